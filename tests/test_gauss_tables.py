"""The tabulated short Gaussian sums for 1/r that the boundary-data route
(Sec. 6.3, Gaussian-sum approximation) uses by default, read from the
generated header and checked independently of the generator: every entry
approximates 1/rho on [1, R] within 0.8 of its tolerance (dense log-spaced
check), all coefficients and exponents are positive (no cancellation in
FP32), and the entries are shorter than the trapezoidal sums of the same
accuracy."""

import math
import os
import re

import numpy as np

import oracle

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2510_21213_gb300", "csrc", "dg_gauss_tables.h")


def _tables():
    txt = open(HDR).read()
    ent = re.search(r"kEntry\[kEntries\] = \{(.*?)\};", txt, re.S).group(1)
    entries = [tuple(float(v) for v in m.split(",")) for m in re.findall(r"\{([^{}]*)\}", ent)]

    def arr(name):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", txt, re.S).group(1)
        return np.array([float(v) for v in body.replace("\n", " ").split(",") if v.strip()])

    return entries, arr("kAlpha"), arr("kCoef")


def test_every_entry_meets_its_tolerance():
    entries, alpha, coef = _tables()
    assert len(entries) >= 20
    assert np.all(alpha > 0) and np.all(coef > 0)
    for (R, tol, n, off, err) in entries:
        n, off = int(n), int(off)
        a, c = alpha[off:off + n], coef[off:off + n]
        rho = np.exp(np.linspace(0.0, math.log(R), 20000))
        s = (c[None, :] * np.exp(-a[None, :] * (rho * rho)[:, None])).sum(axis=1)
        e = np.abs(rho * s - 1.0).max()
        assert e <= 0.8 * tol * 1.01, (R, tol, e)
        assert abs(e - err) <= 0.05 * err + 1e-16, (R, tol, e, err)


def test_entries_are_shorter_than_the_trapezoidal_sums():
    entries, _, _ = _tables()
    for (R, tol, n, _, _) in entries:
        if R < 100:
            continue
        c, _, _ = oracle.gauss_sum_1_over_r(1.0, R, tol)
        assert int(n) * 2 < len(c), (R, tol, int(n), len(c))


def _chain10_range():
    """The distance range the setup uses for chain10 (box [-12, 12]^3, 8^3
    elements, p = 6): the first interior node's distance to a face, and the
    box diagonal, widened by 0.1 %."""
    xi, _ = oracle.gauss_legendre(7)
    rmin = (1.0 - xi.max()) * 3.0 / 2.0 * 0.999
    rmax = 24.0 * math.sqrt(3.0) * 1.001
    return rmin, rmax


def _check(c, a, rmin, rmax):
    r = np.exp(np.linspace(math.log(rmin), math.log(rmax), 20000))
    s = (c[None, :] * np.exp(-a[None, :] * (r * r)[:, None])).sum(axis=1)
    return np.abs(r * s - 1.0).max()


def test_setup_sums_through_the_c_abi():
    from paper_2510_21213_gb300 import dgx

    rmin, rmax = _chain10_range()
    for tol, most in ((1e-7, 40), (1e-12, 60)):
        c0, a0, e0 = dgx.dg_gauss_sum(rmin, rmax, tol, 0)
        c1, a1, e1 = dgx.dg_gauss_sum(rmin, rmax, tol, 1)
        assert len(c0) <= most < len(c1), (tol, len(c0), len(c1))
        for c, a, e in ((c0, a0, e0), (c1, a1, e1)):
            assert e <= tol
            assert _check(c, a, rmin, rmax) <= tol
    # a ratio beyond the tables (R = 1e6): the tabulated construction falls back to the trapezoidal rule
    cf, _, ef = dgx.dg_gauss_sum(1e-6, 1.0, 1e-7, 0)
    ct, _, _ = dgx.dg_gauss_sum(1e-6, 1.0, 1e-7, 1)
    assert len(cf) == len(ct) and ef <= 1e-7
    lib = dgx.load()
    n = dgx.C.c_int32()
    for bad in ((0.0, 1.0, 1e-7, 0), (1.0, 0.5, 1e-7, 0), (0.1, 1.0, 0.0, 0), (0.1, 1.0, 1e-7, 2)):
        assert lib.dg_gauss_sum(*bad, 0, dgx.C.byref(n), None, None, None) == dgx.DG_ERR_INVALID_ARG
    assert lib.dg_gauss_sum(0.1, 1.0, 1e-7, 0, 1, dgx.C.byref(n), None,
                            np.zeros(1).ctypes.data_as(dgx.C.c_void_p), None) == dgx.DG_ERR_INVALID_ARG
