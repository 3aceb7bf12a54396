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
