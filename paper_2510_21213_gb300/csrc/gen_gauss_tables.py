"""Writes dg_gauss_tables.h: short Gaussian sums for 1/rho on [1, R],

    1/rho ~ sum_k c_k exp(-alpha_k rho^2),   max relative error <= 0.8 tol,

for a ladder of ratios R = 2^(j/2) and the two tolerances the solver uses
(1e-7 for the FP32 tables of the mixed modes, 1e-12 for FP64). The setup
rescales an entry to [r_min, r_max] (alpha / r_min^2, c / r_min) for any
ratio r_max / r_min <= R and checks the error again on the actual range.

Construction: the exponents lie on a geometric grid alpha_k in
[lo / R^2, hi]; the coefficients are the nonnegative least-squares solution for
the relative error rho s(rho) - 1 on log-spaced rho, with Lawson's reweighting
toward the minimax error; the smallest grid size K (and the best of a few
(lo, hi)) that meets the tolerance on a dense check is kept. Nonnegative
coefficients keep the FP32 evaluation free of cancellation.

Run from this directory: python gen_gauss_tables.py (needs numpy and scipy;
a few minutes).
"""

import math
import os

import numpy as np
from scipy.optimize import nnls

TOLS = (1e-7, 1e-12)
J_RANGE = range(8, 37)  # R = 2^(j/2): 16 .. 262144
LOS = (0.001, 0.003, 0.01, 0.03, 0.1)
HIS = (3.0, 10.0, 30.0)


def fit(R, K, lo, hi, npts=3000, lawson=25):
    a = np.exp(np.linspace(math.log(lo / R ** 2), math.log(hi), K))
    rho = np.exp(np.linspace(0.0, math.log(R), npts))
    A = rho[:, None] * np.exp(-a[None, :] * (rho * rho)[:, None])
    w = np.full(npts, 1.0 / npts)
    best = (np.inf, None)
    for _ in range(lawson):
        sw = np.sqrt(w)
        c, _ = nnls(A * sw[:, None], sw, maxiter=10000)
        e = np.abs(A @ c - 1.0)
        if e.max() < best[0]:
            best = (e.max(), c.copy())
        w = w * e
        w = w / w.sum()
    return a, best[1]


def max_err(R, a, c, npts=40000):
    rho = np.exp(np.linspace(0.0, math.log(R), npts))
    s = (c[None, :] * np.exp(-a[None, :] * (rho * rho)[:, None])).sum(axis=1)
    return float(np.abs(rho * s - 1.0).max())


def table(R, tol, k0):
    K = max(8, k0)
    while K < 200:
        best = None
        for lo in LOS:
            for hi in HIS:
                a, c = fit(R, K, lo, hi)
                e = max_err(R, a, c)
                if best is None or e < best[0]:
                    best = (e, a, c)
        if best[0] <= 0.8 * tol:
            e, a, c = best
            keep = c > 0
            return K, e, a[keep], c[keep]
        K += 2
    raise RuntimeError(f"no table for R={R} tol={tol}")


def main():
    entries, alphas, coefs = [], [], []
    for tol in TOLS:
        k0 = 8
        for j in J_RANGE:
            R = 2.0 ** (j / 2)
            K, e, a, c = table(R, tol, k0)
            k0 = K - 2
            entries.append((R, tol, len(a), len(alphas), e))
            alphas.extend(a.tolist())
            coefs.extend(c.tolist())
            print(f"tol {tol:g} R {R:10.1f}: {len(a)} terms, max rel err {e:.2e}", flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dg_gauss_tables.h")
    with open(out, "w") as fh:
        fh.write("// Generated by gen_gauss_tables.py (short Gaussian sums for 1/rho on [1, R]); do not edit.\n")
        fh.write("#pragma once\n\nnamespace dg {\nnamespace gtab {\n\n")
        fh.write("struct Entry {\n  double R, tol;\n  int n, off;\n  double err;\n};\n\n")
        fh.write(f"constexpr int kEntries = {len(entries)};\n")
        fh.write("constexpr Entry kEntry[kEntries] = {\n")
        for (R, tol, n, off, e) in entries:
            fh.write(f"    {{{R!r}, {tol!r}, {n}, {off}, {e!r}}},\n")
        fh.write("};\n\n")
        for name, vals in (("kAlpha", alphas), ("kCoef", coefs)):
            fh.write(f"constexpr double {name}[{len(vals)}] = {{\n")
            for i in range(0, len(vals), 4):
                fh.write("    " + ", ".join(repr(v) for v in vals[i:i + 4]) + ",\n")
            fh.write("};\n\n")
        fh.write("}  // namespace gtab\n}  // namespace dg\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
