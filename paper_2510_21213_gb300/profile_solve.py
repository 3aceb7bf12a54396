"""Pair solves of one synthetic Gaussian-orbital system, for profiling:
`repeats` calls of dg_pair_solve_batch on the same `pairs` pair densities
(16 orbitals, 32 atoms, box [-12, 12]^3), in the requested form.

    python -m paper_2510_21213_gb300.profile_solve --n 16 --p 7 --precision learned --pairs 16 --repeats 2
"""

from __future__ import annotations

import argparse

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--p", type=int, default=7)
    ap.add_argument("--precision", default="learned", choices=["fp64", "mixed", "learned"])
    ap.add_argument("--pairs", type=int, default=16)
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--seed", type=int, default=900)
    args = ap.parse_args(argv)

    import torch

    from . import build, dgx, inputs

    build.build()
    dgx.load()
    prec = {"fp64": dgx.DG_PREC_FP64, "mixed": dgx.DG_PREC_MIXED, "learned": dgx.DG_PREC_MIXED_LEARNED}[args.precision]
    lo, hi = [-12.0] * 3, [12.0] * 3
    s = dgx.PoissonSolver(lo, hi, (args.n,) * 3, args.p, precision=prec, rtol=1e-8,
                          nn_weights_path=dgx.default_nn_weights(args.p) if prec == dgx.DG_PREC_MIXED_LEARNED else None)
    xyz, w = s.node_coords()
    spec = inputs.random_system(seed=args.seed, n=args.n, p=args.p, n_orb=16, n_atoms=32)
    psi = inputs.orbitals_torch(spec, torch.tensor(xyz, device="cuda"), torch.tensor(w, device="cuda"))
    rng = np.random.default_rng(5)
    pairs = [tuple(sorted(rng.integers(0, 16, size=2))) for _ in range(args.pairs)]
    f = torch.stack([psi[i] * psi[j] for i, j in pairs]).contiguous()
    for _ in range(args.repeats):
        v, st = s.solve(f)
    torch.cuda.synchronize()
    print(f"{args.precision}: mean PCG iterations {np.mean([x['iters'] for x in st]):.2f}, "
          f"fallbacks {sum(x['used_fallback'] for x in st)}", flush=True)
    s.close()


if __name__ == "__main__":
    main()
