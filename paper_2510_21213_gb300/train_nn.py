"""Trains the network of the learned initial guess on the GPU with the
library's own kernels (dg_nn_train_step: guess, loss, backward, Adam) and
writes a weights file for dg_solver_opts.nn_weights_path.

Training data are pair densities psi_i psi_j of synthetic Gaussian-orbital
systems (inputs.random_system recipe: box [-12, 12]^3, 32 atoms, seeded, one
system per training seed) and their potentials, solved by the library's own
mixed-precision solver to a 1e-8 residual. Each step draws a batch of these
pairs. Validation compares, on held-out seeds, the relative residual of the
guess without and with the network, and the PCG iterations of the mixed
(zero guess) and the learned solver on the same pairs.

    python -m paper_2510_21213_gb300.train_nn --p 7 --n 16 --steps 2000 \\
        --out paper_2510_21213_gb300/weights/dgnn_p7.bin --log train_log.json
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def parse_range(text):
    a, _, b = text.partition("-")
    return list(range(int(a), int(b) + 1)) if b else [int(a)]


def init_params(seed, hidden=32):
    """He-style initialisation of the hidden layers; the output layer starts
    at zero, so training starts from the guess without the network."""
    from . import dgx

    rng = np.random.default_rng(seed)
    out = {}
    for name, shape in dgx.NN_LAYOUT:
        if name.startswith("b"):
            out[name] = np.zeros(shape)
        else:
            fan_in = 27 * shape[3]
            out[name] = rng.standard_normal(shape) * math.sqrt(2.0 / fan_in)
    out["W3"][:] = 0.0
    return dgx.nn_pack(out)


def make_systems(solver, seeds, n, p, n_orb, n_atoms):
    import torch

    from . import inputs

    xyz, w = solver.node_coords()
    xyz_d = torch.tensor(xyz, device="cuda")
    w_d = torch.tensor(w, device="cuda")
    out = []
    for sd in seeds:
        spec = inputs.random_system(seed=sd, n=n, p=p, n_orb=n_orb, n_atoms=n_atoms)
        out.append(inputs.orbitals_torch(spec, xyz_d, w_d).contiguous())
    return out


def pair_batch(psi, rng, B):
    import torch

    N = psi.shape[0]
    idx = []
    for _ in range(B):
        i, j = sorted(rng.integers(0, N, size=2))
        idx.append((int(i), int(j)))
    return torch.stack([psi[i] * psi[j] for i, j in idx]).contiguous(), idx


def make_targets(mixed, psis, rng, per_system, batch=32):
    """(system, i, j) of per_system random pairs of every system and their
    potentials (solved with the mixed solver, float64 on the device)."""
    import torch

    keys, vs = [], []
    for si, psi in enumerate(psis):
        f, idx = pair_batch(psi, rng, per_system)
        for b0 in range(0, per_system, batch):
            v, st = mixed.solve(f[b0:b0 + batch].contiguous())
            vs.append(v)
        keys += [(si, i, j) for i, j in idx]
    return keys, torch.cat(vs)


def validate(dgx, learned, mixed, psis, rng, npairs):
    import torch

    res = {"coarse_rel": [], "net_rel": [], "iters_mixed": [], "iters_learned": [], "time_mixed": 0.0,
           "time_learned": 0.0, "fallbacks": 0}
    for psi in psis:
        f, _ = pair_batch(psi, rng, npairs)
        _, rc = dgx.dg_nn_guess(learned.h, f, use_net=False)
        _, rn = dgx.dg_nn_guess(learned.h, f, use_net=True)
        res["coarse_rel"] += rc.tolist()
        res["net_rel"] += rn.tolist()
        for key, s in (("mixed", mixed), ("learned", learned)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = s.solve(f)
            torch.cuda.synchronize()
            res["time_" + key] += time.perf_counter() - t0
            res["iters_" + key] += [x["iters"] for x in st]
            if key == "learned":
                res["fallbacks"] += sum(x["used_fallback"] for x in st)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--p", type=int, default=7)
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--orbitals", type=int, default=16)
    ap.add_argument("--atoms", type=int, default=32)
    ap.add_argument("--seeds", default="100-163")
    ap.add_argument("--val-seeds", default="900-901")
    ap.add_argument("--val-pairs", type=int, default=16)
    ap.add_argument("--pairs-per-system", type=int, default=8)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=3e-5)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--log", default=None)
    ap.add_argument("--verbose", type=int, default=0)
    args = ap.parse_args(argv)

    import torch

    from . import build, dgx

    build.build()
    dgx.load()
    lo, hi = [-12.0] * 3, [12.0] * 3
    learned = dgx.PoissonSolver(lo, hi, (args.n,) * 3, args.p, precision=dgx.DG_PREC_MIXED_LEARNED,
                                bc_route=dgx.DG_BC_GAUSSSUM, rtol=1e-8, verbose=args.verbose)
    mixed = dgx.PoissonSolver(lo, hi, (args.n,) * 3, args.p, precision=dgx.DG_PREC_MIXED,
                              bc_route=dgx.DG_BC_GAUSSSUM, rtol=1e-8, verbose=args.verbose)
    dgx.dg_nn_set_params(learned.h, init_params(args.init_seed))
    t0 = time.perf_counter()
    train = make_systems(learned, parse_range(args.seeds), args.n, args.p, args.orbitals, args.atoms)
    val = make_systems(learned, parse_range(args.val_seeds), args.n, args.p, args.orbitals, args.atoms)
    t_gen = time.perf_counter() - t0
    rng = np.random.default_rng(1234)
    t0 = time.perf_counter()
    keys, targets = make_targets(mixed, train, rng, args.pairs_per_system)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    log = {"args": vars(args), "t_generate_s": t_gen, "t_targets_s": t_solve, "n_train_pairs": len(keys),
           "loss": []}
    log["val_before"] = validate(dgx, learned, mixed, val, np.random.default_rng(99), args.val_pairs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ema = None
    for step in range(1, args.steps + 1):
        # cosine decay to 5 % of the initial rate
        lr = args.lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * (step - 1) / max(1, args.steps))))
        pick = rng.choice(len(keys), size=args.batch, replace=False)
        f = torch.stack([train[keys[k][0]][keys[k][1]] * train[keys[k][0]][keys[k][2]] for k in pick]).contiguous()
        v = targets[torch.as_tensor(pick, device=targets.device)].contiguous()
        loss, _ = dgx.dg_nn_train_step(learned.h, f, v, lr)
        ema = loss if ema is None else 0.98 * ema + 0.02 * loss
        if step % 50 == 0 or step == 1:
            log["loss"].append((step, loss, ema))
            print(f"step {step:5d}  loss {loss:+.6f}  ema {ema:+.6f}", flush=True)
    torch.cuda.synchronize()
    log["t_train_s"] = time.perf_counter() - t0
    log["val_after"] = validate(dgx, learned, mixed, val, np.random.default_rng(99), args.val_pairs)
    for k in ("val_before", "val_after"):
        v = log[k]
        print(k, "coarse rel %.3e  net rel %.3e  iters mixed %.2f  learned %.2f  fallbacks %d  t %.3f / %.3f s" % (
            np.median(v["coarse_rel"]), np.median(v["net_rel"]), np.mean(v["iters_mixed"]),
            np.mean(v["iters_learned"]), v["fallbacks"], v["time_mixed"], v["time_learned"]), flush=True)
    flat = dgx.dg_nn_get_params(learned.h)
    if args.out:
        dgx.save_nn_weights(args.out, flat, args.p)
    if args.log:
        with open(args.log, "w") as fh:
            json.dump(log, fh, indent=1)
    learned.close()
    mixed.close()


if __name__ == "__main__":
    main()
