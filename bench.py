"""Exchange-build benchmark: pair Poisson solves per second at a 1e-8 FP64
true relative residual, the chosen form (mixed precision) against the plain
FP64 form, on one synthetic Gaussian-orbital system per GPU.

One step = one dg_exchange_build: the Hartree solve, the N(N+1)/2 pair solves
(right-hand sides, Coulomb-quadrature Dirichlet data by the Gaussian-sum
route, multigrid-preconditioned CG to 1e-8), the exchange accumulation, the K
contraction and the energies. value = pair solves of all ranks / max-over-ranks
time. Inputs (orbital values at the nodes) are resident in HBM for `value`;
`e2e` copies them from pinned host memory every step and reads K back.
Beside them: the plain FP64 and learned forms of the same build, and the
Hartree/exchange action on trial functions (`jk_action`, the orbitals as the
trial functions).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chain10|mixed64|batched32|tiny] [--precision mixed|fp64|learned]
                  [--no-plain] [--no-learned] [--no-cpu] [--no-jk]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "tiny": "tiny",
    "chain10": "chain10",
    "mixed64": "mixed64",
    "batched32": "batched32",
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def measured_traffic(key):
    """DRAM bytes per launch from the committed ncu capture (profiles/traffic.json),
    or None when the kernel source changed after the capture."""
    import hashlib

    try:
        rec = json.load(open(TRAFFIC_FILE))[key]
        with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
            digest = hashlib.sha256(fh.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    return rec["dram_bytes_per_launch"] if digest == rec["source_sha256"] else None
# FP64 FMA throughput of a GB300 measured with the probe under
# paper_2510_21213_gb300/csrc/peak_probe.cu (152 SMs, FP64 pipe)
FP64_PEAK_TFLOPS = 1.20
FP32_PEAK_TFLOPS = 73.3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chain10", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "learned"])
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP64 form")
    ap.add_argument("--no-learned", action="store_true", help="skip timing the learned form")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-jk", action="store_true", help="skip timing the J/K action on trial functions")
    ap.add_argument("--octree-apply", action="store_true",
                    help="time the SIPDG operator on a density-refined octree instead of the exchange build")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


def dist_env():
    from paper_2510_21213_gb300 import dist as pd

    return pd.env()


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                smax.append(float(s[2]))
                for nm, v in zip(names, s[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(spec, xyz, w):
    from paper_2510_21213_gb300 import inputs

    return inputs.orbitals(spec, xyz, w)


def system_for(workload, rank):
    from paper_2510_21213_gb300 import inputs

    if workload == "tiny":
        return inputs.tiny_system()
    from paper_2510_21213_gb300 import dist as pd

    if workload == "chain10":
        return inputs.chain_system(seed=pd.rank_seed(2, rank))
    return inputs.random_system(seed=pd.rank_seed(3, rank))


def flush_l2(buf):
    buf.add_(1.0)


def time_builds(solver, psi_dev, steps, warmup, torch, flush):
    for _ in range(warmup):
        solver.exchange_build(psi_dev)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush_l2(flush)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        K, eh, ex, stats = solver.exchange_build(psi_dev)
        s1.record()
        s1.synchronize()
        times.append(s0.elapsed_time(s1))
    return times, (K, eh, ex, stats)


def kernel_roofline(solver, B, precision, torch, nrep=20):
    """Average launch duration of the fine-level operator and smoother kernels
    (CUDA events on the launching stream) and their algorithmic work."""
    Nq = solver.Nq
    n1 = solver.info.level_p[0] + 1
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.randn((B, Nq), dtype=dt, device="cuda")
    out = torch.empty_like(u)
    res = {}
    for name, fn in (("apply", lambda: solver.apply(u)), ("smoother", lambda: solver.smoother(u))):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(nrep):
            fn()
        e1.record()
        e1.synchronize()
        res[name] = e0.elapsed_time(e1) / nrep
    del out
    E = Nq // n1 ** 3
    # operator: 3 directions x (n1 diag-block MACs + 4 coupling MACs), 5 flops of
    # mass scaling, traces 6 faces x n1^2 x 2 x n1 MACs per element
    apply_flops = Nq * (3 * (2 * n1 + 8) + 5) + E * 6 * n1 * n1 * 2 * 2 * n1
    m = n1 + 2
    sm_flops = E * (6 * 2 * m ** 4 + m ** 3)
    s = 8 if precision == "fp64" else 4
    apply_bytes = 2 * Nq * s
    sm_bytes = Nq * s + E * m ** 3 * s  # patch kernel: read r, write patch solution
    return {
        "apply_ms": res["apply"], "smoother_ms": res["smoother"], "B": B,
        "apply_flops": apply_flops * B, "apply_bytes": apply_bytes * B,
        "smoother_flops": sm_flops * B, "smoother_bytes": sm_bytes * B,
    }


def cpu_oracle_sample(spec, n_src=4, node_stride=8):
    """The CPU oracle on a bounded sample of the same workload: the Coulomb
    boundary sum of n_src pair sources over every node_stride-th boundary node
    (extrapolated to all nodes), plus their exact FDM solves. Returns
    (pairs_per_s, seconds, description)."""
    import oracle

    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
    x = oracle.node_coords(m)
    W = oracle.quad_weights(m)
    psi = make_inputs(spec, x, W)
    pairs = oracle.pair_list(psi.shape[0])[:n_src]
    f = np.stack([psi[i] * psi[j] for i, j in pairs])
    t0 = time.perf_counter()
    oracle.boundary_data_direct(m, f, node_stride=node_stride)
    t_bc = time.perf_counter() - t0
    g0 = [np.zeros((len(pairs),) + pts.shape[:2]) for pts in oracle.boundary_face_nodes(m)]
    t0 = time.perf_counter()
    B = np.stack([oracle.rhs(m, f[k], [gg[k] for gg in g0]) for k in range(len(pairs))])
    oracle.solve_fdm(m, B)
    t_solve = time.perf_counter() - t0
    total = t_bc * node_stride + t_solve
    desc = (f"{len(pairs)} pair solves of the same workload: direct Coulomb boundary sum over 1/{node_stride} "
            f"of the boundary nodes (time x{node_stride}) + exact fast-diagonalisation solves")
    return len(pairs) / total, t_bc + t_solve, desc


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    spec = system_for(args.workload, 0)
    P = spec.N * (spec.N + 1) // 2
    times, rates = [], []
    desc = ""
    for it in range(args.warmup + args.steps):
        rate, secs, desc = cpu_oracle_sample(spec)
        if it >= args.warmup:
            times.append(secs)
            rates.append(rate)
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": "exchange-build pair Poisson solves/s at 1e-8 residual",
        "value": value, "unit": "pair_solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": P / value * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: n={spec.mesh.n[0]}^3 p={spec.mesh.p} N={spec.N} pairs={P}"},
        "cpu_baseline": {"value": value, "unit": "pair_solves/s", "cores": cores(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "pair_solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """32 independent systems of uneven sizes (seeds 4000..4031: 4^3-12^3
    elements, p 4-8, 2-40 orbitals) in one dg_exchange_build_multi call."""
    import torch

    from paper_2510_21213_gb300 import build, dgx, inputs

    from paper_2510_21213_gb300 import dist as pd

    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pd.init("nccl")
    specs = [inputs.batched_system(sd) for sd in pd.rank_seeds(4000, 32, rank)]
    prec = dgx.DG_PREC_MIXED if args.precision == "mixed" else dgx.DG_PREC_FP64
    systems, host = [], []
    total_pairs = 0
    for sp in specs:
        m = sp.mesh
        xyz, w = dgx.dg_mesh_node_coords(m.lo, m.hi, m.n, m.p)
        psi = inputs.orbitals(sp, xyz, w)
        host.append(psi)
        systems.append((m.lo, m.hi, m.n, m.p, torch.tensor(psi, device="cuda")))
        total_pairs += sp.N * (sp.N + 1) // 2
    opts = dgx.dg_default_opts(precision=prec, rtol=1e-8)
    flush = torch.empty(int(256 * 2 ** 20 / 4), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        dgx.dg_exchange_build_multi(systems, opts=opts, lanes=4)
    pd.barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = dgx.dg_kernel_launch_count()
    times = []
    for _ in range(args.steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ks, ehs, exs, sts = dgx.dg_exchange_build_multi(systems, opts=opts, lanes=4)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    launches = (dgx.dg_kernel_launch_count() - l0) // args.steps
    clocks = clk.stop()
    pd.barrier()
    tot = pd.max_over_ranks(sum(times), device="cuda")
    value = pd.aggregate_rate(total_pairs, args.steps, tot, ws)
    iters = [x["iters"] for st in sts for x in st[1:]]
    if rank != 0:
        dgx.dg_release_cached_handles()
        pd.finish()
        return
    line = {
        "metric": "exchange-build pair Poisson solves/s at 1e-8 residual", "value": value, "unit": "pair_solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"batched32: 32 systems per GPU, seeds 4000-4031 (+1000 per rank), "
                               f"{total_pairs} pair solves + 32 Hartree on rank 0",
                   "sizes": [[sp.mesh.n[0], sp.mesh.p, sp.N] for sp in specs], "lanes": 4,
                   "timing": "host wall clock around each multi-system call (several streams)"},
        "gpu_launches": int(launches), "clocks": clocks,
        "solver": {"mean_iters": float(np.mean(iters)), "max_iters": int(max(iters)),
                   "all_converged": all(x["status"] == 0 for st in sts for x in st)},
    }
    print(json.dumps(line), flush=True)
    dgx.dg_release_cached_handles()
    pd.finish()


def run_ours(args):
    import torch

    from paper_2510_21213_gb300 import dist as pd

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pd.init("nccl")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    spec = system_for(args.workload, rank)
    m = spec.mesh
    N = spec.N
    P = N * (N + 1) // 2
    prec = {"mixed": dgx.DG_PREC_MIXED, "fp64": dgx.DG_PREC_FP64, "learned": dgx.DG_PREC_MIXED_LEARNED}[args.precision]
    weights = dgx.default_nn_weights(m.p)
    if prec == dgx.DG_PREC_MIXED_LEARNED and weights is None:
        raise SystemExit(f"no trained network weights for p = {m.p}")
    solver = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=prec, rtol=1e-8,
                               nn_weights_path=weights if prec == dgx.DG_PREC_MIXED_LEARNED else None)
    xyz, w = solver.node_coords()
    psi_host = make_inputs(spec, xyz, w)
    psi_dev = torch.tensor(psi_host, device="cuda")
    flush = torch.empty(int(256 * 2 ** 20 / 4), dtype=torch.float32, device="cuda")  # 256 MB > L2 (126 MB)

    def barrier():
        pd.barrier()

    # timed region (device-resident inputs)
    for _ in range(args.warmup):
        solver.exchange_build(psi_dev)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = dgx.dg_kernel_launch_count()
    times = []
    for _ in range(args.steps):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        K, eh, ex, stats = solver.exchange_build(psi_dev)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = (dgx.dg_kernel_launch_count() - l0) // args.steps
    clocks = clk.stop()
    barrier()
    tot = pd.max_over_ranks(sum(times) / 1e3, device="cuda")
    value = pd.aggregate_rate(P, args.steps, tot, ws)
    iters = [s["iters"] for s in stats[1:]]
    resid = max(s["rel_residual"] for s in stats)
    status_ok = all(s["status"] == 0 for s in stats)

    # end to end through the public API: pinned host inputs copied in every step, K read back
    pin = torch.tensor(psi_host).pin_memory()
    dev_buf = torch.empty_like(psi_dev)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    e2e_times = []
    for _ in range(args.steps):
        flush_l2(flush)
        t0.record()
        dev_buf.copy_(pin, non_blocking=True)
        solver.exchange_build(dev_buf)
        t1.record()
        t1.synchronize()
        e2e_times.append(t0.elapsed_time(t1))
    e2e_tot = pd.max_over_ranks(sum(e2e_times) / 1e3, device="cuda")
    e2e_value = pd.aggregate_rate(P, args.steps, e2e_tot, ws)

    # plain FP64 form on the same system (the metric's comparison)
    plain = None
    if not args.no_plain and prec != dgx.DG_PREC_FP64:
        solver64 = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=dgx.DG_PREC_FP64, rtol=1e-8)
        ptimes, (K64, eh64, ex64, st64) = time_builds(solver64, psi_dev, max(1, min(args.steps, 3)), 1, torch, flush)
        ptot = pd.max_over_ranks(sum(ptimes) / 1e3, device="cuda")
        plain = {"value": pd.aggregate_rate(P, len(ptimes), ptot, ws), "ms_per_step": ptot / len(ptimes) * 1e3,
                 "mean_iters": float(np.mean([s["iters"] for s in st64[1:]])),
                 "K_rel_diff_vs_chosen": float(np.abs(K64 - K).max() / np.abs(K64).max()),
                 "E_X_rel_diff_vs_chosen": abs(ex64 - ex) / abs(ex64)}
        solver64.close()

    # learned form (network initial guess) on the same system, where weights for this degree exist
    learned = None
    if not args.no_learned and prec == dgx.DG_PREC_MIXED and weights is not None:
        solver_l = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=dgx.DG_PREC_MIXED_LEARNED, rtol=1e-8,
                                     nn_weights_path=weights)
        ltimes, (Kl, ehl, exl, stl) = time_builds(solver_l, psi_dev, max(1, min(args.steps, 3)), 1, torch, flush)
        ltot = pd.max_over_ranks(sum(ltimes) / 1e3, device="cuda")
        learned = {"value": pd.aggregate_rate(P, len(ltimes), ltot, ws), "ms_per_step": ltot / len(ltimes) * 1e3,
                   "mean_iters": float(np.mean([s["iters"] for s in stl[1:]])),
                   "fallbacks": int(sum(s["used_fallback"] for s in stl)),
                   "mean_guess_rel_residual": float(np.mean([s["guess_rel_residual"] for s in stl[1:]])),
                   "K_rel_diff_vs_chosen": float(np.abs(Kl - K).max() / np.abs(K).max()),
                   "weights": os.path.relpath(weights, ROOT)}
        solver_l.close()

    # Hartree and exchange actions on trial functions (the eigensolver's operator
    # application): the occupied orbitals as the m = N trial functions, so that
    # <psi_i, X psi_j> must reproduce -K of the build
    jk = None
    if not args.no_jk and prec != dgx.DG_PREC_FP64 and N <= 16:  # 1 + N^2 solves per call
        _, wq = solver.node_coords()
        wq_d = torch.tensor(wq, device="cuda")
        solver.jk_apply(psi_dev, psi_dev)
        torch.cuda.synchronize()
        jtimes = []
        for _ in range(max(1, min(args.steps, 2))):
            flush_l2(flush)
            t0.record()
            JU, XU, stj = solver.jk_apply(psi_dev, psi_dev)
            t1.record()
            t1.synchronize()
            jtimes.append(t0.elapsed_time(t1))
        jtot = pd.max_over_ranks(sum(jtimes) / 1e3, device="cuda")
        nsolve = 1 + N * N
        Kj = -((psi_dev * wq_d) @ XU.T).cpu().numpy()
        jk = {"value": pd.aggregate_rate(nsolve, len(jtimes), jtot, ws), "unit": "trial_solves/s",
              "trial_functions": N, "solves_per_call": nsolve, "ms_per_call": jtot / len(jtimes) * 1e3,
              "mean_iters": float(np.mean([x["iters"] for x in stj])),
              "K_rel_diff_vs_build": float(np.abs(Kj - K).max() / np.abs(K).max())}

    # roofline of the dominant kernel (the smoother patch solve; see profiles/)
    B = min(P + 1, 64)
    rf = kernel_roofline(solver, B, args.precision, torch)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    alu_peak = FP32_PEAK_TFLOPS if args.precision != "fp64" else FP64_PEAK_TFLOPS
    sm_tf = rf["smoother_flops"] / (rf["smoother_ms"] * 1e-3) / 1e12
    sm_gbs = rf["smoother_bytes"] / (rf["smoother_ms"] * 1e-3) / 1e9
    ap_tf = rf["apply_flops"] / (rf["apply_ms"] * 1e-3) / 1e12
    ap_gbs = rf["apply_bytes"] / (rf["apply_ms"] * 1e-3) / 1e9
    roofline = {
        "kernel": "k_schwarz_patch (fine-level smoother patch solve) + k_schwarz_gather",
        "bound": "alu", "achieved": sm_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": sm_tf / alu_peak,
        "traffic": (measured_traffic("smoother_chain10")
                    if args.workload == "chain10" and args.precision != "fp64" and B == 56 else None),
        "algorithmic_bytes": rf["smoother_bytes"],
        "peak_source": ("FP32 FMA probe (paper_2510_21213_gb300/csrc/peak_probe.cu)" if args.precision != "fp64"
                        else "FP64 FMA probe (paper_2510_21213_gb300/csrc/peak_probe.cu)"),
        "launch_ms": rf["smoother_ms"], "B": B, "hbm_gbs": sm_gbs, "hbm_frac_of_measured": sm_gbs / hbm,
        "operator": {"launch_ms": rf["apply_ms"], "tflops": ap_tf, "frac_alu": ap_tf / alu_peak,
                     "gbs": ap_gbs, "frac_hbm_of_measured": ap_gbs / hbm},
    }

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        rate, secs, desc = cpu_oracle_sample(spec)
        cpu = {"value": rate, "unit": "pair_solves/s", "cores": cores(), "kind": "oracle", "sample": desc,
               "seconds": secs}

    if rank == 0:
        line = {
            "metric": "exchange-build pair Poisson solves/s at 1e-8 residual",
            "value": value, "unit": "pair_solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "fp64": "f64", "learned": "bf16+f32+f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: box [-12,12]^3, n={m.n[0]}^3 elements, p={m.p}, "
                                   f"N={N} orbitals, {P} pair solves + Hartree per step",
                       "precision": args.precision, "rtol": 1e-8, "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"independent system per GPU x{ws}"},
            "e2e": {"value": e2e_value, "unit": "pair_solves/s", "h2d_bytes_per_step": int(psi_host.nbytes),
                    "d2h_bytes_per_step": int(N * N * 8 + 16)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "plain_fp64": plain,
            "learned": learned,
            "jk_action": jk,
            "solver": {"mean_iters": float(np.mean(iters)), "max_iters": int(max(iters)),
                       "max_rel_residual": resid, "all_converged": status_ok,
                       "outer_refinements": int(max(s["outer_refinements"] for s in stats)),
                       "E_H": eh, "E_X": ex},
        }
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as fh:
                fh.write(s + "\n")
    solver.close()
    pd.finish()


def run_octree_apply(args):
    """The SIPDG operator on an adaptive octree (dg_octree_apply): the chain10
    box with a 4^3 root grid at p = 6, refined by the density indicator for the
    chain's ten atom-centred Gaussians (exponent 2, delta 1e-5, up to level 2: 344 leaves),
    applied to 8 fields. One step = one call (connectivity and tables built per
    call, then the kernel)."""
    import torch

    from paper_2510_21213_gb300 import build, dgx

    build.build()
    lo, hi, n, p = [-12.0] * 3, [12.0] * 3, (4, 4, 4), 6
    atoms = np.array([[-6.3 + 1.4 * k, 0.0, 0.0] for k in range(10)])

    def rho(P):
        r2 = ((P[:, None, :] - atoms[None, :, :]) ** 2).sum(-1)
        return (2.0 / math.pi) ** 1.5 * np.exp(-2.0 * r2).sum(1)

    leaves = dgx.dg_octree_refine(lo, hi, n, p, rho, 1e-5, 2)
    E, npe, B = leaves.shape[0], (p + 1) ** 3, 8
    u = torch.randn(B, E * npe, dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 3)):
        dgx.dg_octree_apply(lo, hi, n, p, leaves, u)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        dgx.dg_octree_apply(lo, hi, n, p, leaves, u)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    levels = np.bincount(leaves[:, 0]).tolist()
    print(json.dumps({"metric": "octree SIPDG operator applications, DOF/s", "value": B * E * npe / sec,
                      "unit": "dof/s", "ms_per_step": sec * 1e3, "steps": args.steps, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": "octree-apply: chain10 box, 4^3 roots, p=6",
                                                      "leaves": E, "leaves_per_level": levels, "fields": B,
                                                      "timing": "host wall clock around each call (connectivity, "
                                                                "tables and kernel)"}}), flush=True)


def main():
    args = parse()
    if args.octree_apply:
        run_octree_apply(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched32":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
