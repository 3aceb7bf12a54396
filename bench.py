"""Exchange-build benchmark: pair Poisson solves per second at a 1e-8 FP64
true relative residual, the chosen form (mixed precision) against the plain
FP64 form, on one synthetic Gaussian-orbital system per GPU.

Default workload `mixed64`: box [-12,12]^3, 16^3 elements, p = 7 (2.1 M
nodes), 64 orbitals on 32 random atoms, i.e. 2080 pair solves + the Hartree
solve per exchange build. One step = one batch of consecutive sources of that
build (the source list is 0 = Hartree density, then the pairs) through
dg_exchange_build_range: every row of the hot path for the batch (pair
densities, right-hand sides, Coulomb Dirichlet data by the Gaussian-sum route,
multigrid-preconditioned CG to 1e-8, exchange accumulation, the batch's
contribution to K, the self-energies). Successive steps take successive
batches, cycling through the build; the batches of one cycle add up to the
whole build's K. The batch is three times the library's solve batch (120
sources at this size), or the whole build when that is smaller (chain10).
value = pair solves of all ranks / max-over-ranks time. Inputs (orbital values
at the nodes) are resident in HBM for `value`; `e2e` copies them from pinned
host memory every step and reads the step's K back. Beside them: the plain
FP64 and learned forms on the same batches, the Hartree/exchange action on
trial functions (`jk_action`, N <= 16 only), the roofline of the dominant
kernel and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mixed64|chain10|batched32|tiny] [--precision mixed|fp64|learned]
                  [--sources-per-step S] [--no-plain] [--no-learned] [--no-cpu] [--no-jk]
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
# ALU peaks of a GB300 from its unit counts at the maximum SM clock (2070 MHz):
# FP32 152 SMs x 128 lanes x 2 flop; FP64 the datasheet's 1.25 TFLOP/s dense
# (about 2 FMA per clock per SM)
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25
# dense TF32 tensor rate: the measured BF16 GEMM peak x the nominal TF32 / BF16
# ratio (1.1 / 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed64", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "learned"])
    ap.add_argument("--sources-per-step", type=int, default=0,
                    help="sources of the build per step (0: three library batches, at most the whole build)")
    ap.add_argument("--batch", type=int, default=0,
                    help="sources solved together by the library (0: its default, about 8 GB of FP64 vectors)")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP64 form")
    ap.add_argument("--no-learned", action="store_true", help="skip timing the learned form")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-jk", action="store_true", help="skip timing the J/K action on trial functions")
    ap.add_argument("--octree", action="store_true",
                    help="time the exchange build on a density-refined octree instead of the uniform mesh")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time only the dominant kernels (operator, smoother, patch solves) at the bench's batch, "
                         "without the exchange builds (the command the ncu captures of profiles/ run)")
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


def step_ranges(total, per_step):
    """Consecutive equal batches [b, e) of the source list 0..total-1 (the
    tail that does not fill a batch is left out of the cycle)."""
    per_step = max(1, min(per_step, total))
    return [(b, b + per_step) for b in range(0, total - per_step + 1, per_step)]


def pairs_in(rng):
    """Pair solves of a source range (source 0 is the Hartree density)."""
    b, e = rng
    return (e - b) - (1 if b == 0 else 0)


def run_steps(solver, psi_dev, ranges, first, count, torch, flush, stream, pin=None, dev_buf=None):
    """`count` steps over ranges[first ...] (cyclic), each timed with CUDA events
    on `stream` after an L2 flush. pin/dev_buf: copy the orbitals from pinned
    host memory inside each step (e2e). Returns (ms per step, pairs per step,
    last (K, E_H, stats), the K of every range seen)."""
    times, pairs, last, Ks = [], [], None, {}
    for k in range(count):
        rng = ranges[(first + k) % len(ranges)]
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        src = psi_dev
        if pin is not None:
            dev_buf.copy_(pin, non_blocking=True)
            src = dev_buf
        K, eh, st = solver.exchange_build_range(src, rng[0], rng[1], stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        pairs.append(pairs_in(rng))
        last = (K, eh, st)
        Ks[rng] = K
    return times, pairs, last, Ks


def kernel_roofline(solver, B, precision, torch, nrep=20):
    """Average launch duration (CUDA events on the launching stream) of the
    fine-level patch solves (the dominant kernel), of the whole smoother
    application (patch solves + gather) and of the operator, with their
    algorithmic work."""
    Nq = solver.Nq
    n1 = solver.info.level_p[0] + 1
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.randn((B, Nq), dtype=dt, device="cuda")
    res = {}
    stream = torch.cuda.current_stream()
    for name, fn in (("apply", lambda: solver.apply(u)), ("smoother", lambda: solver.smoother(u)),
                     ("patch", lambda: solver.patch_solves(u))):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nrep):
            fn()
        e1.record(stream)
        e1.synchronize()
        res[name] = e0.elapsed_time(e1) / nrep
    E = Nq // n1 ** 3
    # operator: 3 directions x (n1 diag-block MACs + 4 coupling MACs), 5 flops of
    # mass scaling, traces 6 faces x n1^2 x 2 x n1 MACs per element
    apply_flops = Nq * (3 * (2 * n1 + 8) + 5) + E * 6 * n1 * n1 * 2 * 2 * n1
    m = n1 + 2
    # patch solve by fast diagonalisation: six 1-D passes of m^4 MACs and the
    # eigenvalue scaling per patch
    patch_flops = E * (6 * 2 * m ** 4 + m ** 3)
    s = 8 if precision == "fp64" else 4
    return {
        "apply_ms": res["apply"], "smoother_ms": res["smoother"], "patch_ms": res["patch"], "B": B, "E": E, "m": m,
        "apply_flops": apply_flops * B, "apply_bytes": 2 * Nq * s * B,
        "patch_flops": patch_flops * B,
        # the patch kernel's own input and output: the residual in, the patch solutions out
        "patch_bytes": (Nq + E * m ** 3) * s * B,
        "smoother_bytes": 2 * Nq * s * B,
    }


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


class OracleSample:
    """The CPU oracle (oracle.exchange_partial: exact fast-diagonalisation
    solves, Dirichlet data by its Gaussian-sum route at 1e-12, the range's K
    contribution) on consecutive source ranges of the same workload."""

    def __init__(self, spec):
        import oracle

        self.oracle = oracle
        self.m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
        self.psi = make_inputs(spec, oracle.node_coords(self.m), oracle.quad_weights(self.m))

    def run(self, rng):
        t0 = time.perf_counter()
        self.oracle.exchange_partial(self.m, self.psi, rng[0], rng[1], method="fdm", g_route="gausssum")
        return time.perf_counter() - t0


def oracle_sources_per_step(workload):
    # bounded CPU work per oracle step (about 2-4 s on 16 cores)
    return {"tiny": 4, "chain10": 8}.get(workload, 2)


def describe(spec, P):
    m = spec.mesh
    return (f"box [{m.lo[0]:g},{m.hi[0]:g}]^3, n={m.n[0]}^3 elements, p={m.p}, N={spec.N} orbitals, "
            f"{P} pair solves + Hartree per exchange build")


def run_reference(args):
    """The oracle as it stands, timed on the host cores on the same workload:
    each step one consecutive batch of sources of the build (cycling), no
    extrapolation: value = pair solves done / time taken."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    spec = system_for(args.workload, 0)
    P = spec.N * (spec.N + 1) // 2
    t_setup = time.perf_counter()
    smp = OracleSample(spec)
    t_setup = time.perf_counter() - t_setup
    per = oracle_sources_per_step(args.workload)
    ranges = step_ranges(P + 1, per)
    for k in range(args.warmup):
        smp.run(ranges[k % len(ranges)])
    times, pairs = [], []
    for k in range(args.steps):
        rng = ranges[(args.warmup + k) % len(ranges)]
        times.append(smp.run(rng))
        pairs.append(pairs_in(rng))
    value = sum(pairs) / sum(times)
    desc = (f"oracle.exchange_partial on {per} consecutive sources per step (cycling through the build's "
            f"{P + 1} sources): Gaussian-sum Dirichlet data, exact fast-diagonalisation solves, the range's K; "
            f"numpy/scipy on {cores()} host threads; timed as run, not extrapolated")
    line = {
        "impl": "reference", "metric": "exchange-build pair Poisson solves/s at 1e-8 residual",
        "value": value, "unit": "pair_solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {describe(spec, P)}", "sources_per_step": per,
                   "setup_s": t_setup},
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
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        # every lane's build is ordered after e0 and before e1 on this stream
        # (each waits on the stream at entry and the stream waits on it at exit)
        e0.record(stream)
        Ks, ehs, exs, sts = dgx.dg_exchange_build_multi(systems, opts=opts, lanes=4, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
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
                   "timing": "CUDA events on the calling stream around each multi-system call (the lanes' "
                             "streams are ordered between them)"},
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
    solver = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=prec, rtol=1e-8, batch=args.batch,
                               nn_weights_path=weights if prec == dgx.DG_PREC_MIXED_LEARNED else None)
    if args.kernels_only:
        rf = kernel_roofline(solver, min(solver.info.batch, P + 1), args.precision, torch)
        print(json.dumps({"kernels_only": True, "workload": args.workload, "precision": args.precision, **rf}),
              flush=True)
        solver.close()
        pd.finish()
        return
    xyz, w = solver.node_coords()
    psi_host = make_inputs(spec, xyz, w)
    psi_dev = torch.tensor(psi_host, device="cuda")
    flush = torch.empty(int(256 * 2 ** 20 / 4), dtype=torch.float32, device="cuda")  # 256 MB > L2 (126 MB)
    stream = torch.cuda.current_stream()
    per_step = args.sources_per_step or 3 * solver.info.batch
    ranges = step_ranges(P + 1, per_step)
    per_step = ranges[0][1] - ranges[0][0]

    # timed region (device-resident inputs): warm-up steps, then `steps` steps
    run_steps(solver, psi_dev, ranges, 0, args.warmup, torch, flush, stream)
    pd.barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = dgx.dg_kernel_launch_count()
    times, pairs, (K, eh, stats), Ks = run_steps(solver, psi_dev, ranges, args.warmup, args.steps, torch, flush,
                                                 stream)
    launches = (dgx.dg_kernel_launch_count() - l0) // args.steps
    clocks = clk.stop()
    pd.barrier()
    tot = pd.max_over_ranks(sum(times) / 1e3, device="cuda")
    value = pd.aggregate_rate(sum(pairs) / args.steps, args.steps, tot, ws)
    iters = [s["iters"] for s in stats if s is not None]
    resid = max(s["rel_residual"] for s in stats)
    status_ok = all(s["status"] == 0 for s in stats)

    # end to end through the public API: pinned host orbitals copied in every
    # step, the step's K read back to the host (inside the call)
    pin = torch.tensor(psi_host).pin_memory()
    dev_buf = torch.empty_like(psi_dev)
    pd.barrier()
    e2e_times, e2e_pairs, _, _ = run_steps(solver, psi_dev, ranges, args.warmup, args.steps, torch, flush, stream,
                                           pin=pin, dev_buf=dev_buf)
    e2e_tot = pd.max_over_ranks(sum(e2e_times) / 1e3, device="cuda")
    e2e_value = pd.aggregate_rate(sum(e2e_pairs) / args.steps, args.steps, e2e_tot, ws)
    del dev_buf, pin

    def other_form(form_prec, nsteps, **kw):
        sv = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=form_prec, rtol=1e-8, batch=args.batch, **kw)
        run_steps(sv, psi_dev, ranges, args.warmup, 1, torch, flush, stream)
        t, pr, (Kf, ehf, stf), Kfs = run_steps(sv, psi_dev, ranges, args.warmup, nsteps, torch, flush, stream)
        ftot = pd.max_over_ranks(sum(t) / 1e3, device="cuda")
        common = [r for r in Kfs if r in Ks]
        dK = max((float(np.abs(Kfs[r] - Ks[r]).max() / np.abs(Kfs[r]).max()) for r in common), default=None)
        out = {"value": pd.aggregate_rate(sum(pr) / nsteps, nsteps, ftot, ws), "ms_per_step": ftot / nsteps * 1e3,
               "steps": nsteps, "mean_iters": float(np.mean([x["iters"] for x in stf])),
               "K_rel_diff_vs_chosen": dK}
        sv.close()
        return out, stf

    # plain FP64 form on the same batches (the metric's comparison)
    plain = None
    if not args.no_plain and prec != dgx.DG_PREC_FP64:
        plain, _ = other_form(dgx.DG_PREC_FP64, max(1, min(args.steps, 2)))

    # learned form (network initial guess) on the same batches, where weights for this degree exist
    learned = None
    if not args.no_learned and prec == dgx.DG_PREC_MIXED and weights is not None:
        learned, stl = other_form(dgx.DG_PREC_MIXED_LEARNED, max(1, min(args.steps, 3)), nn_weights_path=weights)
        learned.update({"fallbacks": int(sum(s["used_fallback"] for s in stl)),
                        "mean_guess_rel_residual": float(np.mean([s["guess_rel_residual"] for s in stl])),
                        "weights": os.path.relpath(weights, ROOT)})

    # Hartree and exchange actions on trial functions (the eigensolver's operator
    # application): the occupied orbitals as the m = N trial functions, so that
    # <psi_i, X psi_j> must reproduce -K of the build
    jk = None
    if not args.no_jk and prec != dgx.DG_PREC_FP64 and N <= 16:  # 1 + N^2 solves per call
        K_full, _, _, _ = solver.exchange_build(psi_dev)
        _, wq = solver.node_coords()
        wq_d = torch.tensor(wq, device="cuda")
        solver.jk_apply(psi_dev, psi_dev)
        torch.cuda.synchronize()
        jtimes = []
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        for _ in range(max(1, min(args.steps, 2))):
            flush_l2(flush)
            t0.record(stream)
            JU, XU, stj = solver.jk_apply(psi_dev, psi_dev)
            t1.record(stream)
            t1.synchronize()
            jtimes.append(t0.elapsed_time(t1))
        jtot = pd.max_over_ranks(sum(jtimes) / 1e3, device="cuda")
        nsolve = 1 + N * N
        Kj = -((psi_dev * wq_d) @ XU.T).cpu().numpy()
        jk = {"value": pd.aggregate_rate(nsolve, len(jtimes), jtot, ws), "unit": "trial_solves/s",
              "trial_functions": N, "solves_per_call": nsolve, "ms_per_call": jtot / len(jtimes) * 1e3,
              "mean_iters": float(np.mean([x["iters"] for x in stj])),
              "K_rel_diff_vs_build": float(np.abs(Kj - K_full).max() / np.abs(K_full).max())}

    # roofline of the dominant kernel: the fine-level patch solves (see profiles/)
    B = min(solver.info.batch, P + 1)
    rf = kernel_roofline(solver, B, args.precision, torch)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1906.3)
    tc_used = args.precision != "fp64" and m.p >= 7
    alu_peak = FP32_PEAK_TFLOPS if args.precision != "fp64" else FP64_PEAK_TFLOPS
    t = rf["patch_ms"] * 1e-3
    # the roofline that bounds the kernel is the one with the longest ideal time
    ideal = {"hbm": rf["patch_bytes"] / (hbm * 1e9)}
    if tc_used:
        # executed on the tensor cores: two dense m^2 x m^2 Kronecker factors per patch
        # (TF32, K padded to 8) at the measured BF16 peak x the nominal TF32 / BF16 ratio
        kpad = (rf["m"] ** 2 + 7) // 8 * 8
        tc_flops = rf["B"] * rf["E"] * 2 * 2 * 128 * 12 * kpad
        ideal["tensor"] = tc_flops / (bf16 * TF32_OVER_BF16 * 1e12)
        # the z factor in FP32: per patch m^2 z lines, each two m x m contractions
        ideal["alu"] = rf["B"] * rf["E"] * 2 * 2 * rf["m"] ** 4 / (alu_peak * 1e12)
    else:
        ideal["alu"] = rf["patch_flops"] / (alu_peak * 1e12)
    bound = max(ideal, key=ideal.get)
    if bound == "hbm":
        ach, peak, unit = rf["patch_bytes"] / t / 1e9, hbm, "GB/s"
        peak_source = "MEASURED_PEAKS.json hbm_gbs (copy bandwidth of this pool's GB300)"
    elif bound == "tensor":
        ach, peak, unit = tc_flops / t / 1e12, bf16 * TF32_OVER_BF16, "TFLOP/s"
        peak_source = "MEASURED_PEAKS.json bf16_tflops x 1.1/2.25 (nominal TF32 / BF16)"
    else:
        ach, peak, unit = rf["patch_flops"] / t / 1e12, alu_peak, "TFLOP/s"
        peak_source = ("FP32: 152 SMs x 128 lanes x 2 flop x 2070 MHz (unit counts)" if args.precision != "fp64"
                       else "FP64: 1.25 TFLOP/s dense (datasheet)")
    kname = "k_schwarz_patch_tc" if tc_used else "k_schwarz_patch"
    roofline = {
        "kernel": f"{kname} (fine-level Schwarz patch solves, {rf['B']} sources)",
        "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
        "traffic": measured_traffic(f"{kname}_{args.workload}_{args.precision}_B{rf['B']}"),
        "algorithmic_bytes": rf["patch_bytes"], "algorithmic_flops": rf["patch_flops"],
        "ideal_ms": {k: v * 1e3 for k, v in ideal.items()}, "peak_source": peak_source,
        "launch_ms": rf["patch_ms"], "B": rf["B"],
        "alu_view": {"tflops": rf["patch_flops"] / t / 1e12, "frac": rf["patch_flops"] / t / 1e12 / alu_peak},
        "smoother_application": {"launch_ms": rf["smoother_ms"], "kernels": f"{kname} + k_schwarz_gather",
                                 "gbs_r_in_z_out": rf["smoother_bytes"] / (rf["smoother_ms"] * 1e-3) / 1e9},
        "operator": {"launch_ms": rf["apply_ms"], "tflops": rf["apply_flops"] / (rf["apply_ms"] * 1e-3) / 1e12,
                     "frac_alu": rf["apply_flops"] / (rf["apply_ms"] * 1e-3) / 1e12 / alu_peak,
                     "gbs": rf["apply_bytes"] / (rf["apply_ms"] * 1e-3) / 1e9,
                     "frac_hbm_of_measured": rf["apply_bytes"] / (rf["apply_ms"] * 1e-3) / 1e9 / hbm},
    }

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        smp = OracleSample(spec)
        n_src = {"tiny": P + 1, "chain10": P + 1}.get(args.workload, 8)
        rng = (0, min(n_src, P + 1))
        secs = smp.run(rng)
        cpu = {"value": pairs_in(rng) / secs, "unit": "pair_solves/s", "cores": cores(), "kind": "oracle",
               "sample": f"oracle.exchange_partial over sources {rng[0]}..{rng[1] - 1} of the same build "
                         f"(Gaussian-sum Dirichlet data, exact fast-diagonalisation solves, the range's K)",
               "seconds": secs}

    if rank == 0:
        line = {
            "metric": "exchange-build pair Poisson solves/s at 1e-8 residual",
            "value": value, "unit": "pair_solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "fp64": "f64", "learned": "bf16+f32+f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {describe(spec, P)}",
                       "step": f"{per_step} consecutive sources of the build per step via dg_exchange_build_range, "
                               f"cycling through {len(ranges)} batches",
                       "precision": args.precision, "rtol": 1e-8, "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"independent system per GPU x{ws}"},
            "e2e": {"value": e2e_value, "unit": "pair_solves/s", "h2d_bytes_per_step": int(psi_host.nbytes),
                    "d2h_bytes_per_step": int(N * N * 8 + 8 + per_step * 48)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "plain_fp64": plain,
            "learned": learned,
            "jk_action": jk,
            "solver": {"mean_iters": float(np.mean(iters)), "max_iters": int(max(iters)),
                       "max_rel_residual": resid, "all_converged": status_ok,
                       "outer_refinements": int(max(s["outer_refinements"] for s in stats))},
        }
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as fh:
                fh.write(s + "\n")
    solver.close()
    pd.finish()


def run_octree(args):
    """Exchange build on an adaptive octree (dg_octree_setup /
    dg_octree_exchange_build): the chain10 box [-12, 12]^3 with an 8^3 root grid
    at p = 6, refined by the density indicator of the chain system's orbitals
    (delta 1e-5, up to level 2), the chain's 10 orbitals evaluated at the
    octree's nodes and orthonormalised with its weights; rtol 1e-8. One step =
    one whole build (Hartree + 55 pairs), timed with CUDA events; value = the
    mixed form (FP32 inner PCG in FP64 refinement), the FP64 form beside it.
    Also the FP64 operator alone on 8 fields (one kernel, CUDA events)."""
    import torch

    from paper_2510_21213_gb300 import build, dgx, inputs

    build.build()
    spec = inputs.chain_system()
    lo, hi, n, p = list(spec.mesh.lo), list(spec.mesh.hi), tuple(spec.mesh.n), spec.mesh.p

    def rho(P):
        return np.sum((spec.coeffs @ inputs.eval_primitives(spec, P)) ** 2, axis=0)

    leaves = dgx.dg_octree_refine(lo, hi, n, p, rho, 1e-5, 2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for prec in (dgx.DG_PREC_MIXED, dgx.DG_PREC_FP64):
        s = dgx.OctreeSolver(lo, hi, n, p, leaves, rtol=1e-8, precision=prec)
        xyz, w = s.node_coords()
        psi = torch.tensor(inputs.orbitals(spec, xyz.cpu().numpy(), w.cpu().numpy()), device="cuda")
        for _ in range(max(args.warmup, 3)):
            K, EH, EX, st = s.exchange_build(psi)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            ev0.record()
            K, EH, EX, st = s.exchange_build(psi)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        res[prec] = {"ms": sum(ms) / len(ms), "K": K, "E_H": EH, "E_X": EX,
                     "iters": float(np.mean([x["iters"] for x in st])),
                     "rounds": float(np.mean([x["outer_refinements"] for x in st]))}
        if prec == dgx.DG_PREC_FP64:
            B = 8
            u = torch.randn(B, s.Nq, dtype=torch.float64, device="cuda")
            out = torch.empty_like(u)
            for _ in range(3):
                s.apply(u, out)
            torch.cuda.synchronize()
            ev0.record()
            for _ in range(20):
                s.apply(u, out)
            ev1.record()
            torch.cuda.synchronize()
            op_ms = ev0.elapsed_time(ev1) / 20
            Nq = s.Nq
        N = psi.shape[0]
        s.close()
    P = N * (N + 1) // 2
    mx, fp = res[dgx.DG_PREC_MIXED], res[dgx.DG_PREC_FP64]
    levels = np.bincount(leaves[:, 0]).tolist()
    print(json.dumps({"metric": "octree exchange build, pair solves/s", "value": (P + 1) / (mx["ms"] / 1e3),
                      "unit": "pair_solves/s", "ms_per_step": mx["ms"], "steps": args.steps,
                      "warmup": max(args.warmup, 3), "higher_is_better": True, "dtype": "f32+f64",
                      "data": "synthetic",
                      "config": {"workload": "octree: chain10 box, 8^3 roots, p=6, density-refined to level 2",
                                 "leaves": int(leaves.shape[0]), "leaves_per_level": levels, "Nq": int(Nq),
                                 "orbitals": N, "sources": P + 1, "rtol": 1e-8, "precision": "mixed",
                                 "mean_inner_iters": mx["iters"], "mean_rounds": mx["rounds"],
                                 "E_H": mx["E_H"], "E_X": mx["E_X"],
                                 "timing": "CUDA events around each whole build (host-synchronised PCG)"},
                      "fp64": {"value": (P + 1) / (fp["ms"] / 1e3), "ms_per_step": fp["ms"], "mean_iters": fp["iters"],
                               "K_rel_diff_vs_mixed": float(np.abs(fp["K"] - mx["K"]).max() / np.abs(fp["K"]).max())},
                      "operator": {"fields": 8, "ms_per_application": op_ms, "dof_per_s": 8 * Nq / (op_ms / 1e3),
                                   "dtype": "f64", "timing": "CUDA events over 20 launches of the operator kernel"}}),
          flush=True)


def main():
    args = parse()
    if args.octree:
        run_octree(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched32":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
