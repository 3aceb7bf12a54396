"""The device-side PCG loop (dg_solver_opts.device_loop = 1, the default):
each PCG solve is one CUDA graph launch whose conditional while-node runs the
iterations and tests convergence on the device. A converged source takes zero
steps from then on, and every per-source sum is independent of the other
sources of the batch, so the potentials, iteration counts and residuals equal
those of the host-driven loop (device_loop = 0) bit for bit."""

import numpy as np
import pytest

from paper_2510_21213_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    dgx.load()
    return dgx


def _sources(dgx, s, spec, n):
    xyz, w = s.node_coords()
    psi = inputs.orbitals(spec, xyz, w)
    f = [psi[i] * psi[j] for i in range(spec.N) for j in range(i, spec.N)][:n]
    return torch.tensor(np.stack(f), device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_loop_equals_host_loop(dgx, prec):
    spec = inputs.chain_system()
    m = spec.mesh
    p = dgx.DG_PREC_FP64 if prec == "fp64" else dgx.DG_PREC_MIXED
    out = {}
    for loop in (0, 1):
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=p, rtol=1e-10, device_loop=loop, batch=12)
        f = _sources(dgx, s, spec, 20)
        f[3] *= 0.0  # a zero source: done at x = 0 without iterations
        f[7] *= 1e6  # a badly scaled one
        v, st = s.solve(f)
        v2, st2 = s.solve(f)  # the second call replays the captured graphs
        out[loop] = (v, st, v2, st2)
        s.close()
    v0, st0, v0b, _ = out[0]
    v1, st1, v1b, _ = out[1]
    assert torch.equal(v0, v1) and torch.equal(v0b, v1b) and torch.equal(v1, v1b)
    assert [x["iters"] for x in st0] == [x["iters"] for x in st1]
    assert [x["outer_refinements"] for x in st0] == [x["outer_refinements"] for x in st1]
    assert [x["rel_residual"] for x in st0] == [x["rel_residual"] for x in st1]
    assert all(x["status"] == 0 for x in st1) and st1[3]["iters"] == 0


def test_device_loop_stops_at_the_iteration_limit(dgx):
    """With max_iter too small to converge the device loop stops at the limit
    like the host loop (DG_ERR_NOT_CONVERGED, same iterate)."""
    spec = inputs.tiny_system()
    m = spec.mesh
    out = {}
    for loop in (0, 1):
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=dgx.DG_PREC_FP64, rtol=1e-14, max_iter=3,
                              device_loop=loop)
        f = _sources(dgx, s, spec, 3)
        v, st = s.solve(f, allow_unconverged=True)
        out[loop] = (v, st)
        s.close()
    assert torch.equal(out[0][0], out[1][0])
    assert [x["iters"] for x in out[0][1]] == [x["iters"] for x in out[1][1]]
    assert all(x["status"] == dgx.DG_ERR_NOT_CONVERGED and x["iters"] <= 3 for x in out[1][1])


def test_device_loop_exchange_build_and_launch_count(dgx):
    """A whole exchange build with the device loop gives the host loop's K; the
    library's launch counter still counts every kernel that ran (first
    iteration plus the loop body per further iteration)."""
    spec = inputs.chain_system()
    m = spec.mesh
    res = {}
    for loop in (0, 1):
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=dgx.DG_PREC_MIXED, rtol=1e-8, device_loop=loop)
        xyz, w = s.node_coords()
        psi = torch.tensor(inputs.orbitals(spec, xyz, w), device="cuda")
        s.exchange_build(psi)
        l0 = dgx.dg_kernel_launch_count()
        K, eh, ex, st = s.exchange_build(psi)
        res[loop] = (K, eh, dgx.dg_kernel_launch_count() - l0)
        s.close()
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]
    # the device loop runs converged sources along until the batch is done, so
    # it launches at least as many kernels as the host loop, and not many more
    assert res[0][2] <= res[1][2] <= 2 * res[0][2]
