"""Batched builds of independent systems with uneven meshes and orbital counts
(dg_exchange_build_multi) against one dg_exchange_build per system, and the
autotuner's cache round trip."""

import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2510_21213_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

os.environ.setdefault("DG_AUTOTUNE_CACHE", os.path.join(tempfile.mkdtemp(), "autotune.jsonl"))


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    dgx.load()
    return dgx


def _systems():
    out = []
    for (n, p, N, seed) in [(4, 4, 3, 11), (2, 3, 2, 12), (4, 5, 4, 13), (2, 6, 2, 14), (2, 2, 5, 15)]:
        mesh = inputs.MeshSpec((-6.0,) * 3, (6.0,) * 3, (n, n, n), p)
        rng = np.random.default_rng(seed)
        atoms = rng.uniform(-2.0, 2.0, size=((N + 1) // 2 + 1, 3))
        spec = inputs.gto_system(mesh, atoms, N, seed)
        m = oracle.Mesh(mesh.lo, mesh.hi, mesh.n, mesh.p)
        psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
        out.append((mesh, psi))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_system_build_equals_single_builds(dgx, precision):
    systems = _systems()
    args = [(m.lo, m.hi, m.n, m.p, torch.tensor(psi, device="cuda")) for (m, psi) in systems]
    opts = dgx.dg_default_opts(precision=precision, rtol=1e-10)
    Ks, ehs, exs, sts = dgx.dg_exchange_build_multi(args, opts=opts, lanes=3)
    for i, (m, psi) in enumerate(systems):
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=precision, rtol=1e-10)
        K, eh, ex, st = s.exchange_build(args[i][4])
        assert all(x["status"] == 0 for x in sts[i]) and len(sts[i]) == len(st)
        assert np.abs(Ks[i] - K).max() <= 1e-13 * np.abs(K).max()
        assert abs(ehs[i] - eh) <= 1e-13 * abs(eh) and abs(exs[i] - ex) <= 1e-13 * abs(ex)
        s.close()
    # first system against the oracle as well (FP64 bound / mixed bound at 1e-10)
    m, psi = systems[0]
    ref = oracle.exchange_build(oracle.Mesh(m.lo, m.hi, m.n, m.p), psi, method="fdm")
    tol = 1e-9 if precision == 0 else 1e-6
    assert np.abs(Ks[0] - ref["K"]).max() <= tol * np.abs(ref["K"]).max()
    dgx.dg_release_cached_handles()


def test_autotuner_chooses_and_caches(dgx):
    s = dgx.PoissonSolver([-6.0] * 3, [6.0] * 3, 4, 5, precision=1)
    b1 = dgx.dg_autotune_batch(s.h, 1000)
    assert 1 <= b1 <= 512
    path = os.environ["DG_AUTOTUNE_CACHE"]
    assert os.path.exists(path) and "p5" in open(path).read()
    b2 = dgx.dg_autotune_batch(s.h, 1000)  # second call is served from the cache
    assert b2 == b1
    assert dgx.dg_autotune_batch(s.h, 3) == min(b1, 3)
    s.close()


def test_many_lanes_with_overlapping_setup_and_capture(dgx):
    """Eight uneven systems of the batched workload on four lanes, mixed form:
    lanes set up handles while other lanes capture their PCG graphs. Every
    build converges and matches a single build of the same system."""
    specs = [inputs.batched_system(4000 + k) for k in range(8)]
    args = []
    for sp in specs:
        m = sp.mesh
        xyz, w = dgx.dg_mesh_node_coords(m.lo, m.hi, m.n, m.p)
        args.append((m.lo, m.hi, m.n, m.p, torch.tensor(inputs.orbitals(sp, xyz, w), device="cuda")))
    opts = dgx.dg_default_opts(precision=1, rtol=1e-8)
    Ks, ehs, exs, sts = dgx.dg_exchange_build_multi(args, opts=opts, lanes=4)
    assert all(x["status"] == 0 for st in sts for x in st)
    for i in (0, len(specs) - 1):
        m = specs[i].mesh
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=1, rtol=1e-8)
        K, eh, ex, st = s.exchange_build(args[i][4])
        assert np.abs(Ks[i] - K).max() <= 1e-12 * np.abs(K).max()
        s.close()
    dgx.dg_release_cached_handles()
