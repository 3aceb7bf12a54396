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
    # FP64 to a 1e-12 residual (parity at 1e-10), mixed to 1e-10 (its stated bound 1e-6)
    rtol = 1e-12 if precision == 0 else 1e-10
    opts = dgx.dg_default_opts(precision=precision, rtol=rtol)
    Ks, ehs, exs, sts = dgx.dg_exchange_build_multi(args, opts=opts, lanes=3)
    for i, (m, psi) in enumerate(systems):
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=precision, rtol=rtol)
        K, eh, ex, st = s.exchange_build(args[i][4])
        assert all(x["status"] == 0 for x in sts[i]) and len(sts[i]) == len(st)
        assert np.abs(Ks[i] - K).max() <= 1e-13 * np.abs(K).max()
        assert abs(ehs[i] - eh) <= 1e-13 * abs(eh) and abs(exs[i] - ex) <= 1e-13 * abs(ex)
        s.close()
    # first system against the oracle as well (FP64 1e-10 / mixed bound 1e-6)
    m, psi = systems[0]
    ref = oracle.exchange_build(oracle.Mesh(m.lo, m.hi, m.n, m.p), psi, method="fdm")
    tol = 1e-10 if precision == 0 else 1e-6
    err = np.abs(Ks[0] - ref["K"]).max() / np.abs(ref["K"]).max()
    print(f"precision {precision}: K of the first system vs the oracle {err:.2e}")
    assert err <= tol
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


def test_autotuner_picks_patch_solve_tile_shape(dgx):
    """At p = 7 in the mixed mode the fine level's patch solves have a
    tensor-core kernel; the autotuner times its tile shapes (patches per work
    item), records the choice in its cache, and a solve with the chosen shape
    gives exactly the result of one without tuning (the shape changes no
    sum)."""
    lo, hi, n, p = [-6.0] * 3, [6.0] * 3, (4, 4, 4), 7
    m = oracle.Mesh(lo, hi, n, p)
    x = oracle.node_coords(m)
    f = torch.tensor(np.stack([np.exp(-np.sum((x - c) ** 2, axis=1)) for c in ((0.3, 0.1, -0.2), (-1.0, 0.5, 0.4))]),
                     device="cuda")
    ref_s = dgx.PoissonSolver(lo, hi, n, p, precision=1, rtol=1e-10)
    v_ref, _ = ref_s.solve(f)
    s = dgx.PoissonSolver(lo, hi, n, p, precision=1, rtol=1e-10)
    dgx.dg_autotune_batch(s.h, 64)
    line = [l for l in open(os.environ["DG_AUTOTUNE_CACHE"]) if "p7" in l and "prec1" in l]
    assert line and '"tc_np": ' in line[-1]
    tc_np = int(line[-1].split('"tc_np": ')[1].split("}")[0])
    print("chosen patches per tensor-core item:", tc_np)
    assert tc_np in (2, 4, 6, 8, 10)
    v, st = s.solve(f)
    assert all(x["status"] == 0 for x in st)
    assert torch.equal(v, v_ref)
    ref_s.close()
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
