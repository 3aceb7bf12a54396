"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs. Element-by-element where the oracle is cheap."""

import math

import numpy as np
import pytest

import oracle
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


def level_meshes(lo, hi, n, p):
    """The hp hierarchy documented in dg_poisson.h: p -> p//2 down to 1, then
    n -> n/2 while every n is even."""
    n = list(n)
    out = [(tuple(n), p)]
    while p > 1:
        p = max(1, p // 2)
        out.append((tuple(n), p))
    while all(v % 2 == 0 and v >= 2 for v in n) and 8 * n[0] * n[1] * n[2] > 512:
        n = [v // 2 for v in n]
        out.append((tuple(n), 1))
    return [oracle.Mesh(lo, hi, nn, pp) for nn, pp in out]


def test_node_coords_and_weights(dgx):
    lo, hi, n, p = [-2.0, -1.0, 0.5], [2.0, 1.5, 2.0], (2, 3, 2), 3
    s = dgx.PoissonSolver(lo, hi, n, p)
    xyz, w = s.node_coords()
    m = oracle.Mesh(lo, hi, n, p)
    assert np.abs(xyz - oracle.node_coords(m)).max() < 1e-14
    assert np.abs(w - oracle.quad_weights(m)).max() < 1e-15
    s.close()


@pytest.mark.parametrize("lo,hi,n,p,form", [
    ([-2.0, -1.0, 0.5], [2.0, 1.5, 2.0], (2, 4, 2), 4, 0),
    ([-3.0] * 3, [3.0] * 3, (4, 4, 4), 7, 0),
    ([-1.0, -2.0, -1.5], [1.0, 2.0, 2.0], (3, 2, 1), 8, 1),
    ([-1.0] * 3, [1.0] * 3, (2, 2, 2), 5, 0),
])
def test_operator_all_levels(dgx, lo, hi, n, p, form):
    s = dgx.PoissonSolver(lo, hi, n, p, penalty_form=form)
    meshes = level_meshes(lo, hi, n, p)
    assert s.info.levels == len(meshes)
    rng = np.random.default_rng(1)
    for l, m in enumerate(meshes):
        A = oracle.assemble_kron(m, penalty_form=form)
        u = rng.standard_normal((3, m.Nq))
        ref = np.stack([A @ uu for uu in u])
        got = s.apply(torch.tensor(u, device="cuda"), level=l).cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-13 * scale, (l, np.abs(got - ref).max() / scale)
        got32 = s.apply(torch.tensor(u, device="cuda", dtype=torch.float32), level=l).cpu().double().numpy()
        assert np.abs(got32 - ref).max() <= 2e-5 * scale
    s.close()


def _gauss_sources(m, centers, exps):
    x = oracle.node_coords(m)
    out = []
    for c, a in zip(centers, exps):
        r2 = np.sum((x - np.asarray(c)) ** 2, axis=1)
        out.append((a / math.pi) ** 1.5 * np.exp(-a * r2))
    return np.stack(out)


def _face_arrays(g_flat, m):
    """Split the library's face vector into the oracle's [T1, T2] arrays."""
    out, off = [], 0
    for d in range(3):
        t = [ax for ax in range(3) if ax != d]
        L1, L2 = m.L[t[0]], m.L[t[1]]
        for _ in range(2):
            out.append(g_flat[off:off + L1 * L2].reshape(L2, L1).T)
            off += L1 * L2
    return out


@pytest.mark.parametrize("route", [0, 1])
def test_boundary_data(dgx, route):
    lo, hi, n, p = [-4.0, -3.0, -3.5], [4.0, 3.5, 3.0], (3, 2, 3), 4
    m = oracle.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(7)
    f = np.concatenate([_gauss_sources(m, [[0.3, -0.2, 0.1], [1.0, 0.5, -0.7]], [1.5, 0.7]),
                        rng.standard_normal((1, m.Nq))])
    s = dgx.PoissonSolver(lo, hi, n, p)
    g = s.boundary_data(torch.tensor(f, device="cuda"), route=route).cpu().numpy()
    ref = oracle.boundary_data_direct(m, f)
    bound = oracle.boundary_data_direct(m, np.abs(f))
    for k in range(f.shape[0]):
        faces = _face_arrays(g[k], m)
        for fi in range(6):
            err = np.abs(faces[fi] - ref[fi][k]).max() / bound[fi][k].max()
            tol = 1e-13 if route == 0 else 3e-12
            assert err < tol, (k, fi, err)
    s.close()


@pytest.mark.parametrize("precision,route,form", [(0, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)])
def test_right_hand_side(dgx, precision, route, form):
    """b = 4 pi W f + Nitsche load of g(f) (steps S1-S4) against the oracle's
    load vector with the direct Coulomb boundary data: the volume part to
    round-off, the boundary load within the route's accuracy (R1 the
    definition, R2 the 1e-12 FP64 or 1e-7 FP32 Gaussian sum)."""
    lo, hi, n, p = [-4.0, -3.0, -3.5], [4.0, 3.5, 3.0], (3, 3, 3), 4
    m = oracle.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(27)
    f = np.concatenate([_gauss_sources(m, [[0.3, -0.2, 0.1], [1.0, 0.5, -0.7]], [1.5, 0.7]),
                        rng.standard_normal((1, m.Nq))])
    s = dgx.PoissonSolver(lo, hi, n, p, precision=precision, bc_route=route, penalty_form=form)
    b = dgx.dg_form_rhs(s.h, torch.tensor(f, device="cuda")).cpu().numpy()
    g = oracle.boundary_data_direct(m, f)
    vol = 4.0 * math.pi * oracle.quad_weights(m) * f
    tol = {(0, 0): 1e-12, (0, 1): 1e-10, (1, 1): 2e-5}[(precision, route)]
    for k in range(f.shape[0]):
        ref = oracle.rhs(m, f[k], [gf[k] for gf in g], penalty_form=form)
        lift_ref = ref - vol[k]
        interior = np.abs(lift_ref) == 0.0  # nodes of no boundary element
        assert interior.any() and not interior.all()
        assert np.abs(b[k][interior] - ref[interior]).max() <= 1e-14 * np.abs(ref).max()
        assert np.abs((b[k] - vol[k]) - lift_ref).max() <= tol * np.abs(lift_ref).max(), k
    s.close()


@pytest.mark.parametrize("lo,hi,n,p,B", [
    ([-8.0] * 3, [8.0] * 3, (4, 4, 4), 4, 3),
    ([-4.0, -3.0, -3.5], [4.0, 3.5, 3.0], (2, 2, 4), 3, 5),
    ([-6.0] * 3, [6.0] * 3, (3, 3, 3), 5, 1),
])
def test_pair_solve_matches_exact_solution(dgx, lo, hi, n, p, B):
    m = oracle.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(11)
    centers = rng.uniform(-1.0, 1.0, size=(B, 3))
    f = _gauss_sources(m, centers, rng.uniform(0.5, 2.0, size=B))
    f[-1] *= -0.5  # a negative source too
    s = dgx.PoissonSolver(lo, hi, n, p, rtol=1e-13, max_iter=400)
    v, stats = s.solve(torch.tensor(f, device="cuda"))
    v = v.cpu().numpy()
    ref, _ = oracle.poisson(m, f, method="fdm")
    for k in range(B):
        assert stats[k]["status"] == 0 and stats[k]["rel_residual"] <= 1e-13
        err = np.abs(v[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err < 1e-10, (k, err)
    s.close()


def test_solver_edge_cases(dgx):
    m = oracle.Mesh([-4.0] * 3, [4.0] * 3, 2, 2)
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, rtol=1e-12)
    f = np.zeros((3, m.Nq))
    f[1] = _gauss_sources(m, [[0.1, 0.2, 0.3]], [1.0])[0]
    f[2, 5] = np.nan
    v, stats = s.solve(torch.tensor(f, device="cuda"), allow_unconverged=True)
    v = v.cpu().numpy()
    assert stats[0]["status"] == 0 and np.all(v[0] == 0.0)
    assert stats[1]["status"] == 0
    assert stats[2]["status"] == dgx.DG_ERR_NONFINITE and np.all(v[2] == 0.0)
    ref, _ = oracle.poisson(m, f[1:2], method="dense")
    assert np.abs(v[1] - ref[0]).max() < 1e-10 * np.abs(ref[0]).max()
    # empty batch is a no-op
    v0, st0 = s.solve(torch.zeros((0, m.Nq), dtype=torch.float64, device="cuda"))
    assert v0.shape[0] == 0 and st0 == []
    s.close()


def test_exchange_build_tiny_system(dgx):
    spec = inputs.tiny_system()
    mm = spec.mesh
    m = oracle.Mesh(mm.lo, mm.hi, mm.n, mm.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m))
    ref = oracle.exchange_build(m, psi, method="fdm")
    s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-12)
    K, eh, ex, stats = s.exchange_build(torch.tensor(psi, device="cuda"))
    assert len(stats) == 4 and all(st["status"] == 0 for st in stats)
    assert np.abs(K - ref["K"]).max() <= 1e-10 * np.abs(ref["K"]).max()
    assert abs(eh - ref["E_H"]) <= 1e-10 * abs(ref["E_H"])
    assert abs(ex - ref["E_X"]) <= 1e-10 * abs(ref["E_X"])
    s.close()


def test_exchange_build_small_random_system_ragged_batches(dgx):
    """Several orbitals, pairs split over batches that do not divide the pair count."""
    m = oracle.Mesh([-6.0] * 3, [6.0] * 3, 2, 4)
    atoms = np.array([[-1.0, 0.2, 0.0], [1.1, -0.3, 0.4], [0.0, 0.9, -0.8]])
    spec = inputs.gto_system(inputs.MeshSpec(tuple(m.lo), tuple(m.hi), m.n, m.p), atoms, 5, 21)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    ref = oracle.exchange_build(m, psi, method="fdm")
    for batch in (4, 7, 0):
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, rtol=1e-12, batch=batch)
        K, eh, ex, stats = s.exchange_build(torch.tensor(psi, device="cuda"))
        assert len(stats) == 16 and all(st["status"] == 0 for st in stats)
        assert np.abs(K - ref["K"]).max() <= 1e-10 * np.abs(ref["K"]).max()
        assert abs(eh - ref["E_H"]) <= 1e-10 * abs(ref["E_H"])
        s.close()


def _patch_reference(A, m, r):
    """sum over element patches (element plus one node layer of every
    neighbour) of R_P^T A_PP^-1 R_P r, from the assembled operator."""
    from oracle import dg_oracle as O

    X, Y, Z = O.global_indices(m)
    inv = np.empty(m.Nq, dtype=int)
    inv[X + m.L[0] * (Y + m.L[1] * Z)] = np.arange(m.Nq)
    A = A.tocsr()
    z = np.zeros_like(r)
    for e in range(m.E):
        ec = (e % m.n[0], (e // m.n[0]) % m.n[1], e // (m.n[0] * m.n[1]))
        rng = [np.arange(max(0, ec[d] * m.n1 - 1), min(m.L[d], (ec[d] + 1) * m.n1 + 1)) for d in range(3)]
        XX, YY, ZZ = np.meshgrid(rng[0], rng[1], rng[2], indexing="ij")
        idx = inv[(XX + m.L[0] * (YY + m.L[1] * ZZ)).ravel()]
        z[:, idx] += np.linalg.solve(A[idx][:, idx].toarray(), r[:, idx].T).T
    return z


@pytest.mark.parametrize("lo,hi,n,p", [
    ([-2.0, -1.0, 0.5], [2.0, 1.5, 2.0], (3, 2, 2), 4),
    ([-3.0] * 3, [3.0] * 3, (2, 2, 2), 7),
])
def test_schwarz_smoother_and_coarse_solve(dgx, lo, hi, n, p):
    s = dgx.PoissonSolver(lo, hi, n, p)
    meshes = level_meshes(lo, hi, n, p)
    rng = np.random.default_rng(3)
    for l, m in enumerate(meshes):
        A = oracle.assemble_kron(m)
        r = rng.standard_normal((2, m.Nq))
        if l == len(meshes) - 1:
            ref = np.linalg.solve(A.toarray(), r.T).T
        else:
            ref = _patch_reference(A, m, r)
        got = s.smoother(torch.tensor(r, device="cuda"), level=l).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (l, np.abs(got - ref).max() / np.abs(ref).max())
        got32 = s.smoother(torch.tensor(r, device="cuda", dtype=torch.float32), level=l).cpu().double().numpy()
        assert np.abs(got32 - ref).max() <= 1e-4 * np.abs(ref).max()
    s.close()


def test_iteration_counts_are_small(dgx):
    """The Schwarz-smoothed V-cycle keeps PCG iterations low and nearly
    independent of the mesh (reported, loosely bounded)."""
    out = {}
    for (n, p) in [(4, 4), (8, 4), (4, 7)]:
        m = oracle.Mesh([-12.0] * 3, [12.0] * 3, n, p)
        f = _gauss_sources(m, [[0.5, -0.3, 0.2]], [0.8])
        s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, rtol=1e-8)
        _, st = s.solve(torch.tensor(f, device="cuda"))
        out[(n, p)] = st[0]["iters"]
        assert st[0]["status"] == 0
        s.close()
    assert max(out.values()) <= 15, out


def test_boundary_data_fp32_route_bound(dgx):
    """Mixed modes evaluate the Gaussian-sum boundary data in FP32 with a 1e-7
    table; the error relative to sum_q |W_q f_q| / r stays below 1e-5."""
    lo, hi, n, p = [-6.0] * 3, [6.0] * 3, (3, 3, 3), 5
    m = oracle.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(17)
    f = np.concatenate([_gauss_sources(m, [[0.3, -0.2, 0.1]], [1.5]), rng.standard_normal((1, m.Nq))])
    s = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED)
    assert s.info.n_gauss_fp32 > 0 and s.info.gauss_relerr_fp32 <= 1e-7
    g = s.boundary_data(torch.tensor(f, device="cuda"), route=1).cpu().numpy()
    ref = oracle.boundary_data_direct(m, f)
    bound = oracle.boundary_data_direct(m, np.abs(f))
    for k in range(f.shape[0]):
        faces = _face_arrays(g[k], m)
        for fi in range(6):
            err = np.abs(faces[fi] - ref[fi][k]).max() / bound[fi][k].max()
            assert err < 1e-5, (k, fi, err)
    s.close()


def test_mixed_precision_exchange_build_error_bounds(dgx):
    """Mixed mode (FP32 multigrid-PCG and boundary data, FP64 residuals and
    refinement) reaches the same 1e-8 FP64 residual; K, E_H, E_X and the
    potentials stay within the stated bounds of the FP64 oracle."""
    m = oracle.Mesh([-8.0] * 3, [8.0] * 3, 4, 5)
    atoms = np.array([[-1.0, 0.2, 0.0], [1.1, -0.3, 0.4], [0.0, 0.9, -0.8]])
    spec = inputs.gto_system(inputs.MeshSpec(tuple(m.lo), tuple(m.hi), m.n, m.p), atoms, 4, 5)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    ref = oracle.exchange_build(m, psi, method="fdm")
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=dgx.DG_PREC_MIXED, rtol=1e-8)
    K, eh, ex, stats = s.exchange_build(torch.tensor(psi, device="cuda"))
    assert all(st["status"] == 0 and st["rel_residual"] <= 1e-8 for st in stats)
    assert all(st["outer_refinements"] >= 1 for st in stats)
    assert np.abs(K - ref["K"]).max() <= 1e-6 * np.abs(ref["K"]).max()
    assert abs(eh - ref["E_H"]) <= 1e-6 * abs(ref["E_H"])
    assert abs(ex - ref["E_X"]) <= 1e-6 * abs(ref["E_X"])
    s.close()


@pytest.mark.parametrize("lo,hi,n,p", [
    ([-2.0, -1.0, 0.5], [2.0, 1.5, 2.0], (2, 4, 2), 6),
    ([-3.0] * 3, [3.0] * 3, (4, 4, 4), 7),
    ([-1.0, -2.0, -1.5], [1.0, 2.0, 2.0], (4, 2, 4), 8),
    ([-1.0] * 3, [1.0] * 3, (6, 6, 6), 5),
    ([-2.0] * 3, [2.0] * 3, (8, 8, 8), 2),
])
def test_transfers_all_levels(dgx, lo, hi, n, p):
    """Prolongation and restriction between every pair of levels against the
    oracle's interpolation matrix P (built from node coordinates) and P^T."""
    s = dgx.PoissonSolver(lo, hi, n, p)
    meshes = level_meshes(lo, hi, n, p)
    assert s.info.levels == len(meshes)
    rng = np.random.default_rng(2)
    for l in range(len(meshes) - 1):
        fine, coarse = meshes[l], meshes[l + 1]
        P = oracle.transfer_matrix(fine, coarse)
        uc = rng.standard_normal((3, coarse.Nq))
        rf = rng.standard_normal((3, fine.Nq))
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
            got = dgx.dg_apply_transfer(s.h, torch.tensor(uc, device="cuda", dtype=dt), l, 0, fine.Nq)
            ref = (P @ uc.T).T
            assert np.abs(got.cpu().double().numpy() - ref).max() <= tol * np.abs(ref).max(), (l, dt)
            got = dgx.dg_apply_transfer(s.h, torch.tensor(rf, device="cuda", dtype=dt), l, 1, coarse.Nq)
            ref = (P.T @ rf.T).T
            assert np.abs(got.cpu().double().numpy() - ref).max() <= tol * np.abs(ref).max(), (l, dt)
    with pytest.raises(dgx.DGError):
        dgx.dg_apply_transfer(s.h, torch.zeros((1, meshes[-1].Nq), device="cuda", dtype=torch.float64),
                              len(meshes) - 1, 0, 1)
    s.close()
