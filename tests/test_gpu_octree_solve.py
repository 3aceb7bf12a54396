"""Poisson solves and the exchange build on the octree auxiliary mesh
(dg_octree_setup / dg_octree_solve / dg_octree_exchange_build) against the
oracle's dense Cholesky solve on meshes with hanging faces (Sec. 6.2, 6.3)."""

import math

import numpy as np
import pytest

import oracle
from oracle import octree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LO, HI = [-1.0, -1.5, -1.0], [1.0, 1.5, 2.0]


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    dgx.load()
    return dgx


def _three_levels(p, lo=LO, hi=HI):
    t = octree.OctreeMesh(lo, hi, (2, 2, 2), p)
    t.refine([(0, 0, 0, 0)])
    t.refine([(1, 1, 1, 1)])
    t.balance()
    return t


def _one_split(p):
    t = octree.OctreeMesh(LO, HI, (2, 1, 1), p)
    t.refine([(0, 1, 0, 0)])
    return t


def _solver(dgx, t, **kw):
    return dgx.OctreeSolver(t.lo, t.hi, t.n, t.p, np.array(t.leaf_list(), dtype=np.int32), **kw)


def _gauss_source(t, centre=(0.2, -0.1, 0.3), alpha=3.0):
    x = t.node_coords()
    d = x - np.asarray(centre)[None, :]
    return np.exp(-alpha * np.einsum("qi,qi->q", d, d))


@pytest.mark.parametrize("mesh,p,form", [("three", 2, 0), ("three", 3, 1), ("one", 5, 0), ("one", 8, 0)])
def test_precond_is_the_inverse_of_the_diagonal_blocks(dgx, mesh, p, form):
    """z = P r equals the exact inverse of the oracle matrix's leaf blocks
    (the fast-diagonalisation factors of every leaf class)."""
    t = _three_levels(p) if mesh == "three" else _one_split(p)
    A = octree.assemble(t, penalty_form=form)
    npe = t.npe
    rng = np.random.default_rng(10 + p)
    r = rng.standard_normal((2, t.Nq))
    ref = np.empty_like(r)
    for e in range(t.E):
        s = slice(e * npe, (e + 1) * npe)
        ref[:, s] = np.linalg.solve(A[s, s], r[:, s].T).T
    s = _solver(dgx, t, penalty_form=form, precond=0)
    got = s.precond(torch.tensor(r, device="cuda")).cpu().numpy()
    s.close()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_node_coords_and_weights_are_the_oracle_ones(dgx):
    t = _three_levels(3)
    s = _solver(dgx, t)
    xyz, w = s.node_coords()
    s.close()
    assert np.abs(xyz.cpu().numpy() - t.node_coords()).max() <= 1e-14
    assert np.abs(w.cpu().numpy() - t.quad_weights()).max() <= 1e-15 * t.quad_weights().max() * 10


@pytest.mark.parametrize("mesh,p,form,pc", [("three", 3, 0, 1), ("three", 2, 1, 1), ("one", 6, 0, 1),
                                            ("three", 7, 0, 1), ("three", 3, 0, 0)])
def test_solve_matches_the_dense_oracle(dgx, mesh, p, form, pc):
    """Coulomb boundary data by direct quadrature, Nitsche load, PCG to rtol
    1e-13 (V-cycle or leaf-block preconditioner): v equals the oracle's
    Cholesky solution of the same system."""
    t = _three_levels(p) if mesh == "three" else _one_split(p)
    f = np.stack([_gauss_source(t), _gauss_source(t, (-0.4, 0.5, 0.9), 1.5)])
    ref = np.stack([octree.poisson(t, fk, penalty_form=form) for fk in f])
    s = _solver(dgx, t, penalty_form=form, rtol=1e-13, precond=pc)
    v, st = s.solve(torch.tensor(f, device="cuda"))
    s.close()
    v = v.cpu().numpy()
    assert all(x["status"] == 0 and x["rel_residual"] <= 1e-13 for x in st)
    assert np.abs(v - ref).max() <= 1e-10 * np.abs(ref).max()
    W = t.quad_weights()
    for k in range(2):
        se_ref = float(np.sum(W * f[k] * ref[k]))
        assert abs(st[k]["self_energy"] - se_ref) <= 1e-11 * abs(se_ref)


def test_solve_edge_cases(dgx):
    """A zero source gives v = 0 in no iterations; a source with a NaN is
    reported (DG_ERR_NONFINITE, v = 0) and leaves the others bit-identical."""
    t = _one_split(3)
    s = _solver(dgx, t, rtol=1e-12)
    f = _gauss_source(t)
    bad = f.copy()
    bad[5] = np.nan
    both = torch.tensor(np.stack([f, np.zeros_like(f), bad, 2.0 * f]), device="cuda")
    v, st = s.solve(both, allow_unconverged=True)
    alone, st1 = s.solve(torch.tensor(np.stack([f, 2.0 * f]), device="cuda"))
    s.close()
    assert st[1]["status"] == 0 and st[1]["iters"] == 0 and float(v[1].abs().max()) == 0.0
    assert st[2]["status"] == -5 and float(v[2].abs().max()) == 0.0
    assert torch.equal(v[0], alone[0]) and torch.equal(v[3], alone[1])
    assert st[0]["iters"] == st1[0]["iters"]


def test_exchange_build_matches_the_oracle_on_a_refined_octree(dgx):
    """Hartree and pair solves, accumulation, K and energies on an octree refined
    by the density indicator of Sec. 6.2 around the two atoms of the tiny
    system: equal to the oracle's dense exchange build."""
    from paper_2510_21213_gb300 import inputs

    spec = inputs.tiny_system()
    lo, hi = list(spec.mesh.lo), list(spec.mesh.hi)
    t = octree.OctreeMesh(lo, hi, (2, 2, 2), 3)

    def rho(P):
        return np.sum(inputs.orbitals(spec, P) ** 2, axis=0)

    octree.refine_to_density(t, rho, 1e-3, 2)
    assert t.E > 8 and any(k[0] == 2 for k in t.leaves)
    psi = inputs.orbitals(spec, t.node_coords())
    ref = octree.exchange_build(t, psi)
    s = _solver(dgx, t, rtol=1e-13)
    K, EH, EX, st = s.exchange_build(torch.tensor(psi, device="cuda"))
    s.close()
    assert all(x["status"] == 0 for x in st)
    assert np.abs(K - ref["K"]).max() <= 1e-10 * np.abs(ref["K"]).max()
    assert abs(EH - ref["E_H"]) <= 1e-10 * abs(ref["E_H"])
    assert abs(EX - ref["E_X"]) <= 1e-10 * abs(ref["E_X"])
    # the Hartree self-energy is 2 E_H
    assert abs(st[0]["self_energy"] - 2.0 * EH) <= 1e-14 * abs(EH)


def test_handle_operator_is_dg_octree_apply(dgx):
    """The handle's operator (tables and connectivity kept on the device) gives
    bit for bit what the per-call dg_octree_apply gives, and refuses aliased
    fields."""
    t = _three_levels(4)
    leaves = np.array(t.leaf_list(), dtype=np.int32)
    u = torch.randn(3, t.Nq, dtype=torch.float64, device="cuda")
    ref = dgx.dg_octree_apply(t.lo, t.hi, t.n, t.p, leaves, u)
    s = _solver(dgx, t)
    got = s.apply(u)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    lib = dgx.load()
    ptr = dgx.C.c_void_p(u.data_ptr())
    assert lib.dg_octree_operator(s.h, ptr, ptr, 3, None) == dgx.DG_ERR_INVALID_ARG
    s.close()


def test_vcycle_is_symmetric_and_positive(dgx):
    """PCG needs a symmetric positive preconditioner: (u, V w) = (V u, w) and
    (u, V u) > 0 for the V-cycle (same Chebyshev polynomial before and after
    the coarse correction, restriction the transpose of prolongation)."""
    t = _three_levels(4)
    s = _solver(dgx, t)
    g = torch.Generator(device="cpu").manual_seed(5)
    u = torch.randn(2, t.Nq, generator=g, dtype=torch.float64).cuda()
    Vu = s.precond(u)
    s.close()
    a = float((u[0] * Vu[1]).sum())
    b = float((Vu[0] * u[1]).sum())
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert float((u[0] * Vu[0]).sum()) > 0 and float((u[1] * Vu[1]).sum()) > 0


def test_vcycle_cuts_iterations_on_a_refined_octree(dgx):
    """On the density-refined octree of the tiny system (three leaf levels,
    hanging faces), the V-cycle preconditioner reaches 1e-10 in a small
    fraction of the leaf-block preconditioner's iterations, with the same
    solution."""
    from paper_2510_21213_gb300 import inputs

    spec = inputs.tiny_system()
    t = octree.OctreeMesh(list(spec.mesh.lo), list(spec.mesh.hi), (2, 2, 2), 4)

    def rho(P):
        return np.sum(inputs.orbitals(spec, P) ** 2, axis=0)

    octree.refine_to_density(t, rho, 1e-5, 3)
    assert sorted({k[0] for k in t.leaves}) == [1, 2, 3]
    f = torch.tensor(rho(t.node_coords())[None, :], device="cuda")
    its = {}
    sol = {}
    for pc in (0, 1):
        s = _solver(dgx, t, rtol=1e-10, precond=pc)
        sol[pc], st = s.solve(f)
        s.close()
        its[pc] = st[0]["iters"]
    assert its[1] <= 30 and its[1] * 5 <= its[0], its
    assert float((sol[1] - sol[0]).abs().max()) <= 1e-7 * float(sol[0].abs().max())


def test_solution_does_not_depend_on_the_batch(dgx):
    """Every per-source sum runs in a fixed order that does not depend on how
    many sources share the call (boundary-data tiles of 16 sources, dots,
    operator blocks): the 18th source of a batch is bit-identical to the same
    source solved alone."""
    t = _three_levels(3)
    s = _solver(dgx, t, rtol=1e-11)
    f = np.stack([_gauss_source(t, (0.1 * k - 0.5, 0.2, -0.1), 1.0 + 0.1 * k) for k in range(18)])
    v, _ = s.solve(torch.tensor(f, device="cuda"))
    v1, _ = s.solve(torch.tensor(f[17:], device="cuda"))
    s.close()
    assert torch.equal(v[17], v1[0])


# Mixed mode: FP32 inner PCG and V-cycle inside FP64 refinement; the boundary
# data as a 3xTF32 GEMM against the FP32 kernel matrix 1/|x_j - x_q| (about
# 1e-7 of sum |W f| / r). Stated bound against the FP64 oracle: 2e-5 of the
# largest entry on v, K, E_H, E_X (as for the uniform mesh's mixed mode).
MIXED_BOUND = 2e-5


@pytest.mark.parametrize("mesh,p", [("three", 3), ("one", 7)])
def test_mixed_precision_solve_matches_the_oracle(dgx, mesh, p):
    """Refined to a 1e-12 FP64 residual of its own right-hand side, the mixed
    mode's potentials are within the mixed bound of the oracle's exact solve
    (the difference is the FP32 boundary data's)."""
    t = _three_levels(p) if mesh == "three" else _one_split(p)
    f = np.stack([_gauss_source(t), _gauss_source(t, (-0.4, 0.5, 0.9), 1.5)])
    ref = np.stack([octree.poisson(t, fk) for fk in f])
    s = _solver(dgx, t, rtol=1e-12, precision=dgx.DG_PREC_MIXED)
    v, st = s.solve(torch.tensor(f, device="cuda"))
    s.close()
    assert all(x["status"] == 0 and x["rel_residual"] <= 1e-12 and x["outer_refinements"] >= 2 for x in st)
    err = np.abs(v.cpu().numpy() - ref).max() / np.abs(ref).max()
    print(f"mixed octree solve, {mesh} p = {p}: {err:.2e} of max |v|")
    assert err <= MIXED_BOUND


def test_mixed_precision_exchange_build_matches_the_oracle(dgx):
    """The mixed mode's exchange build on the density-refined octree of the
    two-atom system at rtol 1e-10: K, E_H, E_X within the mixed bound."""
    from paper_2510_21213_gb300 import inputs

    spec = inputs.tiny_system()
    t = octree.OctreeMesh(list(spec.mesh.lo), list(spec.mesh.hi), (2, 2, 2), 3)

    def rho(P):
        return np.sum(inputs.orbitals(spec, P) ** 2, axis=0)

    octree.refine_to_density(t, rho, 1e-3, 2)
    psi = inputs.orbitals(spec, t.node_coords())
    ref = octree.exchange_build(t, psi)
    s = _solver(dgx, t, rtol=1e-10, precision=dgx.DG_PREC_MIXED)
    K, EH, EX, st = s.exchange_build(torch.tensor(psi, device="cuda"))
    s.close()
    assert all(x["status"] == 0 for x in st)
    eK = np.abs(K - ref["K"]).max() / np.abs(ref["K"]).max()
    eH, eX = abs(EH - ref["E_H"]) / abs(ref["E_H"]), abs(EX - ref["E_X"]) / abs(ref["E_X"])
    print(f"mixed octree build: K {eK:.2e}, E_H {eH:.2e}, E_X {eX:.2e}")
    assert eK <= MIXED_BOUND and eH <= MIXED_BOUND and eX <= MIXED_BOUND
