"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed-form integrals and potentials, polynomial exactness, symmetry, brute
force on tiny meshes and invariances. None of these needs a GPU.

The paper prints no worked numbers for the Poisson / exchange path, so every
pin here is a closed form, an invariant or an independent construction.
"""

import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from oracle import dg_oracle as O
from paper_2510_21213_gb300 import inputs


# ---------------------------------------------------------------------------
# Quadrature and the nodal basis (Sec. 6.2: degree-q nodal GL elements whose
# nodes double as the quadrature rule)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_gl_exact_on_box_monomials(p):
    m = oracle.Mesh([-1.3, -0.4, 0.2], [0.9, 1.6, 2.2], (2, 3, 2), p)
    x = oracle.node_coords(m)
    W = oracle.quad_weights(m)
    assert abs(W.sum() - np.prod(m.hi - m.lo)) < 1e-13 * np.prod(m.hi - m.lo)

    def exact(a, b, c):
        val = 1.0
        for d, k in enumerate((a, b, c)):
            val *= (m.hi[d] ** (k + 1) - m.lo[d] ** (k + 1)) / (k + 1)
        return val

    for (a, b, c) in [(2 * p + 1, 0, 0), (0, 2 * p + 1, 1), (p, p + 1, 2 * p + 1), (2 * p + 1,) * 3]:
        got = np.sum(W * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
        ref = exact(a, b, c)
        assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (a, b, c, got, ref)
    # one degree more is not integrated exactly (the rule is not over-exact)
    a = 2 * p + 2
    m1 = oracle.Mesh([0.0] * 3, [1.0] * 3, (1, 1, 1), p)
    got = np.sum(oracle.quad_weights(m1) * oracle.node_coords(m1)[:, 0] ** a)
    assert abs(got - 1.0 / (a + 1)) > 1e-10


@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_lagrange_interpolates_and_differentiates_polynomials(p):
    xi, _ = oracle.gauss_legendre(p + 1)
    L, dL = oracle.lagrange_eval(xi, xi)
    assert np.allclose(L, np.eye(p + 1), atol=1e-13)
    rng = np.random.default_rng(p)
    coef = rng.standard_normal(p + 1)
    poly = np.polynomial.Polynomial(coef)
    pts = np.linspace(-1.0, 1.0, 11)
    Lp, dLp = oracle.lagrange_eval(xi, pts)
    assert np.allclose(Lp @ poly(xi), poly(pts), atol=1e-12)
    assert np.allclose(dLp @ poly(xi), poly.deriv()(pts), atol=1e-11)


@pytest.mark.parametrize("p", [1, 4, 7])
def test_collocated_mass_is_exact(p):
    """The diagonal GL mass w_a h/2 equals the exact int l_a l_b (Gauss rule
    with more points), so the Kronecker form uses the exact mass."""
    xi, w = oracle.gauss_legendre(p + 1)
    xq, wq = oracle.gauss_legendre(p + 4)
    L, _ = oracle.lagrange_eval(xi, xq)
    Mex = L.T @ (wq[:, None] * L)
    assert np.allclose(Mex, np.diag(w), atol=1e-14)


# ---------------------------------------------------------------------------
# SIPDG operator (Sec. 3.4 eq. sip_bilinear, Sec. 3.5, Sec. 6.3)
# ---------------------------------------------------------------------------
TINY = [
    ([-1.0, -2.0, -1.5], [1.0, 2.0, 2.0], (2, 2, 3), 2),
    ([-3.0] * 3, [3.0] * 3, (3, 3, 3), 1),
    ([-2.0, -1.0, 0.0], [2.0, 1.0, 1.5], (1, 2, 2), 3),
]


@pytest.mark.parametrize("lo,hi,n,p", TINY)
@pytest.mark.parametrize("form", [0, 1])
def test_dense_equals_kronecker_and_spd(lo, hi, n, p, form):
    m = oracle.Mesh(lo, hi, n, p)
    Ad = oracle.assemble_dense(m, penalty_form=form)
    Ak = oracle.assemble_kron(m, penalty_form=form).toarray()
    scale = np.abs(Ad).max()
    assert np.abs(Ad - Ak).max() <= 1e-13 * scale
    assert np.abs(Ad - Ad.T).max() <= 1e-13 * scale
    assert np.linalg.eigvalsh(Ad).min() > 0.0


def _poly_problem(m):
    def u(P):
        return P[..., 0] ** 2 * P[..., 1] - 3.0 * P[..., 2] + P[..., 0] * P[..., 1] * P[..., 2] ** 2 + 0.5

    def lap(P):
        return 2.0 * P[..., 1] + 2.0 * P[..., 0] * P[..., 1]

    x = oracle.node_coords(m)
    f = -lap(x) / (4.0 * math.pi)
    g = [u(pts) for pts in oracle.boundary_face_nodes(m)]
    return u(x), f, g


@pytest.mark.parametrize("lo,hi,n,p", [TINY[0], ([-2.0, -1.0, 0.0], [2.0, 1.0, 1.5], (2, 1, 2), 3)])
@pytest.mark.parametrize("form", [0, 1])
def test_polynomial_reproduction(lo, hi, n, p, form):
    """SIP + Nitsche is consistent: a global Q_p solution with f = -Lap u/(4 pi)
    and g = u on the boundary is reproduced to round-off. This pins the sign
    and weight of every face, boundary and load term."""
    m = oracle.Mesh(lo, hi, n, p)
    uex, f, g = _poly_problem(m)
    b = oracle.rhs(m, f, g, penalty_form=form)
    v = oracle.solve_dense(oracle.assemble_dense(m, penalty_form=form), b)
    assert np.abs(v - uex).max() < 1e-11 * np.abs(uex).max()
    v2 = oracle.solve_fdm(m, b, penalty_form=form)
    assert np.abs(v2 - uex).max() < 1e-11 * np.abs(uex).max()


def test_planted_mistake_is_caught(monkeypatch):
    """Flip the sign of the endpoint derivatives (a wrong normal in the trace of
    grad v): polynomial reproduction must fail."""
    m = oracle.Mesh(*TINY[0])
    real = O.lagrange_eval

    def wrong(nodes, x):
        L, dL = real(nodes, x)
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        ends = np.abs(np.abs(x) - 1.0) < 1e-15
        dL[ends] *= -1.0
        return L, dL

    monkeypatch.setattr(O, "lagrange_eval", wrong)
    uex, f, g = _poly_problem(m)
    b = oracle.rhs(m, f, g)
    v = oracle.solve_dense(oracle.assemble_dense(m), b)
    assert np.abs(v - uex).max() > 1e-3 * np.abs(uex).max()


@pytest.mark.parametrize("lo,hi,n,p", TINY)
def test_fdm_equals_cholesky(lo, hi, n, p):
    m = oracle.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(5)
    b = rng.standard_normal((2, m.Nq))
    A = oracle.assemble_dense(m)
    x1 = np.stack([oracle.solve_dense(A, bb) for bb in b])
    x2 = oracle.solve_fdm(m, b)
    assert np.abs(x1 - x2).max() <= 1e-10 * np.abs(x1).max()


# ---------------------------------------------------------------------------
# Boundary data and Gaussian potentials (Sec. 6.3)
# ---------------------------------------------------------------------------
A_EXP = 2.0
CENTER = np.array([0.35, -0.2, 0.1])


def _unit_gaussian(x):
    r = np.linalg.norm(x - CENTER, axis=-1)
    return (A_EXP / math.pi) ** 1.5 * np.exp(-A_EXP * r * r)


def _erf_potential(x):
    r = np.linalg.norm(x - CENTER, axis=-1)
    return erf(math.sqrt(A_EXP) * r) / r


def test_boundary_data_matches_erf_potential():
    errs = []
    for p in (4, 6, 8):
        m = oracle.Mesh([-8.0] * 3, [8.0] * 3, 4, p)
        g = oracle.boundary_data_direct(m, _unit_gaussian(oracle.node_coords(m)))
        errs.append(max(np.abs(gf - _erf_potential(pts)).max() for gf, pts in zip(g, oracle.boundary_face_nodes(m))))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_boundary_data_direct_brute_force():
    m = oracle.Mesh([-2.0, -1.0, -1.0], [2.0, 1.0, 1.5], (2, 1, 2), 2)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(m.Nq)
    g = oracle.boundary_data_direct(m, f, chunk=7)
    x = oracle.node_coords(m)
    W = oracle.quad_weights(m)
    for face, pts in enumerate(oracle.boundary_face_nodes(m)):
        for (i, j) in [(0, 0), (pts.shape[0] - 1, pts.shape[1] - 1), (1, 2)]:
            ref = sum(W[q] * f[q] / math.dist(pts[i, j], x[q]) for q in range(m.Nq))
            assert abs(g[face][i, j] - ref) < 1e-12 * max(1.0, abs(ref))


def test_gaussian_potential_converges_to_erf():
    """A unit Gaussian charge has v = erf(sqrt(a) r)/r; the discrete solution
    converges to it under p- and h-refinement."""
    errs = {}
    for (n, p) in [(4, 4), (4, 6), (4, 8), (8, 4)]:
        m = oracle.Mesh([-8.0] * 3, [8.0] * 3, n, p)
        x = oracle.node_coords(m)
        v, _ = oracle.poisson(m, _unit_gaussian(x), method="fdm")
        errs[(n, p)] = np.abs(v[0] - _erf_potential(x)).max()
    assert errs[(4, 4)] > errs[(4, 6)] > errs[(4, 8)]
    assert errs[(4, 4)] > 4 * errs[(8, 4)]
    assert errs[(4, 8)] < 5e-3


def test_hartree_self_energy_converges():
    """(rho|rho) of a unit Gaussian of exponent a is sqrt(2a/pi)."""
    ref = math.sqrt(2.0 * A_EXP / math.pi)
    errs = []
    for p in (4, 6, 8):
        m = oracle.Mesh([-8.0] * 3, [8.0] * 3, 4, p)
        x = oracle.node_coords(m)
        f = _unit_gaussian(x)
        v, _ = oracle.poisson(m, f, method="fdm")
        errs.append(abs(np.sum(oracle.quad_weights(m) * f * v[0]) - ref))
    assert errs[0] > 100 * errs[2]
    assert errs[2] < 1e-4


# ---------------------------------------------------------------------------
# Exchange matrix and energies (Sec. 6.1.2 eq. fock_exchange, Sec. 2.3.1)
# ---------------------------------------------------------------------------
def _tiny_continuum():
    """Free-space values for two normalised s-Gaussians (exponent 1) at
    (+-0.7, 0, 0), from the Gaussian product theorem and the Coulomb energy of
    two unit Gaussians, erf(sqrt(ab/(a+b)) R)/R."""
    S = math.exp(-0.98)
    i1111 = 2.0 / math.sqrt(math.pi)
    i1212 = S * S * i1111
    i1122 = math.erf(1.4) / 1.4
    i1112 = S * math.erf(0.7) / 0.7
    return {"K11": i1111 + i1212, "K12": 2.0 * i1112, "E_H": 0.5 * (2 * i1111 + 2 * i1122), "i1111": i1111,
            "i1212": i1212}


def test_tiny_system_converges_to_continuum():
    ref = _tiny_continuum()
    spec = inputs.tiny_system()
    errs = []
    for (n, p) in [(4, 4), (4, 6)]:
        m = oracle.Mesh([-8.0] * 3, [8.0] * 3, n, p)
        psi = inputs.orbitals(spec, oracle.node_coords(m))
        r = oracle.exchange_build(m, psi, method="fdm")
        # pair self-energies (11|11), (12|12), (22|22): sources 1, 2, 3 of the list
        se = r["self"]
        errs.append(max(abs(r["K"][0, 0] - ref["K11"]), abs(r["K"][0, 1] - ref["K12"]), abs(r["E_H"] - ref["E_H"]),
                        abs(se[1] - ref["i1111"]), abs(se[3] - ref["i1111"]), abs(se[2] - ref["i1212"])))
        assert abs(r["E_X"] + 0.5 * np.trace(r["K"])) < 1e-15
        assert abs(se[0] - 2.0 * r["E_H"]) < 1e-14 * se[0]
    assert errs[0] > 10 * errs[1]
    assert errs[1] < 5e-3


def _small_system(seed=11, N=4):
    m = oracle.Mesh([-6.0] * 3, [6.0] * 3, 2, 4)
    atoms = np.array([[-1.0, 0.2, 0.0], [1.1, -0.3, 0.4], [0.0, 0.9, -0.8]])
    spec = inputs.gto_system(inputs.MeshSpec(tuple(m.lo), tuple(m.hi), m.n, m.p), atoms, N, seed)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    return m, psi


def test_exchange_matrix_symmetric_psd_and_rotation_invariant():
    m, psi = _small_system()
    r = oracle.exchange_build(m, psi, method="fdm")
    K = r["K"]
    nrm = np.abs(K).max()
    # the Dirichlet lift makes K non-symmetric at discretisation level only
    assert np.abs(K - K.T).max() < 1e-2 * nrm
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > -1e-10 * nrm
    # K_ii = sum_s (is|si) >= (ii|ii) > 0
    Wq = oracle.quad_weights(m)
    for i in range(psi.shape[0]):
        v, _ = oracle.poisson(m, psi[i] * psi[i], method="fdm")
        self_e = np.sum(Wq * psi[i] * psi[i] * v[0])
        assert self_e > 0 and K[i, i] >= self_e - 1e-12
    # orthogonal rotation of the orbitals: K -> Q K Q^T, energies unchanged
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((psi.shape[0],) * 2))
    r2 = oracle.exchange_build(m, Q @ psi, method="fdm")
    assert np.abs(r2["K"] - Q @ K @ Q.T).max() < 1e-11 * nrm
    assert abs(r2["E_H"] - r["E_H"]) < 1e-11 * abs(r["E_H"])
    assert abs(r2["E_X"] - r["E_X"]) < 1e-11 * abs(r["E_X"])


def test_pair_list_order():
    assert oracle.pair_list(3) == [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    assert len(oracle.pair_list(64)) == 2080


def test_gaussian_sum_route_matches_direct_quadrature():
    """The separable Gaussian-sum evaluation of the Dirichlet data (Sec. 5.2
    applied to Sec. 6.3) agrees with the direct quadrature within its bound."""
    m = oracle.Mesh([-4.0, -3.0, -3.5], [4.0, 3.5, 3.0], (3, 2, 3), 4)
    rng = np.random.default_rng(7)
    f = np.concatenate([rng.standard_normal((1, m.Nq)), _unit_gaussian(oracle.node_coords(m))[None, :]])
    g1 = oracle.boundary_data_direct(m, f)
    g2 = oracle.boundary_data_gausssum(m, f, tol=1e-12)
    bound = oracle.boundary_data_direct(m, np.abs(f))
    for a, b, c in zip(g1, g2, bound):
        assert np.abs(a - b).max() <= 2e-12 * c.max()
    c, a, err = oracle.gauss_sum_1_over_r(0.03, 42.0, 1e-10)
    r = np.exp(np.linspace(math.log(0.03), math.log(42.0), 777))
    assert np.abs((np.exp(-np.outer(r * r, a)) @ c) * r - 1.0).max() <= 1e-10 and err <= 1e-10


def test_ace_operator_pins():
    """The compressed exchange operator: exact on the occupied orbitals
    (V_X psi_i = -W_i), symmetric and negative semidefinite in the quadrature
    inner product, and zero on the W_q-orthogonal complement of span(W)."""
    spec = inputs.chain_system(n=2, p=4, n_orb=3)
    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
    Wq = oracle.quad_weights(m)
    psi = inputs.orbitals(spec, oracle.node_coords(m), Wq)
    build = oracle.exchange_build(m, psi)
    W, K = build["W"], build["K"]
    asym = np.abs(K - K.T).max() / np.abs(K).max()
    got = oracle.ace_apply(build, Wq, psi)
    assert np.abs(got + W).max() <= (1e-10 + 10 * asym) * np.abs(W).max()
    rng = np.random.default_rng(4)
    U = rng.standard_normal((4, Wq.size))
    AU = oracle.ace_apply(build, Wq, U)
    G = (U * Wq) @ AU.T  # <u_a, A u_b>
    assert np.abs(G - G.T).max() <= 1e-12 * np.abs(G).max()
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).max() <= 1e-12 * np.abs(G).max()
    # component of U orthogonal (in the W_q inner product) to span(W): mapped to zero
    Gw = (W * Wq) @ W.T
    Up = U - (np.linalg.solve(Gw, (W * Wq) @ U.T)).T @ W
    assert np.abs(oracle.ace_apply(build, Wq, Up)).max() <= 1e-10 * np.abs(AU).max()


def test_jk_action_pins():
    """The Hartree and exchange actions on trial functions (Sec. 2.3.1):
    on the occupied orbitals the exchange action is minus the build's
    accumulation W (so <psi_i, X psi_j> = -K_ij) and sum_i <psi_i, J psi_i> =
    2 E_H; for one orbital J psi + X psi = 0 (no self-interaction); X is
    linear and negative semidefinite up to the asymmetry of the boundary
    data."""
    spec = inputs.chain_system(n=2, p=4, n_orb=3)
    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
    Wq = oracle.quad_weights(m)
    psi = inputs.orbitals(spec, oracle.node_coords(m), Wq)
    build = oracle.exchange_build(m, psi)
    W, K = build["W"], build["K"]
    JU, XU = oracle.jk_apply(m, psi, psi)
    assert np.abs(XU + W).max() <= 1e-12 * np.abs(W).max()
    assert np.abs((psi * Wq) @ XU.T + K).max() <= 1e-12 * np.abs(K).max()
    assert abs(float(np.sum(Wq * psi * JU)) - 2.0 * build["E_H"]) <= 1e-12 * abs(build["E_H"])
    # one orbital: the pair source psi psi is the density, so X psi = -J psi
    J1, X1 = oracle.jk_apply(m, psi[:1], psi[:1])
    assert np.abs(J1 + X1).max() <= 1e-12 * np.abs(J1).max()
    # linearity in the trial function, and the operator flags
    rng = np.random.default_rng(11)
    U = rng.standard_normal((3, Wq.size))
    JU, XU = oracle.jk_apply(m, psi, U)
    Jc, Xc = oracle.jk_apply(m, psi, (2.0 * U[0] - 3.0 * U[1])[None, :], hartree=True, exchange=True)
    assert np.abs(Xc[0] - (2.0 * XU[0] - 3.0 * XU[1])).max() <= 1e-11 * np.abs(XU).max()
    assert np.abs(Jc[0] - (2.0 * JU[0] - 3.0 * JU[1])).max() <= 1e-11 * np.abs(JU).max()
    assert oracle.jk_apply(m, psi, U, exchange=False)[1] is None
    assert oracle.jk_apply(m, psi, U, hartree=False)[0] is None
    # <u_a, X u_b>: symmetric up to the boundary-data asymmetry seen in K, and
    # its symmetric part negative semidefinite to the same order
    asym = np.abs(K - K.T).max() / np.abs(K).max()
    G = (U * Wq) @ XU.T
    scale = np.abs(G).max()
    assert np.abs(G - G.T).max() <= (1e-12 + 10 * asym) * scale
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).max() <= (1e-12 + 10 * asym) * scale
    assert np.all(np.diag(G) < 0)


def test_transfer_matrix_reproduces_piecewise_polynomials():
    """Prolongation of the hp hierarchy (Sec. 6.4): a field that is, in every
    coarse element, a polynomial of the coarse degree plus its own constant is
    reproduced exactly at the fine nodes, for p-transfers (same mesh) and the
    degree-1 h-transfer (8 children). The per-element constants check that
    every fine node is given its own coarse element."""
    rng = np.random.default_rng(8)
    lo, hi = np.array([-2.0, -1.0, 0.5]), np.array([2.0, 1.5, 2.5])
    cases = [((2, 3, 2), 6, (2, 3, 2), 3), ((2, 2, 2), 3, (2, 2, 2), 1), ((4, 2, 6), 1, (2, 1, 3), 1)]
    for nf, pf, nc, pc in cases:
        fine, coarse = oracle.Mesh(lo, hi, nf, pf), oracle.Mesh(lo, hi, nc, pc)
        jump = rng.standard_normal(coarse.E)

        def field(x, e):
            X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
            poly = 0.3 + X ** pc * Y - 2.0 * Z ** pc + X * Y ** max(pc - 1, 0) * Z
            return poly + jump[e]

        xc = oracle.node_coords(coarse)
        ec = np.repeat(np.arange(coarse.E), coarse.npe)
        xf = oracle.node_coords(fine)
        hc = coarse.h
        idx = np.clip(np.floor((xf - coarse.lo) / hc).astype(int), 0, np.asarray(coarse.n) - 1)
        ef = idx[:, 0] + coarse.n[0] * (idx[:, 1] + coarse.n[1] * idx[:, 2])
        P = oracle.transfer_matrix(fine, coarse)
        got = P @ field(xc, ec)
        ref = field(xf, ef)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (nf, pf, nc, pc)
        # a field of one degree more is not reproduced (the interpolation is not over-exact)
        if pf > pc:
            bad = P @ (xc[:, 0] ** (pc + 1)) - xf[:, 0] ** (pc + 1)
            assert np.abs(bad).max() > 1e-6
