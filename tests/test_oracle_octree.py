"""Pins of the octree auxiliary-mesh oracle (Sec. 6.2) against facts outside
it: without refinement it is the uniform oracle; on meshes with 2:1 hanging
faces the SIPDG problem reproduces Q_p polynomial solutions to round-off
(this pins every face, hanging or not, and the Nitsche terms); the matrix is
symmetric and positive definite; the tree stays 2:1 balanced; the density
indicator drives refinement where the density varies."""

import math

import numpy as np
import pytest

import oracle
from oracle import octree


def _u(P):
    return P[:, 0] ** 2 * P[:, 1] - 3.0 * P[:, 2] + P[:, 0] * P[:, 1] * P[:, 2] ** 2 + 0.5


def _lap_u(P):
    return 2.0 * P[:, 1] + 2.0 * P[:, 0] * P[:, 1]


LO, HI = [-1.0, -1.5, -1.0], [1.0, 1.5, 2.0]


def test_unrefined_octree_is_the_uniform_oracle():
    t = octree.OctreeMesh(LO, HI, (2, 2, 2), 2)
    m = oracle.Mesh(LO, HI, (2, 2, 2), 2)
    assert np.abs(t.node_coords() - oracle.node_coords(m)).max() < 1e-14
    assert np.abs(t.quad_weights() - oracle.quad_weights(m)).max() < 1e-15
    A = octree.assemble(t)
    Ad = oracle.assemble_dense(m)
    assert np.abs(A - Ad).max() <= 1e-12 * np.abs(Ad).max()


def _refined(p):
    t = octree.OctreeMesh(LO, HI, (2, 2, 2), p)
    t.refine([(0, 0, 0, 0)])
    t.refine([(1, 1, 1, 1)])  # level-2 cells next to level-0 leaves: balancing must split those
    t.balance()
    return t


@pytest.mark.parametrize("p", [2, 3])
def test_hanging_faces_reproduce_polynomials(p):
    t = _refined(p)
    assert t.is_balanced()
    levels = {k[0] for k in t.leaves}
    assert levels == {0, 1, 2}
    A = octree.assemble(t)
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-13 * scale
    assert np.linalg.eigvalsh(A).min() > 0.0
    x = t.node_coords()
    b = octree.rhs(t, -_lap_u(x) / (4.0 * math.pi), g=_u)
    v = np.linalg.solve(A, b)
    ref = _u(x)
    assert np.abs(v - ref).max() < 1e-10 * np.abs(ref).max()


def test_wrong_hanging_face_fails_reproduction(monkeypatch):
    """A planted mistake: hanging faces integrated with the larger element's
    size in the face weights. Polynomial reproduction must fail."""
    t = _refined(2)
    real = octree._face_quadrature

    def wrong(mesh, K, d, s, xq, wq):
        axes, w = real(mesh, K, d, s, xq, wq)
        nb = mesh.neighbour_cell(K, d, s)
        L = mesh.leaf_covering(*nb) if nb is not None else None
        if L is not None and L[0] < K[0]:
            w = w * 4.0
        return axes, w

    monkeypatch.setattr(octree, "_face_quadrature", wrong)
    A = octree.assemble(t)
    x = t.node_coords()
    b = octree.rhs(t, -_lap_u(x) / (4.0 * math.pi), g=_u)
    v = np.linalg.solve(A, b)
    assert np.abs(v - _u(x)).max() > 1e-4 * np.abs(_u(x)).max()


def test_weights_and_exactness_on_the_refined_mesh():
    p = 3
    t = _refined(p)
    W = t.quad_weights()
    x = t.node_coords()
    vol = np.prod(np.asarray(HI) - np.asarray(LO))
    assert abs(W.sum() - vol) < 1e-13 * vol
    a = 2 * p + 1
    got = np.sum(W * (x[:, 0] + 2.0) ** a * x[:, 1] ** 2 * x[:, 2])
    ref = (((HI[0] + 2.0) ** (a + 1) - (LO[0] + 2.0) ** (a + 1)) / (a + 1) * (HI[1] ** 3 - LO[1] ** 3) / 3
           * (HI[2] ** 2 - LO[2] ** 2) / 2)
    assert abs(got - ref) < 1e-11 * abs(ref)


def test_density_refinement_is_local_and_balanced():
    c = np.array([0.3, -0.4, 0.6])

    def rho(P):
        r2 = np.sum((P - c) ** 2, axis=1)
        return (8.0 / math.pi) ** 1.5 * np.exp(-8.0 * r2)

    t = octree.OctreeMesh(LO, HI, (2, 2, 2), 3)
    octree.refine_to_density(t, rho, delta=1e-5, max_level=3)
    assert t.is_balanced()
    for k in t.leaves:
        if k[0] < 3:
            assert octree.density_indicator(t, k, rho) <= 1e-5
    # the finest leaves sit where the density is
    deepest = max(k[0] for k in t.leaves)
    assert deepest >= 2
    centres = [t.origin(k) + t.h(k) / 2 for k in t.leaves if k[0] == deepest]
    assert min(np.linalg.norm(cc - c) for cc in centres) < 0.5
    far = [k for k in t.leaves if np.linalg.norm(t.origin(k) + t.h(k) / 2 - c) > 2.0]
    assert far and max(k[0] for k in far) <= 1


def test_adaptive_mesh_beats_uniform_for_a_gaussian_charge():
    """The potential of a normalised Gaussian charge is erf(sqrt(a) r)/r. An
    octree refined by the density indicator reaches a smaller nodal error than
    the uniform mesh with fewer nodes (the reason for adapting the auxiliary
    mesh, Sec. 6.2; measured 2752 nodes at 6.5e-2 against 4096 at 8.9e-2)."""
    from scipy.special import erf

    a = 6.0
    c = np.array([1.4, -1.6, 1.5])
    lo, hi = [-3.0] * 3, [3.0] * 3

    def rho(P):
        r2 = np.sum((P - c) ** 2, axis=1)
        return (a / math.pi) ** 1.5 * np.exp(-a * r2)

    def exact(P):
        r = np.linalg.norm(P - c, axis=1)
        return erf(math.sqrt(a) * r) / r

    def err(t):
        x = t.node_coords()
        v = octree.poisson(t, rho(x))
        return np.abs(v - exact(x)).max() / exact(x).max()

    ad = octree.OctreeMesh(lo, hi, (2, 2, 2), 3)
    octree.refine_to_density(ad, rho, delta=3e-3, max_level=2)
    un = octree.OctreeMesh(lo, hi, (4, 4, 4), 3)
    e_ad, e_un = err(ad), err(un)
    assert ad.Nq < un.Nq and e_ad < 0.8 * e_un, (ad.Nq, e_ad, un.Nq, e_un)


def test_unrefined_exchange_build_is_the_uniform_one():
    from paper_2510_21213_gb300 import inputs

    spec = inputs.tiny_system()
    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, (2, 2, 2), 3)
    t = octree.OctreeMesh(spec.mesh.lo, spec.mesh.hi, (2, 2, 2), 3)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    ref = oracle.exchange_build(m, psi, method="dense")
    got = octree.exchange_build(t, psi)
    assert np.abs(got["K"] - ref["K"]).max() <= 1e-10 * np.abs(ref["K"]).max()
    assert abs(got["E_H"] - ref["E_H"]) <= 1e-10 * abs(ref["E_H"])
    assert abs(got["E_X"] - ref["E_X"]) <= 1e-10 * abs(ref["E_X"])


def test_library_octree_equals_the_oracle():
    """The library's host-side octree construction (dg_octree_refine) gives the
    oracle's leaves, in the oracle's element order."""
    from paper_2510_21213_gb300 import dgx

    c = np.array([0.3, -0.4, 0.6])

    def rho(P):
        r2 = np.sum((P - c) ** 2, axis=1)
        return (8.0 / math.pi) ** 1.5 * np.exp(-8.0 * r2)

    for p, delta, ml in ((3, 1e-5, 3), (2, 1e-4, 2)):
        t = octree.OctreeMesh(LO, HI, (2, 2, 2), p)
        octree.refine_to_density(t, rho, delta=delta, max_level=ml)
        got = dgx.dg_octree_refine(LO, HI, (2, 2, 2), p, rho, delta, ml)
        assert [tuple(r) for r in got] == t.leaf_list()
        assert len({k[0] for k in t.leaves}) > 1
    lib = dgx.load()
    n = dgx.C.c_int32()
    desc = dgx.dg_mesh_desc((dgx.C.c_double * 3)(*LO), (dgx.C.c_double * 3)(*HI), (dgx.C.c_int32 * 3)(2, 2, 2), 2)
    fn = dgx.DENSITY_FN(lambda xyz, k, out, u: None)
    assert lib.dg_octree_refine(dgx.C.byref(desc), 0.0, 2, fn, None, 0, None, dgx.C.byref(n)) == dgx.DG_ERR_INVALID_ARG
    assert lib.dg_octree_refine(dgx.C.byref(desc), 1e-3, 21, fn, None, 0, None, dgx.C.byref(n)) == dgx.DG_ERR_INVALID_ARG


def test_library_face_connectivity_is_reciprocal():
    """dg_octree_faces on a mesh with hanging faces: every same-size face is
    seen from both sides, every hanging face from its small side (kind 2, at
    its quarter) appears among the large side's four neighbours (kind 3) at
    that quarter, and boundary faces lie on the box."""
    from paper_2510_21213_gb300 import dgx

    t = _refined(2)
    leaves = np.array(t.leaf_list(), dtype=np.int32)
    kind, nb, pos = dgx.dg_octree_faces(LO, HI, (2, 2, 2), 2, leaves)
    E = len(leaves)
    assert set(np.unique(kind)) == {0, 1, 2, 3}
    for e in range(E):
        lv = leaves[e][0]
        for f in range(6):
            d, side = f // 2, (1 if f % 2 else -1)
            opp = 2 * d + (0 if side > 0 else 1)
            k = kind[e, f]
            if k == 0:
                cell = leaves[e][1 + d] + side
                assert cell < 0 or cell >= t.n[d] * 2 ** lv
            elif k == 1:
                L = nb[e, f, 0]
                assert leaves[L][0] == lv and kind[L, opp] == 1 and nb[L, opp, 0] == e
            elif k == 2:
                L = nb[e, f, 0]
                assert leaves[L][0] == lv - 1 and kind[L, opp] == 3 and nb[L, opp, pos[e, f]] == e
            else:
                for j in range(4):
                    s = nb[e, f, j]
                    assert leaves[s][0] == lv + 1 and kind[s, opp] == 2 and nb[s, opp, 0] == e and pos[s, opp] == j
    with pytest.raises(dgx.DGError):  # an unbalanced set is rejected
        bad = octree.OctreeMesh(LO, HI, (2, 2, 2), 2)
        bad.refine([(0, 0, 0, 0)])
        bad.refine([(1, 1, 1, 1)])  # no balance()
        dgx.dg_octree_faces(LO, HI, (2, 2, 2), 2, np.array(bad.leaf_list(), dtype=np.int32))


def test_library_rejects_overlapping_leaves():
    """A leaf together with one of its own descendants is not a partition of
    the box: dg_octree_faces refuses it (the root cell (0,0,0,0), its eight
    children and the cell (0,1,0,0) would otherwise all get face kinds)."""
    from paper_2510_21213_gb300 import dgx

    leaves = [(0, 0, 0, 0), (0, 1, 0, 0)] + [(1, a, b, c) for c in range(2) for b in range(2) for a in range(2)]
    with pytest.raises(dgx.DGError):
        dgx.dg_octree_faces(LO, HI, (2, 1, 1), 2, np.array(leaves, dtype=np.int32))
    # the same set without the parent is accepted
    dgx.dg_octree_faces(LO, HI, (2, 1, 1), 2, np.array(leaves[1:], dtype=np.int32))


def test_octree_apply_checks_field_shape_before_any_launch():
    """dg_octree_apply takes no lengths, so the binding refuses a field whose
    width is not n_leaves * (p+1)^3 before the library is called (CPU
    tensors: nothing reaches a device)."""
    torch = pytest.importorskip("torch")
    from paper_2510_21213_gb300 import dgx

    t = _refined(2)
    leaves = np.array(t.leaf_list(), dtype=np.int32)
    width = len(leaves) * 27
    for bad in (torch.zeros(width), torch.zeros(2, width - 1), torch.zeros(2, width + 27)):
        with pytest.raises(ValueError):
            dgx.dg_octree_apply(LO, HI, (2, 2, 2), 2, leaves, bad)


def test_octree_setup_rejects_bad_arguments_without_a_device():
    """dg_octree_setup validates the mesh, the leaf set and its settings on the
    host before any device work: each bad argument is DG_ERR_INVALID_ARG and
    no handle is returned."""
    from paper_2510_21213_gb300 import dgx

    lib = dgx.load()
    C = dgx.C
    t = _refined(2)
    leaves = np.array(t.leaf_list(), dtype=np.int32)
    lp = leaves.ctypes.data_as(C.c_void_p)

    def desc(p=2, n=(2, 2, 2)):
        return dgx.dg_mesh_desc((C.c_double * 3)(*LO), (C.c_double * 3)(*HI), (C.c_int32 * 3)(*n), p)

    good = dict(form=0, eps=0.125, rtol=1e-10, it=100, pc=1, prec=0)
    cases = [dict(good, form=2), dict(good, eps=0.0), dict(good, rtol=0.0), dict(good, rtol=1.0),
             dict(good, it=0), dict(good, pc=2), dict(good, pc=-1), dict(good, prec=2), dict(good, prec=-1)]
    for c in cases:
        h = C.c_void_p(1)
        rc = lib.dg_octree_setup(C.byref(desc()), lp, len(leaves), c["form"], c["eps"], c["rtol"], c["it"], c["pc"],
                                 c["prec"], C.byref(h))
        assert rc == dgx.DG_ERR_INVALID_ARG and not h.value
    h = C.c_void_p(1)
    assert lib.dg_octree_setup(C.byref(desc(p=9)), lp, len(leaves), 0, 0.125, 1e-10, 100, 1, 0,
                               C.byref(h)) == dgx.DG_ERR_INVALID_ARG and not h.value
    # a leaf set that is not 2:1 balanced
    bad = octree.OctreeMesh(LO, HI, (2, 2, 2), 2)
    bad.refine([(0, 0, 0, 0)])
    bad.refine([(1, 1, 1, 1)])
    bl = np.array(bad.leaf_list(), dtype=np.int32)
    assert lib.dg_octree_setup(C.byref(desc()), bl.ctypes.data_as(C.c_void_p), len(bl), 0, 0.125, 1e-10, 100, 1, 0,
                               C.byref(h)) == dgx.DG_ERR_INVALID_ARG and not h.value
    assert lib.dg_octree_setup(C.byref(desc()), lp, len(leaves), 0, 0.125, 1e-10, 100, 1, 0, None) == \
        dgx.DG_ERR_INVALID_ARG
    lib.dg_octree_destroy(None)
