"""The octree SIPDG operator on the GPU (dg_octree_apply) against the
oracle's dense matrix on meshes with hanging faces."""

import numpy as np
import pytest

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


def _three_levels(p):
    t = octree.OctreeMesh(LO, HI, (2, 2, 2), p)
    t.refine([(0, 0, 0, 0)])
    t.refine([(1, 1, 1, 1)])
    t.balance()
    return t


def _one_split(p):
    t = octree.OctreeMesh(LO, HI, (2, 1, 1), p)
    t.refine([(0, 1, 0, 0)])
    return t


@pytest.mark.parametrize("mesh,p,form", [("three", 1, 0), ("three", 2, 0), ("three", 3, 1), ("one", 5, 0),
                                         ("one", 6, 0), ("flat", 3, 0), ("one", 7, 0), ("one", 8, 1)])
def test_octree_operator_vs_oracle(dgx, mesh, p, form):
    if mesh == "three":
        t = _three_levels(p)
        n = (2, 2, 2)
    elif mesh == "one":
        t = _one_split(p)
        n = (2, 1, 1)
    else:
        t = octree.OctreeMesh(LO, HI, (2, 3, 2), p)
        n = (2, 3, 2)
    leaves = np.array(t.leaf_list(), dtype=np.int32)
    A = octree.assemble(t, penalty_form=form)
    rng = np.random.default_rng(p)
    u = rng.standard_normal((3, t.Nq))
    got = dgx.dg_octree_apply(LO, HI, n, p, leaves, torch.tensor(u, device="cuda"), penalty_form=form).cpu().numpy()
    ref = (A @ u.T).T
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_octree_apply_refuses_aliased_fields(dgx):
    """out is written while other blocks still read u: an in-place call is
    refused (DG_ERR_INVALID_ARG) instead of racing."""
    t = _one_split(2)
    leaves = np.array(t.leaf_list(), dtype=np.int32)
    u = torch.zeros((2, t.Nq), dtype=torch.float64, device="cuda")
    lib = dgx.load()
    desc = dgx.dg_mesh_desc((dgx.C.c_double * 3)(*LO), (dgx.C.c_double * 3)(*HI), (dgx.C.c_int32 * 3)(2, 1, 1), 2)
    ptr = dgx.C.c_void_p(u.data_ptr())
    rc = lib.dg_octree_apply(dgx.C.byref(desc), leaves.ctypes.data_as(dgx.C.c_void_p), leaves.shape[0], 0, 0.125,
                             ptr, ptr, 2, None)
    assert rc == dgx.DG_ERR_INVALID_ARG
