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
                                         ("one", 6, 0), ("flat", 3, 0)])
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
