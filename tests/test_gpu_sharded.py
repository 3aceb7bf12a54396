"""One system's exchange build split into source ranges (the per-GPU share of
a sharded build): the partial K of the ranges add up to the whole build's K,
E_H comes from the range holding the Hartree source, on the chain workload in
FP64 and mixed precision."""

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


@pytest.mark.parametrize("precision", [0, 1])
def test_ranges_add_up_to_the_whole_build(dgx, precision):
    from paper_2510_21213_gb300 import dist as pd

    spec = inputs.chain_system(n=4, p=5, n_orb=6)
    m = spec.mesh
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=precision, rtol=1e-10)
    xyz, w = s.node_coords()
    psi = torch.tensor(inputs.orbitals(spec, xyz, w), device="cuda")
    N = psi.shape[0]
    K, eh, ex, st = s.exchange_build(psi)
    total = N * (N + 1) // 2 + 1
    Ksum = np.zeros_like(K)
    ehs = []
    for r in range(3):  # three ranks' shares, one after the other on one GPU
        b, e = pd.shard_range(total, 3, r)
        Kp, ehp, stp = dgx.dg_exchange_build_range(s.h, psi, b, e)
        assert len(stp) == e - b and all(x["status"] == 0 for x in stp)
        Ksum += Kp
        ehs.append(ehp)
    assert np.abs(Ksum - K).max() <= 1e-12 * np.abs(K).max()
    assert ehs[0] == pytest.approx(eh, rel=1e-13) and ehs[1] == 0.0 and ehs[2] == 0.0
    # the rank bookkeeping with one rank (no process group) and the library as the share
    K1, eh1, ex1 = pd.sharded_exchange(lambda b, e: dgx.dg_exchange_build_range(s.h, psi, b, e)[:2], N, 1, 0)
    assert np.abs(K1 - K).max() <= 1e-12 * np.abs(K).max() and ex1 == pytest.approx(ex, rel=1e-12)
    # empty and invalid ranges
    K0, eh0, _ = dgx.dg_exchange_build_range(s.h, psi, 3, 3)
    assert not K0.any() and eh0 == 0.0
    with pytest.raises(dgx.DGError):
        dgx.dg_exchange_build_range(s.h, psi, 0, total + 1)
    s.close()


def test_ace_operator_vs_oracle(dgx):
    """dg_ace_apply after a whole build equals the oracle's compressed exchange
    operator of the oracle's build (FP64, 1e-9), maps psi_i to -W_i, and is
    refused without a whole build."""
    import oracle

    spec = inputs.chain_system(n=2, p=4, n_orb=3)
    m = spec.mesh
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, rtol=1e-12)
    xyz, w = s.node_coords()
    psi_h = inputs.orbitals(spec, xyz, w)
    psi = torch.tensor(psi_h, device="cuda")
    U = torch.tensor(np.random.default_rng(8).standard_normal((5, s.Nq)), device="cuda")
    with pytest.raises(dgx.DGError):  # no build yet
        dgx.dg_ace_apply(s.h, U)
    s.exchange_build(psi)
    om = oracle.Mesh(m.lo, m.hi, m.n, m.p)
    ref = oracle.exchange_build(om, psi_h, method="fdm")
    Wq = oracle.quad_weights(om)
    got = dgx.dg_ace_apply(s.h, U).cpu().numpy()
    want = oracle.ace_apply(ref, Wq, U.cpu().numpy())
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    # exact on the occupied orbitals up to the discretisation-level asymmetry of K
    asym = np.abs(ref["K"] - ref["K"].T).max() / np.abs(ref["K"]).max()
    gp = dgx.dg_ace_apply(s.h, psi).cpu().numpy()
    assert np.abs(gp + ref["W"]).max() <= (1e-9 + 10 * asym) * np.abs(ref["W"]).max()
    dgx.dg_exchange_build_range(s.h, psi, 0, 2)  # a partial build clears the operator
    with pytest.raises(dgx.DGError):
        dgx.dg_ace_apply(s.h, U)
    s.close()
