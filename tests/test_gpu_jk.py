"""The Hartree and exchange actions on trial functions (dg_jk_apply) against
the oracle's exact solves, against the exchange build on the occupied
orbitals, and their argument handling."""

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


def _system(n=2, p=4, n_orb=3):
    spec = inputs.chain_system(n=n, p=p, n_orb=n_orb)
    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    return spec, m, psi


@pytest.mark.parametrize("precision", [0, 1])
def test_jk_action_vs_oracle(dgx, precision):
    spec, m, psi = _system()
    rng = np.random.default_rng(21)
    U = np.concatenate([rng.standard_normal((2, m.Nq)), psi[1:2]])
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=precision, rtol=1e-10)
    JU, XU, st = s.jk_apply(torch.tensor(psi, device="cuda"), torch.tensor(U, device="cuda"))
    assert len(st) == 1 + psi.shape[0] * U.shape[0] and all(x["status"] == 0 for x in st)
    Jr, Xr = oracle.jk_apply(m, psi, U)
    # FP64 solves at rtol 1e-10 / the mixed form's bound at 1e-10
    tol = 1e-8 if precision == 0 else 2e-6
    JU, XU = JU.cpu().numpy(), XU.cpu().numpy()
    for k in range(U.shape[0]):
        assert np.abs(JU[k] - Jr[k]).max() <= tol * np.abs(Jr[k]).max(), k
        assert np.abs(XU[k] - Xr[k]).max() <= tol * np.abs(Xr[k]).max(), k
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_exchange_action_on_orbitals_is_minus_K(dgx, precision):
    """With U = psi the solves are the build's pair solves: <psi_i, X psi_j> =
    -K_ij of dg_exchange_build on the same handle, and sum_i <psi_i, J psi_i> =
    2 E_H."""
    spec, m, psi = _system(n=4, p=5, n_orb=4)
    wq = oracle.quad_weights(m)
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=precision, rtol=1e-10)
    pd = torch.tensor(psi, device="cuda")
    K, eh, ex, _ = s.exchange_build(pd)
    JU, XU, _ = s.jk_apply(pd, pd)
    Kx = -(psi * wq) @ XU.cpu().numpy().T
    # the same sources solved in other batches: equal within the form's bound at 1e-10
    tol = 1e-9 if precision == 0 else 1e-6
    assert np.abs(Kx - K).max() <= tol * np.abs(K).max()
    assert abs(float(np.sum(wq * psi * JU.cpu().numpy())) - 2.0 * eh) <= tol * abs(eh)
    s.close()


def test_one_orbital_has_no_self_interaction(dgx):
    """N = 1, u = psi: the pair source psi psi is the density, so the two
    solves are the same and J psi + X psi = 0 exactly."""
    spec, m, psi = _system(n_orb=1)
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=1, rtol=1e-8)
    pd = torch.tensor(psi[:1], device="cuda")
    JU, XU, st = s.jk_apply(pd, pd)
    assert len(st) == 2
    assert torch.equal(JU + XU, torch.zeros_like(JU))
    assert JU.abs().max().item() > 0
    s.close()


def test_single_operator_and_arguments(dgx):
    spec, m, psi = _system()
    s = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, precision=1, rtol=1e-8)
    pd = torch.tensor(psi, device="cuda")
    U = pd[:2].clone()
    J1, X1, st = s.jk_apply(pd, U)
    J2, X2, st2 = s.jk_apply(pd, U, exchange=False)
    assert X2 is None and len(st2) == 1 and torch.equal(J1, J2)
    J3, X3, st3 = s.jk_apply(pd, U, hartree=False)
    assert J3 is None and len(st3) == psi.shape[0] * 2 and torch.equal(X1, X3)
    lib = dgx.load()
    with pytest.raises(dgx.DGError):
        s.jk_apply(pd, U, hartree=False, exchange=False)
    assert lib.dg_jk_apply(s.h, None, 3, dgx._dev_ptr(U), 2, dgx._dev_ptr(U), None, None, None) == dgx.DG_ERR_INVALID_ARG
    assert lib.dg_jk_apply(s.h, dgx._dev_ptr(pd), 0, dgx._dev_ptr(U), 2, dgx._dev_ptr(U), None, None, None) \
        == dgx.DG_ERR_INVALID_ARG
    assert lib.dg_jk_apply(s.h, dgx._dev_ptr(pd), 3, dgx._dev_ptr(U), 0, dgx._dev_ptr(U), None, None, None) \
        == dgx.DG_ERR_INVALID_ARG
    s.close()
