"""Parity at the full size of the 16^3-element, degree-7, 64-orbital workload
(2.1 M nodes) on sampled sources: the Hartree density and two pair densities
solved on the GPU (FP64 and mixed) against the oracle's exact fast-
diagonalisation solve with its own Gaussian-sum Dirichlet data (that route is
pinned against the direct quadrature in test_oracle_pins.py). The full
exchange build at this size is checked by properties (converged residuals,
E_X = -1/2 tr K, symmetry and PSD of K at discretisation level)."""

import numpy as np
import pytest

import oracle
from paper_2510_21213_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    spec = inputs.random_system(seed=3)
    mm = spec.mesh
    m = oracle.Mesh(mm.lo, mm.hi, mm.n, mm.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    f = np.stack([np.sum(psi * psi, axis=0), psi[0] * psi[1], psi[5] * psi[17]])
    g = oracle.boundary_data_gausssum(m, f, tol=1e-12)
    b = np.stack([oracle.rhs(m, f[k], [gg[k] for gg in g]) for k in range(f.shape[0])])
    ref = oracle.solve_fdm(m, b)
    return dgx, spec, m, psi, f, ref


def test_fullsize_sampled_sources_fp64(setup):
    dgx, spec, m, psi, f, ref = setup
    mm = spec.mesh
    s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-12)
    v, st = s.solve(torch.tensor(f, device="cuda"))
    v = v.cpu().numpy()
    for k in range(f.shape[0]):
        assert st[k]["status"] == 0 and st[k]["rel_residual"] <= 1e-12
        err = np.abs(v[k] - ref[k]).max() / np.abs(ref[k]).max()
        print(f"FP64 source {k}: max |v - v_oracle| / max |v_oracle| = {err:.2e}")
        assert err < 1e-10, (k, err)
    s.close()


def test_fullsize_sampled_sources_mixed(setup):
    """Mixed mode at the metric's 1e-8 FP64 residual keeps smooth-mode error
    that a residual stop does not see (stated bound 2e-5, measured ~5e-6 for
    the Hartree density). At a 1e-10 residual the floor is the FP32 boundary
    data: their contractions run on the tensor cores as 3xTF32 (about 22-bit
    products), measured 1.4e-7 for the Hartree density (3e-8 with FP32 SIMT
    contractions); stated bound 3e-7."""
    dgx, spec, m, psi, f, ref = setup
    mm = spec.mesh
    for rtol, bound in ((1e-8, 2e-5), (1e-10, 3e-7)):
        s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=rtol, precision=dgx.DG_PREC_MIXED)
        v, st = s.solve(torch.tensor(f, device="cuda"))
        v = v.cpu().numpy()
        for k in range(f.shape[0]):
            assert st[k]["status"] == 0 and st[k]["rel_residual"] <= rtol
            err = np.abs(v[k] - ref[k]).max() / np.abs(ref[k]).max()
            assert err < bound, (rtol, k, err)
        s.close()


def test_fullsize_exchange_build_properties(setup):
    dgx, spec, m, psi, f, ref = setup
    mm = spec.mesh
    s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-8, precision=dgx.DG_PREC_MIXED)
    K, eh, ex, st = s.exchange_build(torch.tensor(psi, device="cuda"))
    assert len(st) == 64 * 65 // 2 + 1
    assert all(x["status"] == 0 and x["rel_residual"] <= 1e-8 for x in st)
    assert abs(ex + 0.5 * np.trace(K)) <= 1e-12 * abs(ex)
    nrm = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-2 * nrm
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() >= -1e-8 * nrm
    # E_H from the oracle's Hartree potential agrees with the build's within
    # the mixed-mode bound at a 1e-8 residual (measured ~5e-6)
    eh_ref = 0.5 * float(np.sum(oracle.quad_weights(m) * f[0] * ref[0]))
    assert abs(eh - eh_ref) <= 2e-5 * abs(eh_ref)
    s.close()
