"""Oracle parity of the benchmarked workloads, through the C ABI.

chain10 (8^3 elements, p = 6, 10 orbitals: the Hartree solve and 55 pair
solves): the whole exchange build (K, E_H, E_X and every source's
self-energy (f|f) = sum_q W_q f v, i.e. (rho|rho) and the pair self-energies
(ij|ij)) against the oracle's build, which solves each discrete problem
exactly (fast diagonalisation) with Dirichlet data from its Gaussian-sum route
at 1e-12 (pinned against the direct quadrature in test_oracle_pins.py).

mixed64 (16^3 elements, p = 7, 64 orbitals, 2.1 M nodes): the first 64
sources of the build (the Hartree density and 63 pairs) through
dg_exchange_build_range against the oracle's exchange_partial over the same
range: the range's contribution to K, E_H and the self-energies.

Tolerances: FP64 form solved to a 1e-12 true residual, 1e-10 relative (K by
its largest entry, self-energies by the largest one). Mixed and learned forms
at the metric's 1e-8 residual: the stated bound of the mixed modes on the
potentials, 2e-5 relative, carried to K, E_H, E_X and the self-energies (the
FP32 inner solve leaves smooth error that a 1e-8 residual does not see: E_H
of the 16^3 p = 7 system measured 5e-6; the learned form only changes the
initial guess)."""

import numpy as np
import pytest

import oracle
from paper_2510_21213_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_BOUND = 2e-5


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    dgx.load()
    return dgx


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.fixture(scope="module")
def chain10():
    spec = inputs.chain_system(seed=2)
    mm = spec.mesh
    m = oracle.Mesh(mm.lo, mm.hi, mm.n, mm.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    ref = oracle.exchange_build(m, psi, method="fdm", g_route="gausssum")
    return spec, psi, ref


def _check_build(K, eh, ex, st, ref, tol):
    errs = {"K": _rel(K, ref["K"]), "E_H": abs(eh - ref["E_H"]) / abs(ref["E_H"]),
            "E_X": abs(ex - ref["E_X"]) / abs(ref["E_X"]),
            "self": _rel([x["self_energy"] for x in st], ref["self"])}
    print("errors vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(v <= tol for v in errs.values()), errs
    return errs


def test_chain10_build_fp64_vs_oracle(dgx, chain10):
    spec, psi, ref = chain10
    mm = spec.mesh
    s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-12, max_iter=400)
    K, eh, ex, st = s.exchange_build(torch.tensor(psi, device="cuda"))
    assert all(x["status"] == 0 and x["rel_residual"] <= 1e-12 for x in st)
    _check_build(K, eh, ex, st, ref, 1e-10)
    s.close()


@pytest.mark.parametrize("form", ["mixed", "learned"])
def test_chain10_build_reduced_precision_vs_oracle(dgx, chain10, form):
    spec, psi, ref = chain10
    mm = spec.mesh
    if form == "learned":
        w = dgx.default_nn_weights(mm.p)
        if w is None:
            pytest.skip("no trained weights for this degree")
        s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-8, precision=dgx.DG_PREC_MIXED_LEARNED,
                              nn_weights_path=w)
    else:
        s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-8, precision=dgx.DG_PREC_MIXED)
    K, eh, ex, st = s.exchange_build(torch.tensor(psi, device="cuda"))
    assert all(x["status"] == 0 and x["rel_residual"] <= 1e-8 for x in st)
    _check_build(K, eh, ex, st, ref, MIXED_BOUND)
    s.close()


@pytest.fixture(scope="module")
def mixed64():
    spec = inputs.random_system(seed=3)
    mm = spec.mesh
    m = oracle.Mesh(mm.lo, mm.hi, mm.n, mm.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    K, eh, se = oracle.exchange_partial(m, psi, 0, 64, method="fdm", g_route="gausssum", with_self=True)
    return spec, psi, {"K": K, "E_H": eh, "self": se}


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_mixed64_range_vs_oracle(dgx, mixed64, form):
    spec, psi, ref = mixed64
    mm = spec.mesh
    if form == "fp64":
        s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-12, max_iter=400)
        tol, rtol = 1e-10, 1e-12
    else:
        s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, rtol=1e-8, precision=dgx.DG_PREC_MIXED)
        tol, rtol = MIXED_BOUND, 1e-8
    K, eh, st = s.exchange_build_range(torch.tensor(psi, device="cuda"), 0, 64)
    assert len(st) == 64 and all(x["status"] == 0 and x["rel_residual"] <= rtol for x in st)
    errs = {"K": _rel(K, ref["K"]), "E_H": abs(eh - ref["E_H"]) / abs(ref["E_H"]),
            "self": _rel([x["self_energy"] for x in st], ref["self"])}
    print(form, "errors vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(v <= tol for v in errs.values()), errs
    s.close()
