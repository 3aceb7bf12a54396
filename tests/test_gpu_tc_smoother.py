"""The tensor-core patch solve of the Schwarz smoother (FP32 inner solve of
the mixed modes, degrees 6-8) against the oracle's patch inverses.

The smoother output is sum over element patches of R_P^T A_PP^-1 R_P r
(additive Schwarz, one node layer of overlap). The reference assembles A with
the oracle (Kronecker form) and solves every patch densely. The tensor-core
kernel applies the x-y Kronecker factors of the patches' fast diagonalisation
as TF32 MMAs (10-bit mantissas: inputs rounded to a relative 2^-11, or cut to
2^-10 where the hardware takes FP32 operands as they are) with FP32
accumulation; the z factor and the eigenvalue scaling run in FP32. Its
stated bound is 2e-3 of the output's largest entry (the transform errors of a
few 1e-4 are amplified by the spread of the patch eigenvalues); the SIMT FP32
kernel of the same handle with tc_smoother = 0 stays at 1e-4."""

import numpy as np
import pytest

import oracle
from paper_2510_21213_gb300 import inputs  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_BOUND = 2e-3


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    dgx.load()
    return dgx


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


@pytest.mark.parametrize("lo,hi,n,p,B", [
    ([-3.0] * 3, [3.0] * 3, (4, 4, 4), 7, 3),
    ([-2.0, -1.0, 0.5], [2.0, 1.5, 2.0], (3, 2, 5), 6, 2),
    ([-1.0] * 3, [1.0] * 3, (1, 2, 1), 8, 5),
    ([-4.0, -3.0, -2.5], [4.0, 3.5, 2.0], (5, 4, 3), 7, 23),
    ([-6.0] * 3, [6.0] * 3, (6, 5, 4), 6, 4),
])
def test_tc_patch_solve_vs_oracle(dgx, lo, hi, n, p, B):
    s_tc = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED, tc_smoother=2)
    s_simt = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED, tc_smoother=0)
    m = oracle.Mesh(lo, hi, n, p)
    A = oracle.assemble_kron(m)
    rng = np.random.default_rng(p + B)
    r = rng.standard_normal((B, m.Nq))
    ref = _patch_reference(A, m, r)
    r32 = torch.tensor(r, device="cuda", dtype=torch.float32)
    got = s_tc.smoother(r32, level=0).cpu().double().numpy()
    again = s_tc.smoother(r32, level=0).cpu().double().numpy()
    simt = s_simt.smoother(r32, level=0).cpu().double().numpy()
    scale = np.abs(ref).max()
    err_tc = np.abs(got - ref).max() / scale
    err_simt = np.abs(simt - ref).max() / scale
    print(f"n={n} p={p} B={B}: tensor-core {err_tc:.2e}, SIMT {err_simt:.2e}")
    assert err_simt <= 1e-4
    assert err_tc <= TC_BOUND
    # the tensor-core path ran (TF32 differs from FP32) and is deterministic
    assert np.abs(got - simt).max() > 0
    assert np.array_equal(got, again)
    s_tc.close()
    s_simt.close()


def test_tc_smoother_keeps_iterations_and_result(dgx):
    """A mixed-mode solve with the tensor-core smoother reaches the same FP64
    residual in the same number of PCG iterations (within one) as with the
    SIMT smoother, and the two solutions agree within the mixed bound."""
    from paper_2510_21213_gb300 import inputs as I

    spec = I.chain_system(seed=2)
    mm = spec.mesh
    xyz = oracle.node_coords(oracle.Mesh(mm.lo, mm.hi, mm.n, mm.p))
    w = oracle.quad_weights(oracle.Mesh(mm.lo, mm.hi, mm.n, mm.p))
    psi = I.orbitals(spec, xyz, w)
    f = torch.tensor(np.stack([psi[0] * psi[1], psi[3] * psi[3], psi[2] * psi[7]]), device="cuda")
    out = {}
    for tc in (0, 2):
        s = dgx.PoissonSolver(mm.lo, mm.hi, mm.n, mm.p, precision=dgx.DG_PREC_MIXED, rtol=1e-8, tc_smoother=tc)
        v, st = s.solve(f)
        assert all(x["status"] == 0 and x["rel_residual"] <= 1e-8 for x in st)
        out[tc] = (v.cpu().numpy(), [x["iters"] for x in st])
        s.close()
    print("iterations SIMT / tensor-core smoother:", out[0][1], out[2][1])
    assert all(abs(a - b) <= 1 for a, b in zip(out[0][1], out[2][1]))
    v0, v1 = out[0][0], out[2][0]
    assert np.abs(v1 - v0).max() <= 2e-5 * np.abs(v0).max()


def test_patch_solves_alone(dgx):
    """dg_apply_patch_solves returns every patch's solution before the gather:
    the tensor-core kernel's buffer (degree 7, default on) against the FP64
    SIMT kernel's within the TF32 bound, the FP32 SIMT kernel's within 1e-4;
    entries outside the domain are exactly zero; the gather of the buffer is
    what the smoother returns (checked through the smoother's own result on
    an FP64 handle: sum over patches covering each node)."""
    lo, hi, n, p = [-3.0] * 3, [3.0] * 3, (3, 2, 2), 7
    m = oracle.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((3, m.Nq))
    s64 = dgx.PoissonSolver(lo, hi, n, p)
    s_tc = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED)
    s_simt = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED, tc_smoother=0)
    ref = s64.patch_solves(torch.tensor(r, device="cuda")).cpu().numpy()
    r32 = torch.tensor(r, device="cuda", dtype=torch.float32)
    tc = s_tc.patch_solves(r32).cpu().double().numpy()
    simt = s_simt.patch_solves(r32).cpu().double().numpy()
    scale = np.abs(ref).max()
    assert ref.shape == (3, m.E, (p + 3) ** 3)
    err_tc = np.abs(tc - ref).max() / scale
    err_simt = np.abs(simt - ref).max() / scale
    print(f"patch buffers: tensor-core {err_tc:.2e}, SIMT FP32 {err_simt:.2e}")
    assert err_tc <= TC_BOUND and err_simt <= 1e-4 and not np.array_equal(tc, simt)
    # patches of boundary elements have no nodes beyond the box: those slots are zero
    outside = ref == 0.0
    assert outside.any() and np.all(tc[outside] == 0.0)
    # the gather of the FP64 patch buffer is the FP64 smoother's result
    mp = p + 3
    z = s64.smoother(torch.tensor(r, device="cuda")).cpu().numpy()
    from oracle import dg_oracle as O
    X, Y, Z = O.global_indices(m)
    lex = X + m.L[0] * (Y + m.L[1] * Z)
    acc = np.zeros((3, m.L[0] * m.L[1] * m.L[2]))
    for e in range(m.E):
        ec = (e % m.n[0], (e // m.n[0]) % m.n[1], e // (m.n[0] * m.n[1]))
        lo_n = [ec[d] * m.n1 - (1 if ec[d] > 0 else 0) for d in range(3)]
        hi_n = [min(m.L[d], (ec[d] + 1) * m.n1 + 1) for d in range(3)]
        for kz in range(hi_n[2] - lo_n[2]):
            for jy in range(hi_n[1] - lo_n[1]):
                for ix in range(hi_n[0] - lo_n[0]):
                    g = (lo_n[0] + ix) + m.L[0] * ((lo_n[1] + jy) + m.L[1] * (lo_n[2] + kz))
                    acc[:, g] += ref[:, e, ix + mp * (jy + mp * kz)]
    assert np.abs(acc[:, lex] - z).max() <= 1e-12 * np.abs(z).max()
    for s in (s64, s_tc, s_simt):
        s.close()
