"""What the trained network gains: on held-out systems (seeds never used in
training) at the configuration the network was trained for (16^3 elements,
p = 7, 64 orbitals, 32 atoms), pair solves of the learned form against the
mixed form without the network, both to the same FP64 true residual 1e-8.

The solutions must agree (the network only moves the starting point); the
learned form must need fewer PCG iterations on average."""

import numpy as np
import pytest

from paper_2510_21213_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HELD_OUT = (900, 901)
PAIRS_PER_SYSTEM = 24


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    dgx.load()
    if dgx.default_nn_weights(7) is None:
        pytest.skip("no trained weights for p = 7")
    return dgx


def test_learned_guess_cuts_iterations_on_held_out_systems(dgx):
    lo, hi, n, p = [-12.0] * 3, [12.0] * 3, (16, 16, 16), 7
    kw = dict(bc_route=dgx.DG_BC_GAUSSSUM, rtol=1e-8)
    mixed = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED, **kw)
    learned = dgx.PoissonSolver(lo, hi, n, p, precision=dgx.DG_PREC_MIXED_LEARNED,
                                nn_weights_path=dgx.default_nn_weights(7), **kw)
    xyz, w = mixed.node_coords()
    xyz_d = torch.tensor(xyz, device="cuda")
    w_d = torch.tensor(w, device="cuda")
    rng = np.random.default_rng(7)
    it_m, it_l, fb = [], [], 0
    for seed in HELD_OUT:
        spec = inputs.random_system(seed=seed, n=16, p=7, n_orb=64, n_atoms=32)
        psi = inputs.orbitals_torch(spec, xyz_d, w_d)
        pairs = [tuple(sorted(rng.integers(0, 64, size=2))) for _ in range(PAIRS_PER_SYSTEM)]
        f = torch.stack([psi[i] * psi[j] for i, j in pairs]).contiguous()
        vm, sm = mixed.solve(f)
        vl, sl = learned.solve(f)
        assert all(s["status"] == 0 and s["rel_residual"] <= 1e-8 for s in sm + sl)
        # same solution within the mixed form's stated bound at rtol 1e-8
        err = ((vl - vm).abs().amax(dim=1) / vm.abs().amax(dim=1)).max().item()
        assert err < 2e-5
        it_m += [s["iters"] for s in sm]
        it_l += [s["iters"] for s in sl]
        fb += sum(s["used_fallback"] for s in sl)
    print(f"held-out pairs {len(it_m)}: mean PCG iterations mixed {np.mean(it_m):.2f}, learned {np.mean(it_l):.2f}, "
          f"fallbacks {fb}")
    assert np.mean(it_l) < np.mean(it_m)
    mixed.close()
    learned.close()
