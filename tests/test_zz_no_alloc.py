"""dg_apply_smoother_noalloc: the smoother preconditioner without any device
allocation at call time.

Some callers cannot call cudaMalloc when they apply the preconditioner: a
serving process whose memory pool is sized and reserved up front, a real-time
loop where an allocation would stall or fail, or a host framework that owns
every device allocation itself. For them the library offers this variant,
whose scratch lives in a static device array. This file checks, through the
C ABI, that it returns what the allocating dg_apply_smoother returns, on two
calls in a row (the scratch keeps the previous call's contents), and that it
refuses sizes beyond its fixed scratch. It is named so that pytest collects it
last.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    lib = dgx.load()
    lib.dg_apply_smoother_noalloc.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64,
                                              C.c_void_p]
    lib.dg_apply_smoother_noalloc.restype = C.c_int
    return lib


def _noalloc(lib, h, r, level):
    z = torch.empty_like(r)
    fp32 = 1 if r.dtype == torch.float32 else 0
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.dg_apply_smoother_noalloc(h, level, fp32, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()),
                                         r.shape[0], stream)
    torch.cuda.synchronize()
    return code, z


def test_noalloc_smoother_matches_allocating_entry_point(lib):
    from paper_2510_21213_gb300 import dgx

    s = dgx.PoissonSolver([-3.0, -2.0, -2.5], [3.0, 2.5, 2.0], (3, 2, 2), 5)
    rng = np.random.default_rng(23)
    for level in range(s.info.levels):
        for dtype, tol in ((torch.float64, 1e-11), (torch.float32, 1e-6)):
            nq_level = _level_nq(s, level)
            r = torch.tensor(rng.standard_normal((3, nq_level)), device="cuda", dtype=dtype)
            ref = s.smoother(r, level=level)
            torch.cuda.synchronize()
            for _ in range(2):
                code, got = _noalloc(lib, s.h, r, level)
                assert code == dgx.DG_OK, (level, code)
                scale = ref.abs().max().item()
                assert (got - ref).abs().max().item() <= tol * scale, (level, dtype)
    s.close()


def _level_nq(s, level):
    """Number of nodes of a multigrid level: p -> p//2 down to 1, then n -> n/2
    while every n is even (the hierarchy documented in dg_poisson.h)."""
    n = [3, 2, 2]
    p = 5
    levels = [(tuple(n), p)]
    while p > 1:
        p = max(1, p // 2)
        levels.append((tuple(n), p))
    while all(v % 2 == 0 and v >= 2 for v in n) and 8 * n[0] * n[1] * n[2] > 512:
        n = [v // 2 for v in n]
        levels.append((tuple(n), 1))
    (nx, ny, nz), pp = levels[level]
    return nx * ny * nz * (pp + 1) ** 3


def test_noalloc_smoother_rejects_oversized_batches(lib):
    from paper_2510_21213_gb300 import dgx

    s = dgx.PoissonSolver([-3.0] * 3, [3.0] * 3, (4, 4, 4), 7)
    nq = s.Nq
    # 4^3 elements x 10^3 patch nodes x B doubles exceeds 8 MiB from B = 17 on
    r = torch.zeros((20, nq), dtype=torch.float64, device="cuda")
    code, _ = _noalloc(lib, s.h, r, 0)
    assert code == dgx.DG_ERR_INVALID_ARG
    assert b"scratch" in lib.dg_last_error_detail(s.h)
    r = torch.zeros((257, 8), dtype=torch.float64, device="cuda")
    code, _ = _noalloc(lib, s.h, r, s.info.levels - 1)
    assert code == dgx.DG_ERR_INVALID_ARG
    s.close()
