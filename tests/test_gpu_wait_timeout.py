"""The bounded wait of the tensor-core kernels runs out without a fault.

Every hand-off of the library's tensor-core pipeline is an mbarrier wait
with a clock-cycle limit; when it runs out the kernel reports
DG_ERR_TIMEOUT through device memory and returns. dg_wait_probe runs that
same wait in a one-warp kernel on a barrier that nothing arrives on (a few
milliseconds of limit): the call returns DG_ERR_TIMEOUT, and the CUDA
context stays usable (a solve afterwards succeeds). With the arrival the
wait completes and the call returns DG_OK."""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    lib = dgx.load()
    lib.dg_wait_probe.argtypes = [C.c_int32, C.c_int64, C.c_void_p]
    lib.dg_wait_probe.restype = C.c_int
    return dgx


def test_wait_completes_or_times_out_without_fault(dgx):
    lib = dgx.load()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.dg_wait_probe(1, 1 << 24, s) == dgx.DG_OK
    assert lib.dg_wait_probe(0, 1 << 23, s) == dgx.DG_ERR_TIMEOUT  # about 4 ms at 2 GHz
    assert lib.dg_wait_probe(0, 0, s) == dgx.DG_ERR_INVALID_ARG
    # the context is still usable: a small solve converges
    from oracle import Mesh, node_coords
    m = Mesh([-4.0] * 3, [4.0] * 3, 2, 3)
    x = node_coords(m)
    f = np.exp(-np.sum(x * x, axis=1))[None, :]
    sol = dgx.PoissonSolver(m.lo, m.hi, m.n, m.p, rtol=1e-10)
    _, st = sol.solve(torch.tensor(f, device="cuda"))
    assert st[0]["status"] == 0
    sol.close()
