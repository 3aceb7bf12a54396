// The bounded wait of the library's tensor-core kernels, exposed so that its
// timeout path can be exercised on a GPU without a fault or a hang: a one-
// warp kernel initialises an mbarrier, arrives on it or not, and waits with
// the same bounded helper (tc::mbar_wait) that the patch-solve pipeline uses
// for every hand-off. Without the arrival the wait gives up after `limit`
// clock cycles and the kernel reports DG_ERR_TIMEOUT through device memory;
// the context stays usable.
#include "dg_ctx.h"
#include "dg_tc.h"

namespace dg {

__global__ void k_wait_probe(int arrive, long long limit, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_addr(&bar), 1);
    tc::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0 && arrive) tc::mbar_arrive(tc::smem_addr(&bar));
  __syncthreads();
  const bool ok = tc::mbar_wait(tc::smem_addr(&bar), 0, limit);
  if (threadIdx.x == 0) *status = ok ? DG_OK : DG_ERR_TIMEOUT;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_wait_probe(int32_t arrive, int64_t limit_cycles, void* stream) {
  if (limit_cycles < 1 || limit_cycles > (1LL << 34)) return DG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  {
    DeviceWideGuard guard;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return DG_ERR_NO_MEMORY;
  }
  int status = DG_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(d, 0xff, sizeof(int), s);
  if (e == cudaSuccess) {
    count_launch();
    k_wait_probe<<<1, 32, 0, s>>>(arrive ? 1 : 0, (long long)limit_cycles, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  {
    DeviceWideGuard guard;
    cudaFree(d);
  }
  return e == cudaSuccess ? status : DG_ERR_CUDA;
}
