// Allocation-free variant of the smoother entry point (dg_apply_smoother_noalloc).
//
// Some callers cannot allocate device memory when they apply the
// preconditioner (a serving process with a memory pool sized up front, a
// real-time loop, a host framework that owns every allocation). This file
// keeps the scratch that entry point needs in file-scope device arrays, looks
// their device addresses up once per device and hands those to the kernels.
#include <cstring>
#include <mutex>
#include <string>

#include "dg_ctx.h"

namespace dg {

// Scratch of dg_apply_smoother_noalloc: a file-scope device array (every GPU
// that loads the library holds it until the process exits), so that entry
// point never allocates. Host code must not pass these names to kernels: their
// device addresses come from cudaGetSymbolAddress, once per device.
constexpr long long kNoAllocScratchDoubles = 1LL << 20;  // 8 MiB
constexpr int kNoAllocMaxB = 256;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
static __device__ __align__(256) int g_noalloc_act[kNoAllocMaxB];

struct NoAllocDev {
  double* scratch = nullptr;
  int* act = nullptr;
};
static std::mutex g_noalloc_mu;
static NoAllocDev g_noalloc_dev[256];

// First call on a device (that device current): look the arrays up and fill
// the source list 0..kNoAllocMaxB-1 once. Returns 0 or the CUDA error.
static cudaError_t noalloc_setup(NoAllocDev& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDev& d = g_noalloc_dev[dev];
  if (!d.scratch) {
    // the symbol lookup and the synchronous copy are device-wide operations:
    // hold them off while another thread of this process captures a graph
    // (the multi-system build captures on its lanes)
    DeviceWideGuard guard;
    void* sp = nullptr;
    void* ap = nullptr;
    e = cudaGetSymbolAddress(&sp, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&ap, g_noalloc_act);
    if (e != cudaSuccess) return e;
    int iota[kNoAllocMaxB];
    for (int k = 0; k < kNoAllocMaxB; ++k) iota[k] = k;
    e = cudaMemcpy(ap, iota, sizeof(iota), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    d.act = (int*)ap;
    d.scratch = (double*)sp;
  }
  out = d;
  return cudaSuccess;
}


}  // namespace dg

using namespace dg;

extern "C" {

int dg_apply_smoother_noalloc(dg_handle h, int32_t level, int32_t fp32, const void* r, void* z, int64_t B,
                              void* stream) {
  if (!h || level < 0 || level >= h->nlev || B < 0 || (B > 0 && (!r || !z))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  const bool coarsest = level == h->nlev - 1;
  if (!coarsest && h->opts.smoother != DG_SMOOTH_SCHWARZ) {
    h->err = "dg_apply_smoother_noalloc: only the Schwarz smoother and the coarsest level are supported";
    return DG_ERR_UNSUPPORTED;
  }
  const Level& L = h->levels[level];
  const long long mp = L.op.n1 + 2;
  const long long need = coarsest ? 0 : (long long)L.op.E * mp * mp * mp * B;  // elements of T
  const long long have = fp32 ? 2 * kNoAllocScratchDoubles : kNoAllocScratchDoubles;
  if (B > kNoAllocMaxB || need > have) {
    h->err = "dg_apply_smoother_noalloc: B * elements * (p+3)^3 exceeds the static scratch (8 MiB) or B > 256";
    return DG_ERR_INVALID_ARG;
  }
  NoAllocDev d;
  cudaError_t e = noalloc_setup(d);
  if (e != cudaSuccess) {
    h->err = std::string("dg_apply_smoother_noalloc: set-up: ") + cudaGetErrorString(e);
    return DG_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)B;
  if (coarsest) {
    if (fp32)
      DG_CK(launch_coarse_solve<float>(h->coarse_inv.as<double>(), h->Nc, (const float*)r, (float*)z, d.act, nb, s));
    else
      DG_CK(launch_coarse_solve<double>(h->coarse_inv.as<double>(), h->Nc, (const double*)r, (double*)z, d.act, nb,
                                        s));
  } else if (fp32) {
    DG_CK(launch_schwarz<float>(L.op, L.dop, L.sw_tabs.as<double>(), (const float*)r, (float*)d.scratch, (float*)z,
                                nullptr, 0, 0.0, 0.0, d.act, nb, s, L.tc()));
  } else {
    DG_CK(launch_schwarz<double>(L.op, L.dop, L.sw_tabs.as<double>(), (const double*)r, d.scratch, (double*)z,
                                 nullptr, 0, 0.0, 0.0, d.act, nb, s));
  }
  return DG_OK;
}

}  // extern "C"
