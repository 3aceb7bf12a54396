// Internal definition of the library handle (dg_ctx) and its device buffers,
// shared by the host driver and the allocation-free entry point.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "dg_setup.h"
#include "dg_swtc.h"

namespace dg {

// ---------------------------------------------------------------------------
// Device-wide operations (allocation and freeing, synchronous copies,
// device synchronisation, launches on the legacy stream) must not run in one
// host thread while another thread captures a CUDA graph: a device-wide
// synchronisation invalidates the capture. Captures hold a process-wide lock
// shared (CaptureGuard), device-wide sections hold it exclusively
// (DeviceWideGuard); nested exclusive sections of one thread are counted.
// ---------------------------------------------------------------------------
class DeviceWideGuard {
 public:
  DeviceWideGuard();
  ~DeviceWideGuard();
  DeviceWideGuard(const DeviceWideGuard&) = delete;
  DeviceWideGuard& operator=(const DeviceWideGuard&) = delete;
};
class CaptureGuard {
 public:
  CaptureGuard();
  ~CaptureGuard();
  CaptureGuard(const CaptureGuard&) = delete;
  CaptureGuard& operator=(const CaptureGuard&) = delete;

 private:
  bool shared_;
};

// ---------------------------------------------------------------------------
// device buffer helper
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  // owns its allocation: moved, never copied (a copy would free it twice)
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      DeviceWideGuard guard;
      cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (b <= bytes) return cudaSuccess;
    release();
    DeviceWideGuard guard;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = b;
    return cudaSuccess;
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

// per-level multigrid workspace of one precision
struct LevelWork {
  DevBuf x, b, res, d, invD, z, zp;
};

// One captured phase of a PCG iteration (CUDA graph), valid for one active
// source count and one generation of the workspace buffers.
struct PhaseGraph {
  cudaGraphExec_t exec = nullptr;
  int nact = -1;
  long long gen = -1;
  long long nkernels = 0;
  ~PhaseGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// PCG iterations captured as one graph: the first iteration (variant 0) or
// the preconditioner phase that continues an interrupted solve (variant 1),
// then a conditional while-node whose body runs the preconditioner phase, the
// next operator phase and the device-side convergence test. The loop stops
// when a source converges (so that the host can drop it from the batch), when
// none is left, or at the iteration limit. Valid for one active source count
// and one generation of the workspace buffers; the tolerances and the limit
// are read from device memory.
struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  long long gen = -1;
  long long nk_first = 0, nk_body = 0;  // kernels before the loop and of the loop body
  LoopGraph() = default;
  LoopGraph(const LoopGraph&) = delete;
  LoopGraph& operator=(const LoopGraph&) = delete;
  ~LoopGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

template <typename T>
struct PrecWork {
  std::vector<LevelWork> lev;            // per level (level 0: res, d, invD only)
  DevBuf x, r, z, p, q;                  // CG vectors on the fine level
  int cap = 0;
  PhaseGraph gA, gB;                     // captured PCG phases (operator / preconditioner)
  std::map<std::pair<int, int>, std::unique_ptr<LoopGraph>> gL;  // device-side loops by (variant, sources)
};

struct Level {
  LevelOp op;
  LevelOp* dop = nullptr;
  TransferOp tr;                 // to the next coarser level
  TransferOp* dtr = nullptr;
  double lam_max = 0;            // lambda_max(D^-1 A) (point Jacobi)
  double lam_sw = 0;             // lambda_max(M_S A) estimate (Schwarz)
  DevBuf sw_tabs;                // Schwarz patch tables
  DevBuf sw_tc;                  // tables of the tensor-core patch solve (FP32 inner solve), if used
  SwTcPlan tcp;                  // its device blob (null: SIMT patch solve) and header
  const SwTcPlan* tc() const { return tcp.blob && !tcp.off ? &tcp : nullptr; }
};

struct BcAxisTables {
  int L = 0;
  DevBuf gn;   // [2][NG][L]       exp(-a_k (x_X - face_s)^2)
  DevBuf G;    // [NG][L][L]       exp(-a_k (x_i - x_j)^2)
  DevBuf Gs;   // [L][NG * L]      c_k exp(-a_k (x_i - x_j)^2)
};

// network of the learned initial guess: parameters, Adam state, batch buffers
struct NNState {
  bool have = false;     // parameters set
  bool bf16_ok = false;  // BF16 copies of W2 match prm
  int step = 0;          // Adam steps taken
  DevBuf prm, W2t, W2o, m, v, grad, part;
  DevBuf in, out, a1, a2;
  long long save_ne = -1;  // elements whose activations a1 / a2 hold (-1: none)
};

}  // namespace dg

struct dg_ctx {
  dg_mesh_desc mesh;
  dg_solver_opts opts;
  std::vector<dg::Level> levels;
  int nlev = 0;
  // coarsest level
  int Nc = 0;
  dg::DevBuf coarse_inv;
  // fine-level geometry
  long long Nq = 0;
  std::vector<double> axis_nodes[3];
  dg::DevBuf d_W, d_xq, d_axn;
  int lmax = 0;
  long long nface = 0;
  // boundary-data tables: FP64 (1e-12 Gaussian sum) and, in the mixed modes,
  // FP32 (1e-7 Gaussian sum)
  dg::GaussSum gsum, gsum32;
  int NG = 0, NG32 = 0;
  dg::BcAxisTables bct[3], bct32[3];
  dg::DevBuf flex32, T1_32, T2_32, g32;
  dg::DevBuf gemm_ws;              // split-K partials of the FP32 boundary-data GEMMs
  // workspaces
  dg::PrecWork<double> w64;
  dg::PrecWork<float> w32;
  dg::DevBuf f64, b64, x64, r64;   // [cap][Nq]
  dg::DevBuf flex, T1, T2, g;      // boundary data
  dg::DevBuf part, scal, act, flags, pidx;
  dg::DevBuf loop;  // device-side PCG loop state: done[cap], iters[cap], counter, limit, tol[cap], relres[cap]
  dg::DevBuf tc_err;               // device word: a tensor-core kernel's wait gave up (DG_ERR_TIMEOUT)
  dg::DevBuf Wacc, kpart, Kdev;
  int cap = 0;
  std::vector<int> act_host;  // contents of act (device) as last uploaded
  std::string err;
  long long ws_bytes = 0;
  long long buf_gen = 0;      // bumped whenever a workspace buffer is (re)allocated
  bool use_graphs = true;     // capture the PCG phases as CUDA graphs
  cudaStream_t ws = nullptr;  // the handle's own stream (graph capture needs a non-default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  dg::NNState nn;             // learned initial guess (DG_PREC_MIXED_LEARNED)
  dg::DevBuf dlift_op;        // fine-level LevelOp whose lift tables carry (sigma_c - sigma) (coarse guess)
  // adaptively compressed exchange from the last whole exchange build: W (in
  // Wacc) and K, valid while ace_N > 0
  int ace_N = 0;
  std::vector<double> ace_K;  // [N*N] row-major
  dg::DevBuf ace_part, ace_C;
  ~dg_ctx() {
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ws) cudaStreamDestroy(ws);
  }
};

namespace dg {

#define DG_CK(call)                                                                                    \
  do {                                                                                                 \
    cudaError_t e__ = (call);                                                                          \
    if (e__ != cudaSuccess) {                                                                          \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e__);                                    \
      return e__ == cudaErrorMemoryAllocation ? DG_ERR_NO_MEMORY : DG_ERR_CUDA;                        \
    }                                                                                                  \
  } while (0)

// workspace helpers shared by the translation units of the library
template <typename T>
int ensure_prec(dg_ctx* h, PrecWork<T>& w, int cap);
int ensure_common(dg_ctx* h, int cap);
int upload_act(dg_ctx* h, const std::vector<int>& a, cudaStream_t s);
int autotune_batch(dg_ctx* h, int max_sources, cudaStream_t s);
int prepare(dg_ctx* h, int cap);
int form_rhs(dg_ctx* h, const double* f, int nsrc, cudaStream_t s);
int check_finite(dg_ctx* h, const double* f, int nsrc, std::vector<int>& finite, cudaStream_t s);

// learned initial guess (dg_learned.cu): for the sources in act, sets x64 and
// r64 = b64 - A x64 (b64 formed), rel[k] = ||r64|| / ||b64||, fb[k] = 1 where
// the guess was rejected (x64 = 0, r64 = b64)
// nsrc: sources 0..nsrc-1 of the current chunk (b64 and the boundary data formed)
int learned_guess(dg_ctx* h, int nsrc, const std::vector<int>& act, const std::vector<double>& bnorm2, bool use_net,
                  std::vector<double>& rel, std::vector<int>& fb, cudaStream_t s);
// boundary data of the chunk are held in FP32 (g32) rather than FP64 (g)
bool bc_fp32(const dg_ctx* h);
int nn_load_file(dg_ctx* h, const char* path);

// scalar slots of h->scal, each [cap] doubles
enum { S_BN = 0, S_RR, S_RZ, S_RZN, S_PQ, S_AL, S_BE, S_G1, S_G2, S_G3, S_NSLOT };
inline double* scal(dg_ctx* h, int slot) { return h->scal.as<double>() + (size_t)slot * h->cap; }

#define DG_RET(call)                 \
  do {                               \
    int r__ = (call);                \
    if (r__ != DG_OK) return r__;    \
  } while (0)

}  // namespace dg
