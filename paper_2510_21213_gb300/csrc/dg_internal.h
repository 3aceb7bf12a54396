// Internal declarations of the GB300 DG Poisson / exchange library.
//
// Operator structure used everywhere (Sec. 3.4 eq. sip_bilinear, Sec. 3.5):
// on a uniform axis-aligned mesh with tensor Gauss-Legendre nodal elements the
// SIPDG operator is the Kronecker sum
//     A = Ax (x) My (x) Mz + Mx (x) Ay (x) Mz + Mx (x) My (x) Az,
// where M_d is the (diagonal, collocated) 1-D mass and A_d the global 1-D
// SIPDG matrix of axis d. A_d is block tridiagonal: an element's diagonal
// block depends only on whether the element touches the domain boundary, and
// the coupling to a neighbour is rank 2 (the neighbour's trace and normal
// derivative at the shared face). The kernels apply A matrix-free from these
// 1-D tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "dg_poisson.h"

namespace dg {

// kernels launched by this library in this process (profiling / benchmark
// evidence), and by the calling thread (so that a thread capturing a graph can
// take back exactly the launches it recorded, while other threads launch)
extern std::atomic<long long> g_launch_count;
extern thread_local long long t_launch_count;
inline void count_launch(int n = 1) {
  g_launch_count.fetch_add(n, std::memory_order_relaxed);
  t_launch_count += n;
}
// launches recorded by this thread since `since` (a t_launch_count value) are
// removed from the process count: captured kernels are counted when replayed
inline long long uncount_captured(long long since) {
  const long long n = t_launch_count - since;
  g_launch_count.fetch_sub(n, std::memory_order_relaxed);
  t_launch_count = since;
  return n;
}

constexpr int MAXN1 = 9;    // p <= 8
constexpr int MAXLEV = 16;

// 1-D SIPDG data of one axis of one level (FP64).
struct AxisOp {
  int n;
  double lo, hi, h, sigma;
  // element diagonal blocks [type][a * n1 + i], type bit0 = left boundary
  // element, bit1 = right boundary element
  double Kd[4][MAXN1 * MAXN1];
  // coupling to the left neighbour (its value / reference derivative at its
  // right end) and to the right neighbour (at its left end), per row a
  double cLv[MAXN1], cLd[MAXN1], cRv[MAXN1], cRd[MAXN1];
  double m[MAXN1];            // collocated mass w_a h / 2
  double lift[2][MAXN1];      // Nitsche load coefficients, left / right boundary
};

// One multigrid level; plain data, copied to the device as is.
struct LevelOp {
  int n[3];
  int p, n1, E;
  long long Nq;
  double tl[MAXN1], tr[MAXN1], dl[MAXN1], dr[MAXN1];  // l_i(-1), l_i(1), l_i'(-1), l_i'(1)
  AxisOp ax[3];
};

// Transfer between a level and the next coarser one (plain data).
struct TransferOp {
  int kind;      // 0: same mesh, degree p -> p_c; 1: same degree 1, n -> n/2 (8 children)
  int n1f, n1c;
  // interpolation of coarse nodes to fine nodes: I[child position][a * n1c + i]
  double I[2][MAXN1 * MAXN1];
};

// Overlapping Schwarz smoother of one level: the patch of element e is the
// tensor box of global nodes covering e plus one node of each neighbour along
// every axis. Restricted to such a box the Kronecker-sum operator is again a
// Kronecker sum of restricted 1-D matrices, so each patch solve is exact by
// fast diagonalisation: A_P^-1 = (Sx(x)Sy(x)Sz) diag(1/(lx+ly+lz)) (Sx(x)Sy(x)Sz)^T
// with A~_d S_d = M~_d S_d Lambda_d, S_d^T M~_d S_d = I, per axis and element
// position. Device layout per axis: for each element position e_d,
// [m, oL] (ints, stored as doubles) then S [MP*MP] (row = patch node, col =
// mode) then lambda [MP]; MP = n1 + 2.
constexpr int MAXMP = MAXN1 + 2;
inline int schwarz_axis_stride(int n1) { return 2 + (n1 + 2) * (n1 + 2) + (n1 + 2); }

struct GemmArgs {
  int M, N, K, nb1, nb2;
  const void* A;
  long long sAm, sAk, sA1, sA2;
  const void* B;
  long long sBk, sBn, sB1, sB2;
  void* C;
  long long sCm, sCn, sC1, sC2;
  double alpha, beta;
  // optional workspace (elements of the GEMM's type) for splitting a long K
  // across blocks when there are few output tiles (FP32 path); null = no split
  void* work;
  long long work_elems;
};

// ---------------------------------------------------------------------------
// kernel launchers (dg_apply.cu, dg_vec.cu, dg_bc.cu)
// ---------------------------------------------------------------------------
// out = A u (mode 0), out = rin - A u (mode 1), out -= A u (mode 2)
template <typename T>
cudaError_t launch_apply(const LevelOp& hop, const LevelOp* dop, int mode, const T* u, T* out, const T* rin,
                         const int* act, int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_inv_diag(const LevelOp& hop, const LevelOp* dop, T* invD, cudaStream_t s);

// invD == nullptr: the residual argument is already preconditioned
template <typename T>
cudaError_t launch_cheb_first(T* x, T* d, const T* r, const T* invD, double c, int set_x, long long Nq,
                              const int* act, int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_cheb_step(T* x, T* d, const T* res, const T* invD, double c1, double c2, long long Nq,
                             const int* act, int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_xr(T* x, T* r, const T* p, const T* q, const double* alpha, long long Nq, const int* act,
                         int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_p(T* p, const T* z, const double* beta, long long Nq, const int* act, int nact,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_dot(const T* u, const T* v, const double* w, double* out, double* part, long long Nq,
                       const int* act, int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_zero(T* x, long long Nq, const int* act, int nact, cudaStream_t s);
template <typename Td, typename Ts>
cudaError_t launch_convert(Td* dst, const Ts* src, long long Nq, const int* act, int nact, double scale,
                           int accumulate, cudaStream_t s);

template <typename T>
cudaError_t launch_prolong_add(const TransferOp& htr, const TransferOp* dtr, const LevelOp& fine,
                               const LevelOp& coarse, const T* xc, T* xf, const int* act, int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const TransferOp& htr, const TransferOp* dtr, const LevelOp& fine,
                            const LevelOp& coarse, const T* rf, T* rc, const int* act, int nact, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(const double* Ainv, int Nc, const T* r, T* x, const int* act, int nact,
                                cudaStream_t s);

// Schwarz smoother: zp[rhs][e][MP^3] = A_P^-1 R_P r, then with y = sum_P R_P^T zp:
// mode 0: z = y; 1: z = c1 y, x = z; 2: z = c1 y, x += z; 3: z = c1 z + c2 y, x += z.
// tc (FP32 only, may be null): the level's tensor-core patch solve, used instead
// of the SIMT patch kernel
struct SwTcPlan;
// the patch solves alone: zp[rhs][e][MP^3] = A_P^-1 R_P r
template <typename T>
cudaError_t launch_schwarz_patch(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp,
                                 const int* act, int nact, cudaStream_t s, const SwTcPlan* tc = nullptr);
template <typename T>
cudaError_t launch_schwarz(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp, T* z,
                           T* x, int mode, double c1, double c2, const int* act, int nact, cudaStream_t s,
                           const SwTcPlan* tc = nullptr);

// sources and right-hand sides
cudaError_t launch_pair_sources(const double* psi, int N, const int* pi, const int* pj, int nsrc, long long Nq,
                                double* f, cudaStream_t s);
cudaError_t launch_row_products(const double* A, int NA, const double* B, const int* ia, const int* ib, int n,
                                long long Nq, double c, double* out, cudaStream_t s);
cudaError_t launch_scale(double* x, long long n, double c, cudaStream_t s);
cudaError_t launch_rhs_volume(const double* f, const double* W, double* b, long long Nq, int nsrc,
                              cudaStream_t s);
cudaError_t launch_finite_flags(const double* f, long long Nq, int nsrc, int* flags, cudaStream_t s);
template <typename Tg>
cudaError_t launch_lift(const LevelOp& hop, const LevelOp* dop, const Tg* g, double* b, int nsrc,
                        long long gstride, cudaStream_t s);

// boundary data
template <typename T>
cudaError_t launch_weighted_lex(const LevelOp& hop, const LevelOp* dop, const double* f, const double* W, T* flex,
                                int nsrc, cudaStream_t s);
template <typename T>
cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s);
cudaError_t launch_bc_direct(const LevelOp& hop, const LevelOp* dop, const double* f, const double* W,
                             const double* xq, const double* axis_nodes, int lmax, double* g, int nsrc,
                             long long gstride, long long nface, cudaStream_t s);

// exchange
cudaError_t launch_exch_accum(const double* psi, const double* v, double* Wacc, const int* ptr, const int* eb,
                              const int* es, int N, long long Nq, cudaStream_t s);
cudaError_t launch_kmat(const double* psi, const double* W, const double* Wacc, int N, long long Nq,
                        double* part, int nchunk, double* K, cudaStream_t s);

int kmat_chunks(long long Nq);

// per-element convolutional network of the learned initial guess (dg_nn.cu);
// parameters FP32 [NN_NPARAM], W2 also as BF16 [27][co][ci] (W2t) and [27][ci][co] (W2o)
constexpr int NN_NPARAM = 31170;
constexpr int NN_MAXN1 = 8;
cudaError_t nn_prep(const float* prm, void* W2t, void* W2o, cudaStream_t s);
cudaError_t nn_forward(int n1, const float* prm, const void* W2t, const float* in, float* out, void* a1, void* a2,
                       long long ne, cudaStream_t s);
int nn_backward_blocks(int n1, long long ne);
cudaError_t nn_backward(int n1, const float* prm, const void* W2o, const float* in, const void* a1, const void* a2,
                        const float* gout, float* part, float* grad, long long ne, cudaStream_t s);
cudaError_t nn_adam(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2, float eps,
                    int step, cudaStream_t s);

}  // namespace dg
