// Vector kernels of the multigrid-preconditioned CG (Sec. 6.4), the
// hp-transfers, the coarsest-level solve, the right-hand sides (Sec. 6.1,
// Sec. 6.3) and the exchange accumulation and contraction (Sec. 6.1.2,
// eq. fock_exchange).
//
// Batched fields are [B][Nq]; kernels work on the active right-hand sides
// listed in act[0..nact), so converged sources cost nothing. All reductions
// are deterministic: fixed grids, fixed summation order, FP64 accumulation.
#include <algorithm>

#include "dg_internal.h"

namespace dg {

static constexpr int VT = 256;

// ---------------------------------------------------------------------------
// elementwise
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_cheb_first(T* __restrict__ x, T* __restrict__ d, const T* __restrict__ r,
                             const T* __restrict__ invD, T c, int set_x, long long Nq, const int* __restrict__ act) {
  const long long rhs = act[blockIdx.y];
  const long long off = rhs * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x) {
    const T v = invD ? c * invD[i] * r[off + i] : c * r[off + i];
    d[off + i] = v;
    x[off + i] = set_x ? v : x[off + i] + v;
  }
}

template <typename T>
__global__ void k_cheb_step(T* __restrict__ x, T* __restrict__ d, const T* __restrict__ res,
                            const T* __restrict__ invD, T c1, T c2, long long Nq, const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x) {
    const T v = c1 * d[off + i] + (invD ? c2 * invD[i] * res[off + i] : c2 * res[off + i]);
    d[off + i] = v;
    x[off + i] += v;
  }
}

template <typename T>
__global__ void k_cg_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                        const double* __restrict__ alpha, long long Nq, const int* __restrict__ act) {
  const int rhs = act[blockIdx.y];
  const long long off = (long long)rhs * Nq;
  const T al = (T)alpha[rhs];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x) {
    x[off + i] += al * p[off + i];
    r[off + i] -= al * q[off + i];
  }
}

template <typename T>
__global__ void k_cg_p(T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ beta, long long Nq,
                       const int* __restrict__ act) {
  const int rhs = act[blockIdx.y];
  const long long off = (long long)rhs * Nq;
  const T be = (T)beta[rhs];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
    p[off + i] = z[off + i] + be * p[off + i];
}

template <typename T>
__global__ void k_zero(T* __restrict__ x, long long Nq, const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
    x[off + i] = (T)0;
}

template <typename Td, typename Ts>
__global__ void k_convert(Td* __restrict__ dst, const Ts* __restrict__ src, long long Nq, const int* __restrict__ act,
                          double scale, int accumulate) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)src[off + i] * scale;
    dst[off + i] = accumulate ? (Td)((double)dst[off + i] + v) : (Td)v;
  }
}

static inline dim3 vgrid(long long Nq, int nact) {
  long long gx = (Nq + VT * 4 - 1) / (VT * 4);
  if (gx > 4096) gx = 4096;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)nact);
}

template <typename T>
cudaError_t launch_cheb_first(T* x, T* d, const T* r, const T* invD, double c, int set_x, long long Nq,
                              const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_cheb_first<T><<<vgrid(Nq, nact), VT, 0, s>>>(x, d, r, invD, (T)c, set_x, Nq, act);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cheb_step(T* x, T* d, const T* res, const T* invD, double c1, double c2, long long Nq,
                             const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_cheb_step<T><<<vgrid(Nq, nact), VT, 0, s>>>(x, d, res, invD, (T)c1, (T)c2, Nq, act);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_xr(T* x, T* r, const T* p, const T* q, const double* alpha, long long Nq, const int* act,
                         int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_cg_xr<T><<<vgrid(Nq, nact), VT, 0, s>>>(x, r, p, q, alpha, Nq, act);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_p(T* p, const T* z, const double* beta, long long Nq, const int* act, int nact,
                        cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_cg_p<T><<<vgrid(Nq, nact), VT, 0, s>>>(p, z, beta, Nq, act);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_zero(T* x, long long Nq, const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_zero<T><<<vgrid(Nq, nact), VT, 0, s>>>(x, Nq, act);
  return cudaGetLastError();
}
template <typename Td, typename Ts>
cudaError_t launch_convert(Td* dst, const Ts* src, long long Nq, const int* act, int nact, double scale,
                           int accumulate, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_convert<Td, Ts><<<vgrid(Nq, nact), VT, 0, s>>>(dst, src, Nq, act, scale, accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// deterministic dots: out[rhs] = sum_i u_i v_i (w_i), FP64 accumulation
// ---------------------------------------------------------------------------
static constexpr int DOT_BLOCKS = 304;  // 2 blocks per SM of a 152-SM GB300; fixed for determinism

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void k_dot_partial(const T* __restrict__ u, const T* __restrict__ v, const double* __restrict__ w,
                              double* __restrict__ part, long long Nq, const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  double acc = 0.0;
  if (sizeof(T) == 4 && w == nullptr) {
    // FP32 vectors (the inner solve): each thread's few terms (about 16 when
    // Nq / 4096 blocks run) summed by FP32 FMA, then FP64 across threads; the
    // FP64 pipe would otherwise bound the kernel
    float accf = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
      accf = fmaf((float)u[off + i], (float)v[off + i], accf);
    acc = (double)accf;
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x) {
      double t = (double)u[off + i] * (double)v[off + i];
      if (w) t *= w[i];
      acc += t;
    }
  }
  __shared__ double sh[VT / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < VT / 32 ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_dot_final(const double* __restrict__ part, double* __restrict__ out, int nblk,
                            const int* __restrict__ act) {
  // one warp per active rhs; fixed lane assignment and tree order
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 32) acc += part[(long long)k * nblk + i];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[act[k]] = acc;
}

template <typename T>
cudaError_t launch_dot(const T* u, const T* v, const double* w, double* out, double* part, long long Nq,
                       const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  // blocks per source from Nq alone (about 4096 nodes each, at most DOT_BLOCKS),
  // so a source's summation order never depends on how many sources share the launch
  const int nblk = (int)std::max(1LL, std::min((long long)DOT_BLOCKS, (Nq + 4095) / 4096));
  count_launch();
  k_dot_partial<T><<<dim3(nblk, nact), VT, 0, s>>>(u, v, w, part, Nq, act);
  count_launch();
  k_dot_final<<<nact, 32, 0, s>>>(part, out, nblk, act);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// hp transfers (sum-factorised, one coarse element per block)
// ---------------------------------------------------------------------------
// Prolongation: xf += P xc. For a p-transfer the fine element is the coarse
// element; for an h-transfer (degree 1) the coarse element has 8 children
// whose node positions map into the parent's reference cube.
template <typename T>
__global__ void k_prolong_add(const TransferOp* __restrict__ tr, const T* __restrict__ xc, T* __restrict__ xf,
                              int nxc, int nyc, int nzc, long long Nqc, long long Nqf, const int* __restrict__ act) {
  __shared__ double sI[2][MAXN1 * MAXN1];
  __shared__ double sc[MAXN1 * MAXN1 * MAXN1];
  __shared__ double s1[MAXN1 * MAXN1 * MAXN1];
  __shared__ double s2[MAXN1 * MAXN1 * MAXN1];
  const int n1f = tr->n1f, n1c = tr->n1c;
  const int npc = n1c * n1c * n1c, npf = n1f * n1f * n1f;
  const int ec = blockIdx.x;
  const long long rhs = act[blockIdx.y];
  for (int i = threadIdx.x; i < 2 * MAXN1 * MAXN1; i += blockDim.x) sI[i / (MAXN1 * MAXN1)][i % (MAXN1 * MAXN1)] = tr->I[i / (MAXN1 * MAXN1)][i % (MAXN1 * MAXN1)];
  for (int i = threadIdx.x; i < npc; i += blockDim.x) sc[i] = (double)xc[rhs * Nqc + (long long)ec * npc + i];
  __syncthreads();
  const int nch = tr->kind == 1 ? 8 : 1;
  const int ecx = ec % nxc, ecy = (ec / nxc) % nyc, ecz = ec / (nxc * nyc);
  for (int ch = 0; ch < nch; ++ch) {
    const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
    const double* Ix = sI[tr->kind == 1 ? cx : 0];
    const double* Iy = sI[tr->kind == 1 ? cy : 0];
    const double* Iz = sI[tr->kind == 1 ? cz : 0];
    // stage 1: x direction  s1[k][j][a] = sum_i Ix[a,i] c[k][j][i]
    for (int t = threadIdx.x; t < n1c * n1c * n1f; t += blockDim.x) {
      const int a = t % n1f, jk = t / n1f;
      double acc = 0.0;
      for (int i = 0; i < n1c; ++i) acc += Ix[a * n1c + i] * sc[jk * n1c + i];
      s1[t] = acc;
    }
    __syncthreads();
    // stage 2: y  s2[k][b][a] = sum_j Iy[b,j] s1[k][j][a]
    for (int t = threadIdx.x; t < n1c * n1f * n1f; t += blockDim.x) {
      const int a = t % n1f, b = (t / n1f) % n1f, kk = t / (n1f * n1f);
      double acc = 0.0;
      for (int j = 0; j < n1c; ++j) acc += Iy[b * n1c + j] * s1[(kk * n1c + j) * n1f + a];
      s2[t] = acc;
    }
    __syncthreads();
    // stage 3: z, add into the fine element
    long long ef;
    if (tr->kind == 1) {
      const int nxf = 2 * nxc, nyf = 2 * nyc;
      ef = (long long)(2 * ecx + cx) + (long long)nxf * ((2 * ecy + cy) + (long long)nyf * (2 * ecz + cz));
    } else {
      ef = ec;
    }
    T* dst = xf + rhs * Nqf + ef * npf;
    for (int t = threadIdx.x; t < npf; t += blockDim.x) {
      const int ab = t % (n1f * n1f), c = t / (n1f * n1f);
      double acc = 0.0;
      for (int kk = 0; kk < n1c; ++kk) acc += Iz[c * n1c + kk] * s2[kk * n1f * n1f + ab];
      dst[t] = (T)((double)dst[t] + acc);
    }
    __syncthreads();
  }
}

// Restriction rc = P^T rf (gathers the children of each coarse element).
template <typename T>
__global__ void k_restrict(const TransferOp* __restrict__ tr, const T* __restrict__ rf, T* __restrict__ rc, int nxc,
                           int nyc, int nzc, long long Nqc, long long Nqf, const int* __restrict__ act) {
  __shared__ double sI[2][MAXN1 * MAXN1];
  __shared__ double sf[MAXN1 * MAXN1 * MAXN1];
  __shared__ double s1[MAXN1 * MAXN1 * MAXN1];
  __shared__ double s2[MAXN1 * MAXN1 * MAXN1];
  __shared__ double so[MAXN1 * MAXN1 * MAXN1];
  const int n1f = tr->n1f, n1c = tr->n1c;
  const int npc = n1c * n1c * n1c, npf = n1f * n1f * n1f;
  const int ec = blockIdx.x;
  const long long rhs = act[blockIdx.y];
  for (int i = threadIdx.x; i < 2 * MAXN1 * MAXN1; i += blockDim.x) sI[i / (MAXN1 * MAXN1)][i % (MAXN1 * MAXN1)] = tr->I[i / (MAXN1 * MAXN1)][i % (MAXN1 * MAXN1)];
  for (int i = threadIdx.x; i < npc; i += blockDim.x) so[i] = 0.0;
  const int nch = tr->kind == 1 ? 8 : 1;
  const int ecx = ec % nxc, ecy = (ec / nxc) % nyc, ecz = ec / (nxc * nyc);
  for (int ch = 0; ch < nch; ++ch) {
    const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
    const double* Ix = sI[tr->kind == 1 ? cx : 0];
    const double* Iy = sI[tr->kind == 1 ? cy : 0];
    const double* Iz = sI[tr->kind == 1 ? cz : 0];
    long long ef;
    if (tr->kind == 1) {
      const int nxf = 2 * nxc, nyf = 2 * nyc;
      ef = (long long)(2 * ecx + cx) + (long long)nxf * ((2 * ecy + cy) + (long long)nyf * (2 * ecz + cz));
    } else {
      ef = ec;
    }
    __syncthreads();
    const T* src = rf + rhs * Nqf + ef * npf;
    for (int t = threadIdx.x; t < npf; t += blockDim.x) sf[t] = (double)src[t];
    __syncthreads();
    // stage 1 (x^T): s1[c][b][i] = sum_a Ix[a,i] f[c][b][a]
    for (int t = threadIdx.x; t < n1f * n1f * n1c; t += blockDim.x) {
      const int i = t % n1c, bc = t / n1c;
      double acc = 0.0;
      for (int a = 0; a < n1f; ++a) acc += Ix[a * n1c + i] * sf[bc * n1f + a];
      s1[t] = acc;
    }
    __syncthreads();
    // stage 2 (y^T): s2[c][j][i] = sum_b Iy[b,j] s1[c][b][i]
    for (int t = threadIdx.x; t < n1f * n1c * n1c; t += blockDim.x) {
      const int i = t % n1c, j = (t / n1c) % n1c, c = t / (n1c * n1c);
      double acc = 0.0;
      for (int b = 0; b < n1f; ++b) acc += Iy[b * n1c + j] * s1[(c * n1f + b) * n1c + i];
      s2[t] = acc;
    }
    __syncthreads();
    // stage 3 (z^T): so[k][j][i] += sum_c Iz[c,k] s2[c][j][i]
    for (int t = threadIdx.x; t < npc; t += blockDim.x) {
      const int ji = t % (n1c * n1c), kk = t / (n1c * n1c);
      double acc = 0.0;
      for (int c = 0; c < n1f; ++c) acc += Iz[c * n1c + kk] * s2[c * n1c * n1c + ji];
      so[t] += acc;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < npc; t += blockDim.x) rc[rhs * Nqc + (long long)ec * npc + t] = (T)so[t];
}

// Fixed-size transfers: the degree pairs of the hierarchy (p -> floor(p/2),
// and the degree-1 h-transfer) compiled with their sizes, several coarse
// elements per block, arithmetic in the vector precision T. The per-node
// summation order is that of the generic kernels above (stage by stage, terms
// in index order), so the FP64 results are the same.
template <int N1F, int N1C>
struct PXferCfg {
  static constexpr int NPC = N1C * N1C * N1C, NPF = N1F * N1F * N1F;
  static constexpr int EPB = 1024 / NPF < 1 ? 1 : 1024 / NPF;  // coarse elements per block
  static constexpr int THREADS = 256;
};

// p-transfer prolongation, xf += P xc: the fine element is the coarse element.
template <typename T, int N1F, int N1C>
__global__ void __launch_bounds__(256) k_prolong_p(const TransferOp* __restrict__ tr, const T* __restrict__ xc,
                                                   T* __restrict__ xf, int E, long long Nqc, long long Nqf,
                                                   const int* __restrict__ act) {
  using C = PXferCfg<N1F, N1C>;
  constexpr int NPC = C::NPC, NPF = C::NPF, EPB = C::EPB, NT = C::THREADS;
  constexpr int S1 = N1C * N1C * N1F, S2 = N1C * N1F * N1F;
  __shared__ T sI[N1F * N1C];
  __shared__ T sc[EPB * NPC];
  __shared__ T s1[EPB * S1];
  __shared__ T s2[EPB * S2];
  const long long rhs = act[blockIdx.y];
  const int e0 = blockIdx.x * EPB;
  const int ne = E - e0 < EPB ? E - e0 : EPB;
  for (int i = threadIdx.x; i < N1F * N1C; i += NT) sI[i] = (T)tr->I[0][i];
  const T* src = xc + rhs * Nqc + (long long)e0 * NPC;
  for (int t = threadIdx.x; t < ne * NPC; t += NT) sc[t] = src[t];
  __syncthreads();
  // x: s1[el][k][j][a] = sum_i I[a,i] c[el][k][j][i]
  for (int t = threadIdx.x; t < ne * S1; t += NT) {
    const int el = t / S1, r = t % S1, a = r % N1F, jk = r / N1F;
    T acc = (T)0;
#pragma unroll
    for (int i = 0; i < N1C; ++i) acc += sI[a * N1C + i] * sc[el * NPC + jk * N1C + i];
    s1[t] = acc;
  }
  __syncthreads();
  // y: s2[el][k][b][a] = sum_j I[b,j] s1[el][k][j][a]
  for (int t = threadIdx.x; t < ne * S2; t += NT) {
    const int el = t / S2, r = t % S2, a = r % N1F, b = (r / N1F) % N1F, kk = r / (N1F * N1F);
    T acc = (T)0;
#pragma unroll
    for (int j = 0; j < N1C; ++j) acc += sI[b * N1C + j] * s1[el * S1 + (kk * N1C + j) * N1F + a];
    s2[t] = acc;
  }
  __syncthreads();
  // z, added into the fine elements (contiguous: same element order)
  T* dst = xf + rhs * Nqf + (long long)e0 * NPF;
  for (int t = threadIdx.x; t < ne * NPF; t += NT) {
    const int el = t / NPF, r = t % NPF, ab = r % (N1F * N1F), c = r / (N1F * N1F);
    T acc = (T)0;
#pragma unroll
    for (int kk = 0; kk < N1C; ++kk) acc += sI[c * N1C + kk] * s2[el * S2 + kk * N1F * N1F + ab];
    dst[t] = dst[t] + acc;
  }
}

// p-transfer restriction, rc = P^T rf.
template <typename T, int N1F, int N1C>
__global__ void __launch_bounds__(256) k_restrict_p(const TransferOp* __restrict__ tr, const T* __restrict__ rf,
                                                    T* __restrict__ rc, int E, long long Nqc, long long Nqf,
                                                    const int* __restrict__ act) {
  using C = PXferCfg<N1F, N1C>;
  constexpr int NPC = C::NPC, NPF = C::NPF, EPB = C::EPB, NT = C::THREADS;
  constexpr int S1 = N1F * N1F * N1C, S2 = N1F * N1C * N1C;
  __shared__ T sI[N1F * N1C];
  __shared__ T sf[EPB * NPF];
  __shared__ T s1[EPB * S1];
  __shared__ T s2[EPB * S2];
  const long long rhs = act[blockIdx.y];
  const int e0 = blockIdx.x * EPB;
  const int ne = E - e0 < EPB ? E - e0 : EPB;
  for (int i = threadIdx.x; i < N1F * N1C; i += NT) sI[i] = (T)tr->I[0][i];
  const T* src = rf + rhs * Nqf + (long long)e0 * NPF;
  for (int t = threadIdx.x; t < ne * NPF; t += NT) sf[t] = src[t];
  __syncthreads();
  // x^T: s1[el][c][b][i] = sum_a I[a,i] f[el][c][b][a]
  for (int t = threadIdx.x; t < ne * S1; t += NT) {
    const int el = t / S1, r = t % S1, i = r % N1C, bc = r / N1C;
    T acc = (T)0;
#pragma unroll
    for (int a = 0; a < N1F; ++a) acc += sI[a * N1C + i] * sf[el * NPF + bc * N1F + a];
    s1[t] = acc;
  }
  __syncthreads();
  // y^T: s2[el][c][j][i] = sum_b I[b,j] s1[el][c][b][i]
  for (int t = threadIdx.x; t < ne * S2; t += NT) {
    const int el = t / S2, r = t % S2, i = r % N1C, j = (r / N1C) % N1C, c = r / (N1C * N1C);
    T acc = (T)0;
#pragma unroll
    for (int b = 0; b < N1F; ++b) acc += sI[b * N1C + j] * s1[el * S1 + (c * N1F + b) * N1C + i];
    s2[t] = acc;
  }
  __syncthreads();
  // z^T: rc[el][k][j][i] = sum_c I[c,k] s2[el][c][j][i]
  T* dst = rc + rhs * Nqc + (long long)e0 * NPC;
  for (int t = threadIdx.x; t < ne * NPC; t += NT) {
    const int el = t / NPC, r = t % NPC, ji = r % (N1C * N1C), kk = r / (N1C * N1C);
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < N1F; ++c) acc += sI[c * N1C + kk] * s2[el * S2 + c * N1C * N1C + ji];
    dst[t] = acc;
  }
}

// Degree-1 h-transfer prolongation: one thread per fine node, 4 coarse
// elements (8 children of 8 nodes each) per block of 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_h(const TransferOp* __restrict__ tr, const T* __restrict__ xc,
                                                   T* __restrict__ xf, int nxc, int nyc, int E, long long Nqc,
                                                   long long Nqf, const int* __restrict__ act) {
  __shared__ T sI[2][4];
  const long long rhs = act[blockIdx.y];
  if (threadIdx.x < 8) sI[threadIdx.x >> 2][threadIdx.x & 3] = (T)tr->I[threadIdx.x >> 2][threadIdx.x & 3];
  __syncthreads();
  const int ec = blockIdx.x * 4 + (threadIdx.x >> 6);
  if (ec >= E) return;
  const int ch = (threadIdx.x >> 3) & 7, node = threadIdx.x & 7;
  const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
  const int a = node & 1, b = (node >> 1) & 1, c = node >> 2;
  const T* Ix = sI[cx];
  const T* Iy = sI[cy];
  const T* Iz = sI[cz];
  const T* cc = xc + rhs * Nqc + (long long)ec * 8;
  T cv[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) cv[q] = cc[q];
  // s1[k][j] = sum_i Ix[a,i] c[k][j][i]; s2[k] = sum_j Iy[b,j] s1[k][j]; out = sum_k Iz[c,k] s2[k]
  T s2v[2];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    T s1v[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      T acc = (T)0;
#pragma unroll
      for (int i = 0; i < 2; ++i) acc += Ix[a * 2 + i] * cv[(kk * 2 + j) * 2 + i];
      s1v[j] = acc;
    }
    T acc = (T)0;
#pragma unroll
    for (int j = 0; j < 2; ++j) acc += Iy[b * 2 + j] * s1v[j];
    s2v[kk] = acc;
  }
  T acc = (T)0;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) acc += Iz[c * 2 + kk] * s2v[kk];
  const int ecx = ec % nxc, ecy = (ec / nxc) % nyc, ecz = ec / (nxc * nyc);
  const long long ef = (long long)(2 * ecx + cx) + (long long)(2 * nxc) * ((2 * ecy + cy) + (long long)(2 * nyc) * (2 * ecz + cz));
  T* dst = xf + rhs * Nqf + ef * 8 + node;
  *dst = *dst + acc;
}

// Degree-1 h-transfer restriction: one thread per coarse node, the children
// summed in order; 32 coarse elements per block of 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_h(const TransferOp* __restrict__ tr, const T* __restrict__ rf,
                                                    T* __restrict__ rc, int nxc, int nyc, int E, long long Nqc,
                                                    long long Nqf, const int* __restrict__ act) {
  __shared__ T sI[2][4];
  const long long rhs = act[blockIdx.y];
  if (threadIdx.x < 8) sI[threadIdx.x >> 2][threadIdx.x & 3] = (T)tr->I[threadIdx.x >> 2][threadIdx.x & 3];
  __syncthreads();
  const int ec = blockIdx.x * 32 + (threadIdx.x >> 3);
  if (ec >= E) return;
  const int node = threadIdx.x & 7;
  const int i = node & 1, j = (node >> 1) & 1, kk = node >> 2;
  const int ecx = ec % nxc, ecy = (ec / nxc) % nyc, ecz = ec / (nxc * nyc);
  T so = (T)0;
  for (int ch = 0; ch < 8; ++ch) {
    const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
    const T* Ix = sI[cx];
    const T* Iy = sI[cy];
    const T* Iz = sI[cz];
    const long long ef = (long long)(2 * ecx + cx) + (long long)(2 * nxc) * ((2 * ecy + cy) + (long long)(2 * nyc) * (2 * ecz + cz));
    const T* f = rf + rhs * Nqf + ef * 8;
    T fv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) fv[q] = f[q];
    // s1[c][b] = sum_a Ix[a,i] f[c][b][a]; s2[c] = sum_b Iy[b,j] s1[c][b]; so += sum_c Iz[c,kk] s2[c]
    T s2v[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T s1v[2];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        T acc = (T)0;
#pragma unroll
        for (int a = 0; a < 2; ++a) acc += Ix[a * 2 + i] * fv[(c * 2 + b) * 2 + a];
        s1v[b] = acc;
      }
      T acc = (T)0;
#pragma unroll
      for (int b = 0; b < 2; ++b) acc += Iy[b * 2 + j] * s1v[b];
      s2v[c] = acc;
    }
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < 2; ++c) acc += Iz[c * 2 + kk] * s2v[c];
    so += acc;
  }
  rc[rhs * Nqc + (long long)ec * 8 + node] = so;
}

template <typename T, int N1F, int N1C>
static void launch_xfer_p(bool prolong, const TransferOp* dtr, const LevelOp& fine, const LevelOp& coarse,
                          const T* in, T* out, const int* act, int nact, cudaStream_t s) {
  using C = PXferCfg<N1F, N1C>;
  const dim3 grid((unsigned)((coarse.E + C::EPB - 1) / C::EPB), (unsigned)nact);
  count_launch();
  if (prolong)
    k_prolong_p<T, N1F, N1C><<<grid, C::THREADS, 0, s>>>(dtr, in, out, coarse.E, coarse.Nq, fine.Nq, act);
  else
    k_restrict_p<T, N1F, N1C><<<grid, C::THREADS, 0, s>>>(dtr, in, out, coarse.E, coarse.Nq, fine.Nq, act);
}

// Fixed-size transfer for the level pair if one is compiled; false otherwise.
template <typename T>
static bool launch_xfer_fixed(bool prolong, const TransferOp& htr, const TransferOp* dtr, const LevelOp& fine,
                              const LevelOp& coarse, const T* in, T* out, const int* act, int nact, cudaStream_t s) {
  if (htr.kind == 1) {
    if (htr.n1f != 2 || htr.n1c != 2) return false;
    count_launch();
    if (prolong)
      k_prolong_h<T><<<dim3((unsigned)((coarse.E + 3) / 4), (unsigned)nact), 256, 0, s>>>(
          dtr, in, out, coarse.n[0], coarse.n[1], coarse.E, coarse.Nq, fine.Nq, act);
    else
      k_restrict_h<T><<<dim3((unsigned)((coarse.E + 31) / 32), (unsigned)nact), 256, 0, s>>>(
          dtr, in, out, coarse.n[0], coarse.n[1], coarse.E, coarse.Nq, fine.Nq, act);
    return true;
  }
  const int key = htr.n1f * 16 + htr.n1c;
  switch (key) {
    case 3 * 16 + 2: launch_xfer_p<T, 3, 2>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    case 4 * 16 + 2: launch_xfer_p<T, 4, 2>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    case 5 * 16 + 3: launch_xfer_p<T, 5, 3>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    case 6 * 16 + 3: launch_xfer_p<T, 6, 3>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    case 7 * 16 + 4: launch_xfer_p<T, 7, 4>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    case 8 * 16 + 4: launch_xfer_p<T, 8, 4>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    case 9 * 16 + 5: launch_xfer_p<T, 9, 5>(prolong, dtr, fine, coarse, in, out, act, nact, s); return true;
    default: return false;
  }
}

template <typename T>
cudaError_t launch_prolong_add(const TransferOp& htr, const TransferOp* dtr, const LevelOp& fine,
                               const LevelOp& coarse, const T* xc, T* xf, const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  if (launch_xfer_fixed<T>(true, htr, dtr, fine, coarse, xc, xf, act, nact, s)) return cudaGetLastError();
  count_launch();
  k_prolong_add<T><<<dim3(coarse.E, nact), 128, 0, s>>>(dtr, xc, xf, coarse.n[0], coarse.n[1], coarse.n[2],
                                                         coarse.Nq, fine.Nq, act);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict(const TransferOp& htr, const TransferOp* dtr, const LevelOp& fine,
                            const LevelOp& coarse, const T* rf, T* rc, const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  if (launch_xfer_fixed<T>(false, htr, dtr, fine, coarse, rf, rc, act, nact, s)) return cudaGetLastError();
  count_launch();
  k_restrict<T><<<dim3(coarse.E, nact), 128, 0, s>>>(dtr, rf, rc, coarse.n[0], coarse.n[1], coarse.n[2], coarse.Nq,
                                                      fine.Nq, act);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// coarsest level: x = A_c^{-1} r with the inverse formed at setup (FP64)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_coarse_solve(const double* __restrict__ Ainv, int Nc, const T* __restrict__ r, T* __restrict__ x,
                               const int* __restrict__ act) {
  // grid (row blocks of 32 rows, active sources); one warp per row
  extern __shared__ double sr[];
  const long long off = (long long)act[blockIdx.y] * Nc;
  for (int i = threadIdx.x; i < Nc; i += blockDim.x) sr[i] = (double)r[off + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int r0 = blockIdx.x * 32, r1 = min(Nc, r0 + 32);
  for (int row = r0 + warp; row < r1; row += nw) {
    double acc = 0.0;
    for (int j = lane; j < Nc; j += 32) acc += Ainv[(long long)row * Nc + j] * sr[j];
    acc = warp_sum(acc);
    if (lane == 0) x[off + row] = (T)acc;
  }
}

template <typename T>
cudaError_t launch_coarse_solve(const double* Ainv, int Nc, const T* r, T* x, const int* act, int nact,
                                cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  count_launch();
  k_coarse_solve<T><<<dim3((Nc + 31) / 32, nact), 256, Nc * sizeof(double), s>>>(Ainv, Nc, r, x, act);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// sources, right-hand sides, lift
// ---------------------------------------------------------------------------
// f_b = psi_i psi_j for pair b; pi[b] < 0 marks the Hartree density sum_k psi_k^2.
__global__ void k_pair_sources(const double* __restrict__ psi, int N, const int* __restrict__ pi,
                               const int* __restrict__ pj, long long Nq, double* __restrict__ f) {
  const int b = blockIdx.y;
  const int i = pi[b], j = pj[b];
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    double v;
    if (i < 0) {
      v = 0.0;
      for (int k = 0; k < N; ++k) {
        const double t = psi[(long long)k * Nq + q];
        v += t * t;
      }
    } else {
      v = psi[(long long)i * Nq + q] * psi[(long long)j * Nq + q];
    }
    f[(long long)b * Nq + q] = v;
  }
}

cudaError_t launch_pair_sources(const double* psi, int N, const int* pi, const int* pj, int nsrc, long long Nq,
                                double* f, cudaStream_t s) {
  if (nsrc == 0) return cudaSuccess;
  count_launch();
  k_pair_sources<<<vgrid(Nq, nsrc), VT, 0, s>>>(psi, N, pi, pj, Nq, f);
  return cudaGetLastError();
}

// out[b] = c A[ia[b]] B[ib[b]] pointwise; ia[b] < 0: c sum_k A_k^2 over the NA
// rows of A (the density). Sources of the trial-function solves and the
// Hartree action v_H u.
__global__ void k_row_products(const double* __restrict__ A, int NA, const double* __restrict__ B,
                               const int* __restrict__ ia, const int* __restrict__ ib, long long Nq, double c,
                               double* __restrict__ out) {
  const int b = blockIdx.y;
  const int i = ia[b], j = ib[b];
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    double v;
    if (i < 0) {
      v = 0.0;
      for (int k = 0; k < NA; ++k) {
        const double t = A[(long long)k * Nq + q];
        v += t * t;
      }
    } else {
      v = A[(long long)i * Nq + q] * B[(long long)j * Nq + q];
    }
    out[(long long)b * Nq + q] = c * v;
  }
}

cudaError_t launch_row_products(const double* A, int NA, const double* B, const int* ia, const int* ib, int n,
                                long long Nq, double c, double* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  count_launch();
  k_row_products<<<vgrid(Nq, n), VT, 0, s>>>(A, NA, B, ia, ib, Nq, c, out);
  return cudaGetLastError();
}

__global__ void k_scale(double* __restrict__ x, long long n, double c) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    x[q] *= c;
}

cudaError_t launch_scale(double* x, long long n, double c, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  count_launch();
  k_scale<<<vgrid(n, 1), VT, 0, s>>>(x, n, c);
  return cudaGetLastError();
}

__global__ void k_rhs_volume(const double* __restrict__ f, const double* __restrict__ W, double* __restrict__ b,
                             long long Nq) {
  const long long off = (long long)blockIdx.y * Nq;
  const double fourpi = 12.566370614359172953850573533118;  // 4 pi
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x)
    b[off + q] = fourpi * W[q] * f[off + q];
}

cudaError_t launch_rhs_volume(const double* f, const double* W, double* b, long long Nq, int nsrc, cudaStream_t s) {
  if (nsrc == 0) return cudaSuccess;
  count_launch();
  k_rhs_volume<<<vgrid(Nq, nsrc), VT, 0, s>>>(f, W, b, Nq);
  return cudaGetLastError();
}

__global__ void k_finite_flags(const double* __restrict__ f, long long Nq, int* __restrict__ flags) {
  const long long off = (long long)blockIdx.y * Nq;
  int bad = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(f[off + q]);
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicOr(&flags[blockIdx.y], 1);
}

cudaError_t launch_finite_flags(const double* f, long long Nq, int nsrc, int* flags, cudaStream_t s) {
  if (nsrc == 0) return cudaSuccess;
  count_launch();
  k_finite_flags<<<vgrid(Nq, nsrc), VT, 0, s>>>(f, Nq, flags);
  return cudaGetLastError();
}

// Nitsche load on one face: b[node] += lift_d[side][a_d] * M_t1 * M_t2 * g(t1, t2).
// g layout per source: faces -x,+x,-y,+y,-z,+z, each [L_t2][L_t1] (t1 fastest).
template <typename Tg>
__global__ void k_lift(const LevelOp* __restrict__ op, const Tg* __restrict__ g, double* __restrict__ b, int d,
                       int side, long long face_off, long long gstride) {
  const int n1 = op->n1, npe = n1 * n1 * n1;
  const int t1ax = d == 0 ? 1 : 0, t2ax = d == 2 ? 1 : 2;
  const int L1 = op->n[t1ax] * n1, L2 = op->n[t2ax] * n1;
  const long long total = (long long)L1 * L2 * n1;
  const long long src = blockIdx.y;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int ad = (int)(t % n1);
    const long long tt = t / n1;
    const int T1 = (int)(tt % L1), T2 = (int)(tt / L1);
    const int e1 = T1 / n1, a1 = T1 % n1, e2 = T2 / n1, a2 = T2 % n1;
    const int ed = side == 0 ? 0 : op->n[d] - 1;
    int ec[3], lc[3];
    ec[d] = ed;
    lc[d] = ad;
    ec[t1ax] = e1;
    lc[t1ax] = a1;
    ec[t2ax] = e2;
    lc[t2ax] = a2;
    const long long e = ec[0] + (long long)op->n[0] * (ec[1] + (long long)op->n[1] * ec[2]);
    const int loc = lc[0] + n1 * (lc[1] + n1 * lc[2]);
    const double coef = op->ax[d].lift[side][ad] * op->ax[t1ax].m[a1] * op->ax[t2ax].m[a2];
    const double gv = (double)g[src * gstride + face_off + T1 + (long long)L1 * T2];
    b[src * op->Nq + e * npe + loc] += coef * gv;
  }
}

template <typename Tg>
cudaError_t launch_lift(const LevelOp& hop, const LevelOp* dop, const Tg* g, double* b, int nsrc,
                        long long gstride, cudaStream_t s) {
  if (nsrc == 0) return cudaSuccess;
  long long off = 0;
  for (int d = 0; d < 3; ++d) {
    const int t1ax = d == 0 ? 1 : 0, t2ax = d == 2 ? 1 : 2;
    const long long L1 = (long long)hop.n[t1ax] * hop.n1, L2 = (long long)hop.n[t2ax] * hop.n1;
    for (int side = 0; side < 2; ++side) {
      // faces are launched one after another: nodes of edges and corners get
      // one contribution per face without races
      count_launch();
      k_lift<Tg><<<vgrid(L1 * L2 * hop.n1, nsrc), VT, 0, s>>>(dop, g, b, d, side, off, gstride);
      off += L1 * L2;
    }
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exchange accumulation W_m += sum_{(b, s) in list(m)} psi_s v_b (fixed order)
// ---------------------------------------------------------------------------
__global__ void k_exch_accum(const double* __restrict__ psi, const double* __restrict__ v, double* __restrict__ Wacc,
                             const int* __restrict__ ptr, const int* __restrict__ eb, const int* __restrict__ es,
                             long long Nq) {
  const int m = blockIdx.y;
  const int lo = ptr[m], hi = ptr[m + 1];
  if (lo == hi) return;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    double acc = Wacc[(long long)m * Nq + q];
    for (int t = lo; t < hi; ++t) acc += psi[(long long)es[t] * Nq + q] * v[(long long)eb[t] * Nq + q];
    Wacc[(long long)m * Nq + q] = acc;
  }
}

cudaError_t launch_exch_accum(const double* psi, const double* v, double* Wacc, const int* ptr, const int* eb,
                              const int* es, int N, long long Nq, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  count_launch();
  k_exch_accum<<<vgrid(Nq, N), VT, 0, s>>>(psi, v, Wacc, ptr, eb, es, Nq);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K = Psi diag(W) Wacc^T : partial sums over node chunks, then a fixed-order sum
// ---------------------------------------------------------------------------
static constexpr int KT = 32;   // output tile (KT x KT), 256 threads x 4 outputs
static constexpr int KQ = 64;   // nodes per shared-memory stage

int kmat_chunks(long long Nq) {
  long long c = (Nq + 1023) / 1024;
  if (c > 2048) c = 2048;
  return (int)(c < 1 ? 1 : c);
}

__global__ void k_kmat_partial(const double* __restrict__ psi, const double* __restrict__ W,
                               const double* __restrict__ Wacc, int N, long long Nq, double* __restrict__ part) {
  __shared__ double sa[KQ][KT + 1];
  __shared__ double sb[KQ][KT + 1];
  const int ti = blockIdx.x * KT, tj = blockIdx.y * KT;
  const int nchunk = gridDim.z;
  const long long per = (Nq + nchunk - 1) / nchunk;
  const long long q0 = (long long)blockIdx.z * per;
  const long long q1 = q0 + per < Nq ? q0 + per : Nq;
  const int tx = threadIdx.x % KT, ty = threadIdx.x / KT;  // ty in [0, 8)
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long qs = q0; qs < q1; qs += KQ) {
    for (int t = threadIdx.x; t < KQ * KT; t += blockDim.x) {
      const int qq = t % KQ, r = t / KQ;
      const long long q = qs + qq;
      const int i = ti + r, j = tj + r;
      sa[qq][r] = (q < q1 && i < N) ? psi[(long long)i * Nq + q] * W[q] : 0.0;
      sb[qq][r] = (q < q1 && j < N) ? Wacc[(long long)j * Nq + q] : 0.0;
    }
    __syncthreads();
    for (int qq = 0; qq < KQ; ++qq) {
      const double bj = sb[qq][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] += sa[qq][ty + 8 * r] * bj;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ti + ty + 8 * r, j = tj + tx;
    if (i < N && j < N) part[((long long)blockIdx.z * N + i) * N + j] = acc[r];
  }
}

__global__ void k_kmat_reduce(const double* __restrict__ part, int N, int nchunk, double* __restrict__ K) {
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= N * N) return;
  double acc = 0.0;
  for (int c = 0; c < nchunk; ++c) acc += part[(long long)c * N * N + ij];
  K[ij] = acc;
}

cudaError_t launch_kmat(const double* psi, const double* W, const double* Wacc, int N, long long Nq, double* part,
                        int nchunk, double* K, cudaStream_t s) {
  const int tiles = (N + KT - 1) / KT;
  count_launch();
  k_kmat_partial<<<dim3(tiles, tiles, nchunk), 256, 0, s>>>(psi, W, Wacc, N, Nq, part);
  count_launch();
  k_kmat_reduce<<<(N * N + 255) / 256, 256, 0, s>>>(part, N, nchunk, K);
  return cudaGetLastError();
}

// explicit instantiations
#define INST_T(T)                                                                                              \
  template cudaError_t launch_cheb_first<T>(T*, T*, const T*, const T*, double, int, long long, const int*, int, \
                                            cudaStream_t);                                                     \
  template cudaError_t launch_cheb_step<T>(T*, T*, const T*, const T*, double, double, long long, const int*,   \
                                           int, cudaStream_t);                                                 \
  template cudaError_t launch_cg_xr<T>(T*, T*, const T*, const T*, const double*, long long, const int*, int,    \
                                       cudaStream_t);                                                          \
  template cudaError_t launch_cg_p<T>(T*, const T*, const double*, long long, const int*, int, cudaStream_t);    \
  template cudaError_t launch_dot<T>(const T*, const T*, const double*, double*, double*, long long, const int*, \
                                     int, cudaStream_t);                                                       \
  template cudaError_t launch_zero<T>(T*, long long, const int*, int, cudaStream_t);                             \
  template cudaError_t launch_prolong_add<T>(const TransferOp&, const TransferOp*, const LevelOp&,              \
                                             const LevelOp&, const T*, T*, const int*, int, cudaStream_t);     \
  template cudaError_t launch_restrict<T>(const TransferOp&, const TransferOp*, const LevelOp&, const LevelOp&, \
                                          const T*, T*, const int*, int, cudaStream_t);                        \
  template cudaError_t launch_coarse_solve<T>(const double*, int, const T*, T*, const int*, int, cudaStream_t);
INST_T(double)
INST_T(float)
template cudaError_t launch_convert<double, float>(double*, const float*, long long, const int*, int, double, int,
                                                   cudaStream_t);
template cudaError_t launch_convert<float, double>(float*, const double*, long long, const int*, int, double, int,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, double>(double*, const double*, long long, const int*, int, double, int,
                                                    cudaStream_t);
template cudaError_t launch_lift<double>(const LevelOp&, const LevelOp*, const double*, double*, int, long long,
                                         cudaStream_t);
template cudaError_t launch_lift<float>(const LevelOp&, const LevelOp*, const float*, double*, int, long long,
                                        cudaStream_t);
template cudaError_t launch_convert<float, float>(float*, const float*, long long, const int*, int, double, int,
                                                  cudaStream_t);

}  // namespace dg
