// Dirichlet data of the auxiliary-grid Poisson problems (Sec. 6.3):
//     g(x_b) = sum_q W_q f(x_q) / |x_b - x_q|
// at every Gauss-Legendre node of the six boundary faces.
//
// Route DIRECT evaluates that sum as written (FP64, O(N_faces N_q) per source).
// Route GAUSSSUM replaces 1/r by sum_k c_k exp(-alpha_k r^2) (the separable
// Gaussian-sum approximation of Sec. 5.2), so that, on the tensor grid of
// nodes, the sum for the faces normal to axis d factorises into three 1-D
// contractions per term: along d with the face position, then along the two
// tangential axes. Those contractions run as strided batched GEMMs (k_gemm).
#include <algorithm>

#include "dg_internal.h"

namespace dg {

// Flex[src][X + Lx (Y + Ly Z)] = W_q f_src(q): element-blocked -> global lexicographic.
template <typename T>
__global__ void k_weighted_lex(const LevelOp* __restrict__ op, const double* __restrict__ f,
                               const double* __restrict__ W, T* __restrict__ flex) {
  const long long Nq = op->Nq;
  const int n1 = op->n1, npe = n1 * n1 * n1;
  const int nx = op->n[0], ny = op->n[1];
  const long long Lx = (long long)nx * n1, Ly = (long long)ny * n1;
  const long long src = blockIdx.y;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(q / npe), loc = (int)(q % npe);
    const int a = loc % n1, b = (loc / n1) % n1, c = loc / (n1 * n1);
    const long long X = (long long)(e % nx) * n1 + a;
    const long long Y = (long long)((e / nx) % ny) * n1 + b;
    const long long Z = (long long)(e / (nx * ny)) * n1 + c;
    flex[src * Nq + X + Lx * (Y + Ly * Z)] = (T)(W[q] * f[src * Nq + q]);
  }
}

template <typename T>
cudaError_t launch_weighted_lex(const LevelOp& hop, const LevelOp* dop, const double* f, const double* W, T* flex,
                                int nsrc, cudaStream_t s) {
  if (nsrc == 0) return cudaSuccess;
  long long gx = (hop.Nq + 1023) / 1024;
  if (gx > 4096) gx = 4096;
  count_launch();
  k_weighted_lex<T><<<dim3((unsigned)gx, nsrc), 256, 0, s>>>(dop, f, W, flex);
  return cudaGetLastError();
}
template cudaError_t launch_weighted_lex<double>(const LevelOp&, const LevelOp*, const double*, const double*,
                                                 double*, int, cudaStream_t);
template cudaError_t launch_weighted_lex<float>(const LevelOp&, const LevelOp*, const double*, const double*, float*,
                                                int, cudaStream_t);

// ---------------------------------------------------------------------------
// Strided batched GEMM: C[m,n] = alpha sum_k A[m,k] B[k,n] + beta C[m,n]
// with arbitrary element strides and a two-level batch index.
// 64 x 64 output tile, K step 16, 256 threads with 4 x 4 outputs each.
// ---------------------------------------------------------------------------
// (FP64 instances; FP32 runs on the tensor cores in k_gemm_tc below.)
// FP32 instances keep a compensated running sum across K tiles: each 16-term
// tile is accumulated in registers and then added to (sum, carry) with
// Knuth's TwoSum, so the error does not grow with K (K reaches N_G L ~ 10^4 in
// the boundary-data contractions).
template <typename T>
__device__ __forceinline__ void two_sum_add(T& s, T& c, T a) {
  const T t = s + a;
  const T bp = t - s;
  c += (s - (t - bp)) + (a - bp);
  s = t;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs g, int batch_base) {
  constexpr bool COMP = sizeof(T) == 4;
  __shared__ T sA[16][64 + 1];
  __shared__ T sB[16][64 + 1];
  const int bz = batch_base + blockIdx.z;
  const int b1 = bz / g.nb2, b2 = bz % g.nb2;
  const T* A = (const T*)g.A + b1 * g.sA1 + b2 * g.sA2;
  const T* B = (const T*)g.B + b1 * g.sB1 + b2 * g.sB2;
  T* C = (T*)g.C + b1 * g.sC1 + b2 * g.sC2;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const bool a_k_fast = g.sAk == 1;
  const bool b_n_fast = g.sBn == 1;
  T acc[4][4], sum[4][4], car[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = (T)0;
      sum[i][j] = (T)0;
      car[i][j] = (T)0;
    }
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    for (int t = tid; t < 64 * 16; t += 256) {
      int kk, mm;
      if (a_k_fast) {
        kk = t % 16;
        mm = t / 16;
      } else {
        mm = t % 64;
        kk = t / 64;
      }
      const int m = m0 + mm, k = k0 + kk;
      sA[kk][mm] = (m < g.M && k < g.K) ? A[(long long)m * g.sAm + (long long)k * g.sAk] : (T)0;
      int nn, kb;
      if (b_n_fast) {
        nn = t % 64;
        kb = t / 64;
      } else {
        kb = t % 16;
        nn = t / 16;
      }
      const int n = n0 + nn, kx = k0 + kb;
      sB[kb][nn] = (n < g.N && kx < g.K) ? B[(long long)kx * g.sBk + (long long)n * g.sBn] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    if (COMP) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          two_sum_add(sum[i][j], car[i][j], acc[i][j]);
          acc[i][j] = (T)0;
        }
    }
    __syncthreads();
  }
  const T alpha = (T)g.alpha, beta = (T)g.beta;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      const T v = COMP ? sum[i][j] + car[i][j] : acc[i][j];
      T* cp = C + (long long)m * g.sCm + (long long)n * g.sCn;
      *cp = g.beta != 0.0 ? alpha * v + beta * (*cp) : alpha * v;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 strided batched GEMM on the tensor cores: mma.sync m16n8k8 TF32 with
// the 3xTF32 split (a = a_hi + a_lo, both TF32; a b ~ a_hi b_hi + a_hi b_lo +
// a_lo b_hi, error ~ 2^-22 of |a b|) and the same compensated accumulation
// across 16-term K tiles as k_gemm. 64 x 64 output tile, 4 warps of 32 x 32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int TCA = 20;  // padded row of the A tile (conflict-free fragment loads)
constexpr int TCB = 72;  // padded row of the B tile

// With nsplit > 1, block z covers batch (batch_base + z / nsplit) and the K
// range [kc (z % nsplit), kc (z % nsplit + 1)); its compensated partial sum goes
// to work[split][batch - batch_base][m][n] (nbc batches per launch) and
// k_gemm_splitk_reduce finishes C.
__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g, int batch_base, int nsplit, int kc, int nbc) {
  __shared__ unsigned sAh[64][TCA], sAl[64][TCA];
  __shared__ unsigned sBh[16][TCB], sBl[16][TCB];
  const int bz = batch_base + (int)blockIdx.z / nsplit;
  const int split = (int)blockIdx.z % nsplit;
  const int kbeg = split * kc, kend = min(g.K, kbeg + kc);
  const int b1 = bz / g.nb2, b2 = bz % g.nb2;
  const float* A = (const float*)g.A + b1 * g.sA1 + b2 * g.sA2;
  const float* B = (const float*)g.B + b1 * g.sB1 + b2 * g.sB2;
  float* C = (float*)g.C + b1 * g.sC1 + b2 * g.sC2;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, c4 = lane & 3;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const bool a_k_fast = g.sAk == 1;
  const bool b_n_fast = g.sBn == 1;
  float acc[2][4][4], sum[2][4][4], car[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[i][j][e] = 0.f;
        sum[i][j][e] = 0.f;
        car[i][j][e] = 0.f;
      }
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int t = tid; t < 64 * 16; t += 128) {
      int kk, mm;
      if (a_k_fast) {
        kk = t % 16;
        mm = t / 16;
      } else {
        mm = t % 64;
        kk = t / 64;
      }
      const int m = m0 + mm, k = k0 + kk;
      const float av = (m < g.M && k < kend) ? A[(long long)m * g.sAm + (long long)k * g.sAk] : 0.f;
      const unsigned ah = to_tf32(av);
      sAh[mm][kk] = ah;
      sAl[mm][kk] = to_tf32(av - __uint_as_float(ah));
      int nn, kb;
      if (b_n_fast) {
        nn = t % 64;
        kb = t / 64;
      } else {
        kb = t % 16;
        nn = t / 16;
      }
      const int n = n0 + nn, kx = k0 + kb;
      const float bv = (n < g.N && kx < kend) ? B[(long long)kx * g.sBk + (long long)n * g.sBn] : 0.f;
      const unsigned bh = to_tf32(bv);
      sBh[kb][nn] = bh;
      sBl[kb][nn] = to_tf32(bv - __uint_as_float(bh));
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 16; ks += 8) {
      unsigned ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gq;
        ah[i][0] = sAh[r][ks + c4];
        ah[i][1] = sAh[r + 8][ks + c4];
        ah[i][2] = sAh[r][ks + c4 + 4];
        ah[i][3] = sAh[r + 8][ks + c4 + 4];
        al[i][0] = sAl[r][ks + c4];
        al[i][1] = sAl[r + 8][ks + c4];
        al[i][2] = sAl[r][ks + c4 + 4];
        al[i][3] = sAl[r + 8][ks + c4 + 4];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gq;
        bh[j][0] = sBh[ks + c4][c];
        bh[j][1] = sBh[ks + c4 + 4][c];
        bl[j][0] = sBl[ks + c4][c];
        bl[j][1] = sBl[ks + c4 + 4][c];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          mma_tf32(acc[i][j], al[i], bh[j]);
          mma_tf32(acc[i][j], ah[i], bl[j]);
          mma_tf32(acc[i][j], ah[i], bh[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          two_sum_add(sum[i][j][e], car[i][j][e], acc[i][j][e]);
          acc[i][j][e] = 0.f;
        }
    __syncthreads();
  }
  const float alpha = (float)g.alpha, beta = (float)g.beta;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = m0 + wm + i * 16 + gq + (e >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * c4 + (e & 1);
        if (m >= g.M || n >= g.N) continue;
        const float v = sum[i][j][e] + car[i][j][e];
        if (nsplit > 1) {
          ((float*)g.work)[(((long long)split * nbc + (bz - batch_base)) * g.M + m) * g.N + n] = v;
          continue;
        }
        float* cp = C + (long long)m * g.sCm + (long long)n * g.sCn;
        *cp = g.beta != 0.0 ? alpha * v + beta * (*cp) : alpha * v;
      }
}

// C = alpha sum_split work[split] (+ beta C) for batches batch_base ..
// batch_base + nbc - 1, splits added in order with TwoSum
__global__ void k_gemm_splitk_reduce(GemmArgs g, int nsplit, int batch_base, int nbc) {
  const long long mn = (long long)g.M * g.N, total = (long long)nbc * mn;
  const float* w = (const float*)g.work;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float sum = 0.f, car = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) two_sum_add(sum, car, w[(long long)sp * total + i]);
    const long long bz = batch_base + i / mn, r = i % mn;
    const int m = (int)(r / g.N), n = (int)(r - (long long)m * g.N);
    const int b1 = (int)(bz / g.nb2), b2 = (int)(bz % g.nb2);
    float* cp = (float*)g.C + b1 * g.sC1 + b2 * g.sC2 + (long long)m * g.sCm + (long long)n * g.sCn;
    const float v = sum + car;
    *cp = g.beta != 0.0 ? (float)g.alpha * v + (float)g.beta * (*cp) : (float)g.alpha * v;
  }
}

template <typename T>
cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.nb1 * (long long)g.nb2 <= 0) return cudaSuccess;
  const long long nb = (long long)g.nb1 * g.nb2;
  const dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, 1);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    // a long K is split over blocks into fixed 512-term ranges (from K alone,
    // so a batch's sums do not depend on how many batches share the call);
    // batches go through in chunks that fit the workspace
    int nsplit = 1;
    if (g.work && g.K >= 1024) nsplit = std::min(32, (g.K + 511) / 512);
    const int kc = nsplit > 1 ? ((g.K + nsplit - 1) / nsplit + 15) / 16 * 16 : g.K;
    if (nsplit > 1) nsplit = (g.K + kc - 1) / kc;  // no empty split
    long long per = 65535 / nsplit;
    if (nsplit > 1) per = std::min<long long>(per, g.work_elems / ((long long)nsplit * g.M * g.N));
    if (per < 1) return cudaErrorInvalidValue;  // workspace too small for one batch
    for (long long base = 0; base < nb; base += per) {
      const long long cnt = nb - base < per ? nb - base : per;
      count_launch();
      k_gemm_tc<<<dim3(grid.x, grid.y, (unsigned)(cnt * nsplit)), 128, 0, s>>>(g, (int)base, nsplit, kc, (int)cnt);
      if (nsplit > 1) {
        count_launch();
        const long long total = cnt * g.M * g.N;
        k_gemm_splitk_reduce<<<(unsigned)std::min<long long>((total + 255) / 256, 152LL * 16), 256, 0, s>>>(
            g, nsplit, (int)base, (int)cnt);
      }
    }
  } else {
    for (long long base = 0; base < nb; base += 65535) {
      const long long cnt = nb - base < 65535 ? nb - base : 65535;
      count_launch();
      k_gemm<T><<<dim3(grid.x, grid.y, (unsigned)cnt), 256, 0, s>>>(g, (int)base);
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmArgs&, cudaStream_t);
template cudaError_t launch_gemm<float>(const GemmArgs&, cudaStream_t);

// ---------------------------------------------------------------------------
// Direct quadrature: one thread per face node, all volume nodes in tiles.
// ---------------------------------------------------------------------------
static constexpr int BCT = 128;

__global__ void __launch_bounds__(BCT) k_bc_direct(const LevelOp* __restrict__ op, const double* __restrict__ f,
                                                   const double* __restrict__ W, const double* __restrict__ xq,
                                                   const double* __restrict__ axn, int lmax,
                                                   double* __restrict__ g, long long gstride, long long nface) {
  __shared__ double sx[BCT], sy[BCT], sz[BCT], sf[BCT];
  const long long src = blockIdx.y;
  const long long Nq = op->Nq;
  const int n1 = op->n1;
  const long long t = (long long)blockIdx.x * BCT + threadIdx.x;
  // locate the face node
  double bx = 0, by = 0, bz = 0;
  if (t < nface) {
    long long rem = t;
    for (int d = 0; d < 3; ++d) {
      const int t1ax = d == 0 ? 1 : 0, t2ax = d == 2 ? 1 : 2;
      const long long L1 = (long long)op->n[t1ax] * n1, L2 = (long long)op->n[t2ax] * n1;
      for (int side = 0; side < 2; ++side) {
        if (rem >= 0 && rem < L1 * L2) {
          double c[3];
          c[d] = side == 0 ? op->ax[d].lo : op->ax[d].hi;
          c[t1ax] = axn[t1ax * lmax + (rem % L1)];
          c[t2ax] = axn[t2ax * lmax + (rem / L1)];
          bx = c[0];
          by = c[1];
          bz = c[2];
        }
        rem -= L1 * L2;
      }
    }
  }
  double acc = 0.0;
  for (long long q0 = 0; q0 < Nq; q0 += BCT) {
    const long long q = q0 + threadIdx.x;
    __syncthreads();
    if (q < Nq) {
      sx[threadIdx.x] = xq[3 * q];
      sy[threadIdx.x] = xq[3 * q + 1];
      sz[threadIdx.x] = xq[3 * q + 2];
      sf[threadIdx.x] = W[q] * f[src * Nq + q];
    } else {
      sx[threadIdx.x] = 1e300;
      sy[threadIdx.x] = 0.0;
      sz[threadIdx.x] = 0.0;
      sf[threadIdx.x] = 0.0;
    }
    __syncthreads();
    if (t < nface) {
#pragma unroll 4
      for (int j = 0; j < BCT; ++j) {
        const double dx = bx - sx[j], dy = by - sy[j], dz = bz - sz[j];
        acc += sf[j] / sqrt(dx * dx + dy * dy + dz * dz);
      }
    }
  }
  if (t < nface) g[src * gstride + t] = acc;
}

cudaError_t launch_bc_direct(const LevelOp& hop, const LevelOp* dop, const double* f, const double* W,
                             const double* xq, const double* axis_nodes, int lmax, double* g, int nsrc,
                             long long gstride, long long nface, cudaStream_t s) {
  if (nsrc == 0) return cudaSuccess;
  (void)hop;
  count_launch();
  k_bc_direct<<<dim3((unsigned)((nface + BCT - 1) / BCT), nsrc), BCT, 0, s>>>(dop, f, W, xq, axis_nodes, lmax, g,
                                                                           gstride, nface);
  return cudaGetLastError();
}

}  // namespace dg
