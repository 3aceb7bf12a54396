// Matrix-free SIPDG operator (Sec. 3.4 eq. sip_bilinear with the penalty of
// Sec. 3.5 and Nitsche boundary faces) on the element-blocked layout.
//
// One work item = one element of one right-hand side. For element e the
// kernel needs its own (p+1)^3 values and, for each of its six faces, the
// neighbour's trace and reference normal derivative on that face (2 (p+1)^2
// numbers per face): the off-diagonal blocks of the 1-D operator are rank 2.
// Output node (a, b, c):
//   (Au) = My_b Mz_c [sum_i Kx[a,i] u_ibc + cL.x(-x traces) + cR.x(+x traces)]
//        + Mx_a Mz_c [ ... y ... ] + Mx_a My_b [ ... z ... ]
// with Kx the element's diagonal block (volume term plus its own face terms,
// Nitsche terms on boundary faces).
#include "dg_internal.h"

namespace dg {


// Launch layout: EPB elements per block; in the three 1-D passes each thread
// owns LPT lines of one element (line values in registers, the 1-D block rows
// streamed from shared memory and reused across the lines). Loads of the
// element, the neighbour traces and the final store are spread over all
// threads of the block and coalesced.
// Tuning constants (compile-time; the defaults were chosen by timing on a GB300)
#ifndef DG_APPLY_LPT32
#define DG_APPLY_LPT32 2      // lines per thread, FP32
#endif
#ifndef DG_APPLY_THREADS
#define DG_APPLY_THREADS 256  // threads per block (at least)
#endif
#ifndef DG_APPLY_SMEM
#define DG_APPLY_SMEM 38912   // shared-memory budget of the element slots (bytes)
#endif
#ifndef DG_SMEM_CARVEOUT
#define DG_SMEM_CARVEOUT -1  // shared-memory carveout (percent) asked for the operator and patch kernels; -1: default
#endif
#ifndef DG_APPLY_MINB32
#define DG_APPLY_MINB32 4     // resident blocks per SM asked of ptxas, FP32
#endif
// Element values in shared memory: node (a, b, c) at a + PB b + PB N1 c. With
// an even N1 the rows are padded by one (PB = N1 + 1), so that the x-pass's
// threads, which own consecutive x-lines, fall on different banks.
template <int N1>
struct ApplyPad {
  static constexpr int PB = N1 % 2 == 0 ? N1 + 1 : N1;
  static constexpr int PNPE = PB * N1 * N1;
  // shared-memory index of the element-local node loc = a + N1 b + N1^2 c
  __device__ static __forceinline__ int idx(int loc) { return loc + (PB - N1) * (loc / N1); }
};

template <typename T, int N1>
struct ApplyCfg {
  static constexpr int NPE = N1 * N1 * N1;
  static constexpr int NF = N1 * N1;
  static constexpr int PNPE = ApplyPad<N1>::PNPE;
  static constexpr int LPT = sizeof(T) == 4 ? DG_APPLY_LPT32 : 1;
  static constexpr int TPE = (NF + LPT - 1) / LPT;
  static constexpr int PER_ELEM = (2 * PNPE + 12 * NF + 3) * (int)sizeof(T);
  static constexpr int EPB_T = DG_APPLY_THREADS / TPE < 1 ? 1 : DG_APPLY_THREADS / TPE;
  static constexpr int EPB_S = DG_APPLY_SMEM / PER_ELEM < 1 ? 1 : DG_APPLY_SMEM / PER_ELEM;
  static constexpr int EPB = EPB_T < EPB_S ? EPB_T : EPB_S;
  // the load and trace phases use every thread of the block; the line passes
  // use the first EPB * TPE
  static constexpr int THREADS = EPB * TPE < DG_APPLY_THREADS ? DG_APPLY_THREADS : EPB * TPE;
  // resident blocks per SM asked of ptxas (p = 8 keeps 3: at 4 its registers spill)
  static constexpr int MINB = sizeof(T) == 4 ? (N1 >= 9 ? 3 : DG_APPLY_MINB32) : 2;
};

// one direction of the operator for LPT lines of one element:
// sacc[line] (+)= m1 * m2 * (K_ty v + cLv tv- + cLd td- + cRv tv+ + cRd td+)
template <typename T, int N1, int LPT, int TPE, int DIR, bool ACCUM>
__device__ __forceinline__ void ap_pass(const T* __restrict__ su, T* __restrict__ sacc, const T* __restrict__ K,
                                        const T* __restrict__ cc, const T* __restrict__ tr,
                                        const T* __restrict__ mA, const T* __restrict__ mB, int lt) {
  constexpr int NF = N1 * N1;
  constexpr int PB = ApplyPad<N1>::PB;
  constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? PB : PB * N1);
  T v[LPT][N1];
  int base[LPT], tt[LPT];
  bool ok[LPT];
  T scale[LPT], tvm[LPT], tdm[LPT], tvp[LPT], tdp[LPT];
#pragma unroll
  for (int s = 0; s < LPT; ++s) {
    const int l = lt + TPE * s;
    ok[s] = l < NF;
    const int l1 = ok[s] ? l % N1 : 0, l2 = ok[s] ? l / N1 : 0;
    // line (l1, l2) = (b, c) for x, (a, c) for y, (a, b) for z
    base[s] = DIR == 0 ? PB * l1 + PB * N1 * l2 : (DIR == 1 ? l1 + PB * N1 * l2 : l1 + PB * l2);
    tt[s] = l1 + N1 * l2;
    scale[s] = mA[l1] * mB[l2];
    tvm[s] = tr[(0 * 2 + 0) * NF + tt[s]];
    tdm[s] = tr[(0 * 2 + 1) * NF + tt[s]];
    tvp[s] = tr[(1 * 2 + 0) * NF + tt[s]];
    tdp[s] = tr[(1 * 2 + 1) * NF + tt[s]];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[s][i] = su[base[s] + i * stride];
  }
#pragma unroll 1
  for (int a = 0; a < N1; ++a) {
    T acc[LPT];
    const T c0 = cc[0 * N1 + a], c1 = cc[1 * N1 + a], c2 = cc[2 * N1 + a], c3 = cc[3 * N1 + a];
#pragma unroll
    for (int s = 0; s < LPT; ++s) acc[s] = c0 * tvm[s] + c1 * tdm[s] + c2 * tvp[s] + c3 * tdp[s];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      const T kv = K[a * N1 + i];
#pragma unroll
      for (int s = 0; s < LPT; ++s) acc[s] += kv * v[s][i];
    }
#pragma unroll
    for (int s = 0; s < LPT; ++s)
      if (ok[s]) {
        T* dst = sacc + base[s] + a * stride;
        if (ACCUM)
          *dst += scale[s] * acc[s];
        else
          *dst = scale[s] * acc[s];
      }
  }
}

// Traces (value and reference normal derivative) of the neighbours across the
// two faces of direction D of every slot: st[sl][2 D + side][0 / 1][tt].
template <typename T, int N1, int EPB, int NT, int D>
__device__ __forceinline__ void ap_traces(const T* __restrict__ u, const long long* sbase, const int (*snb)[6],
                                          const T (*sTr)[N1], T* __restrict__ st, int tid) {
  constexpr int NF = N1 * N1, NE = EPB * 2 * NF;
  constexpr int SD = D == 0 ? 1 : (D == 1 ? N1 : NF);
#pragma unroll 1
  for (int t = tid; t < NE; t += NT) {
    const int sl = t / (2 * NF), rem = t % (2 * NF), side = rem / NF, tt = rem % NF;
    const long long b0 = sbase[sl];
    const int nb = snb[sl][2 * D + side];
    T val = 0, der = 0;
    if (b0 >= 0 && nb != 0) {
      const int t1 = tt % N1, t2 = tt / N1;
      const int base = D == 0 ? N1 * t1 + NF * t2 : (D == 1 ? t1 + NF * t2 : t1 + N1 * t2);
      const T* un = u + b0 + (long long)nb * (N1 * NF) + base;
      T vals[N1];
      // an x-line is N1 contiguous values: with N1 * sizeof(T) a multiple of 16
      // bytes (and the field 16-byte aligned, as the library's are) it is read
      // with 16-byte loads, so that a warp's load touches each sector once
      constexpr bool VEC = D == 0 && (N1 * (int)sizeof(T)) % 16 == 0;
      if (VEC && (reinterpret_cast<uintptr_t>(un) & 15) == 0) {
        const uint4* p4 = reinterpret_cast<const uint4*>(un);
#pragma unroll
        for (int w = 0; w < (N1 * (int)sizeof(T)) / 16; ++w) {
          const uint4 q = __ldg(p4 + w);
          if constexpr (sizeof(T) == 4) {
            vals[4 * w] = __uint_as_float(q.x);
            vals[4 * w + 1] = __uint_as_float(q.y);
            vals[4 * w + 2] = __uint_as_float(q.z);
            vals[4 * w + 3] = __uint_as_float(q.w);
          } else {
            vals[2 * w] = __hiloint2double((int)q.y, (int)q.x);
            vals[2 * w + 1] = __hiloint2double((int)q.w, (int)q.z);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < N1; ++i) vals[i] = un[i * SD];
      }
      // the -d neighbour meets us at its right end, the +d neighbour at its left end
      const T* tv = side == 0 ? sTr[1] : sTr[0];
      const T* td = side == 0 ? sTr[3] : sTr[2];
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        val += tv[i] * vals[i];
        der += td[i] * vals[i];
      }
    }
    T* dst = st + ((sl * 6 + 2 * D + side) * 2) * NF + tt;
    dst[0] = val;
    dst[NF] = der;
  }
}

template <typename T, int N1, int MODE>
__global__ void __launch_bounds__(ApplyCfg<T, N1>::THREADS, ApplyCfg<T, N1>::MINB)
    k_apply(const LevelOp* __restrict__ op, const T* __restrict__ u, T* __restrict__ out,
            const T* __restrict__ rin, const int* __restrict__ act, int nact) {
  using C = ApplyCfg<T, N1>;
  constexpr int NPE = C::NPE, NF = C::NF, EPB = C::EPB, NT = C::THREADS, TPE = C::TPE, LPT = C::LPT;
  __shared__ T sK[3][4][NF];
  __shared__ T sC[3][4][N1];
  __shared__ T sM[3][N1];
  __shared__ T sTr[4][N1];
  __shared__ T su[EPB][C::PNPE];
  __shared__ T sacc[EPB][C::PNPE];
  __shared__ T st[EPB][6][2][NF];
  __shared__ long long sbase[EPB];  // rhs * Nq + e * NPE of the slot, or -1
  __shared__ int snb[EPB][6];       // neighbour element offset (elements) per face, 0 = none
  __shared__ int sty[EPB][3];

  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * 4 * NF; i += NT) {
    const int d = i / (4 * NF), r = i % (4 * NF);
    sK[d][r / NF][r % NF] = (T)op->ax[d].Kd[r / NF][r % NF];
  }
  for (int i = tid; i < 3 * N1; i += NT) {
    const int d = i / N1, a = i % N1;
    sC[d][0][a] = (T)op->ax[d].cLv[a];
    sC[d][1][a] = (T)op->ax[d].cLd[a];
    sC[d][2][a] = (T)op->ax[d].cRv[a];
    sC[d][3][a] = (T)op->ax[d].cRd[a];
    sM[d][a] = (T)op->ax[d].m[a];
  }
  for (int i = tid; i < N1; i += NT) {
    sTr[0][i] = (T)op->tl[i];
    sTr[1][i] = (T)op->tr[i];
    sTr[2][i] = (T)op->dl[i];
    sTr[3][i] = (T)op->dr[i];
  }
  const int nx = op->n[0], ny = op->n[1], nz = op->n[2];
  const int E = op->E;
  const long long Nq = op->Nq;
  const int slot = tid / TPE, lt = tid % TPE;
  const long long items = (long long)nact * E;
  const long long groups = (items + EPB - 1) / EPB;
  for (long long grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    __syncthreads();  // tables ready / previous group done with the shared buffers
    for (int sl = tid; sl < EPB; sl += NT) {
      const long long it = grp * EPB + sl;
      if (it < items) {
        const int k = (int)(it / E), e = (int)(it - (long long)k * E);
        sbase[sl] = (long long)act[k] * Nq + (long long)e * NPE;
        const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
        snb[sl][0] = ex > 0 ? -1 : 0;
        snb[sl][1] = ex < nx - 1 ? 1 : 0;
        snb[sl][2] = ey > 0 ? -nx : 0;
        snb[sl][3] = ey < ny - 1 ? nx : 0;
        snb[sl][4] = ez > 0 ? -nx * ny : 0;
        snb[sl][5] = ez < nz - 1 ? nx * ny : 0;
        sty[sl][0] = (ex == 0 ? 1 : 0) | (ex == nx - 1 ? 2 : 0);
        sty[sl][1] = (ey == 0 ? 1 : 0) | (ey == ny - 1 ? 2 : 0);
        sty[sl][2] = (ez == 0 ? 1 : 0) | (ez == nz - 1 ? 2 : 0);
      } else {
        sbase[sl] = -1;
        for (int f = 0; f < 6; ++f) snb[sl][f] = 0;
        sty[sl][0] = sty[sl][1] = sty[sl][2] = 0;
      }
    }
    __syncthreads();
    // own elements (coalesced over consecutive items)
    for (int t = tid; t < EPB * NPE; t += NT) {
      const int sl = t / NPE, loc = t - sl * NPE;
      const long long b0 = sbase[sl];
      su[sl][ApplyPad<N1>::idx(loc)] = b0 >= 0 ? u[b0 + loc] : (T)0;
    }
    // neighbour traces: face f = 2 d + side (side 0: -d neighbour, side 1: +d),
    // one direction at a time so that the line stride is a constant
    ap_traces<T, N1, EPB, NT, 0>(u, sbase, snb, sTr, &st[0][0][0][0], tid);
    ap_traces<T, N1, EPB, NT, 1>(u, sbase, snb, sTr, &st[0][0][0][0], tid);
    ap_traces<T, N1, EPB, NT, 2>(u, sbase, snb, sTr, &st[0][0][0][0], tid);
    __syncthreads();
    if (slot < EPB) {
      ap_pass<T, N1, LPT, TPE, 0, false>(su[slot], sacc[slot], sK[0][sty[slot][0]], sC[0][0], &st[slot][0][0][0],
                                         sM[1], sM[2], lt);
    }
    __syncthreads();
    if (slot < EPB) {
      ap_pass<T, N1, LPT, TPE, 1, true>(su[slot], sacc[slot], sK[1][sty[slot][1]], sC[1][0], &st[slot][2][0][0],
                                        sM[0], sM[2], lt);
    }
    __syncthreads();
    if (slot < EPB) {
      ap_pass<T, N1, LPT, TPE, 2, true>(su[slot], sacc[slot], sK[2][sty[slot][2]], sC[2][0], &st[slot][4][0][0],
                                        sM[0], sM[1], lt);
    }
    __syncthreads();
    for (int t = tid; t < EPB * NPE; t += NT) {
      const int sl = t / NPE, loc = t - sl * NPE;
      const long long b0 = sbase[sl];
      if (b0 >= 0) {
        const long long gi = b0 + loc;
        const T Au = sacc[sl][ApplyPad<N1>::idx(loc)];
        if (MODE == 0) {
          out[gi] = Au;
        } else if (MODE == 1) {
          out[gi] = rin[gi] - Au;
        } else {
          out[gi] = out[gi] - Au;
        }
      }
    }
  }
}

template <typename T, int N1>
static cudaError_t apply_n1(const LevelOp& hop, const LevelOp* dop, int mode, const T* u, T* out, const T* rin,
                            const int* act, int nact, cudaStream_t s) {
  using C = ApplyCfg<T, N1>;
  const long long items = (long long)nact * hop.E;
  long long blocks = (items + C::EPB - 1) / C::EPB;
  if (blocks == 0) return cudaSuccess;
  // persistent-style grid: a few resident blocks per SM loop over element groups
  const long long cap = 152LL * (2048 / C::THREADS) * 2;
  if (blocks > cap) blocks = cap;
#if DG_SMEM_CARVEOUT >= 0
  static bool carve = false;  // ask for the largest shared-memory carveout (more resident blocks)
  if (!carve) {
    cudaFuncSetAttribute(k_apply<T, N1, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, DG_SMEM_CARVEOUT);
    cudaFuncSetAttribute(k_apply<T, N1, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, DG_SMEM_CARVEOUT);
    cudaFuncSetAttribute(k_apply<T, N1, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, DG_SMEM_CARVEOUT);
    carve = true;
  }
#endif
  count_launch();
  if (mode == 0)
    k_apply<T, N1, 0><<<(unsigned)blocks, C::THREADS, 0, s>>>(dop, u, out, rin, act, nact);
  else if (mode == 1)
    k_apply<T, N1, 1><<<(unsigned)blocks, C::THREADS, 0, s>>>(dop, u, out, rin, act, nact);
  else
    k_apply<T, N1, 2><<<(unsigned)blocks, C::THREADS, 0, s>>>(dop, u, out, rin, act, nact);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const LevelOp& hop, const LevelOp* dop, int mode, const T* u, T* out, const T* rin,
                         const int* act, int nact, cudaStream_t s) {
  switch (hop.n1) {
    case 2: return apply_n1<T, 2>(hop, dop, mode, u, out, rin, act, nact, s);
    case 3: return apply_n1<T, 3>(hop, dop, mode, u, out, rin, act, nact, s);
    case 4: return apply_n1<T, 4>(hop, dop, mode, u, out, rin, act, nact, s);
    case 5: return apply_n1<T, 5>(hop, dop, mode, u, out, rin, act, nact, s);
    case 6: return apply_n1<T, 6>(hop, dop, mode, u, out, rin, act, nact, s);
    case 7: return apply_n1<T, 7>(hop, dop, mode, u, out, rin, act, nact, s);
    case 8: return apply_n1<T, 8>(hop, dop, mode, u, out, rin, act, nact, s);
    case 9: return apply_n1<T, 9>(hop, dop, mode, u, out, rin, act, nact, s);
    default: return cudaErrorInvalidValue;
  }
}

// Jacobi diagonal of the Kronecker sum: Kx[a,a] My Mz + Mx Ky[b,b] Mz + Mx My Kz[c,c].
template <typename T>
__global__ void k_inv_diag(const LevelOp* __restrict__ op, T* __restrict__ invD) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= op->Nq) return;
  const int n1 = op->n1, npe = n1 * n1 * n1;
  const int e = (int)(i / npe), loc = (int)(i % npe);
  const int a = loc % n1, b = (loc / n1) % n1, c = loc / (n1 * n1);
  const int nx = op->n[0], ny = op->n[1], nz = op->n[2];
  const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
  const int tyx = (ex == 0 ? 1 : 0) | (ex == nx - 1 ? 2 : 0);
  const int tyy = (ey == 0 ? 1 : 0) | (ey == ny - 1 ? 2 : 0);
  const int tyz = (ez == 0 ? 1 : 0) | (ez == nz - 1 ? 2 : 0);
  const double mx = op->ax[0].m[a], my = op->ax[1].m[b], mz = op->ax[2].m[c];
  const double dval = op->ax[0].Kd[tyx][a * n1 + a] * my * mz + mx * op->ax[1].Kd[tyy][b * n1 + b] * mz +
                      mx * my * op->ax[2].Kd[tyz][c * n1 + c];
  invD[i] = (T)(1.0 / dval);
}

template <typename T>
cudaError_t launch_inv_diag(const LevelOp& hop, const LevelOp* dop, T* invD, cudaStream_t s) {
  const long long n = hop.Nq;
  count_launch();
  k_inv_diag<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dop, invD);
  return cudaGetLastError();
}

template cudaError_t launch_apply<double>(const LevelOp&, const LevelOp*, int, const double*, double*,
                                          const double*, const int*, int, cudaStream_t);
template cudaError_t launch_apply<float>(const LevelOp&, const LevelOp*, int, const float*, float*, const float*,
                                         const int*, int, cudaStream_t);
template cudaError_t launch_inv_diag<double>(const LevelOp&, const LevelOp*, double*, cudaStream_t);
template cudaError_t launch_inv_diag<float>(const LevelOp&, const LevelOp*, float*, cudaStream_t);

}  // namespace dg
