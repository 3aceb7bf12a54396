// Overlapping Schwarz smoother for the hp-multigrid of Sec. 6.4.
//
// The paper does not specify the smoother. With the penalty of Sec. 3.5
// (eps = 1/8, i.e. eight times the coercivity bound) point- and element-block
// Jacobi smoothers leave continuous high-order modes undamped, so each
// multigrid level uses additive Schwarz over element patches with one node of
// overlap, accelerated by Chebyshev iteration. Each patch problem is solved
// exactly by fast diagonalisation (the patch operator is a Kronecker sum of
// restricted 1-D matrices; tables built at setup):
//   k_schwarz_patch:  zp_e = A_P(e)^-1 R_P(e) r        (EPB elements per block,
//                     one thread per patch line in each of the six 1-D passes)
//   k_schwarz_gather: z = sum_e R_P(e)^T zp_e          (each node gathers the
//                     at most 8 patches covering it; no atomics), fused with
//                     the Chebyshev update d = c1 d + c2 z, x += d
#include "dg_internal.h"
#include "dg_swtc.h"

namespace dg {

__host__ __device__ inline int sw_axis_off(const LevelOp* op, int d, int stride) {
  return d == 0 ? 0 : (d == 1 ? op->n[0] * stride : (op->n[0] + op->n[1]) * stride);
}

// Patch kernel layout: each thread owns LPT = 3 lines of the patch in every
// 1-D pass (line values and outputs in registers, the 1-D matrix streamed from
// shared memory and reused across the three lines).
// Tuning constants (compile-time; the defaults were chosen by timing on a GB300)
#ifndef DG_SMEM_CARVEOUT
#define DG_SMEM_CARVEOUT -1  // shared-memory carveout (percent) asked for the patch kernel; -1: default
#endif
// patch lines per thread, FP32: 2 for p = 1 and p >= 7, 3 otherwise (timed per degree)
#ifdef DG_SW_LPT32
#define DG_SW_LPT_OF(N1) DG_SW_LPT32
#else
#define DG_SW_LPT_OF(N1) ((N1) == 2 || (N1) >= 8 ? 2 : 3)
#endif
#ifndef DG_GATHER_WAVE
#define DG_GATHER_WAVE 8   // gather grid: at most this many blocks per SM per source list (0: one block per element)
#endif
#ifndef DG_SW_MINB32
#define DG_SW_MINB32 4     // resident blocks per SM asked of ptxas, FP32
#endif
#ifndef DG_SW_THREADS
#define DG_SW_THREADS 256  // thread budget per block
#endif
#ifndef DG_SW_SMEM
#define DG_SW_SMEM 36864   // shared-memory budget of the patch slots (bytes)
#endif
// Padded FP32 patch layout in shared memory: node (i, j, k) of a patch at
// i + MP j + SY k, patch slots SE apart. The plane and slot strides were
// chosen by counting shared-memory wavefronts of the six 1-D passes for every
// degree (lanes of a warp on lines of one or two patches): the unpadded layout
// puts the y lines MP^2 words apart, a 2-way bank conflict for most MP.
__host__ __device__ constexpr int sw_pad_sy(int N1) {
  return N1 == 2 ? 16 : N1 == 3 ? 39 : N1 == 4 ? 39 : N1 == 6 ? 73 : N1 == 7 ? 85 : N1 == 8 ? 109
                                                                                   : (N1 + 2) * (N1 + 2);
}
__host__ __device__ constexpr int sw_pad_se(int N1) {
  return N1 == 2 ? 69 : N1 == 3 ? 201 : N1 == 4 ? 238 : N1 == 6 ? 598 : N1 == 7 ? 795 : N1 == 8 ? 1106
                                                      : N1 == 9 ? 1332 : (N1 + 2) * (N1 + 2) * (N1 + 2);
}

template <typename T, int N1>
struct SwCfg {
  static constexpr int MP = N1 + 2;
  // plane and slot strides of the shared patch buffer (FP64 keeps the dense layout)
  static constexpr int SY = sizeof(T) == 4 ? sw_pad_sy(N1) : MP * MP;
  static constexpr int SE = sizeof(T) == 4 ? sw_pad_se(N1) : MP * MP * MP;
  static_assert(SY >= MP * MP && SE >= MP * SY, "patch layout overlaps");
  static constexpr int LINES = MP * MP;
  // FP32: two or three lines per thread (shared-memory traffic per FMA / LPT);
  // FP64 is bound by the FP64 pipe, one line per thread keeps registers in check
  static constexpr int LPT = sizeof(T) == 4 ? DG_SW_LPT_OF(N1) : 1;
  static constexpr int TPE = (LINES + LPT - 1) / LPT;  // threads per element
  static constexpr int MINB = sizeof(T) == 4 ? DG_SW_MINB32 : 1;  // resident blocks per SM asked of ptxas
  static constexpr int PER_ELEM = (SE + 3 * MP * MP + 3 * MP) * (int)sizeof(T);
  static constexpr int EPB_T = DG_SW_THREADS / TPE < 1 ? 1 : DG_SW_THREADS / TPE;
  static constexpr int EPB_S = DG_SW_SMEM / PER_ELEM < 1 ? 1 : DG_SW_SMEM / PER_ELEM;
  static constexpr int EPB = EPB_T < EPB_S ? EPB_T : EPB_S;
  static constexpr int THREADS = EPB * TPE;
};

// One 1-D pass over the lines l = lt + TPE s (s < LPT) of one patch, node
// (i, j, k) at i + MP j + SY k. dir 0: x lines (j, k) stride 1; dir 1: y lines
// (i, k) stride MP; dir 2: z lines (i, j) stride SY. Forward: v[q] <- sum_i S[i][q] v[i]; backward:
// v[i] <- sum_q S[i][q] v[q].
template <typename T, int MP, int SY, int TPE, int LPT, int DIR, bool BACKWARD>
__device__ __forceinline__ void sw_pass3(T* __restrict__ buf, const T* __restrict__ S, int lt) {
  constexpr int MP2 = MP * MP;
  constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? MP : SY);
  int base[LPT];
  bool ok[LPT];
#pragma unroll
  for (int s = 0; s < LPT; ++s) {
    const int l = lt + TPE * s;
    ok[s] = l < MP2;
    const int l1 = l % MP, l2 = l / MP;
    base[s] = ok[s] ? (DIR == 0 ? l1 * MP + l2 * SY : (DIR == 1 ? l1 + SY * l2 : l1 + MP * l2)) : 0;
  }
  if (!BACKWARD) {
    // o[q] = sum_i S[i][q] v[i]: inputs streamed row by row, outputs in registers
    T o[LPT][MP];
#pragma unroll
    for (int s = 0; s < LPT; ++s)
#pragma unroll
      for (int q = 0; q < MP; ++q) o[s][q] = (T)0;
#pragma unroll 1
    for (int i = 0; i < MP; ++i) {
      T vi[LPT];
#pragma unroll
      for (int s = 0; s < LPT; ++s) vi[s] = buf[base[s] + i * stride];
#pragma unroll
      for (int q = 0; q < MP; ++q) {
        const T sv = S[i * MP + q];
#pragma unroll
        for (int s = 0; s < LPT; ++s) o[s][q] += sv * vi[s];
      }
    }
#pragma unroll
    for (int s = 0; s < LPT; ++s)
      if (ok[s]) {
#pragma unroll
        for (int q = 0; q < MP; ++q) buf[base[s] + q * stride] = o[s][q];
      }
  } else {
    // o[i] = sum_q S[i][q] v[q]: inputs in registers, IB outputs per line at
    // a time (LPT * IB independent sums in q order), each written when done
    constexpr int IB = MP % 3 == 0 ? 3 : 2;
    T v[LPT][MP];
#pragma unroll
    for (int s = 0; s < LPT; ++s)
#pragma unroll
      for (int q = 0; q < MP; ++q) v[s][q] = buf[base[s] + q * stride];
#pragma unroll 1
    for (int i0 = 0; i0 < MP; i0 += IB) {
      T acc[IB][LPT];
#pragma unroll
      for (int ib = 0; ib < IB; ++ib)
#pragma unroll
        for (int s = 0; s < LPT; ++s) acc[ib][s] = (T)0;
      const int nb = MP - i0 < IB ? MP - i0 : IB;
#pragma unroll
      for (int q = 0; q < MP; ++q) {
#pragma unroll
        for (int ib = 0; ib < IB; ++ib) {
          const T sv = ib < nb ? S[(i0 + ib) * MP + q] : (T)0;
#pragma unroll
          for (int s = 0; s < LPT; ++s) acc[ib][s] += sv * v[s][q];
        }
      }
#pragma unroll
      for (int ib = 0; ib < IB; ++ib)
        if (ib < nb) {
#pragma unroll
          for (int s = 0; s < LPT; ++s)
            if (ok[s]) buf[base[s] + (i0 + ib) * stride] = acc[ib][s];
        }
    }
  }
}

// Division by the patch eigenvalue sum: FP32 takes the fast approximate
// quotient (within 2 ulp; the sums are positive and far from the range
// limits), FP64 the exact one.
__device__ __forceinline__ float sw_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sw_div(double a, double b) { return a / b; }

template <typename T, int N1>
__global__ void __launch_bounds__(SwCfg<T, N1>::THREADS, SwCfg<T, N1>::MINB)
    k_schwarz_patch(const LevelOp* __restrict__ op, const double* __restrict__ tabs, const T* __restrict__ r,
                    T* __restrict__ zp, const int* __restrict__ act, int nact) {
  using C = SwCfg<T, N1>;
  constexpr int MP = C::MP, MP2 = MP * MP, MP3 = MP * MP * MP, NPE = N1 * N1 * N1, STR = 2 + MP2 + MP;
  constexpr int SY = C::SY, SE = C::SE;
  constexpr int EPB = C::EPB, NT = C::THREADS, TPE = C::TPE, LPT = C::LPT;
  __shared__ T sS[EPB][3][MP2];
  __shared__ T sL[EPB][3][MP];
  __shared__ T buf[EPB][SE];
  __shared__ int sm[EPB][3], soL[EPB][3];
  __shared__ int spos[EPB][4];  // element of each slot (-1: none) and its (x, y, z) position
  __shared__ long long srhs[EPB];
  const int nx = op->n[0], ny = op->n[1];
  const int E = op->E;
  const long long Nq = op->Nq;
  // the runtime divisions (item -> source, element -> position) once per slot
  if (threadIdx.x < EPB) {
    const long long it = (long long)blockIdx.x * EPB + threadIdx.x;
    const bool v = it < (long long)nact * E;
    const int ee = v ? (int)(it % E) : 0;
    spos[threadIdx.x][0] = v ? ee : -1;
    spos[threadIdx.x][1] = ee % nx;
    spos[threadIdx.x][2] = (ee / nx) % ny;
    spos[threadIdx.x][3] = ee / (nx * ny);
    srhs[threadIdx.x] = v ? act[it / E] : 0;
  }
  __syncthreads();
  const int slot = threadIdx.x / TPE, lt = threadIdx.x % TPE;
  const bool valid = spos[slot][0] >= 0;
  const int e = valid ? spos[slot][0] : 0;
  const long long rhs = srhs[slot];
  const int pos[3] = {spos[slot][1], spos[slot][2], spos[slot][3]};
  // patch tables of the EPB elements
  for (int t = threadIdx.x; t < EPB * 3 * STR; t += NT) {
    const int sl = t / (3 * STR), rem = t % (3 * STR);
    const int d = rem / STR, k = rem % STR;
    const int pd = spos[sl][1 + d];
    const double* tb = tabs + sw_axis_off(op, d, STR) + (long long)pd * STR;
    if (k < 2) {
      if (k == 0)
        sm[sl][d] = (int)tb[0];
      else
        soL[sl][d] = (int)tb[1];
    } else if (k < 2 + MP2) {
      sS[sl][d][k - 2] = (T)tb[k];
    } else {
      sL[sl][d][k - 2 - MP2] = (T)tb[k];
    }
  }
  __syncthreads();
  const int mx = sm[slot][0], my = sm[slot][1], mz = sm[slot][2];
  const int oLx = soL[slot][0], oLy = soL[slot][1], oLz = soL[slot][2];
  T* b = buf[slot];
  // gather the patch residual (own element plus one node layer of each
  // neighbour), one patch row (j, k) at a time: the row's element offsets are
  // computed once, the row's MP entries are three segments (left neighbour,
  // own element, right neighbour)
  if (valid) {
    const T* rr = r + rhs * Nq;
    for (int row = lt; row < MP2; row += TPE) {
      const int j = row % MP, k = row / MP;
      T* brow = b + j * MP + k * SY;
      if (j >= my || k >= mz) {
#pragma unroll
        for (int i = 0; i < MP; ++i) brow[i] = (T)0;
        continue;
      }
      const int Y = pos[1] * N1 - oLy + j, Z = pos[2] * N1 - oLz + k;
      const int ey = Y / N1, ez = Z / N1;
      const long long rowe = (long long)nx * (ey + (long long)ny * ez);  // element index without x
      const int lyz = N1 * ((Y - ey * N1) + N1 * (Z - ez * N1));
      const T* own = rr + (rowe + pos[0]) * NPE + lyz;
      int i = 0;
      if (oLx) brow[i++] = rr[(rowe + pos[0] - 1) * NPE + lyz + (N1 - 1)];
#pragma unroll
      for (int a = 0; a < N1; ++a) brow[i + a] = own[a];
      i += N1;
      if (i < mx) brow[i++] = rr[(rowe + pos[0] + 1) * NPE + lyz];
      for (; i < MP; ++i) brow[i] = (T)0;
    }
  } else {
    for (int t = lt; t < SE; t += TPE) b[t] = (T)0;
  }
  __syncthreads();
  sw_pass3<T, MP, SY, TPE, LPT, 0, false>(b, sS[slot][0], lt);
  __syncthreads();
  sw_pass3<T, MP, SY, TPE, LPT, 1, false>(b, sS[slot][1], lt);
  __syncthreads();
  sw_pass3<T, MP, SY, TPE, LPT, 2, false>(b, sS[slot][2], lt);
  // scale by 1 / (lx + ly + lz) along this thread's z lines (i, j)
#pragma unroll
  for (int s = 0; s < LPT; ++s) {
    const int l = lt + TPE * s;
    if (l < MP2) {
      const int l1 = l % MP, l2 = l / MP;
#pragma unroll
      for (int k = 0; k < MP; ++k) {
        const int t = l + SY * k;
        const bool in = l1 < mx && l2 < my && k < mz;
        b[t] = in ? sw_div(b[t], sL[slot][0][l1] + sL[slot][1][l2] + sL[slot][2][k]) : (T)0;
      }
    }
  }
  sw_pass3<T, MP, SY, TPE, LPT, 2, true>(b, sS[slot][2], lt);
  __syncthreads();
  sw_pass3<T, MP, SY, TPE, LPT, 1, true>(b, sS[slot][1], lt);
  __syncthreads();
  sw_pass3<T, MP, SY, TPE, LPT, 0, true>(b, sS[slot][0], lt);
  __syncthreads();
  if (!valid) return;
  T* out = zp + (rhs * E + e) * (long long)MP3;
  for (int t = lt; t < MP3; t += TPE) out[t] = b[t % MP2 + SY * (t / MP2)];
}

// Gather block shape: GE elements of NPE nodes per block (several small
// elements per block on the coarse levels), one thread per node.
#ifndef DG_GATHER_THREADS
#define DG_GATHER_THREADS 256  // thread budget of a gather block (at least one element)
#endif
template <int N1>
struct GatherCfg {
  static constexpr int NPE = N1 * N1 * N1;
  static constexpr int GE = DG_GATHER_THREADS / NPE < 1 ? 1 : DG_GATHER_THREADS / NPE;
  static constexpr int THREADS = GE * NPE;
};

// mode 0: z = M r; 1: d = c1 M r, x = d; 2: d = c1 M r, x += d; 3: d = c1 d + c2 M r, x += d
// (d is passed in z). GE elements per block and iteration (grid-stride), one thread per node,
// GS sources per thread (the node's position, neighbour tests and offsets shared by them).
#ifndef DG_GATHER_SOURCES
#define DG_GATHER_SOURCES 4
#endif
template <typename T, int N1, int MODE>
__global__ void __launch_bounds__(GatherCfg<N1>::THREADS)
    k_schwarz_gather(const LevelOp* __restrict__ op, const T* __restrict__ zp, T* __restrict__ z, T* __restrict__ x,
                     T c1, T c2, const int* __restrict__ act, int nact) {
  constexpr int MP = N1 + 2, MP2 = MP * MP, MP3 = MP2 * MP, NPE = N1 * N1 * N1, GE = GatherCfg<N1>::GE;
  constexpr int GS = DG_GATHER_SOURCES;
  const int nx = op->n[0], ny = op->n[1], nz = op->n[2];
  const int E = op->E;
  const long long Nq = op->Nq;
  // this block's sources (GS consecutive entries of the active list)
  const int k0 = blockIdx.y * GS;
  const int ns = min(GS, nact - k0);
  const int slot = threadIdx.x / NPE, loc = threadIdx.x % NPE;
  const int a = loc % N1, bb = (loc / N1) % N1, c = loc / (N1 * N1);
  // element position, advanced by the grid stride without runtime divisions
  const int g = gridDim.x * GE, sx = g % nx, sy = (g / nx) % ny, sz = g / (nx * ny);
  const int e0 = blockIdx.x * GE + slot;
  int ex = e0 % nx, ey = (e0 / nx) % ny, ez = e0 / (nx * ny);
  for (int e = e0; e < E; e += g) {
    const int ix = a + (ex > 0), iy = bb + (ey > 0), iz = c + (ez > 0);
    // neighbour along each axis whose patch also covers this node, if any
    int dx = 0, jx = 0, dy = 0, jy = 0, dz = 0, jz = 0;
    if (a == 0 && ex > 0) {
      dx = -1;
      jx = N1 + (ex > 1);
    } else if (a == N1 - 1 && ex < nx - 1) {
      dx = 1;
    }
    if (bb == 0 && ey > 0) {
      dy = -nx;
      jy = N1 + (ey > 1);
    } else if (bb == N1 - 1 && ey < ny - 1) {
      dy = nx;
    }
    if (c == 0 && ez > 0) {
      dz = -nx * ny;
      jz = N1 + (ez > 1);
    } else if (c == N1 - 1 && ez < nz - 1) {
      dz = nx * ny;
    }
    // offsets (values, within one source's patch buffer) of every contribution;
    // a source's patch buffer holds E MP^3 < 2^31 values
    const int o0 = e * MP3 + ix + MP * iy + MP2 * iz;
    const int ox = (e + dx) * MP3 + jx + MP * iy + MP2 * iz;
    const int oy = (e + dy) * MP3 + ix + MP * jy + MP2 * iz;
    const int oz = (e + dz) * MP3 + ix + MP * iy + MP2 * jz;
    const int oxy = (e + dx + dy) * MP3 + jx + MP * jy + MP2 * iz;
    const int oxz = (e + dx + dz) * MP3 + jx + MP * iy + MP2 * jz;
    const int oyz = (e + dy + dz) * MP3 + ix + MP * jy + MP2 * jz;
    const int oxyz = (e + dx + dy + dz) * MP3 + jx + MP * jy + MP2 * jz;
    const int gi = e * NPE + loc;
#pragma unroll
    for (int j = 0; j < GS; ++j) {
      if (j >= ns) break;
      const long long rhs = act[k0 + j];
      const T* zs = zp + rhs * E * (long long)MP3;
      T* zg = z + rhs * Nq;
      T* xg = x + rhs * Nq;
      T acc = zs[o0];
      if (dx) acc += zs[ox];
      if (dy) acc += zs[oy];
      if (dz) acc += zs[oz];
      if (dx && dy) acc += zs[oxy];
      if (dx && dz) acc += zs[oxz];
      if (dy && dz) acc += zs[oyz];
      if (dx && dy && dz) acc += zs[oxyz];
      if (MODE == 0) {
        zg[gi] = acc;
      } else if (MODE == 1) {
        const T v = c1 * acc;
        zg[gi] = v;
        xg[gi] = v;
      } else if (MODE == 2) {
        const T v = c1 * acc;
        zg[gi] = v;
        xg[gi] += v;
      } else {
        const T v = c1 * zg[gi] + c2 * acc;
        zg[gi] = v;
        xg[gi] += v;
      }
    }
    ex += sx;
    int carry = ex >= nx;
    ex -= carry ? nx : 0;
    ey += sy + carry;
    carry = ey >= ny;
    ey -= carry ? ny : 0;
    ez += sz + carry;
  }
}

template <typename T, int N1>
static cudaError_t schwarz_n1(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp, T* z,
                              T* x, int mode, double c1, double c2, const int* act, int nact, cudaStream_t s,
                              const SwTcPlan* tc) {
  using C = SwCfg<T, N1>;
  const long long items = (long long)nact * hop.E;
#if DG_SMEM_CARVEOUT >= 0
  static bool carve = false;
  if (!carve) {
    cudaFuncSetAttribute(k_schwarz_patch<T, N1>, cudaFuncAttributePreferredSharedMemoryCarveout, DG_SMEM_CARVEOUT);
    carve = true;
  }
#endif
  if (sizeof(T) == 4 && tc && tc->blob) {
    const cudaError_t e = launch_schwarz_patch_tc(hop, dop, *tc, (const float*)r, (float*)zp, act, nact, s);
    if (e != cudaSuccess) return e;
  } else {
    count_launch();
    k_schwarz_patch<T, N1><<<(unsigned)((items + C::EPB - 1) / C::EPB), C::THREADS, 0, s>>>(dop, tabs, r, zp, act,
                                                                                           nact);
  }
  constexpr int GT = GatherCfg<N1>::THREADS;
  // the gather indexes one source's patch buffer with 32-bit offsets
  if ((long long)hop.E * (N1 + 2) * (N1 + 2) * (N1 + 2) >= (1LL << 31)) return cudaErrorInvalidValue;
  long long gx = (hop.E + GatherCfg<N1>::GE - 1) / GatherCfg<N1>::GE;
#if DG_GATHER_WAVE > 0
  const long long ngroups = (nact + DG_GATHER_SOURCES - 1) / DG_GATHER_SOURCES;
  const long long cap = 152LL * DG_GATHER_WAVE / (ngroups > 0 ? ngroups : 1) + 1;
  if (gx > cap) gx = cap;
#endif
  const dim3 grid((unsigned)gx, (unsigned)((nact + DG_GATHER_SOURCES - 1) / DG_GATHER_SOURCES));
  count_launch();
  switch (mode) {
    case 0: k_schwarz_gather<T, N1, 0><<<grid, GT, 0, s>>>(dop, zp, z, x, (T)c1, (T)c2, act, nact); break;
    case 1: k_schwarz_gather<T, N1, 1><<<grid, GT, 0, s>>>(dop, zp, z, x, (T)c1, (T)c2, act, nact); break;
    case 2: k_schwarz_gather<T, N1, 2><<<grid, GT, 0, s>>>(dop, zp, z, x, (T)c1, (T)c2, act, nact); break;
    default: k_schwarz_gather<T, N1, 3><<<grid, GT, 0, s>>>(dop, zp, z, x, (T)c1, (T)c2, act, nact); break;
  }
  return cudaGetLastError();
}

// the patch solves alone (the first kernel of schwarz_n1)
template <typename T, int N1>
static cudaError_t schwarz_patch_n1(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp,
                                    const int* act, int nact, cudaStream_t s, const SwTcPlan* tc) {
  using C = SwCfg<T, N1>;
  if (sizeof(T) == 4 && tc && tc->blob)
    return launch_schwarz_patch_tc(hop, dop, *tc, (const float*)r, (float*)zp, act, nact, s);
  const long long items = (long long)nact * hop.E;
  count_launch();
  k_schwarz_patch<T, N1><<<(unsigned)((items + C::EPB - 1) / C::EPB), C::THREADS, 0, s>>>(dop, tabs, r, zp, act,
                                                                                         nact);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_schwarz_patch(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp,
                                 const int* act, int nact, cudaStream_t s, const SwTcPlan* tc) {
  if (nact == 0) return cudaSuccess;
  switch (hop.n1) {
    case 2: return schwarz_patch_n1<T, 2>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 3: return schwarz_patch_n1<T, 3>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 4: return schwarz_patch_n1<T, 4>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 5: return schwarz_patch_n1<T, 5>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 6: return schwarz_patch_n1<T, 6>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 7: return schwarz_patch_n1<T, 7>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 8: return schwarz_patch_n1<T, 8>(hop, dop, tabs, r, zp, act, nact, s, tc);
    case 9: return schwarz_patch_n1<T, 9>(hop, dop, tabs, r, zp, act, nact, s, tc);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_schwarz(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp, T* z,
                           T* x, int mode, double c1, double c2, const int* act, int nact, cudaStream_t s,
                           const SwTcPlan* tc) {
  if (nact == 0) return cudaSuccess;
  switch (hop.n1) {
    case 2: return schwarz_n1<T, 2>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 3: return schwarz_n1<T, 3>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 4: return schwarz_n1<T, 4>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 5: return schwarz_n1<T, 5>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 6: return schwarz_n1<T, 6>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 7: return schwarz_n1<T, 7>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 8: return schwarz_n1<T, 8>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    case 9: return schwarz_n1<T, 9>(hop, dop, tabs, r, zp, z, x, mode, c1, c2, act, nact, s, tc);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_schwarz_patch<double>(const LevelOp&, const LevelOp*, const double*, const double*,
                                                  double*, const int*, int, cudaStream_t, const SwTcPlan*);
template cudaError_t launch_schwarz_patch<float>(const LevelOp&, const LevelOp*, const double*, const float*, float*,
                                                 const int*, int, cudaStream_t, const SwTcPlan*);
template cudaError_t launch_schwarz<double>(const LevelOp&, const LevelOp*, const double*, const double*, double*,
                                            double*, double*, int, double, double, const int*, int, cudaStream_t,
                                            const SwTcPlan*);
template cudaError_t launch_schwarz<float>(const LevelOp&, const LevelOp*, const double*, const float*, float*,
                                           float*, float*, int, double, double, const int*, int, cudaStream_t,
                                           const SwTcPlan*);

}  // namespace dg
