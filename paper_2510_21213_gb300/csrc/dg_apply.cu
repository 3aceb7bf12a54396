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

template <int N1>
struct ApplyCfg {
  static constexpr int NPE = N1 * N1 * N1;
  static constexpr int NF = N1 * N1;
  static constexpr int EPB = (NPE >= 128) ? 1 : (256 / NPE);
  static constexpr int THREADS = EPB * NPE;
};

template <typename T, int N1, int MODE>
__global__ void __launch_bounds__(ApplyCfg<N1>::THREADS)
    k_apply(const LevelOp* __restrict__ op, const T* __restrict__ u, T* __restrict__ out,
            const T* __restrict__ rin, const int* __restrict__ act, int nact) {
  using C = ApplyCfg<N1>;
  constexpr int NPE = C::NPE, NF = C::NF, EPB = C::EPB, NT = C::THREADS;
  __shared__ T sK[3][4][NF];
  __shared__ T sC[3][4][N1];
  __shared__ T sM[3][N1];
  __shared__ T sTr[4][N1];
  __shared__ T su[EPB][NPE];
  __shared__ T st[EPB][6][2][NF];

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
  const int slot = tid / NPE, loc = tid % NPE;
  const long long item = (long long)blockIdx.x * EPB + slot;
  const bool valid = item < (long long)nact * E;
  const int k = valid ? (int)(item / E) : 0;
  const int e = valid ? (int)(item % E) : 0;
  const long long rhs = valid ? (long long)act[k] : 0;
  const T* ub = u + rhs * Nq;
  if (valid) su[slot][loc] = ub[(long long)e * NPE + loc];
  const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
  __syncthreads();

  // neighbour traces: face f = 2 d + side (side 0: -d neighbour, side 1: +d)
  for (int t = loc; t < 6 * NF; t += NPE) {
    const int f = t / NF, tt = t % NF;
    const int d = f >> 1, side = f & 1;
    const int coord = d == 0 ? ex : (d == 1 ? ey : ez);
    const int nd = d == 0 ? nx : (d == 1 ? ny : nz);
    T val = 0, der = 0;
    const bool has = valid && (side == 0 ? coord > 0 : coord < nd - 1);
    if (has) {
      const int se = d == 0 ? 1 : (d == 1 ? nx : nx * ny);
      const int en = e + (side == 0 ? -se : se);
      const T* un = ub + (long long)en * NPE;
      const int t1 = tt % N1, t2 = tt / N1;
      int base, sd;
      if (d == 0) {
        base = N1 * t1 + NF * t2;
        sd = 1;
      } else if (d == 1) {
        base = t1 + NF * t2;
        sd = N1;
      } else {
        base = t1 + N1 * t2;
        sd = NF;
      }
      // the -d neighbour meets us at its right end, the +d neighbour at its left end
      const T* tv = side == 0 ? sTr[1] : sTr[0];
      const T* td = side == 0 ? sTr[3] : sTr[2];
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const T x = un[base + i * sd];
        val += tv[i] * x;
        der += td[i] * x;
      }
    }
    st[slot][f][0][tt] = val;
    st[slot][f][1][tt] = der;
  }
  __syncthreads();
  if (!valid) return;

  const int a = loc % N1, b = (loc / N1) % N1, c = loc / NF;
  const int tyx = (ex == 0 ? 1 : 0) | (ex == nx - 1 ? 2 : 0);
  const int tyy = (ey == 0 ? 1 : 0) | (ey == ny - 1 ? 2 : 0);
  const int tyz = (ez == 0 ? 1 : 0) | (ez == nz - 1 ? 2 : 0);
  const T* us = su[slot];

  T sx = 0, sy = 0, sz = 0;
#pragma unroll
  for (int i = 0; i < N1; ++i) {
    sx += sK[0][tyx][a * N1 + i] * us[i + N1 * b + NF * c];
    sy += sK[1][tyy][b * N1 + i] * us[a + N1 * i + NF * c];
    sz += sK[2][tyz][c * N1 + i] * us[a + N1 * b + NF * i];
  }
  {
    const int tx = b + N1 * c;
    sx += sC[0][0][a] * st[slot][0][0][tx] + sC[0][1][a] * st[slot][0][1][tx] + sC[0][2][a] * st[slot][1][0][tx] +
          sC[0][3][a] * st[slot][1][1][tx];
    const int ty = a + N1 * c;
    sy += sC[1][0][b] * st[slot][2][0][ty] + sC[1][1][b] * st[slot][2][1][ty] + sC[1][2][b] * st[slot][3][0][ty] +
          sC[1][3][b] * st[slot][3][1][ty];
    const int tz = a + N1 * b;
    sz += sC[2][0][c] * st[slot][4][0][tz] + sC[2][1][c] * st[slot][4][1][tz] + sC[2][2][c] * st[slot][5][0][tz] +
          sC[2][3][c] * st[slot][5][1][tz];
  }
  const T Au = sM[1][b] * sM[2][c] * sx + sM[0][a] * sM[2][c] * sy + sM[0][a] * sM[1][b] * sz;
  const long long gi = rhs * Nq + (long long)e * NPE + loc;
  if (MODE == 0) {
    out[gi] = Au;
  } else if (MODE == 1) {
    out[gi] = rin[gi] - Au;
  } else {
    out[gi] = out[gi] - Au;
  }
}

template <typename T, int N1>
static cudaError_t apply_n1(const LevelOp& hop, const LevelOp* dop, int mode, const T* u, T* out, const T* rin,
                            const int* act, int nact, cudaStream_t s) {
  using C = ApplyCfg<N1>;
  const long long items = (long long)nact * hop.E;
  const long long blocks = (items + C::EPB - 1) / C::EPB;
  if (blocks == 0) return cudaSuccess;
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
