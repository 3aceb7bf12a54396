// Overlapping Schwarz smoother for the hp-multigrid of Sec. 6.4.
//
// The paper does not specify the smoother. With the penalty of Sec. 3.5
// (eps = 1/8, i.e. eight times the coercivity bound) point- and element-block
// Jacobi smoothers leave continuous high-order modes undamped, so each
// multigrid level uses additive Schwarz over element patches with one node of
// overlap, accelerated by Chebyshev iteration. Each patch problem is solved
// exactly by fast diagonalisation (the patch operator is a Kronecker sum of
// restricted 1-D matrices; tables built at setup):
//   k_schwarz_patch:  zp_e = A_P(e)^-1 R_P(e) r        (one block per element)
//   k_schwarz_gather: z    = sum_e R_P(e)^T zp_e       (each node gathers the
//                            at most 8 patches covering it; no atomics)
#include "dg_internal.h"

namespace dg {

__host__ __device__ inline int sw_axis_off(const LevelOp* op, int d, int stride) {
  return d == 0 ? 0 : (d == 1 ? op->n[0] * stride : (op->n[0] + op->n[1]) * stride);
}

template <typename T, int N1>
__global__ void __launch_bounds__(256)
    k_schwarz_patch(const LevelOp* __restrict__ op, const double* __restrict__ tabs, const T* __restrict__ r,
                    T* __restrict__ zp, const int* __restrict__ act) {
  constexpr int MP = N1 + 2, MP3 = MP * MP * MP, NPE = N1 * N1 * N1, STR = 2 + MP * MP + MP;
  __shared__ T sS[3][MP * MP];
  __shared__ T sL[3][MP];
  __shared__ T b0[MP3];
  __shared__ T b1[MP3];
  const int e = blockIdx.x;
  const long long rhs = act[blockIdx.y];
  const int nx = op->n[0], ny = op->n[1];
  const int E = op->E;
  const long long Nq = op->Nq;
  const int pos[3] = {e % nx, (e / nx) % ny, e / (nx * ny)};
  int m[3], oL[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double* tb = tabs + sw_axis_off(op, d, STR) + (long long)pos[d] * STR;
    m[d] = (int)tb[0];
    oL[d] = (int)tb[1];
    for (int i = threadIdx.x; i < MP * MP; i += blockDim.x) sS[d][i] = (T)tb[2 + i];
    for (int i = threadIdx.x; i < MP; i += blockDim.x) sL[d][i] = (T)tb[2 + MP * MP + i];
  }
  // gather the patch residual (own element plus one node layer of the neighbours)
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int i = t % MP, j = (t / MP) % MP, k = t / (MP * MP);
    T v = 0;
    if (i < m[0] && j < m[1] && k < m[2]) {
      const int X = pos[0] * N1 - oL[0] + i, Y = pos[1] * N1 - oL[1] + j, Z = pos[2] * N1 - oL[2] + k;
      const long long en = (long long)(X / N1) + (long long)nx * ((Y / N1) + (long long)ny * (Z / N1));
      const int loc = (X % N1) + N1 * ((Y % N1) + N1 * (Z % N1));
      v = r[rhs * Nq + en * NPE + loc];
    }
    b0[t] = v;
  }
  __syncthreads();
  // forward transforms: b <- (Sx (x) Sy (x) Sz)^T b
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int q = t % MP, jk = t / MP;
    T acc = 0;
    for (int i = 0; i < m[0]; ++i) acc += sS[0][i * MP + q] * b0[jk * MP + i];
    b1[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int i = t % MP, q = (t / MP) % MP, k = t / (MP * MP);
    T acc = 0;
    for (int j = 0; j < m[1]; ++j) acc += sS[1][j * MP + q] * b1[(k * MP + j) * MP + i];
    b0[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int i = t % MP, j = (t / MP) % MP, q = t / (MP * MP);
    T acc = 0;
    for (int k = 0; k < m[2]; ++k) acc += sS[2][k * MP + q] * b0[(k * MP + j) * MP + i];
    const bool in = i < m[0] && j < m[1] && q < m[2];
    b1[t] = in ? acc / (sL[0][i] + sL[1][j] + sL[2][q]) : (T)0;
  }
  __syncthreads();
  // backward transforms: b <- (Sx (x) Sy (x) Sz) b
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int i = t % MP, jk = t / MP;
    T acc = 0;
    for (int q = 0; q < m[0]; ++q) acc += sS[0][i * MP + q] * b1[jk * MP + q];
    b0[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int i = t % MP, j = (t / MP) % MP, k = t / (MP * MP);
    T acc = 0;
    for (int q = 0; q < m[1]; ++q) acc += sS[1][j * MP + q] * b0[(k * MP + q) * MP + i];
    b1[t] = acc;
  }
  __syncthreads();
  T* out = zp + ((long long)rhs * E + e) * MP3;
  for (int t = threadIdx.x; t < MP3; t += blockDim.x) {
    const int ij = t % (MP * MP), k = t / (MP * MP);
    T acc = 0;
    for (int q = 0; q < m[2]; ++q) acc += sS[2][k * MP + q] * b1[q * MP * MP + ij];
    out[t] = acc;
  }
}

template <typename T, int N1>
__global__ void k_schwarz_gather(const LevelOp* __restrict__ op, const T* __restrict__ zp, T* __restrict__ z,
                                 const int* __restrict__ act) {
  constexpr int MP = N1 + 2, MP3 = MP * MP * MP, NPE = N1 * N1 * N1;
  const long long rhs = act[blockIdx.y];
  const int nx = op->n[0], ny = op->n[1], nz = op->n[2];
  const int E = op->E;
  const long long Nq = op->Nq;
  const T* zr = zp + rhs * E * (long long)MP3;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(q / NPE), loc = (int)(q % NPE);
    const int lc[3] = {loc % N1, (loc / N1) % N1, loc / (N1 * N1)};
    const int ec[3] = {e % nx, (e / nx) % ny, e / (nx * ny)};
    const int nn[3] = {nx, ny, nz};
    // per axis: up to two (patch position, coordinate inside that patch)
    int cp[3][2], cc[3][2], cn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cn[d] = 1;
      cp[d][0] = ec[d];
      cc[d][0] = lc[d] + (ec[d] > 0 ? 1 : 0);
      if (lc[d] == 0 && ec[d] > 0) {
        cp[d][1] = ec[d] - 1;
        cc[d][1] = N1 + (ec[d] - 1 > 0 ? 1 : 0);
        cn[d] = 2;
      } else if (lc[d] == N1 - 1 && ec[d] < nn[d] - 1) {
        cp[d][1] = ec[d] + 1;
        cc[d][1] = 0;
        cn[d] = 2;
      }
    }
    T acc = 0;
    for (int u = 0; u < cn[2]; ++u)
      for (int v = 0; v < cn[1]; ++v)
        for (int w = 0; w < cn[0]; ++w) {
          const long long pe = cp[0][w] + (long long)nx * (cp[1][v] + (long long)ny * cp[2][u]);
          acc += zr[pe * MP3 + cc[0][w] + MP * (cc[1][v] + MP * cc[2][u])];
        }
    z[rhs * Nq + q] = acc;
  }
}

template <typename T, int N1>
static cudaError_t schwarz_n1(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp, T* z,
                              const int* act, int nact, cudaStream_t s) {
  count_launch();
  k_schwarz_patch<T, N1><<<dim3(hop.E, nact), 256, 0, s>>>(dop, tabs, r, zp, act);
  long long gx = (hop.Nq + 1023) / 1024;
  if (gx > 4096) gx = 4096;
  count_launch();
  k_schwarz_gather<T, N1><<<dim3((unsigned)gx, nact), 256, 0, s>>>(dop, zp, z, act);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_schwarz(const LevelOp& hop, const LevelOp* dop, const double* tabs, const T* r, T* zp, T* z,
                           const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  switch (hop.n1) {
    case 2: return schwarz_n1<T, 2>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 3: return schwarz_n1<T, 3>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 4: return schwarz_n1<T, 4>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 5: return schwarz_n1<T, 5>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 6: return schwarz_n1<T, 6>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 7: return schwarz_n1<T, 7>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 8: return schwarz_n1<T, 8>(hop, dop, tabs, r, zp, z, act, nact, s);
    case 9: return schwarz_n1<T, 9>(hop, dop, tabs, r, zp, z, act, nact, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_schwarz<double>(const LevelOp&, const LevelOp*, const double*, const double*, double*,
                                            double*, const int*, int, cudaStream_t);
template cudaError_t launch_schwarz<float>(const LevelOp&, const LevelOp*, const double*, const float*, float*,
                                           float*, const int*, int, cudaStream_t);

}  // namespace dg
