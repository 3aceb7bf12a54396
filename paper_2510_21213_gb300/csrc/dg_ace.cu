// Adaptively compressed exchange (ACE) operator from the last whole exchange
// build: the exchange operator of Sec. 2.3.1 (eq. exchange) in the compressed
// form the HF SCF of Sec. 7.2 (two-loop algorithm) applies, rank N and exact
// on the occupied orbitals (the construction the paper cites for ACE). With
// W_j = sum_s psi_s v_sj = -(V_X psi_j) on the quadrature grid and
// K_ij = <psi_i, W_j>, the operator
//     V_X^ACE u = -W K_s^-1 (W^T diag(W_q) u),   K_s = (K + K^T) / 2,
// has rank N, is symmetric and negative semidefinite in the discrete inner
// product, and reproduces V_X psi_i = -W_i on the occupied orbitals (up to
// the discretisation-level asymmetry of K).
//   1. C = W diag(W_q) U^T for m trial vectors (N x m; chunked partial sums,
//      reduced in a fixed order),
//   2. Z = K_s^-1 C by a Cholesky factorisation on the host (N x N),
//   3. Y = -W Z.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dg_ctx.h"

namespace dg {

constexpr int AT = 32;  // output tile
constexpr int AQ = 32;  // nodes per shared-memory step

// part[chunk][i][t] = sum over the chunk's nodes of A_i(q) W_q B_t(q)
__global__ void k_ace_gram_partial(const double* __restrict__ A, const double* __restrict__ B,
                                   const double* __restrict__ W, int na, int nb, long long Nq,
                                   double* __restrict__ part) {
  __shared__ double sa[AQ][AT + 1];
  __shared__ double sb[AQ][AT + 1];
  const int ti = blockIdx.x * AT, tj = blockIdx.y * AT;
  const int nchunk = gridDim.z;
  const long long per = (Nq + nchunk - 1) / nchunk;
  const long long q0 = (long long)blockIdx.z * per;
  const long long q1 = q0 + per < Nq ? q0 + per : Nq;
  const int tx = threadIdx.x % AT, ty = threadIdx.x / AT;  // ty in [0, 8)
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long qs = q0; qs < q1; qs += AQ) {
    for (int t = threadIdx.x; t < AQ * AT; t += blockDim.x) {
      const int qq = t % AQ, r = t / AQ;
      const long long q = qs + qq;
      const int i = ti + r, j = tj + r;
      sa[qq][r] = (q < q1 && i < na) ? A[(long long)i * Nq + q] * W[q] : 0.0;
      sb[qq][r] = (q < q1 && j < nb) ? B[(long long)j * Nq + q] : 0.0;
    }
    __syncthreads();
    for (int qq = 0; qq < AQ; ++qq) {
      const double bj = sb[qq][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] += sa[qq][ty + 8 * r] * bj;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ti + ty + 8 * r, j = tj + tx;
    if (i < na && j < nb) part[((long long)blockIdx.z * na + i) * nb + j] = acc[r];
  }
}

__global__ void k_ace_gram_reduce(const double* __restrict__ part, int na, int nb, int nchunk,
                                  double* __restrict__ C) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= na * nb) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(long long)c * na * nb + k];
  C[k] = s;
}

// Y_t(q) = -sum_j W_j(q) Z[j][t] (Z [N][m] in shared memory, N * m <= ACE_ZMAX)
constexpr int ACE_ZMAX = 4096;
__global__ void k_ace_expand(const double* __restrict__ Wacc, const double* __restrict__ Z, int N, int m,
                             long long Nq, double* __restrict__ Y) {
  __shared__ double sz[ACE_ZMAX];
  for (int i = threadIdx.x; i < N * m; i += blockDim.x) sz[i] = Z[i];
  __syncthreads();
  const int t = blockIdx.y;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < N; ++j) acc += Wacc[(long long)j * Nq + q] * sz[j * m + t];
    Y[(long long)t * Nq + q] = -acc;
  }
}

// in-place Cholesky of the symmetric part of K (n x n, row-major); false if
// it is not positive definite
static bool cholesky_sym(std::vector<double>& L, const std::vector<double>& K, int n) {
  L.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.5 * (K[(size_t)i * n + j] + K[(size_t)j * n + i]);
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[(size_t)i * n + i] = std::sqrt(s);
      } else {
        L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
      }
    }
  return true;
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_ace_apply(dg_handle h, const double* U_dev, int64_t m, double* Y_dev, void* stream) {
  if (!h || m < 0 || (m > 0 && (!U_dev || !Y_dev))) return DG_ERR_INVALID_ARG;
  if (h->ace_N < 1) {
    h->err = "dg_ace_apply: no whole exchange build on this handle";
    return DG_ERR_INVALID_ARG;
  }
  const int N = h->ace_N;
  if (m == 0) return DG_OK;
  if ((long long)N * m > ACE_ZMAX) {
    h->err = "dg_ace_apply: N * m above 4096; apply the operator to fewer vectors at a time";
    return DG_ERR_INVALID_ARG;
  }
  std::vector<double> L;
  if (!cholesky_sym(L, h->ace_K, N)) {
    h->err = "dg_ace_apply: the symmetric part of K is not positive definite";
    return DG_ERR_BREAKDOWN;
  }
  cudaStream_t us = (cudaStream_t)stream;
  DG_CK(cudaEventRecord(h->ev_in, us));
  DG_CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  cudaStream_t s = h->ws;
  const long long Nq = h->Nq;
  const int nm = (int)m;
  const int nchunk = (int)std::max(1LL, std::min(256LL, Nq / 8192));
  {
    DeviceWideGuard guard;
    DG_CK(h->ace_part.ensure(sizeof(double) * (size_t)nchunk * N * nm));
    DG_CK(h->ace_C.ensure(sizeof(double) * (size_t)N * nm));
  }
  const double* Wacc = h->Wacc.as<double>();
  count_launch(2);
  k_ace_gram_partial<<<dim3((N + AT - 1) / AT, (nm + AT - 1) / AT, nchunk), 256, 0, s>>>(
      Wacc, U_dev, h->d_W.as<double>(), N, nm, Nq, h->ace_part.as<double>());
  k_ace_gram_reduce<<<(N * nm + 255) / 256, 256, 0, s>>>(h->ace_part.as<double>(), N, nm, nchunk,
                                                           h->ace_C.as<double>());
  DG_CK(cudaGetLastError());
  std::vector<double> Cm((size_t)N * nm);
  DG_CK(cudaMemcpyAsync(Cm.data(), h->ace_C.p, sizeof(double) * Cm.size(), cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  // Z = K_s^-1 C: forward and back substitution, column by column
  for (int t = 0; t < nm; ++t) {
    for (int i = 0; i < N; ++i) {
      double v = Cm[(size_t)i * nm + t];
      for (int k = 0; k < i; ++k) v -= L[(size_t)i * N + k] * Cm[(size_t)k * nm + t];
      Cm[(size_t)i * nm + t] = v / L[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
      double v = Cm[(size_t)i * nm + t];
      for (int k = i + 1; k < N; ++k) v -= L[(size_t)k * N + i] * Cm[(size_t)k * nm + t];
      Cm[(size_t)i * nm + t] = v / L[(size_t)i * N + i];
    }
  }
  DG_CK(cudaMemcpyAsync(h->ace_C.p, Cm.data(), sizeof(double) * Cm.size(), cudaMemcpyHostToDevice, s));
  count_launch();
  const long long gx = std::max(1LL, std::min((Nq + 255) / 256, 152LL * 8 / nm + 1));
  k_ace_expand<<<dim3((unsigned)gx, nm), 256, 0, s>>>(Wacc, h->ace_C.as<double>(), N, nm, Nq, Y_dev);
  DG_CK(cudaGetLastError());
  DG_CK(cudaStreamSynchronize(s));  // Cm is a host temporary of the upload above
  DG_CK(cudaEventRecord(h->ev_out, s));
  DG_CK(cudaStreamWaitEvent(us, h->ev_out, 0));
  return DG_OK;
}

}  // extern "C"
