// Poisson solves and the exchange build on the octree auxiliary mesh
// (Sec. 6.2 mesh, Sec. 6.3 boundary data, Sec. 6.1.2 eq. fock_exchange).
//
// A handle keeps the leaves' connectivity, sizes, node coordinates and weights
// and the preconditioner tables on the device. The system is the one the
// octree operator (dg_octree.cu) applies: SIPDG with symmetric Nitsche
// boundary terms, hanging faces integrated on the smaller face. It is solved
// by PCG with an element-block Jacobi preconditioner whose blocks are
// inverted exactly by fast diagonalisation:
//
//  * The diagonal block of leaf K is a Kronecker sum
//      A_KK = K_x (x) M_y (x) M_z + M_x (x) K_y (x) M_z + M_x (x) M_y (x) K_z,
//    M_d = (h_d / 2) diag(w) the GL-collocated mass (exact for the degree-2p
//    tangential integrands) and K_d the 1-D matrix of the leaf along d:
//      K_d = (2/h_d) S + sum over the two sides e = -1, +1 of
//            -c (2/h_d) e (l(e) l'(e)^T + l'(e) l(e)^T) + sigma l(e) l(e)^T,
//    c = 1 on a boundary face and 1/2 otherwise, sigma the penalty of the
//    smaller leaf across the face (h_d, or h_d / 2 where four smaller leaves
//    meet the face). The faces' leaf-leaf parts integrate the leaf's own
//    traces over its whole face, so the block separates although the mesh
//    does not.
//  * With K_d S_d = M_d S_d Lambda_d, S_d^T M_d S_d = I, the block inverse is
//    (S_x (x) S_y (x) S_z) (Lambda_x + Lambda_y + Lambda_z)^-1 (S_x (x) S_y (x) S_z)^T.
//    (S_d, Lambda_d) depend on the level, the axis and the two face types only:
//    a few classes per mesh, computed on the host.
//
// Boundary data (Sec. 6.3): g(x) = sum_q W_q f(q) / |x - x_q| at the GL nodes
// of every boundary face, by direct quadrature over all nodes (FP64, fixed
// summation order), then the Nitsche load int_F g (sigma v - d_n v), exact
// with the face's GL rule because g is taken as its degree-p interpolant.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dg_ctx.h"
#include "dg_internal.h"
#include "dg_mg.h"
#include "dg_octree.h"
#include "dg_setup.h"

// One level of the octree hierarchy: the leaves at degree p (the fine level,
// then p-coarsened), with the tables of its operator and of its leaf-block
// preconditioner, and its multigrid workspace.
struct OctLevel {
  int n1 = 0, p = 0;
  long long Nq = 0;
  dg::OctTables T;
  dg::DevBuf cls;     // int [E][3]: 1-D class of each leaf axis
  dg::DevBuf S, lam;  // per class: S [n1][n1] (row node, column mode), lambda [n1]
  int ncls = 0;
  double lam_max = 0;  // lambda_max(P^-1 A) estimate (power iteration at set-up)
  dg::DevBuf I;        // [n1][n1c]: the next coarser level's basis at this level's nodes
  dg::DevBuf x, b, res, d, z, q;  // V-cycle workspace, [cap][Nq] each
};

// Handle of the octree solver (opaque in the C ABI).
struct dg_oct {
  std::string err;
  int n1 = 0, p = 0, E = 0, pform = 0, max_iter = 0, precond = 1;
  int mixed = 0;                 // 1: FP32 inner PCG (FP32 V-cycle) inside FP64 refinement
  double inner_rtol = 1e-4;      // relative reduction of each inner solve
  int maxparts = 6;  // largest face-part count of a leaf (the operator's shared memory)
  double eps = 0.125, rtol = 1e-10;
  long long Nq = 0;
  dg::DevBuf hq, kind, nb, pos;  // leaf sizes [E][3]; connectivity [E][6], [E][6][4], [E][6]
  std::vector<OctLevel> lv;      // lv[0]: the fine level
  dg::DevBuf xq, W;              // node coordinates [Nq][3], quadrature weights [Nq]
  int nbf = 0;                   // boundary faces
  dg::DevBuf xb;                 // their GL nodes [nbf][n1 * n1][3] (lower tangential axis fastest)
  dg::DevBuf lift1d;             // [nbf][n1]: (h_t0 h_t1 / 4)(sigma l_a(e) - e (2/h_d) l_a'(e))
  dg::DevBuf wgl;                // GL weights [n1]
  int nbl = 0;                   // leaves with a boundary face
  dg::DevBuf bleaf;              // [nbl][7]: leaf, then the boundary face index of each face or -1
  // coarse correction of the V-cycle: the uniform root grid at degree 1 and
  // its own h-hierarchy (a uniform solver handle), and the transfer to it
  dg_ctx* root = nullptr;
  long long Nq_root = 0;
  int n_root = 0;                // root cells
  dg::DevBuf rcell;              // int [E]: root cell of each leaf
  dg::DevBuf rJ;                 // double [E][3][2][2]: root basis b at the leaf's degree-1 node a, per axis
  dg::DevBuf rptr, rlist;        // root cell -> its leaves (CSR, leaf order)
  dg::DevBuf rb, rx;             // root-level right-hand side and correction, [cap][Nq_root]
  int cheb_k = 3;                // Chebyshev degree of the octree-level smoother
  double cheb_range = 10.0;      // its interval [lambda_max / range, lambda_max]
  // workspace, sized for `cap` sources
  int cap = 0;
  dg::DevBuf f, g, gpart, b, x, r, z, pv, qv, scal, part, act, flags, pidx, lists, Wacc, kpart, Kdev;
  dg::DevBuf b32, x32, r32, z32, p32, q32;  // FP32 inner solve (mixed)
  // mixed mode: the boundary data as one GEMM per chunk, G = (W f) K with the
  // kernel matrix K[q][j] = 1 / |xb_j - x_q| (FP32, [Nq][nbf n1^2]) kept on
  // the device when it fits the budget below
  dg::DevBuf kmat, wf32, g32, gwork;
  bool has_kmat = false;
  std::vector<int> act_host;
  ~dg_oct() {
    if (root) dg_destroy(root);
  }
};

namespace dg {

static constexpr int OT = 256;
// per-source scalar slots; I_*: those of the FP32 inner solve
enum { O_BB = 0, O_RR, O_RZ, O_RZN, O_PQ, O_AL, O_BE, O_SE, I_BB, I_RR, I_RZ, I_RZN, I_PQ, I_AL, I_BE, O_NSLOT };

static inline dim3 ogrid(long long n, int nsrc) {
  long long gx = (n + OT * 4 - 1) / (OT * 4);
  gx = std::max(1LL, std::min(gx, 4096LL));
  return dim3((unsigned)gx, (unsigned)nsrc);
}

// z = P r on every leaf: the exact inverse of the leaf's diagonal block by
// fast diagonalisation (one block per leaf and source)
template <typename V, int N1>
__global__ void __launch_bounds__(128) k_oct_bjac(const int* __restrict__ cls, const double* __restrict__ S,
                                                  const double* __restrict__ lam, const V* __restrict__ r,
                                                  V* __restrict__ z, long long Nq, const int* __restrict__ act) {
  constexpr int NPE = N1 * N1 * N1, NF = N1 * N1;
  __shared__ V sS[3][NF], sl[3][N1], u[NPE], t[NPE];
  const int e = blockIdx.x;
  const long long off = (long long)act[blockIdx.y] * Nq + (long long)e * NPE;
  for (int i = threadIdx.x; i < 3 * NF; i += blockDim.x) {
    const int d = i / NF;
    sS[d][i % NF] = (V)S[(long long)cls[3 * e + d] * NF + i % NF];
  }
  for (int i = threadIdx.x; i < 3 * N1; i += blockDim.x) {
    const int d = i / N1;
    sl[d][i % N1] = (V)lam[(long long)cls[3 * e + d] * N1 + i % N1];
  }
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) u[i] = r[off + i];
  __syncthreads();
  // forward: t = (S_x (x) S_y (x) S_z)^T u, one axis at a time (mode index replaces node index)
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int m = i % N1, rest = i - m;
    V acc = 0;
#pragma unroll
    for (int a = 0; a < N1; ++a) acc += sS[0][a * N1 + m] * u[rest + a];
    t[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int m = (i / N1) % N1, rest = i - m * N1;
    V acc = 0;
#pragma unroll
    for (int b = 0; b < N1; ++b) acc += sS[1][b * N1 + m] * t[rest + b * N1];
    u[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int m = i / NF, rest = i - m * NF;
    V acc = 0;
#pragma unroll
    for (int c = 0; c < N1; ++c) acc += sS[2][c * N1 + m] * u[rest + c * NF];
    t[i] = acc / (sl[0][i % N1] + sl[1][(i / N1) % N1] + sl[2][m]);
  }
  __syncthreads();
  // back: u = (S_x (x) S_y (x) S_z) t
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int c = i / NF, rest = i - c * NF;
    V acc = 0;
#pragma unroll
    for (int m = 0; m < N1; ++m) acc += sS[2][c * N1 + m] * t[rest + m * NF];
    u[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int b = (i / N1) % N1, rest = i - b * N1;
    V acc = 0;
#pragma unroll
    for (int m = 0; m < N1; ++m) acc += sS[1][b * N1 + m] * u[rest + m * N1];
    t[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int a = i % N1, rest = i - a;
    V acc = 0;
#pragma unroll
    for (int m = 0; m < N1; ++m) acc += sS[0][a * N1 + m] * t[rest + m];
    z[off + i] = acc;
  }
}

// g[k][j] = sum_q W_q f_k(q) / |xb_j - x_q| (Sec. 6.3), direct quadrature. One
// thread per boundary node and BDK sources per block: 1 / |xb_j - x_q| is
// evaluated once for all the block's sources, so the cost per source is about
// one FMA per pair. The nodes x_q and the weighted sources are staged through
// shared memory; every sum runs over q in a fixed order. The reciprocal square
// root: the FP32 hardware estimate (rsqrtf) refined by one Newton-Raphson step
// y <- y (3 - d y^2) / 2 in FP64, which squares its relative error (about
// 2^-22 before, 1e-13 after) at four FP64 operations instead of an FP64 square
// root and division.
static constexpr int BDT = 128, BDQ = 128, BDK = 16;
__global__ void __launch_bounds__(BDT) k_oct_bdata(const double* __restrict__ xb, long long nbn,
                                                   const double* __restrict__ xq, const double* __restrict__ W,
                                                   const double* __restrict__ f, long long Nq, int nsrc,
                                                   double* __restrict__ part) {
  __shared__ double sx[BDQ], sy[BDQ], sz[BDQ], sw[BDK][BDQ];
  const long long j = (long long)blockIdx.x * BDT + threadIdx.x;
  const int k0 = blockIdx.z * BDK;
  const int nk = min(BDK, nsrc - k0);
  // this block's chunk of the nodes q (chunk count fixed by the mesh, not the batch)
  const long long per = (Nq + gridDim.y - 1) / gridDim.y;
  const long long qa = (long long)blockIdx.y * per, qb = min(Nq, qa + per);
  double px = 0.0, py = 0.0, pz = 0.0;
  if (j < nbn) {
    px = xb[3 * j];
    py = xb[3 * j + 1];
    pz = xb[3 * j + 2];
  }
  double acc[BDK];
#pragma unroll
  for (int k = 0; k < BDK; ++k) acc[k] = 0.0;
  for (long long q0 = qa; q0 < qb; q0 += BDQ) {
    const int nq = (int)std::min<long long>(BDQ, qb - q0);
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += BDT) {
      sx[i] = xq[3 * (q0 + i)];
      sy[i] = xq[3 * (q0 + i) + 1];
      sz[i] = xq[3 * (q0 + i) + 2];
    }
    for (int t = threadIdx.x; t < BDK * nq; t += BDT) {
      const int k = t / nq, i = t - k * nq;
      sw[k][i] = k < nk ? W[q0 + i] * f[(long long)(k0 + k) * Nq + q0 + i] : 0.0;
    }
    __syncthreads();
    for (int i = 0; i < nq; ++i) {
      const double dx = px - sx[i], dy = py - sy[i], dz = pz - sz[i];
      const double d2 = dx * dx + dy * dy + dz * dz;
      double y = (double)rsqrtf((float)d2);
      y = y * fma(-0.5, d2 * y * y, 1.5);
#pragma unroll
      for (int k = 0; k < BDK; ++k) acc[k] = fma(sw[k][i], y, acc[k]);
    }
  }
  if (j < nbn) {
    double* pc = part + (long long)blockIdx.y * nsrc * nbn;
#pragma unroll
    for (int k = 0; k < BDK; ++k)
      if (k < nk) pc[(long long)(k0 + k) * nbn + j] = acc[k];
  }
}

// g[k][j] = the chunks' partial sums added in chunk order
__global__ void k_oct_bdata_sum(const double* __restrict__ part, int nch, long long n, double* __restrict__ g) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(long long)c * n + t];
    g[t] = s;
  }
}

// kmat[q][j] = 1 / |xb_j - x_q| in FP32 (the mixed mode's boundary-data
// kernel matrix): FP64 distance, rsqrtf refined by one FP64 Newton step, then
// rounded to FP32
__global__ void k_oct_kmat(const double* __restrict__ xb, long long nbn, const double* __restrict__ xq,
                           long long Nq, float* __restrict__ kmat) {
  const long long n = Nq * nbn;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long q = t / nbn, j = t - q * nbn;
    const double dx = xb[3 * j] - xq[3 * q], dy = xb[3 * j + 1] - xq[3 * q + 1], dz = xb[3 * j + 2] - xq[3 * q + 2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    double y = (double)rsqrtf((float)d2);
    y = y * fma(-0.5, d2 * y * y, 1.5);
    kmat[t] = (float)y;
  }
}

// wf[k][q] = W_q f_k(q) in FP32 (the GEMM's left operand)
__global__ void k_oct_wf32(const double* __restrict__ W, const double* __restrict__ f, long long Nq, int nsrc,
                           float* __restrict__ wf) {
  const long long n = Nq * nsrc;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    wf[t] = (float)(W[t % Nq] * f[t]);
}

__global__ void k_oct_f2d(const float* __restrict__ a, long long n, double* __restrict__ b) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    b[t] = (double)a[t];
}

// node chunks of the boundary-data sum: about four blocks per SM of a GB300 for
// one source tile, at most 64
static int oct_bdata_chunks(long long nbn) {
  const long long bx = (nbn + BDT - 1) / BDT;
  return (int)std::max(1LL, std::min(64LL, (4LL * 152 + bx - 1) / bx));
}

// b[k] += Nitsche load of the boundary data on every boundary face of the leaf
// (one block per leaf with a boundary face and source; a leaf's faces are
// summed by one thread per node, so edges and corners take no races)
template <int N1>
__global__ void k_oct_lift(const int* __restrict__ bleaf, const double* __restrict__ lift1d,
                           const double* __restrict__ w, const double* __restrict__ g, long long nbn,
                           double* __restrict__ b, long long Nq) {
  constexpr int NPE = N1 * N1 * N1, NF = N1 * N1;
  const int* bl = bleaf + 7 * blockIdx.x;
  const int e = bl[0];
  const int k = blockIdx.y;
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int c3[3] = {i % N1, (i / N1) % N1, i / NF};
    double acc = 0.0;
    for (int f = 0; f < 6; ++f) {
      const int bf = bl[1 + f];
      if (bf < 0) continue;
      const int d = f >> 1, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
      const int a = c3[d], b0 = c3[t0], b1 = c3[t1];
      acc += lift1d[(long long)bf * N1 + a] * w[b0] * w[b1] * g[(long long)k * nbn + (long long)bf * NF + b0 + N1 * b1];
    }
    b[(long long)k * Nq + (long long)e * NPE + i] += acc;
  }
}

// per-source scalars: out = num / den, 0 and a breakdown flag (2) when den is not positive or not finite
__global__ void k_oct_ratio(const double* num, const double* den, double* out, const int* act, int nact, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nact) return;
  const int k = act[i];
  const double dn = den[k];
  if (!(dn > 0.0) || !isfinite(dn) || !isfinite(num[k])) {
    out[k] = 0.0;
    flags[k] |= 2;
  } else {
    out[k] = num[k] / dn;
  }
}

__global__ void k_oct_copy_slot(const double* src, double* dst, const int* act, int nact) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nact) dst[act[i]] = src[act[i]];
}

// r = b - q (the true residual once q = A x), and p = z, on the active sources
template <typename V>
__global__ void k_oct_sub(V* __restrict__ r, const V* __restrict__ b, const V* __restrict__ q, long long Nq,
                          const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
    r[off + i] = b[off + i] - q[off + i];
}
template <typename V>
__global__ void k_oct_copy(V* __restrict__ dst, const V* __restrict__ src, long long Nq,
                           const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
    dst[off + i] = src[off + i];
}


// p-transfers between octree levels, one leaf and source per block, sum-factorised
// with I [n1f][n1c] (the coarse basis at the fine nodes):
//   prolongation  xf += (I (x) I (x) I) xc,  restriction  rc = (I (x) I (x) I)^T rf
template <typename V>
__global__ void __launch_bounds__(128) k_oct_prolong_p(const double* __restrict__ I, int n1f, int n1c,
                                                       const V* __restrict__ xc, V* __restrict__ xf,
                                                       long long Nqc, long long Nqf, const int* __restrict__ act) {
  __shared__ V sI[MAXN1 * MAXN1], c0[MAXN1 * MAXN1 * MAXN1], t1[MAXN1 * MAXN1 * MAXN1], t2[MAXN1 * MAXN1 * MAXN1];
  const int e = blockIdx.x;
  const long long k = act[blockIdx.y];
  const int npc = n1c * n1c * n1c, npf = n1f * n1f * n1f;
  for (int i = threadIdx.x; i < n1f * n1c; i += blockDim.x) sI[i] = (V)I[i];
  for (int i = threadIdx.x; i < npc; i += blockDim.x) c0[i] = xc[k * Nqc + (long long)e * npc + i];
  __syncthreads();
  for (int t = threadIdx.x; t < n1c * n1c * n1f; t += blockDim.x) {  // t1[c'][b'][a]
    const int a = t % n1f, r = t / n1f;
    V acc = 0;
    for (int j = 0; j < n1c; ++j) acc += sI[a * n1c + j] * c0[r * n1c + j];
    t1[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n1c * n1f * n1f; t += blockDim.x) {  // t2[c'][b][a]
    const int a = t % n1f, b = (t / n1f) % n1f, c = t / (n1f * n1f);
    V acc = 0;
    for (int j = 0; j < n1c; ++j) acc += sI[b * n1c + j] * t1[(c * n1c + j) * n1f + a];
    t2[t] = acc;
  }
  __syncthreads();
  V* dst = xf + k * Nqf + (long long)e * npf;
  for (int t = threadIdx.x; t < npf; t += blockDim.x) {
    const int ab = t % (n1f * n1f), c = t / (n1f * n1f);
    V acc = 0;
    for (int j = 0; j < n1c; ++j) acc += sI[c * n1c + j] * t2[j * n1f * n1f + ab];
    dst[t] += acc;
  }
}

template <typename V>
__global__ void __launch_bounds__(128) k_oct_restrict_p(const double* __restrict__ I, int n1f, int n1c,
                                                        const V* __restrict__ rf, V* __restrict__ rc,
                                                        long long Nqf, long long Nqc, const int* __restrict__ act) {
  __shared__ V sI[MAXN1 * MAXN1], f0[MAXN1 * MAXN1 * MAXN1], t1[MAXN1 * MAXN1 * MAXN1], t2[MAXN1 * MAXN1 * MAXN1];
  const int e = blockIdx.x;
  const long long k = act[blockIdx.y];
  const int npc = n1c * n1c * n1c, npf = n1f * n1f * n1f;
  for (int i = threadIdx.x; i < n1f * n1c; i += blockDim.x) sI[i] = (V)I[i];
  for (int i = threadIdx.x; i < npf; i += blockDim.x) f0[i] = rf[k * Nqf + (long long)e * npf + i];
  __syncthreads();
  for (int t = threadIdx.x; t < n1f * n1f * n1c; t += blockDim.x) {  // t1[c][b][a']
    const int ac = t % n1c, r = t / n1c;
    V acc = 0;
    for (int a = 0; a < n1f; ++a) acc += sI[a * n1c + ac] * f0[r * n1f + a];
    t1[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n1f * n1c * n1c; t += blockDim.x) {  // t2[c][b'][a']
    const int ac = t % n1c, bc = (t / n1c) % n1c, c = t / (n1c * n1c);
    V acc = 0;
    for (int b = 0; b < n1f; ++b) acc += sI[b * n1c + bc] * t1[(c * n1f + b) * n1c + ac];
    t2[t] = acc;
  }
  __syncthreads();
  V* dst = rc + k * Nqc + (long long)e * npc;
  for (int t = threadIdx.x; t < npc; t += blockDim.x) {
    const int ab = t % (n1c * n1c), cc = t / (n1c * n1c);
    V acc = 0;
    for (int c = 0; c < n1f; ++c) acc += sI[c * n1c + cc] * t2[c * n1c * n1c + ab];
    dst[t] = acc;
  }
}

// degree-1 leaves <-> the degree-1 uniform root grid (each leaf lies in one
// root cell; the root field restricted to a leaf is degree 1 there, so the
// prolongation is exact): J[e][d][a][b] = root basis b at the leaf's node a
template <typename V>
__global__ void k_oct_prolong_root(const int* __restrict__ rcell, const double* __restrict__ J,
                                   const V* __restrict__ xr, V* __restrict__ xf, int E, long long Nqr,
                                   long long Nqf, const int* __restrict__ act) {
  const long long k = act[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < E * 8; t += gridDim.x * blockDim.x) {
    const int e = t >> 3, a = t & 1, b = (t >> 1) & 1, c = t >> 2 & 1;
    const double* Je = J + 12LL * e;
    const V* xe = xr + k * Nqr + 8LL * rcell[e];
    double acc = 0.0;
    for (int cc = 0; cc < 2; ++cc)
      for (int bb = 0; bb < 2; ++bb)
        for (int aa = 0; aa < 2; ++aa)
          acc += Je[0 + 2 * a + aa] * Je[4 + 2 * b + bb] * Je[8 + 2 * c + cc] * xe[aa + 2 * bb + 4 * cc];
    xf[k * Nqf + t] += (V)acc;
  }
}

template <typename V>
__global__ void k_oct_restrict_root(const int* __restrict__ rptr, const int* __restrict__ rlist,
                                    const double* __restrict__ J, const V* __restrict__ rf,
                                    V* __restrict__ rr, int nroot, long long Nqr, long long Nqf,
                                    const int* __restrict__ act) {
  const long long k = act[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nroot * 8; t += gridDim.x * blockDim.x) {
    const int rc = t >> 3, aa = t & 1, bb = (t >> 1) & 1, cc = t >> 2 & 1;
    double acc = 0.0;
    for (int i = rptr[rc]; i < rptr[rc + 1]; ++i) {
      const int e = rlist[i];
      const double* Je = J + 12LL * e;
      const V* re = rf + k * Nqf + 8LL * e;
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a)
            acc += Je[0 + 2 * a + aa] * Je[4 + 2 * b + bb] * Je[8 + 2 * c + cc] * re[a + 2 * b + 4 * c];
    }
    rr[k * Nqr + t] = (V)acc;
  }
}

}  // namespace dg

namespace dg {

template <typename V>
static cudaError_t launch_bjac(const dg_oct* h, const OctLevel& L, const V* r, V* z, const int* act, int nact,
                               cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  const dim3 grid((unsigned)h->E, (unsigned)nact);
  const int* c = L.cls.as<int>();
  const double *S = L.S.as<double>(), *l = L.lam.as<double>();
  count_launch();
  switch (L.n1) {
#define DG_BJ(N)                                                              \
  case N:                                                                     \
    k_oct_bjac<V, N><<<grid, 128, 0, s>>>(c, S, l, r, z, L.Nq, act);          \
    break;
    DG_BJ(2) DG_BJ(3) DG_BJ(4) DG_BJ(5) DG_BJ(6) DG_BJ(7) DG_BJ(8) DG_BJ(9)
#undef DG_BJ
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename V>
static cudaError_t oct_apply(const dg_oct* h, const OctLevel& L, const V* u, V* out, const int* act, int nact,
                             cudaStream_t s) {
  return launch_octree_apply<V>(L.n1, L.T, h->hq.as<double>(), h->kind.as<int>(), h->nb.as<int>(), h->pos.as<int>(),
                             h->E, L.p, h->pform, h->eps, u, out, act, nact, h->maxparts, s);
}

static cudaError_t launch_oct_lift(const dg_oct* h, const double* g, double* b, int nsrc, cudaStream_t s) {
  if (nsrc == 0 || h->nbl == 0) return cudaSuccess;
  const dim3 grid((unsigned)h->nbl, (unsigned)nsrc);
  const long long nbn = (long long)h->nbf * h->n1 * h->n1;
  const int* bl = h->bleaf.as<int>();
  const double* l1 = h->lift1d.as<double>();
  const double* w = h->wgl.as<double>();
  count_launch();
  switch (h->n1) {
#define DG_LF(N)                                                      \
  case N:                                                             \
    k_oct_lift<N><<<grid, 128, 0, s>>>(bl, l1, w, g, nbn, b, h->Nq);  \
    break;
    DG_LF(2) DG_LF(3) DG_LF(4) DG_LF(5) DG_LF(6) DG_LF(7) DG_LF(8) DG_LF(9)
#undef DG_LF
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// 1-D class of one leaf axis: the level and the types of its two faces
// (0 boundary, 1 same-size or larger neighbour, 2 four smaller neighbours)
using OctClass = std::tuple<int, int, int, int>;  // axis, level, type of the -d face, type of the +d face

// (S, lambda) of a class: K S = M S Lambda with S^T M S = I (see the file head)
static void oct_class_fdm(const OctTables& T, int n1, int p, double h, int ty0, int ty1, int pform, double eps,
                          double* S, double* lam) {
  std::vector<double> K((size_t)n1 * n1);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n1; ++b) K[(size_t)a * n1 + b] = (2.0 / h) * T.S[a * n1 + b];
  for (int r = 0; r < 2; ++r) {
    const int ty = r ? ty1 : ty0;
    const double e = r ? 1.0 : -1.0;
    const double c = ty == 0 ? 1.0 : 0.5;
    const double sig = penalty(p, ty == 2 ? h / 2.0 : h, pform, eps);
    for (int a = 0; a < n1; ++a)
      for (int b = 0; b < n1; ++b)
        K[(size_t)a * n1 + b] += -c * (2.0 / h) * e * (T.Le[r][a] * T.dLe[r][b] + T.dLe[r][a] * T.Le[r][b]) +
                                 sig * T.Le[r][a] * T.Le[r][b];
  }
  std::vector<double> mi(n1), C((size_t)n1 * n1), l, V;
  for (int a = 0; a < n1; ++a) mi[a] = 1.0 / std::sqrt(0.5 * h * T.w[a]);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n1; ++b) C[(size_t)a * n1 + b] = mi[a] * K[(size_t)a * n1 + b] * mi[b];
  sym_eig(C, n1, l, V);
  for (int a = 0; a < n1; ++a)
    for (int m = 0; m < n1; ++m) S[(size_t)a * n1 + m] = mi[a] * V[(size_t)a * n1 + m];
  for (int m = 0; m < n1; ++m) lam[m] = l[m];
}

static int oct_ws(dg_oct* h, int cap) {
  if (cap <= h->cap) return DG_OK;
  const size_t vec = sizeof(double) * (size_t)cap * (size_t)h->Nq;
  for (DevBuf* v : {&h->f, &h->b, &h->x, &h->r, &h->z, &h->pv, &h->qv}) DG_CK(v->ensure(vec));
  for (size_t l = 0; l < h->lv.size(); ++l) {
    OctLevel& L = h->lv[l];
    const size_t lvec = sizeof(double) * (size_t)cap * (size_t)L.Nq;
    for (DevBuf* v : {&L.res, &L.d, &L.z, &L.q}) DG_CK(v->ensure(lvec));
    if (l > 0)
      for (DevBuf* v : {&L.x, &L.b}) DG_CK(v->ensure(lvec));
  }
  if (h->mixed) {
    const size_t v32 = sizeof(float) * (size_t)cap * (size_t)h->Nq;
    for (DevBuf* v : {&h->b32, &h->x32, &h->r32, &h->z32, &h->p32, &h->q32}) DG_CK(v->ensure(v32));
    if (h->has_kmat) {
      const size_t nbn = (size_t)h->nbf * h->n1 * h->n1;
      DG_CK(h->wf32.ensure(v32));
      DG_CK(h->g32.ensure(sizeof(float) * (size_t)cap * nbn));
      DG_CK(h->gwork.ensure(sizeof(float) * 32 * (size_t)cap * nbn));
    }
  }
  if (h->root) {
    DG_CK(h->rb.ensure(sizeof(double) * (size_t)cap * (size_t)h->Nq_root));
    DG_CK(h->rx.ensure(sizeof(double) * (size_t)cap * (size_t)h->Nq_root));
    int rc = prepare(h->root, cap);
    if (rc == DG_OK && h->mixed) rc = ensure_prec<float>(h->root, h->root->w32, cap);
    if (rc != DG_OK) {
      h->err = "root-grid workspace: " + h->root->err;
      return rc;
    }
  }
  DG_CK(h->g.ensure(sizeof(double) * (size_t)cap * h->nbf * h->n1 * h->n1));
  DG_CK(h->gpart.ensure(sizeof(double) * (size_t)oct_bdata_chunks((long long)h->nbf * h->n1 * h->n1) * cap * h->nbf *
                        h->n1 * h->n1));
  DG_CK(h->scal.ensure(sizeof(double) * O_NSLOT * (size_t)cap));
  DG_CK(h->part.ensure(sizeof(double) * 304 * (size_t)cap));
  DG_CK(h->act.ensure(sizeof(int) * (size_t)cap));
  DG_CK(h->flags.ensure(sizeof(int) * (size_t)cap));
  DG_CK(h->pidx.ensure(sizeof(int) * 2 * (size_t)cap));
  h->act_host.clear();
  h->cap = cap;
  return DG_OK;
}

static inline double* oslot(dg_oct* h, int i) { return h->scal.as<double>() + (size_t)i * h->cap; }

static int oct_act(dg_oct* h, const std::vector<int>& a, cudaStream_t s) {
  if (a.empty() || a == h->act_host) return DG_OK;
  h->act_host = a;
  DG_CK(cudaMemcpyAsync(h->act.p, h->act_host.data(), sizeof(int) * a.size(), cudaMemcpyHostToDevice, s));
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

// b[k] = 4 pi W f_k + the Nitsche load of f_k's Coulomb boundary data, k < nsrc
static int oct_form_rhs(dg_oct* h, const double* f, int nsrc, cudaStream_t s) {
  const long long nbn = (long long)h->nbf * h->n1 * h->n1;
  if (h->mixed && h->has_kmat) {
    // G = (W f) K: 3xTF32 tensor-core GEMM (M sources, N boundary nodes, K nodes)
    const unsigned gb = (unsigned)std::min<long long>(152LL * 16, (h->Nq * nsrc + 255) / 256);
    count_launch();
    k_oct_wf32<<<gb, 256, 0, s>>>(h->W.as<double>(), f, h->Nq, nsrc, h->wf32.as<float>());
    DG_CK(cudaGetLastError());
    GemmArgs ga{};
    ga.M = nsrc;
    ga.N = (int)nbn;
    ga.K = (int)h->Nq;
    ga.nb1 = ga.nb2 = 1;
    ga.A = h->wf32.p;
    ga.sAm = h->Nq;
    ga.sAk = 1;
    ga.B = h->kmat.p;
    ga.sBk = nbn;
    ga.sBn = 1;
    ga.C = h->g32.p;
    ga.sCm = nbn;
    ga.sCn = 1;
    ga.alpha = 1.0;
    ga.beta = 0.0;
    ga.work = h->gwork.p;
    ga.work_elems = 32LL * h->cap * nbn;
    DG_CK(launch_gemm<float>(ga, s));
    count_launch();
    k_oct_f2d<<<(unsigned)std::min<long long>(4096, (nsrc * nbn + 255) / 256), 256, 0, s>>>(
        h->g32.as<float>(), nsrc * nbn, h->g.as<double>());
    DG_CK(cudaGetLastError());
    DG_CK(launch_rhs_volume(f, h->W.as<double>(), h->b.as<double>(), h->Nq, nsrc, s));
    DG_CK(launch_oct_lift(h, h->g.as<double>(), h->b.as<double>(), nsrc, s));
    return DG_OK;
  }
  count_launch();
  const int nch = oct_bdata_chunks(nbn);
  k_oct_bdata<<<dim3((unsigned)((nbn + BDT - 1) / BDT), (unsigned)nch, (unsigned)((nsrc + BDK - 1) / BDK)), BDT, 0,
                s>>>(h->xb.as<double>(), nbn, h->xq.as<double>(), h->W.as<double>(), f, h->Nq, nsrc,
                     h->gpart.as<double>());
  DG_CK(cudaGetLastError());
  count_launch();
  k_oct_bdata_sum<<<(unsigned)std::min<long long>(4096, (nsrc * nbn + 255) / 256), 256, 0, s>>>(
      h->gpart.as<double>(), nch, nsrc * nbn, h->g.as<double>());
  DG_CK(cudaGetLastError());
  DG_CK(launch_rhs_volume(f, h->W.as<double>(), h->b.as<double>(), h->Nq, nsrc, s));
  DG_CK(launch_oct_lift(h, h->g.as<double>(), h->b.as<double>(), nsrc, s));
  return DG_OK;
}

// finite[k] = 1 when f_k holds no NaN or infinity
static int oct_finite(dg_oct* h, const double* f, int nsrc, std::vector<int>& finite, cudaStream_t s) {
  DG_CK(cudaMemsetAsync(h->flags.p, 0, sizeof(int) * nsrc, s));
  DG_CK(launch_finite_flags(f, h->Nq, nsrc, h->flags.as<int>(), s));
  std::vector<int> fl(nsrc);
  DG_CK(cudaMemcpyAsync(fl.data(), h->flags.p, sizeof(int) * nsrc, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  finite.assign(nsrc, 1);
  for (int k = 0; k < nsrc; ++k) finite[k] = fl[k] == 0;
  return DG_OK;
}


// Chebyshev smoothing of A x = b on octree level l: the semi-iteration on
// P^-1 A (P the leaf-block preconditioner) over [lambda / range, lambda],
// lambda = 1.1 x the level's power-iteration estimate. On exit, if want_res,
// the level's res holds b - A x.
template <typename V>
static int oct_cheb(dg_oct* h, int l, const V* b, V* x, bool zero_init, bool want_res, const int* act, int n,
                    cudaStream_t s) {
  OctLevel& L = h->lv[l];
  V *res = L.res.as<V>(), *d = L.d.as<V>(), *z = L.z.as<V>(), *q = L.q.as<V>();
  const double bmax = 1.1 * L.lam_max, amin = bmax / h->cheb_range;
  const double theta = 0.5 * (bmax + amin), delta = 0.5 * (bmax - amin), sig1 = theta / delta;
  const dim3 vg = ogrid(L.Nq, n);
  auto resid = [&]() -> int {
    DG_CK(oct_apply(h, L, x, q, act, n, s));
    count_launch();
    k_oct_sub<<<vg, OT, 0, s>>>(res, b, q, L.Nq, act);
    DG_CK(cudaGetLastError());
    return DG_OK;
  };
  const V* r0 = b;
  if (!zero_init) {
    DG_RET(resid());
    r0 = res;
  }
  DG_CK(launch_bjac(h, L, r0, z, act, n, s));
  DG_CK(launch_cheb_first<V>(x, d, z, nullptr, 1.0 / theta, zero_init ? 1 : 0, L.Nq, act, n, s));
  double rho_prev = 1.0 / sig1;
  for (int j = 2; j <= h->cheb_k; ++j) {
    DG_RET(resid());
    const double rho = 1.0 / (2.0 * sig1 - rho_prev);
    DG_CK(launch_bjac(h, L, res, z, act, n, s));
    DG_CK(launch_cheb_step<V>(x, d, z, nullptr, rho * rho_prev, 2.0 * rho / delta, L.Nq, act, n, s));
    rho_prev = rho;
  }
  if (want_res) DG_RET(resid());
  return DG_OK;
}

// x = V(b) on octree level l (x overwritten): smoothing, restriction to the
// next coarser degree (or, from degree 1, to the uniform root grid and its own
// V-cycle), prolongation of the correction, smoothing
template <typename V>
static int oct_vcycle(dg_oct* h, int l, const V* b, V* x, const int* act, int n, cudaStream_t s) {
  OctLevel& L = h->lv[l];
  DG_RET(oct_cheb<V>(h, l, b, x, true, true, act, n, s));
  const V* res = L.res.as<V>();
  if (l + 1 < (int)h->lv.size()) {
    OctLevel& C = h->lv[l + 1];
    count_launch();
    k_oct_restrict_p<V><<<dim3((unsigned)h->E, (unsigned)n), 128, 0, s>>>(L.I.as<double>(), L.n1, C.n1, res,
                                                                           C.b.as<V>(), L.Nq, C.Nq, act);
    DG_CK(cudaGetLastError());
    DG_RET(oct_vcycle<V>(h, l + 1, C.b.as<V>(), C.x.as<V>(), act, n, s));
    count_launch();
    k_oct_prolong_p<V><<<dim3((unsigned)h->E, (unsigned)n), 128, 0, s>>>(L.I.as<double>(), L.n1, C.n1, C.x.as<V>(),
                                                                          x, C.Nq, L.Nq, act);
    DG_CK(cudaGetLastError());
  } else {
    const unsigned gr = (unsigned)std::min<long long>(4096, (h->n_root * 8LL + 255) / 256);
    count_launch();
    k_oct_restrict_root<V><<<dim3(gr, (unsigned)n), 256, 0, s>>>(h->rptr.as<int>(), h->rlist.as<int>(),
                                                                  h->rJ.as<double>(), res, h->rb.as<V>(),
                                                                  h->n_root, h->Nq_root, L.Nq, act);
    DG_CK(cudaGetLastError());
    PrecWork<V>* w;
    if constexpr (sizeof(V) == 4)
      w = &h->root->w32;
    else
      w = &h->root->w64;
    MG<V> mg{h->root, w, act, n, s};
    const int rc = mg.vcycle(0, h->rb.as<V>(), h->rx.as<V>());
    if (rc != DG_OK) {
      h->err = "root-grid V-cycle: " + h->root->err;
      return rc;
    }
    const unsigned ge = (unsigned)std::min<long long>(4096, (h->E * 8LL + 255) / 256);
    count_launch();
    k_oct_prolong_root<V><<<dim3(ge, (unsigned)n), 256, 0, s>>>(h->rcell.as<int>(), h->rJ.as<double>(),
                                                                 h->rx.as<V>(), x, h->E, h->Nq_root, L.Nq, act);
    DG_CK(cudaGetLastError());
  }
  DG_RET(oct_cheb<V>(h, l, b, x, false, false, act, n, s));
  return DG_OK;
}

// z = M r: the V-cycle (precond 1) or the leaf-block inverse (precond 0)
template <typename V>
static int oct_precond(dg_oct* h, const V* r, V* z, const int* act, int n, cudaStream_t s) {
  if (h->precond == 0) {
    DG_CK(launch_bjac<V>(h, h->lv[0], r, z, act, n, s));
    return DG_OK;
  }
  return oct_vcycle<V>(h, 0, r, z, act, n, s);
}

// lambda_max(P^-1 A) of level l by 30 power iterations from a fixed
// pseudo-random start (one field, the level's workspace of source 0)
static int oct_lambda(dg_oct* h, int l, cudaStream_t s) {
  OctLevel& L = h->lv[l];
  std::vector<double> v(L.Nq);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  for (auto& x : v) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    x = double((st >> 11) & ((1ull << 53) - 1)) / double(1ull << 53) - 0.5;
  }
  double *x = L.d.as<double>(), *q = L.q.as<double>(), *z = L.z.as<double>();
  DG_CK(cudaMemcpyAsync(x, v.data(), sizeof(double) * L.Nq, cudaMemcpyHostToDevice, s));
  DG_RET(oct_act(h, std::vector<int>{0}, s));
  const int* act = h->act.as<int>();
  double* nrm = oslot(h, O_SE);
  double lam = 0.0, nz = 0.0, nx = 0.0;
  DG_CK(launch_dot(x, x, (const double*)nullptr, nrm, h->part.as<double>(), L.Nq, act, 1, s));
  DG_CK(cudaMemcpyAsync(&nx, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  for (int it = 0; it < 30; ++it) {
    DG_CK(oct_apply(h, L, x, q, act, 1, s));
    DG_CK(launch_bjac(h, L, q, z, act, 1, s));
    DG_CK(launch_dot(z, z, (const double*)nullptr, nrm, h->part.as<double>(), L.Nq, act, 1, s));
    DG_CK(cudaMemcpyAsync(&nz, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
    if (!(nz > 0.0) || !std::isfinite(nz)) {
      h->err = "power iteration of the smoother bound broke down";
      return DG_ERR_BREAKDOWN;
    }
    lam = std::sqrt(nz / nx);
    DG_CK(cudaMemcpyAsync(x, z, sizeof(double) * L.Nq, cudaMemcpyDeviceToDevice, s));
    DG_CK(launch_scale(x, L.Nq, 1.0 / std::sqrt(nz), s));
    nx = 1.0;
  }
  L.lam_max = lam;
  return DG_OK;
}

}  // namespace dg

namespace dg {

// PCG on the sources 0..nsrc-1 of the workspace (b formed): x = A^-1 b to the
// FP64 relative residual rtol. Convergence of the recursive residual is
// confirmed on the true residual b - A x; where the two disagree the
// iteration restarts from the true residual (at most 3 times per source).
static int oct_pcg_mixed(dg_oct* h, int nsrc, const std::vector<int>& finite, std::vector<dg_solve_stats>& st,
                         cudaStream_t s);

static int oct_pcg(dg_oct* h, int nsrc, const std::vector<int>& finite, std::vector<dg_solve_stats>& st,
                   cudaStream_t s) {
  if (h->mixed) return oct_pcg_mixed(h, nsrc, finite, st, s);
  const long long Nq = h->Nq;
  double *b = h->b.as<double>(), *x = h->x.as<double>(), *r = h->r.as<double>(), *z = h->z.as<double>();
  double *p = h->pv.as<double>(), *q = h->qv.as<double>(), *part = h->part.as<double>();
  int* flags = h->flags.as<int>();
  const int* act = h->act.as<int>();
  st.assign(nsrc, dg_solve_stats{});
  DG_CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)nsrc * Nq, s));
  DG_CK(cudaMemsetAsync(flags, 0, sizeof(int) * nsrc, s));
  std::vector<int> all;
  for (int k = 0; k < nsrc; ++k) {
    st[k].guess_rel_residual = 1.0;
    if (finite[k])
      all.push_back(k);
    else
      st[k].status = DG_ERR_NONFINITE;
  }
  if (all.empty()) return DG_OK;
  const dim3 vg = ogrid(Nq, 1);
  auto vgrid_n = [&](int n) { return dim3(vg.x, (unsigned)n); };
  // true residual of the sources in `a` into r, its squared norm into O_RR (host: rt)
  std::vector<double> bb(h->cap), rr(h->cap);
  std::vector<int> fl(h->cap);
  auto true_residual = [&](const std::vector<int>& a) -> int {
    DG_RET(oct_act(h, a, s));
    const int n = (int)a.size();
    DG_CK(oct_apply(h, h->lv[0], x, q, act, n, s));
    count_launch();
    k_oct_sub<<<vgrid_n(n), OT, 0, s>>>(r, b, q, Nq, act);
    DG_CK(cudaGetLastError());
    DG_CK(launch_dot(r, r, (const double*)nullptr, oslot(h, O_RR), part, Nq, act, n, s));
    DG_CK(cudaMemcpyAsync(rr.data(), oslot(h, O_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
    return DG_OK;
  };
  // r = b, z = P r, p = z, rz = (r, z), bb = (b, b)
  DG_RET(oct_act(h, all, s));
  int n = (int)all.size();
  count_launch();
  k_oct_copy<<<vgrid_n(n), OT, 0, s>>>(r, b, Nq, act);
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot(b, b, (const double*)nullptr, oslot(h, O_BB), part, Nq, act, n, s));
  DG_RET(oct_precond(h, r, z, act, n, s));
  count_launch();
  k_oct_copy<<<vgrid_n(n), OT, 0, s>>>(p, z, Nq, act);
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot(r, z, (const double*)nullptr, oslot(h, O_RZ), part, Nq, act, n, s));
  DG_CK(cudaMemcpyAsync(bb.data(), oslot(h, O_BB), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  std::vector<int> active, restarts(nsrc, 0);
  for (int k : all)
    if (bb[k] > 0.0)
      active.push_back(k);  // a zero right-hand side has the solution x = 0
  const double rtol = h->rtol;
  for (int it = 1; it <= h->max_iter && !active.empty(); ++it) {
    DG_RET(oct_act(h, active, s));
    n = (int)active.size();
    DG_CK(oct_apply(h, h->lv[0], p, q, act, n, s));
    DG_CK(launch_dot(p, q, (const double*)nullptr, oslot(h, O_PQ), part, Nq, act, n, s));
    count_launch();
    k_oct_ratio<<<(n + 127) / 128, 128, 0, s>>>(oslot(h, O_RZ), oslot(h, O_PQ), oslot(h, O_AL), act, n, flags);
    DG_CK(cudaGetLastError());
    DG_CK(launch_cg_xr(x, r, p, q, oslot(h, O_AL), Nq, act, n, s));
    DG_CK(launch_dot(r, r, (const double*)nullptr, oslot(h, O_RR), part, Nq, act, n, s));
    DG_CK(cudaMemcpyAsync(rr.data(), oslot(h, O_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaMemcpyAsync(fl.data(), flags, sizeof(int) * nsrc, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
    std::vector<int> cand, next, restart;
    for (int k : active) {
      st[k].iters = it;
      if (fl[k] & 2) {
        st[k].status = DG_ERR_BREAKDOWN;
        st[k].rel_residual = std::sqrt(rr[k] / bb[k]);
      } else if (std::sqrt(rr[k] / bb[k]) <= rtol) {
        cand.push_back(k);
      } else {
        next.push_back(k);
      }
    }
    if (!cand.empty()) {
      DG_RET(true_residual(cand));
      for (int k : cand) {
        const double rel = std::sqrt(rr[k] / bb[k]);
        st[k].rel_residual = rel;
        if (rel <= rtol) continue;
        if (restarts[k] < 3) {
          ++restarts[k];
          restart.push_back(k);
          next.push_back(k);
        } else {
          st[k].status = DG_ERR_NOT_CONVERGED;
        }
      }
    }
    std::sort(next.begin(), next.end());
    active = next;
    if (active.empty()) break;
    // z = P r, beta = (r, z) / rz, rz = (r, z), p = z + beta p (beta = 0 on a restart)
    DG_RET(oct_act(h, active, s));
    n = (int)active.size();
    DG_RET(oct_precond(h, r, z, act, n, s));
    DG_CK(launch_dot(r, z, (const double*)nullptr, oslot(h, O_RZN), part, Nq, act, n, s));
    count_launch();
    k_oct_ratio<<<(n + 127) / 128, 128, 0, s>>>(oslot(h, O_RZN), oslot(h, O_RZ), oslot(h, O_BE), act, n, flags);
    DG_CK(cudaGetLastError());
    count_launch();
    k_oct_copy_slot<<<(n + 127) / 128, 128, 0, s>>>(oslot(h, O_RZN), oslot(h, O_RZ), act, n);
    DG_CK(cudaGetLastError());
    for (int k : restart) DG_CK(cudaMemsetAsync(oslot(h, O_BE) + k, 0, sizeof(double), s));
    DG_CK(launch_cg_p(p, z, oslot(h, O_BE), Nq, act, n, s));
  }
  if (!active.empty()) {  // iteration limit
    DG_RET(true_residual(active));
    for (int k : active) {
      st[k].rel_residual = std::sqrt(rr[k] / bb[k]);
      if (st[k].rel_residual > rtol) st[k].status = DG_ERR_NOT_CONVERGED;
    }
  }
  return DG_OK;
}

// Inner PCG in precision V (the FP32 inner solve of the mixed mode) on the
// sources `srcs`: x = A^-1 b from x = 0 until the recursive residual falls by
// itol or imax iterations; iters[k] += the iterations of source k
template <typename V>
static int oct_cg_inner(dg_oct* h, const V* b, V* x, V* r, V* z, V* p, V* q, const std::vector<int>& srcs,
                        double itol, int imax, std::vector<int>& iters, cudaStream_t s) {
  const long long Nq = h->Nq;
  double* part = h->part.as<double>();
  int* flags = h->flags.as<int>();
  const int* act = h->act.as<int>();
  const dim3 vg = ogrid(Nq, 1);
  std::vector<double> bb(h->cap), rr(h->cap);
  std::vector<int> fl(h->cap);
  DG_RET(oct_act(h, srcs, s));
  int n = (int)srcs.size();
  DG_CK(launch_zero<V>(x, Nq, act, n, s));
  count_launch();
  k_oct_copy<V><<<dim3(vg.x, (unsigned)n), OT, 0, s>>>(r, b, Nq, act);
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot<V>(b, b, (const double*)nullptr, oslot(h, I_BB), part, Nq, act, n, s));
  DG_RET(oct_precond<V>(h, r, z, act, n, s));
  count_launch();
  k_oct_copy<V><<<dim3(vg.x, (unsigned)n), OT, 0, s>>>(p, z, Nq, act);
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot<V>(r, z, (const double*)nullptr, oslot(h, I_RZ), part, Nq, act, n, s));
  DG_CK(cudaMemcpyAsync(bb.data(), oslot(h, I_BB), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  std::vector<int> active;
  for (int k : srcs)
    if (bb[k] > 0.0) active.push_back(k);
  for (int it = 1; it <= imax && !active.empty(); ++it) {
    DG_RET(oct_act(h, active, s));
    n = (int)active.size();
    DG_CK(oct_apply<V>(h, h->lv[0], p, q, act, n, s));
    DG_CK(launch_dot<V>(p, q, (const double*)nullptr, oslot(h, I_PQ), part, Nq, act, n, s));
    count_launch();
    k_oct_ratio<<<(n + 127) / 128, 128, 0, s>>>(oslot(h, I_RZ), oslot(h, I_PQ), oslot(h, I_AL), act, n, flags);
    DG_CK(cudaGetLastError());
    DG_CK(launch_cg_xr<V>(x, r, p, q, oslot(h, I_AL), Nq, act, n, s));
    DG_CK(launch_dot<V>(r, r, (const double*)nullptr, oslot(h, I_RR), part, Nq, act, n, s));
    DG_CK(cudaMemcpyAsync(rr.data(), oslot(h, I_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaMemcpyAsync(fl.data(), flags, sizeof(int) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
    std::vector<int> next;
    for (int k : active) {
      ++iters[k];
      if (!(fl[k] & 2) && rr[k] > itol * itol * bb[k]) next.push_back(k);
    }
    active = next;
    if (active.empty()) break;
    DG_RET(oct_act(h, active, s));
    n = (int)active.size();
    DG_RET(oct_precond<V>(h, r, z, act, n, s));
    DG_CK(launch_dot<V>(r, z, (const double*)nullptr, oslot(h, I_RZN), part, Nq, act, n, s));
    count_launch();
    k_oct_ratio<<<(n + 127) / 128, 128, 0, s>>>(oslot(h, I_RZN), oslot(h, I_RZ), oslot(h, I_BE), act, n, flags);
    DG_CK(cudaGetLastError());
    count_launch();
    k_oct_copy_slot<<<(n + 127) / 128, 128, 0, s>>>(oslot(h, I_RZN), oslot(h, I_RZ), act, n);
    DG_CK(cudaGetLastError());
    DG_CK(launch_cg_p<V>(p, z, oslot(h, I_BE), Nq, act, n, s));
  }
  return DG_OK;
}

// Mixed mode: FP64 iterative refinement around the FP32 inner PCG. Each round
// takes the FP64 residual r = b - A x in FP32, solves A e = r to a reduction
// of inner_rtol, adds e to x in FP64 and recomputes the FP64 residual; a
// source stops when that residual meets rtol (at most 30 rounds).
static int oct_pcg_mixed(dg_oct* h, int nsrc, const std::vector<int>& finite, std::vector<dg_solve_stats>& st,
                         cudaStream_t s) {
  const long long Nq = h->Nq;
  double *b = h->b.as<double>(), *x = h->x.as<double>(), *r = h->r.as<double>(), *q = h->qv.as<double>();
  double* part = h->part.as<double>();
  const int* act = h->act.as<int>();
  st.assign(nsrc, dg_solve_stats{});
  DG_CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)nsrc * Nq, s));
  DG_CK(cudaMemsetAsync(h->flags.p, 0, sizeof(int) * nsrc, s));
  std::vector<int> all;
  for (int k = 0; k < nsrc; ++k) {
    st[k].guess_rel_residual = 1.0;
    if (finite[k])
      all.push_back(k);
    else
      st[k].status = DG_ERR_NONFINITE;
  }
  if (all.empty()) return DG_OK;
  const dim3 vg = ogrid(Nq, 1);
  std::vector<double> bb(h->cap), rr(h->cap);
  DG_RET(oct_act(h, all, s));
  int n = (int)all.size();
  count_launch();
  k_oct_copy<double><<<dim3(vg.x, (unsigned)n), OT, 0, s>>>(r, b, Nq, act);
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot<double>(b, b, (const double*)nullptr, oslot(h, O_BB), part, Nq, act, n, s));
  DG_CK(cudaMemcpyAsync(bb.data(), oslot(h, O_BB), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  std::vector<int> active, iters(h->cap, 0);
  for (int k : all)
    if (bb[k] > 0.0) active.push_back(k);
  for (int round = 1; round <= 30 && !active.empty(); ++round) {
    DG_RET(oct_act(h, active, s));
    n = (int)active.size();
    DG_CK((launch_convert<float, double>(h->b32.as<float>(), r, Nq, act, n, 1.0, 0, s)));
    DG_RET(oct_cg_inner<float>(h, h->b32.as<float>(), h->x32.as<float>(), h->r32.as<float>(), h->z32.as<float>(),
                               h->p32.as<float>(), h->q32.as<float>(), active, h->inner_rtol, h->max_iter, iters, s));
    DG_RET(oct_act(h, active, s));
    DG_CK((launch_convert<double, float>(x, h->x32.as<float>(), Nq, act, n, 1.0, 1, s)));
    DG_CK(oct_apply<double>(h, h->lv[0], x, q, act, n, s));
    count_launch();
    k_oct_sub<double><<<dim3(vg.x, (unsigned)n), OT, 0, s>>>(r, b, q, Nq, act);
    DG_CK(cudaGetLastError());
    DG_CK(launch_dot<double>(r, r, (const double*)nullptr, oslot(h, O_RR), part, Nq, act, n, s));
    DG_CK(cudaMemcpyAsync(rr.data(), oslot(h, O_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
    std::vector<int> next;
    for (int k : active) {
      st[k].outer_refinements = round;
      st[k].iters = iters[k];
      st[k].rel_residual = std::sqrt(rr[k] / bb[k]);
      if (!(st[k].rel_residual <= h->rtol)) next.push_back(k);
    }
    active = next;
  }
  for (int k : active) st[k].status = DG_ERR_NOT_CONVERGED;
  return DG_OK;
}

static int worst_of(const std::vector<dg_solve_stats>& st) {
  int w = DG_OK;
  for (const auto& x : st)
    if (x.status != DG_OK && (w == DG_OK || x.status < w)) w = x.status;
  return w;
}

// self-energies (f|f) = sum_q W_q f v of the chunk's sources
static int oct_self_energies(dg_oct* h, const double* f, int nsrc, std::vector<dg_solve_stats>& st, cudaStream_t s) {
  std::vector<int> a(nsrc);
  for (int k = 0; k < nsrc; ++k) a[k] = k;
  DG_RET(oct_act(h, a, s));
  DG_CK(launch_dot(f, h->x.as<double>(), h->W.as<double>(), oslot(h, O_SE), h->part.as<double>(), h->Nq,
                   h->act.as<int>(), nsrc, s));
  std::vector<double> se(nsrc);
  DG_CK(cudaMemcpyAsync(se.data(), oslot(h, O_SE), sizeof(double) * nsrc, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nsrc; ++k) st[k].self_energy = st[k].status == DG_ERR_NONFINITE ? 0.0 : se[k];
  return DG_OK;
}

static int oct_cap(const dg_oct* h, long long want) {
  // per source: seven fine-level PCG vectors, four smoother vectors per level
  // and two more on the coarser ones; at most about 4 GB, at most 64 sources
  long long per = 7LL * h->Nq;
  for (size_t l = 0; l < h->lv.size(); ++l) per += (l == 0 ? 4LL : 6LL) * h->lv[l].Nq;
  per *= (long long)sizeof(double);
  if (h->mixed) per += 6LL * h->Nq * (long long)sizeof(float);
  long long c = std::max(1LL, std::min(64LL, (4LL << 30) / std::max(1LL, per)));
  return (int)std::max(1LL, std::min(c, want));
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_octree_setup(const dg_mesh_desc* root, const int32_t* leaves, int32_t n_leaves, int32_t penalty_form,
                    double penalty_eps, double rtol, int32_t max_iter, int32_t precond, int32_t precision,
                    dg_oct_handle* out) {
  if (!out) return DG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!root || !leaves || n_leaves < 1 || root->p < 1 || root->p > MAXN1 - 1 ||
      (penalty_form != 0 && penalty_form != 1) || !(penalty_eps > 0.0) || !(rtol > 0.0) || !(rtol < 1.0) ||
      max_iter < 1 || (precond != 0 && precond != 1) || (precision != DG_PREC_FP64 && precision != DG_PREC_MIXED))
    return DG_ERR_INVALID_ARG;
  const int E = n_leaves, n1 = root->p + 1, NPE = n1 * n1 * n1, NF = n1 * n1;
  std::vector<int32_t> kind(6 * (size_t)E), nb(24 * (size_t)E), pos(6 * (size_t)E);
  if (!octree_faces(root, leaves, n_leaves, kind.data(), nb.data(), pos.data())) return DG_ERR_INVALID_ARG;
  if ((long long)E * NPE > (1LL << 31)) return DG_ERR_UNSUPPORTED;
  const long long n_root = (long long)root->n[0] * root->n[1] * root->n[2];
  DeviceWideGuard guard;
  dg_oct* h = new dg_oct();
  h->n1 = n1;
  h->p = root->p;
  h->E = E;
  h->pform = penalty_form;
  h->eps = penalty_eps;
  h->rtol = rtol;
  h->max_iter = max_iter;
  h->precond = precond;
  h->mixed = precision == DG_PREC_MIXED;
  h->maxparts = octree_max_parts(kind.data(), E);
  h->Nq = (long long)E * NPE;
  double xi[MAXN1], w[MAXN1];
  gauss_legendre(n1, xi, w);
  // sizes, origins, nodes and weights
  std::vector<double> hq(3 * (size_t)E), org(3 * (size_t)E), xq(3 * (size_t)h->Nq), W(h->Nq);
  for (int e = 0; e < E; ++e)
    for (int d = 0; d < 3; ++d) {
      hq[3 * (size_t)e + d] = (root->hi[d] - root->lo[d]) / root->n[d] / double(1 << leaves[4 * e]);
      org[3 * (size_t)e + d] = root->lo[d] + leaves[4 * e + 1 + d] * hq[3 * (size_t)e + d];
    }
  for (int e = 0; e < E; ++e) {
    const double* hh = &hq[3 * (size_t)e];
    const double* o = &org[3 * (size_t)e];
    for (int i = 0; i < NPE; ++i) {
      const int a = i % n1, b = (i / n1) % n1, c = i / NF;
      const size_t qi = (size_t)e * NPE + i;
      xq[3 * qi + 0] = o[0] + (xi[a] + 1.0) * hh[0] / 2.0;
      xq[3 * qi + 1] = o[1] + (xi[b] + 1.0) * hh[1] / 2.0;
      xq[3 * qi + 2] = o[2] + (xi[c] + 1.0) * hh[2] / 2.0;
      W[qi] = w[a] * w[b] * w[c] * hh[0] * hh[1] * hh[2] / 8.0;
    }
  }
  auto up = [&](DevBuf& dst, const void* src, size_t bytes) -> int {
    DG_CK(dst.ensure(std::max<size_t>(bytes, 16)));
    DG_CK(cudaMemcpy(dst.p, src, bytes, cudaMemcpyHostToDevice));
    return DG_OK;
  };
  int rc = DG_OK;
  auto fail = [&](int code) {
    delete h;
    return code;
  };
  // levels: degree p, then max(1, p / 2) down to 1 (precond 1), each with its
  // operator tables and its leaf-block classes
  for (int pl = root->p;;) {
    h->lv.emplace_back();
    OctLevel& L = h->lv.back();
    L.p = pl;
    L.n1 = pl + 1;
    L.Nq = (long long)E * L.n1 * L.n1 * L.n1;
    octree_tables(L.n1, L.T);
    const int nf = L.n1 * L.n1;
    std::map<OctClass, int> cmap;
    std::vector<int> cls(3 * (size_t)E);
    std::vector<double> Sv, lv;
    for (int e = 0; e < E; ++e)
      for (int d = 0; d < 3; ++d) {
        int ty[2];
        for (int r = 0; r < 2; ++r) {
          const int k = kind[6 * (size_t)e + 2 * d + r];
          ty[r] = k == 0 ? 0 : (k == 3 ? 2 : 1);
        }
        const OctClass key{d, leaves[4 * e], ty[0], ty[1]};
        auto it = cmap.find(key);
        if (it == cmap.end()) {
          const int id = (int)cmap.size();
          it = cmap.emplace(key, id).first;
          Sv.resize((size_t)(id + 1) * nf);
          lv.resize((size_t)(id + 1) * L.n1);
          oct_class_fdm(L.T, L.n1, L.p, hq[3 * (size_t)e + d], ty[0], ty[1], penalty_form, penalty_eps,
                        Sv.data() + (size_t)id * nf, lv.data() + (size_t)id * L.n1);
        }
        cls[3 * (size_t)e + d] = it->second;
      }
    L.ncls = (int)cmap.size();
    if ((rc = up(L.cls, cls.data(), sizeof(int) * cls.size())) != DG_OK ||
        (rc = up(L.S, Sv.data(), sizeof(double) * Sv.size())) != DG_OK ||
        (rc = up(L.lam, lv.data(), sizeof(double) * lv.size())) != DG_OK)
      return fail(rc);
    if (precond == 0 || pl == 1) break;
    pl = std::max(1, pl / 2);
  }
  // interpolation from each level to the next finer one
  for (size_t l = 0; l + 1 < h->lv.size(); ++l) {
    const int nf1 = h->lv[l].n1, nc1 = h->lv[l + 1].n1;
    double xf[MAXN1], wf[MAXN1], xc[MAXN1], wc[MAXN1], Lc[MAXN1], dLc[MAXN1];
    gauss_legendre(nf1, xf, wf);
    gauss_legendre(nc1, xc, wc);
    std::vector<double> I((size_t)nf1 * nc1);
    for (int a = 0; a < nf1; ++a) {
      lagrange(xc, nc1, xf[a], Lc, dLc);
      for (int j = 0; j < nc1; ++j) I[(size_t)a * nc1 + j] = Lc[j];
    }
    if ((rc = up(h->lv[l].I, I.data(), sizeof(double) * I.size())) != DG_OK) return fail(rc);
  }
  // boundary faces: GL nodes, 1-D lift factors, and per leaf the face indices
  const OctTables& T = h->lv[0].T;
  std::vector<double> xb, l1;
  std::vector<int> bl;
  for (int e = 0; e < E; ++e) {
    int fidx[6] = {-1, -1, -1, -1, -1, -1};
    bool any = false;
    for (int f = 0; f < 6; ++f) {
      if (kind[6 * (size_t)e + f] != 0) continue;
      const int d = f >> 1, r = f & 1, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
      const double* hh = &hq[3 * (size_t)e];
      const double* o = &org[3 * (size_t)e];
      fidx[f] = h->nbf++;
      any = true;
      for (int i1 = 0; i1 < n1; ++i1)
        for (int i0 = 0; i0 < n1; ++i0) {
          double pt[3];
          pt[d] = o[d] + (r ? hh[d] : 0.0);
          pt[t0] = o[t0] + (xi[i0] + 1.0) * hh[t0] / 2.0;
          pt[t1] = o[t1] + (xi[i1] + 1.0) * hh[t1] / 2.0;
          xb.insert(xb.end(), pt, pt + 3);
        }
      const double sig = penalty(h->p, hh[d], penalty_form, penalty_eps);
      const double e1 = r ? 1.0 : -1.0;
      for (int a = 0; a < n1; ++a)
        l1.push_back(hh[t0] * hh[t1] / 4.0 * (sig * T.Le[r][a] - e1 * (2.0 / hh[d]) * T.dLe[r][a]));
    }
    if (!any) continue;
    bl.push_back(e);
    bl.insert(bl.end(), fidx, fidx + 6);
    ++h->nbl;
  }
  if ((rc = up(h->hq, hq.data(), sizeof(double) * hq.size())) != DG_OK ||
      (rc = up(h->kind, kind.data(), sizeof(int) * kind.size())) != DG_OK ||
      (rc = up(h->nb, nb.data(), sizeof(int) * nb.size())) != DG_OK ||
      (rc = up(h->pos, pos.data(), sizeof(int) * pos.size())) != DG_OK ||
      (rc = up(h->xq, xq.data(), sizeof(double) * xq.size())) != DG_OK ||
      (rc = up(h->W, W.data(), sizeof(double) * W.size())) != DG_OK ||
      (rc = up(h->xb, xb.data(), sizeof(double) * xb.size())) != DG_OK ||
      (rc = up(h->lift1d, l1.data(), sizeof(double) * l1.size())) != DG_OK ||
      (rc = up(h->wgl, w, sizeof(double) * n1)) != DG_OK ||
      (rc = up(h->bleaf, bl.data(), sizeof(int) * bl.size())) != DG_OK)
    return fail(rc);
  if (precond == 1) {
    // the root grid at degree 1: each leaf's root cell, the root basis at the
    // leaf's degree-1 nodes, the leaves of every root cell, and the uniform
    // solver handle that carries the root grid's own multigrid hierarchy
    double x2[2], w2[2], L2[2], dL2[2];
    gauss_legendre(2, x2, w2);
    h->n_root = (int)n_root;
    h->Nq_root = n_root * 8;
    std::vector<int> rcell(E), rptr(n_root + 1, 0), rlist(E);
    std::vector<double> J(12 * (size_t)E);
    for (int e = 0; e < E; ++e) {
      const int lvl = leaves[4 * e];
      int ci[3];
      for (int d = 0; d < 3; ++d) {
        ci[d] = leaves[4 * e + 1 + d] >> lvl;
        const int loc = leaves[4 * e + 1 + d] - (ci[d] << lvl);
        for (int a = 0; a < 2; ++a) {
          const double eta = 2.0 * (loc + (x2[a] + 1.0) / 2.0) / double(1 << lvl) - 1.0;
          lagrange(x2, 2, eta, L2, dL2);
          for (int bq = 0; bq < 2; ++bq) J[12 * (size_t)e + 4 * d + 2 * a + bq] = L2[bq];
        }
      }
      rcell[e] = ci[0] + root->n[0] * (ci[1] + root->n[1] * ci[2]);
      ++rptr[rcell[e] + 1];
    }
    for (long long c = 0; c < n_root; ++c) rptr[c + 1] += rptr[c];
    {
      std::vector<int> fill(rptr.begin(), rptr.end() - 1);
      for (int e = 0; e < E; ++e) rlist[fill[rcell[e]]++] = e;
    }
    if ((rc = up(h->rcell, rcell.data(), sizeof(int) * rcell.size())) != DG_OK ||
        (rc = up(h->rJ, J.data(), sizeof(double) * J.size())) != DG_OK ||
        (rc = up(h->rptr, rptr.data(), sizeof(int) * rptr.size())) != DG_OK ||
        (rc = up(h->rlist, rlist.data(), sizeof(int) * rlist.size())) != DG_OK)
      return fail(rc);
    dg_mesh_desc rm = *root;
    rm.p = 1;
    dg_solver_opts o;
    dg_default_opts(&o);
    o.precision = DG_PREC_FP64;
    o.penalty_form = penalty_form;
    o.penalty_eps = penalty_eps;
    if ((rc = dg_poisson_setup(&rm, &o, &h->root)) != DG_OK) {
      h->err = "root-grid solver set-up failed";
      return fail(rc);
    }
    // the mixed mode's boundary-data kernel matrix, when it fits 48 GB (a sixth
    // of a GB300's memory) and the GEMM's int sizes; else the direct FP64 sum
    const long long nbn = (long long)h->nbf * n1 * n1;
    if (h->mixed && h->Nq * nbn * 4 <= (48LL << 30) && h->Nq < (1LL << 31)) {
      if ((rc = [&]() -> int {
            DG_CK(h->kmat.ensure(sizeof(float) * (size_t)(h->Nq * nbn)));
            count_launch();
            k_oct_kmat<<<152 * 16, 256>>>(h->xb.as<double>(), nbn, h->xq.as<double>(), h->Nq, h->kmat.as<float>());
            DG_CK(cudaGetLastError());
            DG_CK(cudaDeviceSynchronize());
            return DG_OK;
          }()) != DG_OK)
        return fail(rc);
      h->has_kmat = true;
    }
    // lambda_max(P^-1 A) of every octree level, for its Chebyshev smoother
    if ((rc = oct_ws(h, 1)) != DG_OK) return fail(rc);
    for (size_t l = 0; l < h->lv.size(); ++l)
      if ((rc = oct_lambda(h, (int)l, nullptr)) != DG_OK) return fail(rc);
  }
  *out = h;
  return DG_OK;
}

void dg_octree_destroy(dg_oct_handle h) {
  if (!h) return;
  DeviceWideGuard guard;
  cudaDeviceSynchronize();
  delete h;
}

const char* dg_octree_error_detail(dg_oct_handle h) { return h ? h->err.c_str() : ""; }

int dg_octree_node_coords(dg_oct_handle h, double* xyz_dev, double* w_dev, void* stream) {
  if (!h || (!xyz_dev && !w_dev)) return DG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (xyz_dev) DG_CK(cudaMemcpyAsync(xyz_dev, h->xq.p, sizeof(double) * 3 * h->Nq, cudaMemcpyDeviceToDevice, s));
  if (w_dev) DG_CK(cudaMemcpyAsync(w_dev, h->W.p, sizeof(double) * h->Nq, cudaMemcpyDeviceToDevice, s));
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_octree_operator(dg_oct_handle h, const double* u_dev, double* out_dev, int64_t B, void* stream) {
  if (!h || B < 0 || B > 65535 || (B > 0 && (!u_dev || !out_dev))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  const size_t bytes = sizeof(double) * (size_t)B * (size_t)h->Nq;
  const char *u0 = (const char*)u_dev, *o0 = (const char*)out_dev;
  if (u0 < o0 + bytes && o0 < u0 + bytes) return DG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DG_CK(oct_apply(h, h->lv[0], u_dev, out_dev, nullptr, (int)B, s));
  return DG_OK;
}

int dg_octree_precond(dg_oct_handle h, const double* r_dev, double* z_dev, int64_t B, void* stream) {
  if (!h || B < 0 || (B > 0 && (!r_dev || !z_dev))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = oct_cap(h, B);
  DG_RET(oct_ws(h, cap));
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    std::vector<int> a(nb);
    for (int k = 0; k < nb; ++k) a[k] = k;
    DG_RET(oct_act(h, a, s));
    DG_RET(oct_precond(h, r_dev + b0 * h->Nq, z_dev + b0 * h->Nq, h->act.as<int>(), nb, s));
  }
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_octree_solve(dg_oct_handle h, const double* f_dev, int64_t B, double* v_dev, dg_solve_stats* stats_host,
                    void* stream) {
  if (!h || B < 0 || (B > 0 && !f_dev)) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = oct_cap(h, B);
  DG_RET(oct_ws(h, cap));
  int worst = DG_OK;
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    const double* f = f_dev + b0 * h->Nq;
    std::vector<int> finite;
    DG_RET(oct_finite(h, f, nb, finite, s));
    DG_RET(oct_form_rhs(h, f, nb, s));
    std::vector<dg_solve_stats> st;
    DG_RET(oct_pcg(h, nb, finite, st, s));
    DG_RET(oct_self_energies(h, f, nb, st, s));
    if (v_dev)
      DG_CK(cudaMemcpyAsync(v_dev + b0 * h->Nq, h->x.p, sizeof(double) * (size_t)nb * h->Nq,
                            cudaMemcpyDeviceToDevice, s));
    if (stats_host) std::copy(st.begin(), st.end(), stats_host + b0);
    const int w = worst_of(st);
    if (w != DG_OK && (worst == DG_OK || w < worst)) worst = w;
  }
  DG_CK(cudaStreamSynchronize(s));
  return worst;
}

int dg_octree_exchange_build(dg_oct_handle h, const double* psi, int32_t N, double* K_host, double* E_H,
                             double* E_X, dg_solve_stats* stats_host, void* stream) {
  if (!h || !psi || N < 1 || N > 4096 || !K_host) return DG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long Nq = h->Nq;
  const int nsrc_total = N * (N + 1) / 2 + 1;
  const int cap = oct_cap(h, nsrc_total);
  DG_RET(oct_ws(h, cap));
  DG_CK(h->Wacc.ensure(sizeof(double) * (size_t)N * Nq));
  const int nch = kmat_chunks(Nq);
  DG_CK(h->kpart.ensure(sizeof(double) * (size_t)nch * N * N));
  DG_CK(h->Kdev.ensure(sizeof(double) * (size_t)N * N));
  DG_CK(cudaMemsetAsync(h->Wacc.p, 0, sizeof(double) * (size_t)N * Nq, s));
  // sources: 0 = the density sum_k psi_k^2, then the pairs (i <= j) row-major
  std::vector<int> si(nsrc_total), sj(nsrc_total);
  si[0] = sj[0] = -1;
  for (int i = 0, k = 1; i < N; ++i)
    for (int j = i; j < N; ++j, ++k) {
      si[k] = i;
      sj[k] = j;
    }
  int worst = DG_OK;
  double eh = 0.0;
  std::vector<int> pack;
  for (int b0 = 0; b0 < nsrc_total; b0 += cap) {
    const int nb = std::min(cap, nsrc_total - b0);
    std::vector<int> pij(si.begin() + b0, si.begin() + b0 + nb);
    pij.resize(cap);
    pij.insert(pij.end(), sj.begin() + b0, sj.begin() + b0 + nb);
    DG_CK(cudaMemcpyAsync(h->pidx.p, pij.data(), sizeof(int) * pij.size(), cudaMemcpyHostToDevice, s));
    DG_CK(launch_pair_sources(psi, N, h->pidx.as<int>(), h->pidx.as<int>() + cap, nb, Nq, h->f.as<double>(), s));
    std::vector<int> finite;
    DG_RET(oct_finite(h, h->f.as<double>(), nb, finite, s));  // synchronises: pij may go
    DG_RET(oct_form_rhs(h, h->f.as<double>(), nb, s));
    std::vector<dg_solve_stats> st;
    DG_RET(oct_pcg(h, nb, finite, st, s));
    DG_RET(oct_self_energies(h, h->f.as<double>(), nb, st, s));
    if (b0 == 0) eh = 0.5 * st[0].self_energy;
    if (stats_host) std::copy(st.begin(), st.end(), stats_host + b0);
    const int w = worst_of(st);
    if (w != DG_OK && (worst == DG_OK || w < worst)) worst = w;
    // W_j += psi_s v_sj and W_s += psi_j v_sj (s != j), per orbital in a fixed order
    std::vector<std::vector<std::pair<int, int>>> per(N);
    for (int k = 0; k < nb; ++k) {
      const int gk = b0 + k;
      if (si[gk] < 0) continue;
      per[sj[gk]].push_back({k, si[gk]});
      if (si[gk] != sj[gk]) per[si[gk]].push_back({k, sj[gk]});
    }
    std::vector<int> ptr(N + 1, 0), eb, es;
    for (int m = 0; m < N; ++m) {
      for (auto& e : per[m]) {
        eb.push_back(e.first);
        es.push_back(e.second);
      }
      ptr[m + 1] = (int)eb.size();
    }
    if (eb.empty()) continue;
    pack.clear();
    pack.insert(pack.end(), ptr.begin(), ptr.end());
    pack.insert(pack.end(), eb.begin(), eb.end());
    pack.insert(pack.end(), es.begin(), es.end());
    DG_CK(h->lists.ensure(sizeof(int) * pack.size()));
    DG_CK(cudaMemcpyAsync(h->lists.p, pack.data(), sizeof(int) * pack.size(), cudaMemcpyHostToDevice, s));
    const int* dl = h->lists.as<int>();
    DG_CK(launch_exch_accum(psi, h->x.as<double>(), h->Wacc.as<double>(), dl, dl + N + 1, dl + N + 1 + eb.size(), N,
                            Nq, s));
    DG_CK(cudaStreamSynchronize(s));  // pack is reused by the next chunk
  }
  DG_CK(launch_kmat(psi, h->W.as<double>(), h->Wacc.as<double>(), N, Nq, h->kpart.as<double>(), nch,
                    h->Kdev.as<double>(), s));
  DG_CK(cudaMemcpyAsync(K_host, h->Kdev.p, sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  if (E_H) *E_H = eh;
  if (E_X) {
    double tr = 0.0;
    for (int i = 0; i < N; ++i) tr += K_host[(size_t)i * N + i];
    *E_X = -0.5 * tr;
  }
  return worst;
}

}  // extern "C"
