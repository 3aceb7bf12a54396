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
#include "dg_octree.h"
#include "dg_setup.h"

// Handle of the octree solver (opaque in the C ABI).
struct dg_oct {
  std::string err;
  int n1 = 0, p = 0, E = 0, pform = 0, max_iter = 0;
  double eps = 0.125, rtol = 1e-10;
  long long Nq = 0;
  dg::OctTables T;
  dg::DevBuf hq, kind, nb, pos;  // leaf sizes [E][3]; connectivity [E][6], [E][6][4], [E][6]
  dg::DevBuf cls;                // int [E][3]: 1-D class of each axis
  dg::DevBuf S, lam;             // per class: S [n1][n1] (row node, column mode), lambda [n1]
  int ncls = 0;
  dg::DevBuf xq, W;              // node coordinates [Nq][3], quadrature weights [Nq]
  int nbf = 0;                   // boundary faces
  dg::DevBuf xb;                 // their GL nodes [nbf][n1 * n1][3] (lower tangential axis fastest)
  dg::DevBuf lift1d;             // [nbf][n1]: (h_t0 h_t1 / 4)(sigma l_a(e) - e (2/h_d) l_a'(e))
  dg::DevBuf wgl;                // GL weights [n1]
  int nbl = 0;                   // leaves with a boundary face
  dg::DevBuf bleaf;              // [nbl][7]: leaf, then the boundary face index of each face or -1
  // workspace, sized for `cap` sources
  int cap = 0;
  dg::DevBuf f, g, b, x, r, z, pv, qv, scal, part, act, flags, pidx, lists, Wacc, kpart, Kdev;
  std::vector<int> act_host;
};

namespace dg {

static constexpr int OT = 256;
enum { O_BB = 0, O_RR, O_RZ, O_RZN, O_PQ, O_AL, O_BE, O_SE, O_NSLOT };

static inline dim3 ogrid(long long n, int nsrc) {
  long long gx = (n + OT * 4 - 1) / (OT * 4);
  gx = std::max(1LL, std::min(gx, 4096LL));
  return dim3((unsigned)gx, (unsigned)nsrc);
}

// z = P r on every leaf: the exact inverse of the leaf's diagonal block by
// fast diagonalisation (one block per leaf and source)
template <int N1>
__global__ void __launch_bounds__(128) k_oct_bjac(const int* __restrict__ cls, const double* __restrict__ S,
                                                  const double* __restrict__ lam, const double* __restrict__ r,
                                                  double* __restrict__ z, long long Nq, const int* __restrict__ act) {
  constexpr int NPE = N1 * N1 * N1, NF = N1 * N1;
  __shared__ double sS[3][NF], sl[3][N1], u[NPE], t[NPE];
  const int e = blockIdx.x;
  const long long off = (long long)act[blockIdx.y] * Nq + (long long)e * NPE;
  for (int i = threadIdx.x; i < 3 * NF; i += blockDim.x) {
    const int d = i / NF;
    sS[d][i % NF] = S[(long long)cls[3 * e + d] * NF + i % NF];
  }
  for (int i = threadIdx.x; i < 3 * N1; i += blockDim.x) {
    const int d = i / N1;
    sl[d][i % N1] = lam[(long long)cls[3 * e + d] * N1 + i % N1];
  }
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) u[i] = r[off + i];
  __syncthreads();
  // forward: t = (S_x (x) S_y (x) S_z)^T u, one axis at a time (mode index replaces node index)
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int m = i % N1, rest = i - m;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < N1; ++a) acc += sS[0][a * N1 + m] * u[rest + a];
    t[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int m = (i / N1) % N1, rest = i - m * N1;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < N1; ++b) acc += sS[1][b * N1 + m] * t[rest + b * N1];
    u[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int m = i / NF, rest = i - m * NF;
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < N1; ++c) acc += sS[2][c * N1 + m] * u[rest + c * NF];
    t[i] = acc / (sl[0][i % N1] + sl[1][(i / N1) % N1] + sl[2][m]);
  }
  __syncthreads();
  // back: u = (S_x (x) S_y (x) S_z) t
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int c = i / NF, rest = i - c * NF;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < N1; ++m) acc += sS[2][c * N1 + m] * t[rest + m * NF];
    u[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int b = (i / N1) % N1, rest = i - b * N1;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < N1; ++m) acc += sS[1][b * N1 + m] * u[rest + m * N1];
    t[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPE; i += blockDim.x) {
    const int a = i % N1, rest = i - a;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < N1; ++m) acc += sS[0][a * N1 + m] * t[rest + m];
    z[off + i] = acc;
  }
}

// g[k][j] = sum_q W_q f_k(q) / |xb_j - x_q| (Sec. 6.3): one thread per boundary
// node, the nodes x_q staged through shared memory in a fixed order
static constexpr int BDT = 128, BDQ = 256;
__global__ void __launch_bounds__(BDT) k_oct_bdata(const double* __restrict__ xb, long long nbn,
                                                   const double* __restrict__ xq, const double* __restrict__ W,
                                                   const double* __restrict__ f, long long Nq, double* __restrict__ g) {
  __shared__ double sx[BDQ], sy[BDQ], sz[BDQ], sw[BDQ];
  const long long j = (long long)blockIdx.x * BDT + threadIdx.x;
  const int k = blockIdx.y;
  const double* fk = f + (long long)k * Nq;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (j < nbn) {
    px = xb[3 * j];
    py = xb[3 * j + 1];
    pz = xb[3 * j + 2];
  }
  double acc = 0.0;
  for (long long q0 = 0; q0 < Nq; q0 += BDQ) {
    const int nq = (int)std::min<long long>(BDQ, Nq - q0);
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += BDT) {
      sx[i] = xq[3 * (q0 + i)];
      sy[i] = xq[3 * (q0 + i) + 1];
      sz[i] = xq[3 * (q0 + i) + 2];
      sw[i] = W[q0 + i] * fk[q0 + i];
    }
    __syncthreads();
    for (int i = 0; i < nq; ++i) {
      const double dx = px - sx[i], dy = py - sy[i], dz = pz - sz[i];
      acc += sw[i] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  if (j < nbn) g[(long long)k * nbn + j] = acc;
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
__global__ void k_oct_sub(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ q,
                          long long Nq, const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
    r[off + i] = b[off + i] - q[off + i];
}
__global__ void k_oct_copy(double* __restrict__ dst, const double* __restrict__ src, long long Nq,
                           const int* __restrict__ act) {
  const long long off = (long long)act[blockIdx.y] * Nq;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nq; i += (long long)gridDim.x * blockDim.x)
    dst[off + i] = src[off + i];
}

}  // namespace dg

namespace dg {

static cudaError_t launch_bjac(const dg_oct* h, const double* r, double* z, const int* act, int nact, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;
  const dim3 grid((unsigned)h->E, (unsigned)nact);
  const int* c = h->cls.as<int>();
  const double *S = h->S.as<double>(), *l = h->lam.as<double>();
  count_launch();
  switch (h->n1) {
#define DG_BJ(N)                                                              \
  case N:                                                                     \
    k_oct_bjac<N><<<grid, 128, 0, s>>>(c, S, l, r, z, h->Nq, act);            \
    break;
    DG_BJ(2) DG_BJ(3) DG_BJ(4) DG_BJ(5) DG_BJ(6) DG_BJ(7) DG_BJ(8) DG_BJ(9)
#undef DG_BJ
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
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
  DG_CK(h->g.ensure(sizeof(double) * (size_t)cap * h->nbf * h->n1 * h->n1));
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
  count_launch();
  k_oct_bdata<<<dim3((unsigned)((nbn + BDT - 1) / BDT), (unsigned)nsrc), BDT, 0, s>>>(
      h->xb.as<double>(), nbn, h->xq.as<double>(), h->W.as<double>(), f, h->Nq, h->g.as<double>());
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

}  // namespace dg

namespace dg {

// PCG on the sources 0..nsrc-1 of the workspace (b formed): x = A^-1 b to the
// FP64 relative residual rtol. Convergence of the recursive residual is
// confirmed on the true residual b - A x; where the two disagree the
// iteration restarts from the true residual (at most 3 times per source).
static int oct_pcg(dg_oct* h, int nsrc, const std::vector<int>& finite, std::vector<dg_solve_stats>& st,
                   cudaStream_t s) {
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
    DG_CK(launch_octree_apply(h->n1, h->T, h->hq.as<double>(), h->kind.as<int>(), h->nb.as<int>(), h->pos.as<int>(),
                              h->E, h->p, h->pform, h->eps, x, q, act, n, s));
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
  DG_CK(launch_bjac(h, r, z, act, n, s));
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
    DG_CK(launch_octree_apply(h->n1, h->T, h->hq.as<double>(), h->kind.as<int>(), h->nb.as<int>(), h->pos.as<int>(),
                              h->E, h->p, h->pform, h->eps, p, q, act, n, s));
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
    DG_CK(launch_bjac(h, r, z, act, n, s));
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
  // seven source vectors per source: at most about 4 GB of workspace, at most 64 sources per chunk
  const long long per = 7LL * h->Nq * (long long)sizeof(double);
  long long c = std::max(1LL, std::min(64LL, (4LL << 30) / std::max(1LL, per)));
  return (int)std::max(1LL, std::min(c, want));
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_octree_setup(const dg_mesh_desc* root, const int32_t* leaves, int32_t n_leaves, int32_t penalty_form,
                    double penalty_eps, double rtol, int32_t max_iter, dg_oct_handle* out) {
  if (!out) return DG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!root || !leaves || n_leaves < 1 || root->p < 1 || root->p > MAXN1 - 1 ||
      (penalty_form != 0 && penalty_form != 1) || !(penalty_eps > 0.0) || !(rtol > 0.0) || !(rtol < 1.0) ||
      max_iter < 1)
    return DG_ERR_INVALID_ARG;
  const int E = n_leaves, n1 = root->p + 1, NPE = n1 * n1 * n1, NF = n1 * n1;
  std::vector<int32_t> kind(6 * (size_t)E), nb(24 * (size_t)E), pos(6 * (size_t)E);
  if (!octree_faces(root, leaves, n_leaves, kind.data(), nb.data(), pos.data())) return DG_ERR_INVALID_ARG;
  if ((long long)E * NPE > (1LL << 31)) return DG_ERR_UNSUPPORTED;
  DeviceWideGuard guard;
  dg_oct* h = new dg_oct();
  h->n1 = n1;
  h->p = root->p;
  h->E = E;
  h->pform = penalty_form;
  h->eps = penalty_eps;
  h->rtol = rtol;
  h->max_iter = max_iter;
  h->Nq = (long long)E * NPE;
  octree_tables(n1, h->T);
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
  // 1-D classes of the block preconditioner
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
        Sv.resize((size_t)(id + 1) * NF);
        lv.resize((size_t)(id + 1) * n1);
        oct_class_fdm(h->T, n1, h->p, hq[3 * (size_t)e + d], ty[0], ty[1], penalty_form, penalty_eps,
                      Sv.data() + (size_t)id * NF, lv.data() + (size_t)id * n1);
      }
      cls[3 * (size_t)e + d] = it->second;
    }
  h->ncls = (int)cmap.size();
  // boundary faces: GL nodes, 1-D lift factors, and per leaf the face indices
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
        l1.push_back(hh[t0] * hh[t1] / 4.0 * (sig * h->T.Le[r][a] - e1 * (2.0 / hh[d]) * h->T.dLe[r][a]));
    }
    if (!any) continue;
    bl.push_back(e);
    bl.insert(bl.end(), fidx, fidx + 6);
    ++h->nbl;
  }
  auto up = [&](DevBuf& dst, const void* src, size_t bytes) -> int {
    DG_CK(dst.ensure(std::max<size_t>(bytes, 16)));
    DG_CK(cudaMemcpy(dst.p, src, bytes, cudaMemcpyHostToDevice));
    return DG_OK;
  };
  int rc = DG_OK;
  if ((rc = up(h->hq, hq.data(), sizeof(double) * hq.size())) != DG_OK ||
      (rc = up(h->kind, kind.data(), sizeof(int) * kind.size())) != DG_OK ||
      (rc = up(h->nb, nb.data(), sizeof(int) * nb.size())) != DG_OK ||
      (rc = up(h->pos, pos.data(), sizeof(int) * pos.size())) != DG_OK ||
      (rc = up(h->cls, cls.data(), sizeof(int) * cls.size())) != DG_OK ||
      (rc = up(h->S, Sv.data(), sizeof(double) * Sv.size())) != DG_OK ||
      (rc = up(h->lam, lv.data(), sizeof(double) * lv.size())) != DG_OK ||
      (rc = up(h->xq, xq.data(), sizeof(double) * xq.size())) != DG_OK ||
      (rc = up(h->W, W.data(), sizeof(double) * W.size())) != DG_OK ||
      (rc = up(h->xb, xb.data(), sizeof(double) * xb.size())) != DG_OK ||
      (rc = up(h->lift1d, l1.data(), sizeof(double) * l1.size())) != DG_OK ||
      (rc = up(h->wgl, w, sizeof(double) * n1)) != DG_OK || (rc = up(h->bleaf, bl.data(), sizeof(int) * bl.size())) != DG_OK) {
    delete h;
    return rc;
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
  DG_CK(launch_octree_apply(h->n1, h->T, h->hq.as<double>(), h->kind.as<int>(), h->nb.as<int>(), h->pos.as<int>(),
                            h->E, h->p, h->pform, h->eps, u_dev, out_dev, nullptr, (int)B, s));
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
    DG_CK(launch_bjac(h, r_dev + b0 * h->Nq, z_dev + b0 * h->Nq, h->act.as<int>(), nb, s));
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
