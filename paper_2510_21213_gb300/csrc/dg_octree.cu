// Adaptive octree auxiliary mesh, host side (Sec. 6.2): the uniform root grid
// refined where the density's quadrature indicator exceeds a threshold, kept
// 2:1 balanced across faces, and the face connectivity the operator on it
// needs (same-size, larger or smaller neighbours, boundary).
//
// Readings: isotropic 8-child splits; indicator Q = |I_K(rho) - sum over the
// children of I_C(rho)| with the degree-p tensor Gauss-Legendre rule of the
// leaf and of each child; a leaf is split while Q > delta and its level is
// below the maximum level.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "dg_ctx.h"
#include "dg_internal.h"
#include "dg_octree.h"
#include "dg_setup.h"

namespace dg {

using Leaf = std::array<int, 4>;  // level, ix, iy, iz

struct Octree {
  double lo[3], H[3];
  int n[3], p;
  std::set<Leaf> leaves;

  double h(int level, int d) const { return H[d] / double(1 << level); }
  long long extent(int level, int d) const { return (long long)n[d] << level; }

  void refine(const std::vector<Leaf>& ks) {
    for (const Leaf& k : ks) {
      if (!leaves.erase(k)) continue;
      for (int c = 0; c < 8; ++c)
        leaves.insert({k[0] + 1, 2 * k[1] + (c & 1), 2 * k[2] + ((c >> 1) & 1), 2 * k[3] + (c >> 2)});
    }
  }

  // leaf containing the cell (level, x, y, z) unless finer leaves cover it
  bool covering(int level, int x, int y, int z, Leaf& out) const {
    for (int lv = level; lv >= 0; --lv) {
      const int s = level - lv;
      const Leaf k{lv, x >> s, y >> s, z >> s};
      if (leaves.count(k)) {
        out = k;
        return true;
      }
    }
    return false;
  }

  // same-level cell across face (d, side); false at the domain boundary
  bool neighbour(const Leaf& k, int d, int side, Leaf& out) const {
    out = k;
    out[1 + d] += side;
    return out[1 + d] >= 0 && out[1 + d] < extent(k[0], d);
  }

  void balance() {
    for (;;) {
      std::set<Leaf> split;
      for (const Leaf& k : leaves)
        for (int d = 0; d < 3; ++d)
          for (int side = -1; side <= 1; side += 2) {
            Leaf nb, L;
            if (!neighbour(k, d, side, nb)) continue;
            if (covering(nb[0], nb[1], nb[2], nb[3], L) && L[0] < k[0] - 1) split.insert(L);
          }
      if (split.empty()) return;
      refine(std::vector<Leaf>(split.begin(), split.end()));
    }
  }

  // element order: root cell (x fastest), then level, z, y, x
  std::vector<Leaf> ordered() const {
    std::vector<Leaf> v(leaves.begin(), leaves.end());
    auto key = [&](const Leaf& k) {
      const int lv = k[0];
      const long long r = (k[1] >> lv) + (long long)n[0] * ((k[2] >> lv) + (long long)n[1] * (k[3] >> lv));
      return std::array<long long, 5>{r, lv, k[3], k[2], k[1]};
    };
    std::sort(v.begin(), v.end(), [&](const Leaf& a, const Leaf& b) { return key(a) < key(b); });
    return v;
  }
};

// integral of rho over the box [o, o + h] by the degree-p tensor GL rule
static double gl_integral(const double* o, const double* h, int n1, const double* xi, const double* w,
                          dg_density_fn rho, void* user, std::vector<double>& pts, std::vector<double>& val) {
  const int np = n1 * n1 * n1;
  pts.resize(3 * (size_t)np);
  val.resize(np);
  for (int c = 0; c < n1; ++c)
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) {
        const int q = a + n1 * (b + n1 * c);
        pts[3 * q + 0] = o[0] + (xi[a] + 1.0) * h[0] / 2.0;
        pts[3 * q + 1] = o[1] + (xi[b] + 1.0) * h[1] / 2.0;
        pts[3 * q + 2] = o[2] + (xi[c] + 1.0) * h[2] / 2.0;
      }
  rho(pts.data(), np, val.data(), user);
  double s = 0.0;
  for (int c = 0; c < n1; ++c)
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) s += w[a] * w[b] * w[c] * val[a + n1 * (b + n1 * c)];
  return s * h[0] * h[1] * h[2] / 8.0;
}

// Face connectivity of a leaf set (see dg_octree_faces); false for a bad mesh
// or leaf set.
bool octree_faces(const dg_mesh_desc* root, const int32_t* leaves, int32_t n_leaves, int32_t* kind,
                         int32_t* nb, int32_t* pos) {
  if (!root || !leaves || n_leaves < 1 || !kind || !nb || !pos) return false;
  Octree t;
  for (int d = 0; d < 3; ++d) {
    if (root->n[d] < 1 || !(root->hi[d] > root->lo[d])) return false;
    t.lo[d] = root->lo[d];
    t.n[d] = root->n[d];
    t.H[d] = (root->hi[d] - root->lo[d]) / root->n[d];
  }
  t.p = root->p;
  std::map<Leaf, int> index;
  for (int e = 0; e < n_leaves; ++e) {
    const Leaf k{leaves[4 * e], leaves[4 * e + 1], leaves[4 * e + 2], leaves[4 * e + 3]};
    if (k[0] < 0 || k[0] > 20) return false;
    for (int d = 0; d < 3; ++d)
      if (k[1 + d] < 0 || k[1 + d] >= t.extent(k[0], d)) return false;
    if (!index.emplace(k, e).second) return false;
    t.leaves.insert(k);
  }
  // a partition: no leaf may lie inside another leaf of the set
  for (int e = 0; e < n_leaves; ++e) {
    const Leaf k{leaves[4 * e], leaves[4 * e + 1], leaves[4 * e + 2], leaves[4 * e + 3]};
    for (int lv = k[0] - 1; lv >= 0; --lv) {
      const int sh = k[0] - lv;
      if (index.count(Leaf{lv, k[1] >> sh, k[2] >> sh, k[3] >> sh})) return false;
    }
  }
  for (int e = 0; e < n_leaves; ++e) {
    const Leaf k{leaves[4 * e], leaves[4 * e + 1], leaves[4 * e + 2], leaves[4 * e + 3]};
    for (int d = 0; d < 3; ++d)
      for (int sd = 0; sd < 2; ++sd) {
        const int f = 2 * d + sd, side = sd ? 1 : -1;
        const long long o = 6LL * e + f;
        for (int j = 0; j < 4; ++j) nb[4 * o + j] = -1;
        pos[o] = -1;
        Leaf c, L;
        if (!t.neighbour(k, d, side, c)) {
          kind[o] = 0;  // boundary
          continue;
        }
        const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
        if (t.covering(c[0], c[1], c[2], c[3], L)) {
          if (L[0] == k[0]) {
            kind[o] = 1;
          } else if (L[0] == k[0] - 1) {
            kind[o] = 2;  // this face is a quarter of L's face: its two tangential bits
            pos[o] = (k[1 + t0] & 1) | ((k[1 + t1] & 1) << 1);
          } else {
            return false;  // not 2:1 balanced
          }
          nb[4 * o] = index.at(L);
          continue;
        }
        // four smaller neighbours: the level + 1 cells touching this face
        kind[o] = 3;
        for (int j = 0; j < 4; ++j) {
          Leaf sl{k[0] + 1, 2 * k[1], 2 * k[2], 2 * k[3]};
          sl[1 + d] = sd ? 2 * k[1 + d] + 2 : 2 * k[1 + d] - 1;
          sl[1 + t0] += j & 1;
          sl[1 + t1] += j >> 1;
          auto it = index.find(sl);
          if (it == index.end()) return false;  // not 2:1 balanced or not a leaf set
          nb[4 * o + j] = it->second;
        }
      }
  }
  return true;
}


// ---------------------------------------------------------------------------
// SIPDG operator on the octree leaves (Sec. 3.4 eq. sip_bilinear with the
// Nitsche boundary terms of Sec. 6.3), matrix-free, one block per leaf and
// source. Volume term: the element's Kronecker sum (GL-collocated mass, exact
// 1-D stiffness). Face terms: traces and normal derivatives of this leaf and of
// its neighbour(s) at Gauss points of the smaller face (a hanging face is
// integrated on each of its four quarters), fluxes
//   v-trace:      -{d_n u} + sigma [u]     (boundary: -d_n u + sigma u)
//   d_n v:        -1/2 [u]                 (boundary: -u)
// with [u] = u_K - u_L along K's outward normal, sigma = (p+1)^2/(eps h) of
// the smaller leaf, and the test-side contraction back onto the leaf's nodes.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double oct_penalty(int p, double h, int form, double eps) {
  const double c = (double)((p + 1) * (p + 1));
  return form == 0 ? c / (eps * h) : c / (eps * h * h);
}

template <int N1>
__global__ void __launch_bounds__(256) k_octree_apply(const OctTables T, const double* __restrict__ hq,
                                                      const int* __restrict__ kind, const int* __restrict__ nbr,
                                                      const int* __restrict__ pos, int E, int p, int pform,
                                                      double eps, const double* __restrict__ u,
                                                      double* __restrict__ out, const int* __restrict__ act) {
  constexpr int NPE = N1 * N1 * N1, NF = N1 * N1;
  __shared__ double sLq[NF], sLh[2][NF], sS[NF], sLe[2][N1], sdLe[2][N1], sw[N1], swq[N1];
  __shared__ double uK[NPE], acc[NPE], uN[NPE];
  __shared__ double VK[NF], DK[NF], VL[NF], DL[NF], pv[NF], pd[NF], qv[NF], qd[NF], F1[NF], F2[NF], G1[NF],
      G2[NF];
  const int e = blockIdx.x;
  const int tid = threadIdx.x, NT = blockDim.x;
  const long long src = act ? act[blockIdx.y] : blockIdx.y;
  const double* ub = u + src * E * NPE;
  double* ob = out + src * E * NPE;
  for (int i = tid; i < NF; i += NT) {
    const int r = i / N1, c = i % N1;
    sLq[i] = T.Lq[r * N1 + c];
    sLh[0][i] = T.Lh[0][r * N1 + c];
    sLh[1][i] = T.Lh[1][r * N1 + c];
    sS[i] = T.S[r * N1 + c];
  }
  for (int i = tid; i < N1; i += NT) {
    sLe[0][i] = T.Le[0][i];
    sLe[1][i] = T.Le[1][i];
    sdLe[0][i] = T.dLe[0][i];
    sdLe[1][i] = T.dLe[1][i];
    sw[i] = T.w[i];
    swq[i] = T.wq[i];
  }
  for (int i = tid; i < NPE; i += NT) uK[i] = ub[(long long)e * NPE + i];
  const double hK[3] = {hq[3LL * e], hq[3LL * e + 1], hq[3LL * e + 2]};
  __syncthreads();
  // volume: sum_d (2/h_d)(h_t0 h_t1 / 4) (S_d (x) W (x) W) u
  for (int i = tid; i < NPE; i += NT) {
    const int ix = i % N1, iy = (i / N1) % N1, iz = i / NF;
    double vx = 0.0, vy = 0.0, vz = 0.0;
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      vx += sS[ix * N1 + a] * uK[a + N1 * iy + NF * iz];
      vy += sS[iy * N1 + a] * uK[ix + N1 * a + NF * iz];
      vz += sS[iz * N1 + a] * uK[ix + N1 * iy + NF * a];
    }
    acc[i] = vx * sw[iy] * sw[iz] * (2.0 / hK[0]) * (hK[1] * hK[2] / 4.0) +
             vy * sw[ix] * sw[iz] * (2.0 / hK[1]) * (hK[0] * hK[2] / 4.0) +
             vz * sw[ix] * sw[iy] * (2.0 / hK[2]) * (hK[0] * hK[1] / 4.0);
  }
  __syncthreads();
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, r = f & 1;
    const double s = r ? 1.0 : -1.0;
    const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    const int str[3] = {1, N1, NF};
    const int sd = str[d], s0 = str[t0], s1 = str[t1];
    // this leaf's face trace and outward normal derivative on its face nodes [t0][t1]
    for (int j = tid; j < NF; j += NT) {
      const int b = j / N1, c = j % N1;
      double v = 0.0, dv = 0.0;
#pragma unroll
      for (int a = 0; a < N1; ++a) {
        const double x = uK[a * sd + b * s0 + c * s1];
        v += sLe[r][a] * x;
        dv += sdLe[r][a] * x;
      }
      VK[j] = v;
      DK[j] = dv * (2.0 / hK[d]) * s;
    }
    __syncthreads();
    const long long o = 6LL * e + f;
    const int kd = kind[o];
    const int nq4 = kd == 3 ? 4 : 1;
    for (int qi = 0; qi < nq4; ++qi) {
      const double* T0K = kd == 3 ? sLh[qi & 1] : sLq;
      const double* T1K = kd == 3 ? sLh[qi >> 1] : sLq;
      for (int q = tid; q < NF; q += NT) {
        const int i = q / N1, jj = q % N1;
        double v = 0.0, dv = 0.0;
        for (int b = 0; b < N1; ++b) {
          double rv = 0.0, rd = 0.0;
#pragma unroll
          for (int c = 0; c < N1; ++c) {
            rv += T1K[jj * N1 + c] * VK[b * N1 + c];
            rd += T1K[jj * N1 + c] * DK[b * N1 + c];
          }
          v += T0K[i * N1 + b] * rv;
          dv += T0K[i * N1 + b] * rd;
        }
        pv[q] = v;
        pd[q] = dv;
      }
      double sig, wscale;
      if (kd == 0) {
        sig = oct_penalty(p, hK[d], pform, eps);
        wscale = hK[t0] * hK[t1] / 4.0;
      } else {
        const int L = kd == 3 ? nbr[4 * o + qi] : nbr[4 * o];
        const double hL[3] = {hq[3LL * L], hq[3LL * L + 1], hq[3LL * L + 2]};
        for (int i = tid; i < NPE; i += NT) uN[i] = ub[(long long)L * NPE + i];
        __syncthreads();
        const int rl = 1 - r;  // the neighbour's face is on its other side
        for (int j = tid; j < NF; j += NT) {
          const int b = j / N1, c = j % N1;
          double v = 0.0, dv = 0.0;
#pragma unroll
          for (int a = 0; a < N1; ++a) {
            const double x = uN[a * sd + b * s0 + c * s1];
            v += sLe[rl][a] * x;
            dv += sdLe[rl][a] * x;
          }
          VL[j] = v;
          DL[j] = dv * (2.0 / hL[d]) * s;
        }
        __syncthreads();
        const int ps = kd == 2 ? pos[o] : 0;
        const double* T0L = kd == 2 ? sLh[ps & 1] : sLq;
        const double* T1L = kd == 2 ? sLh[ps >> 1] : sLq;
        for (int q = tid; q < NF; q += NT) {
          const int i = q / N1, jj = q % N1;
          double v = 0.0, dv = 0.0;
          for (int b = 0; b < N1; ++b) {
            double rv = 0.0, rd = 0.0;
#pragma unroll
            for (int c = 0; c < N1; ++c) {
              rv += T1L[jj * N1 + c] * VL[b * N1 + c];
              rd += T1L[jj * N1 + c] * DL[b * N1 + c];
            }
            v += T0L[i * N1 + b] * rv;
            dv += T0L[i * N1 + b] * rd;
          }
          qv[q] = v;
          qd[q] = dv;
        }
        sig = oct_penalty(p, fmin(hK[d], hL[d]), pform, eps);
        wscale = kd == 3 ? hL[t0] * hL[t1] / 4.0 : hK[t0] * hK[t1] / 4.0;
      }
      __syncthreads();
      for (int q = tid; q < NF; q += NT) {
        const int i = q / N1, jj = q % N1;
        const double wt = swq[i] * swq[jj] * wscale;
        if (kd == 0) {
          F1[q] = wt * (-pd[q] + sig * pv[q]);
          F2[q] = wt * (-pv[q]);
        } else {
          F1[q] = wt * (-0.5 * (pd[q] + qd[q]) + sig * (pv[q] - qv[q]));
          F2[q] = wt * (-0.5 * (pv[q] - qv[q]));
        }
      }
      __syncthreads();
      // back onto this leaf's face nodes: G[b][c] = sum_ij T0K[i][b] T1K[j][c] F[i][j]
      for (int j = tid; j < NF; j += NT) {
        const int b = j / N1, c = j % N1;
        double g1 = 0.0, g2 = 0.0;
        for (int i = 0; i < N1; ++i) {
          double r1 = 0.0, r2 = 0.0;
#pragma unroll
          for (int jj = 0; jj < N1; ++jj) {
            r1 += F1[i * N1 + jj] * T1K[jj * N1 + c];
            r2 += F2[i * N1 + jj] * T1K[jj * N1 + c];
          }
          g1 += T0K[i * N1 + b] * r1;
          g2 += T0K[i * N1 + b] * r2;
        }
        G1[j] = g1;
        G2[j] = g2;
      }
      __syncthreads();
      for (int i = tid; i < NPE; i += NT) {
        const int c3[3] = {i % N1, (i / N1) % N1, i / NF};
        const int a = c3[d], b = c3[t0], c = c3[t1];
        acc[i] += sLe[r][a] * G1[b * N1 + c] + sdLe[r][a] * (2.0 / hK[d]) * s * G2[b * N1 + c];
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < NPE; i += NT) ob[(long long)e * NPE + i] = acc[i];
}

void octree_tables(int n1, OctTables& T) {
  std::memset(&T, 0, sizeof(T));
  double xi[MAXN1], w[MAXN1], xq[MAXN1], wq[MAXN1], L[MAXN1], dL[MAXN1];
  gauss_legendre(n1, xi, w);
  gauss_legendre(n1, xq, wq);  // Gauss points of a face direction (exact for the face integrands)
  for (int a = 0; a < n1; ++a) {
    T.w[a] = w[a];
    T.wq[a] = wq[a];
  }
  for (int i = 0; i < n1; ++i) {
    lagrange(xi, n1, xq[i], L, dL);
    for (int a = 0; a < n1; ++a) T.Lq[i * n1 + a] = L[a];
    for (int c = 0; c < 2; ++c) {
      lagrange(xi, n1, (xq[i] + 2.0 * c - 1.0) / 2.0, L, dL);
      for (int a = 0; a < n1; ++a) T.Lh[c][i * n1 + a] = L[a];
    }
  }
  for (int r = 0; r < 2; ++r) {
    lagrange(xi, n1, r ? 1.0 : -1.0, L, dL);
    for (int a = 0; a < n1; ++a) {
      T.Le[r][a] = L[a];
      T.dLe[r][a] = dL[a];
    }
  }
  // 1-D stiffness: sum_q wq l_a'(xq) l_b'(xq)
  std::vector<double> dq((size_t)n1 * n1);
  for (int i = 0; i < n1; ++i) {
    lagrange(xi, n1, xq[i], L, dL);
    for (int a = 0; a < n1; ++a) dq[(size_t)i * n1 + a] = dL[a];
  }
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n1; ++b) {
      double sum = 0.0;
      for (int i = 0; i < n1; ++i) sum += wq[i] * dq[(size_t)i * n1 + a] * dq[(size_t)i * n1 + b];
      T.S[a * n1 + b] = sum;
    }
}

cudaError_t launch_octree_apply(int n1, const OctTables& T, const double* hq, const int* kind, const int* nb,
                                const int* pos, int E, int p, int pform, double eps, const double* u, double* out,
                                const int* act, int nact, cudaStream_t s) {
  if (nact == 0 || E == 0) return cudaSuccess;
  const dim3 grid((unsigned)E, (unsigned)nact);
  count_launch();
  switch (n1) {
#define DG_OCT_CASE(N)                                                                             \
  case N:                                                                                          \
    k_octree_apply<N><<<grid, 256, 0, s>>>(T, hq, kind, nb, pos, E, p, pform, eps, u, out, act); \
    break;
    DG_OCT_CASE(2)
    DG_OCT_CASE(3)
    DG_OCT_CASE(4)
    DG_OCT_CASE(5)
    DG_OCT_CASE(6)
    DG_OCT_CASE(7)
    DG_OCT_CASE(8)
    DG_OCT_CASE(9)
#undef DG_OCT_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace dg

using namespace dg;

extern "C" {

int dg_octree_refine(const dg_mesh_desc* root, double delta, int32_t max_level, dg_density_fn rho, void* user,
                     int32_t max_leaves, int32_t* leaves_host, int32_t* n_leaves) {
  if (!root || !rho || !n_leaves || !(delta > 0.0) || max_level < 0 || max_level > 20 || root->p < 1 ||
      root->p > MAXN1 - 1 || max_leaves < 0)
    return DG_ERR_INVALID_ARG;
  Octree t;
  for (int d = 0; d < 3; ++d) {
    if (root->n[d] < 1 || !(root->hi[d] > root->lo[d])) return DG_ERR_INVALID_ARG;
    t.lo[d] = root->lo[d];
    t.n[d] = root->n[d];
    t.H[d] = (root->hi[d] - root->lo[d]) / root->n[d];
  }
  t.p = root->p;
  for (int z = 0; z < t.n[2]; ++z)
    for (int y = 0; y < t.n[1]; ++y)
      for (int x = 0; x < t.n[0]; ++x) t.leaves.insert({0, x, y, z});
  const int n1 = t.p + 1;
  double xi[MAXN1], w[MAXN1];
  gauss_legendre(n1, xi, w);
  std::vector<double> pts, val;
  for (;;) {
    std::vector<Leaf> split;
    for (const Leaf& k : t.leaves) {
      if (k[0] >= max_level) continue;
      double o[3], h[3];
      for (int d = 0; d < 3; ++d) {
        h[d] = t.h(k[0], d);
        o[d] = t.lo[d] + k[1 + d] * h[d];
      }
      const double whole = gl_integral(o, h, n1, xi, w, rho, user, pts, val);
      double parts = 0.0;
      for (int c = 0; c < 8; ++c) {
        double oc[3], hc[3];
        for (int d = 0; d < 3; ++d) {
          hc[d] = h[d] / 2.0;
          oc[d] = o[d] + ((c >> d) & 1) * hc[d];
        }
        parts += gl_integral(oc, hc, n1, xi, w, rho, user, pts, val);
      }
      if (std::fabs(whole - parts) > delta) split.push_back(k);
    }
    if (split.empty()) break;
    t.refine(split);
    t.balance();
    if ((long long)t.leaves.size() > (1LL << 24)) return DG_ERR_NO_MEMORY;
  }
  const std::vector<Leaf> v = t.ordered();
  *n_leaves = (int32_t)v.size();
  if (leaves_host) {
    if ((long long)v.size() > max_leaves) return DG_ERR_INVALID_ARG;
    for (size_t i = 0; i < v.size(); ++i)
      for (int j = 0; j < 4; ++j) leaves_host[4 * i + j] = v[i][j];
  }
  return DG_OK;
}

int dg_octree_faces(const dg_mesh_desc* root, const int32_t* leaves, int32_t n_leaves, int32_t* kind, int32_t* nb,
                    int32_t* pos) {
  return octree_faces(root, leaves, n_leaves, kind, nb, pos) ? DG_OK : DG_ERR_INVALID_ARG;
}


int dg_octree_apply(const dg_mesh_desc* root, const int32_t* leaves, int32_t n_leaves, int32_t penalty_form,
                    double penalty_eps, const double* u, double* out, int64_t B, void* stream) {
  if (!root || root->p < 1 || root->p > MAXN1 - 1 || (penalty_form != 0 && penalty_form != 1) ||
      !(penalty_eps > 0.0) || B < 0 || B > 65535 || n_leaves < 1 || (B > 0 && (!u || !out)))
    return DG_ERR_INVALID_ARG;
  const int E = n_leaves;
  if (B > 0) {
    // out is written while other blocks still read u: the two must not overlap
    const size_t bytes = sizeof(double) * (size_t)B * (size_t)E * (size_t)((root->p + 1) * (root->p + 1) * (root->p + 1));
    const char *u0 = (const char*)u, *o0 = (const char*)out;
    if (u0 < o0 + bytes && o0 < u0 + bytes) return DG_ERR_INVALID_ARG;
  }
  std::vector<int32_t> kind(6 * (size_t)E), nb(24 * (size_t)E), pos(6 * (size_t)E);
  if (!octree_faces(root, leaves, n_leaves, kind.data(), nb.data(), pos.data())) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  std::vector<double> hq(3 * (size_t)E);
  for (int e = 0; e < E; ++e)
    for (int d = 0; d < 3; ++d)
      hq[3 * (size_t)e + d] = (root->hi[d] - root->lo[d]) / root->n[d] / double(1 << leaves[4 * e]);
  const int n1 = root->p + 1;
  OctTables T;
  octree_tables(n1, T);
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf dh, dk, dn, dp;
  auto ck = [](cudaError_t e) { return e == cudaSuccess ? DG_OK : (e == cudaErrorMemoryAllocation ? DG_ERR_NO_MEMORY : DG_ERR_CUDA); };
  int rc;
  if ((rc = ck(dh.ensure(sizeof(double) * hq.size()))) != DG_OK) return rc;
  if ((rc = ck(dk.ensure(sizeof(int) * kind.size()))) != DG_OK) return rc;
  if ((rc = ck(dn.ensure(sizeof(int) * nb.size()))) != DG_OK) return rc;
  if ((rc = ck(dp.ensure(sizeof(int) * pos.size()))) != DG_OK) return rc;
  if ((rc = ck(cudaMemcpyAsync(dh.p, hq.data(), sizeof(double) * hq.size(), cudaMemcpyHostToDevice, s))) != DG_OK)
    return rc;
  if ((rc = ck(cudaMemcpyAsync(dk.p, kind.data(), sizeof(int) * kind.size(), cudaMemcpyHostToDevice, s))) != DG_OK)
    return rc;
  if ((rc = ck(cudaMemcpyAsync(dn.p, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice, s))) != DG_OK)
    return rc;
  if ((rc = ck(cudaMemcpyAsync(dp.p, pos.data(), sizeof(int) * pos.size(), cudaMemcpyHostToDevice, s))) != DG_OK)
    return rc;
  if ((rc = ck(launch_octree_apply(n1, T, dh.as<double>(), dk.as<int>(), dn.as<int>(), dp.as<int>(), E, root->p,
                                   penalty_form, penalty_eps, u, out, nullptr, (int)B, s))) != DG_OK)
    return rc;
  // the tables and connectivity are call-local: wait before they are freed
  return ck(cudaStreamSynchronize(s));
}

}  // extern "C"
