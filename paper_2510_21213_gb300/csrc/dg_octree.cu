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

// Every face-quarter of the leaf is processed at once (a face with four smaller
// neighbours has four, every other face one): 6 to 24 "face parts" per leaf,
// each with six NF-sized buffers in dynamic shared memory. Interpolations to and
// from the Gauss points are sum-factorised (one tangential axis at a time).
// Phases, separated by block barriers:
//   1. volume term; this leaf's six face traces; the neighbours' traces of
//      every part, read from global memory
//   2. first tangential contraction (t1) of the four traces of every part
//   3. second contraction (t0) and the fluxes F1 (v-trace), F2 (d_n v)
//   4, 5. the fluxes back onto this leaf's face nodes (t1, then t0)
//   6. the face contributions added into the volume term, and the store
template <int N1>
__device__ __forceinline__ int oct_stride(int d) {
  return d == 0 ? 1 : (d == 1 ? N1 : N1 * N1);
}

struct OctPart {
  int f, L;          // face (2 d + side) and neighbour leaf (-1: boundary)
  int tk0, tk1;      // this leaf's tables along t0, t1: 0 = Lq, 1 = Lh[0], 2 = Lh[1]
  int tl0, tl1;      // the neighbour's
  double sig, wsc;   // penalty and Jacobian of the part's face
};

// V: the field type (double, or float in the FP32 inner solve); tables and
// arithmetic in V too, the leaf sizes and penalties in FP64 until the final cast
template <typename V, int N1>
__global__ void __launch_bounds__(256) k_octree_apply(const OctTables T, const double* __restrict__ hq,
                                                      const int* __restrict__ kind, const int* __restrict__ nbr,
                                                      const int* __restrict__ pos, int E, int p, int pform,
                                                      double eps, const V* __restrict__ u, V* __restrict__ out,
                                                      const int* __restrict__ act) {
  constexpr int NPE = N1 * N1 * N1, NF = N1 * N1;
  extern __shared__ __align__(16) unsigned char pbuf_raw[];
  V* pbuf = (V*)pbuf_raw;  // [nparts][6][NF]
  __shared__ V sTab[3][NF], sS[NF], sLe[2][N1], sdLe[2][N1], sw[N1], swq[N1];
  __shared__ V uK[NPE], acc[NPE], VK[6][2][NF];
  __shared__ OctPart part[24];
  __shared__ int npart;
  __shared__ double hK[3];
  const int e = blockIdx.x;
  const int tid = threadIdx.x, NT = blockDim.x;
  const long long src = act ? act[blockIdx.y] : blockIdx.y;
  const V* ub = u + src * E * NPE;
  V* ob = out + src * E * NPE;
  for (int i = tid; i < NF; i += NT) {
    const int r = i / N1, c = i % N1;
    sTab[0][i] = (V)T.Lq[r * N1 + c];
    sTab[1][i] = (V)T.Lh[0][r * N1 + c];
    sTab[2][i] = (V)T.Lh[1][r * N1 + c];
    sS[i] = (V)T.S[r * N1 + c];
  }
  for (int i = tid; i < N1; i += NT) {
    sLe[0][i] = (V)T.Le[0][i];
    sLe[1][i] = (V)T.Le[1][i];
    sdLe[0][i] = (V)T.dLe[0][i];
    sdLe[1][i] = (V)T.dLe[1][i];
    sw[i] = (V)T.w[i];
    swq[i] = (V)T.wq[i];
  }
  for (int i = tid; i < NPE; i += NT) uK[i] = ub[(long long)e * NPE + i];
  if (tid < 3) hK[tid] = hq[3LL * e + tid];
  __syncthreads();
  // the leaf's face parts, one thread per (face f, quarter qi) slot: part index =
  // the parts of the faces before f, plus qi
  if (tid < 24) {
    const int f = tid >> 2, qi = tid & 3;
    int kd = 0, start = 0, total = 0;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const int kg = kind[6LL * e + g];
      const int ng = kg == 3 ? 4 : 1;
      if (g < f) start += ng;
      if (g == f) kd = kg;
      total += ng;
    }
    if (tid == 0) npart = total;
    if (qi < (kd == 3 ? 4 : 1)) {
      const int d = f >> 1, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
      const long long o = 6LL * e + f;
      OctPart& P = part[start + qi];
      P.f = f;
      P.tk0 = kd == 3 ? 1 + (qi & 1) : 0;
      P.tk1 = kd == 3 ? 1 + (qi >> 1) : 0;
      const int ps = kd == 2 ? pos[o] : 0;
      P.tl0 = kd == 2 ? 1 + (ps & 1) : 0;
      P.tl1 = kd == 2 ? 1 + (ps >> 1) : 0;
      if (kd == 0) {
        P.L = -1;
        P.sig = oct_penalty(p, hK[d], pform, eps);
        P.wsc = hK[t0] * hK[t1] / 4.0;
      } else {
        P.L = kd == 3 ? nbr[4 * o + qi] : nbr[4 * o];
        const double* hL = hq + 3LL * P.L;
        P.sig = oct_penalty(p, fmin(hK[d], hL[d]), pform, eps);
        P.wsc = kd == 3 ? hL[t0] * hL[t1] / 4.0 : hK[t0] * hK[t1] / 4.0;
      }
    }
  }
  __syncthreads();
  const int np = npart;
  // 1. volume: sum_d (2/h_d)(h_t0 h_t1 / 4) (S_d (x) W (x) W) u
  for (int i = tid; i < NPE; i += NT) {
    const int ix = i % N1, iy = (i / N1) % N1, iz = i / NF;
    V vx = 0, vy = 0, vz = 0;
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      vx += sS[ix * N1 + a] * uK[a + N1 * iy + NF * iz];
      vy += sS[iy * N1 + a] * uK[ix + N1 * a + NF * iz];
      vz += sS[iz * N1 + a] * uK[ix + N1 * iy + NF * a];
    }
    acc[i] = vx * sw[iy] * sw[iz] * (V)((2.0 / hK[0]) * (hK[1] * hK[2] / 4.0)) +
             vy * sw[ix] * sw[iz] * (V)((2.0 / hK[1]) * (hK[0] * hK[2] / 4.0)) +
             vz * sw[ix] * sw[iy] * (V)((2.0 / hK[2]) * (hK[0] * hK[1] / 4.0));
  }
  // 1. this leaf's traces and outward normal derivatives on its face nodes [t0][t1]
  for (int t = tid; t < 6 * NF; t += NT) {
    const int f = t / NF, j = t - f * NF;
    const int d = f >> 1, r = f & 1, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    const int b = j / N1, c = j % N1;
    const int sd = oct_stride<N1>(d), base = b * oct_stride<N1>(t0) + c * oct_stride<N1>(t1);
    V v = 0, dv = 0;
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      const V x = uK[a * sd + base];
      v += sLe[r][a] * x;
      dv += sdLe[r][a] * x;
    }
    VK[f][0][j] = v;
    VK[f][1][j] = dv * (V)((2.0 / hK[d]) * (r ? 1.0 : -1.0));
  }
  // 1. the neighbours' traces (on the neighbour's own face nodes) into buffers 0, 1
  for (int t = tid; t < np * NF; t += NT) {
    const int k = t / NF, j = t - k * NF;
    const OctPart& P = part[k];
    const int L = P.L;
    V* B = pbuf + (size_t)k * 6 * NF;
    if (L < 0) continue;
    const int d = P.f >> 1, r = P.f & 1, rl = 1 - r, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    const int b = j / N1, c = j % N1;
    const V* uL = ub + (long long)L * NPE + b * oct_stride<N1>(t0) + c * oct_stride<N1>(t1);
    const int sd = oct_stride<N1>(d);
    V v = 0, dv = 0;
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      const V x = uL[a * sd];
      v += sLe[rl][a] * x;
      dv += sdLe[rl][a] * x;
    }
    B[j] = v;
    B[NF + j] = dv * (V)((2.0 / hq[3LL * L + d]) * (r ? 1.0 : -1.0));
  }
  __syncthreads();
  // 2. first contraction along t1: R_X[b][jj] = sum_c T1[jj][c] X[b][c] into buffers 2..5
  //    (X = this leaf's value, derivative, the neighbour's value, derivative)
  for (int t = tid; t < np * 4 * NF; t += NT) {
    const int k = t / (4 * NF), rem = t - k * 4 * NF, x = rem / NF, q = rem - x * NF;
    const OctPart& P = part[k];
    V* B = pbuf + (size_t)k * 6 * NF;
    if (x >= 2 && P.L < 0) continue;
    const int b = q / N1, jj = q % N1;
    const V* X = x < 2 ? VK[P.f][x] : B + (x - 2) * NF;
    const V* T1 = sTab[x < 2 ? P.tk1 : P.tl1];
    V s = 0;
#pragma unroll
    for (int c = 0; c < N1; ++c) s += T1[jj * N1 + c] * X[b * N1 + c];
    B[(2 + x) * NF + q] = s;
  }
  __syncthreads();
  // 3. second contraction along t0 at the Gauss point (i, jj), and the fluxes into buffers 0, 1
  for (int t = tid; t < np * NF; t += NT) {
    const int k = t / NF, q = t - k * NF;
    const OctPart& P = part[k];
    V* B = pbuf + (size_t)k * 6 * NF;
    const int i = q / N1, jj = q % N1;
    const V* T0K = sTab[P.tk0];
    V pv = 0, pd = 0;
#pragma unroll
    for (int b = 0; b < N1; ++b) {
      pv += T0K[i * N1 + b] * B[2 * NF + b * N1 + jj];
      pd += T0K[i * N1 + b] * B[3 * NF + b * N1 + jj];
    }
    const V wt = swq[i] * swq[jj] * (V)P.wsc;
    const V sig = (V)P.sig;
    V F1, F2;
    if (P.L < 0) {
      F1 = wt * (-pd + sig * pv);
      F2 = wt * (-pv);
    } else {
      const V* T0L = sTab[P.tl0];
      V qv = 0, qd = 0;
#pragma unroll
      for (int b = 0; b < N1; ++b) {
        qv += T0L[i * N1 + b] * B[4 * NF + b * N1 + jj];
        qd += T0L[i * N1 + b] * B[5 * NF + b * N1 + jj];
      }
      F1 = wt * ((V)-0.5 * (pd + qd) + sig * (pv - qv));
      F2 = wt * ((V)-0.5 * (pv - qv));
    }
    B[q] = F1;
    B[NF + q] = F2;
  }
  __syncthreads();
  // 4. back along t1: H_Y[i][c] = sum_jj F_Y[i][jj] T1K[jj][c] into buffers 2, 3
  for (int t = tid; t < np * 2 * NF; t += NT) {
    const int k = t / (2 * NF), rem = t - k * 2 * NF, y = rem / NF, q = rem - y * NF;
    const OctPart& P = part[k];
    V* B = pbuf + (size_t)k * 6 * NF;
    const int i = q / N1, c = q % N1;
    const V* T1 = sTab[P.tk1];
    V s = 0;
#pragma unroll
    for (int jj = 0; jj < N1; ++jj) s += B[y * NF + i * N1 + jj] * T1[jj * N1 + c];
    B[(2 + y) * NF + q] = s;
  }
  __syncthreads();
  // 5. back along t0: G_Y[b][c] = sum_i T0K[i][b] H_Y[i][c] into buffers 4, 5
  for (int t = tid; t < np * 2 * NF; t += NT) {
    const int k = t / (2 * NF), rem = t - k * 2 * NF, y = rem / NF, q = rem - y * NF;
    const OctPart& P = part[k];
    V* B = pbuf + (size_t)k * 6 * NF;
    const int b = q / N1, c = q % N1;
    const V* T0 = sTab[P.tk0];
    V s = 0;
#pragma unroll
    for (int i = 0; i < N1; ++i) s += T0[i * N1 + b] * B[(2 + y) * NF + i * N1 + c];
    B[(4 + y) * NF + q] = s;
  }
  __syncthreads();
  // 6. face contributions onto the leaf's nodes: l_a(e) G1 + l_a'(e) (2/h) s G2, parts in order
  for (int i = tid; i < NPE; i += NT) {
    const int ix = i % N1, iy = (i / N1) % N1, iz = i / NF;
    V a_ = acc[i];
    for (int k = 0; k < np; ++k) {
      const OctPart& P = part[k];
      const V* B = pbuf + (size_t)k * 6 * NF;
      const int d = P.f >> 1, r = P.f & 1;
      // (a, b, c) = the node's coordinates along d, t0, t1
      const int a = d == 0 ? ix : (d == 1 ? iy : iz);
      const int bc = d == 0 ? iy * N1 + iz : (d == 1 ? ix * N1 + iz : ix * N1 + iy);
      a_ += sLe[r][a] * B[4 * NF + bc] + sdLe[r][a] * (V)((2.0 / hK[d]) * (r ? 1.0 : -1.0)) * B[5 * NF + bc];
    }
    ob[(long long)e * NPE + i] = a_;
  }
}

int octree_max_parts(const int32_t* kind, int E) {
  int m = 6;
  for (int e = 0; e < E; ++e) {
    int n = 0;
    for (int f = 0; f < 6; ++f) n += kind[6 * (size_t)e + f] == 3 ? 4 : 1;
    m = std::max(m, n);
  }
  return m;
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

template <typename V>
cudaError_t launch_octree_apply(int n1, const OctTables& T, const double* hq, const int* kind, const int* nb,
                                const int* pos, int E, int p, int pform, double eps, const V* u, V* out,
                                const int* act, int nact, int maxparts, cudaStream_t s) {
  if (nact == 0 || E == 0) return cudaSuccess;
  if (maxparts < 6 || maxparts > 24) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)E, (unsigned)nact);
  const size_t smem = sizeof(V) * (size_t)maxparts * 6 * n1 * n1;
  // threads per block by degree: the phases have (p+1)^2 to 24 (p+1)^2 work items
  const int nthr = n1 <= 3 ? 64 : (n1 <= 5 ? 128 : 256);
  count_launch();
  switch (n1) {
#define DG_OCT_CASE(N)                                                                                       \
  case N: {                                                                                                  \
    cudaError_t e0 = cudaFuncSetAttribute(k_octree_apply<V, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                          (int)smem);                                                        \
    if (e0 != cudaSuccess) return e0;                                                                        \
    k_octree_apply<V, N><<<grid, nthr, smem, s>>>(T, hq, kind, nb, pos, E, p, pform, eps, u, out, act);         \
    break;                                                                                                   \
  }
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
template cudaError_t launch_octree_apply<double>(int, const OctTables&, const double*, const int*, const int*,
                                                 const int*, int, int, int, double, const double*, double*, const int*,
                                                 int, int, cudaStream_t);
template cudaError_t launch_octree_apply<float>(int, const OctTables&, const double*, const int*, const int*,
                                                const int*, int, int, int, double, const float*, float*, const int*,
                                                int, int, cudaStream_t);
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
  if ((rc = ck(launch_octree_apply<double>(n1, T, dh.as<double>(), dk.as<int>(), dn.as<int>(), dp.as<int>(), E, root->p,
                                   penalty_form, penalty_eps, u, out, nullptr, (int)B, octree_max_parts(kind.data(), E),
                                   s))) != DG_OK)
    return rc;
  // the tables and connectivity are call-local: wait before they are freed
  return ck(cudaStreamSynchronize(s));
}

}  // extern "C"
