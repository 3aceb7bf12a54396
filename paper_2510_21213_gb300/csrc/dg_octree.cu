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
#include <map>
#include <set>
#include <vector>

#include "dg_internal.h"
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
  if (!root || !leaves || n_leaves < 1 || !kind || !nb || !pos) return DG_ERR_INVALID_ARG;
  Octree t;
  for (int d = 0; d < 3; ++d) {
    if (root->n[d] < 1 || !(root->hi[d] > root->lo[d])) return DG_ERR_INVALID_ARG;
    t.lo[d] = root->lo[d];
    t.n[d] = root->n[d];
    t.H[d] = (root->hi[d] - root->lo[d]) / root->n[d];
  }
  t.p = root->p;
  std::map<Leaf, int> index;
  for (int e = 0; e < n_leaves; ++e) {
    const Leaf k{leaves[4 * e], leaves[4 * e + 1], leaves[4 * e + 2], leaves[4 * e + 3]};
    if (k[0] < 0 || k[0] > 20) return DG_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
      if (k[1 + d] < 0 || k[1 + d] >= t.extent(k[0], d)) return DG_ERR_INVALID_ARG;
    if (!index.emplace(k, e).second) return DG_ERR_INVALID_ARG;
    t.leaves.insert(k);
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
        if (t.covering(c[0], c[1], c[2], c[3], L)) {
          if (L[0] == k[0]) {
            kind[o] = 1;
          } else if (L[0] == k[0] - 1) {
            kind[o] = 2;  // this face is a quarter of L's face: its two tangential bits
            const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
            pos[o] = (k[1 + t0] & 1) | ((k[1 + t1] & 1) << 1);
          } else {
            return DG_ERR_INVALID_ARG;  // not 2:1 balanced
          }
          nb[4 * o] = index.at(L);
          continue;
        }
        // four smaller neighbours: the level + 1 cells touching this face
        kind[o] = 3;
        const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
        for (int j = 0; j < 4; ++j) {
          Leaf s{k[0] + 1, 2 * k[1], 2 * k[2], 2 * k[3]};
          s[1 + d] = sd ? 2 * k[1 + d] + 2 : 2 * k[1 + d] - 1;
          s[1 + t0] += j & 1;
          s[1 + t1] += j >> 1;
          auto it = index.find(s);
          if (it == index.end()) return DG_ERR_INVALID_ARG;  // not 2:1 balanced or not a leaf set
          nb[4 * o + j] = it->second;
        }
      }
  }
  return DG_OK;
}

}  // extern "C"
