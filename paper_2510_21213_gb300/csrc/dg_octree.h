// Octree auxiliary mesh (Sec. 6.2): connectivity, the operator's 1-D tables
// and the operator launcher (dg_octree.cu), shared with the octree solver
// (dg_octree_solve.cu).
#pragma once

#include <stdint.h>

#include "dg_internal.h"

namespace dg {

// 1-D tables of the octree operator for one degree (n1 nodes per axis)
struct OctTables {
  double w[MAXN1];               // GL weights
  double wq[MAXN1];              // Gauss weights (n1 points per face direction)
  double S[MAXN1 * MAXN1];       // sum_q wq l_a'(xq) l_b'(xq)
  double Lq[MAXN1 * MAXN1];      // [i][a] l_a(xq_i)
  double Lh[2][MAXN1 * MAXN1];   // [c][i][a] l_a((xq_i + 2c - 1) / 2): a larger leaf's basis on half c
  double Le[2][MAXN1];           // l_a(-1), l_a(+1)
  double dLe[2][MAXN1];          // l_a'(-1), l_a'(+1)
};

void octree_tables(int n1, OctTables& T);

// Face connectivity of a leaf set ([E][4] level, ix, iy, iz); per leaf and face
// f = 2 d + side: kind 0 boundary, 1 same-size neighbour, 2 larger neighbour
// (pos: this face's quarter of it), 3 four smaller neighbours (nb[4]). False
// for a bad mesh, a leaf set that is not a partition, or one not 2:1 balanced.
bool octree_faces(const dg_mesh_desc* root, const int32_t* leaves, int32_t n_leaves, int32_t* kind, int32_t* nb,
                  int32_t* pos);

// largest number of face parts of a leaf (a face with four smaller neighbours
// counts four, any other face one): 6..24, the operator's shared-memory size
int octree_max_parts(const int32_t* kind, int E);

// out[k] = A u[k] for the sources k = act[0..nact) (act null: k = 0..nact),
// u and out [.][E][n1^3]; hq [E][3] leaf sizes, kind/nb/pos as octree_faces;
// maxparts = octree_max_parts of the mesh; V = double or float (the fields and
// the arithmetic)
template <typename V>
cudaError_t launch_octree_apply(int n1, const OctTables& T, const double* hq, const int* kind, const int* nb,
                                const int* pos, int E, int p, int pform, double eps, const V* u, V* out,
                                const int* act, int nact, int maxparts, cudaStream_t s);

}  // namespace dg
