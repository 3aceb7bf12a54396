// Tables and launcher of the tensor-core Schwarz patch solve
// (dg_schwarz_tc.cu), shared with the host set-up.
#pragma once

#include <stdint.h>

#include <vector>

#include "dg_internal.h"

namespace dg {

constexpr int SWTC_LBO = 144;        // byte stride of K-adjacent core matrices (128 + 16: conflict-free stores)
// warp roles: consumers first (one thread per TMEM lane: z-step and output;
// at n1 = 8 two warps per lane quarter, each taking every other patch of an
// item), then 4 producer warps (item decode and the residual fill), then the
// MMA issuer
// Tuning switches (compile-time; defaults chosen by timing on a GB300):
// DG_SWTC_ROWFILL: at n1 = 8 fill the residual operand by 16-byte copies of
// element rows (K order permuted, x-halos shared within an item); 0: one
// 4-byte load per operand entry, as at the other degrees.
// DG_SWTC_WIDE: at n1 = 8 two consumer warps per TMEM lane quarter (z factor
// read from shared memory); 0: one warp per quarter with the z factor in
// registers.
#ifndef DG_SWTC_ROWFILL
#define DG_SWTC_ROWFILL 1
#endif
// DG_SWTC_LDG: patches per batch of tensor-memory loads in the consumer warps
// (the next batch is in flight while one is processed).
#ifndef DG_SWTC_LDG
#define DG_SWTC_LDG 1
#endif
#ifndef DG_SWTC_WIDE
#define DG_SWTC_WIDE 0
#endif
__host__ __device__ constexpr int swtc_consumers(int n1) { return n1 == 8 && DG_SWTC_WIDE ? 256 : 128; }
// producers: 4 warps (one thread per operand column in the 4-byte fill), 3 with
// the row fill, so that the CTA has 8 warps: two per SM sub-partition, whose
// register file (16 K registers) then allows up to 255 registers a thread
// (with 9 warps one sub-partition holds three, and the cap is 168)
__host__ __device__ constexpr int swtc_producers(int n1) { return n1 == 8 && DG_SWTC_ROWFILL && !DG_SWTC_WIDE ? 96 : 128; }
__host__ __device__ constexpr int swtc_threads(int n1) { return swtc_consumers(n1) + swtc_producers(n1) + 32; }
// rings of the pipeline: B operands in shared memory, FP32 accumulators in
// tensor memory, item descriptions
constexpr int SWTC_BSLOTS = 2, SWTC_DSLOTS = 3, SWTC_ISLOTS = 4;
constexpr int SWTC_TMEM_COLS = 512;  // three accumulators of up to 128 columns
constexpr int SWTC_MAXCLS = 8;       // position classes per axis
constexpr int SWTC_MAXZCLS = 5;      // position classes along z (at most 5 on a uniform mesh)
constexpr int SWTC_MAXSEG = SWTC_MAXCLS * SWTC_MAXCLS;
constexpr int SWTC_CS = 12;          // B rows / D columns per patch (MP <= 11, padded to a multiple of 4)
constexpr int SWTC_NPMAX = 10;       // patches per work item
constexpr int SWTC_MAXCOLS = 768;    // element columns (nx * ny) staged in shared memory
constexpr int SWTC_MAXNZ = 256;      // elements along z
constexpr int SWTC_MAXACT = 256;     // active sources staged in shared memory (more are read from global)
// floats per z class: S and S^T with rows padded to a multiple of 4 (16-byte
// row loads), lambda (padded), m
#define SWTC_MPP(MP) (((MP) + 3) / 4 * 4)
#define SWTC_ZSTR(MP) (2 * (MP) * SWTC_MPP(MP) + SWTC_MPP(MP) + 4)

// operand geometry for one degree
struct SwTcGeom {
  int mp;       // patch nodes per axis, n1 + 2
  int kpad;     // K of both MMAs: mp^2 padded to a multiple of 8
  int kc;       // 16-byte core-matrix columns along K (kpad / 4)
  int sbo;      // bytes per 8-row group (kc * SWTC_LBO)
  int a_bytes;  // one Kronecker factor in shared memory (ceil(mp^2 / 8) row groups)
  int np;       // patches per work item
  int ncol;     // N of the MMAs: np * SWTC_CS rounded up to a multiple of 16
  int b_bytes;  // the B operand of one stage (ncol / 8 row groups)
};

// Header of a level's table blob (device memory, read by the kernel). Offsets
// are bytes from the blob start; float tables per class.
struct SwTcHead {
  SwTcGeom geom;
  int n1, nx, ny, nz;
  int nseg, ncx, ncy, ncz;
  int* err;             // device word set to DG_ERR_TIMEOUT when a wait gives up
  long long off_cols;   // int [ncol][2]: element columns (ex, ey), grouped by segment
  long long off_zcls;   // int [nz]: class of each z position
  long long off_z;      // float [ncz][SWTC_ZSTR]: Sz [node][mode], Sz^T [mode][node] (rows of SWTC_MPP), lambda_z, m_z
  long long off_xy;     // float [ncx][mp + 1] then [ncy][mp + 1]: lambda, m
  long long off_y;      // float offset of the y classes inside off_xy
  long long off_a;      // per segment: forward factor then inverse factor, a_bytes each
  int seg_col0[SWTC_MAXSEG], seg_ncol[SWTC_MAXSEG], seg_cx[SWTC_MAXSEG], seg_cy[SWTC_MAXSEG];
};

// per-stage description of the work item in flight
struct SwTcItem {
  int np, seg;
  int src[SWTC_NPMAX], elem[SWTC_NPMAX];
  short ex[SWTC_NPMAX], ey[SWTC_NPMAX], ez[SWTC_NPMAX], cz[SWTC_NPMAX];
  // residual offset of patch z-node k relative to its plane (x, y) part, -1 outside the domain
  int zoff[SWTC_NPMAX][SWTC_CS];
  // row fill at n1 = 8: offset of the patch's element in the residual, and
  // flags: bit 0 left overlap along y, bits 1-4 patch nodes along y, bits 6 / 7
  // x-halo left / right taken from the neighbouring patch of the item, bits 8 / 9
  // a left / right neighbour element exists
  long long rbase[SWTC_NPMAX];
  unsigned short pf[SWTC_NPMAX];
};

// static shared memory of the kernel
struct SwTcShared {
  // per B slot: filled by the producers (full), rewritten by the consumers (b2);
  // per accumulator slot: MMA 1 done (d1), MMA 2 done (d2), read out (empty);
  // the two factor copies
  unsigned long long full[SWTC_BSLOTS], b2[SWTC_BSLOTS];
  unsigned long long d1[SWTC_DSLOTS], d2[SWTC_DSLOTS], empty[SWTC_DSLOTS];
  unsigned long long tma_f, tma_i;
  uint32_t tmem;
  int abort;
  int item0[SWTC_MAXSEG + 1];
  SwTcItem item[SWTC_ISLOTS];
  alignas(16) float z[SWTC_MAXZCLS * SWTC_ZSTR(11)];
  // the level's tables, staged once per launch (no global loads on the item path)
  int seg_col0[SWTC_MAXSEG], seg_ncol[SWTC_MAXSEG];
  unsigned char seg_cx[SWTC_MAXSEG], seg_cy[SWTC_MAXSEG];
  short2 cols[SWTC_MAXCOLS];
  unsigned char zcls[SWTC_MAXNZ];
  unsigned short act[SWTC_MAXACT];
  float lxy[2][SWTC_MAXCLS][12];  // per x / y class: lambda [MP], m
};

// a level's tensor-core patch solve: device blob, a host copy of its header,
// and the operand geometry in use (patches per item; the autotuner may pick
// another count, or switch the level to the SIMT patch kernel)
struct SwTcPlan {
  const void* blob = nullptr;
  SwTcHead head;
  SwTcGeom geom;
  bool off = false;
};

// operand geometry for degree n1 - 1 with np patches per item (0: the default,
// the largest count that fits); false if the degree or count does not fit
bool swtc_geometry(int n1, SwTcGeom& g, int np = 0);
// K slot of patch node (j, l) in the residual operand at n1 = 8 (-1: no node)
int swtc_fill_k(int j, int l, int oLx, int mx);
std::vector<unsigned char> schwarz_tc_blob(const LevelOp& L, const std::vector<double>& tabs, int* err_dev);
cudaError_t schwarz_tc_prepare(int n1);
cudaError_t launch_schwarz_patch_tc(const LevelOp& hop, const LevelOp* dop, const SwTcPlan& plan, const float* r,
                                    float* zp, const int* act, int nact, cudaStream_t s);

}  // namespace dg
