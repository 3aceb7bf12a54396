// Tables and launcher of the tensor-core Schwarz patch solve
// (dg_schwarz_tc.cu), shared with the host set-up.
#pragma once

#include <stdint.h>

#include <vector>

#include "dg_internal.h"

namespace dg {

constexpr int SWTC_LBO = 144;        // byte stride of K-adjacent core matrices (128 + 16: conflict-free stores)
// warp roles: 0-3 consumers (one thread per TMEM lane: z-step and output),
// 4-7 producers (item decode and the residual fill), 8 the MMA issuer
constexpr int SWTC_CONSUMERS = 128, SWTC_PRODUCERS = 128;
constexpr int SWTC_THREADS = SWTC_CONSUMERS + SWTC_PRODUCERS + 32;
// rings of the pipeline: B operands in shared memory, FP32 accumulators in
// tensor memory, item descriptions
constexpr int SWTC_BSLOTS = 2, SWTC_DSLOTS = 3, SWTC_ISLOTS = 4;
constexpr int SWTC_TMEM_COLS = 512;  // three accumulators of up to 128 columns
constexpr int SWTC_MAXCLS = 8;       // position classes per axis
constexpr int SWTC_MAXSEG = SWTC_MAXCLS * SWTC_MAXCLS;
constexpr int SWTC_CS = 12;          // B rows / D columns per patch (MP <= 11, padded to a multiple of 4)
constexpr int SWTC_NPMAX = 10;       // patches per work item
constexpr int SWTC_MAXCOLS = 1024;   // element columns (nx * ny) staged in shared memory
constexpr int SWTC_MAXNZ = 256;      // elements along z
constexpr int SWTC_MAXACT = 256;     // active sources staged in shared memory (more are read from global)
#define SWTC_ZSTR(MP) ((MP) * (MP) + (MP) + 1)  // floats per z class: S, lambda, m

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
  long long off_z;      // float [ncz][SWTC_ZSTR]: Sz (row node, col mode), lambda_z, m_z
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
  float z[SWTC_MAXCLS * SWTC_ZSTR(11)];
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
std::vector<unsigned char> schwarz_tc_blob(const LevelOp& L, const std::vector<double>& tabs, int* err_dev);
cudaError_t schwarz_tc_prepare(int n1);
cudaError_t launch_schwarz_patch_tc(const LevelOp& hop, const LevelOp* dop, const SwTcPlan& plan, const float* r,
                                    float* zp, const int* act, int nact, cudaStream_t s);

}  // namespace dg
