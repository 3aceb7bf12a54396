// Tables and launcher of the tensor-core Schwarz patch solve
// (dg_schwarz_tc.cu), shared with the host set-up.
#pragma once

#include <stdint.h>

#include <vector>

#include "dg_internal.h"

namespace dg {

constexpr int SWTC_LBO = 144;        // byte stride of K-adjacent core matrices (128 + 16: conflict-free stores)
constexpr int SWTC_THREADS = 256;    // two warps per TMEM lane quadrant
constexpr int SWTC_TMEM_COLS = 256;  // one FP32 accumulator of up to 256 columns
constexpr int SWTC_MAXCLS = 8;       // position classes per axis
constexpr int SWTC_MAXSEG = SWTC_MAXCLS * SWTC_MAXCLS;
constexpr int SWTC_CS = 12;          // B rows / D columns per patch (MP <= 11, padded to a multiple of 4)
constexpr int SWTC_NPMAX = 21;       // patches per work item
#define SWTC_ZSTR(MP) ((MP) * (MP) + (MP) + 1)  // floats per z class: S, lambda, m

// operand geometry for one degree
struct SwTcGeom {
  int mp;       // patch nodes per axis, n1 + 2
  int kpad;     // K of both MMAs: mp^2 padded to a multiple of 8
  int kc;       // 16-byte core-matrix columns along K (kpad / 4)
  int sbo;      // bytes per 8-row group (kc * SWTC_LBO)
  int a_bytes;  // one Kronecker factor in shared memory (ceil(mp^2 / 8) row groups)
  int np;       // patches per work item
  int ncol;     // N of the MMAs: np * mp rounded up to a multiple of 16
  int b_bytes;  // the B operand (ncol / 8 row groups)
};

// Header of a level's table blob (device memory, read by the kernel). Offsets
// are bytes from the blob start; float tables per class.
struct SwTcHead {
  SwTcGeom geom;
  int n1, nx, ny, nz;
  int nseg, ncz;
  int* err;             // device word set to DG_ERR_TIMEOUT when a wait gives up
  long long off_cols;   // int [ncol][2]: element columns (ex, ey), grouped by segment
  long long off_zcls;   // int [nz]: class of each z position
  long long off_z;      // float [ncz][SWTC_ZSTR]: Sz (row node, col mode), lambda_z, m_z
  long long off_xy;     // float [ncx][mp + 1] then [ncy][mp + 1]: lambda, m
  long long off_y;      // float offset of the y classes inside off_xy
  long long off_a;      // per segment: forward factor then inverse factor, a_bytes each
  int seg_col0[SWTC_MAXSEG], seg_ncol[SWTC_MAXSEG], seg_cx[SWTC_MAXSEG], seg_cy[SWTC_MAXSEG];
};

// static shared memory of the kernel
struct SwTcShared {
  unsigned long long mbar_tma, mbar_mma;
  uint32_t tmem;
  int abort;
  int item0[SWTC_MAXSEG + 1];
  int src[SWTC_NPMAX], elem[SWTC_NPMAX], ez[SWTC_NPMAX], ex[SWTC_NPMAX], ey[SWTC_NPMAX];
  float z[SWTC_MAXCLS * SWTC_ZSTR(11)];
};

// a level's tensor-core patch solve: device blob and a host copy of its header
struct SwTcPlan {
  const void* blob = nullptr;
  SwTcHead head;
};

bool swtc_geometry(int n1, SwTcGeom& g);
std::vector<unsigned char> schwarz_tc_blob(const LevelOp& L, const std::vector<double>& tabs, int* err_dev);
cudaError_t schwarz_tc_prepare(int n1);
cudaError_t launch_schwarz_patch_tc(const LevelOp& hop, const LevelOp* dop, const SwTcPlan& plan, const float* r,
                                    float* zp, const int* act, int nact, cudaStream_t s);

}  // namespace dg
