// Tables and launcher of the tensor-core Schwarz patch solve
// (dg_schwarz_tc.cu), shared with the host set-up.
#pragma once

#include <stdint.h>

#include <vector>

#include "dg_internal.h"
#include "dg_tc.h"

namespace dg {

constexpr int SWTC_LBO = 144;        // byte stride of K-adjacent core matrices (128 + 16: conflict-free stores)
// Warp roles: 4 consumer warps (one thread per TMEM lane), then the producer
// warps (item decode and the residual fill: 4, one thread per operand column,
// in the kernel of degrees 6 and 8; 3 in the degree-7 kernel, so that its CTA
// has 8 warps, two per SM sub-partition, whose 16 K registers then allow up
// to 255 registers a thread; with 9 warps one sub-partition holds three and
// the cap is 168), then one warp whose first thread issues the MMAs.
constexpr int SWTC_CONSUMERS = 128;
// DG_SWTC_ZTC (compile-time): at degree 7 run the z factor on the tensor cores
// too (dg_schwarz_tc8.cu: A operand read from tensor memory, 7 patches per
// item). Measured slower than the FP32 z-step at 16^3 p = 7 with 42 sources
// (1.08 against 0.84 ms per launch: its two-slot pipeline waits on the chain
// fill -> MMA 1 -> z1 -> scaling -> MMA 2 -> z2), so it is off by default.
#ifndef DG_SWTC_ZTC
#define DG_SWTC_ZTC 0
#endif
// DG_SWTC_SPLIT (compile-time): 1 = every CTA takes a share of every class
// pair (balanced mix of item costs, a factor reload per class pair); 0 = each
// CTA a contiguous range of the item list.
#ifndef DG_SWTC_SPLIT
#define DG_SWTC_SPLIT 1
#endif
__host__ __device__ constexpr int swtc_producers(int n1) { return n1 == 8 ? 96 : 128; }
__host__ __device__ constexpr int swtc_threads(int n1) { return SWTC_CONSUMERS + swtc_producers(n1) + 32; }
// rings of the pipeline: B operands in shared memory, FP32 accumulators in
// tensor memory, item descriptions
constexpr int SWTC_BSLOTS = 2, SWTC_DSLOTS = 3, SWTC_ISLOTS = 4;
constexpr int SWTC_TMEM_COLS = 512;  // three accumulators of up to 128 columns
constexpr int SWTC_MAXCLS = 8;       // position classes per axis
constexpr int SWTC_MAXZCLS = 5;      // position classes along z (at most 5 on a uniform mesh)
constexpr int SWTC_MAXSEG = SWTC_MAXCLS * SWTC_MAXCLS;
constexpr int SWTC_CS = 12;          // B rows / D columns per patch (MP <= 11, padded to a multiple of 4)
constexpr int SWTC_NPMAX = 10;       // patches per work item
// degree 7 with DG_SWTC_ZTC: 16 rows / columns per patch, so that each patch's z line
// is one 16-wide operand of the z-factor MMAs; at most 7 patches per item
// (two items in flight, each with two 128-column accumulators)
constexpr int SWTC8_CS = 16, SWTC8_NPMAX = 7;
// z-factor operands of the degree-7 kernel: per z class Sz^T and Sz as 16 x 16
// TF32 matrices, K-major core matrices (16-byte groups of K 128 bytes apart,
// 8-row groups 512 bytes apart)
constexpr int SWTC_ZB_BYTES = 1024, SWTC_ZB_LBO = 128, SWTC_ZB_SBO = 512;
constexpr int SWTC_MAXCOLS = 768;    // element columns (nx * ny) staged in shared memory
constexpr int SWTC_MAXNZ = 256;      // elements along z
constexpr int SWTC_MAXACT = 256;     // active sources staged in shared memory (more are read from global)
// floats per z class: S (rows padded to a multiple of 4), lambda (padded), m
#define SWTC_MPP(MP) (((MP) + 3) / 4 * 4)
#define SWTC_ZSTR(MP) ((MP) * SWTC_MPP(MP) + SWTC_MPP(MP) + 4)

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
  int cs;       // B rows / D columns per patch
  int zb_bytes; // z-factor operands in shared memory (degree 7), 0 otherwise
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
  long long off_z;      // float [ncz][SWTC_ZSTR]: Sz [node][mode] (rows of SWTC_MPP), lambda_z, m_z
  long long off_zb;     // degree 7: per z class the operands Sz^T then Sz (SWTC_ZB_BYTES each)
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
  // degree-7 kernel: z-forward MMAs done (e), z-inverse MMAs done (f), item
  // description slot free (ifree)
  unsigned long long e[2], f[2], ifree[SWTC_ISLOTS];
  uint32_t tmem;
  int abort;
  int item0[SWTC_MAXSEG + 1];
  // degree-7 kernel: this CTA's share of every segment (first item in the
  // segment, count of its items before the segment)
  int mine0[SWTC_MAXSEG], mcum[SWTC_MAXSEG + 1];
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
cudaError_t schwarz_tc8_prepare(const SwTcGeom& g);
cudaError_t launch_schwarz_patch_tc8(const SwTcPlan& plan, const float* r, float* zp, const int* act, int nact,
                                     cudaStream_t s);

// Bounded wait on a shared-memory mbarrier phase (about a second); on a
// timeout the kernel's error word gets DG_ERR_TIMEOUT and the CTA's abort flag
// is set, so that every role leaves its loop.
constexpr long long kSwtcWaitLimit = 1LL << 31;  // clock cycles
__device__ __forceinline__ bool swtc_wait(SwTcShared& sh, const SwTcHead* H, unsigned long long* bar,
                                          uint32_t parity) {
  if (tc::mbar_wait(tc::smem_addr(bar), parity, kSwtcWaitLimit)) return true;
  atomicExch(H->err, DG_ERR_TIMEOUT);
  atomicExch(&sh.abort, 1);
  return false;
}
cudaError_t launch_schwarz_patch_tc(const LevelOp& hop, const LevelOp* dop, const SwTcPlan& plan, const float* r,
                                    float* zp, const int* act, int nact, cudaStream_t s);

}  // namespace dg
