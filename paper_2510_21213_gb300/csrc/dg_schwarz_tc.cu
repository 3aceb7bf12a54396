// Tensor-core patch solve of the overlapping Schwarz smoother (FP32 inner
// solve, levels of degree 6-8): tables, geometry and the kernel (a variant at
// degree 7 that also runs the z factor on the tensor cores, off by default,
// is in dg_schwarz_tc8.cu).
//
// Each patch problem of the smoother is solved exactly by fast
// diagonalisation (Sec. 3.4: the SIPDG operator is a Kronecker sum, so its
// restriction to a tensor box of nodes is one too):
//   z = (Sz (x) Sy (x) Sx) diag(1 / (lz + ly + lx)) (Sz (x) Sy (x) Sx)^T r.
// This kernel applies the two x-y factors as dense contractions on the
// tensor cores and the z factor on the FP32 pipe:
//   MMA 1:  D1[(j',l')][(i,k)] = sum_(j,l) Sy[j][j'] Sx[l][l'] r_i[k][j][l]
//   z-step: thread (j',l') holds D1[(j',l')][(i, 0..MP-1)], the whole z line
//           of patch i, applies Sz^T, the eigenvalue scaling and Sz in
//           registers, and writes the line back as the next B operand
//   MMA 2:  D2[(j,l)][(i,k)] = sum_(j',l') Sy[j][j'] Sx[l][l'] w_i[k][j'][l']
// A operand = the 2-D Kronecker factor (M = 128 TMEM lanes >= MP^2 modes or
// nodes, K = MP^2 padded to a multiple of 8), B operand = MP rows per patch
// (a stride of 12 rows per patch, N <= 256), both TF32 in shared memory, K-major, and
// D in tensor memory (FP32). The Kronecker factors depend on the x and y
// position classes of the element (boundary, next to the boundary, interior),
// so a work item holds patches of one class pair; its factors arrive by bulk
// copy. The residual entries arrive, at degree 7 (element rows of 32 bytes),
// by 16-byte asynchronous copies of whole element rows into a permuted K
// order (swtc_fill_k), the x-halos shared between the x-neighbouring patches
// of an item; at degrees 6 and 8 by coalesced 4-byte loads rounded to TF32 on
// their way into shared memory; zero outside the domain. The output goes to
// the same patch buffer as the SIMT kernel's, [source][element][MP^3]
// (x fastest), for k_schwarz_gather.
#include <algorithm>
#include <cstring>

#include "dg_internal.h"
#include "dg_swtc.h"
#include "dg_tc.h"

namespace dg {

namespace {

// byte offset of element (row, k) in the padded K-major operand layout
inline size_t opnd_off(int row, int k, int sbo) {
  return (size_t)(row / 8) * sbo + (size_t)(k / 4) * SWTC_LBO + (size_t)(row % 8) * 16 + (size_t)(k % 4) * 4;
}

// round to TF32, nearest with ties away from zero (as cvt.rna.tf32.f32)
inline float host_tf32(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

}  // namespace

// K slot of patch node (j, l) in the residual operand of the n1 = 8 kernel,
// for an x position class with left overlap oLx and mx patch nodes: own
// x-node a = l - oLx of row j at 8 j + a (two 16-byte groups per row, filled
// by 16-byte copies of the element row), the left / right x-halo node of row
// j at 8 MP + 2 j + 0 / 1; -1 for a node outside the patch
int swtc_fill_k(int j, int l, int oLx, int mx) {
  constexpr int N1 = 8, MP = N1 + 2;
  const int a = l - oLx;
  if (a >= 0 && a < N1) return N1 * j + a;
  if (l == 0 && oLx == 1) return N1 * MP + 2 * j;
  if (l == oLx + N1 && l < mx) return N1 * MP + 2 * j + 1;
  return -1;
}

bool swtc_geometry(int n1, SwTcGeom& g, int np) {
  g.mp = n1 + 2;
  const int mp2 = g.mp * g.mp;
  if (n1 < 7 || n1 > 9) return false;
  g.kpad = (mp2 + 7) / 8 * 8;
  g.kc = g.kpad / 4;
  g.sbo = g.kc * SWTC_LBO;
  g.a_bytes = ((mp2 + 7) / 8) * g.sbo;
  // patches per item: MP rows of the B operand each, at a stride of cs rows
  // (D columns), so that every tensor-memory load starts at a multiple of 4
  // (degree 7: 16, one z-factor MMA operand per patch); two stages of B must
  // fit next to the two factors (and, at degree 7, the z-factor operands)
  const bool ztc = n1 == 8 && DG_SWTC_ZTC;
  g.cs = ztc ? SWTC8_CS : SWTC_CS;
  const int np_max = ztc ? SWTC8_NPMAX : g.mp == 11 ? 4 : 10;
  if (np < 0 || np > np_max) return false;
  g.np = np > 0 ? np : np_max;
  g.ncol = (g.np * g.cs + 15) / 16 * 16;
  g.b_bytes = (g.ncol / 8) * g.sbo;
  g.zb_bytes = ztc ? SWTC_MAXZCLS * 2 * SWTC_ZB_BYTES : 0;
  // the static shared memory counts in whole kilobytes (the dynamic part is
  // 1024-byte aligned after it)
  const size_t stat = (sizeof(SwTcShared) + 1023) / 1024 * 1024;
  // tensor memory: three accumulators, or at degree 7 two items of two
  // 128-column accumulators each
  const bool tmem_ok = ztc ? g.ncol <= 128 : SWTC_DSLOTS * g.ncol <= SWTC_TMEM_COLS;
  return 2 * (size_t)g.a_bytes + SWTC_BSLOTS * (size_t)g.b_bytes + g.zb_bytes + stat <= 232448 &&
         g.np <= SWTC_NPMAX && tmem_ok;
}

// Host tables of the tensor-core patch solve of one level (layout in
// dg_swtc.h), from the level's Schwarz tables (schwarz_tables). Returns an
// empty vector when the level does not qualify (degree outside 6..8, more
// position classes than supported).
std::vector<unsigned char> schwarz_tc_blob(const LevelOp& L, const std::vector<double>& tabs, int* err_dev) {
  SwTcGeom g;
  if (!swtc_geometry(L.n1, g)) return {};
  const int MP = g.mp, STR = schwarz_axis_stride(L.n1);
  // position classes per axis: positions whose tables are identical share a class
  int cls[3][4096];
  std::vector<int> rep[3];  // representative position of each class
  size_t off = 0;
  for (int d = 0; d < 3; ++d) {
    if (L.n[d] > 4096) return {};
    for (int e = 0; e < L.n[d]; ++e) {
      const double* t = tabs.data() + off + (size_t)e * STR;
      int c = -1;
      for (size_t k = 0; k < rep[d].size(); ++k)
        if (std::memcmp(tabs.data() + off + (size_t)rep[d][k] * STR, t, sizeof(double) * STR) == 0) {
          c = (int)k;
          break;
        }
      if (c < 0) {
        c = (int)rep[d].size();
        rep[d].push_back(e);
      }
      cls[d][e] = c;
    }
    if ((int)rep[d].size() > (d == 2 ? SWTC_MAXZCLS : SWTC_MAXCLS)) return {};
    off += (size_t)L.n[d] * STR;
  }
  if (L.n[0] * L.n[1] > SWTC_MAXCOLS || L.n[2] > SWTC_MAXNZ) return {};
  auto tab = [&](int d, int pos) {
    size_t o = 0;
    for (int dd = 0; dd < d; ++dd) o += (size_t)L.n[dd] * STR;
    return tabs.data() + o + (size_t)pos * STR;
  };
  SwTcHead H;
  std::memset(&H, 0, sizeof(H));
  H.geom = g;
  H.n1 = L.n1;
  H.nx = L.n[0];
  H.ny = L.n[1];
  H.nz = L.n[2];
  H.err = err_dev;
  const int ncx = (int)rep[0].size(), ncy = (int)rep[1].size(), ncz = (int)rep[2].size();
  H.ncx = ncx;
  H.ncy = ncy;
  H.ncz = ncz;
  // segments: class pairs (cx, cy) with their element columns (ex, ey)
  std::vector<int> cols;
  H.nseg = 0;
  for (int cy = 0; cy < ncy; ++cy)
    for (int cx = 0; cx < ncx; ++cx) {
      const int s = H.nseg++;
      H.seg_cx[s] = cx;
      H.seg_cy[s] = cy;
      H.seg_col0[s] = (int)cols.size() / 2;
      for (int ey = 0; ey < L.n[1]; ++ey)
        for (int ex = 0; ex < L.n[0]; ++ex)
          if (cls[0][ex] == cx && cls[1][ey] == cy) {
            cols.push_back(ex);
            cols.push_back(ey);
          }
      H.seg_ncol[s] = (int)cols.size() / 2 - H.seg_col0[s];
    }
  // byte layout
  auto align = [](size_t x) { return (x + 127) / 128 * 128; };
  size_t pos = align(sizeof(SwTcHead));
  H.off_cols = pos;
  pos = align(pos + sizeof(int) * cols.size());
  H.off_zcls = pos;
  pos = align(pos + sizeof(int) * L.n[2]);
  H.off_z = pos;  // per z class: S [MP][MP], lambda [MP], m (as float)
  pos = align(pos + sizeof(float) * (size_t)ncz * SWTC_ZSTR(MP));
  H.off_xy = pos;  // per x class, then per y class: lambda [MP], m (as float)
  pos = align(pos + sizeof(float) * (size_t)(ncx + ncy) * (MP + 1));
  H.off_y = ncx * (MP + 1);
  H.off_zb = pos;  // degree 7: per z class Sz^T and Sz as MMA operands
  pos = align(pos + (L.n1 == 8 && DG_SWTC_ZTC ? (size_t)ncz * 2 * SWTC_ZB_BYTES : 0));
  H.off_a = pos;
  pos += (size_t)H.nseg * 2 * g.a_bytes;
  std::vector<unsigned char> blob(pos, 0);
  std::memcpy(blob.data() + H.off_cols, cols.data(), sizeof(int) * cols.size());
  std::memcpy(blob.data() + H.off_zcls, cls[2], sizeof(int) * L.n[2]);
  float* zt = (float*)(blob.data() + H.off_z);
  const int MPP = SWTC_MPP(MP);
  for (int c = 0; c < ncz; ++c) {
    const double* t = tab(2, rep[2][c]);
    float* o = zt + (size_t)c * SWTC_ZSTR(MP);
    for (int a = 0; a < MP; ++a)
      for (int k = 0; k < MP; ++k) o[a * MPP + k] = (float)t[2 + a * MP + k];
    for (int k = 0; k < MP; ++k) o[MP * MPP + k] = (float)t[2 + MP * MP + k];
    o[MP * MPP + MPP] = (float)t[0];
  }
  if (L.n1 == 8 && DG_SWTC_ZTC) {
    // z-factor MMA operands per z class: Sz^T [n = mode][k = node] (forward)
    // and Sz [n = node][k = mode] (inverse), 16 x 16, zero outside the patch
    auto zoff = [](int n, int k) {
      return (size_t)(n / 8) * SWTC_ZB_SBO + (size_t)(k / 4) * SWTC_ZB_LBO + (size_t)(n % 8) * 16 + (size_t)(k % 4) * 4;
    };
    for (int c = 0; c < ncz; ++c) {
      const double* t = tab(2, rep[2][c]);
      unsigned char* fw = blob.data() + H.off_zb + (size_t)c * 2 * SWTC_ZB_BYTES;
      unsigned char* iv = fw + SWTC_ZB_BYTES;
      for (int node = 0; node < MP; ++node)
        for (int mode = 0; mode < MP; ++mode) {
          const float v = host_tf32((float)t[2 + node * MP + mode]);
          std::memcpy(fw + zoff(mode, node), &v, 4);
          std::memcpy(iv + zoff(node, mode), &v, 4);
        }
    }
  }
  float* xy = (float*)(blob.data() + H.off_xy);
  for (int d = 0; d < 2; ++d)
    for (int c = 0; c < (int)rep[d].size(); ++c) {
      const double* t = tab(d, rep[d][c]);
      float* o = xy + (d == 0 ? 0 : H.off_y) + (size_t)c * (MP + 1);
      for (int k = 0; k < MP; ++k) o[k] = (float)t[2 + MP * MP + k];
      o[MP] = (float)t[0];
    }
  // Kronecker factors per segment: forward (rows = modes (j',l'), K = nodes
  // (j,l)) and inverse (rows = nodes, K = modes), value Sy[j][j'] Sx[l][l'].
  // At n1 = 8 the forward factor's K order is the one the residual fill
  // writes (swtc_fill_k): each patch row's own x-nodes as two aligned 16-byte
  // groups, the x-halo nodes after all rows.
  for (int s = 0; s < H.nseg; ++s) {
    const double* tx = tab(0, rep[0][H.seg_cx[s]]);
    const double* ty = tab(1, rep[1][H.seg_cy[s]]);
    const int oLx = (int)tx[1], mx = (int)tx[0];
    unsigned char* af = blob.data() + H.off_a + (size_t)s * 2 * g.a_bytes;
    unsigned char* ai = af + g.a_bytes;
    for (int j = 0; j < MP; ++j)
      for (int l = 0; l < MP; ++l) {
        const int kf = L.n1 == 8 ? swtc_fill_k(j, l, oLx, mx) : j * MP + l;
        for (int jp = 0; jp < MP; ++jp)
          for (int lp = 0; lp < MP; ++lp) {
            const float v = host_tf32((float)(ty[2 + j * MP + jp] * tx[2 + l * MP + lp]));
            const int node = j * MP + l, mode = jp * MP + lp;
            if (kf >= 0) std::memcpy(af + opnd_off(mode, kf, g.sbo), &v, 4);
            std::memcpy(ai + opnd_off(node, mode, g.sbo), &v, 4);
          }
      }
  }
  std::memcpy(blob.data(), &H, sizeof(H));
  return blob;
}

// ---------------------------------------------------------------------------
// kernel: a pipeline over work items, each CTA taking a share of every class
// pair (or, with DG_SWTC_SPLIT = 0, a contiguous range of the item list).
// Warp roles: producers decode an item and fill its B operand (2 slots),
// the MMA thread issues MMA 1 as soon as a B is full and MMA 2 as soon as the
// consumers have rewritten it, consumers run the z-step of item i and then
// read out item i - 1 (accumulators in 3 TMEM slots, item descriptions in 4).
// Every hand-off is an mbarrier; every wait is bounded.
// ---------------------------------------------------------------------------
template <int N1>
__global__ void __launch_bounds__(swtc_threads(N1), 1)
    k_schwarz_patch_tc(const LevelOp* __restrict__ op, const unsigned char* __restrict__ blob, const SwTcGeom geom,
                       const float* __restrict__ r, float* __restrict__ zp, const int* __restrict__ act, int nact) {
  constexpr int MP = N1 + 2, MP2 = MP * MP, MP3 = MP2 * MP, NPE = N1 * N1 * N1, MPP = SWTC_MPP(MP);
  constexpr int CONS = SWTC_CONSUMERS, PROD = swtc_producers(N1), THREADS = swtc_threads(N1);
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ SwTcShared sh;
  const SwTcHead* H = (const SwTcHead*)blob;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int a_bytes = geom.a_bytes, b_bytes = geom.b_bytes, sbo = geom.sbo, NP = geom.np;
  const int kc = geom.kc, ncol = geom.ncol, nseg = H->nseg;
  const long long off_a = H->off_a;
  unsigned char* sAf = dsm;
  unsigned char* sAi = dsm + a_bytes;
  unsigned char* sB0 = dsm + 2 * a_bytes;
  const int nx = H->nx, ny = H->ny, nz = H->nz;
  const int E = nx * ny * nz;
  const long long Nq = (long long)E * NPE;
  // ---- set-up: barriers, tensor memory, staged tables, item offsets, zeroed B
  if (tid == 0) {
    for (int b = 0; b < SWTC_BSLOTS; ++b) {
      tc::mbar_init(tc::smem_addr(&sh.full[b]), PROD);
      tc::mbar_init(tc::smem_addr(&sh.b2[b]), CONS);
    }
    for (int d = 0; d < SWTC_DSLOTS; ++d) {
      tc::mbar_init(tc::smem_addr(&sh.d1[d]), 1);
      tc::mbar_init(tc::smem_addr(&sh.d2[d]), 1);
      tc::mbar_init(tc::smem_addr(&sh.empty[d]), CONS);
    }
    tc::mbar_init(tc::smem_addr(&sh.tma_f), 1);
    tc::mbar_init(tc::smem_addr(&sh.tma_i), 1);
    tc::mbar_init_fence();
    sh.abort = 0;
    int acc = 0;
    for (int sg = 0; sg < nseg; ++sg) {
      sh.item0[sg] = acc;
      acc += (int)(((long long)H->seg_ncol[sg] * nz * nact + NP - 1) / NP);
    }
    sh.item0[nseg] = acc;
    if (DG_SWTC_SPLIT) {
      // Every CTA takes the same share of every segment (class pair), so that
      // all CTAs get the same mix of interior items and the costlier items of
      // the boundary classes; its position in the split rotates from segment
      // to segment, so that the CTAs that take one item more of a small
      // segment differ. A CTA's share of a segment is a contiguous run.
      int mine = 0;
      const long long G = gridDim.x;
      for (int sg = 0; sg < nseg; ++sg) {
        const long long n = sh.item0[sg + 1] - sh.item0[sg];
        const long long c = (blockIdx.x + 37LL * sg) % G;
        const int lo = (int)(c * n / G), hi = (int)((c + 1) * n / G);
        sh.mine0[sg] = sh.item0[sg] + lo;
        sh.mcum[sg] = mine;
        mine += hi - lo;
      }
      sh.mcum[nseg] = mine;
    }
  }
  if (warp == 0) tc::tmem_alloc(&sh.tmem, SWTC_TMEM_COLS);
  {
    const float* zt = (const float*)(blob + H->off_z);
    for (int i = tid; i < H->ncz * SWTC_ZSTR(MP); i += THREADS) sh.z[i] = zt[i];
    for (int i = tid; i < nseg; i += THREADS) {
      sh.seg_col0[i] = H->seg_col0[i];
      sh.seg_ncol[i] = H->seg_ncol[i];
      sh.seg_cx[i] = (unsigned char)H->seg_cx[i];
      sh.seg_cy[i] = (unsigned char)H->seg_cy[i];
    }
    const int* cols = (const int*)(blob + H->off_cols);
    for (int i = tid; i < nx * ny; i += THREADS) sh.cols[i] = make_short2((short)cols[2 * i], (short)cols[2 * i + 1]);
    const int* zc = (const int*)(blob + H->off_zcls);
    for (int i = tid; i < nz; i += THREADS) sh.zcls[i] = (unsigned char)zc[i];
    for (int i = tid; i < nact && i < SWTC_MAXACT; i += THREADS) sh.act[i] = (unsigned short)act[i];
    const float* xy = (const float*)(blob + H->off_xy);
    for (int i = tid; i < 2 * SWTC_MAXCLS * (MP + 1); i += THREADS) {
      const int d = i / (SWTC_MAXCLS * (MP + 1)), rem = i % (SWTC_MAXCLS * (MP + 1));
      const int c = rem / (MP + 1), k = rem % (MP + 1);
      if (c < (d == 0 ? H->ncx : H->ncy)) sh.lxy[d][c][k] = xy[(d == 0 ? 0 : H->off_y) + (size_t)c * (MP + 1) + k];
    }
    uint4* b4 = (uint4*)sB0;
    for (int i = tid; i < SWTC_BSLOTS * b_bytes / 16; i += THREADS) b4[i] = make_uint4(0, 0, 0, 0);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sh.tmem;
  // without DG_SWTC_SPLIT each CTA takes a contiguous range of items, so that
  // it rarely crosses into another class pair (a new pair costs a reload of
  // both factors)
  const int total = sh.item0[nseg];
  const int per_cta = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  const int first = (int)blockIdx.x * per_cta;
  const int nmine = DG_SWTC_SPLIT ? sh.mcum[nseg] : max(0, min(per_cta, total - first));

  if (tid >= CONS && tid < CONS + PROD) {
    // ================= producers: decode and fill =================
    const int L = tid - CONS;  // B column (j, l) this thread fills (n1 != 8)
    const int jj = L / MP, ll = L % MP;
    // row fill (n1 = 8): slots (zk, jj, half) L, L + PROD, ... of the 2 MP^2
    // per patch, with the y offset of row jj relative to the patch's element for
    // a patch without (0) and with (1) left overlap along y
    constexpr int NSL = (2 * MP2 + PROD - 1) / PROD;
    int f_zk[NSL], f_j[NSL], f_h[NSL], f_own[NSL], f_halo[NSL];
    long long f_yoff[NSL][2];
    bool f_ok[NSL];
#pragma unroll
    for (int u = 0; u < NSL; ++u) {
      if constexpr (N1 != 8) break;
      const int sl = L + PROD * u;
      f_ok[u] = sl < 2 * MP2;
      f_zk[u] = sl / (2 * MP);
      f_j[u] = (sl % (2 * MP)) >> 1;
      f_h[u] = sl & 1;
      const int j = f_j[u], kh = N1 * MP + 2 * j + f_h[u];
      f_own[u] = (2 * j + f_h[u]) * SWTC_LBO;
      f_halo[u] = (kh >> 2) * SWTC_LBO + (kh & 3) * 4;
      f_yoff[u][0] = (long long)(j / N1) * nx * NPE + (j % N1) * N1;
      f_yoff[u][1] = j == 0 ? -(long long)nx * NPE + (N1 - 1) * N1
                            : (long long)((j - 1) / N1) * nx * NPE + ((j - 1) % N1) * N1;
    }
    int seg = 0;  // segment of the current item (items ascend)
    for (int li = 0; li < nmine; ++li) {
      const int b = li % SWTC_BSLOTS;
      // The item is decoded as soon as its description slot is free (item
      // li - 4 read out), before the wait for its B slot (MMA 2 of item li - 2
      // done), which is the longer one: the decode stays off the B slots'
      // critical path. All producers leave together (they share a named barrier).
      bool ok = li < SWTC_ISLOTS || swtc_wait(sh, H, &sh.empty[(li - SWTC_ISLOTS) % SWTC_DSLOTS],
                                              ((li - SWTC_ISLOTS) / SWTC_DSLOTS) & 1);
      if (tc::named_barrier_or(1, PROD, !ok || sh.abort != 0)) break;
      SwTcItem& I = sh.item[li % SWTC_ISLOTS];
      int it;  // item index in the launch's item list
      if (DG_SWTC_SPLIT) {
        while (sh.mcum[seg + 1] <= li) ++seg;
        it = sh.mine0[seg] + li - sh.mcum[seg];
      } else {
        it = first + li;
        while (sh.item0[seg + 1] <= it) ++seg;
      }
      // patch q of a segment: column fastest, then z, then source: each CTA
      // sweeps a slab of one source's elements, so the residual rows it
      // gathers as halos were loaded shortly before (by itself or by the CTAs
      // on the neighbouring slabs) and are still in L2 (counts stay below
      // 2^31: columns x sources x z positions)
      const int q0 = (it - sh.item0[seg]) * NP;
      const int ncs = sh.seg_ncol[seg];
      const int np = min(NP, ncs * nz * nact - q0);
      if (L < np) {
        const int q = q0 + L;
        const int colrel = q % ncs, zq = q / ncs;
        const int ez = zq % nz, a = zq / nz;
        const short2 c = sh.cols[sh.seg_col0[seg] + colrel];
        I.src[L] = a < SWTC_MAXACT ? (int)sh.act[a] : act[a];
        I.ex[L] = c.x;
        I.ey[L] = c.y;
        I.ez[L] = (short)ez;
        I.cz[L] = (short)sh.zcls[ez];
        I.elem[L] = c.x + nx * (c.y + ny * ez);
        if constexpr (N1 == 8) {
          // x-halos shared with the neighbouring patch of the item: the same
          // source, y and z position and the adjacent x position (patch q - 1
          // or q + 1 of the same column run)
          const short2* cs = sh.cols + sh.seg_col0[seg];
          const bool lsh = L > 0 && colrel > 0 && cs[colrel - 1].x == c.x - 1 && cs[colrel - 1].y == c.y;
          const bool rsh = L + 1 < np && colrel + 1 < ncs && cs[colrel + 1].x == c.x + 1 && cs[colrel + 1].y == c.y;
          const int oLy = c.y > 0, my = N1 + oLy + (c.y < ny - 1);
          I.rbase[L] = (long long)I.src[L] * Nq + (long long)(c.x + nx * c.y) * NPE;
          I.pf[L] = (unsigned short)(oLy | (my << 1) | (lsh << 6) | (rsh << 7) | ((c.x > 0) << 8) |
                                     ((c.x < nx - 1) << 9));
        }
      }
      // z offsets of every (patch, z-node): the same for all (x, y) of the patch
      for (int e = L; e < np * MP; e += PROD) {
        const int i = e / MP, k = e - (e / MP) * MP;
        const int ez = ((q0 + i) / ncs) % nz;
        const int oLz = ez > 0, mz = N1 + oLz + (ez < nz - 1);
        const int Z = ez * N1 - oLz + k;
        const int EZ = Z / N1;
        I.zoff[i][k] = k < mz ? EZ * nx * ny * NPE + N1 * N1 * (Z - EZ * N1) : -1;
      }
      if (L == 0) {
        I.np = np;
        I.seg = seg;
      }
      ok = li < SWTC_BSLOTS ||
           swtc_wait(sh, H, &sh.d2[(li - SWTC_BSLOTS) % SWTC_DSLOTS], ((li - SWTC_BSLOTS) / SWTC_DSLOTS) & 1);
      if (tc::named_barrier_or(1, PROD, !ok || sh.abort != 0)) break;
      unsigned char* sB = sB0 + b * b_bytes;
      if constexpr (N1 == 8) {
        // Residual rows by 16-byte copies: row (zk, jj) of patch i holds its
        // 8 own x-nodes (one element row, 32 bytes) at K slots 8 jj .. 8 jj + 7
        // and its x-halo nodes at 8 MP + 2 jj + side (swtc_fill_k). This
        // thread's slots (zk, jj, half) are fixed: per patch it copies one
        // half row and the x-halo node on side `half`, unless that node is an
        // own node of the item's neighbouring patch (copied in shared memory
        // below). Outside the domain the copies fill zeros. The values land
        // as FP32 and the tensor core takes their TF32 part.
#pragma unroll
        for (int i = 0; i < SWTC_NPMAX; ++i) {
          if (i < np) {
            const long long rb = I.rbase[i];
            const int pf = I.pf[i];
            const int oLy = pf & 1, my = (pf >> 1) & 15;
#pragma unroll
            for (int u = 0; u < NSL; ++u) {
              if (f_ok[u]) {
                const int zo = I.zoff[i][f_zk[u]];
                const bool valid = f_j[u] < my && zo >= 0;
                const long long o = rb + (oLy ? f_yoff[u][1] : f_yoff[u][0]) + zo;
                const int row = i * SWTC_CS + f_zk[u];
                unsigned char* rowp = sB + (row >> 3) * sbo + (row & 7) * 16;
                tc::cp_async16(rowp + f_own[u], valid ? r + o + 4 * f_h[u] : r, valid ? 16 : 0);
                if (!((pf >> (6 + f_h[u])) & 1)) {
                  const bool ok_x = valid && ((pf >> (8 + f_h[u])) & 1);
                  tc::cp_async4(rowp + f_halo[u], ok_x ? r + o + (f_h[u] ? NPE : N1 - 1 - NPE) : r, ok_x ? 4 : 0);
                }
              }
            }
          }
        }
        tc::cp_async_wait_all();
        tc::named_barrier(1, PROD);
#pragma unroll
        for (int i = 0; i < SWTC_NPMAX; ++i) {
          if (i < np) {
            const int pf = I.pf[i];
#pragma unroll
            for (int u = 0; u < NSL; ++u) {
              if (f_ok[u] && ((pf >> (6 + f_h[u])) & 1)) {
                const int row = i * SWTC_CS + f_zk[u];
                const int rs = row + (f_h[u] ? SWTC_CS : -SWTC_CS);
                const int ks = N1 * f_j[u] + (f_h[u] ? 0 : N1 - 1);
                const float v =
                    *(const float*)(sB + (rs >> 3) * sbo + (ks >> 2) * SWTC_LBO + (rs & 7) * 16 + (ks & 3) * 4);
                *(float*)(sB + (row >> 3) * sbo + (row & 7) * 16 + f_halo[u]) = v;
              }
            }
          }
        }
      } else if (L < MP2) {
        // this thread's column of B: byte offset of row 0 in its 4-column group.
        // Every value of the item is loaded first (all in flight at once), then
        // rounded to TF32 and stored: coalesced loads, not one-element copies
        unsigned char* col = sB + (L / 4) * SWTC_LBO + (L % 4) * 4;
        float v[SWTC_NPMAX][MP];
#pragma unroll
        for (int i = 0; i < SWTC_NPMAX; ++i) {
          if (i < np) {
            const int ex = I.ex[i], ey = I.ey[i];
            const int oLx = ex > 0, oLy = ey > 0;
            const int mx = N1 + oLx + (ex < nx - 1), my = N1 + oLy + (ey < ny - 1);
            const int X = ex * N1 - oLx + ll, Y = ey * N1 - oLy + jj;
            const bool vx = ll < mx && jj < my;
            const int EX = vx ? X / N1 : 0, EY = vx ? Y / N1 : 0;
            const float* pxy =
                r + (long long)I.src[i] * Nq + (EX + nx * EY) * NPE + (X - EX * N1) + N1 * (Y - EY * N1);
#pragma unroll
            for (int k = 0; k < MP; ++k) {
              const int zo = I.zoff[i][k];
              v[i][k] = (vx && zo >= 0) ? __ldg(pxy + zo) : 0.0f;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < SWTC_NPMAX; ++i) {
          if (i < np) {
#pragma unroll
            for (int k = 0; k < MP; ++k) {
              const int row = i * SWTC_CS + k;
              *(float*)(col + (row >> 3) * sbo + (row & 7) * 16) = tc::to_tf32(v[i][k]);
            }
          }
        }
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(tc::smem_addr(&sh.full[b]));
    }
  } else if (tid >= CONS + PROD) {
    // ================= MMA issuer (one thread) =================
    if (tid == CONS + PROD) {
      const uint32_t idesc = tc::idesc_tf32(128, ncol);
      int seg_f = -1, seg_i = -1;
      uint32_t ph_f = 0, ph_i = 0;
      // MMA 2 of item k: after the consumers rewrote its B
      auto mma2 = [&](int k) -> bool {
        const int b = k % SWTC_BSLOTS, d = k % SWTC_DSLOTS;
        if (!swtc_wait(sh, H, &sh.b2[b], (k / SWTC_BSLOTS) & 1)) return false;
        const int seg = sh.item[k % SWTC_ISLOTS].seg;
        if (seg != seg_i) {
          // the inverse factor is read by MMA 2 of item k - 1: let it finish first
          if (k >= 1 && !swtc_wait(sh, H, &sh.d2[(k - 1) % SWTC_DSLOTS], ((k - 1) / SWTC_DSLOTS) & 1)) return false;
          tc::mbar_expect_tx(tc::smem_addr(&sh.tma_i), (uint32_t)a_bytes);
          tc::bulk_g2s(sAi, blob + off_a + ((size_t)seg * 2 + 1) * a_bytes, (uint32_t)a_bytes,
                       tc::smem_addr(&sh.tma_i));
          if (!swtc_wait(sh, H, &sh.tma_i, ph_i)) return false;
          ph_i ^= 1;
          seg_i = seg;
        }
        tc::fence_after_sync();
        const uint32_t sb = tc::smem_addr(sB0 + b * b_bytes);
        for (int s = 0; s < kc / 2; ++s)
          tc::mma_tf32(tmem + d * ncol, tc::desc_kmajor(tc::smem_addr(sAi) + s * 2 * SWTC_LBO, SWTC_LBO, sbo),
                       tc::desc_kmajor(sb + s * 2 * SWTC_LBO, SWTC_LBO, sbo), idesc, s > 0);
        tc::mma_commit(tc::smem_addr(&sh.d2[d]));
        return true;
      };
      for (int li = 0; li < nmine; ++li) {
        const int b = li % SWTC_BSLOTS, d = li % SWTC_DSLOTS;
        if (!swtc_wait(sh, H, &sh.full[b], (li / SWTC_BSLOTS) & 1)) break;
        // accumulator slot free once item li - 3 is read out
        if (li >= SWTC_DSLOTS &&
            !swtc_wait(sh, H, &sh.empty[(li - SWTC_DSLOTS) % SWTC_DSLOTS], ((li - SWTC_DSLOTS) / SWTC_DSLOTS) & 1))
          break;
        const int seg = sh.item[li % SWTC_ISLOTS].seg;
        if (seg != seg_f) {
          if (li >= 1 && !swtc_wait(sh, H, &sh.d1[(li - 1) % SWTC_DSLOTS], ((li - 1) / SWTC_DSLOTS) & 1)) break;
          tc::mbar_expect_tx(tc::smem_addr(&sh.tma_f), (uint32_t)a_bytes);
          tc::bulk_g2s(sAf, blob + off_a + (size_t)seg * 2 * a_bytes, (uint32_t)a_bytes, tc::smem_addr(&sh.tma_f));
          if (!swtc_wait(sh, H, &sh.tma_f, ph_f)) break;
          ph_f ^= 1;
          seg_f = seg;
        }
        tc::fence_after_sync();
        const uint32_t sb = tc::smem_addr(sB0 + b * b_bytes);
        for (int s = 0; s < kc / 2; ++s)
          tc::mma_tf32(tmem + d * ncol, tc::desc_kmajor(tc::smem_addr(sAf) + s * 2 * SWTC_LBO, SWTC_LBO, sbo),
                       tc::desc_kmajor(sb + s * 2 * SWTC_LBO, SWTC_LBO, sbo), idesc, s > 0);
        tc::mma_commit(tc::smem_addr(&sh.d1[d]));
        if (li >= 1 && !mma2(li - 1)) break;
      }
      if (nmine >= 1 && !sh.abort) mma2(nmine - 1);
    }
  } else {
    // ================= consumers: z-step of item li, output of item li - 1 =================
    const int L = tid;  // TMEM lane: mode (j', l') for the z-step, node (j, l) for the output
    const int jj = L / MP, ll = L % MP;
    const bool active = L < MP2;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
    float S[MP][MP], inv[MP];
    float lxy = 0.f;
    bool vxy = false;
    int cur_seg = -1, cur_cz = -1;
    // output of item k: patch node (l, j, k') of each patch
    auto output = [&](int k) -> bool {
      const int d = k % SWTC_DSLOTS;
      const bool ok = swtc_wait(sh, H, &sh.d2[d], (k / SWTC_DSLOTS) & 1);
      if (__any_sync(0xffffffffu, !ok || sh.abort != 0)) return false;
      tc::fence_after_sync();
      const SwTcItem& I = sh.item[k % SWTC_ISLOTS];
      const uint32_t tcol = tlane + d * ncol;
      const int np = I.np;
      uint32_t nx12[SWTC_CS];  // the next patch's columns, in flight
      tc::tmem_ld12_async(tcol, nx12);
      for (int i = 0; i < np; ++i) {
        tc::tmem_wait12(nx12);
        float v[SWTC_CS];
#pragma unroll
        for (int c = 0; c < SWTC_CS; ++c) v[c] = __uint_as_float(nx12[c]);
        if (i + 1 < np) tc::tmem_ld12_async(tcol + (i + 1) * SWTC_CS, nx12);
        if (active) {
          // streaming stores: the patch solutions are read once, by the gather,
          // long after; evict-first keeps L2 for the residual rows that
          // neighbouring patches still gather
          float* out = zp + ((long long)I.src[i] * E + I.elem[i]) * MP3 + L;
#pragma unroll
          for (int c = 0; c < MP; ++c) __stcs(out + c * MP2, v[c]);
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(tc::smem_addr(&sh.empty[d]));
      return true;
    };
    int li = 0;
    for (; li < nmine; ++li) {
      const int b = li % SWTC_BSLOTS, d = li % SWTC_DSLOTS;
      // full[b] (the producers' item description) then d1[d] (MMA 1 done); full[b]
      // cannot move on before this thread's z-step of the item (b2[b] -> MMA 2)
      const bool ok = swtc_wait(sh, H, &sh.full[b], (li / SWTC_BSLOTS) & 1) &&
                      swtc_wait(sh, H, &sh.d1[d], (li / SWTC_DSLOTS) & 1);
      // tensor-memory loads are warp-collective: a warp leaves as a whole
      if (__any_sync(0xffffffffu, !ok || sh.abort != 0)) break;
      tc::fence_after_sync();
      const SwTcItem& I = sh.item[li % SWTC_ISLOTS];
      const int np = I.np;
      if (I.seg != cur_seg) {
        cur_seg = I.seg;
        const float* tx = sh.lxy[0][sh.seg_cx[cur_seg]];
        const float* ty = sh.lxy[1][sh.seg_cy[cur_seg]];
        lxy = active ? tx[ll] + ty[jj] : 0.f;
        vxy = active && ll < (int)tx[MP] && jj < (int)ty[MP];
        cur_cz = -1;
      }
      unsigned char* sB = sB0 + b * b_bytes;
      const uint32_t tcol = tlane + d * ncol;
      // z-step: Sz^T, scaling, Sz along each patch's z line, back into B as TF32
      uint32_t nx12[SWTC_CS];  // the next patch's columns, in flight
      tc::tmem_ld12_async(tcol, nx12);
      for (int i = 0; i < np; ++i) {
        tc::tmem_wait12(nx12);
        float t[SWTC_CS];
#pragma unroll
        for (int c = 0; c < SWTC_CS; ++c) t[c] = __uint_as_float(nx12[c]);
        if (i + 1 < np) tc::tmem_ld12_async(tcol + (i + 1) * SWTC_CS, nx12);
        const int cz = I.cz[i];
        if (cz != cur_cz) {
          cur_cz = cz;
          const float* zt = sh.z + cz * SWTC_ZSTR(MP);
          const int mzc = (int)zt[MP * MPP + MPP];
#pragma unroll
          for (int a = 0; a < MP; ++a)
#pragma unroll
            for (int c = 0; c < MP; ++c) S[a][c] = zt[a * MPP + c];
#pragma unroll
          for (int c = 0; c < MP; ++c) inv[c] = (vxy && c < mzc) ? 1.0f / (lxy + zt[MP * MPP + c]) : 0.0f;
        }
        if (active) {
          // both contractions as MP independent accumulators updated per step
          float u[MP], w[MP];
#pragma unroll
          for (int c = 0; c < MP; ++c) u[c] = S[0][c] * t[0];
#pragma unroll
          for (int a = 1; a < MP; ++a)
#pragma unroll
            for (int c = 0; c < MP; ++c) u[c] = fmaf(S[a][c], t[a], u[c]);
#pragma unroll
          for (int c = 0; c < MP; ++c) u[c] *= inv[c];
#pragma unroll
          for (int a = 0; a < MP; ++a) w[a] = S[a][0] * u[0];
#pragma unroll
          for (int c = 1; c < MP; ++c)
#pragma unroll
            for (int a = 0; a < MP; ++a) w[a] = fmaf(S[a][c], u[c], w[a]);
          unsigned char* col = sB + (L / 4) * SWTC_LBO + (L % 4) * 4;
#pragma unroll
          for (int a = 0; a < MP; ++a) {
            const int row = i * SWTC_CS + a;
            *(float*)(col + (row >> 3) * sbo + (row & 7) * 16) = tc::to_tf32(w[a]);
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(tc::smem_addr(&sh.b2[b]));
      if (li >= 1 && !output(li - 1)) break;
    }
    if (li == nmine && nmine >= 1) output(nmine - 1);
  }
  // ---- teardown (every role has left its loop)
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, SWTC_TMEM_COLS);
  }
}

template <int N1>
static cudaError_t launch_tc_n1(const LevelOp* dop, const unsigned char* blob, const SwTcGeom& g, const float* r,
                                float* zp, const int* act, int nact, long long items, cudaStream_t s) {
  const int smem = 2 * g.a_bytes + SWTC_BSLOTS * g.b_bytes;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(items, nsm));
  count_launch();
  k_schwarz_patch_tc<N1><<<grid, swtc_threads(N1), smem, s>>>(dop, blob, g, r, zp, act, nact);
  return cudaGetLastError();
}

// Opt the kernel of this degree into the dynamic shared memory it needs (at
// set-up, before any stream capture).
cudaError_t schwarz_tc_prepare(int n1) {
  SwTcGeom g;
  if (!swtc_geometry(n1, g)) return cudaErrorInvalidValue;
  const int smem = 2 * g.a_bytes + SWTC_BSLOTS * g.b_bytes;
  switch (n1) {
    case 7: return cudaFuncSetAttribute(k_schwarz_patch_tc<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case 8:
      if (DG_SWTC_ZTC) return schwarz_tc8_prepare(g);
      return cudaFuncSetAttribute(k_schwarz_patch_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case 9: return cudaFuncSetAttribute(k_schwarz_patch_tc<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_schwarz_patch_tc(const LevelOp& hop, const LevelOp* dop, const SwTcPlan& plan, const float* r,
                                    float* zp, const int* act, int nact, cudaStream_t s) {
  const SwTcHead& head = plan.head;
  const SwTcGeom& g = plan.geom;
  long long items = 0;
  for (int k = 0; k < head.nseg; ++k) items += ((long long)head.seg_ncol[k] * head.nz * nact + g.np - 1) / g.np;
  const unsigned char* b = (const unsigned char*)plan.blob;
  switch (hop.n1) {
    case 7: return launch_tc_n1<7>(dop, b, g, r, zp, act, nact, items, s);
    case 8:
      if (DG_SWTC_ZTC) return launch_schwarz_patch_tc8(plan, r, zp, act, nact, s);
      return launch_tc_n1<8>(dop, b, g, r, zp, act, nact, items, s);
    case 9: return launch_tc_n1<9>(dop, b, g, r, zp, act, nact, items, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
