// Variant of the tensor-core patch solve of the Schwarz smoother at degree 7
// (n1 = 8, patches of 10^3 nodes; compiled in with DG_SWTC_ZTC = 1, see
// dg_swtc.h for its measured speed), FP32 inner solve: all three factors of each patch's
// fast diagonalisation (Sec. 3.4: the restriction of the Kronecker-sum SIPDG
// operator to a tensor box of nodes is a Kronecker sum)
//   z = (Sz (x) Sy (x) Sx) diag(1 / (lz + ly + lx)) (Sz (x) Sy (x) Sx)^T r
// run on the tensor cores (TF32 operands, FP32 accumulation in tensor memory):
//   MMA 1   D1[(j',l')][(i,k)] = sum_(j,l) Sy[j][j'] Sx[l][l'] r_i[k][j][l]
//   MMA z1  E [(j',l')][(i,c)] = sum_k D1[(j',l')][(i,k)] Sz[k][c]
//           (A = D1 read from tensor memory, 16 columns per patch; B = Sz^T)
//   scale   w = E / (lx[l'] + ly[j'] + lz[c]), rounded to TF32, written by
//           the consumer threads (one per tensor-memory lane) as the next B
//   MMA 2   D2[(j,l)][(i,c)]  = sum_(j',l') Sy[j][j'] Sx[l][l'] w[(j',l')][(i,c)]
//   MMA z2  F [(j,l)][(i,k)]  = sum_c D2[(j,l)][(i,c)] Sz[k][c]   (B = Sz)
// and F goes to the patch buffer [source][element][MP^3] (x fastest) that
// k_schwarz_gather sums. Compared with the kernel of degrees 6 and 8 (which
// runs the z factor on the FP32 pipe of the consumer threads), the consumers
// only scale, round and store.
//
// Roles (8 warps): warps 0-3 consumers, 4-6 producers (item decode and the
// residual fill by 16-byte copies of element rows, the K order of the
// forward factor permuted to match: swtc_fill_k), warp 7's first thread
// issues every MMA. Pipeline: two B operand slots, two tensor-memory pairs
// (D1 / D2 in the first 128 columns, E / F in the second), four item
// descriptions. Every hand-off is an mbarrier, every wait bounded; on a
// timeout the kernel sets the level's error word and returns.
#include <algorithm>

#include "dg_internal.h"
#include "dg_swtc.h"
#include "dg_tc.h"

namespace dg {

namespace {
constexpr int N1 = 8, MP = N1 + 2, MP2 = MP * MP, MP3 = MP2 * MP, NPE = N1 * N1 * N1;
constexpr int CS = SWTC8_CS, CONS = SWTC_CONSUMERS, PROD = swtc_producers(8), THREADS = swtc_threads(8);
constexpr int MPP = SWTC_MPP(MP);
static_assert(THREADS == 256, "degree-7 patch kernel: 8 warps");
}  // namespace

__global__ void __launch_bounds__(THREADS, 1)
    k_schwarz_patch_tc8(const unsigned char* __restrict__ blob, const SwTcGeom geom, const float* __restrict__ r,
                        float* __restrict__ zp, const int* __restrict__ act, int nact) {
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
  unsigned char* sZ = sB0 + SWTC_BSLOTS * b_bytes;  // z-factor operands, 2 KB per z class
  const int nx = H->nx, ny = H->ny, nz = H->nz;
  const int E = nx * ny * nz;
  const long long Nq = (long long)E * NPE;
  // ---- set-up: barriers, tensor memory, staged tables, item offsets, zeroed B
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tc::smem_addr(&sh.full[b]), PROD);  // residual operand filled
      tc::mbar_init(tc::smem_addr(&sh.b2[b]), CONS);    // scaled operand written
      tc::mbar_init(tc::smem_addr(&sh.e[b]), 1);        // MMA 1 + z1 done
      tc::mbar_init(tc::smem_addr(&sh.f[b]), 1);        // MMA 2 + z2 done
      tc::mbar_init(tc::smem_addr(&sh.d1[b]), 1);       // MMA 1 done (issuer only)
      tc::mbar_init(tc::smem_addr(&sh.d2[b]), 1);       // MMA 2 done (issuer only)
      tc::mbar_init(tc::smem_addr(&sh.empty[b]), CONS); // tensor-memory pair read out
    }
    for (int k = 0; k < SWTC_ISLOTS; ++k) tc::mbar_init(tc::smem_addr(&sh.ifree[k]), CONS);
    tc::mbar_init(tc::smem_addr(&sh.tma_f), 1);
    tc::mbar_init(tc::smem_addr(&sh.tma_i), 1);
    tc::mbar_init_fence();
    sh.abort = 0;
    // Every CTA takes the same share of every segment (class pair), so that
    // all CTAs get the same mix of interior items and the costlier items of
    // the boundary classes (fewer x-halos shared, several z classes per item);
    // a CTA's share of a segment is a contiguous run of its items.
    // The CTA's position in the split is rotated from segment to segment, so
    // that the CTAs that take one item more of a small segment differ.
    int mine = 0;
    const long long G = gridDim.x;
    for (int sg = 0; sg < nseg; ++sg) {
      const long long n = ((long long)H->seg_ncol[sg] * nz * nact + NP - 1) / NP;
      const long long c = (blockIdx.x + 37LL * sg) % G;
      const int lo = (int)(c * n / G), hi = (int)((c + 1) * n / G);
      sh.mine0[sg] = lo;
      sh.mcum[sg] = mine;
      mine += hi - lo;
    }
    sh.mcum[nseg] = mine;
  }
  if (warp == 0) tc::tmem_alloc(&sh.tmem, SWTC_TMEM_COLS);
  {
    const float* zt = (const float*)(blob + H->off_z);
    for (int i = tid; i < H->ncz * SWTC_ZSTR(MP); i += THREADS) sh.z[i] = zt[i];
    const uint4* zb = (const uint4*)(blob + H->off_zb);
    for (int i = tid; i < H->ncz * 2 * SWTC_ZB_BYTES / 16; i += THREADS) ((uint4*)sZ)[i] = zb[i];
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
  const int nmine = sh.mcum[nseg];

  if (tid >= CONS && tid < CONS + PROD) {
    // ================= producers: decode and fill =================
    const int L = tid - CONS;
    // This thread's fill slots (zk, jj, half): L, L + PROD, ... of the 2 MP^2
    // per patch; per patch a slot is half an element row (16 bytes) and the
    // x-halo node on side `half` of that row. y offset of row jj relative to
    // the patch's element, for a patch without (0) and with (1) left overlap
    // along y.
    constexpr int NSL = (2 * MP2 + PROD - 1) / PROD;
    int f_zk[NSL], f_j[NSL], f_h[NSL], f_own[NSL], f_halo[NSL];
    long long f_yoff[NSL][2];
    bool f_ok[NSL];
#pragma unroll
    for (int u = 0; u < NSL; ++u) {
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
      const int b = li & 1;
      // description slot free once item li - 4 is read out; decoded before the
      // wait for the B slot, which is the longer one
      bool ok = li < SWTC_ISLOTS ||
                swtc_wait(sh, H, &sh.ifree[li % SWTC_ISLOTS], ((li - SWTC_ISLOTS) / SWTC_ISLOTS) & 1);
      if (tc::named_barrier_or(1, PROD, !ok || sh.abort != 0)) break;
      SwTcItem& I = sh.item[li % SWTC_ISLOTS];
      while (sh.mcum[seg + 1] <= li) ++seg;
      // patch q of a segment: column fastest, then z, then source
      const int q0 = (sh.mine0[seg] + li - sh.mcum[seg]) * NP;
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
        // x-halos shared with the neighbouring patch of the item (the same
        // source, y and z position, the adjacent x position)
        const short2* cs = sh.cols + sh.seg_col0[seg];
        const bool lsh = L > 0 && colrel > 0 && cs[colrel - 1].x == c.x - 1 && cs[colrel - 1].y == c.y;
        const bool rsh = L + 1 < np && colrel + 1 < ncs && cs[colrel + 1].x == c.x + 1 && cs[colrel + 1].y == c.y;
        const int oLy = c.y > 0, my = N1 + oLy + (c.y < ny - 1);
        I.rbase[L] = (long long)I.src[L] * Nq + (long long)(c.x + nx * c.y) * NPE;
        I.pf[L] = (unsigned short)(oLy | (my << 1) | (lsh << 6) | (rsh << 7) | ((c.x > 0) << 8) | ((c.x < nx - 1) << 9));
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
      // B slot free once MMA 2 and z2 of item li - 2 are done
      ok = li < 2 || swtc_wait(sh, H, &sh.f[b], ((li - 2) >> 1) & 1);
      if (tc::named_barrier_or(1, PROD, !ok || sh.abort != 0)) break;
      unsigned char* sB = sB0 + b * b_bytes;
      // Residual rows by 16-byte copies: row (zk, jj) of patch i holds its 8
      // own x-nodes (one element row, 32 bytes) at K slots 8 jj .. 8 jj + 7 and
      // its x-halo nodes at 8 MP + 2 jj + side; outside the domain the copies
      // fill zeros. The values land as FP32 and the tensor core takes their
      // TF32 part.
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i) {
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
              const int row = i * CS + f_zk[u];
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
      // x-halos from the neighbouring patch: its own x-node 7 (left halo) or
      // 0 (right halo) of the same row
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i) {
        if (i < np) {
          const int pf = I.pf[i];
#pragma unroll
          for (int u = 0; u < NSL; ++u) {
            if (f_ok[u] && ((pf >> (6 + f_h[u])) & 1)) {
              const int row = i * CS + f_zk[u];
              const int rs = row + (f_h[u] ? CS : -CS);
              const int ks = N1 * f_j[u] + (f_h[u] ? 0 : N1 - 1);
              const float v = *(const float*)(sB + (rs >> 3) * sbo + (ks >> 2) * SWTC_LBO + (rs & 7) * 16 + (ks & 3) * 4);
              *(float*)(sB + (row >> 3) * sbo + (row & 7) * 16 + f_halo[u]) = v;
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
      const uint32_t idesc_xy = tc::idesc_tf32(128, ncol), idesc_z = tc::idesc_tf32(128, 16);
      const uint32_t zbase = tc::smem_addr(sZ);
      int seg_f = -1, seg_i = -1;
      uint32_t ph_f = 0, ph_i = 0;
      // z-factor MMAs of every patch of item I: dst[:, CS i ..] = src[:, CS i ..] x
      // (the class's Sz^T (which = 0) or Sz (which = 1)), K = N = 16
      auto zmma = [&](const SwTcItem& I, uint32_t src, uint32_t dst, int which) {
        for (int i = 0; i < I.np; ++i) {
          const uint32_t zb = zbase + (uint32_t)(I.cz[i] * 2 + which) * SWTC_ZB_BYTES;
          for (int s = 0; s < 2; ++s)
            tc::mma_tf32_tmem_a(dst + CS * i, src + CS * i + 8 * s,
                                tc::desc_kmajor(zb + s * 2 * SWTC_ZB_LBO, SWTC_ZB_LBO, SWTC_ZB_SBO), idesc_z, s > 0);
        }
      };
      // The issuer advances four streams, each in item order: MMA 1 of item k
      // (its residual operand filled, its tensor-memory pair read out by the
      // consumers two items back), z1 of k (MMA 1 of k done), MMA 2 of k (the
      // consumers' scaled operand written), z2 of k (MMA 2 of k done). It polls
      // the conditions and issues whatever is ready, so that the MMAs of two
      // items interleave and no stream waits behind another.
      int nA1 = 0, nA2 = 0, nB1 = 0, nB2 = 0;
      long long t_last = clock64();
      bool fail = false;
      while (nB2 < nmine && !fail && !sh.abort) {
        bool moved = false;
        if (nB2 < nB1 && tc::mbar_test(tc::smem_addr(&sh.d2[nB2 & 1]), (nB2 >> 1) & 1)) {
          const int k = nB2, b = k & 1;
          const uint32_t R1 = tmem + 256 * b;
          tc::fence_after_sync();
          zmma(sh.item[k % SWTC_ISLOTS], R1, R1 + 128, 1);
          tc::mma_commit(tc::smem_addr(&sh.f[b]));
          ++nB2;
          moved = true;
        }
        if (nB1 < nA2 && tc::mbar_test(tc::smem_addr(&sh.b2[nB1 & 1]), (nB1 >> 1) & 1)) {
          const int k = nB1, b = k & 1;
          const uint32_t R1 = tmem + 256 * b;
          const SwTcItem& I = sh.item[k % SWTC_ISLOTS];
          if (I.seg != seg_i) {
            // the inverse factor's last user, MMA 2 of item k - 1, must be done
            fail = (k >= 1 && !swtc_wait(sh, H, &sh.d2[(k - 1) & 1], ((k - 1) >> 1) & 1));
            if (fail) break;
            tc::mbar_expect_tx(tc::smem_addr(&sh.tma_i), (uint32_t)a_bytes);
            tc::bulk_g2s(sAi, blob + off_a + ((size_t)I.seg * 2 + 1) * a_bytes, (uint32_t)a_bytes,
                         tc::smem_addr(&sh.tma_i));
            fail = !swtc_wait(sh, H, &sh.tma_i, ph_i);
            if (fail) break;
            ph_i ^= 1;
            seg_i = I.seg;
          }
          tc::fence_after_sync();
          const uint32_t sb = tc::smem_addr(sB0 + b * b_bytes);
          for (int s = 0; s < kc / 2; ++s)
            tc::mma_tf32(R1, tc::desc_kmajor(tc::smem_addr(sAi) + s * 2 * SWTC_LBO, SWTC_LBO, sbo),
                         tc::desc_kmajor(sb + s * 2 * SWTC_LBO, SWTC_LBO, sbo), idesc_xy, s > 0);
          tc::mma_commit(tc::smem_addr(&sh.d2[b]));
          ++nB1;
          moved = true;
        }
        if (nA2 < nA1 && tc::mbar_test(tc::smem_addr(&sh.d1[nA2 & 1]), (nA2 >> 1) & 1)) {
          const int k = nA2, b = k & 1;
          const uint32_t R1 = tmem + 256 * b;
          tc::fence_after_sync();
          zmma(sh.item[k % SWTC_ISLOTS], R1, R1 + 128, 0);
          tc::mma_commit(tc::smem_addr(&sh.e[b]));
          ++nA2;
          moved = true;
        }
        if (nA1 < nmine && tc::mbar_test(tc::smem_addr(&sh.full[nA1 & 1]), (nA1 >> 1) & 1) &&
            (nA1 < 2 || tc::mbar_test(tc::smem_addr(&sh.empty[nA1 & 1]), ((nA1 - 2) >> 1) & 1))) {
          const int k = nA1, b = k & 1;
          const uint32_t R1 = tmem + 256 * b;
          const SwTcItem& I = sh.item[k % SWTC_ISLOTS];
          if (I.seg != seg_f) {
            // the forward factor's last user, MMA 1 of item k - 1, must be done
            fail = (k >= 1 && !swtc_wait(sh, H, &sh.d1[(k - 1) & 1], ((k - 1) >> 1) & 1));
            if (fail) break;
            tc::mbar_expect_tx(tc::smem_addr(&sh.tma_f), (uint32_t)a_bytes);
            tc::bulk_g2s(sAf, blob + off_a + (size_t)I.seg * 2 * a_bytes, (uint32_t)a_bytes, tc::smem_addr(&sh.tma_f));
            fail = !swtc_wait(sh, H, &sh.tma_f, ph_f);
            if (fail) break;
            ph_f ^= 1;
            seg_f = I.seg;
          }
          tc::fence_after_sync();
          const uint32_t sb = tc::smem_addr(sB0 + b * b_bytes);
          for (int s = 0; s < kc / 2; ++s)
            tc::mma_tf32(R1, tc::desc_kmajor(tc::smem_addr(sAf) + s * 2 * SWTC_LBO, SWTC_LBO, sbo),
                         tc::desc_kmajor(sb + s * 2 * SWTC_LBO, SWTC_LBO, sbo), idesc_xy, s > 0);
          tc::mma_commit(tc::smem_addr(&sh.d1[b]));
          ++nA1;
          moved = true;
        }
        if (moved) {
          t_last = clock64();
        } else if (clock64() - t_last <= kSwtcWaitLimit) {
          __nanosleep(20);  // leave the issue slots to the consumer warp of this sub-partition
        } else {
          atomicExch(H->err, DG_ERR_TIMEOUT);
          atomicExch(&sh.abort, 1);
        }
      }
    }
  } else {
    // ================= consumers: scale item li, output item li - 1 =================
    const int L = tid;  // TMEM lane: mode (j', l') for the scaling, node (j, l) for the output
    const int jj = L / MP, ll = L % MP;
    const bool active = L < MP2;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
    float inv[SWTC_MAXZCLS][MP];  // 1 / (lx + ly + lz) of this lane's mode for every z class
    int cur_seg = -1;
    // output of item k: F of each patch to the patch buffer
    auto output = [&](int k) -> bool {
      const int b = k & 1;
      const bool ok = swtc_wait(sh, H, &sh.f[b], (k >> 1) & 1);
      if (__any_sync(0xffffffffu, !ok || sh.abort != 0)) return false;
      tc::fence_after_sync();
      const SwTcItem& I = sh.item[k % SWTC_ISLOTS];
      const uint32_t tcol = tlane + 256 * b + 128;
      const int np = I.np;
      // every patch's columns loaded at once, then one wait
      uint32_t v[SWTC8_NPMAX][12];
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i)
        if (i < np) tc::tmem_ld12_async(tcol + i * CS, v[i]);
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i) tc::tmem_wait12(v[i]);
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i) {
        if (i < np && active) {
          // streaming stores: the patch solutions are read once, by the gather
          float* out = zp + ((long long)I.src[i] * E + I.elem[i]) * MP3 + L;
#pragma unroll
          for (int c = 0; c < MP; ++c) __stcs(out + c * MP2, __uint_as_float(v[i][c]));
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(tc::smem_addr(&sh.empty[b]));
      tc::mbar_arrive(tc::smem_addr(&sh.ifree[k % SWTC_ISLOTS]));
      return true;
    };
    int li = 0;
    for (; li < nmine; ++li) {
      const int b = li & 1;
      // full[b]: the item description is written; e[b]: E of the item is ready
      const bool ok = swtc_wait(sh, H, &sh.full[b], (li >> 1) & 1) && swtc_wait(sh, H, &sh.e[b], (li >> 1) & 1);
      // tensor-memory loads are warp-collective: a warp leaves as a whole
      if (__any_sync(0xffffffffu, !ok || sh.abort != 0)) break;
      tc::fence_after_sync();
      const SwTcItem& I = sh.item[li % SWTC_ISLOTS];
      const int np = I.np;
      if (I.seg != cur_seg) {
        cur_seg = I.seg;
        const float* tx = sh.lxy[0][sh.seg_cx[cur_seg]];
        const float* ty = sh.lxy[1][sh.seg_cy[cur_seg]];
        const float lxy = active ? tx[ll] + ty[jj] : 0.f;
        const bool vxy = active && ll < (int)tx[MP] && jj < (int)ty[MP];
#pragma unroll
        for (int z = 0; z < SWTC_MAXZCLS; ++z) {
          const float* zt = sh.z + z * SWTC_ZSTR(MP);
          const int mzc = z < H->ncz ? (int)zt[MP * MPP + MPP] : 0;
#pragma unroll
          for (int c = 0; c < MP; ++c) inv[z][c] = (vxy && c < mzc) ? 1.0f / (lxy + zt[MP * MPP + c]) : 0.0f;
        }
      }
      unsigned char* col = sB0 + b * b_bytes + (L / 4) * SWTC_LBO + (L % 4) * 4;
      const uint32_t tcol = tlane + 256 * b + 128;
      // every patch's columns loaded at once, then one wait
      uint32_t tv[SWTC8_NPMAX][12];
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i)
        if (i < np) tc::tmem_ld12_async(tcol + i * CS, tv[i]);
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i) tc::tmem_wait12(tv[i]);
#pragma unroll
      for (int i = 0; i < SWTC8_NPMAX; ++i) {
        if (i >= np) break;
        const int cz = I.cz[i];
        if (active) {
          // the class's scaling row, selected without indexing the register array
          float iv[MP];
#pragma unroll
          for (int c = 0; c < MP; ++c) iv[c] = inv[0][c];
#pragma unroll
          for (int z = 1; z < SWTC_MAXZCLS; ++z)
            if (cz == z)
#pragma unroll
              for (int c = 0; c < MP; ++c) iv[c] = inv[z][c];
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            const int row = i * CS + c;
            *(float*)(col + (row >> 3) * sbo + (row & 7) * 16) = tc::to_tf32(__uint_as_float(tv[i][c]) * iv[c]);
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

static int tc8_smem(const SwTcGeom& g) { return 2 * g.a_bytes + SWTC_BSLOTS * g.b_bytes + g.zb_bytes; }

// Opt the kernel into the dynamic shared memory of geometry g (at set-up,
// before any stream capture).
cudaError_t schwarz_tc8_prepare(const SwTcGeom& g) {
  return cudaFuncSetAttribute(k_schwarz_patch_tc8, cudaFuncAttributeMaxDynamicSharedMemorySize, tc8_smem(g));
}

cudaError_t launch_schwarz_patch_tc8(const SwTcPlan& plan, const float* r, float* zp, const int* act, int nact,
                                     cudaStream_t s) {
  const SwTcHead& head = plan.head;
  const SwTcGeom& g = plan.geom;
  if (head.n1 != 8 || g.cs != SWTC8_CS || g.np > SWTC8_NPMAX || head.ncz > SWTC_MAXZCLS) return cudaErrorInvalidValue;
  long long items = 0;
  for (int k = 0; k < head.nseg; ++k) items += ((long long)head.seg_ncol[k] * head.nz * nact + g.np - 1) / g.np;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(items, nsm));
  count_launch();
  k_schwarz_patch_tc8<<<grid, THREADS, tc8_smem(g), s>>>((const unsigned char*)plan.blob, g, r, zp, act, nact);
  return cudaGetLastError();
}

}  // namespace dg
