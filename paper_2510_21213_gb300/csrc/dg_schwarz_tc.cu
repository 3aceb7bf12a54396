// Tensor-core patch solve of the overlapping Schwarz smoother (FP32 inner
// solve, levels of degree 6-8).
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
// copy, its residual entries by 4-byte asynchronous copies (zero-filled
// outside the domain). The output goes to the same patch buffer as the SIMT
// kernel's, [source][element][MP^3] (x fastest), for k_schwarz_gather.
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

bool swtc_geometry(int n1, SwTcGeom& g) {
  g.mp = n1 + 2;
  const int mp2 = g.mp * g.mp;
  if (n1 < 7 || n1 > 9) return false;
  g.kpad = (mp2 + 7) / 8 * 8;
  g.kc = g.kpad / 4;
  g.sbo = g.kc * SWTC_LBO;
  g.a_bytes = ((mp2 + 7) / 8) * g.sbo;
  // patches per item: MP rows of the B operand each, at a stride of SWTC_CS rows
  // (D columns), so that every tensor-memory load starts at a multiple of 4
  g.np = g.mp == 11 ? 10 : 21;  // the B operand must fit next to two A factors
  g.ncol = (g.np * SWTC_CS + 15) / 16 * 16;
  g.b_bytes = (g.ncol / 8) * g.sbo;
  return 2 * (size_t)g.a_bytes + g.b_bytes + sizeof(SwTcShared) <= 232448;
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
    if ((int)rep[d].size() > SWTC_MAXCLS) return {};
    off += (size_t)L.n[d] * STR;
  }
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
  H.off_a = pos;
  pos += (size_t)H.nseg * 2 * g.a_bytes;
  std::vector<unsigned char> blob(pos, 0);
  std::memcpy(blob.data() + H.off_cols, cols.data(), sizeof(int) * cols.size());
  std::memcpy(blob.data() + H.off_zcls, cls[2], sizeof(int) * L.n[2]);
  float* zt = (float*)(blob.data() + H.off_z);
  for (int c = 0; c < ncz; ++c) {
    const double* t = tab(2, rep[2][c]);
    float* o = zt + (size_t)c * SWTC_ZSTR(MP);
    for (int i = 0; i < MP * MP; ++i) o[i] = (float)t[2 + i];
    for (int k = 0; k < MP; ++k) o[MP * MP + k] = (float)t[2 + MP * MP + k];
    o[MP * MP + MP] = (float)t[0];
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
  // (j,l)) and inverse (rows = nodes, K = modes), value Sy[j][j'] Sx[l][l']
  for (int s = 0; s < H.nseg; ++s) {
    const double* tx = tab(0, rep[0][H.seg_cx[s]]);
    const double* ty = tab(1, rep[1][H.seg_cy[s]]);
    unsigned char* af = blob.data() + H.off_a + (size_t)s * 2 * g.a_bytes;
    unsigned char* ai = af + g.a_bytes;
    for (int j = 0; j < MP; ++j)
      for (int l = 0; l < MP; ++l)
        for (int jp = 0; jp < MP; ++jp)
          for (int lp = 0; lp < MP; ++lp) {
            const float v = host_tf32((float)(ty[2 + j * MP + jp] * tx[2 + l * MP + lp]));
            const int node = j * MP + l, mode = jp * MP + lp;
            std::memcpy(af + opnd_off(mode, node, g.sbo), &v, 4);
            std::memcpy(ai + opnd_off(node, mode, g.sbo), &v, 4);
          }
  }
  std::memcpy(blob.data(), &H, sizeof(H));
  return blob;
}

// ---------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------
constexpr long long kWaitLimit = 1LL << 31;  // clock cycles (about a second) before a wait gives up

template <int N1>
__global__ void __launch_bounds__(SWTC_THREADS, 1)
    k_schwarz_patch_tc(const LevelOp* __restrict__ op, const unsigned char* __restrict__ blob,
                       const float* __restrict__ r, float* __restrict__ zp, const int* __restrict__ act, int nact) {
  constexpr int MP = N1 + 2, MP2 = MP * MP, MP3 = MP2 * MP, NPE = N1 * N1 * N1;
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ SwTcShared sh;
  const SwTcHead* H = (const SwTcHead*)blob;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  const int L = 32 * quad + lane;  // TMEM lane of this thread: mode / node (j, l) = (L / MP, L % MP)
  const bool active = L < MP2;
  const int a_bytes = H->geom.a_bytes, sbo = H->geom.sbo, NP = H->geom.np, kc = H->geom.kc;
  const int ncol = H->geom.ncol;
  unsigned char* sA0 = dsm;
  unsigned char* sA1 = dsm + a_bytes;
  unsigned char* sB = dsm + 2 * a_bytes;
  const int nx = H->nx, ny = H->ny, nz = H->nz;
  const int E = nx * ny * nz;
  const long long Nq = (long long)E * NPE;
  const int* cols = (const int*)(blob + H->off_cols);
  const int* zcls = (const int*)(blob + H->off_zcls);
  // ---- set-up: barriers, tensor memory, z tables, zeroed B operand
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(&sh.mbar_tma), 1);
    tc::mbar_init(tc::smem_addr(&sh.mbar_mma), 1);
    tc::mbar_init_fence();
    sh.abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&sh.tmem, SWTC_TMEM_COLS);
  {
    const float* zt = (const float*)(blob + H->off_z);
    for (int i = tid; i < H->ncz * SWTC_ZSTR(MP); i += SWTC_THREADS) sh.z[i] = zt[i];
    const int nseg = H->nseg;
    if (tid == 0) {
      int acc = 0;
      for (int s = 0; s < nseg; ++s) {
        sh.item0[s] = acc;
        acc += (int)(((long long)H->seg_ncol[s] * nz * nact + NP - 1) / NP);
      }
      sh.item0[nseg] = acc;
    }
    uint4* b4 = (uint4*)sB;
    for (int i = tid; i < H->geom.b_bytes / 16; i += SWTC_THREADS) b4[i] = make_uint4(0, 0, 0, 0);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sh.tmem;
  const uint32_t tlane = tmem + ((uint32_t)(32 * quad) << 16);
  const uint32_t mbar_tma = tc::smem_addr(&sh.mbar_tma), mbar_mma = tc::smem_addr(&sh.mbar_mma);
  const uint32_t idesc = tc::idesc_tf32(128, ncol);
  uint32_t ph_mma = 0, ph_tma = 0;
  int cur_seg = -1;
  // per-thread constants of the current segment and z class
  float lxy = 0.f;
  bool vxy = false;
  int cur_cz = -1;
  float S[MP][MP], inv[MP];
  const int total = sh.item0[H->nseg];
  const int jj = L / MP, ll = L % MP;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    // ---- decode the item: segment, patches (source, element, z position)
    int seg = 0;
    while (sh.item0[seg + 1] <= it) ++seg;
    const long long q0 = (long long)(it - sh.item0[seg]) * NP;
    const int ncs = H->seg_ncol[seg];
    const long long per_z = (long long)ncs * nact;
    const int np = (int)std::min<long long>(NP, per_z * nz - q0);
    if (tid < np) {
      const long long q = q0 + tid;
      const int ez = (int)(q / per_z);
      const long long rem = q - (long long)ez * per_z;
      const int colrel = (int)(rem / nact), a = (int)(rem - (long long)colrel * nact);
      const int ex = cols[2 * (H->seg_col0[seg] + colrel)], ey = cols[2 * (H->seg_col0[seg] + colrel) + 1];
      sh.src[tid] = act[a];
      sh.elem[tid] = ex + nx * (ey + ny * ez);
      sh.ez[tid] = ez;
      sh.ex[tid] = ex;
      sh.ey[tid] = ey;
    }
    // ---- new class pair: bulk-copy its two Kronecker factors (no MMA reads them now)
    if (seg != cur_seg) {
      if (tid == 0) {
        const unsigned char* src = blob + H->off_a + (size_t)seg * 2 * a_bytes;
        tc::mbar_expect_tx(mbar_tma, 2u * (uint32_t)a_bytes);
        tc::bulk_g2s(sA0, src, (uint32_t)a_bytes, mbar_tma);
        tc::bulk_g2s(sA1, src + a_bytes, (uint32_t)a_bytes, mbar_tma);
      }
      const float* xy = (const float*)(blob + H->off_xy);
      const float* tx = xy + (size_t)H->seg_cx[seg] * (MP + 1);
      const float* ty = xy + H->off_y + (size_t)H->seg_cy[seg] * (MP + 1);
      if (active) {
        lxy = tx[ll] + ty[jj];
        vxy = ll < (int)tx[MP] && jj < (int)ty[MP];
      }
      cur_cz = -1;
    }
    __syncthreads();
    // ---- fill B: row (i, k), column (j, l) = residual at patch node (l, j, k)
    if (active) {
      for (int i = half; i < np; i += 2) {
        const int e = sh.elem[i];
        const int ex = sh.ex[i], ey = sh.ey[i], ez = sh.ez[i];
        const int oLx = ex > 0, oLy = ey > 0, oLz = ez > 0;
        const int mx = N1 + oLx + (ex < nx - 1), my = N1 + oLy + (ey < ny - 1), mz = N1 + oLz + (ez < nz - 1);
        const int X = ex * N1 - oLx + ll, Y = ey * N1 - oLy + jj;
        const bool vx = ll < mx && jj < my;
        const int EX = vx ? X / N1 : 0, EY = vx ? Y / N1 : 0;
        const long long bxy =
            (long long)sh.src[i] * Nq + (long long)(EX + nx * EY) * NPE + (X - EX * N1) + N1 * (Y - EY * N1);
        (void)e;
#pragma unroll
        for (int k = 0; k < MP; ++k) {
          const int Z = ez * N1 - oLz + k;
          const bool v = vx && k < mz;
          const int EZ = v ? Z / N1 : 0;
          const float* g = v ? r + bxy + (long long)EZ * nx * ny * NPE + (long long)N1 * N1 * (Z - EZ * N1) : r;
          const int row = i * SWTC_CS + k;
          tc::cp_async4(sB + (size_t)(row / 8) * sbo + (size_t)(L / 4) * SWTC_LBO + (size_t)(row % 8) * 16 +
                            (size_t)(L % 4) * 4,
                        g, v ? 4u : 0u);
        }
      }
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- MMA 1: D = A_fwd x B^T
    if (tid == 0) {
      tc::fence_after_sync();
      bool ok = true;
      if (seg != cur_seg) {
        ok = tc::mbar_wait(mbar_tma, ph_tma, kWaitLimit);
        ph_tma ^= 1;
      }
      if (!ok) {
        atomicExch(H->err, DG_ERR_TIMEOUT);
        sh.abort = 1;
      } else {
        for (int s = 0; s < kc / 2; ++s)
          tc::mma_tf32(tmem, tc::desc_kmajor(tc::smem_addr(sA0) + s * 2 * SWTC_LBO, SWTC_LBO, sbo),
                       tc::desc_kmajor(tc::smem_addr(sB) + s * 2 * SWTC_LBO, SWTC_LBO, sbo), idesc, s > 0);
        tc::mma_commit(mbar_mma);
      }
    }
    cur_seg = seg;
    __syncthreads();
    if (sh.abort) break;
    if (!tc::mbar_wait(mbar_mma, ph_mma, kWaitLimit)) {
      atomicExch(H->err, DG_ERR_TIMEOUT);
      sh.abort = 1;
    }
    ph_mma ^= 1;
    tc::fence_after_sync();
    __syncthreads();
    if (sh.abort) break;
    // ---- z-step: Sz^T, scaling, Sz along each patch's z line, back into B
    for (int i = half; i < np; i += 2) {
      float t[SWTC_CS];
      tc::tmem_ld_x4<SWTC_CS / 4>(tlane + i * SWTC_CS, t);
      tc::tmem_wait_ld();
      const int cz = zcls[sh.ez[i]];
      if (cz != cur_cz) {
        cur_cz = cz;
        const float* zt = sh.z + cz * SWTC_ZSTR(MP);
        const int mzc = (int)zt[MP2 + MP];
#pragma unroll
        for (int a = 0; a < MP; ++a)
#pragma unroll
          for (int b = 0; b < MP; ++b) S[a][b] = zt[a * MP + b];
#pragma unroll
        for (int b = 0; b < MP; ++b) inv[b] = (vxy && b < mzc) ? 1.0f / (lxy + zt[MP2 + b]) : 0.0f;
      }
      if (active) {
        float u[MP];
#pragma unroll
        for (int b = 0; b < MP; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int a = 0; a < MP; ++a) acc = fmaf(S[a][b], t[a], acc);
          u[b] = acc * inv[b];
        }
#pragma unroll
        for (int a = 0; a < MP; ++a) {
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < MP; ++b) acc = fmaf(S[a][b], u[b], acc);
          const int row = i * SWTC_CS + a;
          *(float*)(sB + (size_t)(row / 8) * sbo + (size_t)(L / 4) * SWTC_LBO + (size_t)(row % 8) * 16 +
                    (size_t)(L % 4) * 4) = tc::to_tf32(acc);
        }
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- MMA 2: D = A_inv x B^T
    if (tid == 0) {
      tc::fence_after_sync();
      for (int s = 0; s < kc / 2; ++s)
        tc::mma_tf32(tmem, tc::desc_kmajor(tc::smem_addr(sA1) + s * 2 * SWTC_LBO, SWTC_LBO, sbo),
                     tc::desc_kmajor(tc::smem_addr(sB) + s * 2 * SWTC_LBO, SWTC_LBO, sbo), idesc, s > 0);
      tc::mma_commit(mbar_mma);
    }
    if (!tc::mbar_wait(mbar_mma, ph_mma, kWaitLimit)) {
      atomicExch(H->err, DG_ERR_TIMEOUT);
      sh.abort = 1;
    }
    ph_mma ^= 1;
    tc::fence_after_sync();
    __syncthreads();
    if (sh.abort) break;
    // ---- output: patch node (l, j, k) of patch i
    for (int i = half; i < np; i += 2) {
      float v[SWTC_CS];
      tc::tmem_ld_x4<SWTC_CS / 4>(tlane + i * SWTC_CS, v);
      tc::tmem_wait_ld();
      if (active) {
        float* out = zp + ((long long)sh.src[i] * E + sh.elem[i]) * MP3 + L;
#pragma unroll
        for (int k = 0; k < MP; ++k) out[k * MP2] = v[k];
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  // ---- teardown
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
  const int smem = 2 * g.a_bytes + g.b_bytes;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(items, nsm));
  count_launch();
  k_schwarz_patch_tc<N1><<<grid, SWTC_THREADS, smem, s>>>(dop, blob, r, zp, act, nact);
  return cudaGetLastError();
}

// Opt the kernel of this degree into the dynamic shared memory it needs (at
// set-up, before any stream capture).
cudaError_t schwarz_tc_prepare(int n1) {
  SwTcGeom g;
  if (!swtc_geometry(n1, g)) return cudaErrorInvalidValue;
  const int smem = 2 * g.a_bytes + g.b_bytes;
  switch (n1) {
    case 7: return cudaFuncSetAttribute(k_schwarz_patch_tc<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case 8: return cudaFuncSetAttribute(k_schwarz_patch_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case 9: return cudaFuncSetAttribute(k_schwarz_patch_tc<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_schwarz_patch_tc(const LevelOp& hop, const LevelOp* dop, const SwTcPlan& plan, const float* r,
                                    float* zp, const int* act, int nact, cudaStream_t s) {
  const SwTcHead& head = plan.head;
  const SwTcGeom& g = head.geom;
  long long items = 0;
  for (int k = 0; k < head.nseg; ++k) items += ((long long)head.seg_ncol[k] * head.nz * nact + g.np - 1) / g.np;
  const unsigned char* b = (const unsigned char*)plan.blob;
  switch (hop.n1) {
    case 7: return launch_tc_n1<7>(dop, b, g, r, zp, act, nact, items, s);
    case 8: return launch_tc_n1<8>(dop, b, g, r, zp, act, nact, items, s);
    case 9: return launch_tc_n1<9>(dop, b, g, r, zp, act, nact, items, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
