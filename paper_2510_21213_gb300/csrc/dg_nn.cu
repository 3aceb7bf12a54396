// Per-element 3-D convolutional network for the learned initial guess (not in
// the paper; the learned form of the exchange-build solves).
//
// Network: per element, two input channels on the (p+1)^3 nodes (scaled
// source, scaled coarse-grid solution) -> conv 3x3x3 (2 -> 32) -> ReLU ->
// conv 3x3x3 (32 -> 32) -> ReLU -> conv 3x3x3 (32 -> 2), zero padding at the
// element border. Weights are kept in FP32 (master copy, Adam) and used in
// BF16; activations are stored in BF16; every sum accumulates in FP32.
//
// Layouts: nodes of an element x-fastest, channels last: act[e][node][C].
// Tap t = (dz+1)*9 + (dy+1)*3 + (dx+1). Parameter vector (FP32):
//   W1 [27][2][32] | b1 [32] | W2 [27][32][32] (tap, ci, co) | b2 [32] |
//   W3 [27][32][2] | b3 [2]
// BF16 copies of W2: W2t [27][32 co][32 ci] (forward) and W2o [27][32 ci][32 co]
// (gradient with respect to the layer input).
//
// The 32 -> 32 layer and its two gradients run on the tensor cores with
// mma.sync m16n8k16 (BF16 in, FP32 accumulate); A tiles come from
// channel-last shared memory with ldmatrix (16 nodes x 16 channels), the
// convolution taps are row offsets into a zero-bordered (p+3)^3 grid.
#include <cuda_bf16.h>

#include "dg_internal.h"

namespace dg {

constexpr int NN_OW1 = 0, NN_OB1 = 1728, NN_OW2 = 1760, NN_OB2 = 29408, NN_OW3 = 29440, NN_OB3 = 31168;
static_assert(NN_NPARAM == 31170, "parameter layout");
constexpr int NN_H = 32;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma16816(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int N1>
struct NNCfg {
  static constexpr int P = N1 + 2;
  static constexpr int P3 = P * P * P;
  static constexpr int NPE = N1 * N1 * N1;
  static constexpr int MT = (NPE + 15) / 16;  // 16-node tiles
  static constexpr int THREADS = 256;
};

template <int N1>
__device__ __forceinline__ int pad_index(int n) {
  constexpr int P = N1 + 2;
  const int x = n % N1, y = (n / N1) % N1, z = n / (N1 * N1);
  return (z + 1) * P * P + (y + 1) * P + (x + 1);
}
template <int N1>
__device__ __forceinline__ int tap_offset(int t) {
  constexpr int P = N1 + 2;
  return (t / 9 - 1) * P * P + ((t / 3) % 3 - 1) * P + (t % 3 - 1);
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Shared-memory activations: row p (padded node) holds 32 BF16 channels as four
// 16-byte chunks; chunk c of row p is stored at position c ^ ((p >> 1) & 3), so
// the eight consecutive rows an ldmatrix phase reads fall into distinct banks.
__device__ __forceinline__ int swz(int p, int ch) {
  return p * NN_H + ((((ch >> 3) ^ ((p >> 1) & 3)) << 3) | (ch & 7));
}

constexpr int NN_FWD_THREADS = 512;
constexpr int NN_W2LD = 40;  // padded row of the staged W2 (bank-conflict-free B fragment loads)

template <int N1>
__global__ void __launch_bounds__(NN_FWD_THREADS, 1)
    k_nn_forward(const float* __restrict__ prm, const __nv_bfloat16* __restrict__ W2t, const float* __restrict__ in,
                 float* __restrict__ out, __nv_bfloat16* __restrict__ a1_out, __nv_bfloat16* __restrict__ a2_out,
                 long long ne) {
  using C = NNCfg<N1>;
  constexpr int P3 = C::P3, NPE = C::NPE, MT = C::MT;
  constexpr int NT = NN_FWD_THREADS, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sA1 = (__nv_bfloat16*)smem;                           // [P3][32] swizzled
  __nv_bfloat16* sA2 = sA1 + P3 * NN_H;                                 // [P3][32] swizzled
  __nv_bfloat16* sW2 = sA2 + P3 * NN_H;                                 // [27][32 co][NN_W2LD] (ci)
  float* sIn = (float*)(sW2 + 27 * 32 * NN_W2LD);                      // [P3][2]
  float* sW1 = sIn + 2 * P3;                                           // [27][2][32] + b1
  float* sW3 = sW1 + 1728 + 32;                                        // [27][32][2] + b3
  float* sb2 = sW3 + 1728 + 2;                                         // [32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 2 * P3; i += NT) sIn[i] = 0.f;
  for (int i = tid; i < P3 * NN_H; i += NT) ((unsigned*)sA1)[i] = 0u;  // sA1 and sA2
  for (int i = tid; i < 27 * 32 * 16; i += NT) {
    const int row = i >> 4, c2 = i & 15;
    ((unsigned*)(sW2 + row * NN_W2LD))[c2] = ((const unsigned*)(W2t + row * 32))[c2];
  }
  for (int i = tid; i < 1760; i += NT) sW1[i] = prm[NN_OW1 + i];
  for (int i = tid; i < 1730; i += NT) sW3[i] = prm[NN_OW3 + i];
  for (int i = tid; i < 32; i += NT) sb2[i] = prm[NN_OB2 + i];
  __syncthreads();
  const int g = lane >> 2, c4 = lane & 3;
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int i = tid; i < NPE; i += NT) {
      const int p = pad_index<N1>(i);
      const float2 v = ((const float2*)in)[e * NPE + i];
      sIn[2 * p] = v.x;
      sIn[2 * p + 1] = v.y;
    }
    __syncthreads();
    // layer 1 (2 -> 32), SIMT: thread = (node, group of 8 output channels = one chunk)
    for (int w = tid; w < NPE * 4; w += NT) {
      const int n = w >> 2, cg = (w & 3) * 8;
      const int p = pad_index<N1>(n);
      float acc[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = sW1[1728 + cg + c];
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int q = p + tap_offset<N1>(t);
        const float i0 = sIn[2 * q], i1 = sIn[2 * q + 1];
        const float* wt = sW1 + t * 64 + cg;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += i0 * wt[c] + i1 * wt[32 + c];
      }
      uint4 pk;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(fmaxf(acc[0], 0.f), fmaxf(acc[1], 0.f));
      __nv_bfloat162 h1 = __floats2bfloat162_rn(fmaxf(acc[2], 0.f), fmaxf(acc[3], 0.f));
      __nv_bfloat162 h2 = __floats2bfloat162_rn(fmaxf(acc[4], 0.f), fmaxf(acc[5], 0.f));
      __nv_bfloat162 h3 = __floats2bfloat162_rn(fmaxf(acc[6], 0.f), fmaxf(acc[7], 0.f));
      pk.x = *(unsigned*)&h0;
      pk.y = *(unsigned*)&h1;
      pk.z = *(unsigned*)&h2;
      pk.w = *(unsigned*)&h3;
      *(uint4*)(sA1 + swz(p, cg)) = pk;
    }
    __syncthreads();
    // layer 2 (32 -> 32) on the tensor cores: warp owns node tiles warp, warp + NW, ...
    for (int mt0 = warp; mt0 < MT; mt0 += 2 * NW) {
      float acc[2][4][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
      int rowp[2];
      bool tile_ok[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int mt = mt0 + NW * a;
        tile_ok[a] = mt < MT;
        const int node = mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
        rowp[a] = (tile_ok[a] && node < NPE) ? pad_index<N1>(node) : 0;  // padded row 0 is all zero
      }
      const int khalf = lane >> 4;  // which 8 channels of the 16-channel k step this lane's row address serves
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int off = tap_offset<N1>(t);
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
          // B fragments (k = ci, n = co) from the staged W2[t][co][ci]
          unsigned b[4][2];
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const __nv_bfloat16* wp = sW2 + (t * 32 + nt * 8 + g) * NN_W2LD + kh * 16 + 2 * c4;
            b[nt][0] = *(const unsigned*)wp;
            b[nt][1] = *(const unsigned*)(wp + 8);
          }
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            if (!tile_ok[a]) continue;
            const int qq = rowp[a] == 0 ? 0 : rowp[a] + off;  // rows past the element read the zero corner
            unsigned a0, a1, a2, a3;
            ldsm_x4(smem_u32(sA1 + swz(qq, kh * 16 + khalf * 8)), a0, a1, a2, a3);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) mma16816(acc[a][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
          }
        }
      }
      // epilogue: bias, ReLU, BF16 into sA2 (rows g and g+8, columns 2c4, 2c4+1 of each n tile)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (!tile_ok[a]) continue;
        const int mt = mt0 + NW * a;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int node = mt * 16 + g + 8 * h;
          if (node >= NPE) continue;
          const int p = pad_index<N1>(node);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int co = nt * 8 + 2 * c4;
            const float v0 = fmaxf(acc[a][nt][2 * h] + sb2[co], 0.f);
            const float v1 = fmaxf(acc[a][nt][2 * h + 1] + sb2[co + 1], 0.f);
            *(__nv_bfloat162*)(sA2 + swz(p, co)) = __floats2bfloat162_rn(v0, v1);
          }
        }
      }
    }
    __syncthreads();
    // layer 3 (32 -> 2), SIMT; optional copies of the activations for training
    for (int n = tid; n < NPE; n += NT) {
      const int p = pad_index<N1>(n);
      float o0 = sW3[1728], o1 = sW3[1729];
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int q = p + tap_offset<N1>(t);
        const float* wt = sW3 + t * 64;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint4 raw = *(const uint4*)(sA2 + swz(q, 8 * c));
          const __nv_bfloat162* hv = (const __nv_bfloat162*)&raw;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 v = __bfloat1622float2(hv[k]);
            const int ci = 8 * c + 2 * k;
            o0 += v.x * wt[2 * ci] + v.y * wt[2 * ci + 2];
            o1 += v.x * wt[2 * ci + 1] + v.y * wt[2 * ci + 3];
          }
        }
      }
      ((float2*)out)[e * NPE + n] = make_float2(o0, o1);
    }
    if (a1_out) {
      for (int i = tid; i < NPE * 4; i += NT) {
        const int n = i >> 2, c = i & 3;
        const int p = pad_index<N1>(n);
        ((uint4*)(a1_out + (e * NPE + n) * NN_H))[c] = *(const uint4*)(sA1 + swz(p, 8 * c));
        ((uint4*)(a2_out + (e * NPE + n) * NN_H))[c] = *(const uint4*)(sA2 + swz(p, 8 * c));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// backward: per-block partial gradients, reduced in a fixed order afterwards
// ---------------------------------------------------------------------------
template <int N1>
__global__ void __launch_bounds__(256, 1)
    k_nn_backward(const float* __restrict__ prm, const __nv_bfloat16* __restrict__ W2o, const float* __restrict__ in,
                  const __nv_bfloat16* __restrict__ a1g, const __nv_bfloat16* __restrict__ a2g,
                  const float* __restrict__ gout, float* __restrict__ part, long long ne) {
  using C = NNCfg<N1>;
  constexpr int P3 = C::P3, NPE = C::NPE, MT = C::MT;
  extern __shared__ __align__(16) unsigned char smem[];
  // sA1 holds a1 until the layer-2 weight gradient is done, then g_a1 (masked);
  // the BF16 arrays come first: ldmatrix rows must be 16-byte aligned
  __nv_bfloat16* sA1 = (__nv_bfloat16*)smem;                           // [P3][32]
  __nv_bfloat16* sA2 = sA1 + P3 * NN_H;                                 // [P3][32] -> g_a2 (masked)
  float* sIn = (float*)(sA2 + P3 * NN_H);                              // [P3][2]
  float* sG3 = sIn + 2 * P3;                                           // [P3][2]
  float* sW3 = sG3 + 2 * P3;                                           // [27][32][2]
  float* dW1 = sW3 + 1728;                                             // [27][2][32]
  float* dW3 = dW1 + 1728;                                             // [27][32][2]
  float* db = dW3 + 1728;                                              // b1[32] b2[32] b3[2]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 4 * P3; i += 256) sIn[i] = 0.f;  // sIn and sG3
  for (int i = tid; i < 2 * P3 * NN_H; i += 256) sA1[i] = __float2bfloat16(0.f);
  for (int i = tid; i < 1728; i += 256) sW3[i] = prm[NN_OW3 + i];
  for (int i = tid; i < 1728 * 2 + 66; i += 256) dW1[i] = 0.f;
  // dW2 accumulators: warp owns taps warp, warp + 8, warp + 16, warp + 24 (< 27);
  // per tap 32 (ci) x 32 (co) = 2 x 4 mma tiles
  float accW[4][2][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int c = 0; c < 4; ++c) accW[a][m][n][c] = 0.f;
  __syncthreads();
  const int j = lane >> 3, r = lane & 7, g = lane >> 2, c4 = lane & 3;
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int i = tid; i < NPE; i += 256) {
      const int p = pad_index<N1>(i);
      sIn[2 * p] = in[(e * NPE + i) * 2];
      sIn[2 * p + 1] = in[(e * NPE + i) * 2 + 1];
      sG3[2 * p] = gout[(e * NPE + i) * 2];
      sG3[2 * p + 1] = gout[(e * NPE + i) * 2 + 1];
    }
    for (int i = tid; i < NPE * 16; i += 256) {
      const int n = i >> 4, c = i & 15;
      const int p = pad_index<N1>(n);
      ((__nv_bfloat162*)(sA1 + p * NN_H))[c] = ((const __nv_bfloat162*)(a1g + (e * NPE + n) * NN_H))[c];
      ((__nv_bfloat162*)(sA2 + p * NN_H))[c] = ((const __nv_bfloat162*)(a2g + (e * NPE + n) * NN_H))[c];
    }
    __syncthreads();
    // layer 3 weights: dW3[t][ci][co] += sum_n g3[n][co] a2[n + t][ci]; db3
    for (int w = tid; w < 1728 + 2; w += 256) {
      if (w < 1728) {
        const int t = w / 64, ci = (w / 2) % 32, co = w % 2;
        const int off = tap_offset<N1>(t);
        float acc = 0.f;
        for (int n = 0; n < NPE; ++n) {
          const int p = pad_index<N1>(n);
          acc += sG3[2 * p + co] * __bfloat162float(sA2[(p + off) * NN_H + ci]);
        }
        dW3[w] += acc;
      } else {
        const int co = w - 1728;
        float acc = 0.f;
        for (int n = 0; n < NPE; ++n) acc += sG3[2 * pad_index<N1>(n) + co];
        db[64 + co] += acc;
      }
    }
    __syncthreads();
    // g_a2[n][ci] = (sum_t sum_co W3[t][ci][co] g3[n - t][co]) * (a2[n][ci] > 0), in place of a2
    for (int w = tid; w < NPE * NN_H; w += 256) {
      const int n = w >> 5, ci = w & 31;
      const int p = pad_index<N1>(n);
      float acc = 0.f;
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int q = p - tap_offset<N1>(t);
        acc += sW3[t * 64 + ci * 2] * sG3[2 * q] + sW3[t * 64 + ci * 2 + 1] * sG3[2 * q + 1];
      }
      const float a2v = __bfloat162float(sA2[p * NN_H + ci]);
      sA2[p * NN_H + ci] = __float2bfloat16(a2v > 0.f ? acc : 0.f);
    }
    __syncthreads();
    for (int ci = tid; ci < NN_H; ci += 256) {
      float acc = 0.f;
      for (int n = 0; n < NPE; ++n) acc += __bfloat162float(sA2[pad_index<N1>(n) * NN_H + ci]);
      db[32 + ci] += acc;
    }
    // layer 2 weights on the tensor cores: dW2[t] (ci x co) += sum_n a1[n + t][ci] g_a2[n][co]
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int t = warp + 8 * a;
      if (t >= 27) continue;
      const int off = tap_offset<N1>(t);
#pragma unroll 1
      for (int kt = 0; kt < MT; ++kt) {
        // k = 16 nodes of tile kt; lane row address: node kt*16 + r + 8*(j>>1)
        const int node = kt * 16 + r + 8 * (j >> 1);
        const int pA = node < NPE ? pad_index<N1>(node) + off : 0;
        const int pB = node < NPE ? pad_index<N1>(node) : 0;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          // A (m = ci, k = node): transposed 8x8 blocks of a1[node][ci]
          unsigned a0, a1r, a2r, a3;
          ldsm_x4_t(smem_u32(sA1 + pA * NN_H + m * 16 + 8 * (j & 1)), a0, a1r, a2r, a3);
#pragma unroll
          for (int nh = 0; nh < 2; ++nh) {
            // B (k = node, n = co): transposed blocks of g_a2[node][co], two n-tiles
            unsigned b0, b1, b2, b3;
            ldsm_x4_t(smem_u32(sA2 + pB * NN_H + nh * 16 + 8 * (j & 1)), b0, b1, b2, b3);
            mma16816(accW[a][m][2 * nh], a0, a1r, a2r, a3, b0, b2);
            mma16816(accW[a][m][2 * nh + 1], a0, a1r, a2r, a3, b1, b3);
          }
        }
      }
    }
    __syncthreads();
    // layer 2 input gradient on the tensor cores: g_a1[n][ci] = mask * sum_t sum_co g_a2[n - t][co] W2[t][ci][co],
    // written over a1 (each lane reads the mask of exactly the entries it writes)
    for (int mt = warp; mt < MT; mt += 8) {
      float acc[4][4];
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[b][c] = 0.f;
      const int node = mt * 16 + r + 8 * (j & 1);
      const int prow = node < NPE ? pad_index<N1>(node) : -1;
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int off = tap_offset<N1>(t);
        const int q = prow >= 0 ? prow - off : 0;
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
          unsigned a0, a1r, a2r, a3;
          ldsm_x4(smem_u32(sA2 + q * NN_H + kh * 16 + 8 * (j >> 1)), a0, a1r, a2r, a3);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const __nv_bfloat16* wp = W2o + ((long long)t * 32 + nt * 8 + g) * 32 + kh * 16 + 2 * c4;
            mma16816(acc[nt], a0, a1r, a2r, a3, *(const unsigned*)wp, *(const unsigned*)(wp + 8));
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int nn = mt * 16 + g + 8 * h;
        if (nn >= NPE) continue;
        const int p = pad_index<N1>(nn);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int ci = nt * 8 + 2 * c4;
          __nv_bfloat162* dst = (__nv_bfloat162*)(sA1 + p * NN_H + ci);
          const float2 a1v = __bfloat1622float2(*dst);
          *dst = __floats2bfloat162_rn(a1v.x > 0.f ? acc[nt][2 * h] : 0.f, a1v.y > 0.f ? acc[nt][2 * h + 1] : 0.f);
        }
      }
    }
    __syncthreads();
    // layer 1 weights and biases
    for (int w = tid; w < 1728 + 32; w += 256) {
      if (w < 1728) {
        const int t = w / 64, ci = (w / 32) % 2, co = w % 32;
        const int off = tap_offset<N1>(t);
        float acc = 0.f;
        for (int n = 0; n < NPE; ++n) {
          const int p = pad_index<N1>(n);
          acc += sIn[2 * (p + off) + ci] * __bfloat162float(sA1[p * NN_H + co]);
        }
        dW1[w] += acc;
      } else {
        const int co = w - 1728;
        float acc = 0.f;
        for (int n = 0; n < NPE; ++n) acc += __bfloat162float(sA1[pad_index<N1>(n) * NN_H + co]);
        db[co] += acc;
      }
    }
    __syncthreads();
    // a1 and a2 were overwritten by their gradients at interior nodes only;
    // the zero borders stay, the interiors are reloaded for the next element
  }
  // write this block's partial gradients in parameter order
  float* pb = part + (long long)blockIdx.x * NN_NPARAM;
  for (int i = tid; i < 1728; i += 256) {
    pb[NN_OW1 + i] = dW1[i];
    pb[NN_OW3 + i] = dW3[i];
  }
  for (int i = tid; i < 32; i += 256) {
    pb[NN_OB1 + i] = db[i];
    pb[NN_OB2 + i] = db[32 + i];
  }
  if (tid < 2) pb[NN_OB3 + tid] = db[64 + tid];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int t = warp + 8 * a;
    if (t >= 27) continue;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int ci = m * 16 + g + 8 * h, co = n * 8 + 2 * c4;
          pb[NN_OW2 + (t * 32 + ci) * 32 + co] = accW[a][m][n][2 * h];
          pb[NN_OW2 + (t * 32 + ci) * 32 + co + 1] = accW[a][m][n][2 * h + 1];
        }
  }
}

__global__ void k_nn_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN_NPARAM) return;
  float acc = 0.f;
  for (int b = 0; b < nblk; ++b) acc += part[(long long)b * NN_NPARAM + i];
  grad[i] = acc;
}

// BF16 copies of W2 in both layouts
__global__ void k_nn_prep(const float* __restrict__ prm, __nv_bfloat16* __restrict__ W2t,
                          __nv_bfloat16* __restrict__ W2o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * 32 * 32) return;
  const int t = i / 1024, ci = (i / 32) % 32, co = i % 32;
  const __nv_bfloat16 v = __float2bfloat16(prm[NN_OW2 + i]);
  W2o[i] = v;
  W2t[(t * 32 + co) * 32 + ci] = v;
}

__global__ void k_nn_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                          float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN_NPARAM) return;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  prm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static size_t fwd_smem(int n1) {
  const int P3 = (n1 + 2) * (n1 + 2) * (n1 + 2);
  return 2 * sizeof(__nv_bfloat16) * P3 * NN_H + sizeof(__nv_bfloat16) * 27 * 32 * NN_W2LD + sizeof(float) * 2 * P3 +
         sizeof(float) * (1760 + 1730 + 32);
}
static size_t bwd_smem(int n1) {
  const int P3 = (n1 + 2) * (n1 + 2) * (n1 + 2), NPE = n1 * n1 * n1;
  (void)NPE;
  return sizeof(float) * 4 * P3 + 2 * sizeof(__nv_bfloat16) * P3 * NN_H + sizeof(float) * (1728 * 3 + 66);
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// resident blocks of a kernel per SM at its dynamic shared memory (at least 1)
template <typename K>
static int blocks_per_sm(K kern, size_t smem, int threads = 256) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem) != cudaSuccess || b < 1) b = 1;
  return b;
}

template <int N1>
static cudaError_t nn_fwd_n1(const float* prm, const __nv_bfloat16* W2t, const float* in, float* out,
                             __nv_bfloat16* a1, __nv_bfloat16* a2, long long ne, cudaStream_t s) {
  const size_t sm = fwd_smem(N1);
  static int bps = 0;
  if (!bps) {
    cudaError_t e = cudaFuncSetAttribute(k_nn_forward<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    bps = blocks_per_sm(k_nn_forward<N1>, sm, NN_FWD_THREADS);
  }
  const long long cap = (long long)sm_count() * bps;
  const long long grid = ne < cap ? ne : cap;
  if (grid < 1) return cudaSuccess;
  count_launch();
  k_nn_forward<N1><<<(unsigned)grid, NN_FWD_THREADS, sm, s>>>(prm, W2t, in, out, a1, a2, ne);
  return cudaGetLastError();
}

template <int N1>
static int nn_bwd_blocks(long long ne) {
  static int bps = 0;
  if (!bps) {
    const size_t sm = bwd_smem(N1);
    if (cudaFuncSetAttribute(k_nn_backward<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return 0;
    bps = blocks_per_sm(k_nn_backward<N1>, sm);
  }
  const long long cap = (long long)sm_count() * bps;
  return (int)(ne < cap ? (ne < 1 ? 1 : ne) : cap);
}

template <int N1>
static cudaError_t nn_bwd_n1(const float* prm, const __nv_bfloat16* W2o, const float* in, const __nv_bfloat16* a1,
                             const __nv_bfloat16* a2, const float* gout, float* part, int nblk, long long ne,
                             cudaStream_t s) {
  count_launch();
  k_nn_backward<N1><<<nblk, 256, bwd_smem(N1), s>>>(prm, W2o, in, a1, a2, gout, part, ne);
  return cudaGetLastError();
}

cudaError_t nn_prep(const float* prm, void* W2t, void* W2o, cudaStream_t s) {
  count_launch();
  k_nn_prep<<<(27 * 1024 + 255) / 256, 256, 0, s>>>(prm, (__nv_bfloat16*)W2t, (__nv_bfloat16*)W2o);
  return cudaGetLastError();
}

cudaError_t nn_forward(int n1, const float* prm, const void* W2tv, const float* in, float* out, void* a1v, void* a2v,
                       long long ne, cudaStream_t s) {
  const __nv_bfloat16* W2t = (const __nv_bfloat16*)W2tv;
  __nv_bfloat16* a1 = (__nv_bfloat16*)a1v;
  __nv_bfloat16* a2 = (__nv_bfloat16*)a2v;
  switch (n1) {
    case 2: return nn_fwd_n1<2>(prm, W2t, in, out, a1, a2, ne, s);
    case 3: return nn_fwd_n1<3>(prm, W2t, in, out, a1, a2, ne, s);
    case 4: return nn_fwd_n1<4>(prm, W2t, in, out, a1, a2, ne, s);
    case 5: return nn_fwd_n1<5>(prm, W2t, in, out, a1, a2, ne, s);
    case 6: return nn_fwd_n1<6>(prm, W2t, in, out, a1, a2, ne, s);
    case 7: return nn_fwd_n1<7>(prm, W2t, in, out, a1, a2, ne, s);
    case 8: return nn_fwd_n1<8>(prm, W2t, in, out, a1, a2, ne, s);
    default: return cudaErrorInvalidValue;
  }
}

// blocks (and gradient partials) of the backward kernel for ne elements; 0 on error
int nn_backward_blocks(int n1, long long ne) {
  switch (n1) {
    case 2: return nn_bwd_blocks<2>(ne);
    case 3: return nn_bwd_blocks<3>(ne);
    case 4: return nn_bwd_blocks<4>(ne);
    case 5: return nn_bwd_blocks<5>(ne);
    case 6: return nn_bwd_blocks<6>(ne);
    case 7: return nn_bwd_blocks<7>(ne);
    case 8: return nn_bwd_blocks<8>(ne);
    default: return 0;
  }
}

cudaError_t nn_backward(int n1, const float* prm, const void* W2ov, const float* in, const void* a1v, const void* a2v,
                        const float* gout, float* part, float* grad, long long ne, cudaStream_t s) {
  const __nv_bfloat16* W2o = (const __nv_bfloat16*)W2ov;
  const __nv_bfloat16* a1 = (const __nv_bfloat16*)a1v;
  const __nv_bfloat16* a2 = (const __nv_bfloat16*)a2v;
  const int nblk = nn_backward_blocks(n1, ne);
  if (nblk < 1) return cudaErrorInvalidValue;
  cudaError_t e;
  switch (n1) {
    case 2: e = nn_bwd_n1<2>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    case 3: e = nn_bwd_n1<3>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    case 4: e = nn_bwd_n1<4>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    case 5: e = nn_bwd_n1<5>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    case 6: e = nn_bwd_n1<6>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    case 7: e = nn_bwd_n1<7>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    case 8: e = nn_bwd_n1<8>(prm, W2o, in, a1, a2, gout, part, nblk, ne, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  count_launch();
  k_nn_reduce<<<(NN_NPARAM + 255) / 256, 256, 0, s>>>(part, nblk, grad);
  return cudaGetLastError();
}

cudaError_t nn_adam(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2, float eps,
                    int step, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  count_launch();
  k_nn_adam<<<(NN_NPARAM + 255) / 256, 256, 0, s>>>(prm, grad, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace dg
