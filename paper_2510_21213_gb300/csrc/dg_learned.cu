// Learned initial guess of the pair solves (precision DG_PREC_MIXED_LEARNED;
// not in the paper): the coarse guess x_c from the degree-1 level of the
// multigrid hierarchy (Sec. 6.4), the per-element network of dg_nn.cu that
// corrects it, the energy-optimal scaling and the fallback test, the training
// step (energy-functional loss, backward kernels, Adam) and the dg_nn.h
// entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dg_mg.h"
#include "dg_nn.h"

namespace dg {

static_assert(DG_NN_NPARAM == NN_NPARAM, "parameter count");

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// out[src] = max_q |u[src][q]| (divided by the nodal mass if by_mass); out
// must be zero on entry. Grid (x: node blocks, y: active source); each block
// reduces its nodes (warp shuffles, then shared memory) and issues one atomic
// max. Non-negative doubles order like their bit patterns, so the integer
// atomic max is exact and order-independent.
__global__ void k_maxabs(const float* __restrict__ u, const LevelOp* __restrict__ op, int by_mass,
                         const int* __restrict__ act, long long Nq, double* __restrict__ out) {
  __shared__ double red[32];
  const int n1 = op->n1, npe = n1 * n1 * n1;
  const int src = act[blockIdx.y];
  const float* us = u + (long long)src * Nq;
  double best = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nq; q += (long long)gridDim.x * blockDim.x) {
    double v = fabs((double)us[q]);
    if (by_mass) {
      const int loc = (int)(q % npe);
      v /= op->ax[0].m[loc % n1] * op->ax[1].m[(loc / n1) % n1] * op->ax[2].m[loc / (n1 * n1)];
    }
    best = fmax(best, v);  // a NaN is dropped here; the fallback test catches it later
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0 && best > 0.0)
      atomicMax((unsigned long long*)&out[src], (unsigned long long)__double_as_longlong(best));
  }
}

// network input of nc sources act[0..nc): c0 = (b / m) / sb (right-hand side
// over the nodal mass), c1 = x_c / sx, with sb, sx their per-source maxima;
// laid out [source][element][node][2] (= [source][q][2])
__global__ void k_guess_features(const float* __restrict__ b, const float* __restrict__ xc,
                                 const double* __restrict__ sb, const double* __restrict__ sx,
                                 const LevelOp* __restrict__ op, const int* __restrict__ act, int nc, long long Nq,
                                 float* __restrict__ in) {
  const int n1 = op->n1, npe = n1 * n1 * n1;
  const long long total = (long long)nc * Nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(i / Nq);
    const long long q = i - (long long)kk * Nq;
    const int src = act[kk];
    const long long g = (long long)src * Nq + q;
    const int loc = (int)(q % npe);
    const int a = loc % n1, bb = (loc / n1) % n1, c = loc / (n1 * n1);
    const double m = op->ax[0].m[a] * op->ax[1].m[bb] * op->ax[2].m[c];
    const double ib = sb[src] > 0.0 ? 1.0 / sb[src] : 0.0, ix = sx[src] > 0.0 ? 1.0 / sx[src] : 0.0;
    in[2 * i] = (float)(ib * (double)b[g] / m);
    in[2 * i + 1] = (float)(ix * (double)xc[g]);
  }
}

// x *= num / den per source (unchanged unless both are positive and finite)
__global__ void k_scale_ratio(float* __restrict__ x, const double* __restrict__ num, const double* __restrict__ den,
                              const int* __restrict__ act, int nact, long long Nq) {
  const long long total = (long long)nact * Nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(i / Nq);
    const int src = act[kk];
    const double dn = den[src], nm = num[src];
    if (dn > 0.0 && nm > 0.0 && isfinite(dn) && isfinite(nm))
      x[(long long)src * Nq + (i - (long long)kk * Nq)] *= (float)(nm / dn);
  }
}

// y = x_c (1 + o1) + o0 sx for nc sources act[0..nc) (y = 0 where x_c = 0)
template <typename T>
__global__ void k_guess_combine(const float* __restrict__ xc, const float* __restrict__ out,
                                const double* __restrict__ sx, const int* __restrict__ act, int nc, long long Nq,
                                T* __restrict__ x0) {
  const long long total = (long long)nc * Nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(i / Nq);
    const long long g = (long long)act[kk] * Nq + (i - (long long)kk * Nq);
    const double s = sx[act[kk]];
    const double v = s > 0.0 ? (double)xc[g] * (1.0 + (double)out[2 * i + 1]) + (double)out[2 * i] * s : 0.0;
    x0[g] = (T)v;
  }
}

// x = alpha x, r = b - alpha r with alpha = num / den (0 unless both positive)
__global__ void k_guess_scale(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ b,
                              const double* __restrict__ num, const double* __restrict__ den,
                              const int* __restrict__ act, int nact, long long Nq) {
  const long long total = (long long)nact * Nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(i / Nq);
    const int src = act[kk];
    const long long g = (long long)src * Nq + (i - (long long)kk * Nq);
    const double dn = den[src], nm = num[src];
    const double al = (dn > 0.0 && nm > 0.0 && isfinite(dn) && isfinite(nm)) ? nm / dn : 0.0;
    x[g] = al * x[g];
    r[g] = b[g] - al * r[g];
  }
}

// training loss terms and gradient with respect to the network output for
// B sources: e = y - v (y the network's guess before smoothing, v the target
// potential), L_k = sum_q m_q e_q^2 / nv_k with nv_k = sum_q m_q v_q^2, the
// loss (1/B) sum_k L_k; dL/dy = 2 m e / (B nv), dy/do0 = sx, dy/do1 = x_c.
// e (FP32) is written for the loss reduction.
__global__ void k_train_gout(const float* __restrict__ xc, const float* __restrict__ y, const double* __restrict__ v,
                             const LevelOp* __restrict__ op, const double* __restrict__ sx,
                             const double* __restrict__ nv, int B, long long Nq, float* __restrict__ gout,
                             float* __restrict__ e_out) {
  const int n1 = op->n1, npe = n1 * n1 * n1;
  const long long total = (long long)B * Nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / Nq);
    const int loc = (int)((i - (long long)k * Nq) % npe);
    const double m = op->ax[0].m[loc % n1] * op->ax[1].m[(loc / n1) % n1] * op->ax[2].m[loc / (n1 * n1)];
    const double s = sx[k];
    const double nk = nv[k];
    const double e = (double)y[i] - v[i];
    double g0 = 0.0, g1 = 0.0;
    if (s > 0.0 && nk > 0.0) {
      const double gy = 2.0 * m * e / (nk * (double)B);
      g0 = gy * s;
      g1 = gy * (double)xc[i];
    }
    gout[2 * i] = (float)g0;
    gout[2 * i + 1] = (float)g1;
    e_out[i] = (float)e;
  }
}

static unsigned flat_grid(long long total) {
  const long long b = (total + 255) / 256;
  return (unsigned)std::max(1LL, std::min(b, 152LL * 16));
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
static int nn_require(dg_ctx* h) {
  if (h->levels[0].op.n1 > NN_MAXN1) {
    h->err = "learned guess: the network supports p <= 7";
    return DG_ERR_UNSUPPORTED;
  }
  if (!h->nn.have) {
    h->err = "learned guess: no network parameters set";
    return DG_ERR_INVALID_ARG;
  }
  return DG_OK;
}

static int nn_bf16(dg_ctx* h, cudaStream_t s) {
  NNState& nn = h->nn;
  if (nn.bf16_ok) return DG_OK;
  DG_CK(nn.W2t.ensure(2 * 27 * 1024));
  DG_CK(nn.W2o.ensure(2 * 27 * 1024));
  DG_CK(nn_prep(nn.prm.as<float>(), nn.W2t.p, nn.W2o.p, s));
  nn.bf16_ok = true;
  return DG_OK;
}

static int nn_set(dg_ctx* h, const float* host) {
  for (int i = 0; i < NN_NPARAM; ++i)
    if (!std::isfinite(host[i])) return DG_ERR_INVALID_ARG;
  NNState& nn = h->nn;
  DG_CK(nn.prm.ensure(sizeof(float) * NN_NPARAM));
  DG_CK(nn.m.ensure(sizeof(float) * NN_NPARAM));
  DG_CK(nn.v.ensure(sizeof(float) * NN_NPARAM));
  DG_CK(nn.grad.ensure(sizeof(float) * NN_NPARAM));
  DG_CK(cudaMemcpy(nn.prm.p, host, sizeof(float) * NN_NPARAM, cudaMemcpyHostToDevice));
  DG_CK(cudaMemset(nn.m.p, 0, sizeof(float) * NN_NPARAM));
  DG_CK(cudaMemset(nn.v.p, 0, sizeof(float) * NN_NPARAM));
  nn.step = 0;
  nn.bf16_ok = false;
  nn.have = true;
  nn.save_ne = -1;
  return DG_OK;
}

int nn_load_file(dg_ctx* h, const char* path) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    h->err = std::string("learned guess: cannot open weights file ") + path;
    return DG_ERR_INVALID_ARG;
  }
  char magic[4];
  int32_t hdr[3];
  std::vector<float> prm(NN_NPARAM);
  const bool ok = std::fread(magic, 1, 4, f) == 4 && std::fread(hdr, 4, 3, f) == 3 &&
                  std::memcmp(magic, "DGNN", 4) == 0 && hdr[0] == 1 && hdr[1] == NN_NPARAM &&
                  std::fread(prm.data(), 4, NN_NPARAM, f) == (size_t)NN_NPARAM;
  std::fclose(f);
  if (!ok) {
    h->err = std::string("learned guess: malformed weights file ") + path;
    return DG_ERR_INVALID_ARG;
  }
  if (hdr[2] != h->mesh.p) {
    h->err = "learned guess: weights were trained for another degree p";
    return DG_ERR_INVALID_ARG;
  }
  if (h->levels[0].op.n1 > NN_MAXN1) return DG_ERR_UNSUPPORTED;
  return nn_set(h, prm.data());
}

// activations and input/output buffers for ne elements
static int nn_ensure_io(dg_ctx* h, long long ne, bool io, bool save) {
  const long long npe = (long long)h->levels[0].op.n1 * h->levels[0].op.n1 * h->levels[0].op.n1;
  NNState& nn = h->nn;
  if (io) {
    DG_CK(nn.in.ensure(sizeof(float) * 2 * npe * ne));
    DG_CK(nn.out.ensure(sizeof(float) * 2 * npe * ne));
  }
  if (save) {
    DG_CK(nn.a1.ensure(2ull * 32 * npe * ne));
    DG_CK(nn.a2.ensure(2ull * 32 * npe * ne));
  }
  return DG_OK;
}

// x_c (FP32, w32.x) of the active sources: two V-cycles on the first degree-1
// level l1, applied to the restricted right-hand side, then prolongated level
// by level to the fine level. The restricted right-hand side carries the
// boundary data with the penalty of level l1 (the Nitsche lift in b has the
// fine penalty, 16x that of degree 1 when p = 7; restricted as it is, it would
// impose about 16 g on the coarse boundary): b_c = b + lift_{sigma_l1 - sigma}(g),
// formed in r64 (sources 0..nsrc-1). Sets w32.r = (float) b; uses w32.z, w32.p
// and w32.q as temporaries.
static int coarse_guess(dg_ctx* h, int nsrc, const int* dact, int nact, cudaStream_t s) {
  PrecWork<float>& w = h->w32;
  int l1 = 0;
  while (l1 < h->nlev - 1 && h->levels[l1].op.p > 1) ++l1;
  const long long Nq = h->Nq;
  DG_CK((launch_convert<float, double>(w.r.as<float>(), h->b64.as<double>(), Nq, dact, nact, 1.0, 0, s)));
  const float* src0 = w.r.as<float>();
  if (l1 > 0) {
    if (!h->dlift_op.p) {
      LevelOp D = h->levels[0].op;
      for (int d = 0; d < 3; ++d) {
        const double ds = h->levels[l1].op.ax[d].sigma - D.ax[d].sigma;
        for (int a = 0; a < D.n1; ++a) {
          D.ax[d].lift[0][a] = ds * D.tl[a];
          D.ax[d].lift[1][a] = ds * D.tr[a];
        }
      }
      DeviceWideGuard guard;
      DG_CK(h->dlift_op.ensure(sizeof(LevelOp)));
      DG_CK(cudaMemcpy(h->dlift_op.p, &D, sizeof(LevelOp), cudaMemcpyHostToDevice));
    }
    double* bc = h->r64.as<double>();
    DG_CK((launch_convert<double, double>(bc, h->b64.as<double>(), Nq, dact, nact, 1.0, 0, s)));
    if (bc_fp32(h))
      DG_CK(launch_lift<float>(h->levels[0].op, h->dlift_op.as<LevelOp>(), h->g32.as<float>(), bc, nsrc, h->nface, s));
    else
      DG_CK(launch_lift<double>(h->levels[0].op, h->dlift_op.as<LevelOp>(), h->g.as<double>(), bc, nsrc, h->nface, s));
    DG_CK((launch_convert<float, double>(w.z.as<float>(), bc, Nq, dact, nact, 1.0, 0, s)));
    src0 = w.z.as<float>();
  }
  for (int l = 0; l < l1; ++l) {
    const float* src = l == 0 ? src0 : w.lev[l].b.as<float>();
    DG_CK(launch_restrict<float>(h->levels[l].tr, h->levels[l].dtr, h->levels[l].op, h->levels[l + 1].op, src,
                                 w.lev[l + 1].b.as<float>(), dact, nact, s));
  }
  float* bl = l1 == 0 ? w.r.as<float>() : w.lev[l1].b.as<float>();
  float* xl = l1 == 0 ? w.x.as<float>() : w.lev[l1].x.as<float>();
  MG<float> mg{h, &w, dact, nact, s};
  DG_RET(mg.vcycle(l1, bl, xl));
  if (l1 < h->nlev - 1) {  // the coarsest level is solved exactly by the first cycle
    const Level& L = h->levels[l1];
    float* t = w.p.as<float>();
    float* u = w.q.as<float>();
    DG_CK(launch_apply<float>(L.op, L.dop, 1, xl, t, bl, dact, nact, s));
    DG_RET(mg.vcycle(l1, t, u));
    DG_CK((launch_convert<float, float>(xl, u, L.op.Nq, dact, nact, 1.0, 1, s)));
  }
  for (int l = l1 - 1; l >= 0; --l) {
    float* dst = l == 0 ? w.x.as<float>() : w.lev[l].x.as<float>();
    DG_CK(launch_zero<float>(dst, h->levels[l].op.Nq, dact, nact, s));
    DG_CK(launch_prolong_add<float>(h->levels[l].tr, h->levels[l].dtr, h->levels[l].op, h->levels[l + 1].op,
                                    w.lev[l + 1].x.as<float>(), dst, dact, nact, s));
  }
  return DG_OK;
}


// network guess of the sources act[c0..c0+nc) (device list dact + c0) into x0
template <typename T>
static int nn_apply_chunk(dg_ctx* h, const int* dact_c, int nc, T* x0, bool save, cudaStream_t s) {
  const LevelOp& F = h->levels[0].op;
  const long long Nq = h->Nq;
  const long long ne = (long long)nc * F.E;
  count_launch();
  k_guess_features<<<flat_grid(nc * Nq), 256, 0, s>>>(h->w32.r.as<float>(), h->w32.x.as<float>(), scal(h, S_G1),
                                                       scal(h, S_G3), h->levels[0].dop, dact_c, nc, Nq,
                                                       h->nn.in.as<float>());
  DG_CK(cudaGetLastError());
  DG_CK(nn_forward(F.n1, h->nn.prm.as<float>(), h->nn.W2t.p, h->nn.in.as<float>(), h->nn.out.as<float>(),
                   save ? h->nn.a1.p : nullptr, save ? h->nn.a2.p : nullptr, ne, s));
  count_launch();
  k_guess_combine<T><<<flat_grid(nc * Nq), 256, 0, s>>>(h->w32.x.as<float>(), h->nn.out.as<float>(), scal(h, S_G3),
                                                        dact_c, nc, Nq, x0);
  DG_CK(cudaGetLastError());
  return DG_OK;
}

// x <- Chebyshev smoothing of A x = b32 on the fine level (the V-cycle's
// pre-smoother, Sec. 6.4), starting from x
static int smooth_guess(dg_ctx* h, float* x, const int* dact, int nact, cudaStream_t s) {
  if (h->nlev < 2) return DG_OK;
  MG<float> mg{h, &h->w32, dact, nact, s};
  return mg.cheb(0, h->w32.r.as<float>(), x, false, false);
}

// FP32 guess of the active sources (b64 formed): x_c (w32.x) scaled by its
// energy-optimal factor b^T x_c / x_c^T A x_c, b32 (w32.r), the network's
// correction y (if use_net), then (if smooth) the fine-level Chebyshev
// smoother; the guess in w32.q, w32.z and w32.p are scratch. With save, all
// sources form one network batch and the activations are kept.
static int guess_fp32(dg_ctx* h, int nsrc, const int* dact, int nact, bool use_net, bool save, bool smooth,
                      cudaStream_t s) {
  PrecWork<float>& w = h->w32;
  const long long Nq = h->Nq;
  const LevelOp& F = h->levels[0].op;
  double* part = h->part.as<double>();
  DG_RET(coarse_guess(h, nsrc, dact, nact, s));
  DG_CK(launch_apply<float>(F, h->levels[0].dop, 0, w.x.as<float>(), w.z.as<float>(), nullptr, dact, nact, s));
  DG_CK(launch_dot<float>(w.x.as<float>(), w.r.as<float>(), nullptr, scal(h, S_G1), part, Nq, dact, nact, s));
  DG_CK(launch_dot<float>(w.x.as<float>(), w.z.as<float>(), nullptr, scal(h, S_G2), part, Nq, dact, nact, s));
  count_launch();
  k_scale_ratio<<<flat_grid(nact * Nq), 256, 0, s>>>(w.x.as<float>(), scal(h, S_G1), scal(h, S_G2), dact, nact, Nq);
  DG_CK(cudaGetLastError());
  if (use_net) {
    DG_RET(nn_bf16(h, s));
    // per-source input scales: sb = max |b / m| (S_G1), sx = max |x_c| (S_G3)
    DG_CK(cudaMemsetAsync(scal(h, S_G1), 0, sizeof(double) * h->cap, s));
    DG_CK(cudaMemsetAsync(scal(h, S_G3), 0, sizeof(double) * h->cap, s));
    count_launch(2);
    const dim3 mgrid((unsigned)std::max(1LL, std::min((Nq + 255) / 256, 152LL * 8 / nact + 1)), (unsigned)nact);
    k_maxabs<<<mgrid, 256, 0, s>>>(w.r.as<float>(), h->levels[0].dop, 1, dact, Nq, scal(h, S_G1));
    k_maxabs<<<mgrid, 256, 0, s>>>(w.x.as<float>(), h->levels[0].dop, 0, dact, Nq, scal(h, S_G3));
    DG_CK(cudaGetLastError());
    // network batches of at most ~512 MB of input + output (one batch when saving)
    const int chunk =
        save ? nact : (int)std::max(1LL, std::min<long long>(nact, (512LL << 20) / (16 * Nq)));
    DG_RET(nn_ensure_io(h, (long long)chunk * F.E, true, save));
    for (int c0 = 0; c0 < nact; c0 += chunk)
      DG_RET(nn_apply_chunk<float>(h, dact + c0, std::min(chunk, nact - c0), w.q.as<float>(), save, s));
  } else {
    DG_CK((launch_convert<float, float>(w.q.as<float>(), w.x.as<float>(), Nq, dact, nact, 1.0, 0, s)));
  }
  if (smooth) DG_RET(smooth_guess(h, w.q.as<float>(), dact, nact, s));
  return DG_OK;
}

int learned_guess(dg_ctx* h, int nsrc, const std::vector<int>& act, const std::vector<double>& bnorm2, bool use_net,
                  std::vector<double>& rel, std::vector<int>& fb, cudaStream_t s) {
  if (act.empty()) return DG_OK;
  if (use_net) DG_RET(nn_require(h));
  const long long Nq = h->Nq;
  const int nact = (int)act.size();
  DG_RET(upload_act(h, act, s));
  const int* dact = h->act.as<int>();
  double* x64 = h->x64.as<double>();
  double* r64 = h->r64.as<double>();
  const double* b64 = h->b64.as<double>();
  double* part = h->part.as<double>();
  DG_RET(guess_fp32(h, nsrc, dact, nact, use_net, false, true, s));
  DG_CK((launch_convert<double, float>(x64, h->w32.q.as<float>(), Nq, dact, nact, 1.0, 0, s)));
  // energy-optimal scaling alpha = b^T x0 / x0^T A x0, residual r = b - alpha A x0 (FP64)
  DG_CK(launch_apply<double>(h->levels[0].op, h->levels[0].dop, 0, x64, r64, nullptr, dact, nact, s));
  DG_CK(launch_dot<double>(x64, b64, nullptr, scal(h, S_G1), part, Nq, dact, nact, s));
  DG_CK(launch_dot<double>(x64, r64, nullptr, scal(h, S_G2), part, Nq, dact, nact, s));
  count_launch();
  k_guess_scale<<<flat_grid(nact * Nq), 256, 0, s>>>(x64, r64, b64, scal(h, S_G1), scal(h, S_G2), dact, nact, Nq);
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot<double>(r64, r64, nullptr, scal(h, S_RR), part, Nq, dact, nact, s));
  std::vector<double> rr(h->cap);
  DG_CK(cudaMemcpyAsync(rr.data(), scal(h, S_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  std::vector<int> rej;
  for (int k : act) {
    const double r = bnorm2[k] > 0 ? std::sqrt(std::max(rr[k], 0.0) / bnorm2[k]) : 0.0;
    if (!(r < 1.0)) {
      rej.push_back(k);
      rel[k] = bnorm2[k] > 0 ? 1.0 : 0.0;
      fb[k] = 1;
    } else {
      rel[k] = r;
      fb[k] = 0;
    }
  }
  if (!rej.empty()) {
    DG_RET(upload_act(h, rej, s));
    DG_CK(launch_zero<double>(x64, Nq, h->act.as<int>(), (int)rej.size(), s));
    DG_CK((launch_convert<double, double>(r64, b64, Nq, h->act.as<int>(), (int)rej.size(), 1.0, 0, s)));
  }
  return DG_OK;
}

// workspaces of a network call on B sources (FP32 multigrid work, right-hand sides)
static int nn_prepare(dg_ctx* h, int B) {
  DG_RET(ensure_common(h, B));
  DG_RET(ensure_prec<float>(h, h->w32, B));
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_nn_set_params(dg_handle h, const float* params_host) {
  if (!h || !params_host) return DG_ERR_INVALID_ARG;
  DeviceWideGuard guard;
  if (h->levels[0].op.n1 > NN_MAXN1) return DG_ERR_UNSUPPORTED;
  return nn_set(h, params_host);
}

int dg_nn_get_params(dg_handle h, float* params_host) {
  if (!h || !params_host || !h->nn.have) return DG_ERR_INVALID_ARG;
  DeviceWideGuard guard;
  DG_CK(cudaDeviceSynchronize());
  DG_CK(cudaMemcpy(params_host, h->nn.prm.p, sizeof(float) * NN_NPARAM, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int dg_nn_forward(dg_handle h, const float* in_dev, float* out_dev, int64_t n_elem, int32_t save_act, void* stream) {
  if (!h || n_elem < 0 || (n_elem > 0 && (!in_dev || !out_dev))) return DG_ERR_INVALID_ARG;
  DG_RET(nn_require(h));
  cudaStream_t s = (cudaStream_t)stream;
  DG_RET(nn_bf16(h, s));
  if (save_act) {
    DG_RET(nn_ensure_io(h, std::max<int64_t>(n_elem, 1), false, true));
    h->nn.save_ne = n_elem;
  }
  if (n_elem > 0)
    DG_CK(nn_forward(h->levels[0].op.n1, h->nn.prm.as<float>(), h->nn.W2t.p, in_dev, out_dev,
                     save_act ? h->nn.a1.p : nullptr, save_act ? h->nn.a2.p : nullptr, n_elem, s));
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_nn_backward(dg_handle h, const float* in_dev, const float* gout_dev, float* grad_dev, int64_t n_elem,
                   void* stream) {
  if (!h || !in_dev || !gout_dev || !grad_dev || n_elem < 1) return DG_ERR_INVALID_ARG;
  DG_RET(nn_require(h));
  if (h->nn.save_ne != n_elem) {
    h->err = "dg_nn_backward: no saved activations of this input size";
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DG_RET(nn_bf16(h, s));
  const int n1 = h->levels[0].op.n1;
  const int nblk = nn_backward_blocks(n1, n_elem);
  if (nblk < 1) return DG_ERR_CUDA;
  DG_CK(h->nn.part.ensure(sizeof(float) * (size_t)nblk * NN_NPARAM));
  DG_CK(nn_backward(n1, h->nn.prm.as<float>(), h->nn.W2o.p, in_dev, h->nn.a1.p, h->nn.a2.p, gout_dev,
                    h->nn.part.as<float>(), grad_dev, n_elem, s));
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_nn_adam(dg_handle h, const float* grad_dev, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!h || !grad_dev || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return DG_ERR_INVALID_ARG;
  DG_RET(nn_require(h));
  cudaStream_t s = (cudaStream_t)stream;
  h->nn.step += 1;
  DG_CK(nn_adam(h->nn.prm.as<float>(), grad_dev, h->nn.m.as<float>(), h->nn.v.as<float>(), lr, beta1, beta2, eps,
                h->nn.step, s));
  h->nn.bf16_ok = false;
  DG_RET(nn_bf16(h, s));
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_nn_train_step(dg_handle h, const double* f_dev, const double* v_dev, int64_t B, float lr, double* loss_host,
                     void* stream) {
  if (!h || !f_dev || !v_dev || B < 1 || B > 4096 || !(lr >= 0.f)) return DG_ERR_INVALID_ARG;
  DG_RET(nn_require(h));
  cudaStream_t us = (cudaStream_t)stream;
  DG_CK(cudaEventRecord(h->ev_in, us));
  DG_CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  cudaStream_t s = h->ws;
  const int nb = (int)B;
  const long long Nq = h->Nq;
  const LevelOp& F = h->levels[0].op;
  DG_RET(nn_prepare(h, nb));
  std::vector<int> finite;
  DG_RET(check_finite(h, f_dev, nb, finite, s));
  for (int k = 0; k < nb; ++k)
    if (!finite[k]) return DG_ERR_NONFINITE;
  DG_RET(form_rhs(h, f_dev, nb, s));
  std::vector<int> all(nb);
  for (int k = 0; k < nb; ++k) all[k] = k;
  DG_RET(upload_act(h, all, s));
  const int* dact = h->act.as<int>();
  double* part = h->part.as<double>();
  PrecWork<float>& w = h->w32;
  const long long ne = (long long)nb * F.E;
  // network guess before smoothing (activations kept): y (w.q), x_c (w.x)
  DG_RET(guess_fp32(h, nb, dact, nb, true, true, false, s));
  h->nn.save_ne = -1;  // the buffers now hold this step's activations, not a dg_nn_forward call's
  DG_CK(launch_dot<double>(v_dev, v_dev, h->d_W.as<double>(), scal(h, S_G2), part, Nq, dact, nb, s));
  count_launch();
  k_train_gout<<<flat_grid(nb * Nq), 256, 0, s>>>(w.x.as<float>(), w.q.as<float>(), v_dev, h->levels[0].dop,
                                                   scal(h, S_G3), scal(h, S_G2), nb, Nq, h->nn.out.as<float>(),
                                                   w.p.as<float>());
  DG_CK(cudaGetLastError());
  DG_CK(launch_dot<float>(w.p.as<float>(), w.p.as<float>(), h->d_W.as<double>(), scal(h, S_RR), part, Nq, dact, nb,
                          s));
  const int nblk = nn_backward_blocks(F.n1, ne);
  if (nblk < 1) return DG_ERR_CUDA;
  DG_CK(h->nn.part.ensure(sizeof(float) * (size_t)nblk * NN_NPARAM));
  DG_CK(nn_backward(F.n1, h->nn.prm.as<float>(), h->nn.W2o.p, h->nn.in.as<float>(), h->nn.a1.p, h->nn.a2.p,
                    h->nn.out.as<float>(), h->nn.part.as<float>(), h->nn.grad.as<float>(), ne, s));
  h->nn.step += 1;
  DG_CK(nn_adam(h->nn.prm.as<float>(), h->nn.grad.as<float>(), h->nn.m.as<float>(), h->nn.v.as<float>(), lr, 0.9f,
                0.999f, 1e-8f, h->nn.step, s));
  h->nn.bf16_ok = false;
  DG_RET(nn_bf16(h, s));
  std::vector<double> ee(h->cap), nv(h->cap);
  DG_CK(cudaMemcpyAsync(ee.data(), scal(h, S_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaMemcpyAsync(nv.data(), scal(h, S_G2), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  DG_CK(cudaEventRecord(h->ev_out, s));
  DG_CK(cudaStreamWaitEvent(us, h->ev_out, 0));
  if (loss_host) {
    double L = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double lk = nv[k] > 0 ? ee[k] / nv[k] : 0.0;
      L += lk / nb;
      loss_host[1 + k] = lk;
    }
    loss_host[0] = L;
  }
  return DG_OK;
}

int dg_nn_guess(dg_handle h, const double* f_dev, int64_t B, int32_t use_net, double* x0_dev, double* rel_host,
                void* stream) {
  if (!h || B < 0 || (B > 0 && (!f_dev || !x0_dev))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  if (use_net) DG_RET(nn_require(h));
  cudaStream_t us = (cudaStream_t)stream;
  DG_CK(cudaEventRecord(h->ev_in, us));
  DG_CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  cudaStream_t s = h->ws;
  const int nb = (int)B;
  const long long Nq = h->Nq;
  DG_RET(nn_prepare(h, nb));
  std::vector<int> finite;
  DG_RET(check_finite(h, f_dev, nb, finite, s));
  for (int k = 0; k < nb; ++k)
    if (!finite[k]) return DG_ERR_NONFINITE;
  DG_RET(form_rhs(h, f_dev, nb, s));
  std::vector<int> all(nb);
  for (int k = 0; k < nb; ++k) all[k] = k;
  DG_RET(upload_act(h, all, s));
  DG_CK(launch_dot<double>(h->b64.as<double>(), h->b64.as<double>(), nullptr, scal(h, S_BN), h->part.as<double>(),
                           Nq, h->act.as<int>(), nb, s));
  std::vector<double> bn(h->cap, 0.0), rel(h->cap, 1.0);
  std::vector<int> fb(h->cap, 0);
  DG_CK(cudaMemcpyAsync(bn.data(), scal(h, S_BN), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  DG_RET(learned_guess(h, nb, all, bn, use_net != 0, rel, fb, s));
  DG_CK(cudaMemcpyAsync(x0_dev, h->x64.p, sizeof(double) * Nq * nb, cudaMemcpyDeviceToDevice, s));
  DG_CK(cudaStreamSynchronize(s));
  DG_CK(cudaEventRecord(h->ev_out, s));
  DG_CK(cudaStreamWaitEvent(us, h->ev_out, 0));
  if (rel_host)
    for (int k = 0; k < nb; ++k) rel_host[k] = rel[k];
  return DG_OK;
}

}  // extern "C"
