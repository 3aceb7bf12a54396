// Host driver and C ABI: hp-multigrid-preconditioned CG (Sec. 6.4) over a
// batch of sources, Dirichlet data (Sec. 6.3), the exchange build
// (Sec. 6.1.2, eq. fock_exchange) and the entry points of dg_poisson.h.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <shared_mutex>
#include <vector>

#include "dg_ctx.h"
#include "dg_mg.h"

namespace dg {

static std::shared_mutex g_capture_mu;
static thread_local int t_device_wide = 0;

DeviceWideGuard::DeviceWideGuard() {
  if (t_device_wide++ == 0) g_capture_mu.lock();
}
DeviceWideGuard::~DeviceWideGuard() {
  if (--t_device_wide == 0) g_capture_mu.unlock();
}
CaptureGuard::CaptureGuard() : shared_(t_device_wide == 0) {
  if (shared_) g_capture_mu.lock_shared();
}
CaptureGuard::~CaptureGuard() {
  if (shared_) g_capture_mu.unlock_shared();
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
template <typename T>
int ensure_prec(dg_ctx* h, PrecWork<T>& w, int cap) {
  if (w.cap >= cap && !w.lev.empty()) return DG_OK;
  DeviceWideGuard guard;
  ++h->buf_gen;
  w.lev.resize(h->nlev);
  for (int l = 0; l < h->nlev; ++l) {
    const long long N = h->levels[l].op.Nq;
    LevelWork& L = w.lev[l];
    if (l > 0) {
      DG_CK(L.x.ensure(sizeof(T) * N * cap));
      DG_CK(L.b.ensure(sizeof(T) * N * cap));
    }
    DG_CK(L.res.ensure(sizeof(T) * N * cap));
    DG_CK(L.d.ensure(sizeof(T) * N * cap));
    if (h->opts.smoother == DG_SMOOTH_SCHWARZ && l + 1 < h->nlev) {
      const long long mp = h->levels[l].op.n1 + 2;
      DG_CK(L.zp.ensure(sizeof(T) * (size_t)h->levels[l].op.E * mp * mp * mp * cap));
    }
    if (!L.invD.p) {
      DG_CK(L.invD.ensure(sizeof(T) * N));
      DG_CK(launch_inv_diag<T>(h->levels[l].op, h->levels[l].dop, L.invD.as<T>(), 0));
    }
  }
  const long long N = h->Nq;
  DG_CK(w.x.ensure(sizeof(T) * N * cap));
  DG_CK(w.r.ensure(sizeof(T) * N * cap));
  DG_CK(w.z.ensure(sizeof(T) * N * cap));
  DG_CK(w.p.ensure(sizeof(T) * N * cap));
  DG_CK(w.q.ensure(sizeof(T) * N * cap));
  w.cap = cap;
  DG_CK(cudaDeviceSynchronize());
  return DG_OK;
}

template int ensure_prec<double>(dg_ctx*, PrecWork<double>&, int);
template int ensure_prec<float>(dg_ctx*, PrecWork<float>&, int);

// layout of the device-side loop state: done[cap], iters[cap], counter, limit, then
// (8-byte aligned) tol[cap], relres[cap]
static size_t loop_ints(int cap) { return ((size_t)2 * cap + 2 + 1) / 2 * 2; }
size_t loop_bytes(int cap) { return sizeof(int) * loop_ints(cap) + sizeof(double) * 2 * (size_t)cap; }
static int* loop_done(dg_ctx* h) { return h->loop.as<int>(); }
static int* loop_iters(dg_ctx* h) { return h->loop.as<int>() + h->cap; }
static int* loop_counter(dg_ctx* h) { return h->loop.as<int>() + 2 * h->cap; }
static int* loop_limit(dg_ctx* h) { return h->loop.as<int>() + 2 * h->cap + 1; }
static double* loop_tol(dg_ctx* h) { return (double*)(h->loop.as<int>() + loop_ints(h->cap)); }
static double* loop_relres(dg_ctx* h) { return loop_tol(h) + h->cap; }

int ensure_common(dg_ctx* h, int cap) {
  if (h->cap >= cap) return DG_OK;
  DeviceWideGuard guard;
  ++h->buf_gen;
  const long long N = h->Nq;
  DG_CK(h->f64.ensure(sizeof(double) * N * cap));
  DG_CK(h->b64.ensure(sizeof(double) * N * cap));
  DG_CK(h->x64.ensure(sizeof(double) * N * cap));
  DG_CK(h->r64.ensure(sizeof(double) * N * cap));
  DG_CK(h->part.ensure(sizeof(double) * 304 * cap));
  DG_CK(h->scal.ensure(sizeof(double) * S_NSLOT * cap));
  DG_CK(h->act.ensure(sizeof(int) * cap));
  h->act_host.clear();
  DG_CK(h->flags.ensure(sizeof(int) * cap));
  DG_CK(h->loop.ensure(loop_bytes(cap)));
  DG_CK(h->pidx.ensure(sizeof(int) * 2 * cap));
  DG_CK(h->g.ensure(sizeof(double) * h->nface * cap));
  h->cap = cap;
  return DG_OK;
}

template <typename T>
static int ensure_bc_work(dg_ctx* h, int nsrc, int NG, BcAxisTables* bct, DevBuf& flex, DevBuf& T1, DevBuf& T2) {
  const long long N = h->Nq;
  DG_CK(flex.ensure(sizeof(T) * N * nsrc));
  long long maxface = 0;
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    maxface = std::max(maxface, (long long)bct[t1].L * bct[t2].L);
  }
  const size_t tb = sizeof(T) * 2 * (size_t)NG * maxface * nsrc;
  DG_CK(T1.ensure(tb));
  DG_CK(T2.ensure(tb));
  if (sizeof(T) == 4) DG_CK(h->gemm_ws.ensure(sizeof(float) * (16LL << 20)));  // 64 MB of split-K partials
  return DG_OK;
}

static void account(dg_ctx* h) {
  long long b = 0;
  auto add = [&](const DevBuf& x) { b += (long long)x.bytes; };
  for (auto* w : {&h->f64, &h->b64, &h->x64, &h->r64, &h->flex, &h->T1, &h->T2, &h->g, &h->part, &h->scal,
                  &h->flex32, &h->T1_32, &h->T2_32, &h->g32,
                  &h->act, &h->flags, &h->pidx, &h->Wacc, &h->kpart, &h->Kdev, &h->coarse_inv, &h->d_W, &h->d_xq,
                  &h->d_axn})
    add(*w);
  for (auto& L : h->w64.lev) {
    add(L.x); add(L.b); add(L.res); add(L.d); add(L.invD); add(L.z); add(L.zp);
  }
  for (auto& L : h->w32.lev) {
    add(L.x); add(L.b); add(L.res); add(L.d); add(L.invD); add(L.z); add(L.zp);
  }
  for (auto& L : h->levels) add(L.sw_tabs);
  for (auto* w : {&h->w64.x, &h->w64.r, &h->w64.z, &h->w64.p, &h->w64.q}) add(*w);
  for (auto* w : {&h->w32.x, &h->w32.r, &h->w32.z, &h->w32.p, &h->w32.q}) add(*w);
  for (int d = 0; d < 3; ++d) {
    add(h->bct[d].gn); add(h->bct[d].G); add(h->bct[d].Gs);
    add(h->bct32[d].gn); add(h->bct32[d].G); add(h->bct32[d].Gs);
  }
  h->ws_bytes = b;
}

// device per-rhs scalar update: out = num / den (0 and a breakdown flag when den <= 0 or not finite)
__global__ void k_ratio(const double* num, const double* den, double* out, const int* act, int nact, int* flags,
                        int check) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nact) return;
  const int r = act[k];
  const double dn = den[r];
  if (!(dn > 0.0) || !isfinite(dn) || !isfinite(num[r])) {
    out[r] = 0.0;
    if (check) flags[r] |= 2;
  } else {
    out[r] = num[r] / dn;
  }
}

__global__ void k_copy_slot(const double* src, double* dst, const int* act, int nact) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nact) dst[act[k]] = src[act[k]];
}

// k_ratio for the device-side loop: a source marked done takes a zero step
__global__ void k_ratio_masked(const double* num, const double* den, double* out, const int* act, int nact,
                               int* flags, int check, const int* done) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nact) return;
  const int r = act[k];
  if (done[r]) {
    out[r] = 0.0;
    return;
  }
  const double dn = den[r];
  if (!(dn > 0.0) || !isfinite(dn) || !isfinite(num[r])) {
    out[r] = 0.0;
    if (check) flags[r] |= 2;
  } else {
    out[r] = num[r] / dn;
  }
}

// Device-side convergence test after the operator phase of an iteration (one
// block): every source not yet done records the iteration and its relative
// residual and is done once that meets its tolerance (or is not finite). The
// loop goes on while no source became done in this test, some are left and the
// iteration limit is not reached.
__global__ void k_pcg_check(const double* rr, const double* bn, const double* tol, const int* act, int nact,
                            int* done, int* iters, double* relres, int* counter, const int* limit,
                            cudaGraphConditionalHandle hnd) {
  const int it = *counter + 1;
  const int maxit = *limit;
  int left = 0, now = 0;
  for (int k = threadIdx.x; k < nact; k += blockDim.x) {
    const int r = act[k];
    if (done[r]) continue;
    iters[r] = it;
    const double rel = sqrt(fmax(rr[r], 0.0) / bn[r]);
    relres[r] = rel;
    if (!(rel <= tol[r]) && isfinite(rel)) {
      left = 1;
    } else {
      done[r] = 1;
      now = 1;
    }
  }
  left = __syncthreads_or(left);
  now = __syncthreads_or(now);
  if (threadIdx.x == 0) {
    *counter = it;
    cudaGraphSetConditional(hnd, (left && !now && it < maxit) ? 1u : 0u);
  }
}

// Active source list on the device; re-uploaded only when it changes.
int upload_act(dg_ctx* h, const std::vector<int>& a, cudaStream_t s) {
  if (a.empty()) return DG_OK;
  if (h->act_host == a) return DG_OK;
  DG_CK(cudaMemcpyAsync(h->act.p, a.data(), sizeof(int) * a.size(), cudaMemcpyHostToDevice, s));
  DG_CK(cudaStreamSynchronize(s));
  h->act_host = a;
  return DG_OK;
}

// Runs `body` (kernel launches only) on stream s, through a CUDA graph captured
// on first use and replayed while the active source count and the workspace
// buffers stay the same.
template <typename F>
static int run_phase(dg_ctx* h, PhaseGraph& g, int nact, cudaStream_t s, F&& body) {
  if (!h->use_graphs || s == nullptr) return body();
  if (g.exec && g.nact == nact && g.gen == h->buf_gen) {
    DG_CK(cudaGraphLaunch(g.exec, s));
    count_launch((int)g.nkernels);
    return DG_OK;
  }
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  CaptureGuard cap_guard;  // no device-wide operation of another thread during the capture
  const long long l0 = t_launch_count;
  DG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int rc = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  // kernels counted while capturing did not run; they are counted at replay
  const long long nk = uncount_captured(l0);
  if (rc != DG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  DG_CK(e);
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  DG_CK(ei);
  g.nact = nact;
  g.gen = h->buf_gen;
  g.nkernels = nk;
  DG_CK(cudaGraphLaunch(g.exec, s));
  count_launch((int)nk);
  return DG_OK;
}

// Preconditioned CG in precision T on the fine level for the sources in
// `act0`: solves A x = r (r overwritten by the residual) starting from x = 0
// until ||r||_2 <= tol * ||r_0||_2 or maxit iterations. iters[k] receives the
// iterations used by each source; flags (device) collect breakdowns. Each
// iteration is two device-only phases (operator + updates; preconditioner +
// direction update), replayed as CUDA graphs, and one host read of ||r||^2.
template <typename T>
static int pcg(dg_ctx* h, PrecWork<T>& w, const std::vector<int>& act0, const std::vector<double>& tol, int maxit,
               cudaStream_t s, std::vector<int>& iters, std::vector<double>& relres) {
  const long long Nq = h->Nq;
  T* x = w.x.template as<T>();
  T* r = w.r.template as<T>();
  T* z = w.z.template as<T>();
  T* p = w.p.template as<T>();
  T* q = w.q.template as<T>();
  double* part = h->part.as<double>();
  int* flags = h->flags.as<int>();
  std::vector<int> act = act0;
  int nact = (int)act.size();
  if (nact == 0) return DG_OK;
  DG_RET(upload_act(h, act, s));
  const int* dact = h->act.as<int>();
  MG<T> mg{h, &w, dact, nact, s};
  DG_CK(launch_zero<T>(x, Nq, dact, nact, s));
  DG_CK(launch_dot<T>(r, r, nullptr, scal(h, S_BN), part, Nq, dact, nact, s));
  DG_RET(mg.vcycle(0, r, z));
  DG_CK((launch_convert<T, T>(p, z, Nq, dact, nact, 1.0, 0, s)));
  DG_CK(launch_dot<T>(r, z, nullptr, scal(h, S_RZ), part, Nq, dact, nact, s));
  std::vector<double> bn(h->cap, 0.0), rr(h->cap, 0.0);
  DG_CK(cudaMemcpyAsync(bn.data(), scal(h, S_BN), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  for (int k : act) {
    iters[k] = 0;
    relres[k] = bn[k] > 0 ? 1.0 : 0.0;
  }
  // sources with a zero right-hand side are done at x = 0
  {
    std::vector<int> a2;
    for (int k : act)
      if (bn[k] > 0.0) a2.push_back(k);
    if (a2.size() != act.size()) {
      act = a2;
      nact = (int)act.size();
      if (nact == 0) return DG_OK;
      DG_RET(upload_act(h, act, s));
      mg.nact = nact;
    }
  }
  auto phaseA = [&]() -> int {
    DG_CK(launch_apply<T>(h->levels[0].op, h->levels[0].dop, 0, p, q, nullptr, dact, nact, s));
    DG_CK(launch_dot<T>(p, q, nullptr, scal(h, S_PQ), part, Nq, dact, nact, s));
    count_launch();
    k_ratio<<<(nact + 127) / 128, 128, 0, s>>>(scal(h, S_RZ), scal(h, S_PQ), scal(h, S_AL), dact, nact, flags, 1);
    DG_CK(launch_cg_xr<T>(x, r, p, q, scal(h, S_AL), Nq, dact, nact, s));
    DG_CK(launch_dot<T>(r, r, nullptr, scal(h, S_RR), part, Nq, dact, nact, s));
    return DG_OK;
  };
  auto phaseB = [&]() -> int {
    DG_RET(mg.vcycle(0, r, z));
    DG_CK(launch_dot<T>(r, z, nullptr, scal(h, S_RZN), part, Nq, dact, nact, s));
    count_launch();
    k_ratio<<<(nact + 127) / 128, 128, 0, s>>>(scal(h, S_RZN), scal(h, S_RZ), scal(h, S_BE), dact, nact, flags, 0);
    count_launch();
    k_copy_slot<<<(nact + 127) / 128, 128, 0, s>>>(scal(h, S_RZN), scal(h, S_RZ), dact, nact);
    DG_CK(launch_cg_p<T>(p, z, scal(h, S_BE), Nq, dact, nact, s));
    return DG_OK;
  };
  // device-side loop: always (1), or (2, the default) where an iteration is
  // short enough for the host round trip to matter (at most 2^24 unknowns in
  // the batch)
  const bool dev_loop =
      h->opts.device_loop == 1 || (h->opts.device_loop == 2 && (long long)Nq * nact <= (1LL << 24));
  if (h->use_graphs && s != nullptr && dev_loop) {
    // iterations in graph launches with a device-side loop: each launch runs
    // until a source converges, then the host drops the converged sources and
    // launches the continuation for the others
    int* done = loop_done(h);
    const std::vector<double> tolv(tol.begin(), tol.begin() + h->cap);
    DG_CK(cudaMemcpyAsync(loop_tol(h), tolv.data(), sizeof(double) * h->cap, cudaMemcpyHostToDevice, s));
    DG_CK(cudaMemsetAsync(done, 0, sizeof(int) * h->cap, s));
    const int lim[2] = {0, maxit};  // counter, iteration limit
    DG_CK(cudaMemcpyAsync(loop_counter(h), lim, sizeof(lim), cudaMemcpyHostToDevice, s));
    auto phaseAm = [&]() -> int {
      DG_CK(launch_apply<T>(h->levels[0].op, h->levels[0].dop, 0, p, q, nullptr, dact, nact, s));
      DG_CK(launch_dot<T>(p, q, nullptr, scal(h, S_PQ), part, Nq, dact, nact, s));
      count_launch();
      k_ratio_masked<<<(nact + 127) / 128, 128, 0, s>>>(scal(h, S_RZ), scal(h, S_PQ), scal(h, S_AL), dact, nact,
                                                         flags, 1, done);
      DG_CK(launch_cg_xr<T>(x, r, p, q, scal(h, S_AL), Nq, dact, nact, s));
      DG_CK(launch_dot<T>(r, r, nullptr, scal(h, S_RR), part, Nq, dact, nact, s));
      return DG_OK;
    };
    auto phaseBm = [&]() -> int {
      DG_RET(mg.vcycle(0, r, z));
      DG_CK(launch_dot<T>(r, z, nullptr, scal(h, S_RZN), part, Nq, dact, nact, s));
      count_launch();
      k_ratio_masked<<<(nact + 127) / 128, 128, 0, s>>>(scal(h, S_RZN), scal(h, S_RZ), scal(h, S_BE), dact, nact,
                                                         flags, 0, done);
      count_launch();
      k_copy_slot<<<(nact + 127) / 128, 128, 0, s>>>(scal(h, S_RZN), scal(h, S_RZ), dact, nact);
      DG_CK(launch_cg_p<T>(p, z, scal(h, S_BE), Nq, dact, nact, s));
      return DG_OK;
    };
    std::vector<int> ibuf(2 * (size_t)h->cap + 1);
    std::vector<double> rel(h->cap);
    for (int variant = 0;; variant = 1) {
      std::unique_ptr<LoopGraph>& slot = w.gL[{variant, nact}];
      if (!slot || slot->gen != h->buf_gen) {
        slot.reset(new LoopGraph());
        LoopGraph& L = *slot;
        CaptureGuard cap_guard;  // no device-wide operation of another thread during the capture
        cudaGraph_t g = nullptr;
        DG_CK(cudaGraphCreate(&g, 0));
        struct GraphOwner {
          cudaGraph_t g;
          ~GraphOwner() {
            if (g) cudaGraphDestroy(g);
          }
        } owner{g};
        cudaGraphConditionalHandle hnd;
        DG_CK(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
        auto check = [&]() -> int {
          count_launch();
          k_pcg_check<<<1, 256, 0, s>>>(scal(h, S_RR), scal(h, S_BN), loop_tol(h), dact, nact, done,
                                        loop_iters(h), loop_relres(h), loop_counter(h), loop_limit(h), hnd);
          DG_CK(cudaGetLastError());
          return DG_OK;
        };
        // before the loop: the first operator phase (variant 0) or the
        // preconditioner phase and the next operator phase (variant 1)
        const long long l0 = t_launch_count;
        DG_CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        int rc = variant == 0 ? DG_OK : phaseBm();
        if (rc == DG_OK) rc = phaseAm();
        if (rc == DG_OK) rc = check();
        std::vector<cudaGraphNode_t> sink;
        {
          cudaStreamCaptureStatus cst;
          const cudaGraphNode_t* deps = nullptr;
          size_t nd = 0;
          if (cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess && deps)
            sink.assign(deps, deps + nd);
        }
        cudaGraph_t g_out = nullptr;
        const cudaError_t e1 = cudaStreamEndCapture(s, &g_out);
        const long long nk_first = uncount_captured(l0);  // counted at replay
        if (rc != DG_OK) {
          slot.reset();
          return rc;
        }
        DG_CK(e1);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        DG_CK(cudaGraphAddNode(&cnode, g, sink.data(), nullptr, sink.size(), &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const long long l1 = t_launch_count;
        DG_CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        rc = phaseBm();
        if (rc == DG_OK) rc = phaseAm();
        if (rc == DG_OK) rc = check();
        cudaGraph_t b_out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &b_out);
        const long long nk_body = uncount_captured(l1);
        if (rc != DG_OK) {
          slot.reset();
          return rc;
        }
        DG_CK(e2);
        DG_CK(cudaGraphInstantiate(&L.exec, g, 0));
        L.gen = h->buf_gen;
        L.nk_first = nk_first;
        L.nk_body = nk_body;
      }
      const int it0 = variant == 0 ? 0 : ibuf[2 * (size_t)h->cap];
      DG_CK(cudaGraphLaunch(slot->exec, s));
      DG_CK(cudaMemcpyAsync(ibuf.data(), h->loop.p, sizeof(int) * ibuf.size(), cudaMemcpyDeviceToHost, s));
      DG_CK(cudaMemcpyAsync(rel.data(), loop_relres(h), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
      DG_CK(cudaStreamSynchronize(s));
      const int nit = ibuf[2 * (size_t)h->cap];
      count_launch((int)(slot->nk_first + (long long)std::max(0, nit - it0 - 1) * slot->nk_body));
      std::vector<int> a2;
      for (int k : act) {
        iters[k] = ibuf[(size_t)h->cap + k];
        relres[k] = rel[k];
        if (!ibuf[k]) a2.push_back(k);
      }
      if (a2.empty() || nit >= maxit) break;
      if (a2.size() != act.size()) {
        act = a2;
        nact = (int)act.size();
        DG_RET(upload_act(h, act, s));
        mg.nact = nact;
      }
    }
    return DG_OK;
  }
  for (int it = 1; it <= maxit; ++it) {
    DG_RET(run_phase(h, w.gA, nact, s, phaseA));
    DG_CK(cudaMemcpyAsync(rr.data(), scal(h, S_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
    std::vector<int> a2;
    for (int k : act) {
      iters[k] = it;
      relres[k] = std::sqrt(std::max(rr[k], 0.0) / bn[k]);
      if (!(relres[k] <= tol[k]) && std::isfinite(relres[k])) a2.push_back(k);
    }
    if (a2.empty()) break;
    if (a2.size() != act.size()) {
      act = a2;
      nact = (int)act.size();
      DG_RET(upload_act(h, act, s));
      mg.nact = nact;
    }
    if (it == maxit) break;
    DG_RET(run_phase(h, w.gB, nact, s, phaseB));
  }
  return DG_OK;
}

// FP64 true residual r64 = b64 - A x64 and its relative norm per source.
static int true_residual(dg_ctx* h, const std::vector<int>& act, const std::vector<double>& bnorm2,
                         std::vector<double>& rel, cudaStream_t s) {
  if (act.empty()) return DG_OK;
  DG_RET(upload_act(h, act, s));
  const int* dact = h->act.as<int>();
  const int nact = (int)act.size();
  DG_CK(launch_apply<double>(h->levels[0].op, h->levels[0].dop, 1, h->x64.as<double>(), h->r64.as<double>(),
                             h->b64.as<double>(), dact, nact, s));
  DG_CK(launch_dot<double>(h->r64.as<double>(), h->r64.as<double>(), nullptr, scal(h, S_RR), h->part.as<double>(),
                           h->Nq, dact, nact, s));
  std::vector<double> rr(h->cap);
  DG_CK(cudaMemcpyAsync(rr.data(), scal(h, S_RR), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  for (int k : act) rel[k] = bnorm2[k] > 0 ? std::sqrt(std::max(rr[k], 0.0) / bnorm2[k]) : 0.0;
  return DG_OK;
}

// Solves A x64 = b64 for sources 0..nsrc-1 of the current chunk (b64 filled).
static int solve_chunk(dg_ctx* h, int nsrc, const std::vector<int>& finite, dg_solve_stats* st, cudaStream_t s) {
  const long long Nq = h->Nq;
  const double rtol = h->opts.rtol;
  std::vector<int> act;
  for (int k = 0; k < nsrc; ++k)
    if (finite[k]) act.push_back(k);
  std::vector<int> all(nsrc);
  for (int k = 0; k < nsrc; ++k) all[k] = k;
  DG_RET(upload_act(h, all, s));
  DG_CK(launch_zero<double>(h->x64.as<double>(), Nq, h->act.as<int>(), nsrc, s));
  DG_CK(cudaMemsetAsync(h->flags.p, 0, sizeof(int) * h->cap, s));
  std::vector<double> bnorm2(h->cap, 0.0), rel(h->cap, 1.0);
  if (!act.empty()) {
    DG_RET(upload_act(h, act, s));
    DG_CK(launch_dot<double>(h->b64.as<double>(), h->b64.as<double>(), nullptr, scal(h, S_BN), h->part.as<double>(),
                             Nq, h->act.as<int>(), (int)act.size(), s));
    DG_CK(cudaMemcpyAsync(bnorm2.data(), scal(h, S_BN), sizeof(double) * h->cap, cudaMemcpyDeviceToHost, s));
    DG_CK(cudaStreamSynchronize(s));
  }
  std::vector<int> iters(h->cap, 0), it_inner(h->cap, 0), outer(h->cap, 0);
  const int maxit = h->opts.max_iter;
  const bool mixed = h->opts.precision != DG_PREC_FP64;
  // r64 = b64 (x64 = 0)
  if (!act.empty()) {
    DG_RET(upload_act(h, act, s));
    DG_CK((launch_convert<double, double>(h->r64.as<double>(), h->b64.as<double>(), Nq, h->act.as<int>(),
                                          (int)act.size(), 1.0, 0, s)));
  }
  for (int k : act) rel[k] = bnorm2[k] > 0 ? 1.0 : 0.0;
  // learned form: start from the network's guess (x64, r64, rel set; rejected
  // guesses fall back to x64 = 0)
  std::vector<int> fbk(h->cap, 0);
  if (h->opts.precision == DG_PREC_MIXED_LEARNED) {
    std::vector<int> nz;
    for (int k : act)
      if (bnorm2[k] > 0) nz.push_back(k);
    DG_RET(learned_guess(h, nsrc, nz, bnorm2, h->opts.nn_use_net != 0, rel, fbk, s));
  }
  std::vector<double> grel = rel;
  std::vector<int> todo;
  for (int k : act)
    if (rel[k] > rtol) todo.push_back(k);
  int round = 0;
  while (!todo.empty() && round < 64) {
    ++round;
    DG_RET(upload_act(h, todo, s));
    const int* dact = h->act.as<int>();
    const int nt = (int)todo.size();
    // relative reduction asked of this refinement round, per source: enough for the
    // true residual to reach rtol (FP64), at most inner_rtol (mixed)
    std::vector<double> tolv(h->cap, 1.0), rl(h->cap, 1.0);
    int remaining = 1;
    for (int k : todo) {
      const double need = 0.5 * rtol / std::max(rel[k], 1e-300);
      tolv[k] = mixed ? std::max(need, h->opts.inner_rtol) : std::max(need, 1e-15);
      remaining = std::max(remaining, maxit - iters[k]);
    }
    if (!mixed) {
      DG_CK((launch_convert<double, double>(h->w64.r.as<double>(), h->r64.as<double>(), Nq, dact, nt, 1.0, 0, s)));
      DG_RET(pcg<double>(h, h->w64, todo, tolv, remaining, s, it_inner, rl));
      DG_RET(upload_act(h, todo, s));
      DG_CK((launch_convert<double, double>(h->x64.as<double>(), h->w64.x.as<double>(), Nq, dact, nt, 1.0, 1, s)));
    } else {
      DG_CK((launch_convert<float, double>(h->w32.r.as<float>(), h->r64.as<double>(), Nq, dact, nt, 1.0, 0, s)));
      DG_RET(pcg<float>(h, h->w32, todo, tolv, remaining, s, it_inner, rl));
      DG_RET(upload_act(h, todo, s));
      DG_CK((launch_convert<double, float>(h->x64.as<double>(), h->w32.x.as<float>(), Nq, dact, nt, 1.0, 1, s)));
    }
    for (int k : todo) {
      iters[k] += it_inner[k];
      outer[k] += 1;
    }
    DG_RET(true_residual(h, todo, bnorm2, rel, s));
    if (h->opts.verbose >= 2)
      for (int k : todo)
        std::fprintf(stderr, "  source %d round %d: inner iterations %d (asked %.2e), true residual %.3e\n", k, round,
                     it_inner[k], tolv[k], rel[k]);
    std::vector<int> t2;
    for (int k : todo)
      if (rel[k] > rtol && std::isfinite(rel[k]) && iters[k] < maxit) t2.push_back(k);
    todo = t2;
  }
  std::vector<int> fl(h->cap, 0);
  DG_CK(cudaMemcpyAsync(fl.data(), h->flags.p, sizeof(int) * h->cap, cudaMemcpyDeviceToHost, s));
  int tc_err = 0;
  if (h->tc_err.p) DG_CK(cudaMemcpyAsync(&tc_err, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  if (tc_err) {
    h->err = "a tensor-core patch-solve kernel gave up waiting for its MMA or copy (bounded wait)";
    return DG_ERR_TIMEOUT;
  }
  int worst = DG_OK;
  for (int k = 0; k < nsrc; ++k) {
    dg_solve_stats S;
    S.iters = iters[k];
    S.outer_refinements = mixed ? outer[k] : 0;
    S.used_fallback = fbk[k];
    S.rel_residual = finite[k] ? rel[k] : NAN;
    S.guess_rel_residual = finite[k] ? grel[k] : NAN;
    S.self_energy = 0.0;  // set by the callers that hold the sources
    if (!finite[k])
      S.status = DG_ERR_NONFINITE;
    else if (!(rel[k] <= rtol))
      S.status = (fl[k] & 2) ? DG_ERR_BREAKDOWN : DG_ERR_NOT_CONVERGED;
    else
      S.status = DG_OK;
    if (st) st[k] = S;
    if (S.status != DG_OK && (worst == DG_OK || S.status < worst)) worst = S.status;
  }
  return worst;
}

// Coulomb self-energy of each source of the chunk, (f|f) = sum_q W_q f(q) v(q)
// with v = x64 (Sec. 2.3.1; (ij|ij) for a pair density), into out[0..nsrc).
static int self_energies(dg_ctx* h, const double* f, int nsrc, std::vector<double>& out, cudaStream_t s) {
  out.assign(nsrc, 0.0);
  if (nsrc == 0) return DG_OK;
  std::vector<int> all(nsrc);
  for (int k = 0; k < nsrc; ++k) all[k] = k;
  DG_RET(upload_act(h, all, s));
  DG_CK(launch_dot<double>(f, h->x64.as<double>(), h->d_W.as<double>(), scal(h, S_G1), h->part.as<double>(), h->Nq,
                           h->act.as<int>(), nsrc, s));
  DG_CK(cudaMemcpyAsync(out.data(), scal(h, S_G1), sizeof(double) * nsrc, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

// ---------------------------------------------------------------------------
// boundary data of the sources in f64[0..nsrc) into g[0..nsrc)
// ---------------------------------------------------------------------------
// Gaussian-sum route in precision T (tables bct, NG terms)
template <typename T>
static int boundary_gausssum(dg_ctx* h, const double* f, int nsrc, T* g, BcAxisTables* bct, int NG, DevBuf& flexb,
                             DevBuf& T1b, DevBuf& T2b, cudaStream_t s) {
  const LevelOp& op = h->levels[0].op;
  DG_RET(ensure_bc_work<T>(h, nsrc, NG, bct, flexb, T1b, T2b));
  T* flex = flexb.as<T>();
  DG_CK(launch_weighted_lex<T>(op, h->levels[0].dop, f, h->d_W.as<double>(), flex, nsrc, s));
  const long long Lx = bct[0].L, Ly = bct[1].L, Lz = bct[2].L;
  const long long Nq = h->Nq;
  long long face_off = 0;
  T* T1 = T1b.as<T>();
  T* T2 = T2b.as<T>();
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const long long L1 = bct[t1].L, L2 = bct[t2].L, Ld = bct[d].L;
    const long long tsz = 2LL * NG * L1 * L2;  // per source
    // step 1: contraction along the normal axis with both face positions
    GemmArgs a{};
    a.M = 2 * NG;
    a.K = (int)Ld;
    a.A = bct[d].gn.p;
    a.sAm = Ld;
    a.sAk = 1;
    a.C = T1;
    a.sCm = L1 * L2;
    a.sCn = 1;
    a.alpha = 1.0;
    a.beta = 0.0;
    a.B = flex;
    a.nb1 = nsrc;
    a.sB1 = Nq;
    a.sC1 = tsz;
    if (d == 0) {
      a.N = (int)(Ly * Lz);
      a.nb2 = 1;
      a.sBk = 1;
      a.sBn = Lx;
    } else if (d == 1) {
      a.N = (int)Lx;
      a.nb2 = (int)Lz;
      a.sBk = Lx;
      a.sBn = 1;
      a.sB2 = Lx * Ly;
      a.sC2 = Lx;
    } else {
      a.N = (int)(Lx * Ly);
      a.nb2 = 1;
      a.sBk = Lx * Ly;
      a.sBn = 1;
    }
    DG_CK(launch_gemm<T>(a, s));
    // step 2: along t1 (fastest index), per (source, side, term)
    GemmArgs b{};
    b.M = (int)L2;
    b.N = (int)L1;
    b.K = (int)L1;
    b.nb1 = nsrc * 2;
    b.nb2 = NG;
    b.A = T1;
    b.sAm = L1;
    b.sAk = 1;
    b.sA1 = (long long)NG * L1 * L2;
    b.sA2 = L1 * L2;
    b.B = bct[t1].G.p;
    b.sBk = 1;
    b.sBn = L1;
    b.sB1 = 0;
    b.sB2 = L1 * L1;
    b.C = T2;
    b.sCm = L1;
    b.sCn = 1;
    b.sC1 = (long long)NG * L1 * L2;
    b.sC2 = L1 * L2;
    b.alpha = 1.0;
    b.beta = 0.0;
    DG_CK(launch_gemm<T>(b, s));
    // step 3: along t2 together with the weighted sum over terms
    GemmArgs c{};
    c.M = (int)L2;
    c.N = (int)L1;
    c.K = (int)(NG * L2);
    c.nb1 = nsrc;
    c.nb2 = 2;
    c.A = bct[t2].Gs.p;
    c.sAm = NG * L2;
    c.sAk = 1;
    c.B = T2;
    c.sBk = L1;
    c.sBn = 1;
    c.sB1 = 2LL * NG * L1 * L2;
    c.sB2 = (long long)NG * L1 * L2;
    c.C = g + face_off;
    c.sCm = L1;
    c.sCn = 1;
    c.sC1 = h->nface;
    c.sC2 = L1 * L2;
    c.alpha = 1.0;
    c.beta = 0.0;
    if (sizeof(T) == 4) {  // K = N_G L over few output tiles: split K (FP32 path)
      c.work = h->gemm_ws.p;
      c.work_elems = (long long)(h->gemm_ws.bytes / sizeof(float));
    }
    DG_CK(launch_gemm<T>(c, s));
    face_off += 2 * L1 * L2;
  }
  return DG_OK;
}

// boundary data of the sources f[0..nsrc) into g[0..nsrc) (FP64)
static int boundary_data(dg_ctx* h, int route, const double* f, int nsrc, double* g, cudaStream_t s) {
  const LevelOp& op = h->levels[0].op;
  if (route == DG_BC_DIRECT) {
    DG_CK(launch_bc_direct(op, h->levels[0].dop, f, h->d_W.as<double>(), h->d_xq.as<double>(),
                           h->d_axn.as<double>(), h->lmax, g, nsrc, h->nface, h->nface, s));
    return DG_OK;
  }
  return boundary_gausssum<double>(h, f, nsrc, g, h->bct, h->NG, h->flex, h->T1, h->T2, s);
}

// b64 = 4 pi W f + Nitsche lift of g(f) for f[0..nsrc). The mixed modes
// evaluate the Gaussian-sum route in FP32 with their own (1e-7) table.
bool bc_fp32(const dg_ctx* h) {
  return h->opts.precision != DG_PREC_FP64 && h->opts.bc_route == DG_BC_GAUSSSUM;
}

int form_rhs(dg_ctx* h, const double* f, int nsrc, cudaStream_t s) {
  DG_CK(launch_rhs_volume(f, h->d_W.as<double>(), h->b64.as<double>(), h->Nq, nsrc, s));
  if (bc_fp32(h)) {
    DG_CK(h->g32.ensure(sizeof(float) * h->nface * nsrc));
    DG_RET(boundary_gausssum<float>(h, f, nsrc, h->g32.as<float>(), h->bct32, h->NG32, h->flex32, h->T1_32,
                                    h->T2_32, s));
    DG_CK(launch_lift<float>(h->levels[0].op, h->levels[0].dop, h->g32.as<float>(), h->b64.as<double>(), nsrc,
                             h->nface, s));
  } else {
    DG_RET(boundary_data(h, h->opts.bc_route, f, nsrc, h->g.as<double>(), s));
    DG_CK(launch_lift<double>(h->levels[0].op, h->levels[0].dop, h->g.as<double>(), h->b64.as<double>(), nsrc,
                              h->nface, s));
  }
  return DG_OK;
}

int check_finite(dg_ctx* h, const double* f, int nsrc, std::vector<int>& finite, cudaStream_t s) {
  DG_CK(cudaMemsetAsync(h->flags.p, 0, sizeof(int) * nsrc, s));
  DG_CK(launch_finite_flags(f, h->Nq, nsrc, h->flags.as<int>(), s));
  std::vector<int> fl(nsrc);
  DG_CK(cudaMemcpyAsync(fl.data(), h->flags.p, sizeof(int) * nsrc, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  finite.assign(nsrc, 1);
  for (int k = 0; k < nsrc; ++k) finite[k] = fl[k] ? 0 : 1;
  return DG_OK;
}

static int default_batch(dg_ctx* h) {
  if (h->opts.batch > 0) return h->opts.batch;
  // fill roughly 8 GB of FP64 fine-level vectors
  long long per = h->Nq * 8LL * 12;
  long long b = (8LL << 30) / std::max(per, 1LL);
  return (int)std::max(1LL, std::min(b, 256LL));
}

int prepare(dg_ctx* h, int cap) {
  DG_RET(ensure_common(h, cap));
  if (h->opts.precision == DG_PREC_FP64)
    DG_RET(ensure_prec<double>(h, h->w64, cap));
  else
    DG_RET(ensure_prec<float>(h, h->w32, cap));
  account(h);
  return DG_OK;
}

// ---------------------------------------------------------------------------
// lambda_max(M_S A) of a level by Lanczos from 24 preconditioned CG steps on a
// seeded random right-hand side (FP64); returned with a 8 % safety margin
// (Chebyshev smoothing must not see modes above its interval)
// ---------------------------------------------------------------------------
static int estimate_lambda_schwarz(dg_ctx* h, int l, double* out) {
  Level& L = h->levels[l];
  const long long N = L.op.Nq;
  const long long mp = L.op.n1 + 2;
  DevBuf r, z, p, q, x, zp, part, dsc, dact;
  DG_CK(r.ensure(sizeof(double) * N));
  DG_CK(z.ensure(sizeof(double) * N));
  DG_CK(p.ensure(sizeof(double) * N));
  DG_CK(q.ensure(sizeof(double) * N));
  DG_CK(x.ensure(sizeof(double) * N));
  DG_CK(zp.ensure(sizeof(double) * (size_t)L.op.E * mp * mp * mp));
  DG_CK(part.ensure(sizeof(double) * 304));
  DG_CK(dsc.ensure(sizeof(double) * 4));
  DG_CK(dact.ensure(sizeof(int)));
  DG_CK(cudaMemset(dact.p, 0, sizeof(int)));
  std::vector<double> hr(N);
  unsigned long long st = 0x9E3779B97F4A7C15ull + (unsigned long long)l;
  for (long long i = 0; i < N; ++i) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    hr[i] = ((double)(st >> 11) / 9007199254740992.0) - 0.5;
  }
  DG_CK(cudaMemcpy(r.p, hr.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  const int* a = dact.as<int>();
  double* sc = dsc.as<double>();
  auto dot = [&](const double* u, const double* v, double* res) -> int {
    DG_CK(launch_dot<double>(u, v, nullptr, sc + 3, part.as<double>(), N, a, 1, 0));
    DG_CK(cudaMemcpy(res, sc + 3, sizeof(double), cudaMemcpyDeviceToHost));
    return DG_OK;
  };
  DG_CK(launch_schwarz<double>(L.op, L.dop, L.sw_tabs.as<double>(), r.as<double>(), zp.as<double>(),
                               z.as<double>(), nullptr, 0, 0.0, 0.0, a, 1, 0));
  DG_CK(cudaMemcpy(p.p, z.p, sizeof(double) * N, cudaMemcpyDeviceToDevice));
  double rz = 0.0;
  DG_RET(dot(r.as<double>(), z.as<double>(), &rz));
  std::vector<double> al, be;
  const int K = (int)std::min<long long>(24, N);
  for (int k = 0; k < K; ++k) {
    DG_CK(launch_apply<double>(L.op, L.dop, 0, p.as<double>(), q.as<double>(), nullptr, a, 1, 0));
    double pq = 0.0;
    DG_RET(dot(p.as<double>(), q.as<double>(), &pq));
    if (!(pq > 0.0) || !(rz > 0.0)) break;
    const double alpha = rz / pq;
    DG_CK(cudaMemcpy(sc, &alpha, sizeof(double), cudaMemcpyHostToDevice));
    DG_CK(launch_cg_xr<double>(x.as<double>(), r.as<double>(), p.as<double>(), q.as<double>(), sc, N, a, 1, 0));
    DG_CK(launch_schwarz<double>(L.op, L.dop, L.sw_tabs.as<double>(), r.as<double>(), zp.as<double>(),
                                 z.as<double>(), nullptr, 0, 0.0, 0.0, a, 1, 0));
    double rzn = 0.0;
    DG_RET(dot(r.as<double>(), z.as<double>(), &rzn));
    const double beta = rzn / rz;
    rz = rzn;
    al.push_back(alpha);
    be.push_back(beta);
    DG_CK(cudaMemcpy(sc + 1, &beta, sizeof(double), cudaMemcpyHostToDevice));
    DG_CK(launch_cg_p<double>(p.as<double>(), z.as<double>(), sc + 1, N, a, 1, 0));
    if (!(rz > 0.0)) break;
  }
  const int m = (int)al.size();
  if (m == 0) {
    h->err = "Lanczos estimate of the smoother spectrum failed";
    return DG_ERR_INVALID_ARG;
  }
  std::vector<double> T((size_t)m * m, 0.0);
  for (int k = 0; k < m; ++k) {
    T[(size_t)k * m + k] = 1.0 / al[k] + (k > 0 ? be[k - 1] / al[k - 1] : 0.0);
    if (k + 1 < m) {
      const double o = std::sqrt(std::max(be[k], 0.0)) / al[k];
      T[(size_t)k * m + k + 1] = o;
      T[(size_t)(k + 1) * m + k] = o;
    }
  }
  *out = 1.08 * sym_max_eig(T, m);
  return DG_OK;
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
static int setup(dg_ctx* h) {
  const dg_mesh_desc& m = h->mesh;
  const dg_solver_opts& o = h->opts;
  // level list: degree p -> floor(p/2) down to 1, then n -> n/2 while even
  int n[3] = {m.n[0], m.n[1], m.n[2]};
  int p = m.p;
  std::vector<std::pair<std::array<int, 3>, int>> spec;
  spec.push_back({{n[0], n[1], n[2]}, p});
  while (p > 1) {
    p = std::max(1, p / 2);
    spec.push_back({{n[0], n[1], n[2]}, p});
  }
  // geometric coarsening while every n is even, until a level small enough for
  // the dense coarsest solve (<= 512 unknowns at degree 1) is reached
  while (n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0 && n[0] >= 2 && n[1] >= 2 && n[2] >= 2 &&
         8LL * n[0] * n[1] * n[2] > 512 && (int)spec.size() < MAXLEV) {
    n[0] /= 2;
    n[1] /= 2;
    n[2] /= 2;
    spec.push_back({{n[0], n[1], n[2]}, 1});
  }
  h->nlev = (int)spec.size();
  h->levels.resize(h->nlev);
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->levels[l];
    double sig0[3];
    for (int d = 0; d < 3; ++d) sig0[d] = h->levels[0].op.ax[d].sigma;
    build_level(L.op, spec[l].first.data(), spec[l].second, m.lo, m.hi, o.penalty_form, o.penalty_eps,
                (l > 0 && o.coarse_penalty == 1) ? sig0 : nullptr);
    L.lam_max = level_lambda_max(L.op);
  }
  for (int l = 0; l + 1 < h->nlev; ++l) build_transfer(h->levels[l].tr, h->levels[l].op, h->levels[l + 1].op);
  DG_CK(cudaStreamCreateWithFlags(&h->ws, cudaStreamNonBlocking));
  DG_CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  DG_CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  const LevelOp& Lc = h->levels[h->nlev - 1].op;
  if (Lc.Nq > 4096) {
    h->err = "coarsest multigrid level has more than 4096 unknowns";
    return DG_ERR_UNSUPPORTED;
  }
  h->Nc = (int)Lc.Nq;
  {
    std::vector<double> Ac = level_dense(Lc);
    if (!spd_inverse(Ac, h->Nc)) {
      h->err = "coarsest-level operator is not positive definite";
      return DG_ERR_INVALID_ARG;
    }
    DG_CK(h->coarse_inv.ensure(sizeof(double) * Ac.size()));
    DG_CK(cudaMemcpy(h->coarse_inv.p, Ac.data(), sizeof(double) * Ac.size(), cudaMemcpyHostToDevice));
  }
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->levels[l];
    DG_CK(cudaMalloc(&L.dop, sizeof(LevelOp)));
    DG_CK(cudaMemcpy(L.dop, &L.op, sizeof(LevelOp), cudaMemcpyHostToDevice));
    DG_CK(cudaMalloc(&L.dtr, sizeof(TransferOp)));
    DG_CK(cudaMemcpy(L.dtr, &L.tr, sizeof(TransferOp), cudaMemcpyHostToDevice));
  }
  if (o.smoother == DG_SMOOTH_SCHWARZ) {
    for (int l = 0; l + 1 < h->nlev; ++l) {
      Level& L = h->levels[l];
      const std::vector<double> tb = schwarz_tables(L.op);
      DG_CK(L.sw_tabs.ensure(sizeof(double) * tb.size()));
      DG_CK(cudaMemcpy(L.sw_tabs.p, tb.data(), sizeof(double) * tb.size(), cudaMemcpyHostToDevice));
      DG_RET(estimate_lambda_schwarz(h, l, &L.lam_sw));
      // FP32 inner solve: patch solves on the tensor cores at degrees 7-8 (and 6
      // when asked: there the SIMT kernel is as fast)
      if (o.precision != DG_PREC_FP64 && o.tc_smoother > 0 && (L.op.n1 >= 8 || o.tc_smoother >= 2)) {
        if (!h->tc_err.p) {
          DG_CK(h->tc_err.ensure(sizeof(int)));
          DG_CK(cudaMemset(h->tc_err.p, 0, sizeof(int)));
        }
        const std::vector<unsigned char> blob = schwarz_tc_blob(L.op, tb, h->tc_err.as<int>());
        if (!blob.empty()) {
          DG_CK(schwarz_tc_prepare(L.op.n1));
          DG_CK(L.sw_tc.ensure(blob.size()));
          DG_CK(cudaMemcpy(L.sw_tc.p, blob.data(), blob.size(), cudaMemcpyHostToDevice));
          std::memcpy(&L.tcp.head, blob.data(), sizeof(SwTcHead));
          L.tcp.geom = L.tcp.head.geom;
          L.tcp.blob = L.sw_tc.p;
        }
      }
    }
  }
  // fine-level nodes, weights
  const LevelOp& F = h->levels[0].op;
  h->Nq = F.Nq;
  const int n1 = F.n1;
  double xi[MAXN1], w[MAXN1];
  gauss_legendre(n1, xi, w);
  h->lmax = 0;
  for (int d = 0; d < 3; ++d) {
    const int Ld = F.n[d] * n1;
    h->lmax = std::max(h->lmax, Ld);
    h->axis_nodes[d].resize(Ld);
    const double hd = F.ax[d].h;
    for (int e = 0; e < F.n[d]; ++e)
      for (int a = 0; a < n1; ++a) h->axis_nodes[d][e * n1 + a] = m.lo[d] + hd * (e + (xi[a] + 1.0) / 2.0);
  }
  {
    std::vector<double> W(h->Nq), X(3 * h->Nq);
    const int npe = n1 * n1 * n1;
    for (long long q = 0; q < h->Nq; ++q) {
      const int e = (int)(q / npe), loc = (int)(q % npe);
      const int a = loc % n1, b = (loc / n1) % n1, c = loc / (n1 * n1);
      const int ex = e % F.n[0], ey = (e / F.n[0]) % F.n[1], ez = e / (F.n[0] * F.n[1]);
      W[q] = F.ax[0].m[a] * F.ax[1].m[b] * F.ax[2].m[c];
      X[3 * q] = h->axis_nodes[0][ex * n1 + a];
      X[3 * q + 1] = h->axis_nodes[1][ey * n1 + b];
      X[3 * q + 2] = h->axis_nodes[2][ez * n1 + c];
    }
    DG_CK(h->d_W.ensure(sizeof(double) * h->Nq));
    DG_CK(cudaMemcpy(h->d_W.p, W.data(), sizeof(double) * h->Nq, cudaMemcpyHostToDevice));
    DG_CK(h->d_xq.ensure(sizeof(double) * 3 * h->Nq));
    DG_CK(cudaMemcpy(h->d_xq.p, X.data(), sizeof(double) * 3 * h->Nq, cudaMemcpyHostToDevice));
    std::vector<double> axn(3 * (size_t)h->lmax, 0.0);
    for (int d = 0; d < 3; ++d)
      for (size_t i = 0; i < h->axis_nodes[d].size(); ++i) axn[d * h->lmax + i] = h->axis_nodes[d][i];
    DG_CK(h->d_axn.ensure(sizeof(double) * axn.size()));
    DG_CK(cudaMemcpy(h->d_axn.p, axn.data(), sizeof(double) * axn.size(), cudaMemcpyHostToDevice));
  }
  h->nface = 0;
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    h->nface += 2LL * F.n[t1] * n1 * F.n[t2] * n1;
  }
  // Gaussian-sum tables: accurate on [rmin, rmax], rmin the smallest
  // face-node to volume-node distance (the first interior node along the
  // normal), rmax the box diagonal
  {
    double rmin = 1e300, diag2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      rmin = std::min(rmin, (1.0 - xi[n1 - 1]) * F.ax[d].h / 2.0);
      diag2 += (m.hi[d] - m.lo[d]) * (m.hi[d] - m.lo[d]);
    }
    auto build_tables = [&](double tol, GaussSum& gs, int& NG, BcAxisTables* bct, bool fp32) -> int {
      gs = make_gauss_sum(rmin * 0.999, std::sqrt(diag2) * 1.001, tol, h->opts.gauss_construction == 0);
      NG = (int)gs.c.size();
      if (NG == 0) {
        h->err = "could not build the Gaussian-sum 1/r table";
        return DG_ERR_INVALID_ARG;
      }
      for (int d = 0; d < 3; ++d) {
        const int L = (int)h->axis_nodes[d].size();
        bct[d].L = L;
        const std::vector<double>& x = h->axis_nodes[d];
        std::vector<double> gn(2 * (size_t)NG * L), G((size_t)NG * L * L), Gs((size_t)L * NG * L);
        for (int sd = 0; sd < 2; ++sd) {
          const double xf = sd == 0 ? m.lo[d] : m.hi[d];
          for (int k = 0; k < NG; ++k)
            for (int i = 0; i < L; ++i) gn[((size_t)sd * NG + k) * L + i] = std::exp(-gs.a[k] * (x[i] - xf) * (x[i] - xf));
        }
        for (int k = 0; k < NG; ++k)
          for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) {
              const double v = std::exp(-gs.a[k] * (x[i] - x[j]) * (x[i] - x[j]));
              G[((size_t)k * L + i) * L + j] = v;
              Gs[(size_t)i * NG * L + (size_t)k * L + j] = gs.c[k] * v;
            }
        auto up = [&](DevBuf& dst, const std::vector<double>& src) -> int {
          if (fp32) {
            std::vector<float> t(src.begin(), src.end());
            DG_CK(dst.ensure(sizeof(float) * t.size()));
            DG_CK(cudaMemcpy(dst.p, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice));
          } else {
            DG_CK(dst.ensure(sizeof(double) * src.size()));
            DG_CK(cudaMemcpy(dst.p, src.data(), sizeof(double) * src.size(), cudaMemcpyHostToDevice));
          }
          return DG_OK;
        };
        DG_RET(up(bct[d].gn, gn));
        DG_RET(up(bct[d].G, G));
        DG_RET(up(bct[d].Gs, Gs));
      }
      return DG_OK;
    };
    const double tol = o.bc_tol > 0 ? o.bc_tol : 1e-12;
    DG_RET(build_tables(tol, h->gsum, h->NG, h->bct, false));
    if (o.precision != DG_PREC_FP64) DG_RET(build_tables(1e-7, h->gsum32, h->NG32, h->bct32, true));
  }
  account(h);
  return DG_OK;
}

}  // namespace dg

namespace dg {
std::atomic<long long> g_launch_count{0};
thread_local long long t_launch_count = 0;

template <typename T>
static int apply_smoother_t(dg_ctx* h, PrecWork<T>& w, int level, const T* r, T* z, int nb, cudaStream_t s) {
  const Level& L = h->levels[level];
  const int* a = h->act.as<int>();
  if (level == h->nlev - 1) {
    DG_CK(launch_coarse_solve<T>(h->coarse_inv.as<double>(), h->Nc, r, z, a, nb, s));
  } else if (h->opts.smoother == DG_SMOOTH_SCHWARZ) {
    DG_CK(launch_schwarz<T>(L.op, L.dop, L.sw_tabs.as<double>(), r, w.lev[level].zp.template as<T>(), z, nullptr, 0,
                            0.0, 0.0, a, nb, s, L.tc()));
  } else {
    DG_CK(launch_cheb_first<T>(z, z, r, w.lev[level].invD.template as<T>(), 1.0, 1, L.op.Nq, a, nb, s));
  }
  return DG_OK;
}


}  // namespace dg

using namespace dg;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void dg_default_opts(dg_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = DG_PREC_FP64;
  o->rtol = 1e-8;
  o->max_iter = 500;
  o->penalty_eps = 0.125;
  o->penalty_form = 0;
  o->bc_route = DG_BC_GAUSSSUM;
  o->bc_tol = 0.0;
  o->batch = 0;
  o->smoother = DG_SMOOTH_SCHWARZ;
  o->smoother_degree = 4;
  o->cheb_range = 10.0;
  o->inner_rtol = 1e-4;
  o->nn_weights_path = nullptr;
  o->verbose = 0;
  o->coarse_penalty = 0;
  o->coarse_smoother_degree = 0;
  o->p1_smoother = -1;
  o->gauss_construction = 0;
  o->tc_smoother = 1;
  o->nn_use_net = 1;
  o->device_loop = 2;
}

const char* dg_error_string(int status) {
  switch (status) {
    case DG_OK: return "ok";
    case DG_ERR_INVALID_ARG: return "invalid argument";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_NOT_CONVERGED: return "not converged";
    case DG_ERR_BREAKDOWN: return "CG breakdown";
    case DG_ERR_NONFINITE: return "non-finite input";
    case DG_ERR_TIMEOUT: return "timeout";
    case DG_ERR_NO_MEMORY: return "out of device memory";
    case DG_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* dg_last_error_detail(dg_handle h) { return h ? h->err.c_str() : ""; }

int64_t dg_kernel_launch_count(void) { return g_launch_count.load(); }

int dg_poisson_setup(const dg_mesh_desc* mesh, const dg_solver_opts* opts, dg_handle* out) {
  if (!mesh || !out) return DG_ERR_INVALID_ARG;
  *out = nullptr;
  if (mesh->p < 1 || mesh->p > 8) return DG_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d) {
    if (mesh->n[d] < 1 || mesh->n[d] > 4096) return DG_ERR_INVALID_ARG;
    if (!(mesh->hi[d] > mesh->lo[d]) || !std::isfinite(mesh->lo[d]) || !std::isfinite(mesh->hi[d]))
      return DG_ERR_INVALID_ARG;
  }
  dg_solver_opts o;
  if (opts)
    o = *opts;
  else
    dg_default_opts(&o);
  if (!(o.rtol > 0) || o.max_iter < 1 || !(o.penalty_eps > 0) || (o.penalty_form != 0 && o.penalty_form != 1) ||
      (o.bc_route != DG_BC_DIRECT && o.bc_route != DG_BC_GAUSSSUM) || o.precision < 0 || o.precision > 2 ||
      o.smoother_degree < 1 || o.smoother_degree > 16 || o.batch < 0 ||
      (o.smoother != DG_SMOOTH_JACOBI && o.smoother != DG_SMOOTH_SCHWARZ) ||
      (o.coarse_penalty != 0 && o.coarse_penalty != 1) || o.coarse_smoother_degree < 0 ||
      o.coarse_smoother_degree > 16 || o.p1_smoother < -1 || o.p1_smoother > 1 ||
      (o.gauss_construction != 0 && o.gauss_construction != 1) || o.device_loop < 0 || o.device_loop > 2)
    return DG_ERR_INVALID_ARG;
  if (o.cheb_range <= 1.0) o.cheb_range = 10.0;
  if (o.inner_rtol <= 0.0) o.inner_rtol = 1e-4;
  if (o.precision == DG_PREC_MIXED_LEARNED && mesh->p > NN_MAXN1 - 1) return DG_ERR_UNSUPPORTED;
  dg_ctx* h = new (std::nothrow) dg_ctx();
  if (!h) return DG_ERR_NO_MEMORY;
  h->mesh = *mesh;
  h->opts = o;
  DeviceWideGuard guard;  // set-up allocates, copies synchronously and launches on the legacy stream
  int rc = setup(h);
  if (rc == DG_OK && o.precision == DG_PREC_MIXED_LEARNED && o.nn_weights_path) rc = nn_load_file(h, o.nn_weights_path);
  h->opts.nn_weights_path = nullptr;  // the caller's string is not kept
  if (rc != DG_OK) {
    fprintf(stderr, "dg_poisson_setup: %s\n", h->err.c_str());
    dg_destroy(h);
    return rc;
  }
  *out = h;
  return DG_OK;
}

void dg_destroy(dg_handle h) {
  if (!h) return;
  DeviceWideGuard guard;
  for (auto& L : h->levels) {
    if (L.dop) cudaFree(L.dop);
    if (L.dtr) cudaFree(L.dtr);
  }
  delete h;
}

int dg_get_info(dg_handle h, dg_info* info) {
  if (!h || !info) return DG_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->Nq = h->Nq;
  info->levels = h->nlev;
  info->batch = default_batch(h);
  for (int l = 0; l < h->nlev && l < 16; ++l) {
    info->level_n[l] = h->levels[l].op.n[0];
    info->level_p[l] = h->levels[l].op.p;
  }
  info->coarse_dofs = h->Nc;
  info->n_gauss = h->NG;
  info->gauss_rmin = h->gsum.rmin;
  info->gauss_rmax = h->gsum.rmax;
  info->gauss_relerr = h->gsum.relerr;
  info->n_gauss_fp32 = h->NG32;
  info->gauss_relerr_fp32 = h->gsum32.relerr;
  for (int d = 0; d < 3; ++d) info->sigma[d] = h->levels[0].op.ax[d].sigma;
  account(h);
  info->workspace_bytes = h->ws_bytes;
  return DG_OK;
}

int dg_mesh_node_coords(const dg_mesh_desc* m, double* xyz, double* w) {
  if (!m || m->p < 1 || m->p > 8) return DG_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (m->n[d] < 1 || !(m->hi[d] > m->lo[d])) return DG_ERR_INVALID_ARG;
  const int n1 = m->p + 1, npe = n1 * n1 * n1;
  double xi[MAXN1], wg[MAXN1];
  gauss_legendre(n1, xi, wg);
  double hd[3];
  for (int d = 0; d < 3; ++d) hd[d] = (m->hi[d] - m->lo[d]) / m->n[d];
  const long long Nq = (long long)m->n[0] * m->n[1] * m->n[2] * npe;
  for (long long q = 0; q < Nq; ++q) {
    const int e = (int)(q / npe), loc = (int)(q % npe);
    const int a[3] = {loc % n1, (loc / n1) % n1, loc / (n1 * n1)};
    const int ec[3] = {e % m->n[0], (e / m->n[0]) % m->n[1], e / (m->n[0] * m->n[1])};
    double wq = 1.0;
    for (int d = 0; d < 3; ++d) {
      if (xyz) xyz[3 * q + d] = m->lo[d] + hd[d] * (ec[d] + (xi[a[d]] + 1.0) / 2.0);
      wq *= wg[a[d]] * hd[d] / 2.0;
    }
    if (w) w[q] = wq;
  }
  return DG_OK;
}

int dg_node_coords(dg_handle h, double* xyz, double* w) {
  if (!h) return DG_ERR_INVALID_ARG;
  const LevelOp& F = h->levels[0].op;
  const int n1 = F.n1, npe = n1 * n1 * n1;
  for (long long q = 0; q < h->Nq; ++q) {
    const int e = (int)(q / npe), loc = (int)(q % npe);
    const int a = loc % n1, b = (loc / n1) % n1, c = loc / (n1 * n1);
    const int ex = e % F.n[0], ey = (e / F.n[0]) % F.n[1], ez = e / (F.n[0] * F.n[1]);
    if (xyz) {
      xyz[3 * q] = h->axis_nodes[0][ex * n1 + a];
      xyz[3 * q + 1] = h->axis_nodes[1][ey * n1 + b];
      xyz[3 * q + 2] = h->axis_nodes[2][ez * n1 + c];
    }
    if (w) w[q] = F.ax[0].m[a] * F.ax[1].m[b] * F.ax[2].m[c];
  }
  return DG_OK;
}

int dg_apply_operator(dg_handle h, int32_t level, int32_t fp32, const void* u, void* out, int64_t B, void* stream) {
  if (!h || level < 0 || level >= h->nlev || B < 0 || (B > 0 && (!u || !out))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = (int)std::min<int64_t>(B, 65535);
  DG_RET(ensure_common(h, cap));
  const Level& L = h->levels[level];
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    std::vector<int> a(nb);
    for (int k = 0; k < nb; ++k) a[k] = k;
    DG_RET(upload_act(h, a, s));
    if (fp32)
      DG_CK(launch_apply<float>(L.op, L.dop, 0, (const float*)u + b0 * L.op.Nq, (float*)out + b0 * L.op.Nq, nullptr,
                                h->act.as<int>(), nb, s));
    else
      DG_CK(launch_apply<double>(L.op, L.dop, 0, (const double*)u + b0 * L.op.Nq, (double*)out + b0 * L.op.Nq,
                                 nullptr, h->act.as<int>(), nb, s));
  }
  return DG_OK;
}

int dg_apply_transfer(dg_handle h, int32_t level, int32_t direction, int32_t fp32, const void* in, void* out,
                      int64_t B, void* stream) {
  if (!h || level < 0 || level >= h->nlev - 1 || (direction != 0 && direction != 1) || B < 0 ||
      (B > 0 && (!in || !out)))
    return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = (int)std::min<int64_t>(B, 65535);
  DG_RET(ensure_common(h, cap));
  const Level& L = h->levels[level];
  const Level& Cl = h->levels[level + 1];
  const long long nqf = L.op.Nq, nqc = Cl.op.Nq;
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    std::vector<int> a(nb);
    for (int k = 0; k < nb; ++k) a[k] = k;
    DG_RET(upload_act(h, a, s));
    const int* act = h->act.as<int>();
    if (direction == 0) {
      if (fp32) {
        float* o = (float*)out + b0 * nqf;
        DG_CK(launch_zero<float>(o, nqf, act, nb, s));
        DG_CK(launch_prolong_add<float>(L.tr, L.dtr, L.op, Cl.op, (const float*)in + b0 * nqc, o, act, nb, s));
      } else {
        double* o = (double*)out + b0 * nqf;
        DG_CK(launch_zero<double>(o, nqf, act, nb, s));
        DG_CK(launch_prolong_add<double>(L.tr, L.dtr, L.op, Cl.op, (const double*)in + b0 * nqc, o, act, nb, s));
      }
    } else {
      if (fp32)
        DG_CK(launch_restrict<float>(L.tr, L.dtr, L.op, Cl.op, (const float*)in + b0 * nqf, (float*)out + b0 * nqc,
                                     act, nb, s));
      else
        DG_CK(launch_restrict<double>(L.tr, L.dtr, L.op, Cl.op, (const double*)in + b0 * nqf,
                                      (double*)out + b0 * nqc, act, nb, s));
    }
  }
  return DG_OK;
}

int dg_apply_smoother(dg_handle h, int32_t level, int32_t fp32, const void* r, void* z, int64_t B, void* stream) {
  if (!h || level < 0 || level >= h->nlev || B < 0 || (B > 0 && (!r || !z))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = (int)std::min<int64_t>(B, 4096);
  DG_RET(ensure_common(h, cap));
  if (fp32)
    DG_RET(ensure_prec<float>(h, h->w32, cap));
  else
    DG_RET(ensure_prec<double>(h, h->w64, cap));
  const long long N = h->levels[level].op.Nq;
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    std::vector<int> a(nb);
    for (int k = 0; k < nb; ++k) a[k] = k;
    DG_RET(upload_act(h, a, s));
    if (fp32)
      DG_RET(apply_smoother_t<float>(h, h->w32, level, (const float*)r + b0 * N, (float*)z + b0 * N, nb, s));
    else
      DG_RET(apply_smoother_t<double>(h, h->w64, level, (const double*)r + b0 * N, (double*)z + b0 * N, nb, s));
  }
  return DG_OK;
}

int dg_apply_patch_solves(dg_handle h, int32_t level, int32_t fp32, const void* r, void* zp, int64_t B,
                          void* stream) {
  if (!h || level < 0 || level >= h->nlev - 1 || B < 0 || B > 65535 || (B > 0 && (!r || !zp)))
    return DG_ERR_INVALID_ARG;
  if (h->opts.smoother != DG_SMOOTH_SCHWARZ) {
    h->err = "dg_apply_patch_solves: the handle's smoother is not the Schwarz smoother";
    return DG_ERR_UNSUPPORTED;
  }
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)B;
  DG_RET(ensure_common(h, nb));
  std::vector<int> a(nb);
  for (int k = 0; k < nb; ++k) a[k] = k;
  DG_RET(upload_act(h, a, s));
  const Level& L = h->levels[level];
  if (fp32)
    DG_CK(launch_schwarz_patch<float>(L.op, L.dop, L.sw_tabs.as<double>(), (const float*)r, (float*)zp,
                                      h->act.as<int>(), nb, s, L.tc()));
  else
    DG_CK(launch_schwarz_patch<double>(L.op, L.dop, L.sw_tabs.as<double>(), (const double*)r, (double*)zp,
                                       h->act.as<int>(), nb, s, nullptr));
  return DG_OK;
}

int dg_boundary_data(dg_handle h, int32_t route, const double* f, int64_t B, double* g, int64_t* nface,
                     void* stream) {
  if (!h || (route != DG_BC_DIRECT && route != DG_BC_GAUSSSUM) || B < 0) return DG_ERR_INVALID_ARG;
  if (nface) *nface = h->nface;
  if (!g || B == 0) return DG_OK;
  if (!f) return DG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = std::max(1, std::min(default_batch(h), (int)B));
  DG_RET(ensure_common(h, cap));
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    if (route == DG_BC_GAUSSSUM && bc_fp32(h)) {
      DG_CK(h->g32.ensure(sizeof(float) * h->nface * nb));
      DG_RET(boundary_gausssum<float>(h, f + b0 * h->Nq, nb, h->g32.as<float>(), h->bct32, h->NG32, h->flex32,
                                      h->T1_32, h->T2_32, s));
      std::vector<int> a(nb);
      for (int k = 0; k < nb; ++k) a[k] = k;
      DG_RET(upload_act(h, a, s));
      DG_CK((launch_convert<double, float>(g + b0 * h->nface, h->g32.as<float>(), h->nface, h->act.as<int>(), nb,
                                           1.0, 0, s)));
    } else {
      DG_RET(boundary_data(h, route, f + b0 * h->Nq, nb, g + b0 * h->nface, s));
    }
  }
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_gauss_sum(double rmin, double rmax, double tol, int32_t construction, int32_t max_terms, int32_t* n_terms,
                 double* relerr, double* c, double* alpha) {
  if (!(rmin > 0.0) || !(rmax > rmin) || !(tol > 0.0) || (construction != 0 && construction != 1) || !n_terms)
    return DG_ERR_INVALID_ARG;
  const GaussSum gs = make_gauss_sum(rmin, rmax, tol, construction == 0);
  const int n = (int)gs.c.size();
  if (n == 0) return DG_ERR_UNSUPPORTED;
  if ((c || alpha) && max_terms < n) return DG_ERR_INVALID_ARG;
  *n_terms = n;
  if (relerr) *relerr = gs.relerr;
  for (int k = 0; k < n; ++k) {
    if (c) c[k] = gs.c[k];
    if (alpha) alpha[k] = gs.a[k];
  }
  return DG_OK;
}

int dg_form_rhs(dg_handle h, const double* f, int64_t B, double* b, void* stream) {
  if (!h || B < 0 || (B > 0 && (!f || !b))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap = std::max(1, std::min(default_batch(h), (int)std::min<int64_t>(B, 65535)));
  DG_RET(prepare(h, cap));
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    DG_RET(form_rhs(h, f + b0 * h->Nq, nb, s));
    DG_CK(cudaMemcpyAsync(b + b0 * h->Nq, h->b64.p, sizeof(double) * h->Nq * nb, cudaMemcpyDeviceToDevice, s));
  }
  DG_CK(cudaStreamSynchronize(s));
  return DG_OK;
}

int dg_pair_solve_batch(dg_handle h, const double* f, int64_t B, double* v, dg_solve_stats* stats, void* stream) {
  if (!h || B < 0 || (B > 0 && (!f || !v))) return DG_ERR_INVALID_ARG;
  if (B == 0) return DG_OK;
  // work runs on the handle's stream, ordered after the caller's stream
  cudaStream_t us = (cudaStream_t)stream;
  DG_CK(cudaEventRecord(h->ev_in, us));
  DG_CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  cudaStream_t s = h->ws;
  const int cap = std::max(1, std::min(default_batch(h), (int)std::min<int64_t>(B, 65535)));
  DG_RET(prepare(h, cap));
  int worst = DG_OK;
  for (int64_t b0 = 0; b0 < B; b0 += cap) {
    const int nb = (int)std::min<int64_t>(cap, B - b0);
    const double* fc = f + b0 * h->Nq;
    std::vector<int> finite;
    DG_RET(check_finite(h, fc, nb, finite, s));
    DG_RET(form_rhs(h, fc, nb, s));
    const int rc = solve_chunk(h, nb, finite, stats ? stats + b0 : nullptr, s);
    if (rc == DG_ERR_CUDA || rc == DG_ERR_NO_MEMORY) return rc;
    if (rc != DG_OK && (worst == DG_OK || rc < worst)) worst = rc;
    if (stats) {
      std::vector<double> se;
      DG_RET(self_energies(h, fc, nb, se, s));
      for (int k = 0; k < nb; ++k) stats[b0 + k].self_energy = se[k];
    }
    DG_CK(cudaMemcpyAsync(v + b0 * h->Nq, h->x64.p, sizeof(double) * h->Nq * nb, cudaMemcpyDeviceToDevice, s));
  }
  DG_CK(cudaStreamSynchronize(s));
  DG_CK(cudaEventRecord(h->ev_out, s));
  DG_CK(cudaStreamWaitEvent(us, h->ev_out, 0));
  if (h->opts.verbose) fprintf(stderr, "dg_pair_solve_batch: %lld sources, status %d\n", (long long)B, worst);
  return worst;
}

// Exchange build over the sources [src_begin, src_end) of the list
// 0 = Hartree density, then the pairs (i <= j) row-major: K_host receives
// their contribution to K (the contributions of disjoint ranges add up to K),
// E_H is set when the range holds source 0 (else 0), E_X = -1/2 tr K_host.
static int exchange_build_range(dg_handle h, const double* psi, int32_t N, long long src_begin, long long src_end,
                                double* K_host, double* E_H, double* E_X, dg_solve_stats* stats, void* stream) {
  h->ace_N = 0;  // W and K are rewritten below; valid again only after a whole, successful build
  cudaStream_t us = (cudaStream_t)stream;
  DG_CK(cudaEventRecord(h->ev_in, us));
  DG_CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  cudaStream_t s = h->ws;
  const long long Nq = h->Nq;
  const int P = N * (N + 1) / 2;
  const int nsrc_total = P + 1;
  const int cap = std::max(1, std::min<int>(default_batch(h), (int)(src_end - src_begin)));
  DG_RET(prepare(h, cap));
  DG_CK(h->Wacc.ensure(sizeof(double) * N * Nq));
  const int nch = kmat_chunks(Nq);
  DG_CK(h->kpart.ensure(sizeof(double) * (size_t)nch * N * N));
  DG_CK(h->Kdev.ensure(sizeof(double) * ((size_t)N * N + 4)));
  DG_CK(cudaMemsetAsync(h->Wacc.p, 0, sizeof(double) * N * Nq, s));
  // source list: 0 = Hartree density, then pairs (i <= j) row-major
  std::vector<int> si(nsrc_total), sj(nsrc_total);
  si[0] = -1;
  sj[0] = -1;
  {
    int k = 1;
    for (int i = 0; i < N; ++i)
      for (int j = i; j < N; ++j, ++k) {
        si[k] = i;
        sj[k] = j;
      }
  }
  int worst = DG_OK;
  double eh = 0.0;
  DevBuf lists;
  for (int b0 = (int)src_begin; b0 < (int)src_end; b0 += cap) {
    const int nb = std::min(cap, (int)src_end - b0);
    DG_CK(cudaMemcpyAsync(h->pidx.p, si.data() + b0, sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    DG_CK(cudaMemcpyAsync(h->pidx.as<int>() + cap, sj.data() + b0, sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    DG_CK(launch_pair_sources(psi, N, h->pidx.as<int>(), h->pidx.as<int>() + cap, nb, Nq, h->f64.as<double>(), s));
    std::vector<int> finite;
    DG_RET(check_finite(h, h->f64.as<double>(), nb, finite, s));
    DG_RET(form_rhs(h, h->f64.as<double>(), nb, s));
    const int rc = solve_chunk(h, nb, finite, stats ? stats + (b0 - src_begin) : nullptr, s);
    if (rc == DG_ERR_CUDA || rc == DG_ERR_NO_MEMORY) return rc;
    if (rc != DG_OK && (worst == DG_OK || rc < worst)) worst = rc;
    const double* v = h->x64.as<double>();
    // self-energies (f|f) = sum_q W_q f v of the chunk's sources: the pair
    // self-energies (ij|ij), and for source 0 (rho) E_H = (rho|rho) / 2
    std::vector<double> se;
    DG_RET(self_energies(h, h->f64.as<double>(), nb, se, s));
    if (stats)
      for (int k = 0; k < nb; ++k) stats[b0 - src_begin + k].self_energy = se[k];
    if (b0 == 0) eh = 0.5 * se[0];
    // W_j += psi_s v_sj and W_s += psi_j v_sj (s != j), per orbital in fixed order
    std::vector<std::vector<std::pair<int, int>>> per(N);
    for (int k = 0; k < nb; ++k) {
      const int g = b0 + k;
      if (si[g] < 0) continue;
      per[sj[g]].push_back({k, si[g]});
      if (si[g] != sj[g]) per[si[g]].push_back({k, sj[g]});
    }
    std::vector<int> ptr(N + 1, 0), eb, es;
    for (int m = 0; m < N; ++m) {
      for (auto& e : per[m]) {
        eb.push_back(e.first);
        es.push_back(e.second);
      }
      ptr[m + 1] = (int)eb.size();
    }
    if (!eb.empty()) {
      std::vector<int> pack;
      pack.insert(pack.end(), ptr.begin(), ptr.end());
      pack.insert(pack.end(), eb.begin(), eb.end());
      pack.insert(pack.end(), es.begin(), es.end());
      DG_CK(lists.ensure(sizeof(int) * pack.size()));
      DG_CK(cudaMemcpyAsync(lists.p, pack.data(), sizeof(int) * pack.size(), cudaMemcpyHostToDevice, s));
      const int* dl = lists.as<int>();
      DG_CK(launch_exch_accum(psi, v, h->Wacc.as<double>(), dl, dl + N + 1, dl + N + 1 + eb.size(), N, Nq, s));
      DG_CK(cudaStreamSynchronize(s));  // pack is a host temporary
    }
  }
  DG_CK(launch_kmat(psi, h->d_W.as<double>(), h->Wacc.as<double>(), N, Nq, h->kpart.as<double>(), nch,
                    h->Kdev.as<double>(), s));
  DG_CK(cudaMemcpyAsync(K_host, h->Kdev.p, sizeof(double) * N * N, cudaMemcpyDeviceToHost, s));
  DG_CK(cudaStreamSynchronize(s));
  DG_CK(cudaEventRecord(h->ev_out, s));
  DG_CK(cudaStreamWaitEvent(us, h->ev_out, 0));
  if (E_H) *E_H = eh;
  if (E_X) {
    double tr = 0.0;
    for (int i = 0; i < N; ++i) tr += K_host[(size_t)i * N + i];
    *E_X = -0.5 * tr;
  }
  // a whole build leaves W (Wacc) and K for the compressed exchange operator
  if (src_begin == 0 && src_end == nsrc_total && worst == DG_OK) {
    h->ace_K.assign(K_host, K_host + (size_t)N * N);
    h->ace_N = N;
  } else {
    h->ace_N = 0;
  }
  account(h);
  return worst;
}

int dg_exchange_build(dg_handle h, const double* psi, int32_t N, double* K_host, double* E_H, double* E_X,
                      dg_solve_stats* stats, void* stream) {
  if (!h || N < 1 || !psi || !K_host) return DG_ERR_INVALID_ARG;
  return exchange_build_range(h, psi, N, 0, (long long)N * (N + 1) / 2 + 1, K_host, E_H, E_X, stats, stream);
}

int dg_exchange_build_range(dg_handle h, const double* psi, int32_t N, int64_t src_begin, int64_t src_end,
                            double* K_partial_host, double* E_H, dg_solve_stats* stats, void* stream) {
  if (!h || N < 1 || !psi || !K_partial_host) return DG_ERR_INVALID_ARG;
  const long long total = (long long)N * (N + 1) / 2 + 1;
  if (src_begin < 0 || src_end < src_begin || src_end > total) return DG_ERR_INVALID_ARG;
  if (src_end == src_begin) {
    std::memset(K_partial_host, 0, sizeof(double) * (size_t)N * N);
    if (E_H) *E_H = 0.0;
    return DG_OK;
  }
  return exchange_build_range(h, psi, N, src_begin, src_end, K_partial_host, E_H, nullptr, stats, stream);
}

// Hartree and exchange actions on trial functions (Sec. 2.3.1): the solves of
// psi_j u_k (and of the density for J) in batches, J u = v_H u formed from the
// Hartree solve, X u_k accumulated per trial function over j in ascending order
// and negated at the end.
int dg_jk_apply(dg_handle h, const double* psi, int32_t N, const double* U, int64_t m, double* JU, double* XU,
                dg_solve_stats* stats, void* stream) {
  if (!h || N < 1 || m < 1 || !psi || !U || (!JU && !XU)) return DG_ERR_INVALID_ARG;
  const long long nJ = JU ? 1 : 0;
  const long long total = nJ + (XU ? (long long)N * m : 0);
  if (m > 65535 || total > (1LL << 30)) return DG_ERR_INVALID_ARG;
  cudaStream_t us = (cudaStream_t)stream;
  DG_CK(cudaEventRecord(h->ev_in, us));
  DG_CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  cudaStream_t s = h->ws;
  const long long Nq = h->Nq;
  // solve list: the density (row index -1) for J, then psi_j u_k with j fastest
  std::vector<int> sa((size_t)total), sb((size_t)total);
  {
    size_t t = 0;
    if (JU) {
      sa[t] = -1;
      sb[t++] = 0;
    }
    if (XU)
      for (int k = 0; k < (int)m; ++k)
        for (int j = 0; j < N; ++j, ++t) {
          sa[t] = j;
          sb[t] = k;
        }
  }
  const int cap = (int)std::max<long long>(1, std::min<long long>(default_batch(h), total));
  DG_RET(prepare(h, cap));
  if (XU) DG_CK(cudaMemsetAsync(XU, 0, sizeof(double) * (size_t)m * Nq, s));
  DevBuf idx, lists;
  DG_CK(idx.ensure(sizeof(int) * 2 * (size_t)std::max<long long>(cap, m)));
  int* ia = idx.as<int>();
  int* ib = ia + std::max<long long>(cap, m);
  int worst = DG_OK;
  for (long long b0 = 0; b0 < total; b0 += cap) {
    const int nb = (int)std::min<long long>(cap, total - b0);
    DG_CK(cudaMemcpyAsync(ia, sa.data() + b0, sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    DG_CK(cudaMemcpyAsync(ib, sb.data() + b0, sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    DG_CK(launch_row_products(psi, N, U, ia, ib, nb, Nq, 1.0, h->f64.as<double>(), s));
    std::vector<int> finite;
    DG_RET(check_finite(h, h->f64.as<double>(), nb, finite, s));
    DG_RET(form_rhs(h, h->f64.as<double>(), nb, s));
    const int rc = solve_chunk(h, nb, finite, stats ? stats + b0 : nullptr, s);
    if (rc == DG_ERR_CUDA || rc == DG_ERR_NO_MEMORY) return rc;
    if (rc != DG_OK && (worst == DG_OK || rc < worst)) worst = rc;
    if (stats) {
      std::vector<double> se;
      DG_RET(self_energies(h, h->f64.as<double>(), nb, se, s));
      for (int k = 0; k < nb; ++k) stats[b0 + k].self_energy = se[k];
    }
    const double* v = h->x64.as<double>();
    std::vector<int> ja, jb;
    if (JU && b0 == 0) {
      // J u_k = v_H u_k, v_H in slot 0
      ja.assign((size_t)m, 0);
      jb.resize((size_t)m);
      for (int k = 0; k < (int)m; ++k) jb[k] = k;
      DG_CK(cudaMemcpyAsync(ia, ja.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
      DG_CK(cudaMemcpyAsync(ib, jb.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
      DG_CK(launch_row_products(v, 1, U, ia, ib, (int)m, Nq, 1.0, JU, s));
    }
    // XU_k += psi_j v_(jk) for the batch's exchange solves, per k in ascending j
    std::vector<int> ptr((size_t)m + 1, 0), eb, es;
    if (XU) {
      std::vector<std::vector<std::pair<int, int>>> per((size_t)m);
      for (int k = 0; k < nb; ++k) {
        const long long g = b0 + k;
        if (sa[g] < 0) continue;
        per[sb[g]].push_back({k, sa[g]});
      }
      for (int k = 0; k < (int)m; ++k) {
        for (auto& e : per[k]) {
          eb.push_back(e.first);
          es.push_back(e.second);
        }
        ptr[k + 1] = (int)eb.size();
      }
    }
    if (!eb.empty()) {
      std::vector<int> pack;
      pack.insert(pack.end(), ptr.begin(), ptr.end());
      pack.insert(pack.end(), eb.begin(), eb.end());
      pack.insert(pack.end(), es.begin(), es.end());
      DG_CK(lists.ensure(sizeof(int) * pack.size()));
      DG_CK(cudaMemcpyAsync(lists.p, pack.data(), sizeof(int) * pack.size(), cudaMemcpyHostToDevice, s));
      const int* dl = lists.as<int>();
      DG_CK(launch_exch_accum(psi, v, XU, dl, dl + m + 1, dl + m + 1 + eb.size(), (int)m, Nq, s));
    }
    DG_CK(cudaStreamSynchronize(s));  // the index lists are host temporaries
  }
  if (XU) DG_CK(launch_scale(XU, (long long)m * Nq, -1.0, s));
  DG_CK(cudaStreamSynchronize(s));
  DG_CK(cudaEventRecord(h->ev_out, s));
  DG_CK(cudaStreamWaitEvent(us, h->ev_out, 0));
  account(h);
  return worst;
}

}  // extern "C"
