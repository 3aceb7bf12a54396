// Exchange builds of many independent systems of uneven sizes in one call
// (dg_exchange_build_multi) and the autotuner that picks the source-batch
// size of each mesh.
//
// GB300 layout of the work: systems are sorted by estimated cost (pair count
// times nodes) and pulled from a shared queue by `lanes` host threads; each
// lane owns one handle per mesh (cached across calls), and each handle runs
// on its own non-blocking stream with its PCG phases replayed as CUDA graphs,
// so the kernels of small systems from different lanes overlap on the GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <sys/stat.h>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dg_ctx.h"

namespace dg {

// ---------------------------------------------------------------------------
// autotuner: source-batch size per (n, p, precision)
// ---------------------------------------------------------------------------
struct TuneEntry {
  int batch = 0;
  double us_per_source = 0.0;
  int tc_np = -1;  // fine-level patch solve: patches per tensor-core item, 0 = SIMT kernel, -1 = not tuned
};

static std::mutex g_tune_mu;
static std::map<std::string, TuneEntry> g_tune;
static bool g_tune_loaded = false;

static std::string tune_path() {
  const char* p = std::getenv("DG_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/dgx_autotune.jsonl";
}

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE* f = std::fopen(tune_path().c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char key[256];
    int batch = 0, tc_np = -1;
    double us = 0.0;
    // {"key": "...", "batch": B, "us_per_source": U, "tc_np": P}
    const int got = std::sscanf(line, " {\"key\": \"%255[^\"]\", \"batch\": %d, \"us_per_source\": %lf, \"tc_np\": %d",
                                key, &batch, &us, &tc_np);
    if (got >= 3 && batch > 0) g_tune[key] = TuneEntry{batch, us, got == 4 ? tc_np : -1};
  }
  std::fclose(f);
}

static void tune_store_locked() {
  const std::string path = tune_path();
  const size_t cut = path.find_last_of('/');
  if (cut != std::string::npos && cut > 0) mkdir(path.substr(0, cut).c_str(), 0755);  // one level, may exist
  FILE* f = std::fopen(path.c_str(), "w");
  if (!f) return;  // cache is an optimisation only
  for (const auto& kv : g_tune)
    std::fprintf(f, "{\"key\": \"%s\", \"batch\": %d, \"us_per_source\": %.6g, \"tc_np\": %d}\n", kv.first.c_str(),
                 kv.second.batch, kv.second.us_per_source, kv.second.tc_np);
  std::fclose(f);
}

static std::string tune_key(const dg_ctx* h) {
  char buf[160];
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::snprintf(buf, sizeof(buf), "%s|n%dx%dx%d|p%d|prec%d|sm%d|cp%d", prop.name, h->mesh.n[0], h->mesh.n[1],
                h->mesh.n[2], h->mesh.p, h->opts.precision, h->opts.smoother, h->opts.coarse_penalty);
  return buf;
}

// Times one fine-level operator application plus one smoother application
// on B fields in the solve precision; returns microseconds per field.
template <typename T>
static double probe_us_per_source(dg_ctx* h, PrecWork<T>& w, int B, cudaStream_t s) {
  const Level& L = h->levels[0];
  std::vector<int> a(B);
  for (int k = 0; k < B; ++k) a[k] = k;
  if (upload_act(h, a, s) != DG_OK) return 1e300;
  const int* dact = h->act.as<int>();
  T* u = w.p.template as<T>();
  T* out = w.q.template as<T>();
  cudaMemsetAsync(u, 0, sizeof(T) * h->Nq * B, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto once = [&]() {
    launch_apply<T>(L.op, L.dop, 0, u, out, nullptr, dact, B, s);
    if (h->nlev > 1 && h->opts.smoother == DG_SMOOTH_SCHWARZ)
      launch_schwarz<T>(L.op, L.dop, L.sw_tabs.as<double>(), out, w.lev[0].zp.template as<T>(), u, nullptr, 0, 0.0,
                        0.0, dact, B, s, L.tc());
  };
  once();
  cudaEventRecord(e0, s);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) once();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 1000.0 * ms / reps / B;
}

// Applies a tuned patch-solve variant to the fine level: np > 0 tensor-core
// items of np patches, 0 the SIMT kernel (no change without a tensor-core plan).
static void apply_tc_choice(dg_ctx* h, int np) {
  SwTcPlan& P = h->levels[0].tcp;
  if (!P.blob || np < 0) return;
  ++h->buf_gen;  // captured PCG phases embed the old variant: capture again
  SwTcGeom g;
  if (np == 0) {
    P.off = true;
  } else if (swtc_geometry(h->levels[0].op.n1, g, np)) {
    P.geom = g;
    P.off = false;
  }
}

// Tile shape of the fine level's tensor-core patch solve (patches per work
// item, i.e. the MMA width N), timed at batch B with the operator + smoother
// probe; the fastest is kept. The shape does not change any result (every
// output element is the same sum in the same order whatever the item size),
// so tuned and untuned builds agree exactly; the switch to the SIMT kernel,
// which changes the rounding, is left to the caller (tc_smoother). -1 without
// a plan.
static int autotune_tc(dg_ctx* h, int B, cudaStream_t s) {
  SwTcPlan& P = h->levels[0].tcp;
  if (!P.blob || P.off || h->opts.precision == DG_PREC_FP64) return -1;
  const SwTcGeom keep = P.geom;
  std::vector<int> cand;
  for (int np : {2, 4, 6, 8, 10}) {
    SwTcGeom g;
    if (swtc_geometry(h->levels[0].op.n1, g, np)) cand.push_back(np);
  }
  int pick = keep.np;
  double best = 1e300;
  for (int np : cand) {
    apply_tc_choice(h, np);
    const double t = probe_us_per_source<float>(h, h->w32, B, s);
    if (t < best) {
      best = t;
      pick = np;
    }
  }
  P.geom = keep;
  P.off = false;
  apply_tc_choice(h, pick);
  return pick;
}

// Batch size for a handle: the smallest candidate whose per-source time is
// within 10 % of the best candidate's (bigger batches cost memory and leave
// fewer sources for other lanes), then the fine level's patch-solve variant.
// Results cached per device name and mesh.
int autotune_batch(dg_ctx* h, int max_sources, cudaStream_t s) {
  const std::string key = tune_key(h);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      apply_tc_choice(h, it->second.tc_np);
      return std::min(it->second.batch, std::max(1, max_sources));
    }
  }
  // candidates bounded by memory: about 2 GB of fine-level vectors per handle
  const long long per_source = h->Nq * 8LL * 16;
  const int mem_cap = (int)std::max(1LL, std::min(512LL, (2LL << 30) / std::max(per_source, 1LL)));
  std::vector<int> cand;
  for (int b : {8, 16, 32, 64, 128, 256, 512})
    if (b <= mem_cap) cand.push_back(b);
  if (cand.empty()) cand.push_back(std::max(1, mem_cap));
  const int bmax = cand.back();
  if (ensure_common(h, bmax) != DG_OK) return std::max(1, std::min(bmax, max_sources));
  double best = 1e300;
  std::vector<double> t(cand.size(), 1e300);
  const bool f32 = h->opts.precision != DG_PREC_FP64;
  if ((f32 ? ensure_prec<float>(h, h->w32, bmax) : ensure_prec<double>(h, h->w64, bmax)) != DG_OK)
    return std::max(1, std::min(bmax, max_sources));
  for (size_t i = 0; i < cand.size(); ++i) {
    t[i] = f32 ? probe_us_per_source<float>(h, h->w32, cand[i], s) : probe_us_per_source<double>(h, h->w64, cand[i], s);
    best = std::min(best, t[i]);
  }
  int pick = bmax;
  double pick_t = best;
  for (size_t i = 0; i < cand.size(); ++i)
    if (t[i] <= 1.10 * best) {
      pick = cand[i];
      pick_t = t[i];
      break;
    }
  const int tc_np = f32 ? autotune_tc(h, pick, s) : -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = TuneEntry{pick, pick_t, tc_np};
    tune_store_locked();
  }
  return std::min(pick, std::max(1, max_sources));
}

// ---------------------------------------------------------------------------
// handle cache for the multi-system builds: one handle per (mesh, options, lane)
// ---------------------------------------------------------------------------
static std::mutex g_cache_mu;
static std::map<std::string, dg_ctx*> g_cache;

static std::string cache_key(const dg_mesh_desc& m, const dg_solver_opts& o, int lane) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%.17g,%.17g,%.17g,%.17g,%.17g,%.17g|%d,%d,%d|%d|%d,%.17g,%d,%.17g,%d,%d,%.17g,%d,%d,"
                "%.17g,%.17g,%d,%d,%d,%d|%d",
                m.lo[0], m.lo[1], m.lo[2], m.hi[0], m.hi[1], m.hi[2], m.n[0], m.n[1], m.n[2], m.p, o.precision, o.rtol,
                o.max_iter, o.penalty_eps, o.penalty_form, o.bc_route, o.bc_tol, o.smoother, o.smoother_degree,
                o.cheb_range, o.inner_rtol, o.coarse_penalty, o.coarse_smoother_degree, o.p1_smoother, o.gauss_construction, lane);
  std::string k(buf);
  if (o.nn_weights_path) k += std::string("|") + o.nn_weights_path;
  return k;
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_exchange_build_multi(const dg_mesh_desc* meshes, const double* const* psi_devs, const int32_t* Ns,
                            int32_t nsys, const dg_solver_opts* opts, double* const* K_hosts, double* E_H,
                            double* E_X, dg_solve_stats* const* stats_hosts, int32_t lanes, void* cuda_stream) {
  if (!meshes || !psi_devs || !Ns || nsys < 0 || !K_hosts) return DG_ERR_INVALID_ARG;
  if (nsys == 0) return DG_OK;
  dg_solver_opts o;
  if (opts)
    o = *opts;
  else
    dg_default_opts(&o);
  for (int i = 0; i < nsys; ++i)
    if (!psi_devs[i] || Ns[i] < 1 || !K_hosts[i]) return DG_ERR_INVALID_ARG;
  if (lanes <= 0) lanes = 4;
  lanes = std::min(lanes, nsys);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  // most expensive systems first
  std::vector<int> order(nsys);
  for (int i = 0; i < nsys; ++i) order[i] = i;
  auto cost = [&](int i) {
    const double nq = (double)meshes[i].n[0] * meshes[i].n[1] * meshes[i].n[2] * std::pow(meshes[i].p + 1, 3);
    return nq * Ns[i] * (Ns[i] + 1) / 2.0;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::atomic<int> next{0};
  std::atomic<int> worst{DG_OK};
  auto lane_fn = [&](int lane) {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nsys) break;
      const int i = order[k];
      dg_ctx* h = nullptr;
      const std::string key = cache_key(meshes[i], o, lane);
      {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) h = it->second;
      }
      if (!h) {
        dg_handle nh = nullptr;
        const int rc = dg_poisson_setup(&meshes[i], &o, &nh);
        if (rc != DG_OK) {
          int w = worst.load();
          while ((w == DG_OK || rc < w) && !worst.compare_exchange_weak(w, rc)) {
          }
          continue;
        }
        h = nh;
        if (o.batch <= 0) h->opts.batch = autotune_batch(h, Ns[i] * (Ns[i] + 1) / 2 + 1, h->ws);
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cache[key] = h;
      }
      const int rc = dg_exchange_build(h, psi_devs[i], Ns[i], K_hosts[i], E_H ? &E_H[i] : nullptr,
                                       E_X ? &E_X[i] : nullptr, stats_hosts ? stats_hosts[i] : nullptr, cuda_stream);
      if (rc != DG_OK) {
        int w = worst.load();
        while ((w == DG_OK || rc < w) && !worst.compare_exchange_weak(w, rc)) {
        }
      }
    }
  };
  std::vector<std::thread> th;
  for (int l = 1; l < lanes; ++l) th.emplace_back(lane_fn, l);
  lane_fn(0);
  for (auto& t : th) t.join();
  return worst.load();
}

void dg_release_cached_handles(void) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto& kv : g_cache) dg_destroy(kv.second);
  g_cache.clear();
}

int dg_autotune_batch(dg_handle h, int32_t max_sources, int32_t* batch) {
  if (!h || !batch) return DG_ERR_INVALID_ARG;
  *batch = autotune_batch(h, max_sources > 0 ? max_sources : 1 << 20, h->ws);
  h->opts.batch = *batch;
  return DG_OK;
}

}  // extern "C"
