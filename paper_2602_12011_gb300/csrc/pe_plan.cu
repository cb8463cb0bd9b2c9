// pe_plan.cu -- uneven-batch execution plans (row G3): the whole batched log-likelihood (prep,
// tile scan, persistent fused kernel, reduction) over many (detector, sample) pairs with their
// own grid lengths and active ranges, captured once into a CUDA graph with pre-allocated
// scratch, plus the project autotuner that picks the forward kernel's register-budget variant and
// persistent grid size for a workload and caches the choice in a JSON file.
//
// Tuning changes launch parameters only (never the 128-bin tile that fixes the reduction order),
// so a tuned launch gives bit-identical results to the default one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <sys/stat.h>

#include "pe_internal.h"
#include "pe_kernels.h"
#include "pe_plan.h"
#include "pespace_gb300.h"

namespace pe {
namespace {

std::mutex g_mu;
std::map<std::string, TuneChoice> g_cache;
bool g_loaded = false;

std::string cache_path() {
  const char* p = getenv("PE_TUNE_CACHE");
  if (p && *p) return p;
  const char* x = getenv("XDG_CACHE_HOME");
  if (x && *x) return std::string(x) + "/pespace_gb300/tune.json";
  const char* h = getenv("HOME");
  if (h && *h) return std::string(h) + "/.cache/pespace_gb300/tune.json";
  return "";
}

void mkdirs_for(const std::string& path) {
  for (size_t i = 1; i < path.size(); ++i)
    if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
}

// File format: one JSON object, one entry per line:  "key": {"variant": v, "ctas_per_sm": c, "ms": t},
void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    char* q0 = strchr(line, '"');
    if (!q0) continue;
    char* q1 = strchr(q0 + 1, '"');
    if (!q1) continue;
    std::string key(q0 + 1, q1 - q0 - 1);
    TuneChoice c{};
    if (sscanf(q1 + 1, ": {\"variant\": %d, \"ctas_per_sm\": %d, \"ms\": %lf", &c.variant, &c.ctas_per_sm, &c.ms) == 3 &&
        c.variant >= 0 && c.variant < kFwdVariants && c.ctas_per_sm >= 1 && c.ctas_per_sm <= 64)
      g_cache[key] = c;
  }
  fclose(f);
}

void save_locked() {
  const std::string path = cache_path();
  if (path.empty()) return;
  mkdirs_for(path);
  const std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : g_cache) {
    fprintf(f, "\"%s\": {\"variant\": %d, \"ctas_per_sm\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(), kv.second.variant,
            kv.second.ctas_per_sm, kv.second.ms, (++i < g_cache.size()) ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
}

int sm_count_now() {
  int dev = 0, n = 1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

}  // namespace

std::string tune_key(const DetSet& ds, int B, unsigned mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  char buf[256];
  std::string k;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) k = prop.name; else { cudaGetLastError(); k = "gpu"; }
  snprintf(buf, sizeof(buf), "|sm=%d|B=%d|mask=%u|nb=", sm_count_now(), B, mask);
  k += buf;
  for (int i = 0; i < ds.ndet; ++i) {
    snprintf(buf, sizeof(buf), "%s%d@%lld", i ? "," : "", ds.d[i].nb, ds.d[i].k0);
    k += buf;
  }
  for (char& c : k)
    if (c == '"' || c == '\\' || c == '\n') c = '_';
  return k;
}

bool lookup_tuned(const DetSet& ds, int B, unsigned mask, TuneChoice* out) {
  const std::string key = tune_key(ds, B, mask);
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  *out = it->second;
  return true;
}

TuneChoice default_choice() { return TuneChoice{kFwdDefaultVariant, 8, 0.0}; }

int grid_for(const TuneChoice& c, long long max_tiles) {
  const long long g = std::min<long long>(max_tiles, (long long)sm_count_now() * c.ctas_per_sm);
  return (int)std::max<long long>(g, 1);
}

// Times every (variant, CTAs per SM) candidate of the forward kernel on the prepared work list
// (coefficients, active counts and tile offsets already on the device) and returns the fastest.
cudaError_t autotune_fwd(const DetSet& ds, int B, unsigned mask, const SampleCoef* coef, const int* nend,
                         const long long* off, double* part, long long max_tiles, cudaStream_t st, TuneChoice* best) {
  static const int kCtas[] = {2, 4, 8, 16};
  const int prec = mask_prec(mask);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  TuneChoice b{-1, 0, 1e30};
  for (int v = 0; v < kFwdVariants && e == cudaSuccess; ++v) {
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
      TuneChoice c{v, kCtas[ci], 0.0};
      const int grid = grid_for(c, max_tiles);
      if ((e = launch_loglike_fwd_variant(v, prec, ds, B, coef, nend, off, part, grid, st)) != cudaSuccess) break;  // warm
      float best_ms = 1e30f;
      for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        e = launch_loglike_fwd_variant(v, prec, ds, B, coef, nend, off, part, grid, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        best_ms = std::min(best_ms, ms);
      }
      if (e == cudaSuccess && best_ms < b.ms) { b = c; b.ms = best_ms; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  *best = b;
  return cudaSuccess;
}

void store_tuned(const DetSet& ds, int B, unsigned mask, const TuneChoice& c) {
  const std::string key = tune_key(ds, B, mask);
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  g_cache[key] = c;
  save_locked();
}

}  // namespace pe

// ------------------------------------------------------------------------------------------
// Plans
// ------------------------------------------------------------------------------------------
struct pe_plan_s {
  pe::DetSet ds;
  int B;
  unsigned mask;
  void* scratch;
  pe::TuneChoice choice;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

namespace {
bool dev_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

extern "C" {

pe_status pe_plan_create(const pe_detector* dets, int ndet, int B, unsigned mode_mask, const double* theta_dev,
                         double* out_logl_dev, double* out_dhhh_dev, int32_t* out_status_dev, int autotune,
                         pe_plan* out) {
  if (out == nullptr) return pe::set_error(PE_EINVAL, "pe_plan_create: out is NULL");
  *out = nullptr;
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (B < 1 || B > (1 << 20)) return pe::set_error(PE_EINVAL, "pe_plan_create: B outside [1, 2^20]");
  if (!pe::fwd_mask_ok(mode_mask)) return pe::set_error(PE_EINVAL, "pe_plan_create: bad mode mask");
  if (!dev_ptr(theta_dev) || !dev_ptr(out_logl_dev) || (out_dhhh_dev && !dev_ptr(out_dhhh_dev)) ||
      (out_status_dev && !dev_ptr(out_status_dev)))
    return pe::set_error(PE_EINVAL, "pe_plan_create: theta and outputs must be device pointers");
  const size_t P = (size_t)ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * pe::tiles_of(ds.d[i].nb, pe::fwd_tile_bins(pe::mask_prec(mode_mask)));
  const size_t o_nend = a256((size_t)B * sizeof(pe::SampleCoef));
  const size_t o_off = a256(o_nend + P * sizeof(int));
  const size_t o_part = a256(o_off + (P + 1) * sizeof(long long));
  const size_t bytes = o_part + (size_t)max_tiles * 6 * sizeof(double);
  pe_plan_s* pl = new (std::nothrow) pe_plan_s();
  if (!pl) return pe::set_error(PE_ENOMEM, "pe_plan_create: host allocation failed");
  pl->ds = ds;
  pl->B = B;
  pl->mask = mode_mask;
  if (cudaMalloc(&pl->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return pe::set_error(PE_ENOMEM, "pe_plan_create: scratch allocation failed");
  }
  unsigned char* sc = static_cast<unsigned char*>(pl->scratch);
  pe::SampleCoef* coef = reinterpret_cast<pe::SampleCoef*>(sc);
  int* nend = reinterpret_cast<int*>(sc + o_nend);
  long long* off = reinterpret_cast<long long*>(sc + o_off);
  double* part = reinterpret_cast<double*>(sc + o_part);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  pl->choice = pe::default_choice();
  if (e == cudaSuccess && !pe::lookup_tuned(ds, B, mode_mask, &pl->choice) && autotune) {
    e = pe::launch_prep(theta_dev, B, mode_mask, ds, coef, nend, nullptr, cs);
    if (e == cudaSuccess) e = pe::launch_scan_tiles(nend, (int)P, off, pe::fwd_tile_bins(pe::mask_prec(mode_mask)), cs);
    pe::TuneChoice best;
    if (e == cudaSuccess) e = pe::autotune_fwd(ds, B, mode_mask, coef, nend, off, part, max_tiles, cs, &best);
    if (e == cudaSuccess) {
      pl->choice = best;
      pe::store_tuned(ds, B, mode_mask, best);
    }
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = pe::launch_prep(theta_dev, B, mode_mask, ds, coef, nend, out_status_dev, cs);
    if (e1 == cudaSuccess) e1 = pe::launch_scan_tiles(nend, (int)P, off, pe::fwd_tile_bins(pe::mask_prec(mode_mask)), cs);
    if (e1 == cudaSuccess)
      e1 = pe::launch_loglike_fwd_variant(pl->choice.variant, pe::mask_prec(mode_mask), ds, B, coef, nend, off, part,
                                          pe::grid_for(pl->choice, max_tiles), cs);
    if (e1 == cudaSuccess) e1 = pe::launch_reduce(ds, B, off, part, coef, out_logl_dev, out_dhhh_dev, cs);
    e = cudaStreamEndCapture(cs, &pl->graph);
    if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (pl->graph) cudaGraphDestroy(pl->graph);
    cudaFree(pl->scratch);
    delete pl;
    char msg[256];
    snprintf(msg, sizeof(msg), "pe_plan_create: %s", cudaGetErrorString(e));
    return pe::set_error(PE_ECUDA, msg);
  }
  *out = pl;
  return PE_OK;
}

pe_status pe_plan_launch(pe_plan plan, void* stream) {
  if (plan == nullptr) return pe::set_error(PE_EINVAL, "pe_plan_launch: plan is NULL");
  cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof(msg), "pe_plan_launch: %s", cudaGetErrorString(e));
    return pe::set_error(PE_ECUDA, msg);
  }
  return PE_OK;
}

pe_status pe_plan_info(pe_plan plan, int* fwd_variant, int* ctas_per_sm, double* tuned_ms) {
  if (plan == nullptr) return pe::set_error(PE_EINVAL, "pe_plan_info: plan is NULL");
  if (fwd_variant) *fwd_variant = plan->choice.variant;
  if (ctas_per_sm) *ctas_per_sm = plan->choice.ctas_per_sm;
  if (tuned_ms) *tuned_ms = plan->choice.ms;
  return PE_OK;
}

pe_status pe_autotune(const pe_detector* dets, int ndet, const double* theta_dev, int B, unsigned mode_mask,
                      int* out_variant, int* out_ctas_per_sm, double* out_ms) {
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (B < 1 || B > (1 << 20)) return pe::set_error(PE_EINVAL, "pe_autotune: B outside [1, 2^20]");
  if (!pe::fwd_mask_ok(mode_mask)) return pe::set_error(PE_EINVAL, "pe_autotune: bad mode mask");
  if (!dev_ptr(theta_dev)) return pe::set_error(PE_EINVAL, "pe_autotune: theta must be a device pointer");
  const size_t P = (size_t)ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * pe::tiles_of(ds.d[i].nb, pe::fwd_tile_bins(pe::mask_prec(mode_mask)));
  const size_t o_nend = a256((size_t)B * sizeof(pe::SampleCoef));
  const size_t o_off = a256(o_nend + P * sizeof(int));
  const size_t o_part = a256(o_off + (P + 1) * sizeof(long long));
  const size_t bytes = o_part + (size_t)max_tiles * 6 * sizeof(double);
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return pe::set_error(PE_ENOMEM, "pe_autotune: scratch allocation failed");
  }
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  pe::SampleCoef* coef = reinterpret_cast<pe::SampleCoef*>(sc);
  int* nend = reinterpret_cast<int*>(sc + o_nend);
  long long* off = reinterpret_cast<long long*>(sc + o_off);
  double* part = reinterpret_cast<double*>(sc + o_part);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  pe::TuneChoice best = pe::default_choice();
  if (e == cudaSuccess) e = pe::launch_prep(theta_dev, B, mode_mask, ds, coef, nend, nullptr, cs);
  if (e == cudaSuccess) e = pe::launch_scan_tiles(nend, (int)P, off, pe::fwd_tile_bins(pe::mask_prec(mode_mask)), cs);
  if (e == cudaSuccess) e = pe::autotune_fwd(ds, B, mode_mask, coef, nend, off, part, max_tiles, cs, &best);
  if (cs) cudaStreamDestroy(cs);
  cudaFree(scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof(msg), "pe_autotune: %s", cudaGetErrorString(e));
    return pe::set_error(PE_ECUDA, msg);
  }
  pe::store_tuned(ds, B, mode_mask, best);
  if (out_variant) *out_variant = best.variant;
  if (out_ctas_per_sm) *out_ctas_per_sm = best.ctas_per_sm;
  if (out_ms) *out_ms = best.ms;
  return PE_OK;
}

pe_status pe_plan_destroy(pe_plan plan) {
  if (plan == nullptr) return PE_OK;
  cudaDeviceSynchronize();
  cudaGraphExecDestroy(plan->exec);
  cudaGraphDestroy(plan->graph);
  cudaFree(plan->scratch);
  cudaGetLastError();
  delete plan;
  return PE_OK;
}

}  // extern "C"
