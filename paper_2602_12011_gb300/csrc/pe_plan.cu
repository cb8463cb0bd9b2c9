// pe_plan.cu -- uneven-batch execution plans (row G3): the whole batched log-likelihood (prep,
// tile scan, persistent fused kernel, reduction) over many (detector, sample) pairs with their
// own grid lengths and active ranges, captured once into a CUDA graph with pre-allocated
// scratch, plus the project autotuner that picks the forward kernel's work-item size (128-bin
// sub-tiles per item), register-budget variant and persistent grid size for a workload and
// caches the choice in a JSON file.
//
// Every choice keeps one partial per 128-bin sub-tile in the same fixed reduction order, so a
// tuned launch gives bit-identical results to the default one.
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
#include "pe_fault.h"

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

// File format: one JSON object, one entry per line:
//   "key": {"variant": v, "ctas_per_sm": c, "subtiles": r, "ms": t},
// (entries without "subtiles" are from an earlier format and are ignored, so they are re-tuned)
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
    if (sscanf(q1 + 1, ": {\"variant\": %d, \"ctas_per_sm\": %d, \"subtiles\": %d, \"ms\": %lf", &c.variant,
               &c.ctas_per_sm, &c.subtiles, &c.ms) == 4 &&
        c.variant >= 0 && c.variant < kFwdVariants && c.ctas_per_sm >= 1 && c.ctas_per_sm <= 64 &&
        (c.subtiles == 1 || c.subtiles == 2 || c.subtiles == 4 || c.subtiles == 8))
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
    fprintf(f, "\"%s\": {\"variant\": %d, \"ctas_per_sm\": %d, \"subtiles\": %d, \"ms\": %.6f}%s\n",
            kv.first.c_str(), kv.second.variant, kv.second.ctas_per_sm, kv.second.subtiles, kv.second.ms,
            (++i < g_cache.size()) ? "," : "");
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

TuneChoice default_choice(int prec) { return TuneChoice{kFwdDefaultVariant, 8, fwd_default_subtiles(prec), 0.0}; }

int grid_for(const TuneChoice& c, long long max_tiles) {
  const long long g = std::min<long long>(max_tiles, (long long)sm_count_now() * c.ctas_per_sm);
  return (int)std::max<long long>(g, 1);
}

// Two stages on the prepared work list: every (register-budget variant, CTAs per SM) at the
// precision's default sub-tiles per item, then every sub-tile count (1, 2, 4, 8) at the best of
// those. Each candidate: one warm launch, the best of two timed ones.
cudaError_t autotune_fwd(const DetSet& ds, int B, unsigned mask, const SampleCoef* coef, const int* nend,
                         const long long* off, long long* offi, double* part, long long max_tiles, cudaStream_t st,
                         TuneChoice* best) {
  static const int kCtas[] = {2, 4, 8, 16};
  static const int kSub[] = {1, 2, 4, 8};
  const int prec = mask_prec(mask);
  const int P = ds.ndet * B;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  auto time_one = [&](const TuneChoice& c, float* out_ms) -> cudaError_t {
    const int grid = grid_for(c, max_tiles);
    cudaError_t r = cudaSuccess;
    if (c.subtiles > 1) r = launch_scan_tiles(nend, P, offi, c.subtiles * kTileBins, st);
    if (r == cudaSuccess)
      r = launch_loglike_fwd_variant(c.variant, prec, ds, B, coef, nend, off, offi, c.subtiles, part, grid, st);  // warm
    float bm = 1e30f;
    for (int k = 0; k < 2 && r == cudaSuccess; ++k) {
      cudaEventRecord(e0, st);
      r = launch_loglike_fwd_variant(c.variant, prec, ds, B, coef, nend, off, offi, c.subtiles, part, grid, st);
      cudaEventRecord(e1, st);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
      bm = std::min(bm, ms);
    }
    *out_ms = bm;
    return r;
  };
  TuneChoice b{-1, 0, fwd_default_subtiles(prec), 1e30};
  for (int v = 0; v < kFwdVariants && e == cudaSuccess; ++v)
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
      TuneChoice c{v, kCtas[ci], fwd_default_subtiles(prec), 0.0};
      float ms = 0.f;
      e = time_one(c, &ms);
      if (e == cudaSuccess && ms < b.ms) { b = c; b.ms = ms; }
    }
  const int r0 = b.subtiles;
  for (int si = 0; si < 4 && e == cudaSuccess; ++si) {
    if (kSub[si] == r0) continue;
    TuneChoice c = b;
    c.subtiles = kSub[si];
    float ms = 0.f;
    e = time_one(c, &ms);
    if (e == cudaSuccess && ms < b.ms) { b = c; b.ms = ms; }
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
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * pe::tiles_of(ds.d[i].nb, pe::kTileBins);
  const size_t o_nend = a256((size_t)B * sizeof(pe::SampleCoef));
  const size_t o_off = a256(o_nend + P * sizeof(int));
  const size_t o_offi = a256(o_off + (P + 1) * sizeof(long long));
  const size_t o_part = a256(o_offi + (P + 1) * sizeof(long long));
  const size_t bytes = o_part + (size_t)max_tiles * 6 * sizeof(double);
  pe_plan_s* pl = new (std::nothrow) pe_plan_s();
  if (!pl) return pe::set_error(PE_ENOMEM, "pe_plan_create: host allocation failed");
  pl->ds = ds;
  pl->B = B;
  pl->mask = mode_mask;
  if (pe::dmalloc(&pl->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return pe::set_error(PE_ENOMEM, "pe_plan_create: scratch allocation failed");
  }
  unsigned char* sc = static_cast<unsigned char*>(pl->scratch);
  pe::SampleCoef* coef = reinterpret_cast<pe::SampleCoef*>(sc);
  int* nend = reinterpret_cast<int*>(sc + o_nend);
  long long* off = reinterpret_cast<long long*>(sc + o_off);
  long long* offi = reinterpret_cast<long long*>(sc + o_offi);
  double* part = reinterpret_cast<double*>(sc + o_part);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  pl->choice = pe::default_choice(pe::mask_prec(mode_mask));
  if (e == cudaSuccess && !pe::lookup_tuned(ds, B, mode_mask, &pl->choice) && autotune) {
    e = pe::launch_prep(theta_dev, B, mode_mask, ds, coef, nend, nullptr, cs);
    if (e == cudaSuccess) e = pe::launch_scan_tiles(nend, (int)P, off, pe::kTileBins, cs);
    pe::TuneChoice best;
    if (e == cudaSuccess) e = pe::autotune_fwd(ds, B, mode_mask, coef, nend, off, offi, part, max_tiles, cs, &best);
    if (e == cudaSuccess) {
      pl->choice = best;
      pe::store_tuned(ds, B, mode_mask, best);
    }
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = pe::launch_prep(theta_dev, B, mode_mask, ds, coef, nend, out_status_dev, cs);
    if (e1 == cudaSuccess) e1 = pe::launch_fwd_offsets(nend, (int)P, off, offi, pl->choice.subtiles, cs);
    if (e1 == cudaSuccess)
      e1 = pe::launch_loglike_fwd_variant(pl->choice.variant, pe::mask_prec(mode_mask), ds, B, coef, nend, off, offi,
                                          pl->choice.subtiles, part, pe::grid_for(pl->choice, max_tiles), cs);
    if (e1 == cudaSuccess) e1 = pe::launch_reduce(ds, B, off, part, coef, out_logl_dev, out_dhhh_dev, cs);
    e = cudaStreamEndCapture(cs, &pl->graph);
    if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pe::dfree(pl->scratch);
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

pe_status pe_plan_info(pe_plan plan, int* fwd_variant, int* ctas_per_sm, int* subtiles, double* tuned_ms) {
  if (plan == nullptr) return pe::set_error(PE_EINVAL, "pe_plan_info: plan is NULL");
  if (fwd_variant) *fwd_variant = plan->choice.variant;
  if (ctas_per_sm) *ctas_per_sm = plan->choice.ctas_per_sm;
  if (subtiles) *subtiles = plan->choice.subtiles;
  if (tuned_ms) *tuned_ms = plan->choice.ms;
  return PE_OK;
}

pe_status pe_tune_set(const pe_detector* dets, int ndet, int B, unsigned mode_mask, int fwd_variant, int ctas_per_sm,
                      int subtiles) {
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (B < 1 || B > (1 << 20)) return pe::set_error(PE_EINVAL, "pe_tune_set: B outside [1, 2^20]");
  if (!pe::fwd_mask_ok(mode_mask)) return pe::set_error(PE_EINVAL, "pe_tune_set: bad mode mask");
  if (fwd_variant < 0 || fwd_variant >= pe::kFwdVariants || ctas_per_sm < 1 || ctas_per_sm > 64 ||
      (subtiles != 1 && subtiles != 2 && subtiles != 4 && subtiles != 8))
    return pe::set_error(PE_EINVAL, "pe_tune_set: choice out of range");
  pe::store_tuned(ds, B, mode_mask, pe::TuneChoice{fwd_variant, ctas_per_sm, subtiles, 0.0});
  return PE_OK;
}

pe_status pe_autotune(const pe_detector* dets, int ndet, const double* theta_dev, int B, unsigned mode_mask,
                      int* out_variant, int* out_ctas_per_sm, int* out_subtiles, double* out_ms) {
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (B < 1 || B > (1 << 20)) return pe::set_error(PE_EINVAL, "pe_autotune: B outside [1, 2^20]");
  if (!pe::fwd_mask_ok(mode_mask)) return pe::set_error(PE_EINVAL, "pe_autotune: bad mode mask");
  if (!dev_ptr(theta_dev)) return pe::set_error(PE_EINVAL, "pe_autotune: theta must be a device pointer");
  const size_t P = (size_t)ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * pe::tiles_of(ds.d[i].nb, pe::kTileBins);
  const size_t o_nend = a256((size_t)B * sizeof(pe::SampleCoef));
  const size_t o_off = a256(o_nend + P * sizeof(int));
  const size_t o_offi = a256(o_off + (P + 1) * sizeof(long long));
  const size_t o_part = a256(o_offi + (P + 1) * sizeof(long long));
  const size_t bytes = o_part + (size_t)max_tiles * 6 * sizeof(double);
  void* scratch = nullptr;
  if (pe::dmalloc(&scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return pe::set_error(PE_ENOMEM, "pe_autotune: scratch allocation failed");
  }
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  pe::SampleCoef* coef = reinterpret_cast<pe::SampleCoef*>(sc);
  int* nend = reinterpret_cast<int*>(sc + o_nend);
  long long* off = reinterpret_cast<long long*>(sc + o_off);
  long long* offi = reinterpret_cast<long long*>(sc + o_offi);
  double* part = reinterpret_cast<double*>(sc + o_part);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  pe::TuneChoice best = pe::default_choice(pe::mask_prec(mode_mask));
  if (e == cudaSuccess) e = pe::launch_prep(theta_dev, B, mode_mask, ds, coef, nend, nullptr, cs);
  if (e == cudaSuccess) e = pe::launch_scan_tiles(nend, (int)P, off, pe::kTileBins, cs);
  if (e == cudaSuccess) e = pe::autotune_fwd(ds, B, mode_mask, coef, nend, off, offi, part, max_tiles, cs, &best);
  if (cs) cudaStreamDestroy(cs);
  pe::dfree(scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof(msg), "pe_autotune: %s", cudaGetErrorString(e));
    return pe::set_error(PE_ECUDA, msg);
  }
  pe::store_tuned(ds, B, mode_mask, best);
  if (out_variant) *out_variant = best.variant;
  if (out_ctas_per_sm) *out_ctas_per_sm = best.ctas_per_sm;
  if (out_subtiles) *out_subtiles = best.subtiles;
  if (out_ms) *out_ms = best.ms;
  return PE_OK;
}

pe_status pe_plan_destroy(pe_plan plan) {
  if (plan == nullptr) return PE_OK;
  cudaDeviceSynchronize();
  cudaGraphExecDestroy(plan->exec);
  cudaGraphDestroy(plan->graph);
  pe::dfree(plan->scratch);
  cudaGetLastError();
  delete plan;
  return PE_OK;
}

}  // extern "C"
