// pe_api.cu -- host implementation of the C ABI in include/pespace_gb300.h: detector handles,
// argument validation, pointer-kind handling, stream-ordered scratch and kernel launches.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <thread>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <string>
#include <vector>

#include "pe_internal.h"
#include "pe_grad.h"
#include "pe_kernels.h"
#include "pe_measure.h"
#include "pe_plan.h"
#include "pespace_gb300.h"
#include "pe_fault.h"

struct pe_detector_s {
  int device;
  pe_detector_config cfg;
  double T;
  long long k0;
  int nb;
  void* mem;           // one allocation for every per-bin table
  double* f;
  double* f13;
  double* fm13;
  double* lnf3;
  double* fm76;
  double* fpow;        // [3][nb] f^(-5/6), f^(-1/2), f^(-5/3)
  double2* sca;
  double2* z;
  double2* dg;
  double* gg;
  double* psd_model;   // [3][nb] analytic PSD
  double* dd_dev;      // [3]
  double2* sct;        // [kSinTab] sincos table
  float4* sctw;        // [kSinTab] the same as double words
  float2* fw;          // [nb] double words of f, pi f L, f L / 2, sin(pi f L), cos(pi f L)
  float2* aw;
  float2* atw;
  float2* saw;
  float2* caw;
  float2* f13w;        // [nb] f^(1/3), f^(-7/6) as double words
  float2* fm76w;
  float4* zw;          // [nb] z as a double-word pair
  float4* dgw;         // [3][nb] dg / dg_scale as double words
  float2* ggw;         // [3][nb] gg / gg_scale as double words
  float* f32;          // [5][nb] FP32 f, f^(1/3), f^(-1/3), ln f/3, f^(-7/6) (precision study)
  float2* scaf;        // [nb] FP32 (sin a, cos a), z, then dg / dg_scale [3][nb]
  float2* zf;
  float2* dgf;
  float* ggf;          // [3][nb] FP32 gg / gg_scale
  double dd[3];
  int has_data;
  pe::DetDev dev;
};

namespace {

thread_local std::string g_err;

pe_status fail(pe_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define PE_CUDA(call)                                                                             \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(PE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Bounded wait for the call's stream before host outputs are read (PE_ETIMEOUT past the limit).
#define PE_WAIT(st)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = pe::wait_stream(st);                                                            \
    if (e_ == cudaErrorNotReady)                                                                     \
      return fail(PE_ETIMEOUT, "stream did not finish within %g s; the work stays queued",          \
                  pe_get_wait_limit());                                                              \
    if (e_ != cudaSuccess) return fail(PE_ECUDA, "stream wait failed: %s", cudaGetErrorString(e_)); \
  } while (0)

// Where a caller's buffer lives: host memory (pageable or pinned), memory the current device can
// use directly (its own device memory, or managed memory), or another device's memory.
enum PtrKind { kPtrHost = 0, kPtrDevice = 1, kPtrOtherDevice = 2 };
PtrKind ptr_kind(const void* p) {
  if (p == nullptr) return kPtrHost;
  int dev = -1;
  cudaPointerAttributes a;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kPtrHost;
  }
  if (a.type == cudaMemoryTypeManaged) return kPtrDevice;
  if (a.type == cudaMemoryTypeDevice) return a.device == dev ? kPtrDevice : kPtrOtherDevice;
  return kPtrHost;
}
bool is_device_ptr(const void* p) { return ptr_kind(p) == kPtrDevice; }
// PE_EINVAL (with a message) if any of the caller's buffers is another device's memory
pe_status check_local(const char* who, std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs)
    if (ptr_kind(p) == kPtrOtherDevice)
      return fail(PE_EINVAL, "%s: a buffer lives on another device than the current one", who);
  return PE_OK;
}

std::once_flag g_pool_once;
void setup_pool() {
  std::call_once(g_pool_once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long thr = ~0ull;  // keep freed blocks cached in the pool
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

// Stream-ordered scratch for one call: every buffer is released on the call's stream.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> bufs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* p : bufs) pe::dfree_async(p, st);
  }
  template <class T>
  cudaError_t alloc(T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = pe::dmalloc_async(&q, n * sizeof(T) + 16, st);
    if (e != cudaSuccess) return e;
    bufs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
};

double det_arm_s(const pe_detector_config& c) { return c.arm_m / pe::kC; }

// double -> double word (hi = nearest float, lo = nearest float of the remainder)
float2 host_dw(double a) {
  const float h = static_cast<float>(a);
  return make_float2(h, static_cast<float>(a - static_cast<double>(h)));
}

void fill_dev(pe_detector_s* d) {
  pe::DetDev& D = d->dev;
  memset(&D, 0, sizeof(D));
  const pe_detector_config& c = d->cfg;
  D.T = d->T;
  D.k0 = d->k0;
  D.nb = d->nb;
  D.orbit = c.orbit;
  D.tdi_gen = c.tdi_gen;
  D.L = det_arm_s(c);
  D.R = pe::kAuS;
  D.alpha0_ht = c.alpha0_rad / pe::kPi;
  D.rate_ht = 2.0 / pe::kYearS;
  D.alpha0_t = 0.5 * D.alpha0_ht;
  D.rate_t = 1.0 / pe::kYearS;
  if (c.orbit == PE_ORBIT_HELIO) {
    const double e = D.L / (2.0 * std::sqrt(3.0) * D.R);
    D.eRh = 0.5 * e * D.R;
    D.eR3h = 1.5 * e * D.R;
    D.eRs3 = std::sqrt(3.0) * e * D.R;
    for (int i = 0; i < 3; ++i) {
      const double b = 2.0 * pe::kPi * i / 3.0 + c.cartwheel0_rad;
      D.cb[i] = std::cos(b);
      D.sb[i] = std::sin(b);
    }
    // offsets as linear forms in the basis (cos 2a, sin 2a, cos a, sin a) plus a constant:
    //   x = eRh (c2 cb + s2 sb) - eR3h cb,  y = eRh (s2 cb - c2 sb) - eR3h sb,  z = -eRs3 (c cb + s sb)
    for (int i = 0; i < 3; ++i) {
      const double cb = D.cb[i], sb = D.sb[i];
      const double row[3][5] = {{D.eRh * cb, D.eRh * sb, 0.0, 0.0, -D.eR3h * cb},
                                {-D.eRh * sb, D.eRh * cb, 0.0, 0.0, -D.eR3h * sb},
                                {0.0, 0.0, -D.eRs3 * cb, -D.eRs3 * sb, 0.0}};
      for (int j = 0; j < 3; ++j)
        for (int m = 0; m < 5; ++m) D.Mo[i][j][m] = row[j][m];
    }
  } else {
    D.rgeo = D.L / std::sqrt(3.0);
    D.geo_rate_ht = 2.0 / c.geo_period_s;
    D.geo_rate_t = 1.0 / c.geo_period_s;
    const double nl = c.geo_lon_rad, nbt = c.geo_lat_rad;
    const double n[3] = {std::cos(nbt) * std::cos(nl), std::cos(nbt) * std::sin(nl), std::sin(nbt)};
    D.e1[0] = -std::sin(nl); D.e1[1] = std::cos(nl); D.e1[2] = 0.0;
    D.e2[0] = n[1] * D.e1[2] - n[2] * D.e1[1];
    D.e2[1] = n[2] * D.e1[0] - n[0] * D.e1[2];
    D.e2[2] = n[0] * D.e1[1] - n[1] * D.e1[0];
    // spacecraft i at phase phi_0 + 2 pi i/3: r (cos(phi_0 + b_i) e1 + sin(phi_0 + b_i) e2)
    //   = cos phi_0 r (cos b_i e1 + sin b_i e2) + sin phi_0 r (-sin b_i e1 + cos b_i e2)
    for (int i = 0; i < 3; ++i) {
      const double cbi = std::cos(2.0 * pe::kPi * i / 3.0), sbi = std::sin(2.0 * pe::kPi * i / 3.0);
      for (int j = 0; j < 3; ++j) {
        D.Mo[i][j][0] = D.rgeo * (cbi * D.e1[j] + sbi * D.e2[j]);
        D.Mo[i][j][1] = D.rgeo * (-sbi * D.e1[j] + cbi * D.e2[j]);
        D.Mo[i][j][2] = D.Mo[i][j][3] = D.Mo[i][j][4] = 0.0;
      }
    }
  }
  D.Rw = host_dw(D.R);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int m = 0; m < 5; ++m) D.Mof[i][j][m] = static_cast<float>(D.Mo[i][j][m]);
  D.ratew = host_dw(D.rate_t);
  D.alpha0w = host_dw(D.alpha0_t);
  D.geo_ratew = host_dw(D.geo_rate_t);
  // double-word t_f carries ~6e-14 relative error (a dozen rounded operations); below 2^23 s the
  // heliocentric angle (1 turn a year) and below 2^21 s the geocentric one (1 turn in ~4 days) stay
  // within ~1e-13 turn of their FP64 values; beyond, the unit forms them in FP64
  D.tfw_max = (c.orbit == PE_ORBIT_HELIO) ? 8388608.0f : 2097152.0f;
  D.f = d->f; D.f13 = d->f13; D.fm13 = d->fm13; D.lnf3 = d->lnf3; D.fm76 = d->fm76;
  D.fm56 = d->fpow; D.fm12 = d->fpow + d->nb; D.fm53 = d->fpow + 2 * (size_t)d->nb;
  D.sca = d->sca; D.z = d->z; D.dg = d->dg; D.gg = d->gg; D.dd = d->dd_dev; D.sct = d->sct;
  D.sctw = d->sctw; D.fw = d->fw; D.aw = d->aw; D.atw = d->atw; D.saw = d->saw; D.caw = d->caw;
  D.zw = d->zw; D.dgw = d->dgw; D.ggw = d->ggw; D.f13w = d->f13w; D.fm76w = d->fm76w;
  const size_t nbz = (size_t)d->nb;
  D.ff = d->f32; D.f13f = d->f32 + nbz; D.fm13f = d->f32 + 2 * nbz; D.lnf3f = d->f32 + 3 * nbz; D.fm76f = d->f32 + 4 * nbz;
  D.scaf = d->scaf; D.zf = d->zf; D.dgf = d->dgf; D.ggf = d->ggf;
  D.rate_tf = (float)D.rate_t; D.alpha0_tf = (float)D.alpha0_t; D.geo_rate_tf = (float)D.geo_rate_t;
  D.Rf = (float)D.R; D.Lf = (float)D.L;
  D.dg_scale = 1.0;
  D.gg_scale = 1.0;
}

// Power of two above |x| (1 for zero or non-finite x): the double-word tables hold x / scale < 1.
double pow2_above(double x) {
  if (!(x > 0.0) || !std::isfinite(x)) return 1.0;
  return std::ldexp(1.0, std::ilogb(x) + 1);
}

pe_status check_dets(const pe_detector* dets, int ndet, pe::DetSet* ds) {
  if (dets == nullptr) return fail(PE_EINVAL, "dets is NULL");
  if (ndet < 1 || ndet > pe::kMaxDet) return fail(PE_EINVAL, "ndet=%d outside [1, %d]", ndet, pe::kMaxDet);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return fail(PE_ECUDA, "no CUDA device"); }
  memset(ds, 0, sizeof(*ds));
  ds->ndet = ndet;
  for (int i = 0; i < ndet; ++i) {
    if (dets[i] == nullptr) return fail(PE_EINVAL, "dets[%d] is NULL", i);
    if (!dets[i]->has_data) return fail(PE_ESTATE, "dets[%d] has no data (call pe_set_data_psd first)", i);
    if (dets[i]->device != dev) return fail(PE_EINVAL, "dets[%d] lives on device %d, current is %d", i, dets[i]->device, dev);
    ds->d[i] = dets[i]->dev;
  }
  return PE_OK;
}

int g_sm_count = 0;
int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 1;
  }
  return g_sm_count;
}

}  // namespace

extern "C" {

int pe_abi_version(void) { return 1; }

const char* pe_last_error(void) { return g_err.c_str(); }

pe_status pe_create_detector(const pe_detector_config* cfg, double T_obs, int64_t k0, int64_t nbins, pe_detector* out) {
  if (cfg == nullptr || out == nullptr) return fail(PE_EINVAL, "cfg/out is NULL");
  *out = nullptr;
  if (!(T_obs > 0.0) || !std::isfinite(T_obs)) return fail(PE_EINVAL, "T_obs must be positive");
  if (k0 < 1) return fail(PE_EINVAL, "k0 must be >= 1 (no DC bin)");
  if (nbins < 1 || nbins > (1 << 26)) return fail(PE_EINVAL, "nbins=%lld outside [1, 2^26]", (long long)nbins);
  if (cfg->orbit != PE_ORBIT_HELIO && cfg->orbit != PE_ORBIT_GEO) return fail(PE_EINVAL, "orbit must be 0 or 1");
  if (cfg->tdi_gen != 15 && cfg->tdi_gen != 20) return fail(PE_EINVAL, "tdi_gen must be 15 or 20");
  if (!(cfg->arm_m > 0.0)) return fail(PE_EINVAL, "arm_m must be positive");
  if (cfg->orbit == PE_ORBIT_GEO && !(cfg->geo_period_s > 0.0)) return fail(PE_EINVAL, "geo_period_s must be positive");
  setup_pool();
  pe_detector_s* d = new (std::nothrow) pe_detector_s();
  if (!d) return fail(PE_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&d->device) != cudaSuccess) { cudaGetLastError(); delete d; return fail(PE_ECUDA, "no CUDA device"); }
  d->cfg = *cfg;
  d->T = T_obs;
  d->k0 = k0;
  d->nb = (int)nbins;
  const size_t nb = (size_t)nbins;
  // double2: sincos table + sca, z (2 nb) + dg (3 nb); float4: double-word sincos table, zw (nb),
  // dgw (3 nb); doubles: f, f13, fm13, lnf3, fm76 (5 nb) + fpow (3 nb) + gg (3 nb) + psd_model (3 nb) + dd (3,
  // padded); float2: fw, aw, atw, saw, caw, f13w, fm76w (7 nb) + ggw (3 nb) + scaf, zf (2 nb) +
  // dgf (3 nb); float: five FP32 grid tables (5 nb) + ggf (3 nb)
  const size_t n_d = 14 * nb + 8, n_d2 = 5 * nb + pe::kSinTab, n_f4 = pe::kSinTab + 4 * nb, n_f2 = 15 * nb,
               n_f = 8 * nb;
  const size_t bytes = n_d2 * sizeof(double2) + n_f4 * sizeof(float4) + n_d * sizeof(double) +
                       n_f2 * sizeof(float2) + n_f * sizeof(float);
  cudaError_t e = pe::dmalloc(&d->mem, bytes);
  if (e != cudaSuccess) { cudaGetLastError(); delete d; return fail(PE_ENOMEM, "pe::dmalloc(%zu) failed", bytes); }
  double2* p2 = static_cast<double2*>(d->mem);
  d->sct = p2; p2 += pe::kSinTab;
  d->sca = p2; p2 += nb;
  d->z = p2; p2 += nb;
  d->dg = p2; p2 += 3 * nb;
  float4* p4 = reinterpret_cast<float4*>(p2);
  d->sctw = p4; p4 += pe::kSinTab;
  d->zw = p4; p4 += nb;
  d->dgw = p4; p4 += 3 * nb;
  double* p = reinterpret_cast<double*>(p4);
  d->f = p; p += nb;
  d->f13 = p; p += nb;
  d->fm13 = p; p += nb;
  d->lnf3 = p; p += nb;
  d->fm76 = p; p += nb;
  d->fpow = p; p += 3 * nb;
  d->gg = p; p += 3 * nb;
  d->psd_model = p; p += 3 * nb;
  d->dd_dev = p; p += 8;
  float2* pf = reinterpret_cast<float2*>(p);
  d->fw = pf; pf += nb;
  d->aw = pf; pf += nb;
  d->atw = pf; pf += nb;
  d->saw = pf; pf += nb;
  d->caw = pf; pf += nb;
  d->f13w = pf; pf += nb;
  d->fm76w = pf; pf += nb;
  d->ggw = pf; pf += 3 * nb;
  d->scaf = pf; pf += nb;
  d->zf = pf; pf += nb;
  d->dgf = pf; pf += 3 * nb;
  float* pff = reinterpret_cast<float*>(pf);
  d->f32 = pff; pff += 5 * nb;
  d->ggf = pff;
  fill_dev(d);
  const double L = det_arm_s(*cfg);
  if ((e = pe::launch_sincos_table(d->sct, 0)) != cudaSuccess ||
      (e = pe::launch_grid_tables(T_obs, k0, d->nb, L, d->f, d->f13, d->fm13, d->lnf3, d->fm76, d->fpow, d->sca,
                                  d->z, 0)) != cudaSuccess ||
      (e = pe::launch_psd_model(d->f, d->nb, L, cfg->oms_m_rtHz, cfg->acc_ms2_rtHz, cfg->psd_shaping, cfg->tdi_gen,
                                d->psd_model, 0)) != cudaSuccess ||
      (e = pe::launch_dw_tables(d->f, d->f13, d->fm76, d->sca, d->z, d->sct, d->nb, L, d->fw, d->aw, d->atw, d->saw,
                                d->caw, d->f13w, d->fm76w, d->zw, d->sctw, 0)) != cudaSuccess ||
      (e = pe::launch_f32_tables(d->f, d->f13, d->fm13, d->lnf3, d->fm76, d->sca, d->z, d->nb, d->f32,
                                 d->f32 + nb, d->f32 + 2 * nb, d->f32 + 3 * nb, d->f32 + 4 * nb, d->scaf, d->zf, 0)) !=
          cudaSuccess ||
      (e = cudaMemset(d->dd_dev, 0, 3 * sizeof(double))) != cudaSuccess ||
      (e = cudaDeviceSynchronize()) != cudaSuccess) {
    cudaGetLastError();
    pe::dfree(d->mem);
    delete d;
    return fail(PE_ECUDA, "detector table set-up failed: %s", cudaGetErrorString(e));
  }
  *out = d;
  return PE_OK;
}

pe_status pe_destroy_detector(pe_detector det) {
  if (det == nullptr) return PE_OK;
  cudaDeviceSynchronize();
  pe::dfree(det->mem);
  cudaGetLastError();
  delete det;
  return PE_OK;
}

pe_status pe_psd_model(pe_detector det, double* out_psd) {
  if (det == nullptr || out_psd == nullptr) return fail(PE_EINVAL, "det/out_psd is NULL");
  PE_CUDA(cudaMemcpy(out_psd, det->psd_model, 3 * (size_t)det->nb * sizeof(double), cudaMemcpyDeviceToHost));
  return PE_OK;
}

pe_status pe_data_norm(pe_detector det, double* out_dd) {
  if (det == nullptr || out_dd == nullptr) return fail(PE_EINVAL, "det/out_dd is NULL");
  if (!det->has_data) return fail(PE_ESTATE, "no data set");
  for (int c = 0; c < 3; ++c) out_dd[c] = det->dd[c];
  return PE_OK;
}

static pe_status set_data_device(pe_detector det, const double2* data_dev, const double* psd_dev) {
  const int nb = det->nb;
  double* parts = nullptr;
  int* bad = nullptr;
  const int nblk = (nb + pe::kTileBins - 1) / pe::kTileBins;
  PE_CUDA(pe::dmalloc(&parts, (size_t)nblk * 3 * sizeof(double)));
  if (pe::dmalloc(&bad, sizeof(int)) != cudaSuccess) { pe::dfree(parts); return fail(PE_ENOMEM, "cudaMalloc failed"); }
  cudaMemset(bad, 0, sizeof(int));
  int g = 0;
  const double L = det_arm_s(det->cfg);
  cudaError_t e = pe::launch_data_tables(det->f, det->sca, det->z, nb, det->T, L, det->cfg.tdi_gen, data_dev,
                                         psd_dev ? psd_dev : det->psd_model, det->dg, det->gg, parts, bad, &g, 0);
  if (e == cudaSuccess) e = pe::launch_sum_parts(parts, g, 3, det->dd_dev, 0);
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(det->dd, det->dd_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost);
  // double-word copies of the whitened tables for the mixed-precision path, scaled by powers of two
  // near their maxima
  double* mxp = nullptr;
  const int n3 = 3 * nb;
  if (e == cudaSuccess) e = pe::dmalloc(&mxp, ((size_t)(n3 + pe::kTileBins - 1) / pe::kTileBins * 2 + 2) * sizeof(double));
  double mx[2] = {0.0, 0.0};
  if (e == cudaSuccess) {
    double* out = mxp;
    e = pe::launch_table_max(det->dg, det->gg, n3, mxp + 2, out, 0);
    if (e == cudaSuccess) e = cudaMemcpy(mx, out, 2 * sizeof(double), cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) {
    det->dev.dg_scale = pow2_above(mx[0]);
    det->dev.gg_scale = pow2_above(mx[1]);
    e = pe::launch_dw_data(det->dg, det->gg, n3, 1.0 / det->dev.dg_scale, 1.0 / det->dev.gg_scale, det->dgw, det->ggw,
                           det->dgf, det->ggf, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (mxp) pe::dfree(mxp);
  pe::dfree(parts);
  pe::dfree(bad);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(PE_ECUDA, "data tables: %s", cudaGetErrorString(e)); }
  if (hbad) { det->has_data = 0; return fail(PE_EINVAL, "PSD has a non-positive or non-finite value"); }
  det->has_data = 1;
  return PE_OK;
}

pe_status pe_set_data_psd(pe_detector det, const double* data_aet, const double* psd_aet, int ptr_is_device) {
  if (det == nullptr || data_aet == nullptr) return fail(PE_EINVAL, "det/data is NULL");
  const size_t nb = (size_t)det->nb;
  if (ptr_is_device) return set_data_device(det, reinterpret_cast<const double2*>(data_aet), psd_aet);
  double2* dd = nullptr;
  double* pd = nullptr;
  PE_CUDA(pe::dmalloc(&dd, 3 * nb * sizeof(double2)));
  if (psd_aet && pe::dmalloc(&pd, 3 * nb * sizeof(double)) != cudaSuccess) {
    pe::dfree(dd);
    return fail(PE_ENOMEM, "cudaMalloc failed");
  }
  cudaError_t e = pe::upload(dd, data_aet, 3 * nb * sizeof(double2));
  if (e == cudaSuccess && psd_aet) e = pe::upload(pd, psd_aet, 3 * nb * sizeof(double));
  pe_status st = PE_OK;
  if (e != cudaSuccess) st = fail(PE_ECUDA, "upload failed: %s", cudaGetErrorString(e));
  else st = set_data_device(det, dd, pd);
  pe::dfree(dd);
  if (pd) pe::dfree(pd);
  return st;
}

static pe_status signal_device(pe_detector det, const double* theta, unsigned mode_mask, double2* out_dev,
                               cudaStream_t st) {
  Scratch sc(st);
  double* th = nullptr;
  pe::SampleCoef* coef = nullptr;
  int* nend = nullptr;
  int* status = nullptr;
  PE_CUDA(sc.alloc(&coef, 1));
  PE_CUDA(sc.alloc(&nend, 1));
  PE_CUDA(sc.alloc(&status, 1));
  if (is_device_ptr(theta)) {
    th = const_cast<double*>(theta);
  } else {
    for (int i = 0; i < PE_NPARAM; ++i)
      if (!std::isfinite(theta[i])) return fail(PE_EINVAL, "theta[%d] is not finite", i);
    PE_CUDA(sc.alloc(&th, PE_NPARAM));
    PE_CUDA(pe::upload_async(th, theta, PE_NPARAM * sizeof(double), st));
  }
  pe::DetSet ds;
  memset(&ds, 0, sizeof(ds));
  ds.ndet = 1;
  ds.d[0] = det->dev;
  PE_CUDA(pe::launch_prep(th, 1, mode_mask, ds, coef, nend, status, st));
  PE_CUDA(pe::launch_signal(det->dev, coef, out_dev, pe::mask_prec(mode_mask), st));
  int hs = 0;
  PE_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  PE_WAIT(st);
  if (hs) return fail(PE_EINVAL, "theta is outside the parameter domain");
  return PE_OK;
}

pe_status pe_signal_aet(pe_detector det, const double* theta, unsigned mode_mask, double* out, void* stream) {
  if (det == nullptr || theta == nullptr || out == nullptr) return fail(PE_EINVAL, "det/theta/out is NULL");
  if (!pe::fwd_mask_ok(mode_mask)) return fail(PE_EINVAL, "bad mode mask 0x%x", mode_mask);
  if (check_local("pe_signal_aet", {theta, out}) != PE_OK) return PE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (is_device_ptr(out)) return signal_device(det, theta, mode_mask, reinterpret_cast<double2*>(out), st);
  double2* tmp = nullptr;
  const size_t n = 3 * (size_t)det->nb;
  PE_CUDA(pe::dmalloc(&tmp, n * sizeof(double2)));
  pe_status s = signal_device(det, theta, mode_mask, tmp, st);
  if (s == PE_OK) {
    cudaError_t e = cudaMemcpy(out, tmp, n * sizeof(double2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = fail(PE_ECUDA, "download failed: %s", cudaGetErrorString(e));
  }
  pe::dfree(tmp);
  return s;
}

pe_status pe_inject(pe_detector det, const double* theta_inj, unsigned mode_mask, const double* normals) {
  if (det == nullptr || theta_inj == nullptr) return fail(PE_EINVAL, "det/theta is NULL");
  if (mode_mask == 0 || (mode_mask & ~PE_MODE_ALL)) return fail(PE_EINVAL, "bad mode mask 0x%x", mode_mask);
  const size_t n = 3 * (size_t)det->nb;
  double2* h = nullptr;
  double2* nd = nullptr;
  PE_CUDA(pe::dmalloc(&h, n * sizeof(double2)));
  pe_status s = signal_device(det, theta_inj, mode_mask, h, 0);
  if (s == PE_OK && normals) {
    cudaError_t e = pe::dmalloc(&nd, n * sizeof(double2));
    if (e == cudaSuccess) e = pe::upload(nd, normals, n * sizeof(double2));
    if (e == cudaSuccess) e = pe::launch_inject(det->nb, det->T, det->psd_model, nd, h, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { cudaGetLastError(); s = fail(PE_ECUDA, "noise injection failed: %s", cudaGetErrorString(e)); }
  }
  if (s == PE_OK) s = set_data_device(det, h, nullptr);
  pe::dfree(h);
  if (nd) pe::dfree(nd);
  return s;
}

pe_status pe_loglike_batch(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask,
                           double* out_logl, double* out_dhhh, int32_t* out_status, void* stream) {
  pe::DetSet ds;
  pe_status s0 = check_dets(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (theta == nullptr || out_logl == nullptr) return fail(PE_EINVAL, "theta/out_logl is NULL");
  if (B < 1 || B > (1 << 20)) return fail(PE_EINVAL, "B=%d outside [1, 2^20]", B);
  if (!pe::fwd_mask_ok(mode_mask)) return fail(PE_EINVAL, "bad mode mask 0x%x", mode_mask);
  if (check_local("pe_loglike_batch", {theta, out_logl, out_dhhh, out_status}) != PE_OK) return PE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch sc(st);
  const int P = ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * pe::tiles_of(ds.d[i].nb, pe::kTileBins);
  const double* th = theta;
  if (!is_device_ptr(theta)) {
    double* t = nullptr;
    PE_CUDA(sc.alloc(&t, (size_t)B * PE_NPARAM));
    PE_CUDA(pe::upload_async(t, theta, (size_t)B * PE_NPARAM * sizeof(double), st));
    th = t;
  }
  pe::SampleCoef* coef = nullptr;
  int* nend = nullptr;
  long long* off = nullptr;
  long long* offi = nullptr;
  double* part = nullptr;
  pe::TuneChoice tc = pe::default_choice(pe::mask_prec(mode_mask));
  pe::lookup_tuned(ds, B, mode_mask, &tc);
  PE_CUDA(sc.alloc(&coef, B));
  PE_CUDA(sc.alloc(&nend, P));
  PE_CUDA(sc.alloc(&off, P + 1));
  if (tc.subtiles > 1) PE_CUDA(sc.alloc(&offi, P + 1));
  PE_CUDA(sc.alloc(&part, (size_t)max_tiles * 6));
  const bool h_logl = !is_device_ptr(out_logl);
  const bool h_dhhh = out_dhhh && !is_device_ptr(out_dhhh);
  const bool h_stat = out_status && !is_device_ptr(out_status);
  double* logl = out_logl;
  double* dhhh = out_dhhh;
  int32_t* stat = out_status;
  if (h_logl) PE_CUDA(sc.alloc(&logl, B));
  if (h_dhhh) PE_CUDA(sc.alloc(&dhhh, (size_t)B * ndet * 6));
  if (h_stat) PE_CUDA(sc.alloc(&stat, B));
  PE_CUDA(pe::launch_prep(th, B, mode_mask, ds, coef, nend, stat, st));
  PE_CUDA(pe::launch_fwd_offsets(nend, P, off, offi, tc.subtiles, st));
  void* prof = nullptr;
  pe::profile_begin(st, &prof);
  PE_CUDA(pe::launch_loglike_fwd_variant(tc.variant, pe::mask_prec(mode_mask), ds, B, coef, nend, off, offi,
                                         tc.subtiles, part, pe::grid_for(tc, max_tiles), st));
  pe::profile_end(st, prof);
  PE_CUDA(pe::launch_reduce(ds, B, off, part, coef, logl, dhhh, st));
  if (h_logl) PE_CUDA(cudaMemcpyAsync(out_logl, logl, (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (h_dhhh)
    PE_CUDA(cudaMemcpyAsync(out_dhhh, dhhh, (size_t)B * ndet * 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (h_stat) PE_CUDA(cudaMemcpyAsync(out_status, stat, (size_t)B * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (h_logl || h_dhhh || h_stat) PE_WAIT(st);
  return PE_OK;
}

pe_status pe_loglike_grad_batch(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask,
                                double* out_logl, double* out_grad, int32_t* out_status, void* stream) {
  pe::DetSet ds;
  pe_status s0 = check_dets(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (theta == nullptr || out_grad == nullptr) return fail(PE_EINVAL, "theta/out_grad is NULL");
  if (B < 1 || B > (1 << 20)) return fail(PE_EINVAL, "B=%d outside [1, 2^20]", B);
  if ((mode_mask & PE_MODE_ALL) == 0 || (mode_mask & ~(PE_MODE_ALL | PE_PREC_MIXED)))
    return fail(PE_EINVAL, "bad mode mask 0x%x (the gradient takes PE_PREC_MIXED, not PE_PREC_FP32)", mode_mask);
  const bool mixed = (mode_mask & PE_PREC_MIXED) != 0;
  mode_mask &= PE_MODE_ALL;
  if (check_local("pe_loglike_grad_batch", {theta, out_logl, out_grad, out_status}) != PE_OK) return PE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch sc(st);
  const int P = ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * ((ds.d[i].nb + pe::kTileBins - 1) / pe::kTileBins);
  const double* th = theta;
  if (!is_device_ptr(theta)) {
    double* t = nullptr;
    PE_CUDA(sc.alloc(&t, (size_t)B * PE_NPARAM));
    PE_CUDA(pe::upload_async(t, theta, (size_t)B * PE_NPARAM * sizeof(double), st));
    th = t;
  }
  pe::SampleCoef* coef = nullptr;
  pe::SampleGrad* sg = nullptr;
  int* nend = nullptr;
  long long* off = nullptr;
  double* part = nullptr;
  const int W = pe::grad_partial_width();
  PE_CUDA(sc.alloc(&coef, B));
  PE_CUDA(sc.alloc(&sg, B));
  PE_CUDA(sc.alloc(&nend, P));
  PE_CUDA(sc.alloc(&off, P + 1));
  PE_CUDA(sc.alloc(&part, (size_t)max_tiles * W));
  const bool h_logl = out_logl && !is_device_ptr(out_logl);
  const bool h_grad = !is_device_ptr(out_grad);
  const bool h_stat = out_status && !is_device_ptr(out_status);
  double* logl = out_logl;
  double* grad = out_grad;
  int32_t* stat = out_status;
  if (h_logl) PE_CUDA(sc.alloc(&logl, B));
  if (h_grad) PE_CUDA(sc.alloc(&grad, (size_t)B * PE_NPARAM));
  if (h_stat) PE_CUDA(sc.alloc(&stat, B));
  PE_CUDA(pe::launch_prep_grad(th, B, mode_mask, ds, coef, sg, nend, stat, st));
  PE_CUDA(pe::launch_scan_tiles(nend, P, off, pe::kTileBins, st));
  // a persistent grid of the kernel's resident CTAs per SM, each with its tape region
  const long long g = std::max<long long>(
      1, std::min<long long>(max_tiles, (long long)sm_count() * pe::grad_tape_ctas_per_sm(mixed)));
  double* tape = nullptr;
  PE_CUDA(sc.alloc(&tape, (size_t)g * pe::grad_tape_doubles_per_cta()));
  void* prof = nullptr;
  pe::profile_begin(st, &prof);
  PE_CUDA(pe::launch_grad_fwd(ds, B, coef, sg, nend, off, part, (int)g, mixed, tape, st));
  pe::profile_end(st, prof);
  PE_CUDA(pe::launch_grad_reduce(ds, B, off, part, coef, sg, logl, grad, st));
  if (h_logl) PE_CUDA(cudaMemcpyAsync(out_logl, logl, (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (h_grad)
    PE_CUDA(cudaMemcpyAsync(out_grad, grad, (size_t)B * PE_NPARAM * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (h_stat) PE_CUDA(cudaMemcpyAsync(out_status, stat, (size_t)B * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (h_logl || h_grad || h_stat) PE_WAIT(st);
  return PE_OK;
}

pe_status pe_fisher(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask, double* out_F,
                    void* stream) {
  pe::DetSet ds;
  pe_status s0 = check_dets(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (theta == nullptr || out_F == nullptr) return fail(PE_EINVAL, "theta/out_F is NULL");
  if (B < 1 || B > (1 << 16)) return fail(PE_EINVAL, "B=%d outside [1, 2^16]", B);
  if (mode_mask == 0 || (mode_mask & ~PE_MODE_ALL)) return fail(PE_EINVAL, "bad mode mask 0x%x", mode_mask);
  if (check_local("pe_fisher", {theta, out_F}) != PE_OK) return PE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch sc(st);
  const int P = ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * ((ds.d[i].nb + pe::kTileBins - 1) / pe::kTileBins);
  const double* th = theta;
  if (!is_device_ptr(theta)) {
    double* t = nullptr;
    PE_CUDA(sc.alloc(&t, (size_t)B * PE_NPARAM));
    PE_CUDA(pe::upload_async(t, theta, (size_t)B * PE_NPARAM * sizeof(double), st));
    th = t;
  }
  pe::SampleCoef* coef = nullptr;
  pe::SampleGrad* sg = nullptr;
  int* nend = nullptr;
  long long* off = nullptr;
  double* part = nullptr;
  const int W = pe::fisher_partial_width();
  PE_CUDA(sc.alloc(&coef, B));
  PE_CUDA(sc.alloc(&sg, B));
  PE_CUDA(sc.alloc(&nend, P));
  PE_CUDA(sc.alloc(&off, P + 1));
  PE_CUDA(sc.alloc(&part, (size_t)max_tiles * W));
  const bool h_F = !is_device_ptr(out_F);
  double* F = out_F;
  if (h_F) PE_CUDA(sc.alloc(&F, (size_t)B * 121));
  PE_CUDA(pe::launch_prep_grad(th, B, mode_mask, ds, coef, sg, nend, nullptr, st));
  PE_CUDA(pe::launch_scan_tiles(nend, P, off, pe::kTileBins, st));
  const long long g = std::min<long long>(max_tiles, (long long)sm_count() * 16);
  void* prof = nullptr;
  pe::profile_begin(st, &prof);
  PE_CUDA(pe::launch_fisher_fwd(ds, B, coef, sg, nend, off, part, (int)std::max<long long>(g, 1), st));
  pe::profile_end(st, prof);
  PE_CUDA(pe::launch_fisher_reduce(ds, B, off, part, coef, F, st));
  if (h_F) {
    PE_CUDA(cudaMemcpyAsync(out_F, F, (size_t)B * 121 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PE_WAIT(st);
  }
  return PE_OK;
}

// Fisher-Gaussian approximation of the posterior on a parameter subset (Sec. 2.2: C = F^-1 of
// Eq. eq_ll_fisher, the other parameters held at theta0 as in Sec. 3.3): F on the subset is the
// sub-block of the full Fisher matrix; C = F_sub^-1 by Cholesky; samples theta0 + L z with
// C = L L^T and z the caller's standard normals.
pe_status pe_fisher_gaussian(const pe_detector* dets, int ndet, const double* theta0, unsigned mode_mask,
                             const int32_t* idx, int k, const double* normals, int n, double* out_cov,
                             double* out_samples) {
  if (theta0 == nullptr || idx == nullptr || out_cov == nullptr) return fail(PE_EINVAL, "theta0/idx/out_cov is NULL");
  if (k < 1 || k > PE_NPARAM) return fail(PE_EINVAL, "k=%d outside [1, 11]", k);
  if (n < 0 || (n > 0 && (normals == nullptr || out_samples == nullptr)))
    return fail(PE_EINVAL, "normals/out_samples required for n > 0");
  for (int i = 0; i < k; ++i) {
    if (idx[i] < 0 || idx[i] >= PE_NPARAM) return fail(PE_EINVAL, "idx[%d]=%d out of range", i, idx[i]);
    for (int j = 0; j < i; ++j)
      if (idx[j] == idx[i]) return fail(PE_EINVAL, "idx has a repeated parameter");
  }
  double F[PE_NPARAM * PE_NPARAM];
  pe_status st = pe_fisher(dets, ndet, theta0, 1, mode_mask, F, nullptr);
  if (st != PE_OK) return st;
  // sub-block and its Cholesky factor F_sub = R R^T
  double A[PE_NPARAM][PE_NPARAM], R[PE_NPARAM][PE_NPARAM] = {};
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) A[i][j] = F[idx[i] * PE_NPARAM + idx[j]];
  for (int j = 0; j < k; ++j) {
    double d = A[j][j];
    for (int m = 0; m < j; ++m) d -= R[j][m] * R[j][m];
    if (!(d > 0.0)) return fail(PE_EINVAL, "Fisher sub-block is not positive definite");
    R[j][j] = std::sqrt(d);
    for (int i = j + 1; i < k; ++i) {
      double v = A[i][j];
      for (int m = 0; m < j; ++m) v -= R[i][m] * R[j][m];
      R[i][j] = v / R[j][j];
    }
  }
  // C = F_sub^-1 = R^-T R^-1: invert the lower-triangular R column by column
  double Ri[PE_NPARAM][PE_NPARAM] = {};
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < k; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int m = 0; m < i; ++m) v -= R[i][m] * Ri[m][c];
      Ri[i][c] = v / R[i][i];
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double v = 0.0;
      for (int m = 0; m < k; ++m) v += Ri[m][i] * Ri[m][j];
      out_cov[i * k + j] = v;
    }
  // samples: delta = L z with L = R^-T (lower factor of C), so C = L L^T
  for (int sidx = 0; sidx < n; ++sidx) {
    for (int p = 0; p < PE_NPARAM; ++p) out_samples[(size_t)sidx * PE_NPARAM + p] = theta0[p];
    for (int i = 0; i < k; ++i) {
      double v = 0.0;
      for (int m = 0; m < k; ++m) v += Ri[m][i] * normals[(size_t)sidx * k + m];
      out_samples[(size_t)sidx * PE_NPARAM + idx[i]] += v;
    }
  }
  return PE_OK;
}

}  // extern "C"

namespace {
std::atomic<double> g_wait_limit_s{600.0};
}

#ifdef PE_FAULT_INJECTION
#include "pespace_gb300_test.h"
// ---- test build: host-side fault injection and live-allocation count (pe_fault.h)
namespace {
std::atomic<int> g_fault_kind{-1};      // armed kind, -1 none
std::atomic<long> g_fault_nth{0};       // the armed event's index (1-based) among its kind
std::atomic<long> g_fault_seen[3];      // events of each kind since the last arm
std::atomic<long> g_fault_fired{0};
std::atomic<long> g_live{0};
std::once_flag g_fault_env_once;

void fault_env() {
  std::call_once(g_fault_env_once, [] {
    const char* v = getenv("PE_FAULT");
    if (!v || !*v) return;
    const char* names[3] = {"alloc", "upload", "launch"};
    for (int k = 0; k < 3; ++k) {
      const size_t n = strlen(names[k]);
      if (strncmp(v, names[k], n) == 0) {
        long nth = 1;
        if (v[n] == ':') nth = strtol(v + n + 1, nullptr, 10);
        g_fault_nth.store(nth > 0 ? nth : 1);
        g_fault_kind.store(k);
      }
    }
  });
}
}  // namespace

namespace pe {
bool fault_now(int kind) {
  fault_env();
  const long n = ++g_fault_seen[kind];
  if (g_fault_kind.load() == kind && n == g_fault_nth.load()) {
    ++g_fault_fired;
    return true;
  }
  return false;
}
void live_add(long d) { g_live += d; }
int checked_take_kernels();
int checked_take_grad();
}  // namespace pe

extern "C" {
pe_status pe_test_fault_arm(int kind, long nth) {
  if (kind < -1 || kind > 2 || nth < 0) return fail(PE_EINVAL, "pe_test_fault_arm: kind in -1..2, nth >= 0");
  fault_env();   // PE_FAULT is read once, before the arm below replaces it
  for (auto& c : g_fault_seen) c.store(0);
  g_fault_fired.store(0);
  g_fault_kind.store(nth > 0 ? kind : -1);
  g_fault_nth.store(nth);
  return PE_OK;
}
long pe_test_fault_count(int kind) { return (kind >= 0 && kind <= 2) ? g_fault_seen[kind].load() : -1; }
long pe_test_fault_fired(void) { return g_fault_fired.load(); }
long pe_test_live_allocations(void) { return g_live.load(); }
int pe_test_checked_take(void) {
  const int a = pe::checked_take_kernels(), b = pe::checked_take_grad();
  return (a < 0 || b < 0) ? -1 : (a | b);
}
}  // extern "C"
#endif

namespace pe {
cudaError_t wait_stream(cudaStream_t st) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev, st);
  if (e == cudaSuccess) {
    const double limit = g_wait_limit_s.load();
    const auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
      e = cudaEventQuery(ev);
      if (e != cudaErrorNotReady) break;
      if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit) break;
      if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  cudaEventDestroy(ev);
  if (e == cudaErrorNotReady) cudaGetLastError();
  return e;
}
}  // namespace pe

extern "C" {
pe_status pe_set_wait_limit(double seconds) {
  if (!(seconds > 0.0) || !std::isfinite(seconds)) return fail(PE_EINVAL, "wait limit must be positive and finite");
  g_wait_limit_s.store(seconds);
  return PE_OK;
}
double pe_get_wait_limit(void) { return g_wait_limit_s.load(); }
}  // extern "C"

namespace pe {
// Detector-handle validation for entry points defined in other translation units: fills the
// device views of dets[0..ndet) and sets pe_last_error on failure.
pe_status detset_from_handles(const pe_detector* dets, int ndet, DetSet* ds) { return check_dets(dets, ndet, ds); }
// Records a message for pe_last_error and returns st.
pe_status set_error(pe_status st, const char* msg) { return fail(st, "%s", msg); }

int fwd_blocks_per_sm() {
  static int n = 0;
  if (n == 0) n = 8;
  return n;
}
}  // namespace pe
