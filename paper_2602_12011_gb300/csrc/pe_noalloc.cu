// pe_noalloc.cu -- pe_loglike_batch_noalloc: the batched log-likelihood with its scratch in a
// fixed, file-scope device array instead of memory allocated per call.
//
// Who needs it: a caller that must not allocate device memory while it runs, for example a
// sampler embedded in a host application that reserves the GPU's memory for its own pool at
// start-up (so a library cudaMalloc can fail at an arbitrary point), or a latency-critical loop
// that must never enter the allocator or wait on its implicit synchronisation. Such a caller
// allocates its inputs and outputs once, up front, and this entry point then touches no
// allocator at all.
//
// The scratch lives in g_noalloc_scratch below: kNoAllocScratchBytes (32 MiB) per device. CUDA
// loads this file's module lazily, so the array is committed on a device by the first call there,
// and held until the process exits. Every call looks up its device address with
// cudaGetSymbolAddress on the current device (the host-side symbol is only a stand-in, not a
// device address); once the module is loaded the lookup allocates nothing, and no cached address
// can outlive a device reset.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "pe_internal.h"
#include "pe_kernels.h"
#include "pespace_gb300.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// device (or managed) memory of the current device
bool device_ptr(const void* p) {
  if (p == nullptr) return false;
  int dev = -1;
  cudaPointerAttributes a;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the scratch array on the current device, looked up on every call.
pe_status scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof(msg), "pe_loglike_batch_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return pe::set_error(PE_ECUDA, msg);
  }
  *out = p;
  return PE_OK;
}

}  // namespace

extern "C" pe_status pe_loglike_batch_noalloc(const pe_detector* dets, int ndet, const double* theta, int B,
                                              unsigned mode_mask, double* out_logl, double* out_dhhh,
                                              int32_t* out_status, void* stream) {
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (B < 1) return pe::set_error(PE_EINVAL, "pe_loglike_batch_noalloc: B must be >= 1");
  if (!pe::fwd_mask_ok(mode_mask)) return pe::set_error(PE_EINVAL, "pe_loglike_batch_noalloc: bad mode mask");
  if (!device_ptr(theta) || !device_ptr(out_logl) || (out_dhhh && !device_ptr(out_dhhh)) ||
      (out_status && !device_ptr(out_status)))
    return pe::set_error(PE_EINVAL,
                         "pe_loglike_batch_noalloc: theta and every output must be device pointers of the current device");
  // Scratch layout: coefficients [B], active bins [P], sub-tile offsets [P+1], work-item offsets
  // [P+1], sub-tile partials [sub-tiles][6]. The work items take the precision's default number of
  // sub-tiles (no tuned choice is read here).
  const size_t P = (size_t)ndet * B;
  const int R = pe::fwd_default_subtiles(pe::mask_prec(mode_mask));
  size_t max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (size_t)B * pe::tiles_of(ds.d[i].nb, pe::kTileBins);
  const size_t o_coef = 0;
  const size_t o_nend = align256(o_coef + (size_t)B * sizeof(pe::SampleCoef));
  const size_t o_off = align256(o_nend + P * sizeof(int));
  const size_t o_offi = align256(o_off + (P + 1) * sizeof(long long));
  const size_t o_part = align256(o_offi + (P + 1) * sizeof(long long));
  const size_t need = o_part + max_tiles * 6 * sizeof(double);
  if (need > kNoAllocScratchBytes) {
    char msg[320];
    snprintf(msg, sizeof(msg),
             "pe_loglike_batch_noalloc: B=%d on these grids needs %zu bytes of scratch, more than the fixed %zu; "
             "split the batch (about %zu bytes per sample)",
             B, need, kNoAllocScratchBytes, need / (size_t)B);
    return pe::set_error(PE_EINVAL, msg);
  }
  void* base = nullptr;
  pe_status s1 = scratch_address(&base);
  if (s1 != PE_OK) return s1;
  unsigned char* sc = static_cast<unsigned char*>(base);
  pe::SampleCoef* coef = reinterpret_cast<pe::SampleCoef*>(sc + o_coef);
  int* nend = reinterpret_cast<int*>(sc + o_nend);
  long long* off = reinterpret_cast<long long*>(sc + o_off);
  long long* offi = reinterpret_cast<long long*>(sc + o_offi);
  double* part = reinterpret_cast<double*>(sc + o_part);
  // Every scratch element a kernel reads is written earlier in the same call (coefficients and
  // active counts by the prep kernel, offsets by the scan, one partial per tile by the forward
  // kernel), so nothing is cleared between calls.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
    cudaGetLastError();
    nsm = 1;
  }
  cudaError_t e = pe::launch_prep(theta, B, mode_mask, ds, coef, nend, out_status, st);
  if (e == cudaSuccess) e = pe::launch_fwd_offsets(nend, (int)P, off, offi, R, st);
  const size_t g = max_tiles < (size_t)nsm * pe::fwd_blocks_per_sm() ? max_tiles : (size_t)nsm * pe::fwd_blocks_per_sm();
  if (e == cudaSuccess) e = pe::launch_loglike_fwd(ds, B, coef, nend, off, offi, R, part, (int)(g > 0 ? g : 1),
                                                     pe::mask_prec(mode_mask), st);
  if (e == cudaSuccess) e = pe::launch_reduce(ds, B, off, part, coef, out_logl, out_dhhh, st);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "pe_loglike_batch_noalloc: launch failed: %s", cudaGetErrorString(e));
    return pe::set_error(PE_ECUDA, msg);
  }
  return PE_OK;
}
