// pe_kernels.h -- host-callable launch wrappers of the kernels in pe_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "pe_internal.h"

namespace pe {

cudaError_t launch_grid_tables(double T, long long k0, int nb, double L, double* f, double* f13, double* fm13,
                               double* lnf3, double* fm76, double* fpow, double2* sca, double2* z, cudaStream_t st);
cudaError_t launch_sincos_table(double2* tab, cudaStream_t st);
cudaError_t launch_psd_model(const double* f, int nb, double L, double oms, double acc, int shaping, int tdi_gen,
                             double* out, cudaStream_t st);
cudaError_t launch_data_tables(const double* f, const double2* sca, const double2* z, int nb, double T, double L,
                               int tdi_gen, const double2* data, const double* psd, double2* dg, double* gg,
                               double* dd_part, int* bad, int* nblocks, cudaStream_t st);
cudaError_t launch_sum_parts(const double* part, int n, int w, double* out, cudaStream_t st);
cudaError_t launch_prep(const double* theta, int B, unsigned mask, const DetSet& ds, SampleCoef* coef, int* nend,
                        int* status, cudaStream_t st);
// Tile offsets of the uneven (detector, sample) work list for tiles of tile_bins bins (kTileBins
// times 1, 2, 4 or 8): off[p] = sum over pairs before p of ceil(nend / tile_bins), off[P] = total.
cudaError_t launch_scan_tiles(const int* nend, int P, long long* off, int tile_bins, cudaStream_t st);
// The log-likelihood kernel's offsets: off over 128-bin sub-tiles (partials) and offi over work
// items of R sub-tiles (not written when R == 1: the kernel then takes off for both).
cudaError_t launch_fwd_offsets(const int* nend, int P, long long* off, long long* offi, int R, cudaStream_t st);
inline long long tiles_of(int nb, int tile_bins) { return (nb + tile_bins - 1) / tile_bins; }
cudaError_t launch_dw_tables(const double* f, const double* f13, const double* fm76, const double2* sca,
                             const double2* z, const double2* tab, int nb, double L, float2* fw, float2* aw,
                             float2* atw, float2* saw, float2* caw, float2* f13w, float2* fm76w, float4* zw,
                             float4* tabw, cudaStream_t st);
// max over n entries of max(|Re dg|, |Im dg|) and gg -> out[2]; mx_part: [ceil(n/128)][2] scratch
cudaError_t launch_table_max(const double2* dg, const double* gg, int n, double* mx_part, double* out, cudaStream_t st);
cudaError_t launch_dw_data(const double2* dg, const double* gg, int n, double inv_dgs, double inv_ggs, float4* dgw,
                           float2* ggw, float2* dgf, float* ggf, cudaStream_t st);
// FP32 copies of the grid tables (precision study)
cudaError_t launch_f32_tables(const double* f, const double* f13, const double* fm13, const double* lnf3,
                              const double* fm76, const double2* sca, const double2* z, int nb, float* ff, float* f13f,
                              float* fm13f, float* lnf3f, float* fm76f, float2* scaf, float2* zf, cudaStream_t st);
// prec: kPrecFP64, kPrecMixed or kPrecFP32 forward kernel; R: sub-tiles per work item (1, 2, 4, 8)
cudaError_t launch_loglike_fwd(const DetSet& ds, int B, const SampleCoef* coef, const int* nend, const long long* off,
                               const long long* offi, int R, double* part, int grid, int prec, cudaStream_t st);
// Register-budget variants of the forward kernel (min resident CTAs per SM 2, 3, 4), per precision.
constexpr int kFwdVariants = 3;
constexpr int kFwdDefaultVariant = 1;
cudaError_t launch_loglike_fwd_variant(int variant, int prec, const DetSet& ds, int B, const SampleCoef* coef,
                                       const int* nend, const long long* off, const long long* offi, int R,
                                       double* part, int grid, cudaStream_t st);
int fwd_variant_min_blocks(int variant);
int fwd_variant_max_blocks_per_sm(int variant, int prec);
cudaError_t launch_reduce(const DetSet& ds, int B, const long long* off, const double* part, const SampleCoef* coef,
                          double* logl, double* dhhh, cudaStream_t st);
cudaError_t launch_signal(const DetDev& D, const SampleCoef* coef, double2* out, int prec, cudaStream_t st);
cudaError_t launch_inject(int nb, double T, const double* psd, const double2* normals, double2* h, cudaStream_t st);

// Mode mask of the forward entry points: at least one PE_MODE_* bit, optionally one precision flag.
inline bool fwd_mask_ok(unsigned m) {
  return (m & PE_MODE_ALL) != 0u && (m & ~(PE_MODE_ALL | PE_PREC_MIXED | PE_PREC_FP32)) == 0u &&
         (m & (PE_PREC_MIXED | PE_PREC_FP32)) != (PE_PREC_MIXED | PE_PREC_FP32);
}
inline int mask_prec(unsigned m) {
  return (m & PE_PREC_MIXED) ? kPrecMixed : ((m & PE_PREC_FP32) ? kPrecFP32 : kPrecFP64);
}

// CTAs per SM the persistent forward kernel can keep resident (occupancy query).
int fwd_blocks_per_sm();

// Defined in pe_api.cu: handle validation and error reporting shared with other entry points.
pe_status detset_from_handles(const pe_detector* dets, int ndet, DetSet* ds);
pe_status set_error(pe_status st, const char* msg);
// Bounded host wait for the work queued so far on st (an event polled with cudaEventQuery until
// the limit pe_set_wait_limit set): cudaSuccess, cudaErrorNotReady when the limit ran out (the
// work stays queued), or the stream's error.
cudaError_t wait_stream(cudaStream_t st);

}  // namespace pe
