// pe_kernels.h -- host-callable launch wrappers of the kernels in pe_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "pe_internal.h"

namespace pe {

cudaError_t launch_grid_tables(double T, long long k0, int nb, double L, double* f, double* f13, double* fm13,
                               double* lnf3, double* fm76, double2* sca, double2* z, cudaStream_t st);
cudaError_t launch_sincos_table(double2* tab, cudaStream_t st);
cudaError_t launch_psd_model(const double* f, int nb, double L, double oms, double acc, int shaping, int tdi_gen,
                             double* out, cudaStream_t st);
cudaError_t launch_data_tables(const double* f, const double2* sca, const double2* z, int nb, double T, double L,
                               int tdi_gen, const double2* data, const double* psd, double2* dg, double* gg,
                               double* dd_part, int* bad, int* nblocks, cudaStream_t st);
cudaError_t launch_sum_parts(const double* part, int n, int w, double* out, cudaStream_t st);
cudaError_t launch_prep(const double* theta, int B, unsigned mask, const DetSet& ds, SampleCoef* coef, int* nend,
                        int* status, cudaStream_t st);
cudaError_t launch_scan_tiles(const int* nend, int P, long long* off, cudaStream_t st);
cudaError_t launch_loglike_fwd(const DetSet& ds, int B, const SampleCoef* coef, const int* nend, const long long* off,
                               double* part, int grid, cudaStream_t st);
// Register-budget variants of the forward kernel (min resident CTAs per SM 2, 3, 4).
constexpr int kFwdVariants = 3;
constexpr int kFwdDefaultVariant = 1;
cudaError_t launch_loglike_fwd_variant(int variant, const DetSet& ds, int B, const SampleCoef* coef, const int* nend,
                                       const long long* off, double* part, int grid, cudaStream_t st);
int fwd_variant_min_blocks(int variant);
int fwd_variant_max_blocks_per_sm(int variant);
cudaError_t launch_reduce(const DetSet& ds, int B, const long long* off, const double* part, const SampleCoef* coef,
                          double* logl, double* dhhh, cudaStream_t st);
cudaError_t launch_signal(const DetDev& D, const SampleCoef* coef, double2* out, cudaStream_t st);
cudaError_t launch_inject(int nb, double T, const double* psd, const double2* normals, double2* h, cudaStream_t st);

// CTAs per SM the persistent forward kernel can keep resident (occupancy query).
int fwd_blocks_per_sm();

// Defined in pe_api.cu: handle validation and error reporting shared with other entry points.
pe_status detset_from_handles(const pe_detector* dets, int ndet, DetSet* ds);
pe_status set_error(pe_status st, const char* msg);

}  // namespace pe
