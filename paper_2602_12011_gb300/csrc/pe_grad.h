// pe_grad.h -- launch wrappers of the gradient and Fisher kernels (pe_grad.cu).
#pragma once
#include <cuda_runtime.h>

#include "pe_internal.h"

namespace pe {

cudaError_t launch_prep_grad(const double* theta, int B, unsigned mask, const DetSet& ds, SampleCoef* coef,
                             SampleGrad* sgrad, int* nend, int* status, cudaStream_t st);
cudaError_t launch_grad_fwd(const DetSet& ds, int B, const SampleCoef* coef, const SampleGrad* sgrad, const int* nend,
                            const long long* off, double* part, int grid, bool mixed, double* tape,
                            cudaStream_t st);
cudaError_t launch_grad_reduce(const DetSet& ds, int B, const long long* off, const double* part,
                               const SampleCoef* coef, const SampleGrad* sgrad, double* logl, double* grad,
                               cudaStream_t st);
cudaError_t launch_fisher_fwd(const DetSet& ds, int B, const SampleCoef* coef, const SampleGrad* sgrad,
                              const int* nend, const long long* off, double* part, int grid, cudaStream_t st);
cudaError_t launch_fisher_reduce(const DetSet& ds, int B, const long long* off, const double* part,
                                 const SampleCoef* coef, double* F, cudaStream_t st);
int grad_partial_width();
// Gradient: resident CTAs per SM of its persistent kernels, and the doubles of tape each CTA of
// the grid needs (launch_grad_fwd's tape holds grid x that many)
int grad_tape_ctas_per_sm(bool mixed);
size_t grad_tape_doubles_per_cta();
int fisher_partial_width();

}  // namespace pe
