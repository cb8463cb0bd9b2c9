// pe_mlp.h -- launch wrappers of the surrogate's tensor-core layers and elementwise kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace pe {

// C[M,N] = A[M,K] Bt[N,K]^T (bf16 operands, fp32 accumulation in TMEM, tcgen05.mma; pe_umma.cu).
// epi 0: C; epi 1: C + bias -> C (fp32) and SiLU -> Hout (bf16); epi 2: C + bias -> C.
// Requires K % 64 == 0, N % 64 == 0, 16-byte aligned A and Bt; any M >= 1.
cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int epi,
                    const float* bias, __nv_bfloat16* Hout, cudaStream_t st);
// Once per device before the first gemm_tn (outside any stream capture): kernel attributes and
// the tensor-map encoder.
cudaError_t umma_prepare();
// Error code recorded by a GEMM launch since the last call (0 none; 1-3 a barrier wait that ran out
// of time: TMA slot, TMA data, accumulator), cleared when read; -1 if it cannot be read.
int umma_take_error();
cudaError_t transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int Cn, cudaStream_t st);
cudaError_t f32_to_bf16(const float* in, __nv_bfloat16* out, size_t n, cudaStream_t st);
cudaError_t silu_bwd(const float* dH, const float* Z, __nv_bfloat16* dZ, float* dZf, size_t n, cudaStream_t st);
cudaError_t mse(const float* Y, const float* T, float* dYf, __nv_bfloat16* dY, double* part, size_t n, float scale,
                int* nblocks, cudaStream_t st);
cudaError_t colsum(const float* dZ, float* db, int R, int Cn, cudaStream_t st);
// Adam with the step's learning rate and bias corrections read from par (device, {lr, bc1, bc2}).
cudaError_t adam(float* w, const float* g, float* m, float* v, size_t n, const float* par, float b1, float b2, float eps,
                 cudaStream_t st);
// par = {lr_t, 1 - b1^t, 1 - b2^t} for the step the device counters ctr describe (cosine schedule).
cudaError_t train_step_params(const int* ctr, float* par, double lr, int total_steps, float b1, float b2,
                              cudaStream_t st);
// ctr[0..2] += 1 (step in epoch, global step, Adam steps).
cudaError_t train_step_advance(int* ctr, cudaStream_t st);

}  // namespace pe
