// pe_mlp.h -- launch wrappers of the surrogate's tensor-core layers and elementwise kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace pe {

// C[M,N] = A[M,K] Bt[N,K]^T (bf16 operands, fp32 accumulation, mma.sync m16n8k16).
// epi 0: C; epi 1: C + bias -> C (fp32) and SiLU -> Hout (bf16); epi 2: C + bias -> C.
cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int epi,
                    const float* bias, __nv_bfloat16* Hout, cudaStream_t st);
cudaError_t transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int Cn, cudaStream_t st);
cudaError_t f32_to_bf16(const float* in, __nv_bfloat16* out, size_t n, cudaStream_t st);
cudaError_t silu_bwd(const float* dH, const float* Z, __nv_bfloat16* dZ, float* dZf, size_t n, cudaStream_t st);
cudaError_t mse(const float* Y, const float* T, float* dYf, __nv_bfloat16* dY, double* part, size_t n, float scale,
                int* nblocks, cudaStream_t st);
cudaError_t colsum(const float* dZ, float* db, int R, int Cn, cudaStream_t st);
cudaError_t adam(float* w, const float* g, float* m, float* v, __nv_bfloat16* wb, size_t n, float lr, float b1, float b2,
                 float eps, int t, cudaStream_t st);

}  // namespace pe
