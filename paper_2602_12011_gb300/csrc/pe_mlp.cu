// pe_mlp.cu -- the surrogate's dense layers on tensor cores (BF16 operands, FP32 accumulation):
// one tiled GEMM C[M,N] = A[M,K] Bt[N,K]^T (both operands K-contiguous) on mma.sync m16n8k16, with
// an optional bias + SiLU epilogue, plus the elementwise and transpose kernels of the forward and
// backward passes and the Adam update. Layer l: Z = H W^T + b, H' = SiLU(Z), with W stored [out][in].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pe_mlp.h"

namespace pe {

constexpr int GB_M = 64, GB_N = 64, GB_K = 32;
constexpr int GPAD = 8;  // bf16 elements of padding per shared-memory row (keeps ldmatrix conflict-free)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldmatrix_x4(unsigned r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }

// C[M,N] = A[M,K] Bt[N,K]^T; requires M % 64 == 0, N % 64 == 0, K % 32 == 0 and 16-byte aligned
// rows. 4 warps, each a 32x32 sub-tile (2 x 4 mma tiles). epi: 0 store C (fp32); 1 Z = C + bias
// (fp32, stored to C) and H = SiLU(Z) as bf16 to Hout; 2 C + bias.
__global__ void __launch_bounds__(128) k_gemm_tn(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Bt,
                                                 float* __restrict__ C, int M, int N, int K, int epi,
                                                 const float* __restrict__ bias, __nv_bfloat16* __restrict__ Hout) {
  __shared__ __align__(16) __nv_bfloat16 As[GB_M][GB_K + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GB_N][GB_K + GPAD];
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GB_K) {
    // 64 rows x 32 bf16 = 64 x 4 chunks of 16 bytes per operand; 128 threads x 2 chunks
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int idx = tid + c * 128;
      const int r = idx >> 2, q = (idx & 3) * 8;
      *reinterpret_cast<uint4*>(&As[r][q]) = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + k0 + q);
      *reinterpret_cast<uint4*>(&Bs[r][q]) = *reinterpret_cast<const uint4*>(Bt + (size_t)(n0 + r) * K + k0 + q);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; kk += 16) {
      unsigned af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int row = wm + i * 16 + (lane & 15);
        const int col = kk + (lane >> 4) * 8;
        ldmatrix_x4(af[i], &As[row][col]);
      }
#pragma unroll
      for (int jp = 0; jp < 2; ++jp) {
        // two n8 tiles at once: matrices (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
        unsigned bf[4];
        const int nrow = wn + jp * 16 + (lane & 7) + ((lane >> 4) << 3);
        const int col = kk + ((lane >> 3) & 1) * 8;
        ldmatrix_x4(bf, &Bs[nrow][col]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][jp * 2 + 0], af[i], bf[0], bf[1]);
          mma_bf16(acc[i][jp * 2 + 1], af[i], bf[2], bf[3]);
        }
      }
    }
    __syncthreads();
  }
  // epilogue: thread holds rows (lane/4, +8), cols 2*(lane%4), +1 of each 16x8 tile
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm + i * 16 + (lane >> 2) + h * 8;
        const int col = n0 + wn + j * 8 + (lane & 3) * 2;
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (epi >= 1) {
          v0 += bias[col];
          v1 += bias[col + 1];
        }
        if (epi == 1)
          *reinterpret_cast<__nv_bfloat162*>(Hout + (size_t)row * N + col) = __floats2bfloat162_rn(silu(v0), silu(v1));
        *reinterpret_cast<float2*>(C + (size_t)row * N + col) = make_float2(v0, v1);
      }
}

// out[c][r] = in[r][c] (bf16), in: [R][Cn]
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out, int R, int Cn) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j;
    if (r < R && c < Cn) t[j][threadIdx.x] = in[(size_t)r * Cn + c];
  }
  __syncthreads();
  const int oc = r0 + threadIdx.x, orb = blockIdx.x * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int orow = orb + j;
    if (orow < Cn && oc < R) out[(size_t)orow * R + oc] = t[threadIdx.x][j];
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// dZ = dH * SiLU'(Z) (bf16 out); SiLU'(z) = s (1 + z (1 - s)), s = sigmoid(z)
__global__ void k_silu_bwd(const float* __restrict__ dH, const float* __restrict__ Z, __nv_bfloat16* __restrict__ dZ,
                           float* __restrict__ dZf, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z = Z[i];
  const float s = 1.0f / (1.0f + __expf(-z));
  const float g = dH[i] * s * (1.0f + z * (1.0f - s));
  dZ[i] = __float2bfloat16_rn(g);
  if (dZf) dZf[i] = g;
}

// MSE loss on standardised targets: L = mean (y - t)^2 over rows x cols; dY = 2 (y - t)/(R C)
// (fp32 and bf16); per-block partial sums of (y - t)^2.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dYf,
                      __nv_bfloat16* __restrict__ dY, double* __restrict__ part, size_t n, float scale) {
  __shared__ double red[256];
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (i < n) {
    const float d = Y[i] - T[i];
    e2 = (double)d * d;
    const float g = 2.0f * d * scale;
    if (dYf) dYf[i] = g;
    dY[i] = __float2bfloat16_rn(g);
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// db[c] = sum_r dZ[r][c] (fixed order over rows)
__global__ void k_colsum(const float* __restrict__ dZ, float* __restrict__ db, int R, int Cn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cn) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += dZ[(size_t)r * Cn + c];
  db[c] = s;
}

// Adam on fp32 master weights; also refreshes the bf16 copy. t: 1-based step.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ wb, size_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

// ---- launch wrappers -------------------------------------------------------------------------
cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int epi,
                    const float* bias, __nv_bfloat16* Hout, cudaStream_t st) {
  if (M % GB_M || N % GB_N || K % GB_K) return cudaErrorInvalidValue;
  dim3 grid(N / GB_N, M / GB_M);
  k_gemm_tn<<<grid, 128, 0, st>>>(A, Bt, C, M, N, K, epi, bias, Hout);
  return cudaGetLastError();
}
cudaError_t transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int Cn, cudaStream_t st) {
  dim3 grid((Cn + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, st>>>(in, out, R, Cn);
  return cudaGetLastError();
}
cudaError_t f32_to_bf16(const float* in, __nv_bfloat16* out, size_t n, cudaStream_t st) {
  k_f32_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t silu_bwd(const float* dH, const float* Z, __nv_bfloat16* dZ, float* dZf, size_t n, cudaStream_t st) {
  k_silu_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dH, Z, dZ, dZf, n);
  return cudaGetLastError();
}
cudaError_t mse(const float* Y, const float* T, float* dYf, __nv_bfloat16* dY, double* part, size_t n, float scale,
                int* nblocks, cudaStream_t st) {
  *nblocks = (int)((n + 255) / 256);
  k_mse<<<*nblocks, 256, 0, st>>>(Y, T, dYf, dY, part, n, scale);
  return cudaGetLastError();
}
cudaError_t colsum(const float* dZ, float* db, int R, int Cn, cudaStream_t st) {
  k_colsum<<<(Cn + 127) / 128, 128, 0, st>>>(dZ, db, R, Cn);
  return cudaGetLastError();
}
cudaError_t adam(float* w, const float* g, float* m, float* v, __nv_bfloat16* wb, size_t n, float lr, float b1, float b2,
                 float eps, int t, cudaStream_t st) {
  const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, g, m, v, wb, n, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace pe
