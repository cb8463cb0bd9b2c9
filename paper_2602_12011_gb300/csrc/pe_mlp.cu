// pe_mlp.cu -- the elementwise and transpose kernels of the surrogate's forward and backward passes
// and the Adam update (the dense products themselves are pe_umma.cu's tcgen05 GEMM). Layer l:
// Z = H W^T + b, H' = SiLU(Z), with W stored [out][in].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pe_mlp.h"
#include "pe_fault.h"

namespace pe {

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

// Adam on fp32 master weights. The step's learning rate and bias corrections come from the device
// (par = {lr_t, 1 - b1^t, 1 - b2^t}, written by k_train_step_params), so that one captured
// training step serves every step of a run.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       size_t n, const float* __restrict__ par, float b1, float b2, float eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float lr = par[0], bc1 = par[1], bc2 = par[2];
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Schedule of one training step from the device counters ctr = {step in epoch, global step, Adam
// steps taken}: cosine learning rate lr (0.02 + 0.98 (1 + cos(pi g/(G-1)))/2) at global step g of G,
// and the bias corrections of Adam step t = ctr[2] + 1.
__global__ void k_train_step_params(const int* __restrict__ ctr, float* __restrict__ par, double lr, int total_steps,
                                    float b1, float b2) {
  const double frac = (double)ctr[1] / (double)(total_steps > 1 ? total_steps - 1 : 1);
  par[0] = (float)(lr * (0.02 + 0.98 * 0.5 * (1.0 + cos(3.14159265358979 * frac))));
  const float t = (float)(ctr[2] + 1);
  par[1] = 1.f - powf(b1, t);
  par[2] = 1.f - powf(b2, t);
}

__global__ void k_train_step_advance(int* ctr) {
  ctr[0] += 1;
  ctr[1] += 1;
  ctr[2] += 1;
}

// ---- launch wrappers -------------------------------------------------------------------------
cudaError_t transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int Cn, cudaStream_t st) {
  dim3 grid((Cn + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, st>>>(in, out, R, Cn);
  return pe::launch_status();
}
cudaError_t f32_to_bf16(const float* in, __nv_bfloat16* out, size_t n, cudaStream_t st) {
  k_f32_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return pe::launch_status();
}
cudaError_t silu_bwd(const float* dH, const float* Z, __nv_bfloat16* dZ, float* dZf, size_t n, cudaStream_t st) {
  k_silu_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dH, Z, dZ, dZf, n);
  return pe::launch_status();
}
cudaError_t mse(const float* Y, const float* T, float* dYf, __nv_bfloat16* dY, double* part, size_t n, float scale,
                int* nblocks, cudaStream_t st) {
  *nblocks = (int)((n + 255) / 256);
  k_mse<<<*nblocks, 256, 0, st>>>(Y, T, dYf, dY, part, n, scale);
  return pe::launch_status();
}
cudaError_t colsum(const float* dZ, float* db, int R, int Cn, cudaStream_t st) {
  k_colsum<<<(Cn + 127) / 128, 128, 0, st>>>(dZ, db, R, Cn);
  return pe::launch_status();
}
cudaError_t adam(float* w, const float* g, float* m, float* v, size_t n, const float* par, float b1, float b2, float eps,
                 cudaStream_t st) {
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, g, m, v, n, par, b1, b2, eps);
  return pe::launch_status();
}
cudaError_t train_step_params(const int* ctr, float* par, double lr, int total_steps, float b1, float b2,
                              cudaStream_t st) {
  k_train_step_params<<<1, 1, 0, st>>>(ctr, par, lr, total_steps, b1, b2);
  return pe::launch_status();
}
cudaError_t train_step_advance(int* ctr, cudaStream_t st) {
  k_train_step_advance<<<1, 1, 0, st>>>(ctr);
  return pe::launch_status();
}

}  // namespace pe
