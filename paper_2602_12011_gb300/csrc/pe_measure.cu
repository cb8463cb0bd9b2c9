// pe_measure.cu -- measurement helpers of the benchmark: CUDA-event timing of the fused
// kernels on their own stream, and the FP64 and FP32 FMA throughputs that bound them.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "pe_measure.h"
#include "pespace_gb300.h"

namespace pe {
namespace {
std::mutex g_mu;
bool g_on = false;
struct EvPair { cudaEvent_t a, b; };
std::vector<EvPair> g_ev;
}  // namespace

void profile_begin(cudaStream_t st, void** token) {
  *token = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  EvPair* p = new EvPair;
  if (cudaEventCreate(&p->a) != cudaSuccess || cudaEventCreate(&p->b) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return;
  }
  cudaEventRecord(p->a, st);
  *token = p;
}

void profile_end(cudaStream_t st, void* token) {
  if (!token) return;
  EvPair* p = static_cast<EvPair*>(token);
  cudaEventRecord(p->b, st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_ev.push_back(*p);
  delete p;
}

// 8 independent FMA chains per thread; the result is stored so nothing is dead code.
template <class T>
__global__ void k_fma_peak(T* out, T a, T b, int iters) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// FMA throughput of type T over about `seconds` of back-to-back launches, in TFLOP/s (FMA = 2).
template <class T>
pe_status fma_peak(double seconds, int iters, double* out_tflops) {
  if (out_tflops == nullptr || !(seconds > 0.0)) return PE_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return PE_ECUDA;
  }
  const int blocks = nsm * 8, threads = 256;
  T* d = nullptr;
  if (cudaMalloc(&d, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return PE_ENOMEM; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_peak<T><<<blocks, threads>>>(d, T(0.999999), T(1e-7), iters);  // warm-up
  double total_ms = 0.0, flops = 0.0;
  pe_status st = PE_OK;
  while (total_ms < seconds * 1e3) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, threads>>>(d, T(0.999999), T(1e-7), iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); st = PE_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    total_ms += ms;
    flops += 2.0 * 8.0 * iters * (double)blocks * threads;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (st == PE_OK) *out_tflops = flops / (total_ms * 1e-3) / 1e12;
  return st;
}

}  // namespace pe

extern "C" {

pe_status pe_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(pe::g_mu);
  pe::g_on = on != 0;
  return PE_OK;
}

pe_status pe_profile_read(double* total_ms, int64_t* launches) {
  if (total_ms == nullptr || launches == nullptr) return PE_EINVAL;
  std::vector<pe::EvPair> ev;
  {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    ev.swap(pe::g_ev);
  }
  double tot = 0.0;
  pe_status st = PE_OK;
  for (auto& p : ev) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
      cudaGetLastError();
      st = PE_ECUDA;
    }
    tot += ms;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  *total_ms = tot;
  *launches = (int64_t)ev.size();
  return st;
}

pe_status pe_measure_fp64_peak(double seconds, double* out_tflops) {
  return pe::fma_peak<double>(seconds, 4096, out_tflops);
}

pe_status pe_measure_fp32_peak(double seconds, double* out_tflops) {
  return pe::fma_peak<float>(seconds, 65536, out_tflops);
}

}  // extern "C"
