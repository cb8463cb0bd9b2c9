// pe_fault.h -- the library's device allocations, host-to-device uploads and launch-status reads go
// through these helpers, so that a test build can make any one of them fail on the host and count
// what stays allocated; and the index checks of the hot kernels' test build.
//
// Normal build: each helper is the plain CUDA call, and PE_CHK(cond, code) is `true`.
// Test build (-DPE_FAULT_INJECTION -DPE_CHECKED, libpespace_gb300_test.so):
//   - fault injection: the n-th allocation, upload or launch-status read after pe_test_fault_arm
//     (or the PE_FAULT environment variable, "alloc[:n]", "upload[:n]" or "launch[:n]", read once)
//     returns an error instead of doing its work (an allocation or upload is then not made; a
//     launch has happened and only its status is replaced), and the number of live device
//     allocations is counted;
//   - PE_CHK(cond, code): where cond fails, the kernel ORs code into this translation unit's
//     device error word (read and cleared by the host) and skips the access instead of making it.
// Nothing here faults or waits on a GPU.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace pe {

enum FaultKind { kFaultAlloc = 0, kFaultUpload = 1, kFaultLaunch = 2 };

#ifdef PE_FAULT_INJECTION
bool fault_now(int kind);          // counts the event; true if it is the armed one
void live_add(long d);             // live device allocations made through the helpers
#else
inline bool fault_now(int) { return false; }
inline void live_add(long) {}
#endif

inline cudaError_t dmalloc_bytes(void** p, size_t bytes) {
  if (fault_now(kFaultAlloc)) { *p = nullptr; return cudaErrorMemoryAllocation; }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) live_add(1);
  return e;
}
inline cudaError_t dmalloc_async_bytes(void** p, size_t bytes, cudaStream_t st) {
  if (fault_now(kFaultAlloc)) { *p = nullptr; return cudaErrorMemoryAllocation; }
  const cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e == cudaSuccess) live_add(1);
  return e;
}
template <class T>
inline cudaError_t dmalloc(T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = dmalloc_bytes(&q, bytes);
  *p = static_cast<T*>(q);
  return e;
}
template <class T>
inline cudaError_t dmalloc_async(T** p, size_t bytes, cudaStream_t st) {
  void* q = nullptr;
  const cudaError_t e = dmalloc_async_bytes(&q, bytes, st);
  *p = static_cast<T*>(q);
  return e;
}
inline cudaError_t dfree(void* p) {
  if (p) live_add(-1);
  return cudaFree(p);
}
inline cudaError_t dfree_async(void* p, cudaStream_t st) {
  if (p) live_add(-1);
  return cudaFreeAsync(p, st);
}
inline cudaError_t upload(void* dst, const void* src, size_t bytes) {
  if (fault_now(kFaultUpload)) return cudaErrorInvalidValue;
  return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}
inline cudaError_t upload_async(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (fault_now(kFaultUpload)) return cudaErrorInvalidValue;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}
// status of the kernel launched just before
inline cudaError_t launch_status() {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && fault_now(kFaultLaunch)) return cudaErrorLaunchOutOfResources;
  return e;
}

}  // namespace pe

#ifdef PE_CHECKED
// one error word per translation unit (no relocatable device code), read by pe_checked_take_local
static __device__ int g_pe_check;
#define PE_CHK(cond, code) ((cond) ? true : (atomicOr(&g_pe_check, (code)), false))
static inline int pe_checked_take_local() {
  int v = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_pe_check, sizeof(int)) != cudaSuccess) return -1;
  if (v != 0 && cudaMemcpyToSymbol(g_pe_check, &zero, sizeof(int)) != cudaSuccess) return -1;
  return v;
}
#else
#define PE_CHK(cond, code) true
static inline int pe_checked_take_local() { return 0; }
#endif
