// pe_umma.cu -- the surrogate's dense-layer GEMM on the 5th-generation tensor cores (tcgen05):
// C[M,N] = A[M,K] Bt[N,K]^T with both operands K-contiguous bf16, fp32 accumulation in tensor
// memory (TMEM), operands staged by TMA (cp.async.bulk.tensor) into 128-byte-swizzled shared
// memory through a multi-stage mbarrier pipeline, and a fused bias / SiLU epilogue read back from
// TMEM with tcgen05.ld.
//
// One CTA of 128 threads computes one 128 x BN output tile (BN = 128 or 64):
//   warp 0, lane 0  TMA producer: per 64-wide K block, one A box (64 x 128) and one B box (64 x BN)
//                   into the next free stage, completion counted in bytes on that stage's
//                   "full" barrier;
//   warp 1, lane 0  MMA issuer: four tcgen05.mma (M 128, N BN, K 16) per K block from shared-memory
//                   descriptors; tcgen05.commit frees the stage ("empty" barrier) once its MMAs are
//                   done, and a last commit signals the accumulator ("accum" barrier);
//   warps 0-3       epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 16 fp32 columns per
//                   tcgen05.ld, adds the bias (staged in shared memory), applies SiLU, and writes
//                   fp32 C and bf16 H into the (by then idle) operand stages in the 128-byte swizzled
//                   layout of TMA; one thread then stores the tile with cp.async.bulk.tensor (rows
//                   past M are clipped by the tensor map).
// Every wait on a barrier is bounded (about one second of %globaltimer); on a timeout the kernel
// records an error code, drains its own TMA copies and MMAs (again bounded), frees its TMEM and
// returns, and the host reads the code (umma_take_error).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "pe_mlp.h"
#include "pe_fault.h"

namespace pe {
namespace umma {

constexpr int BM = 128;          // tile rows = TMEM lanes
constexpr int BK = 64;           // K per stage: one 128-byte swizzle row of bf16
constexpr int UK = 16;           // K per tcgen05.mma of kind::f16
constexpr int STAGES = 3;
constexpr uint64_t kWaitNs = 1000000000ull;   // bound of every barrier wait

__device__ int g_umma_error;     // first error code of any launch since the host last read it

template <int BN>
struct Layout {
  static constexpr int kA = BM * BK * 2;          // bytes of one A stage
  static constexpr int kB = BN * BK * 2;          // bytes of one B stage
  static constexpr int kBars = 2 * STAGES + 1;    // full[], empty[], accum
  static constexpr int kBytes = STAGES * (kA + kB) + 8 * kBars + 16;
  static constexpr int kDyn = kBytes + 1024;      // slack for the 1024-byte alignment of the base
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the completion of the barrier phase of the given parity, at most kWaitNs
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (!mbar_try_wait(bar, parity))
    if (gtime() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(src))
               : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzle layout that
// TMA's SWIZZLE_128B writes: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte
// offset), tile base 1024-byte aligned. Fields: start address >> 4 in bits 0-13, leading byte
// offset >> 4 in bits 16-29 (unused by swizzled K-major tiles; 1), stride byte offset >> 4 in bits
// 32-45, descriptor version 1 in bits 46-47, swizzle mode 2 (128 bytes) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int BN>
__device__ __forceinline__ uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }

// epi 0: C = acc; 1: Z = acc + bias -> C and SiLU(Z) -> Hout (bf16); 2: C = acc + bias
template <int BN>
__global__ void __launch_bounds__(128) k_umma_gemm(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB,
                                                   const __grid_constant__ CUtensorMap tmC,
                                                   const __grid_constant__ CUtensorMap tmH, int M, int N, int K,
                                                   int epi, const float* __restrict__ bias) {
  using Lay = Layout<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * Lay::kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * (Lay::kA + Lay::kB));
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  __shared__ int s_fail;
  __shared__ int s_armed[STAGES];       // TMA copies issued per stage
  __shared__ int s_taken[STAGES];       // ... and consumed by the MMA issuer
  __shared__ float s_bias[BN];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      s_armed[s] = s_taken[s] = 0;
    }
    mbar_init(accum, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (threadIdx.x < BN) s_bias[threadIdx.x] = (epi >= 1) ? bias[n0 + threadIdx.x] : 0.f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
        atomicCAS(&g_umma_error, 0, 1);
        s_fail = 1;
        break;
      }
      if (*(volatile int*)&s_fail) break;
      mbar_expect_tx(&full[s], (uint32_t)(Lay::kA + Lay::kB));
      tma_load_2d(sA + s * Lay::kA, &tmA, kb * BK, m0, &full[s]);
      tma_load_2d(sB + s * Lay::kB, &tmB, kb * BK, n0, &full[s]);
      s_armed[s] += 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16<BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        atomicCAS(&g_umma_error, 0, 2);
        s_fail = 1;
        break;
      }
      s_taken[s] += 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = sw128_desc(smem_addr(sA + s * Lay::kA));
      const uint64_t bd = sw128_desc(smem_addr(sB + s * Lay::kB));
#pragma unroll
      for (int k = 0; k < BK / UK; ++k) {
        // advance along K inside the swizzle row: 16 bf16 = 32 bytes = 2 in the >> 4 address field
        mma_bf16(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (kb > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accum);   // arrives once every MMA issued above has completed (also after a failure)
  }
  __syncwarp();

  // ---- epilogue: TMEM -> registers -> bias / SiLU -> shared (TMA layout) -> TMA store
  const bool ready = mbar_wait(accum, 0);
  if (!ready && lane == 0) {
    atomicCAS(&g_umma_error, 0, 3);
    s_fail = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!s_fail) {
    // every MMA has completed, so the operand stages are free: C tile as BN/32 boxes of 32 fp32
    // columns x 128 rows, then H as BN/64 boxes of 64 bf16 columns x 128 rows, 16 KB each, rows of
    // 128 bytes whose 16-byte chunks sit at chunk ^ (row & 7) (TMA's 128-byte swizzle)
    uint8_t* sC = base;
    uint8_t* sH = base + (BN / 32) * 16384;
    const int r = warp * 32 + lane;           // tile row of this thread = its TMEM lane
    const int sw = r & 7;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] += s_bias[c0 + i];
      uint8_t* crow = sC + (c0 / 32) * 16384 + r * 128;
      const int k0 = (c0 % 32) / 4;           // first 16-byte chunk of these 16 columns in the row
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4*>(crow + (((k0 + j) ^ sw) << 4)) =
            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      if (epi == 1) {
        __nv_bfloat162 h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(silu(v[2 * i]), silu(v[2 * i + 1]));
        uint8_t* hrow = sH + (c0 / 64) * 16384 + r * 128;
        const int kh = (c0 % 64) / 8;         // 16 bf16 = 2 chunks
        *reinterpret_cast<uint4*>(hrow + (((kh + 0) ^ sw) << 4)) = *reinterpret_cast<uint4*>(&h[0]);
        *reinterpret_cast<uint4*>(hrow + (((kh + 1) ^ sw) << 4)) = *reinterpret_cast<uint4*>(&h[4]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> TMA reads
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int g = 0; g < BN / 32; ++g) tma_store_2d(&tmC, n0 + 32 * g, m0, sC + g * 16384);
      if (epi == 1)
        for (int g = 0; g < BN / 64; ++g) tma_store_2d(&tmH, n0 + 64 * g, m0, sH + g * 16384);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // shared memory read out
    }
  } else if (threadIdx.x == 0) {
    // drain: every TMA copy issued but never consumed must land before the CTA's shared memory goes
    for (int s = 0; s < STAGES; ++s)
      for (int j = s_taken[s]; j < s_armed[s]; ++j) (void)mbar_wait(&full[s], (uint32_t)j & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
  }
}

// ---- host side --------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// rows x cols row-major (cols contiguous), box box_cols x box_rows, 128-byte swizzle (box_cols x
// element size = 128 bytes), zero fill for loads out of range (stores are clipped there)
static bool make_map(CUtensorMap* map, const void* ptr, CUtensorMapDataType type, int elem_bytes, int rows, int cols,
                     int box_cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * elem_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, type, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
static cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(k_umma_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Layout<BN>::kDyn);
}

template <int BN>
static cudaError_t launch(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int epi,
                          const float* bias, __nv_bfloat16* Hout, cudaStream_t st) {
  CUtensorMap ma, mb, mc, mh;
  const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (!make_map(&ma, A, bf, 2, M, K, BK, BM) || !make_map(&mb, Bt, bf, 2, N, K, BK, BN) ||
      !make_map(&mc, C, f32, 4, M, N, 32, BM))
    return cudaErrorInvalidValue;
  if (epi == 1) {
    if (!make_map(&mh, Hout, bf, 2, M, N, 64, BM)) return cudaErrorInvalidValue;
  } else {
    mh = mc;   // not read
  }
  dim3 grid((unsigned)(N / BN), (unsigned)((M + BM - 1) / BM));
  k_umma_gemm<BN><<<grid, 128, Layout<BN>::kDyn, st>>>(ma, mb, mc, mh, M, N, K, epi, bias);
  return pe::launch_status();
}

}  // namespace umma

cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int epi,
                    const float* bias, __nv_bfloat16* Hout, cudaStream_t st) {
  // TMA: 16-byte aligned bases and row strides; whole 64-wide K blocks; N a multiple of the tile
  if (M <= 0 || N <= 0 || K <= 0 || K % umma::BK || N % 64) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt) | reinterpret_cast<uintptr_t>(C) |
       reinterpret_cast<uintptr_t>(Hout)) & 15)
    return cudaErrorInvalidValue;
  if (epi == 1 && Hout == nullptr) return cudaErrorInvalidValue;
  if (epi >= 1 && bias == nullptr) return cudaErrorInvalidValue;
  if (N % 128 == 0) return umma::launch<128>(A, Bt, C, M, N, K, epi, bias, Hout, st);
  return umma::launch<64>(A, Bt, C, M, N, K, epi, bias, Hout, st);
}

cudaError_t umma_prepare() {
  // the dynamic shared-memory opt-in of both tile widths (current device) and the tensor-map
  // encoder, before any launch (and so outside any stream capture)
  if (!umma::encode_fn()) return cudaErrorNotSupported;
  cudaError_t e = umma::set_smem_attr<128>();
  if (e == cudaSuccess) e = umma::set_smem_attr<64>();
  return e;
}

int umma_take_error() {
  int code = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbol(&code, umma::g_umma_error, sizeof(int)) != cudaSuccess) return -1;
  if (code != 0 && cudaMemcpyToSymbol(umma::g_umma_error, &zero, sizeof(int)) != cudaSuccess) return -1;
  return code;
}

}  // namespace pe
