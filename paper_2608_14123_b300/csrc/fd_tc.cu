// Fast-diagonalization solve on the 5th-generation tensor cores (tcgen05,
// kind::f16 with BF16 operands and FP32 accumulation in TMEM), Eqs. (9)-(11).
//
// Per element the residual patch r_s (ns^3 <= 16^3) is a 16 x 16 x 16 BF16
// tensor; each of the six mode products (S1^T, S2^T, S3^T, S3, S2, S1 along
// a, b, c) is a GEMM with M = 256 rows (the two non-contracted indices), K =
// 16 (the contracted index) and N = 16, issued as two M = 128 MMAs into 32
// TMEM columns.  The result comes back by tcgen05.ld (one TMEM row per thread)
// and is written, transposed where the next product contracts another index,
// as the next BF16 A operand.  The scaling by 1/(g0 + g1 l1 + g2 l2 + g3 l3)
// and the weights W are applied in FP32; the weighted patch is stored in FP32
// for the combine kernel.
//
// Operand layout: K-major, no swizzle ("core matrices" of 8 rows x 16 bytes);
// element (row r, k) of a 128 x 16 tile at byte (r/8)*256 + (k/8)*128 +
// (r%8)*16 + (k%8)*2, i.e. leading-dimension byte offset 128 (next core
// matrix along K) and stride byte offset 256 (next 8-row group).
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>

#include "dgfas_internal.h"

#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
      return DGFAS_ERR_CUDA;                                                  \
    }                                                                         \
  } while (0)

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in bits 16-29, stride byte offset >> 4 in bits 32-45,
// descriptor version 1 in bits 46-47, base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1),
// B BF16 (bits 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait for the given phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 16 columns of FP32 from TMEM: thread (lane) gets its row's 16 values
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// byte offset of (row, k) in a K-major no-swizzle tile with 16 K columns
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

}  // namespace tc

using namespace tc;

// Self-test: D[128][16] = A[128][16] B[16][16]^T with integer-valued BF16
// operands (exact in FP32), A[r][k] = (r + 2k) % 7 - 3, B[n][k] = (3n + k) % 5 - 2.
__global__ void k_tc_selftest(float* __restrict__ out, int* __restrict__ flag) {
  __shared__ __align__(1024) unsigned char sA[128 * 16 * 2];
  __shared__ __align__(1024) unsigned char sB[16 * 16 * 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = tid; t < 128 * 16; t += blockDim.x) {
    const int r = t / 16, k = t % 16;
    *reinterpret_cast<__nv_bfloat16*>(sA + tile_off(r, k)) = __float2bfloat16((float)((r + 2 * k) % 7 - 3));
  }
  for (int t = tid; t < 16 * 16; t += blockDim.x) {
    const int n = t / 16, k = t % 16;
    *reinterpret_cast<__nv_bfloat16*>(sB + tile_off(n, k)) = __float2bfloat16((float)((3 * n + k) % 5 - 2));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(smem_u32(&mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    mma_bf16(tmem, sdesc(smem_u32(sA), 128, 256), sdesc(smem_u32(sB), 128, 256), idesc_bf16(128, 16), 0);
    commit(smem_u32(&mbar));
  }
  const bool ok = mbar_wait(smem_u32(&mbar), 0);
  fence_after();
  if (!ok && lane == 0) atomicExch(flag, 1);
  float v[16];
  tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
  for (int q = 0; q < 16; ++q) out[(32 * warp + lane) * 16 + q] = ok ? v[q] : 0.0f;
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

extern "C" int dgfas_tc_selftest(float* out_host, int* timeout_host) {
  if (!out_host || !timeout_host) return DGFAS_ERR_INVALID;
  float* d = nullptr;
  int* f = nullptr;
  CK(cudaMalloc(&d, 128 * 16 * sizeof(float)));
  CK(cudaMalloc(&f, sizeof(int)));
  CK(cudaMemset(f, 0, sizeof(int)));
  k_tc_selftest<<<1, 128>>>(d, f);
  ++g_kernels;
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out_host, d, 128 * 16 * sizeof(float), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(timeout_host, f, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(d);
  cudaFree(f);
  return DGFAS_OK;
}
