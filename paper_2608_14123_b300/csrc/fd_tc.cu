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
#include <algorithm>
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

// ---------------------------------------------------------------- FD on tensor cores
// operand tile geometry: K-major tiles (gather, D^-1 step) use LBO 128 / SBO 256
// in the first 4096 B; MN-major tiles use a padded M stride
#define TC_MN_SBO 144
#define TC_MN_LBO (16 * TC_MN_SBO)
#define TC_TILE (2 * TC_MN_LBO + 16)
struct FdTcSmem {
  unsigned char A[2][2][TC_TILE];        // ping-pong A operand, two M = 128 tiles each
  unsigned char B[6][16 * 16 * 2];       // per direction: S^T (n = out, k = in) and S
  float lam[3][16], W[3][16];
  int gmap[3][16];                       // patch position -> (neighbour offset + 1) << 8 | node, or -1
  int nb[27];                            // the element's 27-neighbourhood
  uint64_t mbar;
  uint32_t tslot;
};
// the operand buffers double as the staging area of one FP32 patch (<= 16^3)
static_assert(sizeof(((FdTcSmem*)nullptr)->A) >= 16 * 16 * 16 * sizeof(float), "patch staging");

__device__ __forceinline__ uint4 pack8(const float* v) {
  uint4 o;
  __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]),
                  p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
  o.x = *reinterpret_cast<uint32_t*>(&p0);
  o.y = *reinterpret_cast<uint32_t*>(&p1);
  o.z = *reinterpret_cast<uint32_t*>(&p2);
  o.w = *reinterpret_cast<uint32_t*>(&p3);
  return o;
}

// 16 values of rows m0..m0+15 (m0 % 16 == 0) at column k of an MN-major tile
// pair: (m, k) at byte (m/8)*TC_MN_SBO + (k/8)*TC_MN_LBO + (k%8)*16 + (m%8)*2
// of tile m/128 (descriptor: leading byte offset = next core matrix along K,
// stride byte offset = next core matrix along M).  The core matrices along M
// are 144 B apart instead of 128 so that lanes writing different M groups at
// one k land in different banks.
__device__ __forceinline__ void st_mn(unsigned char* tile2, int m0, int k, const float* v) {
  unsigned char* t = tile2 + (m0 >> 7) * TC_TILE;
  const int ml = m0 & 127;
  const uint32_t off = (uint32_t)((ml >> 3) * TC_MN_SBO + (k >> 3) * TC_MN_LBO + (k & 7) * 16);
  *reinterpret_cast<uint4*>(t + off) = pack8(v);
  *reinterpret_cast<uint4*>(t + off + TC_MN_SBO) = pack8(v + 8);
}

// 16 values k = 0..15 of row m of a K-major tile pair
__device__ __forceinline__ void st_k(unsigned char* tile2, int m, const float* v) {
  unsigned char* t = tile2 + (m >> 7) * TC_TILE;
  const int ml = m & 127;
  const uint32_t off = (uint32_t)((ml >> 3) * 256 + (ml & 7) * 16);
  *reinterpret_cast<uint4*>(t + off) = pack8(v);
  *reinterpret_cast<uint4*>(t + off + 128) = pack8(v + 8);
}

// one mode product: D = A B^T for both M tiles (A K-major or MN-major);
// returns false on a timed-out wait
__device__ __forceinline__ bool tc_step(FdTcSmem& s, int ain, int bsel, bool mn, uint32_t tmem,
                                        uint32_t& phase) {
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_bf16(128, 16) | (mn ? (1u << 15) : 0u);
    const uint64_t bd = sdesc(smem_u32(s.B[bsel]), 128, 256);
    const uint32_t lbo = mn ? TC_MN_LBO : 128, sbo = mn ? TC_MN_SBO : 256;
    mma_bf16(tmem, sdesc(smem_u32(s.A[ain][0]), lbo, sbo), bd, idesc, 0);
    mma_bf16(tmem + 16, sdesc(smem_u32(s.A[ain][1]), lbo, sbo), bd, idesc, 0);
    commit(smem_u32(&s.mbar));
  }
  // only the issuing thread polls the barrier; the others wait at the CTA
  // barrier (no issue slots spent spinning) and order their TMEM reads after it
  const bool ok0 = threadIdx.x == 0 ? mbar_wait(smem_u32(&s.mbar), phase) : true;
  phase ^= 1u;
  const bool ok = __syncthreads_and(ok0 ? 1 : 0) != 0;
  fence_after();
  return ok;
}

// this thread's TMEM row of tile `t` (row 128 t + 32 w + lane), 16 FP32 values
__device__ __forceinline__ void tc_read1(uint32_t tmem, int t, float* v) {
  const int warp = threadIdx.x >> 5;
  tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * t, v);
}

// TN, TM > 0: instantiation for N = TN nodes and TM overlap layers, whose
// gather resolves the row's three source segments at compile time; TN = 0:
// any N and m (per-position gather maps).  VEC (TN % 4 == 0, TM even, r
// 16-byte aligned): the segments are read as float4 (own nodes) and float2
// (layers), 4 loads per row at p = 7 instead of 12 (each lane's loads touch
// distinct 32-byte sectors, so the load count sets the L1 traffic).
template <int TN, int TM, bool VEC = false>
__global__ void __launch_bounds__(128, 8) k_fd_tc(const LevelView<float> L, const float* __restrict__ r,
                                                  float* __restrict__ patch, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  FdTcSmem& s = *reinterpret_cast<FdTcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = TN > 0 ? TN : L.N, m = TN > 0 ? TM : L.m, nsm = L.nsm, N3 = N * N * N;
  const size_t NS3 = (size_t)nsm * nsm * nsm;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&s.tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(smem_u32(&s.mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s.tslot;
  // Subdomains of width <= 12: every row index (X, Y) of the six products
  // with X >= 12 (rows 192..255: warps 2 and 3 of the second M tile) or
  // Y >= 12 (lanes 12..15 of every 16) belongs to no patch position, so those
  // rows are not read back from TMEM (whole warps) or not written as the next
  // operand (single lanes).  Their operand entries keep whatever they hold,
  // which must be finite: such rows of A only produce such rows of D, and
  // such columns (K) meet the zero-padded rows of the S tiles, where 0 x Inf
  // or 0 x NaN would poison the sum.  The buffers are zeroed here, every
  // later write is a finite BF16 value except the FP32 patch staging, whose
  // only bytes outside the regions rewritten before the next product are
  // zeroed again per element (below).
  constexpr bool kSkipHi = TN > 0 && TN + 2 * TM <= 12;
  constexpr int kStagedTail = TC_TILE - 4096;   // bytes of a tile beyond the K-major span
  static_assert(kStagedTail % 16 == 0 && kStagedTail / 16 <= 128, "tail zeroing");
  if (kSkipHi) {
    uint4* z = reinterpret_cast<uint4*>(&s.A[0][0][0]);
    for (int t = tid; t < (int)(sizeof(s.A) / sizeof(uint4)); t += 128) z[t] = make_uint4(0, 0, 0, 0);
    fence_async_smem();
    __syncthreads();
  }
  uint32_t phase = 0;
  bool alive = true;
  int prev = -1;   // variant triple of the tables currently in shared memory
  for (int e = blockIdx.x; e < L.ne && alive; e += gridDim.x) {
    if (L.cls[e] == DGFAS_FROZEN) continue;
    __syncthreads();   // the previous element's patch store has read s.W
    if (kSkipHi && tid < kStagedTail / 16) {
      // the FP32 patch staging overwrote bytes [4096, TC_TILE) of A[0]'s
      // first tile, which the K-major gather does not rewrite and the
      // skipped rows of the MN-major products would leave in place: FP32 bit
      // patterns read as BF16 can be Inf or NaN, and 0 x NaN is NaN
      reinterpret_cast<uint4*>(s.A[0][0] + 4096)[tid] = make_uint4(0, 0, 0, 0);
    }
    const int v1 = L.var[3 * e], v2 = L.var[3 * e + 1], v3 = L.var[3 * e + 2];
    const int key = v1 | (v2 << 4) | (v3 << 8);
    if (tid < 27) s.nb[tid] = L.nbr27[27 * e + tid];
    if (key != prev) {
      // the per-variant tables (B operands S_d^T and S_d from the setup-time
      // BF16 tiles, eigenvalues, weights, gather map) change only with the
      // element's side variants: reloaded when the triple differs from the
      // previous element's (the same for the whole CTA)
      const int vv[3] = {v1, v2, v3};
      for (int t = tid; t < 6 * 32; t += 128) {
        const int slot = t >> 5, q = t & 31, d = slot >> 1, which = slot & 1;
        reinterpret_cast<uint4*>(s.B[slot])[q] = L.Btc[(vv[d] * 2 + which) * 32 + q];
      }
      if (tid < 48) {
        const int d = tid / 16, q = tid % 16, v = vv[d];
        const int nd = N + m * (((v >> 2) == 0) + ((v & 3) == 0));
        const bool in = q < nd;
        s.lam[d][q] = in ? L.lam[v * nsm + q] : 1.0f;
        s.W[d][q] = in ? L.W[v * nsm + q] : 0.0f;
        int code = -1;
        if (in) {
          int a = q, o, ix;
          if ((v >> 2) == 0 && a < m) {
            o = -1;
            ix = N - m + a;
          } else {
            if ((v >> 2) == 0) a -= m;
            o = a < N ? 0 : 1;
            ix = a < N ? a : a - N;
          }
          code = ((o + 1) << 8) | ix;
        }
        s.gmap[d][q] = code;
      }
      prev = key;
    }
    __syncthreads();
    const int n1 = N + m * (((v1 >> 2) == 0) + ((v1 & 3) == 0));
    const int n2 = N + m * (((v2 >> 2) == 0) + ((v2 & 3) == 0));
    const int n3 = N + m * (((v3 >> 2) == 0) + ((v3 & 3) == 0));
    // gather R_s r into A[0] (K-major): rows (c, b) = 16 c + b, K = a; one
    // thread per row, whose three possible sources (the x-neighbours left,
    // own, right of the row's y/z neighbour) are resolved once; the row is
    // written as two 16-byte stores
    for (int row = tid; row < 256; row += 128) {
      const int c = row >> 4, b = row & 15;
      float vals[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) vals[q] = 0.0f;
      const int my = s.gmap[1][b], mz = s.gmap[2][c];
      if (my >= 0 && mz >= 0) {
        const int* nb = s.nb + 3 * (my >> 8) + 9 * (mz >> 8);
        const long long line = ((mz & 255) * N + (my & 255)) * N;
        if constexpr (TN > 0) {
          // segments of the row along a: left layers (x-neighbour -1), own
          // nodes, right layers (x-neighbour +1)
          const float* p0 = nb[0] >= 0 ? r + (long long)nb[0] * N3 + line : nullptr;
          const float* p1 = nb[1] >= 0 ? r + (long long)nb[1] * N3 + line : nullptr;
          const float* p2 = nb[2] >= 0 ? r + (long long)nb[2] * N3 + line : nullptr;
          const bool li = (v1 >> 2) == 0, ri = (v1 & 3) == 0;
          if constexpr (VEC) {
            static_assert(TN % 4 == 0 && TM % 2 == 0 && TN + 2 * TM <= 16, "vector gather");
            float own[TN], lft[TM], rgt[TM];
#pragma unroll
            for (int v = 0; v < TN / 4; ++v) {
              const float4 t = p1 ? __ldg(reinterpret_cast<const float4*>(p1) + v)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
              own[4 * v] = t.x; own[4 * v + 1] = t.y; own[4 * v + 2] = t.z; own[4 * v + 3] = t.w;
            }
#pragma unroll
            for (int v = 0; v < TM / 2; ++v) {
              const float2 t0 = (li && p0) ? __ldg(reinterpret_cast<const float2*>(p0 + TN - TM) + v)
                                           : make_float2(0.f, 0.f);
              const float2 t2 = (ri && p2) ? __ldg(reinterpret_cast<const float2*>(p2) + v)
                                           : make_float2(0.f, 0.f);
              lft[2 * v] = t0.x; lft[2 * v + 1] = t0.y;
              rgt[2 * v] = t2.x; rgt[2 * v + 1] = t2.y;
            }
            if (li) {
#pragma unroll
              for (int q = 0; q < TM; ++q) vals[q] = lft[q];
#pragma unroll
              for (int q = 0; q < TN; ++q) vals[TM + q] = own[q];
#pragma unroll
              for (int q = 0; q < TM; ++q) vals[TM + TN + q] = rgt[q];   // zero unless ri
            } else {
#pragma unroll
              for (int q = 0; q < TN; ++q) vals[q] = own[q];
#pragma unroll
              for (int q = 0; q < TM; ++q) vals[TN + q] = rgt[q];
            }
          } else if (li) {
#pragma unroll
            for (int a = 0; a < TM; ++a) vals[a] = p0 ? p0[TN - TM + a] : 0.0f;
#pragma unroll
            for (int a = 0; a < TN; ++a) vals[TM + a] = p1 ? p1[a] : 0.0f;
            if (ri) {
#pragma unroll
              for (int a = 0; a < TM; ++a)
                if (2 * TM + TN + a - TM < 16) vals[TM + TN + a] = p2 ? p2[a] : 0.0f;
            }
          } else {
#pragma unroll
            for (int a = 0; a < TN; ++a) vals[a] = p1 ? p1[a] : 0.0f;
            if (ri) {
#pragma unroll
              for (int a = 0; a < TM; ++a)
                if (TN + a < 16) vals[TN + a] = p2 ? p2[a] : 0.0f;
            }
          }
        } else {
          const long long b0 = nb[0] >= 0 ? (long long)nb[0] * N3 + line : -1;
          const long long b1 = nb[1] >= 0 ? (long long)nb[1] * N3 + line : -1;
          const long long b2 = nb[2] >= 0 ? (long long)nb[2] * N3 + line : -1;
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int mx = s.gmap[0][q];
            if (mx < 0) continue;
            const int o = mx >> 8;
            const long long bs = o == 0 ? b0 : (o == 1 ? b1 : b2);
            if (bs >= 0) vals[q] = r[bs + (mx & 255)];
          }
        }
      }
      unsigned char* t = s.A[0][0] + (row >> 7) * TC_TILE;
      const int ml = row & 127;
      *reinterpret_cast<uint4*>(t + (ml >> 3) * 256 + (ml & 7) * 16) = pack8(vals);
      *reinterpret_cast<uint4*>(t + (ml >> 3) * 256 + (ml & 7) * 16 + 128) = pack8(vals + 8);
    }
    const float g0 = L.g[4 * e], g1 = L.g[4 * e + 1], g2 = L.g[4 * e + 2], g3 = L.g[4 * e + 3];
    float x[16];
    // 1: S1^T along a (A K-major): rows (c, b) -> x a'; write rows (c, a'), K = b (MN-major)
    if (!(alive = tc_step(s, 0, 0, false, tmem, phase))) break;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (kSkipHi && t == 1 && warp >= 2) continue;   // rows with first index >= 12
      const int rr = 128 * t + 32 * warp + lane;
      tc_read1(tmem, t, x);   // warp-collective: every lane reads
      if (kSkipHi && (rr & 15) >= 12) continue;   // second index >= 12: no patch position
      st_mn(s.A[1][0], 16 * (rr >> 4), rr & 15, x);
    }
    // 2: S2^T along b: rows (c, a') -> x b'; write rows (a', b'), K = c (MN-major)
    if (!(alive = tc_step(s, 1, 2, true, tmem, phase))) break;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (kSkipHi && t == 1 && warp >= 2) continue;   // rows with first index >= 12
      const int rr = 128 * t + 32 * warp + lane;
      tc_read1(tmem, t, x);   // warp-collective: every lane reads
      if (kSkipHi && (rr & 15) >= 12) continue;   // second index >= 12: no patch position
      st_mn(s.A[0][0], 16 * (rr & 15), rr >> 4, x);
    }
    // 3: S3^T along c: rows (a', b') -> x c'; scale by D^-1 in FP32; same rows, K = c' (K-major)
    if (!(alive = tc_step(s, 0, 4, true, tmem, phase))) break;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (kSkipHi && t == 1 && warp >= 2) continue;   // rows with first index >= 12
      const int rr = 128 * t + 32 * warp + lane;
      tc_read1(tmem, t, x);   // warp-collective: every lane reads
      if (kSkipHi && (rr & 15) >= 12) continue;   // second index >= 12: no patch position
      const float d0 = g0 + g1 * s.lam[0][rr >> 4] + g2 * s.lam[1][rr & 15];
#pragma unroll
      for (int q = 0; q < 16; ++q) x[q] = __fdividef(x[q], d0 + g3 * s.lam[2][q]);
      st_k(s.A[1][0], rr, x);
    }
    // 4: S3 along c: rows (a', b') -> x c''; write rows (a', c''), K = b' (MN-major)
    if (!(alive = tc_step(s, 1, 5, false, tmem, phase))) break;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (kSkipHi && t == 1 && warp >= 2) continue;   // rows with first index >= 12
      const int rr = 128 * t + 32 * warp + lane;
      tc_read1(tmem, t, x);   // warp-collective: every lane reads
      if (kSkipHi && (rr & 15) >= 12) continue;   // second index >= 12: no patch position
      st_mn(s.A[0][0], 16 * (rr >> 4), rr & 15, x);
    }
    // 5: S2 along b: rows (a', c'') -> x b''; write rows (c'', b''), K = a' (MN-major)
    if (!(alive = tc_step(s, 0, 3, true, tmem, phase))) break;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (kSkipHi && t == 1 && warp >= 2) continue;   // rows with first index >= 12
      const int rr = 128 * t + 32 * warp + lane;
      tc_read1(tmem, t, x);   // warp-collective: every lane reads
      if (kSkipHi && (rr & 15) >= 12) continue;   // second index >= 12: no patch position
      st_mn(s.A[1][0], 16 * (rr & 15), rr >> 4, x);
    }
    // 6: S1 along a: rows (c'', b'') -> x a''; weight, stage the patch in the
    // (now free) operand buffers in its global layout and copy it out with
    // coalesced stores.  Staged positions outside the element's variant
    // extents are not written; the combine step never reads them.
    if (!(alive = tc_step(s, 1, 1, true, tmem, phase))) break;
    {
      float* Pst = reinterpret_cast<float*>(&s.A[0][0][0]);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (kSkipHi && t == 1 && warp >= 2) continue;   // rows with first index >= 12
        const int rr = 128 * t + 32 * warp + lane;
        tc_read1(tmem, t, x);
        const int cc = rr >> 4, bb = rr & 15;
        if (cc < n3 && bb < n2) {
          const float w = s.W[2][cc] * s.W[1][bb];
          float* row = Pst + (cc * nsm + bb) * nsm;
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < n1) row[q] = x[q] * w * s.W[0][q];
        }
      }
      __syncthreads();
      float* P = patch + (size_t)e * NS3;
      for (int t = tid; t < (int)NS3; t += 128) P[t] = Pst[t];
    }
  }
  if (!alive && tid == 0) atomicExch(err, 1);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

int launch_fd_tc(Ctx& c, int l, const float* r) {
  LevelHost& H = c.lv[l];
  const int smem = (int)sizeof(FdTcSmem) + 1024;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // CTAs per SM: the autotuner's choice, else the 8 that registers allow
  const int per_sm = H.tune.fdtc > 0 ? std::min(H.tune.fdtc, 8) : 8;
  const int grid = std::min(H.ne, nsm * per_sm);
  auto go = [&](auto kern) -> int {
    static bool attr = false;   // one per instantiation
    if (!attr) {
      CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      attr = true;
    }
    kern<<<grid, 128, smem, c.stream>>>(H.v32, r, (float*)c.patch, c.tc_err);
    return DGFAS_OK;
  };
  int rc;
  const int key = 16 * H.N + H.m;
  switch (key) {
    case 16 * 8 + 2:
      // the vector gather needs r 16-byte aligned (element and line offsets
      // are multiples of 8 floats)
      rc = ((uintptr_t)r % 16 == 0) ? go(k_fd_tc<8, 2, true>) : go(k_fd_tc<8, 2>);
      break;
    case 16 * 9 + 2: rc = go(k_fd_tc<9, 2>); break;
    case 16 * 10 + 2: rc = go(k_fd_tc<10, 2>); break;
    case 16 * 11 + 2: rc = go(k_fd_tc<11, 2>); break;
    case 16 * 9 + 3: rc = go(k_fd_tc<9, 3>); break;
    default: rc = go(k_fd_tc<0, 0>); break;
  }
  if (rc != DGFAS_OK) return rc;
  ++g_kernels;
  CK(cudaGetLastError());
  return DGFAS_OK;
}

// Self-test of an MN-major A operand (no swizzle): element (m, k) of the
// 128 x 16 tile at byte (m/8)*128 + (k/8)*2048 + (k%8)*16 + (m%8)*2 (core
// matrices of 8 k-rows x 8 m-values).  Two MMAs read it with the two possible
// assignments of the core-matrix strides to the descriptor's leading / stride
// byte offsets (LBO = 128, SBO = 2048 and the swap); the buffer is sized so
// that either reading stays inside it.  out [2][128][16].
__global__ void k_tc_selftest_mn(float* __restrict__ out, int* __restrict__ flag) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char* sA = dyn;                 // 40 KB region, the tile in its first 4 KB
  unsigned char* sB = dyn + 40 * 1024;     // 512 B
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = tid; t < 40 * 1024 / 4; t += blockDim.x) reinterpret_cast<uint32_t*>(sA)[t] = 0u;
  __syncthreads();
  for (int t = tid; t < 128 * 16; t += blockDim.x) {
    const int r = t / 16, k = t % 16;
    const uint32_t off = (r >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (r & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(sA + off) = __float2bfloat16((float)((r + 2 * k) % 7 - 3));
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
    const uint32_t idesc = idesc_bf16(128, 16) | (1u << 15);   // A MN-major
    const uint64_t bd = sdesc(smem_u32(sB), 128, 256);
    mma_bf16(tmem, sdesc(smem_u32(sA), 128, 2048), bd, idesc, 0);
    mma_bf16(tmem + 16, sdesc(smem_u32(sA), 2048, 128), bd, idesc, 0);
    commit(smem_u32(&mbar));
  }
  const bool ok = mbar_wait(smem_u32(&mbar), 0);
  fence_after();
  if (!ok && lane == 0) atomicExch(flag, 1);
  float v0[16], v1[16];
  tc_read1(tmem, 0, v0);
  tc_read1(tmem, 1, v1);
  for (int q = 0; q < 16; ++q) {
    out[(32 * warp + lane) * 16 + q] = ok ? v0[q] : 0.0f;
    out[2048 + (32 * warp + lane) * 16 + q] = ok ? v1[q] : 0.0f;
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

extern "C" int dgfas_tc_selftest_mn(float* out_host, int* timeout_host) {
  if (!out_host || !timeout_host) return DGFAS_ERR_INVALID;
  float* d = nullptr;
  int* f = nullptr;
  const int smem = 40 * 1024 + 1024;
  CK(cudaFuncSetAttribute(k_tc_selftest_mn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CK(cudaMalloc(&d, 2 * 128 * 16 * sizeof(float)));
  CK(cudaMalloc(&f, sizeof(int)));
  CK(cudaMemset(f, 0, sizeof(int)));
  k_tc_selftest_mn<<<1, 128, smem>>>(d, f);
  ++g_kernels;
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out_host, d, 2 * 128 * 16 * sizeof(float), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(timeout_host, f, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(d);
  cudaFree(f);
  return DGFAS_OK;
}
