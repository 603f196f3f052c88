// aa_gemm_tc.cu -- C = A B^T for the learned warm start on the fifth-
// generation tensor cores of sm_103a.
//
// A [M x K] and B [N x K] are BF16, both K-contiguous (row-major with
// leading dimensions lda, ldb).  One CTA computes a 128 x BN tile of C:
//   * one thread issues tensor-memory-accelerator copies
//     (cp.async.bulk.tensor.2d, 128-byte swizzle) of 128 x 64 and BN x 64
//     operand tiles into a ring of shared-memory stages (full / empty
//     mbarriers);
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
//     N = BN, K = 16 per instruction) with the accumulator in tensor memory
//     (TMEM), and frees each stage with tcgen05.commit;
//   * after the last K block all four warps read the accumulator back with
//     tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows of the tile) and
//     apply the epilogue of aa_gemm_bf16_nt (bias, GELU, BF16 or FP32 store,
//     pre-activation store, accumulation into an FP32 C).
// The tensor maps zero-fill out-of-range rows and K columns, so ragged M, N
// and K need no special path; the epilogue bounds-checks its stores.
//
// Every mbarrier wait is bounded (one second on the device's global timer).
// A role that gives up raises a shared abort flag that ends the others'
// waits; the CTA then lets its copies in flight land (bounded), writes NaN
// over its tile, frees its TMEM, records the timeout for aa_gemm_tc_status
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/aa.h"

namespace {

constexpr int TC_BM = 128;       // rows of C per CTA: one MMA of M = 128
constexpr int TC_BK = 64;        // K per stage: 64 BF16 = one 128-byte swizzled row
constexpr int TC_THREADS = 128;  // 4 warps: warp w reads TMEM lanes 32w..32w+31

template <int BN>
struct TcCfg {
  static constexpr int STAGES = BN == 256 ? 4 : 6;
  static constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2;  // 16 KB
  static constexpr uint32_t B_BYTES = BN * TC_BK * 2;     // 16 or 32 KB
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;  // + slack for 1024-byte alignment
};

__device__ int g_tc_timeout;  // set by a CTA whose bounded wait ran out

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtime_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mb_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mb_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, "
      "0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity; false after one second on the
// global timer, or as soon as *abort is set by another role (abort may be
// null: no early exit).
__device__ bool mb_wait(uint32_t bar, uint32_t parity, volatile int *abort) {
  if (mb_try(bar, parity)) return true;
  const uint64_t t0 = gtime_ns();
  for (uint32_t i = 0; i < (1u << 26); ++i) {
    if (mb_try(bar, parity)) return true;
    if ((i & 63u) == 63u) {
      if (abort && *abort) return false;
      if (gtime_ns() - t0 > 1000000000ull) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by the
// tensor map with 128-byte swizzle: rows of 128 bytes, 8-row swizzle atoms
// 1024 bytes apart (stride byte offset), the leading byte offset unused for
// a K extent inside one atom; bits 46-48 = 0b001, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
template <int BN>
__device__ __forceinline__ uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, "
      "%3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

// Epilogue of one thread: 32 accumulator columns of row `row` starting at
// column `col` (bias, accumulation into FP32 C, pre-activation store, GELU,
// BF16 or FP32 store; vector accesses when the chunk is whole and aligned).
__device__ __forceinline__ void store_chunk(float (&v)[32], int row, int col, int N, void *C, int ldc,
                                            const float *__restrict__ bias, float *P, int ldp, int epi,
                                            bool vec32, bool vec16, bool vecp) {
  const bool full = col + 32 <= N;
  if (epi & 1) {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (col + i < N) v[i] += __ldg(bias + col + i);
  }
  if (epi & 16) {
    const float *cr = (const float *)C + (size_t)row * ldc + col;
    if (full && vec32) {
#pragma unroll
      for (int i = 0; i < 32; i += 4) {
        const float4 q = *(const float4 *)(cr + i);
        v[i] += q.x;
        v[i + 1] += q.y;
        v[i + 2] += q.z;
        v[i + 3] += q.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (col + i < N) v[i] += cr[i];
    }
  }
  if (epi & 8) {
    float *pr = P + (size_t)row * ldp + col;
    if (full && vecp) {
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *(float4 *)(pr + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (col + i < N) pr[i] = v[i];
    }
  }
  if (epi & 2) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = gelu_f(v[i]);
  }
  if (epi & 4) {
    __nv_bfloat16 *cr = (__nv_bfloat16 *)C + (size_t)row * ldc + col;
    if (full && vec16) {
#pragma unroll
      for (int i = 0; i < 32; i += 8) {
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[i], v[i + 1]);
        const __nv_bfloat162 h1 = __floats2bfloat162_rn(v[i + 2], v[i + 3]);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[i + 4], v[i + 5]);
        const __nv_bfloat162 h3 = __floats2bfloat162_rn(v[i + 6], v[i + 7]);
        uint4 q;
        q.x = *(const uint32_t *)&h0;
        q.y = *(const uint32_t *)&h1;
        q.z = *(const uint32_t *)&h2;
        q.w = *(const uint32_t *)&h3;
        *(uint4 *)(cr + i) = q;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (col + i < N) cr[i] = __float2bfloat16_rn(v[i]);
    }
  } else {
    float *cr = (float *)C + (size_t)row * ldc + col;
    if (full && vec32) {
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *(float4 *)(cr + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (col + i < N) cr[i] = v[i];
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int M, int N, int K, void *C, int ldc, const float *__restrict__ bias, float *P,
                   int ldp, int epi) {
  using Cfg = TcCfg<BN>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S], bar_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int nk = (K + TC_BK - 1) / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(su32(&bar_full[s]), 1);
      mb_init(su32(&bar_empty[s]), 1);
    }
    mb_init(su32(&bar_done), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {  // the whole warp allocates BN TMEM columns (a power of two >= 32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&s_tmem)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // producer: stage s holds K block kb = s, s + S, ...; a stage is reused
    // once the MMAs that read it have committed to its empty barrier
    int kb = 0;
    for (; kb < nk; ++kb) {
      const int s = kb % S;
      if (kb >= S && !mb_wait(su32(&bar_empty[s]), ((kb / S) & 1) ^ 1, &s_abort)) {
        s_abort = 1;
        break;
      }
      const uint32_t full = su32(&bar_full[s]);
      const uint32_t dst = base + (uint32_t)s * Cfg::STAGE_BYTES;
      mb_expect_tx(full, Cfg::STAGE_BYTES);
      tma_load_2d(dst, &tmA, kb * TC_BK, m0, full);
      tma_load_2d(dst + Cfg::A_BYTES, &tmB, kb * TC_BK, n0, full);
    }
    if (s_abort) {  // let the copies already issued land before the CTA exits
      for (int j = (kb > S ? kb - S : 0); j < kb; ++j)
        (void)mb_wait(su32(&bar_full[j % S]), (j / S) & 1, nullptr);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16<BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % S;
      if (!mb_wait(su32(&bar_full[s]), (kb / S) & 1, &s_abort)) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = base + (uint32_t)s * Cfg::STAGE_BYTES, b0 = a0 + Cfg::A_BYTES;
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k)  // 16 BF16 = 32 bytes along the swizzled row
        umma_bf16(tmem, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc,
                  (kb | k) != 0 ? 1u : 0u);
      umma_commit(su32(&bar_empty[s]));
    }
    umma_commit(su32(&bar_done));  // arrives once every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: row m0 + 32 warp + lane, BN columns in chunks of 32
  const bool good =
      __all_sync(0xffffffffu, mb_wait(su32(&bar_done), 0, nullptr) && !s_abort);  // warp-uniform
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  const bool vec32 = ((ldc & 3) == 0) && (((uintptr_t)C & 15u) == 0);
  const bool vec16 = ((ldc & 7) == 0) && (((uintptr_t)C & 15u) == 0);
  const bool vecp = P && ((ldp & 3) == 0) && (((uintptr_t)P & 15u) == 0);
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    if (n0 + c0 >= N) break;  // warp-uniform: tcgen05.ld needs the whole warp
    float v[32];
    if (good) {
      tmem_ld32(trow + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = __int_as_float(0x7fc00000);
    }
    if (row < M) store_chunk(v, row, n0 + c0, N, C, ldc, bias, P, ldp, epi, vec32, vec16, vecp);
    __syncwarp();  // reconverge before the next warp-wide tcgen05.ld
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                 : "memory");
  }
  if (threadIdx.x == 0 && !good) atomicExch(&g_tc_timeout, 1);
}


// Persistent form for grids of more tiles than SMs: one CTA per SM walks the
// tiles tile = blockIdx.x + i gridDim.x.  Warp 0 (one thread) keeps the
// stage ring full across tile boundaries, warp 1 (one thread) issues the MMAs
// of tile i into accumulator i % 2 of two in tensor memory (2 BN columns),
// and warps 2-5 read accumulator i % 2 back while the MMAs of tile i + 1 run
// into the other one.  Accumulator hand-off: tfull[a] (tcgen05.commit after
// the tile's last MMA) and tempty[a] (one arrive per epilogue warp after its
// last tcgen05.ld of the tile).  Epilogue warp w reads TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31.  Waits, abort and clean-up as in
// gemm_tc_kernel.
constexpr int TCP_THREADS = 192;

__device__ __forceinline__ void mb_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(TCP_THREADS, 1)
    gemm_tcp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    int M, int N, int K, void *C, int ldc, const float *__restrict__ bias, float *P,
                    int ldp, int epi) {
  using Cfg = TcCfg<BN>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S], bar_tfull[2], bar_tempty[2], bar_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const int tiles_n = (N + BN - 1) / BN;
  const int ntiles = tiles_n * ((M + TC_BM - 1) / TC_BM);
  const int nk = (K + TC_BK - 1) / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(su32(&bar_full[s]), 1);
      mb_init(su32(&bar_empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mb_init(su32(&bar_tfull[a]), 1);
      mb_init(su32(&bar_tempty[a]), 4);
    }
    mb_init(su32(&bar_done), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&s_tmem)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  bool good = true;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;  // K blocks issued so far, over all tiles
      for (int tile = blockIdx.x; tile < ntiles && !s_abort; tile += gridDim.x) {
        const int m0 = (tile / tiles_n) * TC_BM, n0 = (tile % tiles_n) * BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % S;
          if (g >= S && !mb_wait(su32(&bar_empty[s]), ((g / S) & 1) ^ 1, &s_abort)) {
            s_abort = 1;
            break;
          }
          const uint32_t full = su32(&bar_full[s]);
          const uint32_t dst = base + (uint32_t)s * Cfg::STAGE_BYTES;
          mb_expect_tx(full, Cfg::STAGE_BYTES);
          tma_load_2d(dst, &tmA, kb * TC_BK, m0, full);
          tma_load_2d(dst + Cfg::A_BYTES, &tmB, kb * TC_BK, n0, full);
        }
      }
      if (s_abort) {  // let the copies already issued land before the CTA exits
        for (int j = (g > S ? g - S : 0); j < g; ++j)
          (void)mb_wait(su32(&bar_full[j % S]), (j / S) & 1, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16<BN>();
      int g = 0, i = 0;
      for (int tile = blockIdx.x; tile < ntiles && !s_abort; tile += gridDim.x, ++i) {
        const int acc = i & 1;
        // the epilogue has drained this accumulator's previous tile
        if (i >= 2 && !mb_wait(su32(&bar_tempty[acc]), ((i >> 1) & 1) ^ 1, &s_abort)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % S;
          if (!mb_wait(su32(&bar_full[s]), (g / S) & 1, &s_abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = base + (uint32_t)s * Cfg::STAGE_BYTES, b0 = a0 + Cfg::A_BYTES;
#pragma unroll
          for (int k = 0; k < TC_BK / 16; ++k)
            umma_bf16(d, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc,
                      (kb | k) != 0 ? 1u : 0u);
          umma_commit(su32(&bar_empty[s]));
        }
        if (!ok) {
          s_abort = 1;
          break;
        }
        umma_commit(su32(&bar_tfull[acc]));
      }
      umma_commit(su32(&bar_done));  // arrives once every MMA issued above has completed
      (void)mb_wait(su32(&bar_done), 0, nullptr);
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const bool vec32 = ((ldc & 3) == 0) && (((uintptr_t)C & 15u) == 0);
    const bool vec16 = ((ldc & 7) == 0) && (((uintptr_t)C & 15u) == 0);
    const bool vecp = P && ((ldp & 3) == 0) && (((uintptr_t)P & 15u) == 0);
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int acc = i & 1;
      good = __all_sync(0xffffffffu, mb_wait(su32(&bar_tfull[acc]), (i >> 1) & 1, &s_abort));
      if (!good) {
        if (lane == 0) s_abort = 1;  // stop the other roles too
        break;
      }
      tc_fence_after();
      const int m0 = (tile / tiles_n) * TC_BM, n0 = (tile % tiles_n) * BN;
      const int row = m0 + q * 32 + lane;
      const uint32_t trow = tmem + (uint32_t)(acc * BN) + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;  // warp-uniform
        float v[32];
        tmem_ld32(trow + (uint32_t)c0, v);
        if (row < M) store_chunk(v, row, n0 + c0, N, C, ldc, bias, P, ldp, epi, vec32, vec16, vecp);
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mb_arrive(su32(&bar_tempty[acc]));
    }
    if (!good) {
      // tiles this warp did not finish: NaN over its rows of them
      for (int tile = blockIdx.x + i * (int)gridDim.x; tile < ntiles; tile += gridDim.x) {
        const int m0 = (tile / tiles_n) * TC_BM, n0 = (tile % tiles_n) * BN;
        const int row = m0 + q * 32 + lane;
        for (int c0 = 0; c0 < BN && n0 + c0 < N; c0 += 32) {
          float v[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) v[k] = __int_as_float(0x7fc00000);
          if (row < M)
            store_chunk(v, row, n0 + c0, N, C, ldc, nullptr, P, ldp, epi & ~(1 | 2 | 16), vec32,
                        vec16, vecp);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
  }
  if (threadIdx.x == 64 && s_abort) atomicExch(&g_tc_timeout, 1);
}

// ------------------------------------------------------------------- host

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return (EncodeTiledFn)p;
  }();
  return fn;
}

// 2D map over a [rows x K] BF16 matrix (K contiguous, leading dimension ld
// elements): boxes of 64 K columns by box_rows rows, 128-byte swizzle,
// zero fill outside the matrix.
bool make_map(CUtensorMap *map, const void *ptr, int rows, int K, int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2u};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1u, 1u};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// SMs of the current device (0 if the query fails).
int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return n;
}

template <int BN>
int launch_tc(int M, int N, int K, const void *A, int lda, const void *B, int ldb, void *C, int ldc,
              const float *bias, float *pre, int ldp, int epi, cudaStream_t stream) {
  using Cfg = TcCfg<BN>;
  if (cudaFuncSetAttribute(gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           Cfg::SMEM) != cudaSuccess)
    return AA_ECUDA;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, TC_BM) || !make_map(&mb, B, N, K, ldb, BN)) return AA_ECUDA;
  dim3 grid((N + BN - 1) / BN, (M + TC_BM - 1) / TC_BM);
  if (grid.y > 65535) return AA_EINVAL;
  const int nsm = sm_count();
  if (nsm > 0 && (long)grid.x * grid.y > 2L * nsm) {
    // more than two waves of tiles: the persistent form, one CTA per SM
    if (cudaFuncSetAttribute(gemm_tcp_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg::SMEM) != cudaSuccess)
      return AA_ECUDA;
    gemm_tcp_kernel<BN><<<nsm, TCP_THREADS, Cfg::SMEM, stream>>>(ma, mb, M, N, K, C, ldc, bias, pre,
                                                                 ldp, epi);
  } else {
    gemm_tc_kernel<BN><<<grid, TC_THREADS, Cfg::SMEM, stream>>>(ma, mb, M, N, K, C, ldc, bias, pre,
                                                                ldp, epi);
  }
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" int aa_gemm_bf16_nt_tc(int M, int N, int K, const void *A, int lda, const void *B,
                                  int ldb, void *C, int ldc, const float *bias, float *pre, int ldp,
                                  int epi, void *stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return AA_EINVAL;
  if (K % 8 || lda % 8 || ldb % 8 || lda < K || ldb < K || !al16(A) || !al16(B)) return AA_EINVAL;
  if (ldc < N || ((epi & 8) && ldp < N)) return AA_EINVAL;
  if (((epi & 1) && !bias) || ((epi & 8) && !pre)) return AA_EINVAL;
  if ((epi & 16) && (epi & 4)) return AA_EINVAL;
  // 128 x 256 tiles when they still give every SM at least one tile,
  // else 128 x 128
  const long tiles256 = (long)((N + 255) / 256) * ((M + TC_BM - 1) / TC_BM);
  cudaStream_t s = (cudaStream_t)stream;
  if (N > 128 && tiles256 >= 148)
    return launch_tc<256>(M, N, K, A, lda, B, ldb, C, ldc, bias, pre, ldp, epi, s);
  return launch_tc<128>(M, N, K, A, lda, B, ldb, C, ldc, bias, pre, ldp, epi, s);
}

extern "C" int aa_gemm_tc_status(void *stream) {
  int v = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost,
                                (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return AA_ECUDA;
  if (!v) return AA_OK;
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_tc_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice,
                              (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return AA_ECUDA;
  return AA_ETIMEOUT;
}
