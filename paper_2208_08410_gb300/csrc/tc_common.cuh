// tcgen05 / TMA / mbarrier helpers (inline PTX) and the operand rounding
// shared by the tensor-core Gram kernels: the per-row-block SYRK of the dense
// plan (k_gram_tc.cu) and the grouped SYRK of the server (k_serve_tc.cu).
// Tile geometry: MMA M = 128 rows of At (block I) by N = 256 rows (block J);
// one pipeline stage holds one 128-byte swizzle row of K for both slabs
// (32 TF32 or 64 BF16 contraction indices).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tsvd {
namespace {

constexpr int TC_EPI_WARPS = 16;  // 4 TMEM lane quarters x 4 column groups of 64
constexpr int TC_EPI_COLS = 64;   // accumulator columns per epilogue thread
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;  // TMA warp, MMA warp, epilogue warps
constexpr int TM = 128;          // MMA M (rows of At from block I)
constexpr int TN = 256;          // MMA N (rows of At from block J)
constexpr int ROW_BYTES = 128;   // K bytes per stage: one 128-byte swizzle row
constexpr int A_SLAB = TM * ROW_BYTES;  // 16 KB
constexpr int B_SLAB = TN * ROW_BYTES;  // 32 KB
constexpr int MMA_K_BYTES = 32;  // K bytes per MMA (8 TF32 or 16 BF16)

template <int PREC>
struct Cfg {
  static constexpr bool kBf16 = PREC == TSVD_GRAM_BF16X3;
  static constexpr int kElem = kBf16 ? 2 : 4;                       // bytes per operand element
  static constexpr int kTK = ROW_BYTES / kElem;                     // K rows per stage
  static constexpr int kParts = PREC == TSVD_GRAM_TF32 ? 1 : 2;     // hi (and lo / mid) operands
  static constexpr int kStageBytes = kParts * (A_SLAB + B_SLAB);
  static constexpr int kStages = kParts == 2 ? 2 : 4;
  static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
};

__host__ __device__ constexpr int stage_rows(int precision) { return precision == TSVD_GRAM_BF16X3 ? 64 : 32; }

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false on timeout (after limit_ns) or when
// *err is raised.  The clock and *err are read every 256 failed tries, or on
// every try when the limit is below 100 us (the test-only short limits).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  const uint32_t mask = limit_ns < 100000ull ? 0u : 255u;
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try(bar, parity)) return true;
    if ((spin & mask) == 0) {
      if (*(volatile int *)err) return false;
      if (global_timer_ns() - t0 > limit_ns) {
        atomicExch(err, 2);
        return false;
      }
    }
  }
}

// Wait for this CTA's own asynchronous work (a TMA load or the MMAs behind a
// commit) to complete before the CTA frees TMEM and exits.  It does not give
// up when *err is raised: that work completes by itself; the wait is bounded
// by kWaitLimitNs only as a guard.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try(bar, parity)) return true;
    if ((spin & 255u) == 0 && global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// UMMA shared-memory descriptor of a K-major operand whose rows are one
// swizzle row of ROWB bytes (128-byte or 64-byte swizzle, as the TMA wrote
// them): 8-row core-matrix groups 8 * ROWB bytes apart (SBO), start address in
// 16-byte units.
template <int ROWB>
__device__ __forceinline__ uint64_t umma_desc_k(uint32_t saddr) {
  static_assert(ROWB == 128 || ROWB == 64, "128- or 64-byte swizzle rows");
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * ROWB) >> 4) << 32;      // stride byte offset
  d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family)
  d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;  // swizzle mode: 128B (2) or 64B (4)
  return d;
}

__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) { return umma_desc_k<128>(saddr); }

// Instruction descriptor, kind::tf32: D F32, A/B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Instruction descriptor, kind::f16 with BF16 A and B: D F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

template <int PREC>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  if (PREC == TSVD_GRAM_BF16X3)
    umma_bf16(tmem_d, a, b, idesc_bf16(TM, TN), acc);
  else
    umma_tf32(tmem_d, a, b, idesc_tf32(TM, TN), acc);
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// acc[0..15] += TMEM columns [taddr, taddr+16) of this thread's lane (one
// statement so the load, its wait and the round-to-nearest adds stay together)
__device__ __forceinline__ void tmem_add16(uint32_t taddr, float *acc) {
  asm volatile(
      "{\n .reg .f32 t<16>;\n"
      " tcgen05.ld.sync.aligned.32x32b.x16.b32 {t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15}, [%16];\n"
      " tcgen05.wait::ld.sync.aligned;\n"
      " add.rn.f32 %0, %0, t0;\n add.rn.f32 %1, %1, t1;\n add.rn.f32 %2, %2, t2;\n add.rn.f32 %3, %3, t3;\n"
      " add.rn.f32 %4, %4, t4;\n add.rn.f32 %5, %5, t5;\n add.rn.f32 %6, %6, t6;\n add.rn.f32 %7, %7, t7;\n"
      " add.rn.f32 %8, %8, t8;\n add.rn.f32 %9, %9, t9;\n add.rn.f32 %10, %10, t10;\n add.rn.f32 %11, %11, t11;\n"
      " add.rn.f32 %12, %12, t12;\n add.rn.f32 %13, %13, t13;\n add.rn.f32 %14, %14, t14;\n add.rn.f32 %15, %15, t15;\n"
      "}\n"
      : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+f"(acc[4]), "+f"(acc[5]), "+f"(acc[6]),
        "+f"(acc[7]), "+f"(acc[8]), "+f"(acc[9]), "+f"(acc[10]), "+f"(acc[11]), "+f"(acc[12]), "+f"(acc[13]),
        "+f"(acc[14]), "+f"(acc[15])
      : "r"(taddr)
      : "memory");
}

// *p += (double)x with a fire-and-forget global reduction
__device__ __forceinline__ void red_add_f64_from_f32(double *p, float x) {
  asm volatile("{\n .reg .f64 d;\n cvt.f64.f32 d, %1;\n red.global.add.f64 [%0], d;\n}\n" ::"l"(p), "f"(x)
               : "memory");
}

// ---------------------------------------------------------------- TF32 rounding
// Round an FP32 value to the nearest TF32 value (10 explicit mantissa bits),
// ties to even, by integer arithmetic on the encoding; non-finite values pass.
__device__ __forceinline__ float tf32_rne(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // Inf / NaN unchanged
  return __uint_as_float((u + 0x0fffu + ((u >> 13) & 1u)) & 0xffffe000u);
}

// Round an FP32 value to the nearest BF16 value (8 significant bits), ties to
// even, returned as its 16-bit encoding; NaN stays NaN, Inf stays Inf.
__device__ __forceinline__ uint16_t bf16_rne_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ float bf16_bits_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

}  // namespace
}  // namespace tsvd
