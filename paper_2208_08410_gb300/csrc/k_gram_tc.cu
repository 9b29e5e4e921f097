// Dense Gram accumulation G += A_b^T A_b on the 5th-generation tensor cores
// (tcgen05 + TMEM + TMA), the Gram step of the method (B = X^T X, Alg. 2;
// block by block over row batches, Sec. V-C / Alg. 3).
//
// Two kernels per row block:
//  1. prep: transpose A_b (rows x n, row-major) into At (n x Kp, K-major, the
//     row index becomes contiguous) and round every value to TF32 with
//     round-to-nearest-even.  For TF32X3 it also writes lo = tf32(a - hi), so
//     a = hi + lo to ~2^-22 relative and hi*hi + hi*lo + lo*hi recovers the
//     FP32 product to about FP32 accuracy (3xTF32, Ootomo & Yokota 2022).
//     For BF16X3 it writes two BF16 parts hi = bf16(a), mid = bf16(a - hi)
//     (both nearest-even) and the products hi*hi + hi*mid + mid*hi run as
//     kind::f16 MMAs (BF16 x 3, Henry, Tang & Heinecke 2019).
//     Kp is rows rounded up to one stage of K (32 TF32 or 64 BF16 rows) and
//     the pad is zero.
//  2. syrk: a persistent warp-specialised kernel.  A work unit is one
//     128 x 256 tile (I, J) of G with J0 <= I0 + 127 (only tiles touching the
//     lower triangle: the symmetric task reuse of Sec. V-C) and one slice of
//     the K = row range.  Warp 0 streams 128-row (A operand) and 256-row
//     (B operand) slabs of At into a 4-stage shared-memory ring with TMA
//     (64-byte swizzle rows for the split precisions, 128-byte for plain
//     TF32; no multicast); warp 1 issues tcgen05.mma kind::tf32
//     (M=128, N=256, K=8) or kind::f16 with BF16 operands (K=16) into one of
//     two 256-column TMEM accumulators, one
//     short K segment at a time; warps 2-17 drain the other accumulator with
//     tcgen05.ld into FP32 registers (round-to-nearest adds), so draining one
//     segment overlaps the MMAs of the next, and add each unit's sum into the
//     FP64 G with coalesced atomics.
// Every wait is bounded (global timer); on timeout the kernel raises an error
// flag, stops issuing, waits (bounded) for its own copies and MMAs, frees
// TMEM and returns.
//
// Two more uses of the same kernels:
//  - a column block of a wide A (m < n, Eq. 3: the Gram is A A^T): its
//    contraction index is already contiguous in memory, so prep_rows_kernel
//    only rounds and splits (no transpose) before the same SYRK;
//  - one task of the orthogonal batching (Sec. V-C, Fig. 2c-d): panel J is
//    prepped into rows [0, bs) of the operand and panel I into rows
//    [bs, 2 bs), and the SYRK visits only the rectangle of tiles that holds
//    A_J^T A_I (rectangular mode: every element of those tiles is stored).
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace tsvd {
namespace {

// ---------------------------------------------------------------- prep kernel
// At[c][r] = round(A[r][c]) (and the second part).  A block of 32 x 8 threads
// moves a 32-row x 128-column strip as four 32 x 32 tiles through shared
// memory, so both the reads (along a row of A) and the writes (along a row of
// At) are coalesced; 16 loads per thread are in flight before the first store.
template <int PREC>
__global__ void __launch_bounds__(256) prep_kernel(const float *__restrict__ A, int64_t rows, int64_t n, int64_t ld,
                                                   void *__restrict__ hi_, void *__restrict__ lo_, int64_t Kp) {
  __shared__ float s[4][32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t row_strips = Kp / 32, strips = row_strips * ((n + 127) / 128);
  for (int64_t strip = blockIdx.x; strip < strips; strip += gridDim.x) {
  const int64_t r0 = (strip % row_strips) * 32;
  const int64_t c0 = (strip / row_strips) * 128;
  __syncthreads();  // the previous strip's reads of s are done
#pragma unroll
  for (int t = 0; t < 4; ++t) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + ty + 8 * i, c = c0 + 32 * t + tx;
      s[t][ty + 8 * i][tx] = (r < rows && c < n) ? __ldg(A + r * ld + c) : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 4; ++t) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t c = c0 + 32 * t + ty + 8 * i, r = r0 + tx;
      if (c < n && r < Kp) {
        const float x = s[t][tx][ty + 8 * i];
        if (PREC == TSVD_GRAM_BF16X3) {
          const uint16_t h = bf16_rne_bits(x);
          static_cast<uint16_t *>(hi_)[c * Kp + r] = h;
          static_cast<uint16_t *>(lo_)[c * Kp + r] = bf16_rne_bits(x - bf16_bits_value(h));  // x - h is exact
        } else {
          const float h = tf32_rne(x);
          static_cast<float *>(hi_)[c * Kp + r] = h;
          if (PREC == TSVD_GRAM_TF32X3) static_cast<float *>(lo_)[c * Kp + r] = tf32_rne(x - h);
        }
      }
    }
  }
  }
}

// The same rounding (+ split) for an operand whose contraction index is
// already contiguous: At[c][r] = round(X[r][c]) with X[r][c] = A[c ld + r]
// (the column block of a wide A, whose Gram A A^T is Eq. 3's).  No transpose:
// each thread reads and writes four consecutive r of one row c; r in
// [rows, Kp) is the zero pad.
template <int PREC>
__global__ void __launch_bounds__(256) prep_rows_kernel(const float *__restrict__ A, int64_t rows, int64_t n,
                                                        int64_t ld, void *__restrict__ hi_, void *__restrict__ lo_,
                                                        int64_t Kp, int vec) {
  const int64_t q4 = Kp / 4, total = n * q4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / q4, r = (i % q4) * 4;
    const float *src = A + c * ld + r;
    float x[4];
    if (vec && r + 3 < rows) {
      const float4 t = __ldg(reinterpret_cast<const float4 *>(src));
      x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = r + j < rows ? __ldg(src + j) : 0.f;
    }
    if (PREC == TSVD_GRAM_BF16X3) {
      uint16_t h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        h[j] = bf16_rne_bits(x[j]);
        l[j] = bf16_rne_bits(x[j] - bf16_bits_value(h[j]));  // x - h is exact
      }
      *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(hi_) + c * Kp + r) =
          make_uint2((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16));
      *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(lo_) + c * Kp + r) =
          make_uint2((uint32_t)l[0] | ((uint32_t)l[1] << 16), (uint32_t)l[2] | ((uint32_t)l[3] << 16));
    } else {
      float h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = tf32_rne(x[j]);
      *reinterpret_cast<float4 *>(static_cast<float *>(hi_) + c * Kp + r) = make_float4(h[0], h[1], h[2], h[3]);
      if (PREC == TSVD_GRAM_TF32X3)
        *reinterpret_cast<float4 *>(static_cast<float *>(lo_) + c * Kp + r) =
            make_float4(tf32_rne(x[0] - h[0]), tf32_rne(x[1] - h[1]), tf32_rne(x[2] - h[2]), tf32_rne(x[3] - h[3]));
    }
  }
}

// ---------------------------------------------------------------- syrk kernel
struct TcArgs {
  double *G;
  int64_t ldg;        // row stride of G
  int rect_bi0;       // rectangular mode (rect_nbj > 0): I blocks rect_bi0 + t / rect_nbj,
  int rect_nbj;       // J blocks t % rect_nbj, every element of those tiles stored
  int64_t n;
  int64_t Kp;         // padded K (rows) of At
  int64_t ksplit;     // rows per work unit (multiple of stage rows * seg_stages)
  int seg_stages;     // stages per TMEM accumulation segment
  int n_splits;
  int n_tiles;
  int n_iblk;         // ceil(n / 128)
  int *err;
  uint64_t wait_ns;   // limit of the pipeline waits (kWaitLimitNs unless a caller sets a shorter one)
};

// tile t -> (bi, bj): tiles are listed by I block; block bi has bi/2 + 1 tiles
__device__ __forceinline__ void tc_tile(int t, int &bi, int &bj) {
  // C(b) = number of tiles before block b: q(q+1) for b = 2q, (q+1)^2 for b = 2q+1
  int lo = 0, hi = 1 << 16;
  while (lo < hi) {  // largest b with C(b) <= t
    const int mid = (lo + hi + 1) >> 1;
    const long long q = mid >> 1;
    const long long c = (mid & 1) ? (q + 1) * (q + 1) : q * (q + 1);
    if (c <= t) lo = mid; else hi = mid - 1;
  }
  const long long q = lo >> 1;
  const long long cb = (lo & 1) ? (q + 1) * (q + 1) : q * (q + 1);
  bi = lo;
  bj = (int)(t - cb);
}

__device__ __forceinline__ void unit_tile(const TcArgs &a, int t, int &bi, int &bj) {
  if (a.rect_nbj > 0) {
    bi = a.rect_bi0 + t / a.rect_nbj;
    bj = t % a.rect_nbj;
  } else {
    tc_tile(t, bi, bj);
  }
}

// Stage geometry of the dense SYRK: one stage holds ROWB bytes of K (one
// swizzle row) for the 128-row and 256-row slabs of every part.  The split
// precisions take 64-byte rows (16 TF32 or 32 BF16 indices per stage, four
// 48 KB stages); plain TF32 takes 128-byte rows (four 48 KB stages).  Both
// fill 192 KB of shared memory; the shorter rows of the split precisions give
// the TMA three stages of lead instead of one at the same bytes in flight.
template <int PREC, int ROWB>
struct Geo {
  static constexpr int kParts = Cfg<PREC>::kParts;
  static constexpr int kTK = ROWB / Cfg<PREC>::kElem;  // K rows per stage
  static constexpr int kASlab = TM * ROWB, kBSlab = TN * ROWB;
  static constexpr int kStageBytes = kParts * (kASlab + kBSlab);
  static constexpr int kStages = (192 * 1024 / kStageBytes) < 8 ? 192 * 1024 / kStageBytes : 8;
  static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int kMmaPerStage = ROWB / MMA_K_BYTES;  // MMAs per part product and stage
};

// The tensor core adds each MMA into the FP32 TMEM accumulator with a
// directed (toward-zero) rounding, so a long accumulation chain drifts low by
// about 0.4 ulp per MMA.  The accumulator is therefore restarted every
// `seg_stages` stages (a segment of 16-48 MMAs) and the segment sums are
// added into FP32 registers of the epilogue warps with round-to-nearest;
// only the sum over a whole work unit goes to the FP64 G.
template <int PREC, int ROWB>
__global__ void __launch_bounds__(TC_THREADS, 1)
syrk_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, TcArgs a) {
  using C = Geo<PREC, ROWB>;
  constexpr int A_SLAB = C::kASlab, B_SLAB = C::kBSlab;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::kStages * C::kStageBytes);
  // bars: full[kStages], empty[kStages], tfull[2], tempty[2], final
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * C::kStages + 5);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + C::kStages);
  const uint32_t tfull0 = smem_u32(bars + 2 * C::kStages), tempty0 = smem_u32(bars + 2 * C::kStages + 2);
  const uint32_t final_bar = smem_u32(bars + 2 * C::kStages + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TK = C::kTK;
  const int units = a.n_tiles * a.n_splits;
  const int64_t seg_rows = (int64_t)a.seg_stages * TK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, TC_EPI_WARPS);
    }
    mbar_init(final_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int t = u % a.n_tiles, sp = u / a.n_tiles;
        int bi, bj;
        unit_tile(a, t, bi, bj);
        const int64_t k0 = (int64_t)sp * a.ksplit;
        const int64_t k1 = min(a.Kp, k0 + a.ksplit);
        for (int64_t kk = k0; kk < k1; kk += TK, ++it) {
          const uint32_t s = it % C::kStages, ph = (it / C::kStages) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err, a.wait_ns)) { ok = false; break; }
          unsigned char *st = smem + s * C::kStageBytes;
          mbar_expect_tx(full0 + 8 * s, C::kStageBytes);
          const int x = (int)kk;
          tma_load_2d(smem_u32(st), &map_hi, x, bi * TM, full0 + 8 * s);
          tma_load_2d(smem_u32(st + A_SLAB), &map_hi, x, bj * TN, full0 + 8 * s);
          tma_load_2d(smem_u32(st + A_SLAB + B_SLAB / 2), &map_hi, x, bj * TN + TN / 2, full0 + 8 * s);
          if (C::kParts == 2) {
            unsigned char *sl = st + A_SLAB + B_SLAB;
            tma_load_2d(smem_u32(sl), &map_lo, x, bi * TM, full0 + 8 * s);
            tma_load_2d(smem_u32(sl + A_SLAB), &map_lo, x, bj * TN, full0 + 8 * s);
            tma_load_2d(smem_u32(sl + A_SLAB + B_SLAB / 2), &map_lo, x, bj * TN + TN / 2, full0 + 8 * s);
          }
        }
      }
      // Drain: the last kStages loads may still be in flight when the MMA
      // warp stopped early (a wait gave up here or in another CTA), so wait
      // for them to land before the CTA exits.  Every earlier load has landed:
      // its stage was refilled only after the MMAs that read it completed.  On
      // the normal path these loads were consumed and the waits return at once.
      {
        const uint32_t from = it > (uint32_t)C::kStages ? it - C::kStages : 0;
        for (uint32_t j = from; j < it; ++j) mbar_drain(full0 + 8 * (j % C::kStages), (j / C::kStages) & 1u);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t it = 0, sc = 0;  // stage counter, segment counter
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int sp = u / a.n_tiles;
        const int64_t k0 = (int64_t)sp * a.ksplit;
        const int64_t k1 = min(a.Kp, k0 + a.ksplit);
        for (int64_t g0 = k0; g0 < k1 && ok; g0 += seg_rows, ++sc) {
          const int64_t g1 = min(k1, g0 + seg_rows);
          const uint32_t acc = sc & 1u, aph = (sc >> 1) & 1u;
          if (!mbar_wait(tempty0 + 8 * acc, aph ^ 1u, a.err, a.wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem + acc * TN;
          uint32_t first = 1;
          for (int64_t kk = g0; kk < g1; kk += TK, ++it) {
            const uint32_t s = it % C::kStages, ph = (it / C::kStages) & 1u;
            if (!mbar_wait(full0 + 8 * s, ph, a.err, a.wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * C::kStageBytes);
            const uint64_t dah = umma_desc_k<ROWB>(st), dbh = umma_desc_k<ROWB>(st + A_SLAB);
#pragma unroll
            for (int kq = 0; kq < C::kMmaPerStage; ++kq) {
              const uint64_t off = (uint64_t)(kq * MMA_K_BYTES) >> 4;  // descriptor start, 16-byte units
              if (C::kParts == 2) {
                const uint32_t sl = st + A_SLAB + B_SLAB;
                const uint64_t dal = umma_desc_k<ROWB>(sl), dbl = umma_desc_k<ROWB>(sl + A_SLAB);
                umma<PREC>(dtm, dal + off, dbh + off, first ? 0u : 1u);  // small terms first
                first = 0;
                umma<PREC>(dtm, dah + off, dbl + off, 1u);
              }
              umma<PREC>(dtm, dah + off, dbh + off, first ? 0u : 1u);
              first = 0;
            }
            umma_commit(empty0 + 8 * s);  // frees the stage when these MMAs finish
          }
          if (!ok) break;
          umma_commit(tfull0 + 8 * acc);  // segment sum ready for the epilogue
        }
      }
      // wait for every MMA this thread issued before TMEM is released
      // (also after a wait gave up: the MMAs in flight complete by themselves)
      umma_commit(final_bar);
      mbar_drain(final_bar, 0);
    }
  } else {
    // ------------------------------------------------ epilogue: TMEM -> registers -> FP64 G
    const int q = warp & 3;                     // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;              // which 64 of the 256 columns
    const int row = q * 32 + lane;
    float accr[TC_EPI_COLS];
#pragma unroll
    for (int j = 0; j < TC_EPI_COLS; ++j) accr[j] = 0.f;
    uint32_t sc = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int t = u % a.n_tiles, sp = u / a.n_tiles;
      int bi, bj;
      unit_tile(a, t, bi, bj);
      const int64_t k0 = (int64_t)sp * a.ksplit;
      const int64_t k1 = min(a.Kp, k0 + a.ksplit);
      for (int64_t g0 = k0; g0 < k1; g0 += seg_rows, ++sc) {
        const uint32_t acc = sc & 1u, aph = (sc >> 1) & 1u;
        if (!mbar_wait(tfull0 + 8 * acc, aph, a.err, a.wait_ns)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * TN + h * TC_EPI_COLS;
#pragma unroll
        for (int c = 0; c < TC_EPI_COLS / 16; ++c) tmem_add16(tbase + c * 16, accr + c * 16);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
      }
      if (!ok) break;
      const int64_t gi = (int64_t)bi * TM + row;
      const int64_t jbase = (int64_t)bj * TN + h * TC_EPI_COLS;
      // columns gj <= gi of this row (the lower triangle of G), stored at G[gj][gi];
      // in rectangular mode every column of the tile
      const int jlim = gi >= a.n ? 0
                       : a.rect_nbj > 0 ? TC_EPI_COLS
                                        : (int)min((int64_t)TC_EPI_COLS, gi - jbase + 1);
      double *gp = a.G + jbase * a.ldg + gi;
      const int64_t stride = a.ldg;
#pragma unroll
      for (int j = 0; j < TC_EPI_COLS; ++j) {
        if (j < jlim) red_add_f64_from_f32(gp, accr[j]);
        gp += stride;
        accr[j] = 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

tsvd_status get_encode(EncodeTiledFn *out) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TSVD_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) {
      set_error_text("cuTensorMapEncodeTiled not available");
      return TSVD_ECUDA;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = fn;
  return TSVD_OK;
}

// At viewed as n rows of Kp elements; the box is one swizzle row of K (rowb =
// 128 or 64 bytes) by 128 rows, so every x coordinate the kernel passes is a
// multiple of rowb bytes
tsvd_status make_map(CUtensorMap *map, const void *base, int64_t n, int64_t Kp, int precision, int rowb = 128) {
  EncodeTiledFn enc;
  TSVD_TRY(get_encode(&enc));
  const bool bf = precision == TSVD_GRAM_BF16X3;
  const int64_t elem = bf ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)(Kp * elem)};
  if (rowb != 128 && rowb != 64) return TSVD_EINVAL;
  const cuuint32_t box[2] = {(cuuint32_t)(rowb / elem), (cuuint32_t)TM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         const_cast<void *>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE,
                         rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_text("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return TSVD_ECUDA;
  }
  return TSVD_OK;
}

int64_t padded_k(int64_t rows, int precision) {
  return round_up(std::max<int64_t>(rows, 1), stage_rows(precision));
}

int tc_parts(int precision) { return precision == TSVD_GRAM_TF32 ? 1 : 2; }
int64_t tc_elem(int precision) { return precision == TSVD_GRAM_BF16X3 ? 2 : 4; }

template <int PREC, int ROWB>
tsvd_status launch_syrk(const CUtensorMap &mh, const CUtensorMap &ml, const TcArgs &a, int grid,
                        cudaStream_t stream) {
  using G = Geo<PREC, ROWB>;
  TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(syrk_tc_kernel<PREC, ROWB>), G::kSmem));
  syrk_tc_kernel<PREC, ROWB><<<grid, TC_THREADS, G::kSmem, stream>>>(mh, ml, a);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace

tsvd_status tc_make_map(CUtensorMap *map, const void *base, int64_t n, int64_t Kp, int precision) {
  return make_map(map, base, n, Kp, precision);
}

size_t gram_tc_scratch_bytes(int64_t rows, int64_t n, int precision) {
  if (precision == TSVD_GRAM_FP32 || rows <= 0 || n <= 0) return 0;
  // status word (first 1024 bytes), then At (n x Kp) per part, 1024-byte aligned;
  // +1024 lets the caller's 256-byte aligned pointer be rounded up
  return 2048 + (size_t)tc_parts(precision) *
                    (size_t)round_up(n * padded_k(rows, precision) * tc_elem(precision), 1024);
}

// Swizzle row bytes of the dense SYRK's stages: 64 for the split precisions,
// 128 for plain TF32; TSVD_TC_ROW (64 or 128) overrides it.
static int tc_row_bytes(int precision) {
  const char *e = getenv("TSVD_TC_ROW");
  if (e && (atoi(e) == 64 || atoi(e) == 128)) return atoi(e);
  return precision == TSVD_GRAM_TF32 ? 128 : 64;
}

// K rows per stage of the dense SYRK
static int tc_stage_k(int precision, int rowb) { return rowb / (precision == TSVD_GRAM_BF16X3 ? 2 : 4); }

// Stages per TMEM accumulation segment: K rows per segment (bounds the
// truncation drift of one FP32 accumulation chain to 16-24 MMAs: 128 rows of
// TF32, 64 of 3xTF32, 128 of BF16x3) over the rows of a stage; TSVD_TC_SEG
// overrides the rows per segment (a multiple of the stage's rows).
static int tc_seg_stages(int precision, int rowb) {
  const int tk = tc_stage_k(precision, rowb);
  int rows = precision == TSVD_GRAM_TF32X3 ? 64 : 128;
  const char *e = getenv("TSVD_TC_SEG");
  if (e) rows = std::max(tk, atoi(e));
  return std::max(1, rows / tk);
}

namespace {

// Scratch layout of one Gram chunk: status word (first 1024 bytes), then At
// (n x Kp) per part, each 1024-byte aligned.
struct TcLayout {
  int parts = 1;
  int64_t Kp = 0;
  int *err = nullptr;
  void *hi = nullptr, *lo = nullptr;
};

tsvd_status tc_layout(int64_t rows, int64_t n, int precision, void *scratch, size_t scratch_bytes, TcLayout *L) {
  if (precision != TSVD_GRAM_TF32 && precision != TSVD_GRAM_TF32X3 && precision != TSVD_GRAM_BF16X3)
    return TSVD_EINVAL;
  if (n > (int64_t)TM * 65535) return TSVD_EUNSUPPORTED;
  if (!scratch || scratch_bytes < gram_tc_scratch_bytes(rows, n, precision)) return TSVD_EINVAL;
  if ((reinterpret_cast<uintptr_t>(scratch) & 255) != 0) return TSVD_EINVAL;
  L->parts = tc_parts(precision);
  L->Kp = padded_k(rows, precision);
  const int64_t part_bytes = round_up(n * L->Kp * tc_elem(precision), 1024);
  unsigned char *base = static_cast<unsigned char *>(scratch);
  L->err = reinterpret_cast<int *>(base);  // status word: 0 ok, nonzero = a bounded wait gave up
  const uintptr_t al = (reinterpret_cast<uintptr_t>(base) + 1024 + 1023) & ~uintptr_t(1023);
  L->hi = reinterpret_cast<void *>(al);
  L->lo = L->parts == 2 ? reinterpret_cast<void *>(al + part_bytes) : L->hi;
  if (al + (size_t)L->parts * part_bytes > reinterpret_cast<uintptr_t>(base) + scratch_bytes) return TSVD_EINVAL;
  return TSVD_OK;
}

}  // namespace

namespace {

// transpose + rounding (+ split) of A (rows x n, stride ld) into rows [0, n)
// of the At parts at hi / lo; Kp is a multiple of 32, the prep row tile
tsvd_status prep_raw(const float *A, int64_t rows, int64_t n, int64_t ld, int precision, void *hi, void *lo,
                     int64_t Kp, cudaStream_t stream) {
  const int64_t strips = (Kp / 32) * ceil_div(n, 128);
  const int64_t grid = std::min<int64_t>(strips, 0x7fffffffLL);
  dim3 block(32, 8);
  if (precision == TSVD_GRAM_BF16X3)
    prep_kernel<TSVD_GRAM_BF16X3><<<(unsigned)grid, block, 0, stream>>>(A, rows, n, ld, hi, lo, Kp);
  else if (precision == TSVD_GRAM_TF32X3)
    prep_kernel<TSVD_GRAM_TF32X3><<<(unsigned)grid, block, 0, stream>>>(A, rows, n, ld, hi, lo, Kp);
  else
    prep_kernel<TSVD_GRAM_TF32><<<(unsigned)grid, block, 0, stream>>>(A, rows, n, ld, hi, lo, Kp);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// K slices: about 8 units per SM balance the persistent grid; fewer, longer
// units keep the FP64 reductions into G (one 128 x 256 tile per unit) small,
// so slices are never shorter than 4096 rows
void tc_ksplit(TcArgs &a, int precision, int rowb, int sms) {
  const int64_t quantum = (int64_t)tc_stage_k(precision, rowb) * a.seg_stages;
  const int64_t want_units = 8LL * sms;
  int64_t splits = std::max<int64_t>(1, ceil_div(want_units, a.n_tiles));
  int64_t ks = round_up(ceil_div(a.Kp, splits), quantum);
  ks = std::max<int64_t>(ks, std::min<int64_t>(round_up(4096, quantum), round_up(a.Kp, quantum)));
  const char *e = getenv("TSVD_TC_KSPLIT");
  if (e) ks = std::max<int64_t>(quantum, round_up(atoll(e), quantum));
  a.ksplit = ks;
  a.n_splits = (int)ceil_div(a.Kp, ks);
}

tsvd_status run_syrk(const TcLayout &L, const TcArgs &a0, int precision, int sms, cudaStream_t stream,
                     cudaEvent_t ev0, cudaEvent_t ev1, bool reset_status) {
  TcArgs a = a0;
  const int rowb = tc_row_bytes(precision);
  a.seg_stages = tc_seg_stages(precision, rowb);
  CUtensorMap mh, ml;
  TSVD_TRY(make_map(&mh, L.hi, a.n, a.Kp, precision, rowb));
  TSVD_TRY(make_map(&ml, L.lo, a.n, a.Kp, precision, rowb));
  tc_ksplit(a, precision, rowb, sms);
  a.err = L.err;
  if (a.wait_ns == 0) a.wait_ns = kWaitLimitNs;
  if (reset_status) TSVD_CUDA(cudaMemsetAsync(L.err, 0, 4, stream));
  const int64_t units = (int64_t)a.n_tiles * a.n_splits;
  const int grid = (int)std::min<int64_t>(units, sms);
  if (ev0) TSVD_CUDA(cudaEventRecord(ev0, stream));
  if (precision == TSVD_GRAM_TF32)
    TSVD_TRY((rowb == 64 ? launch_syrk<TSVD_GRAM_TF32, 64>(mh, ml, a, grid, stream)
                         : launch_syrk<TSVD_GRAM_TF32, 128>(mh, ml, a, grid, stream)));
  else if (precision == TSVD_GRAM_TF32X3)
    TSVD_TRY((rowb == 64 ? launch_syrk<TSVD_GRAM_TF32X3, 64>(mh, ml, a, grid, stream)
                         : launch_syrk<TSVD_GRAM_TF32X3, 128>(mh, ml, a, grid, stream)));
  else
    TSVD_TRY((rowb == 64 ? launch_syrk<TSVD_GRAM_BF16X3, 64>(mh, ml, a, grid, stream)
                         : launch_syrk<TSVD_GRAM_BF16X3, 128>(mh, ml, a, grid, stream)));
  if (ev1) TSVD_CUDA(cudaEventRecord(ev1, stream));
  return TSVD_OK;
}

}  // namespace

tsvd_status launch_gram_tc_t(const float *A, int64_t rows, int64_t n, int64_t ld, double *G, int precision,
                             void *scratch, size_t scratch_bytes, cudaStream_t stream, cudaEvent_t ev0,
                             cudaEvent_t ev1, bool reset_status, uint64_t wait_ns) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  if (di.cc_major != 10) return TSVD_EUNSUPPORTED;
  TcLayout L;
  TSVD_TRY(tc_layout(rows, n, precision, scratch, scratch_bytes, &L));
  const int vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const int64_t total = n * (L.Kp / 4);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), (int64_t)di.sms * 16));
  if (precision == TSVD_GRAM_BF16X3)
    prep_rows_kernel<TSVD_GRAM_BF16X3><<<grid, 256, 0, stream>>>(A, rows, n, ld, L.hi, L.lo, L.Kp, vec);
  else if (precision == TSVD_GRAM_TF32X3)
    prep_rows_kernel<TSVD_GRAM_TF32X3><<<grid, 256, 0, stream>>>(A, rows, n, ld, L.hi, L.lo, L.Kp, vec);
  else
    prep_rows_kernel<TSVD_GRAM_TF32><<<grid, 256, 0, stream>>>(A, rows, n, ld, L.hi, L.lo, L.Kp, vec);
  TSVD_LAUNCHED();
  return launch_gram_tc_syrk(rows, n, G, precision, scratch, scratch_bytes, stream, ev0, ev1, reset_status,
                             wait_ns);
}

tsvd_status launch_gram_tc_prep(const float *A, int64_t rows, int64_t n, int64_t ld, int precision, void *scratch,
                                size_t scratch_bytes, cudaStream_t stream) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  if (di.cc_major != 10) return TSVD_EUNSUPPORTED;  // tcgen05 needs the sm_100 family
  TcLayout L;
  TSVD_TRY(tc_layout(rows, n, precision, scratch, scratch_bytes, &L));
  return prep_raw(A, rows, n, ld, precision, L.hi, L.lo, L.Kp, stream);
}

tsvd_status launch_gram_tc_syrk(int64_t rows, int64_t n, double *G, int precision, void *scratch, size_t scratch_bytes,
                                cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1, bool reset_status,
                                uint64_t wait_ns) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  if (di.cc_major != 10) return TSVD_EUNSUPPORTED;
  TcLayout L;
  TSVD_TRY(tc_layout(rows, n, precision, scratch, scratch_bytes, &L));
  // persistent tcgen05 SYRK over the lower-triangle tiles
  TcArgs a{};
  a.G = G;
  a.ldg = n;
  a.n = n;
  a.Kp = L.Kp;
  a.n_iblk = (int)ceil_div(n, TM);
  a.wait_ns = wait_ns;
  {
    const int64_t q = (a.n_iblk) >> 1;  // tiles = C(n_iblk)
    a.n_tiles = (int)((a.n_iblk & 1) ? (q + 1) * (q + 1) : q * (q + 1));
  }
  return run_syrk(L, a, precision, di.sms, stream, ev0, ev1, reset_status);
}

tsvd_status launch_gram_tc_rect(const float *AJ, const float *AI, int64_t rows, int64_t bs, int64_t nJ, int64_t nI,
                                int64_t ld, double *G, int precision, void *scratch, size_t scratch_bytes,
                                cudaStream_t stream, bool reset_status) {
  if (rows <= 0 || nJ <= 0 || nI <= 0) return TSVD_OK;
  if (bs % TN != 0 || nJ > bs || nI > bs) return TSVD_EINVAL;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  if (di.cc_major != 10) return TSVD_EUNSUPPORTED;
  TcLayout L;
  TSVD_TRY(tc_layout(rows, 2 * bs, precision, scratch, scratch_bytes, &L));
  // At rows [0, nJ): panel J; rows [bs, bs + nI): panel I.  Rows [nJ, bs) and
  // [bs + nI, 2 bs) keep whatever they held: the tiles that read them only
  // produce entries outside the J x I block, which the caller ignores
  const int64_t off = bs * L.Kp * tc_elem(precision);
  TSVD_TRY(prep_raw(AJ, rows, nJ, ld, precision, L.hi, L.lo, L.Kp, stream));
  TSVD_TRY(prep_raw(AI, rows, nI, ld, precision, static_cast<unsigned char *>(L.hi) + off,
                    static_cast<unsigned char *>(L.lo) + off, L.Kp, stream));
  TcArgs a{};
  a.G = G;
  a.ldg = 2 * bs;
  a.n = 2 * bs;
  a.Kp = L.Kp;
  a.n_iblk = (int)ceil_div(2 * bs, TM);
  a.rect_bi0 = (int)(bs / TM);
  a.rect_nbj = (int)ceil_div(nJ, TN);
  a.n_tiles = (int)ceil_div(nI, TM) * a.rect_nbj;
  return run_syrk(L, a, precision, di.sms, stream, nullptr, nullptr, reset_status);
}

tsvd_status launch_gram_tc(const float *A, int64_t rows, int64_t n, int64_t ld, double *G, int precision,
                           void *scratch, size_t scratch_bytes, cudaStream_t stream, cudaEvent_t ev0,
                           cudaEvent_t ev1, bool reset_status, uint64_t wait_ns) {
  if (rows <= 0) return TSVD_OK;
  TSVD_TRY(launch_gram_tc_prep(A, rows, n, ld, precision, scratch, scratch_bytes, stream));
  return launch_gram_tc_syrk(rows, n, G, precision, scratch, scratch_bytes, stream, ev0, ev1, reset_status,
                             wait_ns);
}

}  // namespace tsvd
