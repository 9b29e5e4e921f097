// Left singular vectors of a dense row block (Alg. 1):
//     U_b = A_b V diag(sigma)^-1,   u_l = A v_l / ||A v_l||
// computed in one extra pass over A after all right vectors are known.
//
// A is rows x n row-major; V is n x k column-major.  A block of 256 threads
// owns 64 rows; each warp keeps 8 rows x 16 columns of partial sums in
// registers.  A lane reads four consecutive entries of a row with one 16-byte
// load (coalesced across the warp, 16 such loads in flight per lane); the
// matching 4 x 16 entries of V come from shared memory, where V is staged 256
// rows at a time, column by column (j contiguous, so the staging writes and
// the 16-byte reads are free of bank conflicts).  Each staged value of V feeds
// 8 rows.  Columns are processed 16 at a time (A is re-read for k > 16).
#include <cuda.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"

namespace tsvd {

__device__ int g_left_status;  // nonzero once a bounded wait of the TMA kernel gave up

namespace {

constexpr int LT = 256;   // threads
constexpr int LR = 8;     // rows per warp
constexpr int LK = 16;    // columns per pass
constexpr int LJ = 256;   // V rows staged per step (= 32 lanes x 4 x 2)

__global__ void __launch_bounds__(LT, 1)
left_dense_kernel(const float *__restrict__ A, int64_t rows, int64_t n, int64_t ld,
                  const float *__restrict__ V, int64_t ldv, int64_t k, const double *__restrict__ sigma,
                  float *__restrict__ U, int64_t ldu, int l0, int vec) {
  __shared__ __align__(16) float Vs[LK][LJ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * (LT / 32) * LR + (int64_t)warp * LR;
  float acc[LR][LK];
#pragma unroll
  for (int r = 0; r < LR; ++r)
#pragma unroll
    for (int t = 0; t < LK; ++t) acc[r][t] = 0.f;
  const int kc = (int)min((int64_t)LK, k - l0);
  const float *arow[LR];
#pragma unroll
  for (int r = 0; r < LR; ++r) arow[r] = A + min(row0 + r, rows - 1) * ld;  // clamp: rows past the end are not stored

  for (int64_t j0 = 0; j0 < n; j0 += LJ) {
    __syncthreads();
    for (int e = threadIdx.x; e < LJ * LK; e += LT) {
      const int jj = e % LJ, t = e / LJ;
      const int64_t j = j0 + jj;
      Vs[t][jj] = (t < kc && j < n) ? __ldg(V + (int64_t)(l0 + t) * ldv + j) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int jj = 128 * s + 4 * lane;
      const int64_t j = j0 + jj;
      float4 a[LR];
      if (vec && j + 3 < n) {
#pragma unroll
        for (int r = 0; r < LR; ++r) a[r] = __ldg(reinterpret_cast<const float4 *>(arow[r] + j));
      } else {
#pragma unroll
        for (int r = 0; r < LR; ++r) {
          a[r].x = j < n ? __ldg(arow[r] + j) : 0.f;
          a[r].y = j + 1 < n ? __ldg(arow[r] + j + 1) : 0.f;
          a[r].z = j + 2 < n ? __ldg(arow[r] + j + 2) : 0.f;
          a[r].w = j + 3 < n ? __ldg(arow[r] + j + 3) : 0.f;
        }
      }
#pragma unroll
      for (int t = 0; t < LK; ++t) {
        const float4 vq = *reinterpret_cast<const float4 *>(&Vs[t][jj]);
#pragma unroll
        for (int r = 0; r < LR; ++r) {
          float x = acc[r][t];
          x = fmaf(a[r].x, vq.x, x);
          x = fmaf(a[r].y, vq.y, x);
          x = fmaf(a[r].z, vq.z, x);
          x = fmaf(a[r].w, vq.w, x);
          acc[r][t] = x;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < LR; ++r) {
#pragma unroll
    for (int t = 0; t < LK; ++t) acc[r][t] = warp_sumf(acc[r][t]);
  }
  // lane t < kc writes column l0+t of every row
#pragma unroll
  for (int t = 0; t < LK; ++t) {
    if (lane == t && t < kc) {
      const double sg = __ldg(sigma + l0 + t);
#pragma unroll
      for (int r = 0; r < LR; ++r) {
        const int64_t row = row0 + r;
        if (row < rows) U[row + (int64_t)(l0 + t) * ldu] = sg > 0.0 ? (float)((double)acc[r][t] / sg) : 0.f;
      }
    }
  }
}


// ---------------------------------------------------------------- TMA variant
// Same arithmetic, but a persistent block streams 64-row x 128-column tiles
// of A and the matching 128 x 16 tile of V^T into a four-stage shared-memory
// ring with TMA, three tiles ahead, so HBM latency is hidden by the copy
// engine instead of by warp occupancy.  Each warp owns RW rows of the tile
// (RW x 16 accumulators per thread): 8 warps of 8 rows by default.  Per
// 128-column chunk a thread reads RW float4 of A and 16 float4 of V^T from
// shared memory for 64 RW FMAs, so 8 rows per warp move 96 KB of shared
// memory per chunk and SM (16 warps of 4 rows: 160 KB), below the 32 KB of A
// the chunk brings from HBM at the link's pace.
constexpr int TLH = 16;                         // columns of V per sweep
constexpr int TR = 64;                          // rows per tile (warps x RW)
constexpr int TJ = 128;                         // columns per chunk (32 lanes x 4)
constexpr int T_ABYTES = TR * TJ * 4;           // 32 KB
constexpr int T_VBYTES = LK * TJ * 4;           // 8 KB
constexpr int T_STAGE = T_ABYTES + T_VBYTES;    // 40 KB
constexpr int T_NST = 4;                        // stages (three tiles in flight)
constexpr int T_SMEM = T_NST * T_STAGE + 1024 + 64;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait_l(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t spin = 0;; ++spin) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if ((spin & 255u) == 255u) {
      if (*(volatile int *)&g_left_status) return false;
      if (global_timer_ns() - t0 > kWaitLimitNs) {
        atomicExch(&g_left_status, 1);
        return false;
      }
    }
  }
}

// Wait for a TMA load this CTA issued to land before the CTA exits, also after
// a wait gave up (the load completes by itself); bounded only as a guard.
__device__ __forceinline__ bool mbar_drain_l(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t spin = 0;; ++spin) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if ((spin & 255u) == 255u && global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
}

template <int RW>
__global__ void __launch_bounds__(TR / RW * 32, 1)
left_tma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV, int64_t rows,
                int64_t n, int64_t k, const double *__restrict__ sigma, float *__restrict__ U, int64_t ldu, int l0) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + T_NST * T_STAGE);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles = ceil_div_dev(rows, TR);
  const int64_t chunks = ceil_div_dev(n, TJ);
  const int kc = (int)min((int64_t)LK, k - l0);
  if (threadIdx.x == 0) {
    for (int b = 0; b < T_NST; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the block's work: tiles blockIdx.x, +gridDim.x, ...; each tile = `chunks` chunks
  const int64_t my_tiles = tiles > blockIdx.x ? ceil_div_dev(tiles - blockIdx.x, gridDim.x) : 0;
  const int64_t total = my_tiles * chunks;
  auto issue = [&](int64_t c) {  // chunk sequence number c -> stage c % T_NST
    const int64_t tile = blockIdx.x + (c / chunks) * gridDim.x;
    const int j0 = (int)((c % chunks) * TJ);
    const uint32_t st = su32(sm + (c % T_NST) * T_STAGE);
    const uint32_t bar = su32(full + (c % T_NST));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(T_STAGE) : "memory");
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(st), "l"(reinterpret_cast<uint64_t>(&mapA)), "r"(j0), "r"((int)(tile * TR)), "r"(bar) : "memory");
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(st + T_ABYTES), "l"(reinterpret_cast<uint64_t>(&mapV)), "r"(j0), "r"(l0), "r"(bar) : "memory");
  };
  if (threadIdx.x == 0) {
    for (int64_t c = 0; c < T_NST - 1 && c < total; ++c) issue(c);
  }
  constexpr int TRW = RW;
  float acc[1][TRW][TLH];
  bool ok = true;
  int64_t stop = total;  // the chunk at which a failed wait ended the loop
  for (int64_t c = 0; c < total; ++c) {
    const int64_t cj = c % chunks;
    if (cj == 0) {
#pragma unroll
      for (int r = 0; r < TRW; ++r)
#pragma unroll
        for (int t = 0; t < TLH; ++t) acc[0][r][t] = 0.f;
    }
    // stage (c + T_NST - 1) % T_NST was released by the sync at the end of iteration c - 1
    if (threadIdx.x == 0 && c + T_NST - 1 < total) issue(c + T_NST - 1);
    if (!mbar_wait_l(su32(full + (c % T_NST)), (uint32_t)((c / T_NST) & 1))) ok = false;
    if (__syncthreads_or(!ok)) {
      stop = c;
      break;
    }
    const float *As = reinterpret_cast<const float *>(sm + (c % T_NST) * T_STAGE);
    const float *Vs = reinterpret_cast<const float *>(sm + (c % T_NST) * T_STAGE + T_ABYTES);
    const int jj = 4 * lane;
#pragma unroll
    for (int h = 0; h < 1; ++h) {
      float4 a[TRW];
#pragma unroll
      for (int r = 0; r < TRW; ++r) a[r] = *reinterpret_cast<const float4 *>(As + (warp * TRW + r) * TJ + jj);
#pragma unroll
      for (int t = 0; t < TLH; ++t) {
        const float4 vq = *reinterpret_cast<const float4 *>(Vs + (h * TLH + t) * TJ + jj);
#pragma unroll
        for (int r = 0; r < TRW; ++r) {
          float x = acc[h][r][t];
          x = fmaf(a[r].x, vq.x, x);
          x = fmaf(a[r].y, vq.y, x);
          x = fmaf(a[r].z, vq.z, x);
          x = fmaf(a[r].w, vq.w, x);
          acc[h][r][t] = x;
        }
      }
    }
    __syncthreads();  // every warp is done with this stage before it is refilled
    if (cj == chunks - 1) {
      const int64_t tile = blockIdx.x + (c / chunks) * gridDim.x;
      const int64_t row0 = tile * TR + warp * TRW;
#pragma unroll
      for (int r = 0; r < TRW; ++r)
#pragma unroll
        for (int t = 0; t < TLH; ++t) acc[0][r][t] = warp_sumf(acc[0][r][t]);
      // lane t writes column l0 + t of the warp's rows (select, no dynamic indexing)
#pragma unroll
      for (int r = 0; r < TRW; ++r) {
        float v = 0.f;
#pragma unroll
        for (int t = 0; t < TLH; ++t) v = (lane == t) ? acc[0][r][t] : v;
        const int64_t row = row0 + r;
        if (lane < kc && row < rows) {
          const double sg = __ldg(sigma + l0 + lane);
          U[row + (int64_t)(l0 + lane) * ldu] = sg > 0.0 ? (float)((double)v / sg) : 0.f;
        }
      }
    }
  }
  // After an early stop, chunks stop .. stop + T_NST - 1 may have been issued
  // and not waited for: let them land before the CTA exits.
  if (stop < total && threadIdx.x == 0) {
    for (int64_t j = stop; j < total && j < stop + T_NST; ++j)
      mbar_drain_l(su32(full + (j % T_NST)), (uint32_t)((j / T_NST) & 1));
  }
  __syncthreads();
}

// ---------------------------------------------------------------- tensor-core variant
// The same product on the tensor cores: mma.sync m16n8k8 with TF32 operands
// in the 3xTF32 split (x = hi + lo, hi = tf32(x), lo = tf32(x - hi); the
// products hi*hi + hi*lo + lo*hi carry the FP32 product to ~2^-20, Ootomo &
// Yokota 2022; split_tf32 below).  A persistent block of 8 warps streams the same 64-row x
// 128-column tiles of A and 16 x 128 tiles of V^T through a four-stage TMA
// ring, now as 32-column boxes with the 128-byte swizzle, so the fragment
// loads below are free of bank conflicts.  Warp w owns rows 16 (w & 3) ..
// +15 of the tile and columns 64 (w >> 2) .. +63 of every chunk (eight
// k-steps of 8); per k-step it loads one A fragment and two V^T fragments
// (16 columns of U), splits them and issues 6 MMAs into three accumulators
// per column tile (one per product: three independent chains).  The tensor
// core rounds its accumulation toward zero, so the accumulators are
// restarted every chunk (8 MMAs each) and added into FP32 sums with
// round-to-nearest.  At the end of a tile the two warps of a row group add
// their halves through shared memory and write U.
constexpr int MW = 8;                            // warps
constexpr int M_SUB = 32;                        // floats per swizzled box row (128 bytes)
constexpr int M_ASUB = TR * M_SUB * 4;           // 8 KB: one 64 x 32 box of A
constexpr int M_VSUB = LK * M_SUB * 4;           // 2 KB: one 16 x 32 box of V^T
constexpr int M_STAGE = 4 * M_ASUB + 4 * M_VSUB; // 40 KB: a 64 x 128 chunk of A, 16 x 128 of V^T
constexpr int M_RED = MW * 32 * 8 * 4;           // 8 KB: partial sums of the k-halves
constexpr int M_NST = 4;                         // stages (three chunks in flight)
constexpr int M_SMEM = M_NST * M_STAGE + M_RED + 1024 + 64;

// byte offset of element (r, c) of a box of 32-float rows written with the 128-byte swizzle
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((((c >> 2) ^ r) & 7) << 4) + ((c & 3) << 2));
}

// x = hi + lo: hi is x rounded to TF32's 10 stored mantissa bits (nearest, ties
// away from zero) by an integer add and mask, lo = x - hi exactly (|lo| <=
// 2^-11 |x|), passed as FP32: the tensor core reads its top 19 bits, so the
// split drops at most 2^-21 |x|.  (|x| within 2^-11 of FLT_MAX would round hi
// to infinity; such A overflows the Gram matrix long before.)
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(MW * 32, 1)
left_mma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV, int64_t rows,
                int64_t n, int64_t k, const double *__restrict__ sigma, float *__restrict__ U, int64_t ldu, int l0) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  float *red = reinterpret_cast<float *>(sm + M_NST * M_STAGE);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + M_NST * M_STAGE + M_RED);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;         // fragment row group and thread in group
  const int rg = warp & 3, kh = warp >> 2;       // row group (16 rows) and k-half of a chunk
  const int64_t tiles = ceil_div_dev(rows, TR);
  const int64_t chunks = ceil_div_dev(n, TJ);
  const int kc = (int)min((int64_t)LK, k - l0);
  if (threadIdx.x == 0) {
    for (int b = 0; b < M_NST; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t my_tiles = tiles > blockIdx.x ? ceil_div_dev(tiles - blockIdx.x, gridDim.x) : 0;
  const int64_t total = my_tiles * chunks;
  // the four columns of U this lane writes (D fragment: 2q, 2q + 1 of both column tiles)
  // and their 1 / sigma (0 where sigma is 0: a zero column)
  float inv[2][2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int t = nt * 8 + 2 * q + e;
      const double sg = t < kc ? __ldg(sigma + l0 + t) : 0.0;
      inv[nt][e] = sg > 0.0 ? (float)(1.0 / sg) : 0.f;
    }
  auto issue = [&](int64_t c) {  // chunk sequence number c -> stage c % M_NST
    const int64_t tile = blockIdx.x + (c / chunks) * gridDim.x;
    const int j0 = (int)((c % chunks) * TJ);
    const uint32_t st = su32(sm + (c % M_NST) * M_STAGE);
    const uint32_t bar = su32(full + (c % M_NST));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(M_STAGE) : "memory");
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              st + s * M_ASUB),
          "l"(reinterpret_cast<uint64_t>(&mapA)), "r"(j0 + s * M_SUB), "r"((int)(tile * TR)), "r"(bar)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              st + 4 * M_ASUB + s * M_VSUB),
          "l"(reinterpret_cast<uint64_t>(&mapV)), "r"(j0 + s * M_SUB), "r"(l0), "r"(bar)
          : "memory");
    }
  };
  int64_t issued = 0;  // chunks issued so far (thread 0)
  if (threadIdx.x == 0) {
    for (; issued < M_NST - 1 && issued < total; ++issued) issue(issued);
  }
  float sum[2][4];
  bool ok = true;
  int64_t stop = total;
  for (int64_t c = 0; c < total; ++c) {
    const int64_t cj = c % chunks;
    if (cj == 0) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) sum[nt][e] = 0.f;
    }
    // stage (c + M_NST - 1) % M_NST was released by the barrier at the end of iteration c - 1
    if (threadIdx.x == 0 && issued < total) issue(issued++);
    if (!mbar_wait_l(su32(full + (c % M_NST)), (uint32_t)((c / M_NST) & 1))) ok = false;
    if (__syncthreads_or(!ok)) {
      stop = c;
      break;
    }
    const unsigned char *As = sm + (c % M_NST) * M_STAGE;
    const unsigned char *Vs = As + 4 * M_ASUB;
    float acc[3][2][4];  // [product][column tile]: six independent chains
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[p][nt][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
      const int col = kh * 64 + ks * 8;          // first column of this k-step within the chunk
      const unsigned char *ab = As + (col >> 5) * M_ASUB;
      const unsigned char *vb = Vs + (col >> 5) * M_VSUB;
      const int cc = col & 31;
      const int r0 = rg * 16 + g;
      uint32_t ah[4], al[4];
      split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0, cc + q)), ah[0], al[0]);
      split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0 + 8, cc + q)), ah[1], al[1]);
      split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0, cc + q + 4)), ah[2], al[2]);
      split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0 + 8, cc + q + 4)), ah[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int t = nt * 8 + g;                // column of U (row of V^T)
        uint32_t bh0, bl0, bh1, bl1;
        split_tf32(*reinterpret_cast<const float *>(vb + sw128(t, cc + q)), bh0, bl0);
        split_tf32(*reinterpret_cast<const float *>(vb + sw128(t, cc + q + 4)), bh1, bl1);
        mma_tf32(acc[0][nt], al, bh0, bh1);      // small terms in their own chains
        mma_tf32(acc[1][nt], ah, bl0, bl1);
        mma_tf32(acc[2][nt], ah, bh0, bh1);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) sum[nt][e] += (acc[0][nt][e] + acc[1][nt][e]) + acc[2][nt][e];
    __syncthreads();  // every warp is done with this stage before it is refilled
    if (cj == chunks - 1) {
      // the k-half 1 warps hand their sums to the k-half 0 warps of the same row group
      float *rp = red + (rg * 32 + lane) * 8;
      if (kh == 1) {
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) rp[nt * 4 + e] = sum[nt][e];
      }
      __syncthreads();
      if (kh == 0) {
        const int64_t tile = blockIdx.x + (c / chunks) * gridDim.x;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = nt * 8 + 2 * q + (e & 1);                   // D fragment: column 2q (+1)
            const int64_t row = tile * TR + rg * 16 + g + (e >> 1) * 8;  // rows g and g + 8
            const float v = sum[nt][e] + rp[nt * 4 + e];
            if (t < kc && row < rows) U[row + (int64_t)(l0 + t) * ldu] = v * inv[nt][e & 1];
          }
      }
      __syncthreads();  // red is free again
    }
  }
  // after an early stop, chunks stop .. issued - 1 were issued and not all waited for
  if (stop < total && threadIdx.x == 0) {
    for (int64_t j = stop; j < issued; ++j) mbar_drain_l(su32(full + (j % M_NST)), (uint32_t)((j / M_NST) & 1));
  }
  __syncthreads();
}

// Warp-specialised form of the same tensor-core product: a ninth warp issues
// the TMA loads, each stage is handed back by an "empty" mbarrier that every
// consumer warp arrives on when it is done with it, and the two k-halves of a
// row group meet at the end of a tile through a pair of mbarriers instead of
// block barriers, so a warp that finishes a chunk early starts the next one.
// Every wait is bounded; a wait that gives up raises g_left_status, the other
// warps see it in their own waits, and each warp leaves its loop by itself.
constexpr int MWS_THREADS = (MW + 1) * 32;
// shared memory of the warp-specialised kernel with NST stages: + full[NST], empty[NST], red_full, red_empty
constexpr int mws_smem(int nst) { return nst * M_STAGE + M_RED + 1024 + 16 * nst + 64; }

template <int M_NST>
__global__ void __launch_bounds__(MWS_THREADS, 1)
left_mma_ws_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                   int64_t rows, int64_t n, int64_t k, const double *__restrict__ sigma, float *__restrict__ U,
                   int64_t ldu, int l0) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  float *red = reinterpret_cast<float *>(sm + M_NST * M_STAGE);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + M_NST * M_STAGE + M_RED);
  uint64_t *empty = full + M_NST;
  uint64_t *red_full = empty + M_NST, *red_empty = red_full + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles = ceil_div_dev(rows, TR);
  const int64_t chunks = ceil_div_dev(n, TJ);
  const int kc = (int)min((int64_t)LK, k - l0);
  if (threadIdx.x == 0) {
    for (int b = 0; b < M_NST; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + b)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(empty + b)), "r"(MW) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(su32(red_full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(su32(red_empty)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t my_tiles = tiles > blockIdx.x ? ceil_div_dev(tiles - blockIdx.x, gridDim.x) : 0;
  const int64_t total = my_tiles * chunks;
  if (warp == MW) {
    // ------------------------------------------------ producer
    if (lane == 0) {
      int64_t issued = 0;
      for (; issued < total; ++issued) {
        const int64_t c = issued;
        if (c >= M_NST && !mbar_wait_l(su32(empty + (c % M_NST)), (uint32_t)(((c / M_NST) - 1) & 1))) break;
        const int64_t tile = blockIdx.x + (c / chunks) * gridDim.x;
        const int j0 = (int)((c % chunks) * TJ);
        const uint32_t st = su32(sm + (c % M_NST) * M_STAGE);
        const uint32_t bar = su32(full + (c % M_NST));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(M_STAGE) : "memory");
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  st + s * M_ASUB),
              "l"(reinterpret_cast<uint64_t>(&mapA)), "r"(j0 + s * M_SUB), "r"((int)(tile * TR)), "r"(bar)
              : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  st + 4 * M_ASUB + s * M_VSUB),
              "l"(reinterpret_cast<uint64_t>(&mapV)), "r"(j0 + s * M_SUB), "r"(l0), "r"(bar)
              : "memory");
        }
      }
      // the last M_NST loads may not have been consumed (a consumer stopped early):
      // let them land before the block exits
      for (int64_t j = issued > M_NST ? issued - M_NST : 0; j < issued; ++j)
        mbar_drain_l(su32(full + (j % M_NST)), (uint32_t)((j / M_NST) & 1));
    }
  } else {
    // ------------------------------------------------ consumers
    const int g = lane >> 2, q = lane & 3;
    const int rg = warp & 3, kh = warp >> 2;
    float inv[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int t = nt * 8 + 2 * q + e;
        const double sg = t < kc ? __ldg(sigma + l0 + t) : 0.0;
        inv[nt][e] = sg > 0.0 ? (float)(1.0 / sg) : 0.f;
      }
    float sum[2][4];
    int64_t tix = 0;  // tiles finished by this block
    for (int64_t c = 0; c < total; ++c) {
      const int64_t cj = c % chunks;
      if (cj == 0) {
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) sum[nt][e] = 0.f;
      }
      if (!mbar_wait_l(su32(full + (c % M_NST)), (uint32_t)((c / M_NST) & 1))) break;
      const unsigned char *As = sm + (c % M_NST) * M_STAGE;
      const unsigned char *Vs = As + 4 * M_ASUB;
      float acc[3][2][4];
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[p][nt][e] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const int col = kh * 64 + ks * 8;
        const unsigned char *ab = As + (col >> 5) * M_ASUB;
        const unsigned char *vb = Vs + (col >> 5) * M_VSUB;
        const int cc = col & 31;
        const int r0 = rg * 16 + g;
        uint32_t ah[4], al[4];
        split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0, cc + q)), ah[0], al[0]);
        split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0 + 8, cc + q)), ah[1], al[1]);
        split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0, cc + q + 4)), ah[2], al[2]);
        split_tf32(*reinterpret_cast<const float *>(ab + sw128(r0 + 8, cc + q + 4)), ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int t = nt * 8 + g;
          uint32_t bh0, bl0, bh1, bl1;
          split_tf32(*reinterpret_cast<const float *>(vb + sw128(t, cc + q)), bh0, bl0);
          split_tf32(*reinterpret_cast<const float *>(vb + sw128(t, cc + q + 4)), bh1, bl1);
          mma_tf32(acc[0][nt], al, bh0, bh1);
          mma_tf32(acc[1][nt], ah, bl0, bl1);
          mma_tf32(acc[2][nt], ah, bh0, bh1);
        }
      }
      // the stage's operands are in registers or consumed: hand it back
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(empty + (c % M_NST))) : "memory");
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) sum[nt][e] += (acc[0][nt][e] + acc[1][nt][e]) + acc[2][nt][e];
      if (cj == chunks - 1) {
        float *rp = red + (rg * 32 + lane) * 8;
        if (kh == 1) {
          // wait until the k-half 0 warps have read the previous tile's sums
          if (tix > 0 && !mbar_wait_l(su32(red_empty), (uint32_t)((tix - 1) & 1))) break;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) rp[nt * 4 + e] = sum[nt][e];
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(su32(red_full)) : "memory");
        } else {
          if (!mbar_wait_l(su32(red_full), (uint32_t)(tix & 1))) break;
          float other[2][4];
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) other[nt][e] = rp[nt * 4 + e];
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(su32(red_empty)) : "memory");
          const int64_t tile = blockIdx.x + (c / chunks) * gridDim.x;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int t = nt * 8 + 2 * q + (e & 1);
              const int64_t row = tile * TR + rg * 16 + g + (e >> 1) * 8;
              if (t < kc && row < rows) U[row + (int64_t)(l0 + t) * ldu] = (sum[nt][e] + other[nt][e]) * inv[nt][e & 1];
            }
        }
        ++tix;
      }
    }
  }
  __syncthreads();
}

typedef CUresult (*EncodeTiledFnL)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

tsvd_status encode_2d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer, int64_t stride_elems,
                      uint32_t box_inner, uint32_t box_outer,
                      CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE) {
  static EncodeTiledFnL fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TSVD_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) return TSVD_ECUDA;
    fn = reinterpret_cast<EncodeTiledFnL>(p);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)stride_elems * 4};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TSVD_OK : TSVD_ECUDA;
}

// The other factor of a wide A (Eq. 3: the power method found the left
// vectors U, then V = A^T U Sigma^-1, Alg. 1) for a block of its
// columns: V[j][l] = sum_i A[i][j] U[i][l] / sigma_l for the block's K
// columns j, over the d rows i.  One thread per column (the loads of A along
// a row are coalesced across the warp); U is staged 32 rows at a time in
// shared memory, row-major, and read as broadcasts.
constexpr int kLtRows = 32;
constexpr int kLtMaxK = 32;

__global__ void __launch_bounds__(256) left_trans_kernel(const float *__restrict__ A, int64_t K, int64_t d, int64_t ld,
                                                         const float *__restrict__ U, int64_t ldu, int k,
                                                         const double *__restrict__ sigma, float *__restrict__ V,
                                                         int64_t ldv) {
  __shared__ __align__(16) float Us[kLtRows][kLtMaxK];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float acc[kLtMaxK];
#pragma unroll
  for (int l = 0; l < kLtMaxK; ++l) acc[l] = 0.f;
  for (int64_t i0 = 0; i0 < d; i0 += kLtRows) {
    __syncthreads();
    for (int e = threadIdx.x; e < kLtRows * kLtMaxK; e += blockDim.x) {
      const int ii = e / kLtMaxK, l = e % kLtMaxK;
      Us[ii][l] = (i0 + ii < d && l < k) ? __ldg(U + (i0 + ii) + (int64_t)l * ldu) : 0.f;
    }
    __syncthreads();
    if (j < K) {
      const int64_t nr = min((int64_t)kLtRows, d - i0);
      for (int64_t ii = 0; ii < nr; ++ii) {
        const float a = __ldg(A + (i0 + ii) * ld + j);
        const float4 *u4 = reinterpret_cast<const float4 *>(Us[ii]);
#pragma unroll
        for (int q = 0; q < kLtMaxK / 4; ++q) {
          const float4 u = u4[q];
          acc[4 * q] = fmaf(a, u.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(a, u.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(a, u.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(a, u.w, acc[4 * q + 3]);
        }
      }
    }
  }
  if (j < K) {
#pragma unroll
    for (int l = 0; l < kLtMaxK; ++l) {
      if (l < k) {
        const double s = __ldg(sigma + l);
        V[j + (int64_t)l * ldv] = s > 0.0 ? (float)((double)acc[l] / s) : 0.f;
      }
    }
  }
}

}  // namespace

tsvd_status launch_left_trans(const float *A, int64_t K, int64_t d, int64_t ld, const float *U, int64_t ldu,
                              int64_t k, const double *sigma, float *V, int64_t ldv, cudaStream_t stream) {
  if (K <= 0 || k <= 0) return TSVD_OK;
  for (int64_t l0 = 0; l0 < k; l0 += kLtMaxK) {
    const int kk = (int)std::min<int64_t>(kLtMaxK, k - l0);
    left_trans_kernel<<<(unsigned)ceil_div(K, 256), 256, 0, stream>>>(A, K, d, ld, U + l0 * ldu, ldu, kk, sigma + l0,
                                                                    V + l0 * ldv, ldv);
    TSVD_LAUNCHED();
  }
  return TSVD_OK;
}

// The device word the TMA-fed left kernels raise when a bounded wait gives up
// (shared by every launch on the device: a caller zeroes it before its pass
// and reads it after)
tsvd_status left_status_word(int **p) {
  TSVD_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(p), g_left_status));
  return TSVD_OK;
}

// Rows per warp of the CUDA-core TMA kernel: 8, or 4 with TSVD_LEFT_RW=4
static int left_rows_per_warp() {
  const char *e = getenv("TSVD_LEFT_RW");
  return e && atoi(e) == 4 ? 4 : 8;
}

// The TMA-fed form: 2 (default) the tensor cores with a producer warp and per-stage
// mbarriers, 1 the tensor cores with a block barrier per chunk, 0 the CUDA cores (TSVD_LEFT_MMA)
static int left_form() {
  const char *e = getenv("TSVD_LEFT_MMA");
  if (!e) return 2;
  const int v = atoi(e);
  return v == 0 || v == 1 ? v : 2;
}
static bool left_use_mma() { return left_form() != 0; }

// TMA stages of the warp-specialised kernel: 4, or 5 with TSVD_LEFT_STAGES=5
static int left_ws_stages() {
  const char *e = getenv("TSVD_LEFT_STAGES");
  return e && atoi(e) == 5 ? 5 : 4;
}

tsvd_status launch_left_dense(const float *A, int64_t rows, int64_t n, int64_t ld, const float *V,
                              int64_t ldv, int64_t k, const double *sigma, float *U, int64_t ldu,
                              cudaStream_t stream) {
  if (rows <= 0 || k <= 0) return TSVD_OK;
  const int64_t rows_per_block = (LT / 32) * LR;
  const int64_t blocks = ceil_div(rows, rows_per_block);
  if (blocks > 0x7fffffffLL) return TSVD_EINVAL;
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  // TMA needs 16-byte aligned bases and strides
  const bool tma = vec && di.cc_major == 10 && (ldv % 4 == 0) && ((reinterpret_cast<uintptr_t>(V) & 15) == 0) &&
                   rows >= TR && n >= 64;
  for (int64_t l0 = 0; l0 < k; l0 += LK) {
    if (tma && left_use_mma()) {
      CUtensorMap ma, mv;
      TSVD_TRY(encode_2d(&ma, A, n, rows, ld, M_SUB, TR, CU_TENSOR_MAP_SWIZZLE_128B));
      TSVD_TRY(encode_2d(&mv, V, n, k, ldv, M_SUB, LK, CU_TENSOR_MAP_SWIZZLE_128B));
      const int64_t tiles = ceil_div(rows, TR);
      const int grid = (int)std::min<int64_t>(tiles, di.sms);
      if (left_form() == 2 && left_ws_stages() == 5) {
        TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(left_mma_ws_kernel<5>), mws_smem(5)));
        left_mma_ws_kernel<5><<<grid, MWS_THREADS, mws_smem(5), stream>>>(ma, mv, rows, n, k, sigma, U, ldu, (int)l0);
      } else if (left_form() == 2) {
        TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(left_mma_ws_kernel<4>), mws_smem(4)));
        left_mma_ws_kernel<4><<<grid, MWS_THREADS, mws_smem(4), stream>>>(ma, mv, rows, n, k, sigma, U, ldu, (int)l0);
      } else {
        TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(left_mma_kernel), M_SMEM));
        left_mma_kernel<<<grid, MW * 32, M_SMEM, stream>>>(ma, mv, rows, n, k, sigma, U, ldu, (int)l0);
      }
      TSVD_LAUNCHED();
    } else if (tma) {
      CUtensorMap ma, mv;
      TSVD_TRY(encode_2d(&ma, A, n, rows, ld, TJ, TR));
      TSVD_TRY(encode_2d(&mv, V, n, k, ldv, TJ, LK));
      const int64_t tiles = ceil_div(rows, TR);
      const int grid = (int)std::min<int64_t>(tiles, di.sms);
      if (left_rows_per_warp() == 4) {
        TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(left_tma_kernel<4>), T_SMEM));
        left_tma_kernel<4><<<grid, TR / 4 * 32, T_SMEM, stream>>>(ma, mv, rows, n, k, sigma, U, ldu, (int)l0);
      } else {
        TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(left_tma_kernel<8>), T_SMEM));
        left_tma_kernel<8><<<grid, TR / 8 * 32, T_SMEM, stream>>>(ma, mv, rows, n, k, sigma, U, ldu, (int)l0);
      }
      TSVD_LAUNCHED();
    } else {
      left_dense_kernel<<<(unsigned)blocks, LT, 0, stream>>>(A, rows, n, ld, V, ldv, k, sigma, U, ldu, (int)l0,
                                                             vec ? 1 : 0);
      TSVD_LAUNCHED();
    }
  }
  return TSVD_OK;
}

}  // namespace tsvd
