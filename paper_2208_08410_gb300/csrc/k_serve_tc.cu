// Grouped tensor-core SYRK of the t-SVD server: the Gram step of the method
// (B = X^T X, Alg. 2; G = A A^T for wide requests, Eq. 3) for every request
// of a wave whose Gram dimension d is large enough to fill 128 x 256 tiles,
// in three grouped launches:
//  1. prep: each request's A is rounded and split into the K-major TF32
//     operand pair hi = tf32(a), lo = tf32(a - hi) (3xTF32, Ootomo & Yokota
//     2022), d rows of Kp contraction indices, zero-padded.  A tall request
//     (G = A^T A) is transposed through shared memory; a wide one (G = A A^T)
//     already has its contraction index contiguous.
//  2. SYRK: a persistent warp-specialised tcgen05 kernel over the units of
//     all requests.  A unit is one 128 x 256 tile touching the lower triangle
//     over its request's WHOLE contraction range, so no two units write the
//     same entries and no atomics are used: a request's Gram matrix is
//     bitwise the same in any wave.  TMA streams the hi / lo slabs (tensor
//     maps of every request in device memory), one thread issues three
//     tcgen05.mma kind::tf32 per K step (lo.hi, hi.lo, hi.hi) into a TMEM
//     accumulator restarted every 64 rows, and the epilogue warps add the
//     segment sums in FP32 registers with round-to-nearest and carry them
//     into the FP64 matrix every 8 segments (512 rows), in place: the first
//     carry of a unit stores, the later ones add.
//  3. finish: the stored entries (gj <= gi, kept at G64[gj d + gi]) are
//     mirrored and the FP32 copy the power kernel iterates on is written.
// Every wait is bounded; on a timeout the SYRK raises the wave's status word
// (read by the power kernel, which then reports TSVD_ETIMEDOUT for the
// request), lets its own loads and MMAs complete, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "serve.cuh"
#include "tc_common.cuh"

namespace tsvd {
namespace {

constexpr int kCarry = 8;                      // TMEM segments summed in FP32 before the FP64 carry
constexpr int kSegStages = 2;                  // stages per TMEM segment (64 contraction indices)
using SC = Cfg<TSVD_GRAM_TF32X3>;

// first index i with start[i + 1] > x (start: n + 1 nondecreasing prefix sums)
__device__ __forceinline__ int find_owner(const int64_t *start, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- grouped prep
// Strip s of request t: contraction indices [32 (s % ks), +32) by operand rows
// [128 (s / ks), +128), ks = Kp / 32.  Block (32, 8).
__global__ void __launch_bounds__(256) srv_tc_prep_kernel(const SrvReq *__restrict__ reqs,
                                                          const SrvTcReq *__restrict__ tcs, int n_tc,
                                                          const int64_t *__restrict__ start, int64_t n_strips) {
  __shared__ float s[4][32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t g = blockIdx.x; g < n_strips; g += gridDim.x) {
    const int t = find_owner(start, n_tc, g);
    const SrvTcReq &c = tcs[t];
    const SrvReq &q = reqs[c.req];
    const int64_t sl = g - start[t], ks = c.Kp / 32;
    const int64_t x0 = (sl % ks) * 32, c0 = (sl / ks) * 128;
    const float *__restrict__ A = q.A;
    if (!q.trans) {
      // tall: At[cc][x] = A[x][cc] (x < K = m rows, cc < d = n columns): transpose
      __syncthreads();  // the previous strip's reads of s are done
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t x = x0 + ty + 8 * i, cc = c0 + 32 * u + tx;
          s[u][ty + 8 * i][tx] = (x < c.K && cc < c.d) ? __ldg(A + x * q.n + cc) : 0.f;
        }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t cc = c0 + 32 * u + ty + 8 * i, x = x0 + tx;
          if (cc < c.d) {
            const float a = s[u][tx][ty + 8 * i];
            const float h = tf32_rne(a);
            c.hi[cc * c.Kp + x] = h;
            c.lo[cc * c.Kp + x] = tf32_rne(a - h);
          }
        }
    } else {
      // wide: At[cc][x] = A[cc][x] (cc < d = m rows, x < K = n columns): already K-major
      for (int r = ty; r < 128; r += 8) {
        const int64_t cc = c0 + r, x = x0 + tx;
        if (cc < c.d) {
          const float a = x < c.K ? __ldg(A + cc * q.n + x) : 0.f;
          const float h = tf32_rne(a);
          c.hi[cc * c.Kp + x] = h;
          c.lo[cc * c.Kp + x] = tf32_rne(a - h);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- grouped finish
// Tile f of request t: the 32 x 32 block (bi, bj), bi <= bj, of the upper
// triangle (row-major blocks of T = ceil(d / 32), listed row by row).  The
// entries (r, c), r <= c, hold G(r, c); mirrored to (c, r); G32 = fl32(G64).
__device__ __forceinline__ void upper_block(int64_t f, int64_t T, int64_t &bi, int64_t &bj) {
  // row bi starts at bi T - bi (bi - 1) / 2
  int64_t lo = 0, hi = T - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (mid * T - mid * (mid - 1) / 2 <= f) lo = mid; else hi = mid - 1;
  }
  bi = lo;
  bj = bi + (f - (bi * T - bi * (bi - 1) / 2));
}

__global__ void __launch_bounds__(256) srv_tc_finish_kernel(const SrvTcReq *__restrict__ tcs, int n_tc,
                                                            const int64_t *__restrict__ start, int64_t n_tiles) {
  __shared__ double s[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t g = blockIdx.x; g < n_tiles; g += gridDim.x) {
    const int t = find_owner(start, n_tc, g);
    const SrvTcReq &c = tcs[t];
    const int64_t d = c.d, T = (d + 31) / 32;
    int64_t bi, bj;
    upper_block(g - start[t], T, bi, bj);
    __syncthreads();
    // read the stored block rows [32 bi, +32) x columns [32 bj, +32): entries with row <= column
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = 32 * bi + ty + 8 * i, cc = 32 * bj + tx;
      double v = 0.0;
      if (r < d && cc < d && r <= cc) {
        v = c.G64[r * d + cc];
        c.G32[r * d + cc] = (float)v;
      }
      s[ty + 8 * i][tx] = v;
    }
    __syncthreads();
    // write the mirror: (cc, r) for r < cc
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t cc = 32 * bj + ty + 8 * i, r = 32 * bi + tx;
      if (r < d && cc < d && r < cc) {
        const double v = s[tx][ty + 8 * i];
        c.G64[cc * d + r] = v;
        c.G32[cc * d + r] = (float)v;
      }
    }
  }
}

// ---------------------------------------------------------------- grouped SYRK
// The same pipeline as the dense plan's SYRK (TMA warp, MMA warp, 16 epilogue
// warps, two 256-column TMEM accumulators), over units of many requests, each
// unit a full-K tile whose sums the epilogue carries into G64 in place.
__global__ void __launch_bounds__(TC_THREADS, 1)
srv_syrk_tc_kernel(const CUtensorMap *__restrict__ maps, const SrvTcReq *__restrict__ tcs,
                   const SrvTcUnit *__restrict__ units, int n_units, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SC::kStages * SC::kStageBytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * SC::kStages + 5);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + SC::kStages);
  const uint32_t tfull0 = smem_u32(bars + 2 * SC::kStages), tempty0 = smem_u32(bars + 2 * SC::kStages + 2);
  const uint32_t final_bar = smem_u32(bars + 2 * SC::kStages + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TK = SC::kTK;  // 32 contraction indices per stage
  constexpr int64_t kSegRows = (int64_t)kSegStages * TK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SC::kStages; ++s) {
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
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const SrvTcUnit un = units[u];
        const int64_t Kp = tcs[un.tc].Kp;
        const CUtensorMap *mh = maps + 2 * un.tc, *ml = maps + 2 * un.tc + 1;
        // the maps were written into a reused device buffer by a copy before this
        // launch: acquire them for the tensor-map proxy before the first load
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mh))
                     : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(ml))
                     : "memory");
        for (int64_t kk = 0; kk < Kp; kk += TK, ++it) {
          const uint32_t s = it % SC::kStages, ph = (it / SC::kStages) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err, kWaitLimitNs)) { ok = false; break; }
          unsigned char *st = smem + s * SC::kStageBytes;
          mbar_expect_tx(full0 + 8 * s, SC::kStageBytes);
          const int x = (int)kk;
          tma_load_2d(smem_u32(st), mh, x, un.bi * TM, full0 + 8 * s);
          tma_load_2d(smem_u32(st + A_SLAB), mh, x, un.bj * TN, full0 + 8 * s);
          tma_load_2d(smem_u32(st + A_SLAB + B_SLAB / 2), mh, x, un.bj * TN + TN / 2, full0 + 8 * s);
          unsigned char *sl = st + A_SLAB + B_SLAB;
          tma_load_2d(smem_u32(sl), ml, x, un.bi * TM, full0 + 8 * s);
          tma_load_2d(smem_u32(sl + A_SLAB), ml, x, un.bj * TN, full0 + 8 * s);
          tma_load_2d(smem_u32(sl + A_SLAB + B_SLAB / 2), ml, x, un.bj * TN + TN / 2, full0 + 8 * s);
        }
      }
      // the last kStages loads may still be in flight when the MMA warp stopped early
      const uint32_t from = it > (uint32_t)SC::kStages ? it - SC::kStages : 0;
      for (uint32_t j = from; j < it; ++j) mbar_drain(full0 + 8 * (j % SC::kStages), (j / SC::kStages) & 1u);
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t it = 0, sc = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const int64_t Kp = tcs[units[u].tc].Kp;
        for (int64_t g0 = 0; g0 < Kp && ok; g0 += kSegRows, ++sc) {
          const int64_t g1 = min(Kp, g0 + kSegRows);
          const uint32_t acc = sc & 1u, aph = (sc >> 1) & 1u;
          if (!mbar_wait(tempty0 + 8 * acc, aph ^ 1u, err, kWaitLimitNs)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem + acc * TN;
          uint32_t first = 1;
          for (int64_t kk = g0; kk < g1; kk += TK, ++it) {
            const uint32_t s = it % SC::kStages, ph = (it / SC::kStages) & 1u;
            if (!mbar_wait(full0 + 8 * s, ph, err, kWaitLimitNs)) { ok = false; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * SC::kStageBytes);
            const uint64_t dah = umma_desc_sw128(st), dbh = umma_desc_sw128(st + A_SLAB);
            const uint32_t sl = st + A_SLAB + B_SLAB;
            const uint64_t dal = umma_desc_sw128(sl), dbl = umma_desc_sw128(sl + A_SLAB);
#pragma unroll
            for (int kq = 0; kq < ROW_BYTES / MMA_K_BYTES; ++kq) {
              const uint64_t off = (uint64_t)(kq * MMA_K_BYTES) >> 4;
              umma<TSVD_GRAM_TF32X3>(dtm, dal + off, dbh + off, first ? 0u : 1u);  // small terms first
              first = 0;
              umma<TSVD_GRAM_TF32X3>(dtm, dah + off, dbl + off, 1u);
              umma<TSVD_GRAM_TF32X3>(dtm, dah + off, dbh + off, 1u);
            }
            umma_commit(empty0 + 8 * s);
          }
          if (!ok) break;
          umma_commit(tfull0 + 8 * acc);
        }
      }
      umma_commit(final_bar);
      mbar_drain(final_bar, 0);
    }
  } else {
    // ------------------------------------------------ epilogue: TMEM -> FP32 registers -> FP64 G64 in place
    const int q = warp & 3;                 // TMEM lane quarter
    const int h = (warp - 2) >> 2;          // which 64 of the 256 columns
    const int row = q * 32 + lane;
    float accr[TC_EPI_COLS];
#pragma unroll
    for (int j = 0; j < TC_EPI_COLS; ++j) accr[j] = 0.f;
    uint32_t sc = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const SrvTcUnit un = units[u];
      const SrvTcReq &c = tcs[un.tc];
      const int64_t d = c.d, Kp = c.Kp;
      const int64_t gi = (int64_t)un.bi * TM + row;
      const int64_t jbase = (int64_t)un.bj * TN + h * TC_EPI_COLS;
      // columns gj <= gi (lower triangle) inside the matrix
      int jlim = gi >= d ? 0 : (int)min((int64_t)TC_EPI_COLS, gi - jbase + 1);
      jlim = (int)max((int64_t)0, min((int64_t)jlim, d - jbase));
      bool first_carry = true;
      int seg_in_unit = 0;
      for (int64_t g0 = 0; g0 < Kp; g0 += kSegRows, ++sc) {
        const uint32_t acc = sc & 1u, aph = (sc >> 1) & 1u;
        if (!mbar_wait(tfull0 + 8 * acc, aph, err, kWaitLimitNs)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * TN + h * TC_EPI_COLS;
#pragma unroll
        for (int cq = 0; cq < TC_EPI_COLS / 16; ++cq) tmem_add16(tbase + cq * 16, accr + cq * 16);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
        ++seg_in_unit;
        if (seg_in_unit % kCarry == 0 || g0 + kSegRows >= Kp) {
          // carry into FP64: entry (gi, gj) stored at G64[gj d + gi] (lanes: consecutive gi)
          double *gp = c.G64 + jbase * d + gi;
#pragma unroll
          for (int j = 0; j < TC_EPI_COLS; ++j) {
            if (j < jlim) {
              if (first_carry)
                *gp = (double)accr[j];
              else
                *gp += (double)accr[j];
            }
            gp += d;
            accr[j] = 0.f;
          }
          first_carry = false;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

int64_t srv_tc_prep_strips(int64_t d, int64_t Kp) { return (Kp / 32) * ((d + 127) / 128); }

int64_t srv_tc_finish_tiles(int64_t d) {
  const int64_t T = (d + 31) / 32;
  return T * (T + 1) / 2;
}

int64_t srv_tc_tiles(int64_t d) {
  // 128-row blocks bi, 256-row blocks bj <= bi / 2 (J0 <= I0 + 127)
  const int64_t nb = (d + TM - 1) / TM, q = nb >> 1;
  return (nb & 1) ? (q + 1) * (q + 1) : q * (q + 1);
}

tsvd_status launch_srv_syrk_tc(const SrvReq *reqs, const SrvTcReq *tcs, int n_tc, const int64_t *prep_start,
                               int64_t n_prep, const int64_t *fin_start, int64_t n_fin, const CUtensorMap *maps,
                               const SrvTcUnit *units, int n_units, int32_t *err, cudaStream_t stream) {
  if (n_tc <= 0 || n_units <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  if (di.cc_major != 10) return TSVD_EUNSUPPORTED;
  TSVD_CUDA(cudaMemsetAsync(err, 0, 4, stream));
  const dim3 blk(32, 8);
  const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n_prep, (int64_t)di.sms * 16));
  srv_tc_prep_kernel<<<gp, blk, 0, stream>>>(reqs, tcs, n_tc, prep_start, n_prep);
  TSVD_LAUNCHED();
  TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(srv_syrk_tc_kernel), SC::kSmem));
  const int grid = std::min(n_units, di.sms);
  srv_syrk_tc_kernel<<<grid, TC_THREADS, SC::kSmem, stream>>>(maps, tcs,
                                                              units, n_units, err);
  TSVD_LAUNCHED();
  const unsigned gf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n_fin, (int64_t)di.sms * 16));
  srv_tc_finish_kernel<<<gf, blk, 0, stream>>>(tcs, n_tc, fin_start, n_fin);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
