// Dense Gram accumulation G += A_b^T A_b on CUDA cores in FP32 (the plain
// FP32 path of the method's Gram step: B = X^T X, Alg. 2; computed block by
// block over row batches of A, Sec. V-C / Alg. 3).
//
// Layout: A_b is rows x n row-major (stride ld), so the contraction index is
// the row and both operand tiles are contiguous along their output index.
// Each CTA owns one 128 x 128 tile (I, J) of the lower block triangle of G
// (J <= I, the symmetric-task reuse of Sec. V-C) and a contiguous slice of the
// rows (split-K); partial sums are FP32 in registers and are added into the
// FP64 result with one atomic per element, so G stays exact to FP64 across
// slices and blocks.  Element G[i][j] (i >= j) is stored at row j, column i
// of the n x n FP64 buffer (upper-triangle storage).
#include <algorithm>

#include "common.cuh"

namespace tsvd {
namespace {

constexpr int BM = 128;   // tile edge
constexpr int BK = 8;     // rows per pipeline step
constexpr int NT = 256;   // threads per CTA (16 x 16, 8 x 8 outputs each)

__device__ __forceinline__ void tile_of(int64_t t, int &bi, int &bj) {
  // t enumerates (bi, bj) with 0 <= bj <= bi in row order of the lower triangle
  int b = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(b + 1) * (b + 2) / 2 <= t) ++b;
  while ((int64_t)b * (b + 1) / 2 > t) --b;
  bi = b;
  bj = (int)(t - (int64_t)b * (b + 1) / 2);
}

__device__ __forceinline__ float4 load4(const float *row, int64_t c, int64_t n, bool vec) {
  if (vec && c + 3 < n) return __ldg(reinterpret_cast<const float4 *>(row + c));
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c < n) r.x = __ldg(row + c);
  if (c + 1 < n) r.y = __ldg(row + c + 1);
  if (c + 2 < n) r.z = __ldg(row + c + 2);
  if (c + 3 < n) r.w = __ldg(row + c + 3);
  return r;
}

// X[r][c] = A[c ld + r]: four consecutive r of column c, zero outside (c < n, r < k1)
__device__ __forceinline__ float4 load4t(const float *A, int64_t c, int64_t n, int64_t r, int64_t k1, int64_t ld,
                                         bool vec) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c >= n) return v;
  const float *p = A + c * ld + r;
  if (vec && r + 3 < k1) return __ldg(reinterpret_cast<const float4 *>(p));
  if (r < k1) v.x = __ldg(p);
  if (r + 1 < k1) v.y = __ldg(p + 1);
  if (r + 2 < k1) v.z = __ldg(p + 2);
  if (r + 3 < k1) v.w = __ldg(p + 3);
  return v;
}

// Triangular mode (nbj == 0): AI == AJ == A, tiles of the lower block
// triangle.  Rectangular mode (nbj > 0, a task of the orthogonal batching):
// G[gj][gi] += sum_r AJ[r][gj] AI[r][gi] for every gj < nJ, gi < nI, tiles
// enumerated row by row over ceil(nJ / 128) J blocks.  trans: the operand is
// X with X[r][c] = A[c ld + r] (a column block of a wide A: its Gram X^T X is
// A A^T, Eq. 3); the loads then run along r and the tile is transposed on its
// way into shared memory.
__global__ void __launch_bounds__(NT, 2)
syrk_simt_kernel(const float *__restrict__ AI, const float *__restrict__ AJ, int64_t rows, int64_t nI, int64_t nJ,
                 int64_t ld, double *__restrict__ G, int64_t ldg, int nbj, int64_t rows_per_split, int vec,
                 int trans) {
  int bi, bj;
  if (nbj > 0) {
    bi = (int)(blockIdx.x / nbj);
    bj = (int)(blockIdx.x % nbj);
  } else {
    tile_of(blockIdx.x, bi, bj);
  }
  const int64_t I0 = (int64_t)bi * BM, J0 = (int64_t)bj * BM;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t k1 = min(rows, k0 + rows_per_split);
  if (k0 >= k1) return;

  __shared__ __align__(16) float sI[2][BK][BM];
  __shared__ __align__(16) float sJ[2][BK][BM];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lr = tid >> 5;         // row of the step this thread loads
  const int lc = (tid & 31) * 4;   // first column it loads
  const bool diag = nbj == 0 && bi == bj;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra, rb;
  const int tc = tid >> 1, tk = (tid & 1) * 4;  // trans: column and first row this thread loads
  auto fetch = [&](int64_t kk) {
    if (trans) {
      ra = load4t(AI, I0 + tc, nI, kk + tk, k1, ld, vec);
      rb = diag ? ra : load4t(AJ, J0 + tc, nJ, kk + tk, k1, ld, vec);
      return;
    }
    const int64_t r = kk + lr;
    if (r < k1) {
      ra = load4(AI + r * ld, I0 + lc, nI, vec);
      rb = diag ? ra : load4(AJ + r * ld, J0 + lc, nJ, vec);
    } else {
      ra = rb = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto put = [&](int buf) {
    if (trans) {
      sI[buf][tk][tc] = ra.x;
      sI[buf][tk + 1][tc] = ra.y;
      sI[buf][tk + 2][tc] = ra.z;
      sI[buf][tk + 3][tc] = ra.w;
      sJ[buf][tk][tc] = rb.x;
      sJ[buf][tk + 1][tc] = rb.y;
      sJ[buf][tk + 2][tc] = rb.z;
      sJ[buf][tk + 3][tc] = rb.w;
    } else {
      *reinterpret_cast<float4 *>(&sI[buf][lr][lc]) = ra;
      *reinterpret_cast<float4 *>(&sJ[buf][lr][lc]) = rb;
    }
  };

  fetch(k0);
  put(0);
  __syncthreads();

  int cur = 0;
  for (int64_t kk = k0; kk < k1; kk += BK) {
    const bool more = kk + BK < k1;
    if (more) fetch(kk + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4 *>(&sI[cur][k][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&sI[cur][k][64 + tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&sJ[cur][k][ty * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&sJ[cur][k][64 + ty * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) put(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }

  // acc[i][j] = sum_r AI[r][gi] AJ[r][gj]; store G[gi][gj] at row gj, column gi
  // (triangular mode: only gi >= gj)
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t gj = J0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
    if (gj >= nJ) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t gi = I0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
      if (gi < nI && (nbj > 0 || gi >= gj)) atomicAdd(G + gj * ldg + gi, (double)acc[i][j]);
    }
  }
}

int64_t simt_splits(int64_t rows, int64_t tiles, int sms, int64_t *per_out) {
  // enough CTAs for ~4 waves at 2 CTAs/SM, but at least 1024 rows per slice
  const int64_t want = 8LL * sms;
  int64_t splits = std::max<int64_t>(1, ceil_div(want, tiles));
  int64_t per = round_up(ceil_div(rows, splits), BK);
  if (per < 1024) per = round_up(std::min<int64_t>(rows, 1024), BK);
  splits = ceil_div(rows, per);
  if (splits > 65535) {
    per = round_up(ceil_div(rows, 65535), BK);
    splits = ceil_div(rows, per);
  }
  *per_out = per;
  return splits;
}

}  // namespace

tsvd_status launch_gram_simt(const float *A, int64_t rows, int64_t n, int64_t ld, double *G,
                             cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int64_t nb = ceil_div(n, BM);
  const int64_t tiles = nb * (nb + 1) / 2;
  int64_t per = 0;
  const int64_t splits = simt_splits(rows, tiles, di.sms, &per);
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  if (ev0) TSVD_CUDA(cudaEventRecord(ev0, stream));
  syrk_simt_kernel<<<grid, NT, 0, stream>>>(A, A, rows, n, n, ld, G, n, 0, per, vec ? 1 : 0, 0);
  TSVD_LAUNCHED();
  if (ev1) TSVD_CUDA(cudaEventRecord(ev1, stream));
  return TSVD_OK;
}

tsvd_status launch_gram_simt_t(const float *A, int64_t rows, int64_t n, int64_t ld, double *G,
                               cudaStream_t stream) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int64_t nb = ceil_div(n, BM);
  const int64_t tiles = nb * (nb + 1) / 2;
  int64_t per = 0;
  const int64_t splits = simt_splits(rows, tiles, di.sms, &per);
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  syrk_simt_kernel<<<grid, NT, 0, stream>>>(A, A, rows, n, n, ld, G, n, 0, per, vec ? 1 : 0, 1);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_gram_simt_rect(const float *AJ, const float *AI, int64_t rows, int64_t nJ, int64_t nI, int64_t ld,
                                  double *G, int64_t ldg, cudaStream_t stream) {
  if (rows <= 0 || nJ <= 0 || nI <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int64_t nbi = ceil_div(nI, BM), nbj = ceil_div(nJ, BM);
  const int64_t tiles = nbi * nbj;
  if (tiles > 0x7fffffffLL) return TSVD_EUNSUPPORTED;
  int64_t per = 0;
  const int64_t splits = simt_splits(rows, tiles, di.sms, &per);
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(AI) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(AJ) & 15) == 0);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  syrk_simt_kernel<<<grid, NT, 0, stream>>>(AI, AJ, rows, nI, nJ, ld, G, ldg, (int)nbj, per, vec ? 1 : 0, 0);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
