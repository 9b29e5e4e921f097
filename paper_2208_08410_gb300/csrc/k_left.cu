// Left singular vectors of a dense row block (Alg. 1 l.11-13):
//     U_b = A_b V diag(sigma)^-1,   u_l = A v_l / ||A v_l||
// computed in one extra pass over A after all right vectors are known.
//
// A is rows x n row-major; V is n x k column-major.  A block of 256 threads
// owns 64 rows; each warp keeps 8 rows x 16 columns of partial sums in
// registers while the lanes stride along the row (coalesced loads of A).  V
// is staged through shared memory 256 rows at a time (transposed to
// [j][l]), so each staged value feeds 8 rows.  Columns are processed 16 at a
// time (A is re-read for k > 16).
#include <algorithm>

#include "common.cuh"

namespace tsvd {
namespace {

constexpr int LT = 256;   // threads
constexpr int LR = 8;     // rows per warp
constexpr int LK = 16;    // columns per pass
constexpr int LJ = 256;   // V rows staged per step

__global__ void __launch_bounds__(LT, 1)
left_dense_kernel(const float *__restrict__ A, int64_t rows, int64_t n, int64_t ld,
                  const float *__restrict__ V, int64_t ldv, int64_t k, const double *__restrict__ sigma,
                  float *__restrict__ U, int64_t ldu, int l0) {
  __shared__ __align__(16) float Vs[LJ][LK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * (LT / 32) * LR + (int64_t)warp * LR;
  float acc[LR][LK];
#pragma unroll
  for (int r = 0; r < LR; ++r)
#pragma unroll
    for (int t = 0; t < LK; ++t) acc[r][t] = 0.f;
  const int kc = (int)std::min<int64_t>(LK, k - l0);

  for (int64_t j0 = 0; j0 < n; j0 += LJ) {
    __syncthreads();
    for (int e = threadIdx.x; e < LJ * LK; e += LT) {
      const int jj = e % LJ, t = e / LJ;  // consecutive threads read consecutive j of one column
      const int64_t j = j0 + jj;
      Vs[jj][t] = (t < kc && j < n) ? __ldg(V + (int64_t)(l0 + t) * ldv + j) : 0.f;
    }
    __syncthreads();
    const int jmax = (int)std::min<int64_t>(LJ, n - j0);
    for (int jj = lane; jj < jmax; jj += 32) {
      const float4 *vq = reinterpret_cast<const float4 *>(&Vs[jj][0]);
      const float4 q0 = vq[0], q1 = vq[1], q2 = vq[2], q3 = vq[3];
      const float vv[LK] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                            q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
#pragma unroll
      for (int r = 0; r < LR; ++r) {
        const int64_t row = row0 + r;
        const float a = row < rows ? __ldg(A + row * ld + j0 + jj) : 0.f;
#pragma unroll
        for (int t = 0; t < LK; ++t) acc[r][t] = fmaf(a, vv[t], acc[r][t]);
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
      const double s = __ldg(sigma + l0 + t);
#pragma unroll
      for (int r = 0; r < LR; ++r) {
        const int64_t row = row0 + r;
        if (row < rows) U[row + (int64_t)(l0 + t) * ldu] = s > 0.0 ? (float)((double)acc[r][t] / s) : 0.f;
      }
    }
  }
}

}  // namespace

tsvd_status launch_left_dense(const float *A, int64_t rows, int64_t n, int64_t ld, const float *V,
                              int64_t ldv, int64_t k, const double *sigma, float *U, int64_t ldu,
                              cudaStream_t stream) {
  if (rows <= 0 || k <= 0) return TSVD_OK;
  const int64_t rows_per_block = (LT / 32) * LR;
  const int64_t blocks = ceil_div(rows, rows_per_block);
  if (blocks > 0x7fffffffLL) return TSVD_EINVAL;
  for (int64_t l0 = 0; l0 < k; l0 += LK) {
    left_dense_kernel<<<(unsigned)blocks, LT, 0, stream>>>(A, rows, n, ld, V, ldv, k, sigma, U, ldu, (int)l0);
    TSVD_LAUNCHED();
  }
  return TSVD_OK;
}

}  // namespace tsvd
