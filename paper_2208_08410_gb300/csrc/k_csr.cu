// Sparse (CSR) kernels: the implicit Gram application and the left vectors.
//
// Fused pair (Sec. IV and Alg. 4 on one GPU; the Gram B = A^T A is never
// formed): for each row r of a row block
//     y_r = sum_p values[p] * v[col_idx[p]]          (gather, group reduction)
//     w[col_idx[p]] += values[p] * y_r               (FP32 atomics)
//     ss += y_r^2                                    (FP64)
// A group of G lanes (4..32, chosen from the mean row length) owns a row:
// column indices and values are read with coalesced loads along the row, the
// row sum is a shuffle reduction inside the group, and the scatter reuses the
// lines the gather just brought into L1.  y_r never leaves registers.
//
// Column-chunked pair (the same operator when v and w exceed what L2 holds):
// the columns are cut into C chunks and every row's sorted entries into C
// runs (split points found by binary search once per row).  Pass 1 forms
// y = A v one chunk at a time (the gathers from v_c hit L2), pass 2 adds
// A^T y into w one chunk at a time (the atomics on w_c stay in L2); the CSR
// is read twice instead of once, but the random accesses no longer go to DRAM.
//
// Left vectors (Alg. 1): U[r][l] = sum_p values[p] * V[col_p][l] /
// sigma_l, with V stored row-major (n x ldk) so one gather fetches all of a
// row's deflation coordinates at once.
#include <algorithm>

#include "common.cuh"

namespace tsvd {
namespace {

constexpr int CT = 256;

template <int G, bool SCATTER>
__global__ void __launch_bounds__(CT) csr_pair_kernel(int64_t rows, const int64_t *__restrict__ row_ptr,
                                                      const int32_t *__restrict__ col_idx,
                                                      const float *__restrict__ values,
                                                      const float *__restrict__ v, float *__restrict__ w,
                                                      double *__restrict__ ss) {
  constexpr int RPW = 32 / G;  // rows per warp step
  const int lane = threadIdx.x & 31;
  const int sub = lane % G, grp = lane / G;
  const int64_t base = __ldg(row_ptr);
  const int64_t warp_global = ((int64_t)blockIdx.x * CT + threadIdx.x) >> 5;
  const int64_t nwarps_total = ((int64_t)gridDim.x * CT) >> 5;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << (G & 31)) - 1u) << (grp * G));
  double ssq = 0.0;
  for (int64_t rb = warp_global * RPW; rb < rows; rb += nwarps_total * RPW) {
    const int64_t r = rb + grp;
    int64_t p0 = 0, p1 = 0;
    if (r < rows) {
      p0 = __ldg(row_ptr + r) - base;
      p1 = __ldg(row_ptr + r + 1) - base;
    }
    float y = 0.f;
    for (int64_t p = p0 + sub; p < p1; p += G) y = fmaf(__ldg(values + p), __ldg(v + __ldg(col_idx + p)), y);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) y += __shfl_xor_sync(gmask, y, o);
    if (sub == 0 && r < rows) ssq += (double)y * (double)y;
    if (SCATTER) {
      for (int64_t p = p0 + sub; p < p1; p += G) atomicAdd(w + __ldg(col_idx + p), __ldg(values + p) * y);
    }
  }
  __shared__ double red[33];
  ssq = block_sum(ssq, red);
  if (threadIdx.x == 0 && ssq != 0.0) atomicAdd(ss, ssq);
}

template <int G>
__global__ void __launch_bounds__(CT) csr_left_kernel(int64_t rows, const int64_t *__restrict__ row_ptr,
                                                      const int32_t *__restrict__ col_idx,
                                                      const float *__restrict__ values,
                                                      const float *__restrict__ Vr, int64_t ldk, int64_t k,
                                                      const double *__restrict__ sigma, float *__restrict__ U,
                                                      int64_t ldu) {
  constexpr int RPW = 32 / G;
  constexpr int KT = 16;
  const int lane = threadIdx.x & 31;
  const int sub = lane % G, grp = lane / G;
  const int64_t base = __ldg(row_ptr);
  const int64_t warp_global = ((int64_t)blockIdx.x * CT + threadIdx.x) >> 5;
  const int64_t nwarps_total = ((int64_t)gridDim.x * CT) >> 5;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << (G & 31)) - 1u) << (grp * G));
  for (int64_t rb = warp_global * RPW; rb < rows; rb += nwarps_total * RPW) {
    const int64_t r = rb + grp;
    int64_t p0 = 0, p1 = 0;
    if (r < rows) {
      p0 = __ldg(row_ptr + r) - base;
      p1 = __ldg(row_ptr + r + 1) - base;
    }
    for (int64_t l0 = 0; l0 < k; l0 += KT) {
      float acc[KT];
#pragma unroll
      for (int t = 0; t < KT; ++t) acc[t] = 0.f;
      for (int64_t p = p0 + sub; p < p1; p += G) {
        const float a = __ldg(values + p);
        const float *vr = Vr + (int64_t)__ldg(col_idx + p) * ldk + l0;
#pragma unroll
        for (int t = 0; t < KT; ++t)
          if (l0 + t < k) acc[t] = fmaf(a, __ldg(vr + t), acc[t]);
      }
#pragma unroll
      for (int t = 0; t < KT; ++t) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(gmask, acc[t], o);
      }
      if (r < rows) {
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          if (sub == t % G && l0 + t < k) {
            const double s = __ldg(sigma + l0 + t);
            U[r + (l0 + t) * ldu] = s > 0.0 ? (float)((double)acc[t] / s) : 0.f;
          }
        }
      }
    }
  }
}

// split[r * (nch-1) + b - 1] = offset (from the row's start) of its first entry
// with column >= b * cw, b = 1 .. nch-1; needs the row's columns sorted
__global__ void csr_split_kernel(int64_t rows, const int64_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col_idx, int nch, int64_t cw,
                                 int32_t *__restrict__ split) {
  const int64_t base = __ldg(row_ptr);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = __ldg(row_ptr + r) - base, p1 = __ldg(row_ptr + r + 1) - base;
    int64_t lo = p0;
    for (int b = 1; b < nch; ++b) {
      const int64_t target = (int64_t)b * cw;
      int64_t hi = p1;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(col_idx + mid) < target) lo = mid + 1; else hi = mid;
      }
      split[r * (nch - 1) + b - 1] = (int32_t)(lo - p0);
    }
  }
}

// entries of chunk c of row r: [p0 + s_c, p0 + s_{c+1}) with s_0 = 0, s_nch = row length.
// The two passes stream the row pointers, split points, column indices and
// values once per chunk; those loads are marked evict-first (ld.global.cs) so
// that they do not push the chunk of v (pass 1) or w (pass 2) out of L2.
__device__ __forceinline__ void chunk_range(const int32_t *split, int64_t r, int nch, int c, int64_t p0, int64_t p1,
                                            int64_t &q0, int64_t &q1) {
  q0 = c == 0 ? p0 : p0 + __ldcs(split + r * (nch - 1) + c - 1);
  q1 = c == nch - 1 ? p1 : p0 + __ldcs(split + r * (nch - 1) + c);
}

// pass 1: y[r] (c == 0: =, else +=) sum over the row's chunk-c entries of values * v[col]
template <int G>
__global__ void __launch_bounds__(CT) csr_chunk_y_kernel(int64_t rows, const int64_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col_idx,
                                                         const float *__restrict__ values,
                                                         const int32_t *__restrict__ split, int nch, int c,
                                                         const float *__restrict__ v, float *__restrict__ y) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane % G, grp = lane / G;
  const int64_t base = __ldg(row_ptr);
  const int64_t warp_global = ((int64_t)blockIdx.x * CT + threadIdx.x) >> 5;
  const int64_t nwarps_total = ((int64_t)gridDim.x * CT) >> 5;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << (G & 31)) - 1u) << (grp * G));
  for (int64_t rb = warp_global * RPW; rb < rows; rb += nwarps_total * RPW) {
    const int64_t r = rb + grp;
    int64_t q0 = 0, q1 = 0;
    if (r < rows) chunk_range(split, r, nch, c, __ldcs(row_ptr + r) - base, __ldcs(row_ptr + r + 1) - base, q0, q1);
    float t = 0.f;
    for (int64_t p = q0 + sub; p < q1; p += G) t = fmaf(__ldcs(values + p), __ldg(v + __ldcs(col_idx + p)), t);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) t += __shfl_xor_sync(gmask, t, o);
    if (sub == 0 && r < rows) y[r] = c == 0 ? t : y[r] + t;
  }
}

// pass 2: w[col] += values * y[r] over the row's chunk-c entries (scatter), and
// with c == 0 the block's sum of y[r]^2 into *ss
template <int G>
__global__ void __launch_bounds__(CT) csr_chunk_w_kernel(int64_t rows, const int64_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col_idx,
                                                         const float *__restrict__ values,
                                                         const int32_t *__restrict__ split, int nch, int c,
                                                         const float *__restrict__ y, float *__restrict__ w,
                                                         double *__restrict__ ss, int scatter) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane % G, grp = lane / G;
  const int64_t base = __ldg(row_ptr);
  const int64_t warp_global = ((int64_t)blockIdx.x * CT + threadIdx.x) >> 5;
  const int64_t nwarps_total = ((int64_t)gridDim.x * CT) >> 5;
  double ssq = 0.0;
  for (int64_t rb = warp_global * RPW; rb < rows; rb += nwarps_total * RPW) {
    const int64_t r = rb + grp;
    if (r >= rows) continue;
    const float yr = __ldg(y + r);
    if (c == 0 && sub == 0) ssq += (double)yr * (double)yr;
    if (scatter) {
      int64_t q0, q1;
      chunk_range(split, r, nch, c, __ldcs(row_ptr + r) - base, __ldcs(row_ptr + r + 1) - base, q0, q1);
      for (int64_t p = q0 + sub; p < q1; p += G) atomicAdd(w + __ldcs(col_idx + p), __ldcs(values + p) * yr);
    }
  }
  if (c == 0) {
    __shared__ double red[33];
    ssq = block_sum(ssq, red);
    if (threadIdx.x == 0 && ssq != 0.0) atomicAdd(ss, ssq);
  }
}

int pick_group(double avg_nnz) {
  if (avg_nnz <= 6.0) return 4;
  if (avg_nnz <= 20.0) return 8;
  if (avg_nnz <= 56.0) return 16;
  return 32;
}

}  // namespace

tsvd_status launch_csr_pair(int64_t rows, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                            const float *values, const float *v, float *w, double *ss, int scatter,
                            double avg_nnz, cudaStream_t stream) {
  (void)n;
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int G = pick_group(avg_nnz);
  const int64_t rows_per_block = (CT / 32) * (32 / G);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, rows_per_block), (int64_t)di.sms * 16));
  const unsigned gb = (unsigned)blocks;
#define TSVD_PAIR(GG)                                                                            \
  if (scatter)                                                                                   \
    csr_pair_kernel<GG, true><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, v, w, ss);  \
  else                                                                                           \
    csr_pair_kernel<GG, false><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, v, w, ss);
  switch (G) {
    case 4: TSVD_PAIR(4); break;
    case 8: TSVD_PAIR(8); break;
    case 16: TSVD_PAIR(16); break;
    default: TSVD_PAIR(32); break;
  }
#undef TSVD_PAIR
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_csr_split(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx, int nch, int64_t cw,
                             int32_t *split, cudaStream_t stream) {
  if (rows <= 0 || nch < 2) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, 256), (int64_t)di.sms * 16));
  csr_split_kernel<<<(unsigned)blocks, 256, 0, stream>>>(rows, row_ptr, col_idx, nch, cw, split);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_csr_chunk_y(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx, const float *values,
                               const int32_t *split, int nch, int c, const float *v, float *y, double avg_nnz,
                               cudaStream_t stream) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int G = pick_group(avg_nnz / nch);
  const int64_t rows_per_block = (CT / 32) * (32 / G);
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, rows_per_block), (int64_t)di.sms * 16));
  switch (G) {
    case 4: csr_chunk_y_kernel<4><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, v, y); break;
    case 8: csr_chunk_y_kernel<8><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, v, y); break;
    case 16: csr_chunk_y_kernel<16><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, v, y); break;
    default: csr_chunk_y_kernel<32><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, v, y); break;
  }
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_csr_chunk_w(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx, const float *values,
                               const int32_t *split, int nch, int c, const float *y, float *w, double *ss, int scatter,
                               double avg_nnz, cudaStream_t stream) {
  if (rows <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int G = pick_group(avg_nnz / nch);
  const int64_t rows_per_block = (CT / 32) * (32 / G);
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, rows_per_block), (int64_t)di.sms * 16));
  switch (G) {
    case 4: csr_chunk_w_kernel<4><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, y, w, ss, scatter); break;
    case 8: csr_chunk_w_kernel<8><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, y, w, ss, scatter); break;
    case 16: csr_chunk_w_kernel<16><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, y, w, ss, scatter); break;
    default: csr_chunk_w_kernel<32><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, split, nch, c, y, w, ss, scatter); break;
  }
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_csr_left(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx,
                            const float *values, const float *Vr, int64_t ldk, int64_t k,
                            const double *sigma, float *U, int64_t ldu, double avg_nnz,
                            cudaStream_t stream) {
  if (rows <= 0 || k <= 0) return TSVD_OK;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int G = pick_group(avg_nnz);
  const int64_t rows_per_block = (CT / 32) * (32 / G);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, rows_per_block), (int64_t)di.sms * 16));
  const unsigned gb = (unsigned)blocks;
  switch (G) {
    case 4: csr_left_kernel<4><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, Vr, ldk, k, sigma, U, ldu); break;
    case 8: csr_left_kernel<8><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, Vr, ldk, k, sigma, U, ldu); break;
    case 16: csr_left_kernel<16><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, Vr, ldk, k, sigma, U, ldu); break;
    default: csr_left_kernel<32><<<gb, CT, 0, stream>>>(rows, row_ptr, col_idx, values, Vr, ldk, k, sigma, U, ldu); break;
  }
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
