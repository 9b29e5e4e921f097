// One triplet of the sparse power method in one cooperative launch: the
// iteration of Alg. 2 with the implicit operator of Alg. 4 (w = A^T (A v), never forming
// A^T A) and Hotelling's correction w -= V (sigma^2 . V^T v) (Eq. 2), for a
// CSR matrix held on the device.  It serves small operators, where a dozen
// kernels and a host round trip per application would cost more than the
// application itself.  Three bounded grid barriers per application:
//   pair   y_r = sum_p values[p] v[col_p] for every row (a group of G lanes
//          per row, shuffle reduction), then w[col_p] += values[p] y_r
//          (FP32 atomics);                                        -> barrier
//   deflate  every block reduces the partial projections c_j = V_j . v of
//          its own copy (same order in every block), then w_i -= sum_j
//          sigma_j^2 c_j V_ij (FP32) and the partial ||w||^2, v.w, v.v
//          (FP64);                                                -> barrier
//   next   every block reduces the three norms and takes the same decision
//          (the test of the explicit loop: rank, |v.w| / (||v|| ||w||) >=
//          1 - eps, forced count, max_iter); then v' = w / ||w||, w = 0,
//          and the partial projections of v' for the next step.  -> barrier
// The iterate alternates between the two buffers v (application 1 reads it)
// and vn, as in the host loop; info receives the applications, the status,
// the done flag and the application that stopped the triplet, so the caller
// finds the result the same way.
#include <algorithm>

#include "common.cuh"

namespace tsvd {
namespace {

constexpr int PT = 256;
constexpr int kMaxL = 32;  // deflation columns handled (the CSR plans allow k + 4 <= kVecPartStride)

struct CsrPowerArgs {
  int64_t m, n;
  const int64_t *rp;
  const int32_t *ci;
  const float *va;
  const float *Vr;  // n x ldk row-major, columns 0..l-1 are the earlier vectors
  int64_t ldk;
  const double *sig2;
  int l;
  float *buf0, *buf1;  // the iterate's two buffers; buf0 holds v0 on entry
  float *w;            // n floats, zero on entry (left zero)
  double *part;        // gridDim.x x ps
  int ps;
  unsigned *bar;
  int *err;
  double eps;
  int max_iter;
  int iters_override;
  double rank_scale;
  int *info;  // [0] applications, [1] status, [2] done, [3] stopping application
};

template <int G>
__global__ void __launch_bounds__(PT) csr_power_kernel(CsrPowerArgs a) {
  __shared__ double red[33];
  __shared__ float cs[kMaxL];
  __shared__ double scal[4];
  __shared__ double cpart[PT / 32][kMaxL];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gt = (int64_t)blockIdx.x * PT + threadIdx.x, gs = (int64_t)gridDim.x * PT;
  const int l = a.l;
  const int NRM = kMaxL;  // norm partials at [NRM, NRM + 3)
  double *mypart = a.part + (int64_t)blockIdx.x * a.ps;

  // partial projections c_j = V_j . x of this block's elements (FP32 per thread, FP64 across)
  auto proj_partials = [&](const float *x) {
    float acc[kMaxL];
#pragma unroll
    for (int j = 0; j < kMaxL; ++j) acc[j] = 0.f;
    for (int64_t i = gt; i < a.n; i += gs) {
      const float xi = x[i];
      const float *row = a.Vr + i * a.ldk;
#pragma unroll
      for (int j = 0; j < kMaxL; ++j)
        if (j < l) acc[j] = fmaf(__ldg(row + j), xi, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kMaxL; ++j) {
      if (j < l) {
        const double t = warp_sum((double)acc[j]);
        if (lane == 0) cpart[warp][j] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x < l) {
      double t = 0.0;
      for (int w = 0; w < PT / 32; ++w) t += cpart[w][threadIdx.x];
      mypart[threadIdx.x] = t;
    }
    __syncthreads();
  };

  if (l > 0) proj_partials(a.buf0);
  if (!grid_barrier(a.bar, a.err)) return;

  const int sub = lane % G, grp = lane / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << (G & 31)) - 1u) << (grp * G));
  const int64_t wg = gt >> 5, nwg = gs >> 5;  // global warp index and count
  for (int it = 0;; ++it) {
    const float *cur = (it & 1) ? a.buf1 : a.buf0;
    float *nxt = (it & 1) ? a.buf0 : a.buf1;
    // ---- pair: w += A^T (A cur)
    for (int64_t rb = wg * (32 / G); rb < a.m; rb += nwg * (32 / G)) {
      const int64_t r = rb + grp;
      int64_t p0 = 0, p1 = 0;
      if (r < a.m) {
        p0 = __ldg(a.rp + r);
        p1 = __ldg(a.rp + r + 1);
      }
      float y = 0.f;
      for (int64_t p = p0 + sub; p < p1; p += G) y = fmaf(__ldg(a.va + p), __ldcg(cur + __ldg(a.ci + p)), y);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) y += __shfl_xor_sync(gmask, y, o);
      for (int64_t p = p0 + sub; p < p1; p += G) atomicAdd(a.w + __ldg(a.ci + p), __ldg(a.va + p) * y);
    }
    if (!grid_barrier(a.bar, a.err)) return;
    // ---- deflate: w -= V (sigma^2 . c), partial norms.  c_j summed over the blocks' partials
    // by warp j % 8 (the same order in every block)
    for (int j = warp; j < l; j += PT / 32) {
      double t = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(a.part + (int64_t)b * a.ps + j);
      t = warp_sum(t);
      if (lane == 0) cs[j] = (float)(__ldg(a.sig2 + j) * t);
    }
    __syncthreads();
    double ww = 0.0, vw = 0.0, vv = 0.0;
    for (int64_t i = gt; i < a.n; i += gs) {
      const float vf = __ldcg(cur + i);
      float wf = __ldcg(a.w + i);
      const float *row = a.Vr + i * a.ldk;
      for (int j = 0; j < l; ++j) wf = fmaf(-__ldg(row + j), cs[j], wf);
      a.w[i] = wf;
      const double wi = (double)wf, vi = (double)vf;
      ww += wi * wi;
      vw += vi * wi;
      vv += vi * vi;
    }
    ww = block_sum(ww, red);
    vw = block_sum(vw, red);
    vv = block_sum(vv, red);
    if (threadIdx.x == 0) {
      mypart[NRM] = ww;
      mypart[NRM + 1] = vw;
      mypart[NRM + 2] = vv;
    }
    if (!grid_barrier(a.bar, a.err)) return;
    // ---- decision (identical in every block) and the next iterate; the three norms
    // summed over the blocks' partials by warps 0..2
    if (warp < 3) {
      double t = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(a.part + (int64_t)b * a.ps + NRM + warp);
      t = warp_sum(t);
      if (lane == 0) scal[warp] = t;
    }
    __syncthreads();
    const double tw = scal[0], tvw = scal[1], tvv = scal[2];
    __syncthreads();
    if (threadIdx.x == 0) {
      const int it1 = it + 1;
      const double nw = sqrt(tw);
      int st = 0, done = 0;
      double sc = 0.0;
      if (!(nw > 1e-30 * a.rank_scale)) {
        st = 2;
        done = 1;
      } else {
        sc = 1.0 / nw;
        if (a.iters_override > 0) {
          done = it1 >= a.iters_override;
        } else {
          const double cosv = fabs(tvw) / (nw * sqrt(tvv));
          done = cosv >= 1.0 - a.eps;
          if (!done && it1 >= a.max_iter) {
            done = 1;
            st = 1;
          }
        }
      }
      scal[0] = sc;
      scal[1] = (double)st;
      scal[2] = (double)done;
      if (blockIdx.x == 0 && done) {
        a.info[0] = it1;
        a.info[1] = st;
        a.info[2] = 1;
        a.info[3] = it1;
      }
    }
    __syncthreads();
    const double sc = scal[0];
    const int st = (int)scal[1];
    const bool done = scal[2] != 0.0;
    if (st == 2) {
      // B v0 vanished: the result stays v0 (cur); w is cleared for the caller
      for (int64_t i = gt; i < a.n; i += gs) a.w[i] = 0.f;
      return;
    }
    for (int64_t i = gt; i < a.n; i += gs) {
      nxt[i] = (float)((double)__ldcg(a.w + i) * sc);
      a.w[i] = 0.f;
    }
    if (done) return;
    __syncthreads();
    if (l > 0) proj_partials(nxt);
    if (!grid_barrier(a.bar, a.err)) return;
  }
}

}  // namespace

size_t csr_power_part_bytes(int grid) { return (size_t)grid * (kMaxL + 4) * sizeof(double); }

tsvd_status launch_csr_power(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci, const float *va,
                             const float *Vr, int64_t ldk, const double *sig2, int64_t l, float *buf0, float *buf1,
                             float *w, double *part, size_t part_bytes, unsigned *bar, int *err, double eps,
                             int max_iter, int iters_override, double rank_scale, int *info, double avg_nnz,
                             int max_blocks, cudaStream_t stream) {
  if (m <= 0 || n <= 0 || l < 0 || l > kMaxL) return TSVD_EINVAL;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const int G = avg_nnz <= 6.0 ? 4 : avg_nnz <= 20.0 ? 8 : avg_nnz <= 56.0 ? 16 : 32;
  void *fn = G == 4 ? (void *)csr_power_kernel<4>
             : G == 8 ? (void *)csr_power_kernel<8>
             : G == 16 ? (void *)csr_power_kernel<16>
                       : (void *)csr_power_kernel<32>;
  int per_sm = 0;
  TSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PT, 0));
  if (per_sm < 1) return TSVD_EUNSUPPORTED;
  const int64_t rows_per_block = (PT / 32) * (32 / G);
  int64_t grid = std::min<int64_t>({(int64_t)di.sms * per_sm, ceil_div(m, rows_per_block),
                                    (int64_t)std::max(1, max_blocks)});
  grid = std::max<int64_t>(grid, 1);
  if (part_bytes < csr_power_part_bytes((int)grid)) return TSVD_EINVAL;
  CsrPowerArgs a;
  a.m = m;
  a.n = n;
  a.rp = rp;
  a.ci = ci;
  a.va = va;
  a.Vr = Vr;
  a.ldk = ldk;
  a.sig2 = sig2;
  a.l = (int)l;
  a.buf0 = buf0;
  a.buf1 = buf1;
  a.w = w;
  a.part = part;
  a.ps = kMaxL + 4;
  a.bar = bar;
  a.err = err;
  a.eps = eps;
  a.max_iter = max_iter > 0 ? max_iter : 10000;
  a.iters_override = iters_override;
  a.rank_scale = rank_scale;
  a.info = info;
  void *args[] = {&a};
  TSVD_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(PT), args, 0, stream));
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
