// Vector kernels of the streamed (CSR) power step.
//
// After the fused pair has produced w = A^T (A v0) for all row blocks, these
// kernels finish one step of Alg. 2 in the Hotelling form of Eq. 2:
//     c_j   = v_j^T v0                    (j < l)
//     w    -= sum_j sigma_j^2 c_j v_j
//     v1    = w / ||w||,  cos = |v0 . w| / (||v0|| ||w||),  stop if cos >= 1 - eps
// The vectors are FP32 (n can be 2^25); every sum is FP64 and reduced in a
// fixed order, so the decision is deterministic.  The decision is written to
// a small device info block that the host reads once per application, since
// the next application needs another pass over the streamed matrix anyway.
#include <algorithm>

#include "common.cuh"

namespace tsvd {
namespace {

constexpr int VT = 256;

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// per-block partial of sum x^2 (x FP64)
__global__ void sumsq_f64_kernel(const double *__restrict__ x, int64_t n, double *part, int ps) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) s += x[i] * x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * ps] = s;
}

// one block: out[o] = sum over blocks of part[b*ps + off + o], o < count
__global__ void reduce_parts_kernel(const double *__restrict__ part, int ps, int nblocks, int off,
                                    int count, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = warp; o < count; o += nw) {
    double t = 0.0;
    for (int b = lane; b < nblocks; b += 32) t += part[(int64_t)b * ps + off + o];
    t = warp_sum(t);
    if (lane == 0) out[o] = t;
  }
}

__global__ void normalize_finish_kernel(double *scal) {
  if (threadIdx.x == 0) {
    const double xx = scal[3];
    scal[4] = xx > 0.0 ? 1.0 / sqrt(xx) : 0.0;
  }
}

__global__ void scale_f64_to_f32_kernel(const double *__restrict__ x, float *__restrict__ v, int64_t n,
                                        const double *scal) {
  const double s = scal[4];
  for (int64_t i = gtid(); i < n; i += gstride()) v[i] = (float)(x[i] * s);
}

// partial c_j = sum_i Vr[i*ldk + j0 + j] v[i] for j < cols (cols <= 32).  Each thread sums
// its few elements (n / grid threads; 128 at n = 2^25) in FP32, the warp and block sums
// are FP64: the FP64 pipe of this part is narrow, and an FP64 product per (i, j) made
// these kernels FP64-bound
__global__ void __launch_bounds__(VT) proj_partial_kernel(const float *__restrict__ Vr, int64_t ldk,
                                                          int j0, int cols, const float *__restrict__ v,
                                                          int64_t n, double *part, int ps) {
  float acc[kVecMaxCols];
#pragma unroll
  for (int j = 0; j < kVecMaxCols; ++j) acc[j] = 0.f;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float vi = v[i];
    const float *row = Vr + i * ldk + j0;
#pragma unroll
    for (int j = 0; j < kVecMaxCols; ++j)
      if (j < cols) acc[j] = fmaf(__ldg(row + j), vi, acc[j]);
  }
  __shared__ double sm[VT / 32][kVecMaxCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kVecMaxCols; ++j) {
    const double t = warp_sum((double)acc[j]);
    if (lane == 0) sm[warp][j] = t;
  }
  __syncthreads();
  if (threadIdx.x < cols) {
    double t = 0.0;
    for (int w = 0; w < VT / 32; ++w) t += sm[w][threadIdx.x];
    part[(int64_t)blockIdx.x * ps + 1 + j0 + threadIdx.x] = t;
  }
}

__global__ void coef_kernel(const double *c, const double *sig2, int l, int orth_only, double *coef) {
  for (int j = threadIdx.x; j < l; j += blockDim.x) coef[j] = orth_only ? c[j] : sig2[j] * c[j];
}

// w[i] = base[i] - sum_j Vr[i*ldk+j] coef[j] (the l corrections in FP32, like the
// iterate itself); partial ww, vw, vv of the stored FP32 values, in FP64
__global__ void __launch_bounds__(VT) deflate_kernel(const float *__restrict__ Vr, int64_t ldk, int l,
                                                     const double *__restrict__ coef,
                                                     const float *__restrict__ v, float *w, int64_t n,
                                                     int orth_only, double *part, int ps, int off) {
  __shared__ float cs[256];
  __shared__ double red[33];
  for (int j = threadIdx.x; j < l && j < 256; j += blockDim.x) cs[j] = (float)coef[j];
  __syncthreads();
  double ww = 0.0, vw = 0.0, vv = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float vf = v[i];
    float wf = orth_only ? vf : w[i];
    const float *row = Vr + i * ldk;
    for (int j = 0; j < l; ++j) wf = fmaf(-__ldg(row + j), j < 256 ? cs[j] : (float)coef[j], wf);
    w[i] = wf;
    const double wi = (double)wf, vi = (double)vf;
    ww += wi * wi;
    vw += vi * wi;
    vv += vi * vi;
  }
  ww = block_sum(ww, red);
  vw = block_sum(vw, red);
  vv = block_sum(vv, red);
  if (threadIdx.x == 0) {
    double *p = part + (int64_t)blockIdx.x * ps + off;
    p[0] = ww;
    p[1] = vw;
    p[2] = vv;
  }
}

// decide: scal[0..2] = ww, vw, vv; info[0] += 1 unless orth_only; info[1] status; info[2] done;
// info[3] the application (1-based) at which the triplet stopped, 0 while it runs.
// ctr (not with orth_only): the triplet's application counter; an application queued after
// the one that stopped the triplet does nothing.  The counter lives in device memory, so
// every application of a triplet launches with the same arguments (a captured graph
// replays them)
__global__ void decide_kernel(double *scal, int *info, double eps, int max_iter, int iters_override,
                              double rank_scale, int orth_only, int *ctr) {
  if (threadIdx.x != 0) return;
  int app = 0;
  if (!orth_only && ctr) {
    app = ++(*ctr);
    if (info[3] != 0 && info[3] < app) return;
  }
  const double ww = scal[0], vw = scal[1], vv = scal[2];
  const double nw = sqrt(ww);
  scal[4] = nw > 0.0 ? 1.0 / nw : 0.0;
  if (orth_only) {
    info[2] = 1;
    return;
  }
  const int it = info[0] + 1;
  info[0] = it;
  if (!(nw > 1e-30 * rank_scale)) {
    info[1] = 2;
    info[2] = 1;
    info[3] = app ? app : it;
    return;
  }
  const double cosv = fabs(vw) / (nw * sqrt(vv));
  scal[5] = cosv;
  int done;
  if (iters_override > 0) {
    done = it >= iters_override;
  } else {
    done = cosv >= 1.0 - eps;
    if (!done && it >= max_iter) {
      done = 1;
      info[1] = 1;
    }
  }
  info[2] = done;
  if (done) info[3] = app ? app : it;
}

__global__ void scale_f32_kernel(const float *__restrict__ w, float *__restrict__ out, int64_t n,
                                 const double *scal, const int *info, const int *ctr) {
  if (ctr) {
    const int stop = info[3];
    if (stop != 0 && stop < *ctr) return;  // an earlier application stopped the triplet
  }
  const double s = scal[4];
  for (int64_t i = gtid(); i < n; i += gstride()) out[i] = (float)((double)w[i] * s);
}

// block arg-max of |v| (ties -> lowest index): part[b*ps+0] = value, [1] = index
__global__ void argmax_kernel(const float *__restrict__ v, int64_t n, double *part, int ps) {
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double m = fabs((double)v[i]);
    if (m > best) { best = m; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  __shared__ double sb[32];
  __shared__ long long si[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sb[warp] = best; si[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sb[w] > best || (sb[w] == best && si[w] < bi)) { best = sb[w]; bi = si[w]; }
    part[(int64_t)blockIdx.x * ps] = best;
    part[(int64_t)blockIdx.x * ps + 1] = (double)bi;
  }
}

__global__ void argmax_finish_kernel(const double *part, int ps, int nblocks, const float *v, double *scal) {
  if (threadIdx.x != 0) return;
  double gb = -1.0;
  int64_t gi = 0;
  for (int b = 0; b < nblocks; ++b) {
    const double cb = part[(int64_t)b * ps];
    const int64_t ci = (int64_t)part[(int64_t)b * ps + 1];
    if (cb > gb || (cb == gb && ci < gi)) { gb = cb; gi = ci; }
  }
  scal[6] = v[gi] < 0.f ? -1.0 : 1.0;
}

__global__ void store_column_kernel(float *v, float *Vr, int64_t ldk, int64_t l, int64_t n,
                                    const double *scal, int use_sign) {
  const float s = use_sign ? (float)scal[6] : 1.f;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float x = v[i] * s;
    v[i] = x;
    Vr[i * ldk + l] = x;
  }
}

}  // namespace

size_t vec_scratch_bytes(int grid) {
  return (size_t)grid * kVecPartStride * sizeof(double) + 4096;
}

static int vec_grid(int64_t n, const VecScratch &sc) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, VT), sc.grid));
}

tsvd_status launch_vec_normalize_f64_to_f32(const double *x, float *v, int64_t n, VecScratch sc,
                                            cudaStream_t stream) {
  const int g = vec_grid(n, sc);
  sumsq_f64_kernel<<<g, VT, 0, stream>>>(x, n, sc.part, kVecPartStride);
  TSVD_LAUNCHED();
  reduce_parts_kernel<<<1, 32, 0, stream>>>(sc.part, kVecPartStride, g, 0, 1, sc.scal + 3);
  TSVD_LAUNCHED();
  normalize_finish_kernel<<<1, 32, 0, stream>>>(sc.scal);
  TSVD_LAUNCHED();
  scale_f64_to_f32_kernel<<<g, VT, 0, stream>>>(x, v, n, sc.scal);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_vec_deflate_step(int64_t n, const float *Vr, int64_t ldk, const double *sig2,
                                    int64_t l, const float *v, float *w, float *vnext, double eps,
                                    int max_iter, int iters_override, double scale, VecScratch sc,
                                    int orth_only, cudaStream_t stream, int *ctr) {
  const int g = vec_grid(n, sc);
  if (l + 4 > kVecPartStride) return TSVD_EUNSUPPORTED;
  if (l > 0) {
    for (int64_t j0 = 0; j0 < l; j0 += kVecMaxCols) {
      const int cols = (int)std::min<int64_t>(kVecMaxCols, l - j0);
      proj_partial_kernel<<<g, VT, 0, stream>>>(Vr, ldk, (int)j0, cols, v, n, sc.part, kVecPartStride);
      TSVD_LAUNCHED();
    }
    reduce_parts_kernel<<<1, 256, 0, stream>>>(sc.part, kVecPartStride, g, 1, (int)l, sc.coef);
    TSVD_LAUNCHED();
    coef_kernel<<<1, 256, 0, stream>>>(sc.coef, sig2, (int)l, orth_only, sc.coef);
    TSVD_LAUNCHED();
  }
  deflate_kernel<<<g, VT, 0, stream>>>(Vr, ldk, (int)l, sc.coef, v, w, n, orth_only, sc.part,
                                       kVecPartStride, (int)(kVecPartStride - 3));
  TSVD_LAUNCHED();
  reduce_parts_kernel<<<1, 96, 0, stream>>>(sc.part, kVecPartStride, g, kVecPartStride - 3, 3, sc.scal);
  TSVD_LAUNCHED();
  decide_kernel<<<1, 32, 0, stream>>>(sc.scal, sc.info, eps, max_iter, iters_override, scale, orth_only,
                                      orth_only ? nullptr : ctr);
  TSVD_LAUNCHED();
  scale_f32_kernel<<<g, VT, 0, stream>>>(w, vnext, n, sc.scal, sc.info, orth_only ? nullptr : ctr);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_vec_store_column(int64_t n, const float *v, float *Vr, int64_t ldk, int64_t l,
                                    int sign_convention, VecScratch sc, cudaStream_t stream) {
  const int g = vec_grid(n, sc);
  if (sign_convention) {
    argmax_kernel<<<g, VT, 0, stream>>>(v, n, sc.part, kVecPartStride);
    TSVD_LAUNCHED();
    argmax_finish_kernel<<<1, 32, 0, stream>>>(sc.part, kVecPartStride, g, v, sc.scal);
    TSVD_LAUNCHED();
  }
  store_column_kernel<<<g, VT, 0, stream>>>(const_cast<float *>(v), Vr, ldk, l, n, sc.scal,
                                            sign_convention);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
