// Deflated power iteration on a dense Gram matrix, kept on the device.
//
// Restates Alg. 2 (v1 = B v0, v1 /= ||v1||, stop when
// |v0 . v1| >= 1 - eps) with B deflated in the Hotelling form that Eq. 2
// reduces to for exact earlier triplets:
//     w = G v0 - sum_{j<l} sigma_j^2 v_j (v_j^T v0)
// and closes with sigma_l^2 = v_l^T G v_l (Alg. 1: sigma = ||A v||).
//
// The Gram matrix is deflated once per triplet (rank-1 update in FP64 of
// the FP64 upper triangle, tsvd_gram_deflate) and the FP32 copy the loop
// reads is rounded from the deflated FP64 matrix, so an iteration is one
// GEMV with the deflated matrix and the copy's rounding error is relative to
// the spectrum that remains (deflating the FP32 copy itself would leave
// errors of ~2^-24 sigma_0^2, larger than the small eigenvalues still to
// find).  sigma_l^2 = v_l^T G v_l is formed as v_l^T G_defl v_l +
// sum_{j<l} sigma_j^2 (v_j . v_l)^2.  One cooperative
// launch runs the whole loop; each block owns a contiguous range of rows and
// an iteration has a single bounded grid barrier:
//   w = G32_defl v for the block's rows (FP32 products, FP64 row sums) and
//   the block's partial ||w||^2, v.w, v.v (FP64) -> barrier -> every block
//   reduces the partials in the same fixed order, so all blocks take the same
//   convergence decision without a host round trip.
// Also here: the symmetrising copy G64 -> G32, the Philox-4x32-10 start
// draws, and small conversions.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "philox.cuh"

namespace tsvd {
namespace {

constexpr int PT = 512;             // threads per block of the power kernel
constexpr int kMaxPowerBlocks = 1024;

struct PowerArgs {
  int64_t n;
  const float *G32;
  const double *G64;
  const double *V64;
  const double *sig2;
  int l;
  double *x;
  double eps;
  int max_iter;
  int iters_override;
  int sign_convention;
  double *out_sigma2;
  int *info;
  float *wb0, *wb1;    // n each: the FP32 iterate (unnormalised w) in two buffers
  double *part;        // gridDim.x * ps
  int ps;              // partial stride (doubles)
  unsigned *bar;       // 2 counters
  int *err;
  int64_t rows_per_block;
  int keep8;           // row pairs p with (p mod 8) < keep8 are read with normal loads, the others
                       // evict-first, so the kept share of G32 stays in L2 across iterations
};

// s + e == a + b exactly (Knuth's TwoSum, FP32, no FMA contraction possible)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Warp sum of FP32 values carried as an unevaluated hi + lo pair (every
// partial addition is error-free); every lane ends with the same pair.
// GB300's FP64 pipe is narrow, so the row sums stay in FP32 and only lane 0
// forms the FP64 value.
__device__ __forceinline__ void warp_sum_f32x2(float &hi, float &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ho = __shfl_xor_sync(0xffffffffu, hi, o);
    const float lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, ho, s, e);
    hi = s;
    lo = lo + lo2 + e;
  }
}

// sum of part[c*ps + off] over blocks c = lane, lane+32, ... (the loads are
// issued together, then added in a fixed order)
__device__ __forceinline__ double lane_partials(const double *part, int ps, int off, int lane) {
  double v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int c = lane + 32 * u;
    v[u] = c < (int)gridDim.x ? __ldcg(part + (int64_t)c * ps + off) : 0.0;
  }
  double t = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) t += v[u];
  for (int c = lane + 256; c < (int)gridDim.x; c += 32) t += __ldcg(part + (int64_t)c * ps + off);
  return t;
}

// reduce part[c*ps + off] over all blocks c, same order in every block
__device__ double reduce_partials(const double *part, int ps, int off, double *red) {
  if (threadIdx.x < 32) {
    double t = lane_partials(part, ps, off, threadIdx.x);
    t = warp_sum(t);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(PT, 1) power_dense_kernel(PowerArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *vs = reinterpret_cast<float *>(smem_raw);                                // n floats (padded)
  double *coef = reinterpret_cast<double *>(smem_raw + ((a.n + 3) / 4) * 16);    // l doubles
  __shared__ double red[33];
  __shared__ double wred[3 * (PT / 32)];
  __shared__ double s_scal[4];

  const int64_t n = a.n;
  const int l = a.l;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t r1 = min(n, r0 + a.rows_per_block);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = PT / 32;
  const int ps = a.ps;
  double *mypart = a.part + (int64_t)blockIdx.x * ps;
  const bool vec = (n % 4 == 0);

  // ---- prologue: v0 = x / ||x|| (Alg. 2)
  double s = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
    const double xi = __ldcg(a.x + i);
    s += xi * xi;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) mypart[0] = s;
  if (!grid_barrier(a.bar, a.err)) return;
  const double xx = reduce_partials(a.part, ps, 0, red);
  if (threadIdx.x == 0) s_scal[0] = xx > 0.0 ? 1.0 / sqrt(xx) : 0.0;
  __syncthreads();
  double vscale = s_scal[0];
  __syncthreads();
  const double rank_scale = (l == 0) ? 1.0 : __ldcg(a.sig2);

  int it = 0, status = 0;
  const float *vsrc = nullptr;  // FP32 iterate of the previous step (unnormalised)
  float *wnext = a.wb0;
  for (;;) {
    // ---- v = w_prev / ||w_prev|| into shared memory (FP32)
    if (it == 0) {
      for (int64_t j = threadIdx.x; j < n; j += PT) vs[j] = (float)(__ldcg(a.x + j) * vscale);
    } else {
      const float sc = (float)vscale;
      int64_t j = threadIdx.x;
      for (; j + 7 * PT < n; j += 8 * PT) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = __ldcg(vsrc + j + u * PT);
#pragma unroll
        for (int u = 0; u < 8; ++u) vs[j + u * PT] = t[u] * sc;
      }
      for (; j < n; j += PT) vs[j] = __ldcg(vsrc + j) * sc;
    }
    __syncthreads();
    // ---- w = G32_defl v for this block's rows, partial ||w||^2, v.w, v.v
    double ww = 0.0, vw = 0.0, vv = 0.0;
    for (int64_t i = r0 + 2 * warp; i < r1; i += 2 * nwarps) {
      // rows i and i+1 (the second may be past the block's range)
      const bool two = i + 1 < r1;
      const float *g0 = a.G32 + i * n;
      const float *g1 = a.G32 + (two ? i + 1 : i) * n;
      float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
      if (vec) {
        const float4 *ga = reinterpret_cast<const float4 *>(g0);
        const float4 *gb = reinterpret_cast<const float4 *>(g1);
        const float4 *v4 = reinterpret_cast<const float4 *>(vs);
        const int64_t n4 = n >> 2;
        const bool keep = ((i >> 1) & 7) < a.keep8;
        int64_t q = lane;
        // sixteen independent 16-byte loads in flight per lane
        for (; q + 32 * 7 < n4; q += 32 * 8) {
          float4 ra[8], rb[8];
          if (keep) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              ra[u] = __ldg(ga + q + 32 * u);
              rb[u] = __ldg(gb + q + 32 * u);
            }
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              ra[u] = __ldcs(ga + q + 32 * u);
              rb[u] = __ldcs(gb + q + 32 * u);
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 vq = v4[q + 32 * u];
            p0 = fmaf(ra[u].x, vq.x, p0); p1 = fmaf(ra[u].y, vq.y, p1);
            p2 = fmaf(ra[u].z, vq.z, p2); p3 = fmaf(ra[u].w, vq.w, p3);
            q0 = fmaf(rb[u].x, vq.x, q0); q1 = fmaf(rb[u].y, vq.y, q1);
            q2 = fmaf(rb[u].z, vq.z, q2); q3 = fmaf(rb[u].w, vq.w, q3);
          }
        }
        for (; q < n4; q += 32) {
          const float4 xa = __ldg(ga + q), xb = __ldg(gb + q), vq = v4[q];
          p0 = fmaf(xa.x, vq.x, p0); p1 = fmaf(xa.y, vq.y, p1);
          p2 = fmaf(xa.z, vq.z, p2); p3 = fmaf(xa.w, vq.w, p3);
          q0 = fmaf(xb.x, vq.x, q0); q1 = fmaf(xb.y, vq.y, q1);
          q2 = fmaf(xb.z, vq.z, q2); q3 = fmaf(xb.w, vq.w, q3);
        }
      } else {
        for (int64_t q = lane; q < n; q += 32) {
          p0 = fmaf(__ldg(g0 + q), vs[q], p0);
          q0 = fmaf(__ldg(g1 + q), vs[q], q0);
        }
      }
      float h0, e0, h1, e1, sa, ea, sb2, eb;
      two_sum(p0, p1, sa, ea);
      two_sum(p2, p3, sb2, eb);
      two_sum(sa, sb2, h0, e0);
      e0 += ea + eb;
      two_sum(q0, q1, sa, ea);
      two_sum(q2, q3, sb2, eb);
      two_sum(sa, sb2, h1, e1);
      e1 += ea + eb;
      warp_sum_f32x2(h0, e0);
      warp_sum_f32x2(h1, e1);
      if (lane == 0) {
        // the iterate is stored in FP32; the sums use exactly the stored values,
        // so 1/||w|| normalises the stored vector to FP64 accuracy
        const double t0 = (double)(float)((double)h0 + (double)e0);
        const double t1 = (double)(float)((double)h1 + (double)e1);
        const double v0i = (double)vs[i];
        wnext[i] = (float)t0;
        ww += t0 * t0;
        vw += v0i * t0;
        vv += v0i * v0i;
        if (two) {
          const double v1i = (double)vs[i + 1];
          wnext[i + 1] = (float)t1;
          ww += t1 * t1;
          vw += v1i * t1;
          vv += v1i * v1i;
        }
      }
    }
    // block sums of the three values (only lane 0 of each warp holds any)
    if (lane == 0) {
      wred[3 * warp] = ww;
      wred[3 * warp + 1] = vw;
      wred[3 * warp + 2] = vv;
    }
    __syncthreads();
    // partials alternate between two slots, so a block still reading the
    // previous iteration's sums is never overwritten
    const int slot = 1 + (it & 1) * 3;
    if (threadIdx.x == 0) {
      double t0 = 0.0, t1 = 0.0, t2 = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        t0 += wred[3 * w];
        t1 += wred[3 * w + 1];
        t2 += wred[3 * w + 2];
      }
      mypart[slot] = t0;
      mypart[slot + 1] = t1;
      mypart[slot + 2] = t2;
    }
    if (!grid_barrier(a.bar, a.err)) return;

    // ---- identical decision in every block (warp 0 reduces, thread 0 decides:
    // FP64 division and square roots are slow on this part, so no other thread
    // repeats them)
    if (warp == 0) {
      double t0 = lane_partials(a.part, ps, slot, lane);
      double t1 = lane_partials(a.part, ps, slot + 1, lane);
      double t2 = lane_partials(a.part, ps, slot + 2, lane);
      t0 = warp_sum(t0);
      t1 = warp_sum(t1);
      t2 = warp_sum(t2);
      if (lane == 0) {
        const int it1 = it + 1;
        const double nw = sqrt(t0);
        int st = 0, done = 0;
        double sc = 0.0;
        if (!(nw > 1e-30 * rank_scale)) {
          st = 2;
          done = 1;
        } else {
          sc = 1.0 / nw;
          const double cosv = fabs(t1) / (nw * sqrt(t2));
          if (a.iters_override > 0) {
            done = it1 >= a.iters_override;
          } else {
            done = cosv >= 1.0 - a.eps;
            if (!done && it1 >= a.max_iter) {
              done = 1;
              st = 1;
            }
          }
        }
        s_scal[0] = sc;
        s_scal[1] = (double)st;
        s_scal[2] = (double)done;
      }
    }
    __syncthreads();
    ++it;
    const int st = (int)s_scal[1];
    const bool done = s_scal[2] != 0.0;
    if (st == 2) {
      status = 2;
      break;
    }
    vsrc = wnext;
    vscale = s_scal[0];
    wnext = (wnext == a.wb0) ? a.wb1 : a.wb0;
    __syncthreads();  // s_scal is rewritten in the next iteration
    if (done) {
      status = st;
      break;
    }
  }

  // ---- the block's rows of v_l (FP64) into x
  if (status == 2) {
    // rank(A) < l+1: v = v0 made orthogonal to v_0..v_{l-1} (two passes), sigma = 0.
    // v0 is the vector of the step whose B v0 vanished (x itself on the first step).
    for (int64_t i = r0 + threadIdx.x; i < r1; i += PT)
      a.x[i] = it <= 1 ? __ldcg(a.x + i) * vscale : (double)__ldcg(vsrc + i) * vscale;
    for (int pass = 0; pass < 2; ++pass) {
      __syncthreads();
      for (int j = warp; j < l; j += nwarps) {
        const double *vj = a.V64 + (int64_t)j * n;
        double t = 0.0;
        for (int64_t i = r0 + lane; i < r1; i += 32) t += __ldg(vj + i) * a.x[i];
        t = warp_sum(t);
        if (lane == 0) mypart[7 + j] = t;
      }
      if (!grid_barrier(a.bar, a.err)) return;
      for (int j = warp; j < l; j += nwarps) {
        double t = lane_partials(a.part, ps, 7 + j, lane);
        t = warp_sum(t);
        if (lane == 0) coef[j] = t;
      }
      __syncthreads();
      double nn = 0.0;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
        double wi = a.x[i];
        for (int j = 0; j < l; ++j) wi -= __ldg(a.V64 + (int64_t)j * n + i) * coef[j];
        a.x[i] = wi;
        nn += wi * wi;
      }
      nn = block_sum(nn, red);
      if (threadIdx.x == 0) mypart[7 + l] = nn;
      if (!grid_barrier(a.bar, a.err)) return;
      const double tn = reduce_partials(a.part, ps, 7 + l, red);
      if (threadIdx.x == 0) s_scal[0] = tn > 0.0 ? 1.0 / sqrt(tn) : 0.0;
      __syncthreads();
      const double sc = s_scal[0];
      __syncthreads();
      for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) a.x[i] *= sc;
    }
  } else {
    for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) a.x[i] = (double)__ldcg(vsrc + i) * vscale;
  }
  __syncthreads();

  // ---- sign convention: largest |v_i| positive, lowest index on ties
  if (a.sign_convention) {
    double best = -1.0;
    int64_t bidx = 0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
      const double m = fabs(a.x[i]);
      if (m > best) { best = m; bidx = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    __shared__ double sb[32];
    __shared__ long long si[32];
    if (lane == 0) { sb[warp] = best; si[warp] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nwarps; ++w)
        if (sb[w] > best || (sb[w] == best && si[w] < bidx)) { best = sb[w]; bidx = si[w]; }
      mypart[8 + l] = best;
      mypart[9 + l] = (double)bidx;
    }
    if (!grid_barrier(a.bar, a.err)) return;
    if (threadIdx.x == 0) {
      double gb = -1.0;
      int64_t gi = 0;
      for (int c = 0; c < (int)gridDim.x; ++c) {
        const double cb = __ldcg(a.part + (int64_t)c * ps + 8 + l);
        const int64_t ci = (int64_t)__ldcg(a.part + (int64_t)c * ps + 9 + l);
        if (cb > gb || (cb == gb && ci < gi)) { gb = cb; gi = ci; }
      }
      s_scal[0] = __ldcg(a.x + gi) < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    const double sign = s_scal[0];
    __syncthreads();  // every block reads x[gi] before any block flips its rows
    if (!grid_barrier(a.bar, a.err)) return;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) a.x[i] *= sign;
  }

  // ---- sigma^2 = v^T G v = v^T G_defl v (upper triangle of the deflated FP64
  // matrix) + sum_{j<l} sigma_j^2 (v_j . v)^2, once per triplet
  if (!grid_barrier(a.bar, a.err)) return;
  double q = 0.0;
  if (status != 2) {
    for (int64_t i = r0 + warp; i < r1; i += nwarps) {
      const double *g = a.G64 + i * n;
      double t = 0.0;
      for (int64_t j = i + lane; j < n; j += 32) {
        const double gv = __ldg(g + j) * __ldcg(a.x + j);
        t += (j == i) ? gv : 2.0 * gv;
      }
      t = warp_sum(t);
      if (lane == 0) q += t * __ldcg(a.x + i);
    }
    for (int j = warp; j < l; j += nwarps) {
      const double *vj = a.V64 + (int64_t)j * n;
      double t = 0.0;
      for (int64_t i = r0 + lane; i < r1; i += 32) t += __ldg(vj + i) * __ldcg(a.x + i);
      t = warp_sum(t);
      if (lane == 0) mypart[11 + l + j] = t;
    }
  }
  q = block_sum(q, red);
  if (threadIdx.x == 0) mypart[10 + l] = q;
  if (!grid_barrier(a.bar, a.err)) return;
  if (blockIdx.x == 0) {
    double tq = reduce_partials(a.part, ps, 10 + l, red);
    if (status != 2) {
      for (int j = 0; j < l; ++j) {
        const double c = reduce_partials(a.part, ps, 11 + l + j, red);
        tq += __ldg(a.sig2 + j) * c * c;
      }
    }
    if (threadIdx.x == 0) {
      *a.out_sigma2 = status == 2 ? 0.0 : fmax(tq, 0.0);
      a.info[0] = it;
      a.info[1] = status;
      a.info[2] = 0;
    }
  }
}

// FULL64: also mirror the upper triangle of G64 into its lower triangle, so
// that every row of G64 holds the full symmetric row
template <bool FULL64>
__global__ void symmetrize_kernel(int64_t n, double *__restrict__ G64, float *__restrict__ G32) {
  // 32 x 32 tiles: G32[i][j] = G64[min(i,j)][max(i,j)]
  __shared__ float t[32][33];
  __shared__ double t64[FULL64 ? 32 : 1][33];
  const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (bj >= bi) {
    // tile in the upper triangle: direct copy (row i <= col j) and mirrored copy
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = bi + r, j = bj + tx;
      double g = 0.0;
      if (i < n && j < n) g = j >= i ? G64[i * n + j] : G64[j * n + i];
      const float v = (float)g;
      t[r][tx] = v;
      if (FULL64) t64[FULL64 ? r : 0][tx] = g;
      if (i < n && j < n) G32[i * n + j] = v;
    }
    __syncthreads();
    if (bj != bi) {
      for (int r = ty; r < 32; r += 8) {
        const int64_t i = bj + r, j = bi + tx;  // mirrored tile
        if (i < n && j < n) {
          G32[i * n + j] = t[tx][r];
          if (FULL64) G64[i * n + j] = t64[FULL64 ? tx : 0][r];
        }
      }
    } else if (FULL64) {
      // diagonal tile: its strict lower part from the tile (only upper entries were read)
      for (int r = ty; r < 32; r += 8) {
        const int64_t i = bi + r, j = bj + tx;
        if (i < n && j < n && tx < r) G64[i * n + j] = t64[FULL64 ? tx : 0][r];
      }
    }
  }
}

__global__ void start_draws_kernel(uint32_t k0, uint32_t k1, uint32_t lword, int64_t n, double *x) {
  const int64_t pairs = (n + 1) / 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    double z0, z1;
    start_normal_pair(k0, k1, lword, p, &z0, &z1);
    x[2 * p] = z0;
    if (2 * p + 1 < n) x[2 * p + 1] = z1;
  }
}

__global__ void philox_raw_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox10(c, key[2 * i], key[2 * i + 1]);
    out[4 * i] = c[0];
    out[4 * i + 1] = c[1];
    out[4 * i + 2] = c[2];
    out[4 * i + 3] = c[3];
  }
}

// Hotelling deflation by one extracted triplet, in FP64: for the upper
// triangle of G64 (entry (i, j), j >= i, at i n + j) G64 -= sigma2 v_i v_j,
// and the FP32 copy of the deflated matrix, both halves.  32 x 32 tiles of
// the upper triangle; each mirrored FP32 tile goes through shared memory.
__global__ void deflate_gram_kernel(int64_t n, double *__restrict__ G64, float *__restrict__ G32,
                                    const double *__restrict__ v, const double *__restrict__ sigma2) {
  __shared__ float t[32][33];
  const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
  if (bj < bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const double s2 = __ldg(sigma2);
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bi + r, j = bj + tx;
    float f = 0.f;
    if (i < n && j < n && j >= i) {
      const double g = fma(-s2 * __ldg(v + i), __ldg(v + j), G64[i * n + j]);
      G64[i * n + j] = g;
      f = (float)g;
      G32[i * n + j] = f;
    }
    t[r][tx] = f;
  }
  __syncthreads();
  // mirrored entries come from the tile (a diagonal tile mirrors only its strict upper part)
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bj + r, j = bi + tx;
    if (i < n && j < n && (bj != bi || r > tx)) G32[i * n + j] = t[tx][r];
  }
}

__global__ void sigma_kernel(const double *sig2, double *sigma, int64_t k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) sigma[i] = sqrt(fmax(sig2[i], 0.0));
}

__global__ void f64_to_f32_kernel(const double *src, float *dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

}  // namespace

// per-block partial layout (doubles): [0] ||x||^2, [1..3] and [4..6] the
// loop's ||w||^2, v.w, v.v in alternating iterations, [7..7+l) and [7+l] the
// rank-deficient projection, [8+l], [9+l] the sign search, [10+l] v^T G v,
// [11+l .. 11+2l) v_j . v; regions written after the loop never overlap ones
// a slower block may still read
static int64_t power_part_stride(int64_t l) { return round_up(2 * l + 12, 4); }

size_t power_scratch_bytes(int64_t n, int64_t l) {
  const size_t ps = (size_t)power_part_stride(l);
  return 256 + 2 * (size_t)round_up(n, 64) * sizeof(float) + (size_t)kMaxPowerBlocks * ps * sizeof(double);
}

tsvd_status launch_power_dense(int64_t n, const float *G32, const double *G64, const double *V64,
                               const double *sigma2, int64_t l, double *x, double eps,
                               int max_iter, int iters_override, int sign_convention,
                               double *out_sigma2, int *info, void *scratch, size_t scratch_bytes,
                               cudaStream_t stream) {
  if (n <= 0 || l < 0 || !G32 || !G64 || !x || !out_sigma2 || !info || !scratch) return TSVD_EINVAL;
  if (l > 0 && (!V64 || !sigma2)) return TSVD_EINVAL;
  if (scratch_bytes < power_scratch_bytes(n, l)) return TSVD_EINVAL;
  if ((reinterpret_cast<uintptr_t>(scratch) & 255) != 0) return TSVD_EINVAL;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const size_t smem = (size_t)round_up(n, 4) * sizeof(float) + 16 + (size_t)l * sizeof(double);
  if (smem > di.smem_optin) return TSVD_EUNSUPPORTED;
  if (smem > 48 * 1024) TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(power_dense_kernel), smem));
  int per_sm = 0;
  TSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, power_dense_kernel, PT, smem));
  if (per_sm < 1) return TSVD_EUNSUPPORTED;
  int64_t grid = std::min<int64_t>({(int64_t)di.sms * per_sm, ceil_div(n, 16), kMaxPowerBlocks});
  grid = std::max<int64_t>(grid, 1);
  const int64_t rows_per_block = ceil_div(n, grid);
  grid = ceil_div(n, rows_per_block);

  unsigned char *s = static_cast<unsigned char *>(scratch);
  PowerArgs a;
  a.n = n; a.G32 = G32; a.G64 = G64; a.V64 = V64; a.sig2 = sigma2; a.l = (int)l; a.x = x;
  a.eps = eps; a.max_iter = max_iter > 0 ? max_iter : 10000; a.iters_override = iters_override;
  a.sign_convention = sign_convention; a.out_sigma2 = out_sigma2; a.info = info;
  a.bar = reinterpret_cast<unsigned *>(s);
  a.err = reinterpret_cast<int *>(s + 64);
  a.wb0 = reinterpret_cast<float *>(s + 256);
  a.wb1 = a.wb0 + round_up(n, 64);
  a.part = reinterpret_cast<double *>(a.wb1 + round_up(n, 64));
  a.ps = (int)power_part_stride(l);
  a.rows_per_block = rows_per_block;
  // G32 is read once per iteration.  When it is larger than ~60 % of L2, only
  // that share of its rows (every row pair whose index mod 8 is below keep8,
  // spread over all blocks) uses normal loads; the rest are evict-first, so
  // they do not push the kept rows out and those are L2 hits next iteration.
  const double l2_share = 0.6 * (double)di.l2_bytes, g_bytes = 4.0 * (double)n * (double)n;
  a.keep8 = g_bytes <= l2_share ? 8 : (int)(8.0 * l2_share / g_bytes);
  TSVD_CUDA(cudaMemsetAsync(s, 0, 256, stream));
  void *args[] = {&a};
  TSVD_CUDA(cudaLaunchCooperativeKernel((void *)power_dense_kernel, dim3((unsigned)grid), dim3(PT),
                                        args, smem, stream));
  TSVD_LAUNCHED();
  // surface a barrier timeout in info[2]
  TSVD_CUDA(cudaMemcpyAsync(info + 2, a.err, sizeof(int), cudaMemcpyDeviceToDevice, stream));
  return TSVD_OK;
}

tsvd_status launch_symmetrize(int64_t n, double *G64, float *G32, cudaStream_t stream, bool full64) {
  const int64_t nb = ceil_div(n, 32);
  if (nb > 65535) return TSVD_EUNSUPPORTED;
  dim3 grid((unsigned)nb, (unsigned)nb), block(32, 8);
  if (full64)
    symmetrize_kernel<true><<<grid, block, 0, stream>>>(n, G64, G32);
  else
    symmetrize_kernel<false><<<grid, block, 0, stream>>>(n, G64, G32);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_start_draws(uint64_t seed, int64_t l, int64_t n, double *x, cudaStream_t stream) {
  const uint64_t s = splitmix64(seed);
  const int64_t pairs = (n + 1) / 2;
  const int64_t blocks = std::min<int64_t>(ceil_div(pairs, 256), 65535);
  start_draws_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, stream>>>(
      (uint32_t)s, (uint32_t)(s >> 32), (uint32_t)l, n, x);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_philox_raw(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count,
                              cudaStream_t stream) {
  if (count <= 0) return TSVD_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(count, 256), 65535);
  philox_raw_kernel<<<(unsigned)blocks, 256, 0, stream>>>(ctr, key, out, count);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// ---------------------------------------------------------------- no-allocation variant
// Scratch of tsvd_power_dense_noalloc: one file-scope device array sized for
// the largest problem it accepts.  Every GPU that loads the library holds it
// until the process exits.  Host code may not use the array's name as a
// device address (on the host it is only a stand-in for the symbol), so its
// device address is looked up per device with cudaGetSymbolAddress, with that
// device current.  The address belongs to the device's context: it is kept
// with the context it was found in and looked up again when the current
// context is a different one (the primary context recreated after
// cudaDeviceReset loads the module again, possibly at another address).
constexpr int64_t kNoallocScratchBytes =
    256 + 2 * TSVD_NOALLOC_MAX_N * 4 + (int64_t)kMaxPowerBlocks * ((2 * TSVD_NOALLOC_MAX_L + 12 + 3) / 4 * 4) * 8;
static __device__ __align__(256) unsigned char g_power_noalloc_scratch[kNoallocScratchBytes];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

static tsvd_status current_context(CUcontext *ctx) {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TSVD_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) {
      set_error_text("cuCtxGetCurrent not available");
      return TSVD_ECUDA;
    }
    fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  *ctx = nullptr;
  if (fn(ctx) != CUDA_SUCCESS) return TSVD_ECUDA;
  return TSVD_OK;
}

static tsvd_status noalloc_scratch(void **out) {
  static std::mutex mu;
  static void *addr[128] = {};
  static CUcontext ctx_of[128] = {};
  int dev = -1;
  TSVD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return TSVD_EUNSUPPORTED;
  CUcontext ctx = nullptr;
  TSVD_TRY(current_context(&ctx));
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev] || !ctx || ctx_of[dev] != ctx) {
    void *p = nullptr;
    // (the lookup also makes the device's primary context current if no
    // runtime call on this thread has done so yet)
    TSVD_CUDA(cudaGetSymbolAddress(&p, g_power_noalloc_scratch));
    if (!p) return TSVD_ECUDA;
    TSVD_TRY(current_context(&ctx));
    addr[dev] = p;
    ctx_of[dev] = ctx;
  }
  *out = addr[dev];
  return TSVD_OK;
}

tsvd_status launch_power_dense_noalloc(int64_t n, const float *G32, const double *G64, const double *V64,
                                       const double *sigma2, int64_t l, double *x, double eps, int max_iter,
                                       int iters_override, int sign_convention, double *out_sigma2, int *info,
                                       cudaStream_t stream) {
  if (n > TSVD_NOALLOC_MAX_N || l > TSVD_NOALLOC_MAX_L) {
    set_error_text("tsvd_power_dense_noalloc: n must be <= " + std::to_string(TSVD_NOALLOC_MAX_N) +
                   " and l <= " + std::to_string(TSVD_NOALLOC_MAX_L) + " (fixed static scratch)");
    return TSVD_EINVAL;
  }
  void *scratch = nullptr;
  TSVD_TRY(noalloc_scratch(&scratch));
  const size_t need = power_scratch_bytes(n, l);
  if (need > (size_t)kNoallocScratchBytes) return TSVD_EINVAL;
  return launch_power_dense(n, G32, G64, V64, sigma2, l, x, eps, max_iter, iters_override, sign_convention,
                            out_sigma2, info, scratch, (size_t)kNoallocScratchBytes, stream);
}

tsvd_status launch_gram_deflate(int64_t n, double *G64, float *G32, const double *v, const double *sigma2,
                                cudaStream_t stream) {
  if (n <= 0) return TSVD_OK;
  const int64_t nb = ceil_div(n, 32);
  if (nb > 65535) return TSVD_EUNSUPPORTED;
  dim3 grid((unsigned)nb, (unsigned)nb), block(32, 8);
  deflate_gram_kernel<<<grid, block, 0, stream>>>(n, G64, G32, v, sigma2);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_sigma_from_sigma2(const double *sig2, double *sigma, int64_t k, cudaStream_t stream) {
  sigma_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, stream>>>(sig2, sigma, k);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_f64_to_f32(const double *src, float *dst, int64_t count, cudaStream_t stream) {
  if (count <= 0) return TSVD_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(count, 256), 65535);
  f64_to_f32_kernel<<<(unsigned)blocks, 256, 0, stream>>>(src, dst, count);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
