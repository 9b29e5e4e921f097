// Deflated power iteration on a dense Gram matrix, kept on the device.
//
// Restates Alg. 2 l.10-15 (v1 = B v0, v1 /= ||v1||, stop when
// |v0 . v1| >= 1 - eps) with B deflated in the Hotelling form that Eq. 2
// reduces to for exact earlier triplets:
//     w = G v0 - sum_{j<l} sigma_j^2 v_j (v_j^T v0)
// and closes with sigma_l^2 = v_l^T G v_l (Alg. 1 l.11-13: sigma = ||A v||).
//
// One cooperative launch runs the whole loop: each block owns a contiguous
// range of rows; two bounded grid barriers per iteration separate
//   A: w_raw = G32 v (FP32 products, FP64 row sums) and partial v_j^T v
//   B: deflation, partial ||w||^2, v.w, v.v (FP64)
//   C: every block reduces the partials in the same fixed order, so all
//      blocks take the same convergence decision without a host round trip.
// Also here: the symmetrising copy G64 -> G32, the Philox-4x32-10 start
// draws, and small conversions.
#include <algorithm>
#include <mutex>

#include "common.cuh"

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
  double *wb0, *wb1;   // n each
  double *part;        // gridDim.x * ps
  int ps;              // partial stride (doubles)
  unsigned *bar;       // 2 counters
  int *err;
  int64_t rows_per_block;
};

// reduce part[c*ps + off] over all blocks c, same order in every block
__device__ double reduce_partials(const double *part, int ps, int off, double *red) {
  double t = 0.0;
  if (threadIdx.x < 32) {
    for (int c = threadIdx.x; c < (int)gridDim.x; c += 32) t += __ldcg(part + (int64_t)c * ps + off);
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
  float *vs = reinterpret_cast<float *>(smem_raw);                          // n floats (padded)
  double *coef = reinterpret_cast<double *>(smem_raw + ((a.n + 3) / 4) * 16);  // l doubles
  __shared__ double red[33];
  __shared__ double s_scal[4];

  const int64_t n = a.n;
  const int l = a.l;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t r1 = min(n, r0 + a.rows_per_block);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = PT / 32;
  const int ps = a.ps;
  double *mypart = a.part + (int64_t)blockIdx.x * ps;
  const bool vec = (n % 4 == 0);

  // ---- prologue: v0 = x / ||x|| (Alg. 2 l.4)
  double s = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
    const double xi = __ldcg(a.x + i);
    s += xi * xi;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) mypart[0] = s;
  if (!grid_barrier(a.bar, a.err)) return;
  const double xx = reduce_partials(a.part, ps, 0, red);
  const double *vsrc = a.x;
  double vscale = xx > 0.0 ? 1.0 / sqrt(xx) : 0.0;
  const double rank_scale = (l == 0) ? 1.0 : __ldcg(a.sig2);

  int it = 0, status = 0;
  double *wnext = a.wb0;
  for (;;) {
    // ---- phase A: w_raw = G32 v, partial c_j = v_j^T v
    for (int64_t j = threadIdx.x; j < n; j += PT) vs[j] = (float)(__ldcg(vsrc + j) * vscale);
    __syncthreads();
    for (int64_t i = r0 + warp; i < r1; i += nwarps) {
      const float *g = a.G32 + i * n;
      float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
      if (vec) {
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        const float4 *v4 = reinterpret_cast<const float4 *>(vs);
        const int64_t n4 = n >> 2;
        for (int64_t q = lane; q < n4; q += 32) {
          const float4 gq = __ldg(g4 + q);
          const float4 vq = v4[q];
          acc0 = fmaf(gq.x, vq.x, acc0);
          acc1 = fmaf(gq.y, vq.y, acc1);
          acc2 = fmaf(gq.z, vq.z, acc2);
          acc3 = fmaf(gq.w, vq.w, acc3);
        }
      } else {
        for (int64_t q = lane; q < n; q += 32) acc0 = fmaf(__ldg(g + q), vs[q], acc0);
      }
      double t = ((double)acc0 + (double)acc1) + ((double)acc2 + (double)acc3);
      t = warp_sum(t);
      if (lane == 0) wnext[i] = t;
    }
    for (int j = warp; j < l; j += nwarps) {
      const double *vj = a.V64 + (int64_t)j * n;
      double t = 0.0;
      for (int64_t i = r0 + lane; i < r1; i += 32) t += __ldg(vj + i) * (__ldcg(vsrc + i) * vscale);
      t = warp_sum(t);
      if (lane == 0) mypart[1 + j] = t;
    }
    if (!grid_barrier(a.bar, a.err)) return;

    // ---- phase B: deflate (Hotelling), partial norms
    for (int j = warp; j < l; j += nwarps) {
      double t = 0.0;
      for (int c = lane; c < (int)gridDim.x; c += 32) t += __ldcg(a.part + (int64_t)c * ps + 1 + j);
      t = warp_sum(t);
      if (lane == 0) coef[j] = __ldg(a.sig2 + j) * t;
    }
    __syncthreads();
    double ww = 0.0, vw = 0.0, vv = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
      double wi = __ldcg(wnext + i);
      for (int j = 0; j < l; ++j) wi -= __ldg(a.V64 + (int64_t)j * n + i) * coef[j];
      wnext[i] = wi;
      const double vi = __ldcg(vsrc + i) * vscale;
      ww += wi * wi;
      vw += vi * wi;
      vv += vi * vi;
    }
    ww = block_sum(ww, red);
    vw = block_sum(vw, red);
    vv = block_sum(vv, red);
    if (threadIdx.x == 0) {
      mypart[1 + l] = ww;
      mypart[2 + l] = vw;
      mypart[3 + l] = vv;
    }
    if (!grid_barrier(a.bar, a.err)) return;

    // ---- phase C: identical decision in every block
    const double tww = reduce_partials(a.part, ps, 1 + l, red);
    const double tvw = reduce_partials(a.part, ps, 2 + l, red);
    const double tvv = reduce_partials(a.part, ps, 3 + l, red);
    ++it;
    const double nw = sqrt(tww);
    if (!(nw > 1e-30 * rank_scale)) {
      status = 2;
      break;
    }
    const double cosv = fabs(tvw) / (nw * sqrt(tvv));
    vsrc = wnext;
    vscale = 1.0 / nw;
    wnext = (wnext == a.wb0) ? a.wb1 : a.wb0;
    bool done;
    if (a.iters_override > 0) {
      done = it >= a.iters_override;
    } else {
      done = cosv >= 1.0 - a.eps;
      if (!done && it >= a.max_iter) {
        done = true;
        status = 1;
      }
    }
    if (done) break;
  }

  if (status == 2) {
    // rank(A) < l+1: v = v0 made orthogonal to v_0..v_{l-1} (two passes), sigma = 0
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = warp; j < l; j += nwarps) {
        const double *vj = a.V64 + (int64_t)j * n;
        double t = 0.0;
        for (int64_t i = r0 + lane; i < r1; i += 32) t += __ldg(vj + i) * (__ldcg(vsrc + i) * vscale);
        t = warp_sum(t);
        if (lane == 0) mypart[1 + j] = t;
      }
      if (!grid_barrier(a.bar, a.err)) return;
      for (int j = warp; j < l; j += nwarps) {
        double t = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32) t += __ldcg(a.part + (int64_t)c * ps + 1 + j);
        t = warp_sum(t);
        if (lane == 0) coef[j] = t;
      }
      __syncthreads();
      double nn = 0.0;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
        double wi = __ldcg(vsrc + i) * vscale;
        for (int j = 0; j < l; ++j) wi -= __ldg(a.V64 + (int64_t)j * n + i) * coef[j];
        wnext[i] = wi;
        nn += wi * wi;
      }
      nn = block_sum(nn, red);
      if (threadIdx.x == 0) mypart[1 + l] = nn;
      if (!grid_barrier(a.bar, a.err)) return;
      const double tn = reduce_partials(a.part, ps, 1 + l, red);
      vsrc = wnext;
      vscale = tn > 0.0 ? 1.0 / sqrt(tn) : 0.0;
      wnext = (wnext == a.wb0) ? a.wb1 : a.wb0;
    }
  }

  // ---- sign convention: largest |v_i| positive, lowest index on ties
  double sign = 1.0;
  if (a.sign_convention) {
    double best = -1.0;
    int64_t bidx = 0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) {
      const double m = fabs(__ldcg(vsrc + i));
      if (m > best) { best = m; bidx = i; }
    }
    // block arg-max (ties -> lower index)
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
      mypart[1 + l] = best;
      mypart[2 + l] = (double)bidx;
    }
    if (!grid_barrier(a.bar, a.err)) return;
    if (threadIdx.x == 0) {
      double gb = -1.0;
      int64_t gi = 0;
      for (int c = 0; c < (int)gridDim.x; ++c) {
        const double cb = __ldcg(a.part + (int64_t)c * ps + 1 + l);
        const int64_t ci = (int64_t)__ldcg(a.part + (int64_t)c * ps + 2 + l);
        if (cb > gb || (cb == gb && ci < gi)) { gb = cb; gi = ci; }
      }
      s_scal[0] = __ldcg(vsrc + gi) < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    sign = s_scal[0];
  }

  // ---- write v_l and the Rayleigh quotient v^T G64 v (upper triangle)
  const double fs = sign * vscale;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += PT) a.x[i] = __ldcg(vsrc + i) * fs;
  double q = 0.0;
  if (status != 2) {
    for (int64_t i = r0 + warp; i < r1; i += nwarps) {
      const double *g = a.G64 + i * n;
      double t = 0.0;
      for (int64_t j = i + lane; j < n; j += 32) {
        const double gv = __ldg(g + j) * __ldcg(vsrc + j);
        t += (j == i) ? gv : 2.0 * gv;
      }
      t = warp_sum(t);
      if (lane == 0) q += t * __ldcg(vsrc + i);
    }
    q *= vscale * vscale;
  }
  q = block_sum(q, red);
  if (threadIdx.x == 0) mypart[3 + l] = q;
  if (!grid_barrier(a.bar, a.err)) return;
  if (blockIdx.x == 0) {
    const double tq = reduce_partials(a.part, ps, 3 + l, red);
    if (threadIdx.x == 0) {
      *a.out_sigma2 = status == 2 ? 0.0 : fmax(tq, 0.0);
      a.info[0] = it;
      a.info[1] = status;
      a.info[2] = 0;
    }
  }
}

__global__ void symmetrize_kernel(int64_t n, const double *__restrict__ G64, float *__restrict__ G32) {
  // 32 x 32 tiles: G32[i][j] = G64[min(i,j)][max(i,j)]
  __shared__ float t[32][33];
  const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (bj >= bi) {
    // tile in the upper triangle: direct copy (row i <= col j) and mirrored copy
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = bi + r, j = bj + tx;
      float v = 0.f;
      if (i < n && j < n) v = (float)(j >= i ? G64[i * n + j] : G64[j * n + i]);
      t[r][tx] = v;
      if (i < n && j < n) G32[i * n + j] = v;
    }
    __syncthreads();
    if (bj != bi) {
      for (int r = ty; r < 32; r += 8) {
        const int64_t i = bj + r, j = bi + tx;  // mirrored tile
        if (i < n && j < n) G32[i * n + j] = t[tx][r];
      }
    }
  }
}

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c, k0, k1);
  }
}

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void start_draws_kernel(uint32_t k0, uint32_t k1, uint32_t lword, int64_t n, double *x) {
  const int64_t pairs = (n + 1) / 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), lword, 0x54535644u};
    philox10(c, k0, k1);
    const uint64_t a = ((uint64_t)c[0] << 32) | c[1];
    const uint64_t b = ((uint64_t)c[2] << 32) | c[3];
    const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(b >> 11) * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    x[2 * p] = rad * cs;
    if (2 * p + 1 < n) x[2 * p + 1] = rad * sn;
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

size_t power_scratch_bytes(int64_t n, int64_t l) {
  const size_t ps = (size_t)round_up(l + 8, 4);
  return 256 + 2 * (size_t)round_up(n, 32) * sizeof(double) + (size_t)kMaxPowerBlocks * ps * sizeof(double);
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
  static thread_local size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    TSVD_CUDA(cudaFuncSetAttribute(power_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    configured = smem;
  }
  int per_sm = 0;
  TSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, power_dense_kernel, PT, smem));
  if (per_sm < 1) return TSVD_EUNSUPPORTED;
  int64_t grid = std::min<int64_t>({(int64_t)di.sms * per_sm, ceil_div(n, 32), kMaxPowerBlocks});
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
  a.wb0 = reinterpret_cast<double *>(s + 256);
  a.wb1 = a.wb0 + round_up(n, 32);
  a.part = a.wb1 + round_up(n, 32);
  a.ps = (int)round_up(l + 8, 4);
  a.rows_per_block = rows_per_block;
  TSVD_CUDA(cudaMemsetAsync(s, 0, 256, stream));
  void *args[] = {&a};
  TSVD_CUDA(cudaLaunchCooperativeKernel((void *)power_dense_kernel, dim3((unsigned)grid), dim3(PT),
                                        args, smem, stream));
  TSVD_LAUNCHED();
  // surface a barrier timeout in info[2]
  TSVD_CUDA(cudaMemcpyAsync(info + 2, a.err, sizeof(int), cudaMemcpyDeviceToDevice, stream));
  return TSVD_OK;
}

tsvd_status launch_symmetrize(int64_t n, const double *G64, float *G32, cudaStream_t stream) {
  const int64_t nb = ceil_div(n, 32);
  dim3 grid((unsigned)nb, (unsigned)nb), block(32, 8);
  symmetrize_kernel<<<grid, block, 0, stream>>>(n, G64, G32);
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
// device address is looked up once per device with cudaGetSymbolAddress.
constexpr int64_t kNoallocScratchBytes =
    256 + 2 * TSVD_NOALLOC_MAX_N * 8 + (int64_t)kMaxPowerBlocks * ((TSVD_NOALLOC_MAX_L + 8 + 3) / 4 * 4) * 8;
static __device__ __align__(256) unsigned char g_power_noalloc_scratch[kNoallocScratchBytes];

static tsvd_status noalloc_scratch(void **out) {
  static std::mutex mu;
  static void *addr[128] = {};
  int dev = -1;
  TSVD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return TSVD_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    TSVD_CUDA(cudaGetSymbolAddress(&p, g_power_noalloc_scratch));
    if (!p) return TSVD_ECUDA;
    addr[dev] = p;
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
