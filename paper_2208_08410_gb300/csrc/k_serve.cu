// Grouped kernels of the t-SVD server: many small requests per launch.
//
// Grouped SYRK (the Gram step of Alg. 2, B = X^T X, for every request of a
// wave at once; G = A A^T for wide requests, Eq. 3).  One CTA per 64 x 64
// tile of one request's lower triangle, over that request's whole K range:
// 32-row slabs of both operand blocks go through shared memory, each thread
// keeps a 4 x 4 block of FP32 sums, and every 512 rows the FP32 sums are
// added into FP64 registers.  No atomics, so a request's Gram does not depend
// on what else is in the wave.  The epilogue writes the tile and its mirror
// into the FP64 matrix and its FP32 copy.
//
// Grouped power (Alg. 1 with Alg. 2 for each triplet, Hotelling
// deflation).  One thread-block cluster per request; CTA c of C owns rows
// [c R, (c+1) R) of G (R = ceil(d / C)), kept in shared memory when they fit.
// An iteration: w = G32 v for the CTA's rows (FP32 products, error-free FP32
// row sums), the rows of w stored into every CTA's next-iterate buffer and
// the CTA's partial ||w||^2, v.w, v.v (pairs of FP32 numbers, ~48 bits, since
// the FP64 pipe of this part is narrow) into every CTA's partial slots through
// distributed shared memory, one cluster barrier, then every CTA adds the C
// partials in rank order and takes the same decision (FP64).  The iterate is
// normalised inside the next product (w = s G r for the stored r), so one
// application has one cluster barrier and two block barriers.  After the loop every
// CTA holds the whole v_l.  The CTA's rows of the FP64 Gram are kept deflated
// (Hotelling, in FP64) and its rows of the FP32 copy are rounded from them,
// so the copy's rounding error is relative to the spectrum that remains;
// sigma_l^2 = v_l^T G v_l is formed as v_l^T G_defl v_l + sum_{j<l}
// sigma_j^2 (v_j . v_l)^2 from row partials (one more exchange).
//
// After the k triplets the same cluster forms the other factor (Alg. 1:
// U = A V Sigma^-1 for tall requests, V = A^T U Sigma^-1
// for wide ones), writes U, sigma, V and the per-triplet info into the
// request's output region and raises its completion flag (a release store
// into the server's device flag array, which the server copies to the host),
// so a request completes as soon as its own cluster finishes.
#include "philox.cuh"
#include "serve.cuh"

namespace tsvd {
namespace {

// ---------------------------------------------------------------- grouped SYRK
__global__ void __launch_bounds__(256) srv_syrk_kernel(const SrvReq *__restrict__ reqs,
                                                       const SrvTile *__restrict__ tiles) {
  __shared__ __align__(16) float sI[32][kSrvTile + 4];
  __shared__ __align__(16) float sJ[32][kSrvTile + 4];
  const SrvTile t = tiles[blockIdx.x];
  const SrvReq &q = reqs[t.req];
  const float *__restrict__ A = q.A;
  const int64_t ld = q.n;
  const bool tr = q.trans != 0;
  const int64_t d = tr ? q.m : q.n, K = tr ? q.n : q.m;
  const int64_t i0 = (int64_t)t.ti * kSrvTile, j0 = (int64_t)t.tj * kSrvTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = 0.f;
      accd[a][b] = 0.0;
    }
  int slabs = 0;
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + 256 * u;  // 0 .. 2047
      // tall: element (kk, ii) is A[k0 + kk][i0 + ii] (coalesced along ii);
      // wide: it is A[i0 + ii][k0 + kk] (coalesced along kk)
      const int kk = tr ? (e & 31) : (e >> 6);
      const int ii = tr ? (e >> 5) : (e & 63);
      const int64_t gk = k0 + kk, gi = i0 + ii, gj = j0 + ii;
      float vi = 0.f, vj = 0.f;
      if (gk < K) {
        if (gi < d) vi = tr ? __ldg(A + gi * ld + gk) : __ldg(A + gk * ld + gi);
        if (gj < d) vj = tr ? __ldg(A + gj * ld + gk) : __ldg(A + gk * ld + gj);
      }
      sI[kk][ii] = vi;
      sJ[kk][ii] = vj;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float4 a = *reinterpret_cast<const float4 *>(&sI[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4 *>(&sJ[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
    }
    __syncthreads();
    if (++slabs == 16) {  // 512 rows of FP32 sums into FP64
      slabs = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          accd[a][b] += (double)acc[a][b];
          acc[a][b] = 0.f;
        }
    }
  }
  double *__restrict__ G64 = q.G64;
  float *__restrict__ G32 = q.G32;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
      if (i < d && j < d) {
        const double v = accd[a][b] + (double)acc[a][b];
        G64[i * d + j] = v;
        G32[i * d + j] = (float)v;
        if (t.ti != t.tj) {
          G64[j * d + i] = v;
          G32[j * d + i] = (float)v;
        }
      }
    }
}

// ---------------------------------------------------------------- cluster helpers
__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cta_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster arrives; release/acquire at cluster scope
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_peer_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Unevaluated FP32 pairs (h, l), value h + l: the FP64 pipe of this part is
// narrow, so the per-row sums of the power loop are kept as pairs on the FP32
// pipe.  a*b is split exactly into p + pe (FMA), h + p into s + e (two-sum), and
// the low part collects both errors, so a pair carries about 48 bits.
__device__ __forceinline__ void ff_add_prod(float &h, float &l, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  float s, e;
  two_sum(h, p, s, e);
  h = s;
  l = __fadd_rn(l, __fadd_rn(e, pe));
}
__device__ __forceinline__ void ff_add(float &h, float &l, float h2, float l2) {
  float s, e;
  two_sum(h, h2, s, e);
  h = s;
  l = __fadd_rn(l, __fadd_rn(e, l2));
}
__device__ __forceinline__ double ff_value(float h, float l) { return (double)h + (double)l; }

constexpr int kMaxCluster = 8;
static_assert(kSrvPowerThreads == 256 && kMaxCluster == 8, "the partial sums reduce over 8 lanes");

constexpr int kPartSlot = kSrvMaxK + 4;  // doubles per (parity, rank) slot

struct PowerSmem {
  float *vb[2];    // d (padded) each: the iterate, scaled in place at the start of an iteration
  double *part;    // [2][kMaxCluster][kPartSlot]
  double *xs;      // d: FP64 start draws, then v_l
  float *Gs;       // R x d rows of G32 (resident mode)
};

__device__ __forceinline__ int64_t pad4(int64_t x) { return (x + 3) & ~int64_t(3); }

// ---------------------------------------------------------------- grouped power
__global__ void __launch_bounds__(kSrvPowerThreads, 2) srv_power_kernel(const SrvReq *__restrict__ reqs,
                                                                       int n_reqs) {
  extern __shared__ __align__(16) unsigned char srv_smem[];
  __shared__ double wred[3 * (kSrvPowerThreads / 32)];
  __shared__ double red[33];
  __shared__ double s_scal[4];
  __shared__ double s2hist[kSrvMaxK];   // sigma_j^2 of the triplets found so far
  __shared__ __align__(16) float ostage[kSrvOtherChunk * kSrvMaxK];  // other factor: a chunk of V or U
  __shared__ double cpart[kSrvMaxK + 1];  // this CTA's v^T G_defl v and v_j . v partials
  const uint32_t C = cta_count(), rank = cta_rank();
  // self-checks of the launch (every CTA of a cluster takes the same branch): a cluster
  // past the descriptors has nothing to do; a request whose descriptor names another
  // cluster size than the launch has is failed, not run on a wrong partition of its rows
  if (blockIdx.x / C >= (unsigned)n_reqs) return;
  const SrvReq &q = reqs[blockIdx.x / C];
  const int64_t d = q.trans ? q.m : q.n;
  const int k = q.k;
  const int64_t R = srv_rows_per_cta(d, C);  // a multiple of 4, so every CTA's row range starts 16-byte aligned
  const int64_t r0 = min(d, (int64_t)rank * R), r1 = min(d, r0 + R);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = kSrvPowerThreads / 32;
  if (q.cluster != (int32_t)C || (q.gram_err && *reinterpret_cast<const volatile int32_t *>(q.gram_err) != 0)) {
    // the tensor-core SYRK that formed this request's G gave up on a bounded wait (or the
    // launch's cluster size is not the descriptor's): no results; every triplet reports
    // the failure (every CTA reads the same words, written before this launch, so the
    // whole cluster takes this branch)
    if (rank == 0) {
      for (int l = threadIdx.x; l < k; l += kSrvPowerThreads) {
        q.oS[l] = 0.0;
        q.oInfo[4 * l] = 0;
        q.oInfo[4 * l + 1] = 0;
        q.oInfo[4 * l + 2] = 1;
        q.oInfo[4 * l + 3] = 0;
      }
    }
    __threadfence_system();
    cluster_sync_all();
    if (rank == 0 && threadIdx.x == 0)
      asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(q.flag), "r"(q.ticket) : "memory");
    return;
  }
  const int64_t dp = pad4(d);
  PowerSmem sm;
  sm.vb[0] = reinterpret_cast<float *>(srv_smem);
  sm.vb[1] = sm.vb[0] + dp;
  sm.part = reinterpret_cast<double *>(sm.vb[1] + dp);
  sm.xs = sm.part + 2 * kMaxCluster * kPartSlot;
  sm.Gs = reinterpret_cast<float *>(sm.xs + dp);
  const bool res = q.resident != 0;
  float *Grow0 = res ? sm.Gs : q.G32 + r0 * d;  // row r of this CTA at Grow0 + (r - r0) * d
  if (res) {
    for (int64_t e = threadIdx.x; e < (r1 - r0) * d; e += kSrvPowerThreads) sm.Gs[e] = q.G32[r0 * d + e];
  }
  // pw = 2^-E, 2^E the largest diagonal entry of G (every CTA forms the same power
  // of two): the stored iterates are r = pw G v, whose entries stay below 2 d, so
  // the products G_ij r_j stay inside the FP32 range up to max G_ii of about 1e31;
  // the pair sums take qs r (qs = 2^20), whose squares stay inside it down to
  // about 1e-25 max G_ii.  Scaling by powers of two is exact.
  float gmax = 0.f;
  for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) gmax = fmaxf(gmax, fabsf(q.G32[i * d + i]));
  {
    float *fred = reinterpret_cast<float *>(wred);
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if (lane == 0) fred[warp] = gmax;
    __syncthreads();
    gmax = fred[0];
    for (int w = 1; w < nwarps; ++w) gmax = fmaxf(gmax, fred[w]);
    __syncthreads();
  }
  int shift = 0;
  if (gmax > 0.f && gmax < INFINITY) shift = -ilogbf(gmax);
  shift = max(-126, min(126, shift));
  const float pw = __int_as_float((shift + 127) << 23);
  constexpr float qs = 1048576.f;  // 2^20
  const double pq2 = (double)pw * (double)pw * (double)qs * (double)qs;
  // every CTA of the cluster is running before any of them stores into another's
  // shared memory
  cluster_sync_all();
  uint32_t phase = 0;  // running count of cluster exchanges (selects the partial slots)
  const bool vec = (d % 4) == 0;
  double sig0sq = 1.0;  // sigma_0^2 (every CTA forms the same value)

  for (int l = 0; l < k; ++l) {
    // ---- start vector x ~ N(0,1)^d (every CTA draws all of it), v0 = x / ||x||
    if (q.x_start) {
      for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.xs[i] = q.x_start[(int64_t)l * d + i];
    } else {
      for (int64_t p = threadIdx.x; p < (d + 1) / 2; p += kSrvPowerThreads) {
        double z0, z1;
        start_normal_pair(q.key0, q.key1, (uint32_t)l, p, &z0, &z1);
        sm.xs[2 * p] = z0;
        if (2 * p + 1 < d) sm.xs[2 * p + 1] = z1;
      }
    }
    __syncthreads();
    double xx = 0.0;
    for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) xx += sm.xs[i] * sm.xs[i];
    xx = block_sum(xx, red);
    const double inv = xx > 0.0 ? 1.0 / sqrt(xx) : 0.0;
    for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.vb[0][i] = (float)(sm.xs[i] * inv);
    const double rank_scale = l == 0 ? 1.0 : sig0sq;
    const double floor_s = 1e-30 * rank_scale * 1e-30 * rank_scale * pq2;  // floor^2 in the units of the sums
    int cur = 0, it = 0, status = 0;
    // vb[cur] holds the raw iterate r (pw G v of the previous application; x / ||x||
    // at first) and v = sc r is the unit iterate of this one: pw G v is formed as
    // pw sc (G r), so no pass over the iterate is needed to normalise it
    float sc = 1.f;
    double vscale = 1.0;  // on exit: v_l = vscale * vb[cur]
    __syncthreads();
    for (;;) {
      const float *v = sm.vb[cur];
      float *nxt = sm.vb[cur ^ 1];
      float wwh = 0.f, wwl = 0.f, vwh = 0.f, vwl = 0.f, vvh = 0.f, vvl = 0.f;
      // four rows per warp step (r0 and R are multiples of 4): four independent
      // dot products and warp reductions in flight; rows past r1 repeat the
      // last row and are dropped
      for (int64_t rb = r0 + 4 * warp; rb < r1; rb += 4 * nwarps) {
        const int nr = (int)min((int64_t)4, r1 - rb);
        const float *g[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) g[u] = Grow0 + (min(rb + u, r1 - 1) - r0) * d;
        float p[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u][0] = p[u][1] = p[u][2] = p[u][3] = 0.f;
        if (vec) {
          const float4 *v4 = reinterpret_cast<const float4 *>(v);
          for (int64_t c = lane; c < d / 4; c += 32) {
            const float4 b = v4[c];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 a = reinterpret_cast<const float4 *>(g[u])[c];
              p[u][0] = fmaf(a.x, b.x, p[u][0]);
              p[u][1] = fmaf(a.y, b.y, p[u][1]);
              p[u][2] = fmaf(a.z, b.z, p[u][2]);
              p[u][3] = fmaf(a.w, b.w, p[u][3]);
            }
          }
        } else {
          for (int64_t c = lane; c < d; c += 32) {
            const float b = v[c];
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u][0] = fmaf(g[u][c], b, p[u][0]);
          }
        }
        float h[4], e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float sa, ea, sb, eb;
          two_sum(p[u][0], p[u][1], sa, ea);
          two_sum(p[u][2], p[u][3], sb, eb);
          two_sum(sa, sb, h[u], e[u]);
          e[u] += ea + eb;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float ho = __shfl_xor_sync(0xffffffffu, h[u], o);
            const float lo2 = __shfl_xor_sync(0xffffffffu, e[u], o);
            float sx, ex;
            two_sum(h[u], ho, sx, ex);
            h[u] = sx;
            e[u] = e[u] + lo2 + ex;
          }
        }
        // every lane holds the four sums; lane u finishes row rb + u: the stored entry
        // is pw times the FP32 rounding of sc (h + e), and the pair sums use exactly
        // the stored entry and v_r
        if (lane < nr) {
          float hu = h[0], eu = e[0];
#pragma unroll
          for (int u = 1; u < 4; ++u) {
            if (lane == u) {
              hu = h[u];
              eu = e[u];
            }
          }
          const float rr = __fmul_rn(__fmul_rn(__fadd_rn(hu, eu), sc), pw);
          const float ts = __fmul_rn(rr, qs);
          const float vr = __fmul_rn(v[rb + lane], sc);
          ff_add_prod(wwh, wwl, ts, ts);
          ff_add_prod(vwh, vwl, vr, ts);
          ff_add_prod(vvh, vvl, vr, vr);
          nxt[rb + lane] = rr;
        }
      }
      // lanes 0..3 hold the warp's partial sums
#pragma unroll
      for (int o = 2; o > 0; o >>= 1) {
        const float a0 = __shfl_xor_sync(0xffffffffu, wwh, o), a1 = __shfl_xor_sync(0xffffffffu, wwl, o);
        const float b0 = __shfl_xor_sync(0xffffffffu, vwh, o), b1 = __shfl_xor_sync(0xffffffffu, vwl, o);
        const float c0 = __shfl_xor_sync(0xffffffffu, vvh, o), c1 = __shfl_xor_sync(0xffffffffu, vvl, o);
        ff_add(wwh, wwl, a0, a1);
        ff_add(vwh, vwl, b0, b1);
        ff_add(vvh, vvl, c0, c1);
      }
      if (lane == 0) {
        float *wr = reinterpret_cast<float *>(wred) + 6 * warp;
        wr[0] = wwh;
        wr[1] = wwl;
        wr[2] = vwh;
        wr[3] = vwl;
        wr[4] = vvh;
        wr[5] = vvl;
      }
      __syncthreads();
      // this CTA's rows of w into the same place of every other CTA's next iterate
      if (C > 1) {
        const uint32_t base = smem_addr(nxt + r0);
        const int64_t n4 = (r1 - r0 + 3) / 4;  // r0 is a multiple of 4; the tail stays inside the padding
        for (int64_t e = threadIdx.x; e < n4 * (C - 1); e += kSrvPowerThreads) {
          const uint32_t c = (uint32_t)(e / n4);
          const uint32_t peer = c >= rank ? c + 1 : c;
          const int64_t q4 = e % n4;
          const float4 x = reinterpret_cast<const float4 *>(nxt + r0)[q4];
          const uint32_t pa = peer_addr(base + 16 * (uint32_t)q4, peer);
          asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(pa), "f"(x.x), "f"(x.y), "f"(x.z),
                       "f"(x.w)
                       : "memory");
        }
      }
      const int par = (int)(phase & 1u);
      if (warp == 0) {
        // the warps' pairs, summed over lanes 0..7 (xor tree: every lane ends with the
        // sums), then lane c stores them into CTA c's slot for this rank
        float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (lane < nwarps) {
          const float *wr = reinterpret_cast<const float *>(wred) + 6 * lane;
#pragma unroll
          for (int t = 0; t < 6; ++t) x[t] = wr[t];
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          float y[6];
#pragma unroll
          for (int t = 0; t < 6; ++t) y[t] = __shfl_xor_sync(0xffffffffu, x[t], o);
#pragma unroll
          for (int t = 0; t < 6; t += 2) ff_add(x[t], x[t + 1], y[t], y[t + 1]);
        }
        if (lane < (int)C) {
          const uint32_t pa = peer_addr(smem_addr(sm.part + (par * kMaxCluster + rank) * kPartSlot), (uint32_t)lane);
          asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(pa), "f"(x[0]), "f"(x[1]) : "memory");
          asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(pa + 8), "f"(x[2]), "f"(x[3]) : "memory");
          asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(pa + 16), "f"(x[4]), "f"(x[5]) : "memory");
        }
      }
      cluster_sync_all();
      ++phase;
      if (warp == 0) {
        // the C ranks' pairs, same xor tree in every CTA, so all take the same decision
        float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (lane < (int)C) {
          const float *ps = reinterpret_cast<const float *>(sm.part + (par * kMaxCluster + lane) * kPartSlot);
#pragma unroll
          for (int t = 0; t < 6; ++t) x[t] = ps[t];
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          float y[6];
#pragma unroll
          for (int t = 0; t < 6; ++t) y[t] = __shfl_xor_sync(0xffffffffu, x[t], o);
#pragma unroll
          for (int t = 0; t < 6; t += 2) ff_add(x[t], x[t + 1], y[t], y[t + 1]);
        }
        if (lane == 0) {
          // t0 = ||r||^2 qs^2, t1 = (v.r) qs, t2 = v.v for the new r = pw w
          const double t0 = ff_value(x[0], x[1]), t1 = ff_value(x[2], x[3]), t2 = ff_value(x[4], x[5]);
          const int it1 = it + 1;
          int st = 0, done = 0;
          float scn = 0.f;
          double vs = 0.0;
          if (!(t0 > floor_s)) {  // ||w|| <= floor: B v0 vanished
            st = 2;
            done = 1;
          } else {
            // 1 / ||r|| = qs / sqrt(t0): FP32 for the next application (its scale only),
            // FP64 on exit
            scn = x[0] > 1e-30f ? __fmul_rn(rsqrtf(x[0]), qs) : (float)((double)qs / sqrt(t0));
            if (q.iters_override) {
              done = it1 >= q.iters_override[l];
            } else {
              // |v . w| / (||v|| ||w||) >= 1 - eps, squared: both sides are non-negative
              const double c1 = 1.0 - q.eps;
              done = t1 * t1 >= c1 * c1 * t0 * t2;
              if (!done && it1 >= q.max_iter) {
                done = 1;
                st = 1;
              }
            }
            if (done) vs = (double)qs / sqrt(t0);
          }
          s_scal[0] = vs;
          s_scal[1] = (double)st;
          s_scal[2] = (double)done;
          s_scal[3] = (double)scn;
        }
      }
      __syncthreads();
      ++it;
      const int st = (int)s_scal[1];
      const bool done = s_scal[2] != 0.0;
      if (st == 2) {
        status = 2;  // vb[cur] still holds the raw iterate of this step
        break;
      }
      sc = (float)s_scal[3];
      cur ^= 1;
      if (done) {
        vscale = s_scal[0];
        status = st;
        break;
      }
    }
    // ---- v_l (FP64, whole vector, every CTA)
    __syncthreads();
    if (status == 2) {
      for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.xs[i] = (double)sm.vb[cur][i];
      for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < l; ++j) {
          const double *vj = q.V64 + (int64_t)j * d;
          double c = 0.0;
          for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) c += vj[i] * sm.xs[i];
          c = block_sum(c, red);
          for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.xs[i] -= c * vj[i];
          __syncthreads();
        }
        double nn = 0.0;
        for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) nn += sm.xs[i] * sm.xs[i];
        nn = block_sum(nn, red);
        const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.xs[i] *= sc;
        __syncthreads();
      }
    } else {
      for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.xs[i] = (double)sm.vb[cur][i] * vscale;
    }
    __syncthreads();
    if (q.sign_convention) {
      // largest |v_i| positive, lowest index on ties (same scan in every CTA)
      if (threadIdx.x == 0) {
        double best = -1.0;
        int64_t bi = 0;
        for (int64_t i = 0; i < d; ++i) {
          const double a = fabs(sm.xs[i]);
          if (a > best) {
            best = a;
            bi = i;
          }
        }
        s_scal[3] = sm.xs[bi] < 0.0 ? -1.0 : 1.0;
      }
      __syncthreads();
      const double sg = s_scal[3];
      for (int64_t i = threadIdx.x; i < d; i += kSrvPowerThreads) sm.xs[i] *= sg;
      __syncthreads();
    }
    // ---- sigma_l^2 = v^T G_defl v + sum_{j<l} sigma_j^2 (v_j . v)^2 from this
    // CTA's rows, exchanged like the partials
    double qv = 0.0;
    if (status != 2) {
      for (int64_t r = r0 + warp; r < r1; r += nwarps) {
        const double *g = q.G64 + r * d;
        double t = 0.0;
        for (int64_t c = lane; c < d; c += 32) t += g[c] * sm.xs[c];
        t = warp_sum(t);
        if (lane == 0) qv += t * sm.xs[r];
      }
      for (int j = warp; j < l; j += nwarps) {
        const double *vj = q.V64 + (int64_t)j * d;  // rows this CTA wrote itself
        double t = 0.0;
        for (int64_t r = r0 + lane; r < r1; r += 32) t += vj[r] * sm.xs[r];
        t = warp_sum(t);
        if (lane == 0) cpart[1 + j] = t;
      }
    }
    qv = block_sum(qv, red);
    if (threadIdx.x == 0) cpart[0] = qv;
    __syncthreads();
    const int par = (int)(phase & 1u);
    const int ncp = status == 2 ? 1 : l + 1;
    if (threadIdx.x < (unsigned)ncp) {
      const uint32_t slot = smem_addr(sm.part + (par * kMaxCluster + rank) * kPartSlot + threadIdx.x);
      for (uint32_t c = 0; c < C; ++c) st_peer_f64(peer_addr(slot, c), cpart[threadIdx.x]);
    }
    cluster_sync_all();
    ++phase;
    double s2 = 0.0;
    for (uint32_t c = 0; c < C; ++c) s2 += sm.part[(par * kMaxCluster + c) * kPartSlot];
    if (status != 2) {
      for (int j = 0; j < l; ++j) {
        double cj = 0.0;
        for (uint32_t c = 0; c < C; ++c) cj += sm.part[(par * kMaxCluster + c) * kPartSlot + 1 + j];
        s2 += s2hist[j] * cj * cj;
      }
    }
    s2 = status == 2 ? 0.0 : fmax(s2, 0.0);
    if (l == 0) sig0sq = s2;
    __syncthreads();
    if (threadIdx.x == 0) s2hist[l] = s2;
    // ---- outputs of triplet l (each CTA its rows; rank 0 the scalars)
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kSrvPowerThreads) {
      q.V64[(int64_t)l * d + r] = sm.xs[r];
      q.vout[(int64_t)l * d + r] = (float)sm.xs[r];
    }
    if (rank == 0 && threadIdx.x == 0) {
      q.sig2[l] = s2;
      q.info[4 * l] = it;
      q.info[4 * l + 1] = status;
      q.info[4 * l + 2] = 0;
      q.info[4 * l + 3] = 0;
    }
    // ---- Hotelling deflation of this CTA's rows: FP64 Gram in FP64, FP32 copy rounded from it
    if (l + 1 < k && status != 2) {
      for (int64_t r = r0 + warp; r < r1; r += nwarps) {
        double *g64 = q.G64 + r * d;
        float *g32 = Grow0 + (r - r0) * d;
        const double cr = s2 * sm.xs[r];
        for (int64_t c = lane; c < d; c += 32) {
          const double g = fma(-cr, sm.xs[c], g64[c]);
          g64[c] = g;
          g32[c] = (float)g;
        }
      }
    }
    __syncthreads();
  }

  // ---- other factor (Alg. 1) for this request, split over the cluster
  cluster_sync_all();  // every CTA's rows of vout are written
  const int64_t m = q.m, n = q.n;
  const float *__restrict__ A = q.A;
  if (q.no_other) {
    // the caller forms the other factor itself
  } else if (!q.trans) {
    // U[r][l] = sum_j A[r][j] V[j][l] / sigma_l; this CTA's rows of U, one row per warp at a time,
    // V staged in chunks of kSrvOtherChunk rows (l-major) in shared memory
    const int64_t Rm = (m + C - 1) / C;
    const int64_t u0 = min(m, (int64_t)rank * Rm), u1 = min(m, u0 + Rm);
    for (int64_t rb = u0; rb < u1; rb += nwarps) {
      const int64_t r = rb + warp;
      float acc[kSrvMaxK];
#pragma unroll
      for (int l = 0; l < kSrvMaxK; ++l) acc[l] = 0.f;
      for (int64_t j0 = 0; j0 < n; j0 += kSrvOtherChunk) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSrvOtherChunk * kSrvMaxK; e += kSrvPowerThreads) {
          const int l = e / kSrvOtherChunk, jj = e % kSrvOtherChunk;
          ostage[e] = (j0 + jj < n && l < k) ? q.vout[(int64_t)l * n + j0 + jj] : 0.f;
        }
        __syncthreads();
        if (r < u1) {
          for (int jj = lane; jj < kSrvOtherChunk; jj += 32) {
            const float x = (j0 + jj < n) ? __ldg(A + r * n + j0 + jj) : 0.f;
#pragma unroll
            for (int l = 0; l < kSrvMaxK; ++l) acc[l] = fmaf(x, ostage[l * kSrvOtherChunk + jj], acc[l]);
          }
        }
      }
      float mine = 0.f;
#pragma unroll
      for (int l = 0; l < kSrvMaxK; ++l) {
        const float t = warp_sumf(acc[l]);
        mine = (lane == l) ? t : mine;
      }
      if (r < u1 && lane < k) {
        const double sg = s2hist[lane];
        q.oU[(int64_t)lane * m + r] = sg > 0.0 ? (float)((double)mine / sqrt(sg)) : 0.f;
      }
    }
  } else {
    // V[j][l] = sum_r A[r][j] U[r][l] / sigma_l; this CTA's columns of V, one per thread,
    // U staged in chunks of kSrvOtherChunk rows (row-major) in shared memory
    const int64_t Rn = (n + C - 1) / C;
    const int64_t c0 = min(n, (int64_t)rank * Rn), c1 = min(n, c0 + Rn);
    for (int64_t jb = c0; jb < c1; jb += kSrvPowerThreads) {
      const int64_t j = jb + threadIdx.x;
      float acc[kSrvMaxK];
#pragma unroll
      for (int l = 0; l < kSrvMaxK; ++l) acc[l] = 0.f;
      for (int64_t rb = 0; rb < m; rb += kSrvOtherChunk) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSrvOtherChunk * kSrvMaxK; e += kSrvPowerThreads) {
          const int rr = e / kSrvMaxK, l = e % kSrvMaxK;
          ostage[e] = (rb + rr < m && l < k) ? q.vout[(int64_t)l * m + rb + rr] : 0.f;
        }
        __syncthreads();
        const int64_t rn = min((int64_t)kSrvOtherChunk, m - rb);
        if (j < c1) {
          for (int64_t rr = 0; rr < rn; ++rr) {
            const float x = __ldg(A + (rb + rr) * n + j);
            const float *ur = ostage + rr * kSrvMaxK;  // same address across the warp
#pragma unroll
            for (int l = 0; l < kSrvMaxK; ++l) acc[l] = fmaf(x, ur[l], acc[l]);
          }
        }
      }
      if (j < c1) {
#pragma unroll
        for (int l = 0; l < kSrvMaxK; ++l) {
          if (l < k) {
            const double sg = s2hist[l];
            q.oV[(int64_t)l * n + j] = sg > 0.0 ? (float)((double)acc[l] / sqrt(sg)) : 0.f;
          }
        }
      }
    }
  }
  // the power vectors (this CTA's rows) and, from rank 0, sigma and the per-triplet info
  float *ovec = q.trans ? q.oU : q.oV;
  for (int l = 0; l < k; ++l)
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kSrvPowerThreads) ovec[(int64_t)l * d + r] = q.vout[(int64_t)l * d + r];
  if (rank == 0) {
    for (int l = threadIdx.x; l < k; l += kSrvPowerThreads) {
      q.oS[l] = sqrt(s2hist[l]);
      for (int t = 0; t < 4; ++t) q.oInfo[4 * l + t] = q.info[4 * l + t];
    }
  }
  __threadfence_system();
  cluster_sync_all();
  if (rank == 0 && threadIdx.x == 0) {
    __threadfence_system();
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(q.flag), "r"(q.ticket) : "memory");
  }
}

}  // namespace

size_t srv_power_smem(int64_t d, int cluster, int resident) {
  const int64_t dp = (d + 3) & ~int64_t(3);
  size_t b = 2 * dp * 4 + 2 * kMaxCluster * kPartSlot * 8 + dp * 8;
  if (resident) b += (size_t)srv_rows_per_cta(d, cluster) * d * 4;
  return b;
}

tsvd_status launch_srv_syrk(const SrvReq *reqs, const SrvTile *tiles, int n_tiles, cudaStream_t stream) {
  if (n_tiles <= 0) return TSVD_OK;
  srv_syrk_kernel<<<n_tiles, 256, 0, stream>>>(reqs, tiles);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_srv_power(const SrvReq *reqs, int n_reqs, int cluster, size_t smem, cudaStream_t stream) {
  if (n_reqs <= 0) return TSVD_OK;
  if (cluster < 1 || cluster > kMaxCluster || (cluster & (cluster - 1))) return TSVD_EINVAL;
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  if (smem > di.smem_optin) return TSVD_EINVAL;
  // the kernel's static arrays (~17 KB) count toward the 48 KB a launch gets without
  // opting in, so the attribute is raised for any size above what is already allowed
  cudaFuncAttributes fa;
  TSVD_CUDA(cudaFuncGetAttributes(&fa, srv_power_kernel));
  if (fa.sharedSizeBytes + smem > di.smem_optin) return TSVD_EINVAL;
  TSVD_TRY(ensure_dynamic_smem(reinterpret_cast<const void *>(srv_power_kernel), smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_reqs * cluster));
  cfg.blockDim = dim3(kSrvPowerThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TSVD_CUDA(cudaLaunchKernelEx(&cfg, srv_power_kernel, reqs, n_reqs));
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
