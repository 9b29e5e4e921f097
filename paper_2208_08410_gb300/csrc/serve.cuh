// Grouped kernels of the t-SVD server (internal header).
//
// A wave of requests runs as three grouped launches, each over all requests of
// the wave at once:
//   1. grouped SYRK: every 64 x 64 tile of every request's Gram matrix
//      (G = A^T A when m >= n, G = A A^T when m < n: Eq. 3), written as the
//      symmetric FP64 matrix and its FP32 copy;
//   2. grouped power: one thread-block cluster per request runs Alg. 1/2 for
//      all k triplets (Hotelling deflation of the FP32 copy, FP64 Rayleigh
//      quotient and convergence test);
//      then, in the same cluster, the other factor: U = A V Sigma^-1 (m >= n)
//      or V = A^T U Sigma^-1 (m < n), Alg. 1; the cluster
//      writes U, sigma, V and the per-triplet info into the request's output
//      region in device memory and then raises the request's completion flag
//      (a word of a device array the server polls), so each request
//      completes on its own.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace tsvd {

// One request as the device sees it (all pointers are device memory).
struct SrvReq {
  const float *A;    // m x n, row-major, row stride n
  int64_t m, n;
  int32_t trans;     // 0: d = n, G = A^T A;  1: d = m, G = A A^T
  int32_t k;
  double *G64;       // d x d, full symmetric, row-major
  float *G32;        // d x d FP32 copy (deflated in place triplet by triplet)
  double *V64;       // d x k column-major: the power method's vectors
  double *sig2;      // k
  int32_t *info;     // 4 per triplet: applications, status (0 ok, 1 no convergence, 2 rank), 0, 0
  float *vout;       // d x k column-major FP32 copy of V64
  double eps;
  int32_t max_iter;
  int32_t sign_convention;
  const int32_t *iters_override;  // k applications per triplet (convergence test skipped), or null
  uint32_t key0, key1;  // Philox key of the start draws (splitmix64 of the seed)
  int32_t cluster;      // CTAs that run this request's power method (1, 2, 4, 8)
  int32_t resident;     // 1: the power kernel keeps the CTA's rows of G32 in shared memory
  // results in device memory, and the completion flag
  float *oU;            // m x k column-major
  float *oV;            // n x k column-major
  double *oS;           // k
  int32_t *oInfo;       // 4 k
  uint32_t *flag;       // set to `ticket` (release, gpu scope) once everything above is written
  uint32_t ticket;
  int32_t no_other;     // 1: skip the other factor (oU when m >= n); the power vectors, sigma and info are written
  const double *x_start;  // d x k column-major start draws used as x_l, or null (Philox draws of key0/key1);
                          // may alias V64: column l is read before the triplet's vector overwrites it
  const int32_t *gram_err;  // status word of the tensor-core SYRK that formed G (nonzero: a bounded wait
                            // gave up, G is not valid), or null for the CUDA-core SYRK
};

// One request of the grouped tensor-core SYRK (3xTF32): its operand At (d rows
// of Kp contraction indices, K-major, TF32 hi and lo parts) and its Gram
// matrix.  The SYRK stores each tile's entries (gi, gj), gj <= gi, at
// G64[gj d + gi]; the finish pass mirrors them and writes the FP32 copy.
struct SrvTcReq {
  int32_t req;       // index of the request in the wave's SrvReq array
  int32_t pad;
  int64_t d, K, Kp;  // Gram dimension, contraction length, K padded to a stage (32)
  float *hi, *lo;    // d x Kp each, 1024-byte aligned
  double *G64;
  float *G32;
};

// Work unit of the grouped tensor-core SYRK: one 128 x 256 tile (bi, bj),
// bj * 256 <= bi * 128 + 127, over the request's whole contraction range.
struct SrvTcUnit {
  int32_t tc, bi, bj, pad;  // tc: index into the SrvTcReq array
};

// Work item of the grouped SYRK: request, tile row, tile column (ti >= tj).
struct SrvTile {
  int32_t req, ti, tj, pad;
};

constexpr int kSrvTile = 64;         // SYRK tile edge
constexpr int kSrvMaxDim = 2048;     // largest d the cluster power kernel takes
constexpr int kSrvMaxK = 32;         // largest k
constexpr int kSrvPowerThreads = 256;
constexpr int kSrvOtherChunk = 128;   // rows of V (tall) or U (wide) staged per step of the other factor

// rows of G each CTA of a cluster owns: ceil(d / cluster) rounded up to 4
__host__ __device__ inline int64_t srv_rows_per_cta(int64_t d, int64_t cluster) {
  return ((d + cluster - 1) / cluster + 3) & ~int64_t(3);
}

// largest power-of-two cluster size <= c that leaves no CTA of the cluster without rows
__host__ __device__ inline int srv_clamp_cluster(int64_t d, int c) {
  while (c > 1 && srv_rows_per_cta(d, c) * (c - 1) >= d) c >>= 1;
  return c > 1 ? c : 1;
}

// Every pointer the grouped kernels dereference is set (host check before a
// launch; the kernels themselves do not test them).
inline bool srv_req_complete(const SrvReq &q) {
  if (!q.G64 || !q.G32 || !q.V64 || !q.sig2 || !q.info || !q.vout || !q.oS || !q.oInfo || !q.flag) return false;
  if (q.no_other) return q.trans ? q.oU != nullptr : q.oV != nullptr;  // the power vectors' copy
  return q.A && q.oU && q.oV;
}

// Dynamic shared memory of the power kernel for (d, cluster, resident).
size_t srv_power_smem(int64_t d, int cluster, int resident);

tsvd_status launch_srv_syrk(const SrvReq *reqs, const SrvTile *tiles, int n_tiles, cudaStream_t stream);

// Grouped tensor-core SYRK of the requests in `tcs` (device arrays): prep
// (round and split each A into its K-major hi / lo operand), the SYRK over
// `units` (maps: 2 per request, hi then lo, 64-byte aligned, device memory),
// then the finish pass (mirror, FP32 copy).  prep_start and fin_start are the
// n_tc + 1 prefix sums of each request's prep strips and finish tiles
// (srv_tc_prep_strips, srv_tc_finish_tiles).  err: the wave's status word,
// zeroed here.
constexpr int kSrvTcTM = 128, kSrvTcTN = 256, kSrvTcKStage = 32;
int64_t srv_tc_prep_strips(int64_t d, int64_t Kp);
int64_t srv_tc_finish_tiles(int64_t d);
int64_t srv_tc_tiles(int64_t d);  // 128 x 256 tiles touching the lower triangle
tsvd_status launch_srv_syrk_tc(const SrvReq *reqs, const SrvTcReq *tcs, int n_tc, const int64_t *prep_start,
                               int64_t n_prep, const int64_t *fin_start, int64_t n_fin, const CUtensorMap *maps,
                               const SrvTcUnit *units, int n_units, int32_t *err, cudaStream_t stream);
// All requests of one launch share the cluster size; `smem` covers the largest.
tsvd_status launch_srv_power(const SrvReq *reqs, int n_reqs, int cluster, size_t smem, cudaStream_t stream);

}  // namespace tsvd
