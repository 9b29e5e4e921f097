// Shared host/device helpers of the tsvd library (internal header).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "tsvd.h"

namespace tsvd {

// ---------------------------------------------------------------- host side
void set_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void set_error_text(const std::string &s);
// kernel launches made by this thread (counted at launch; a replayed graph adds its kernel nodes)
void count_launches(int64_t n);
// Raise `func`'s dynamic shared-memory limit on the current device to at least
// `bytes`.  The limit belongs to the process (every host thread sees it), so
// the record of what was set is process-wide and the limit only grows.
tsvd_status ensure_dynamic_smem(const void *func, size_t bytes);

// A failed call's error is also this thread's last error; it is read here
// (cudaGetLastError), so a later launch check does not report it again.
#define TSVD_CUDA(call)                                                         \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      (void)cudaGetLastError();                                                 \
      ::tsvd::set_cuda_error(e_, #call, __FILE__, __LINE__);                    \
      return TSVD_ECUDA;                                                        \
    }                                                                           \
  } while (0)

#define TSVD_LAUNCHED()                                                         \
  do {                                                                          \
    cudaError_t e_ = cudaGetLastError();                                        \
    if (e_ != cudaSuccess) {                                                    \
      ::tsvd::set_cuda_error(e_, "kernel launch", __FILE__, __LINE__);          \
      return TSVD_ECUDA;                                                        \
    }                                                                           \
    ::tsvd::count_launch();                                                     \
  } while (0)

#define TSVD_TRY(expr)                                                          \
  do {                                                                          \
    tsvd_status s_ = (expr);                                                    \
    if (s_ != TSVD_OK) return s_;                                               \
  } while (0)

// Per-thread count of kernels this library launched (reported per call).
void count_launch();
int64_t launches_so_far();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int cc_major = 0, cc_minor = 0;
  size_t smem_optin = 0;
  size_t l2_bytes = 0;
};
tsvd_status device_info(DeviceInfo *out);

// Page-locked host memory backed by transparent huge pages: an anonymous
// mapping aligned to the huge-page size, advised MADV_HUGEPAGE, touched, then
// registered with cudaHostRegister (portable).  Copy engines translate a
// large page-locked range through far fewer host page-table entries than with
// the base pages of cudaHostAlloc, which keeps block copies at the link rate
// while kernels run beside them.  pinned_free takes only pointers returned by
// pinned_alloc (TSVD_EINVAL otherwise).
tsvd_status pinned_alloc(void **ptr, size_t bytes);
tsvd_status pinned_free(void *ptr);

// ------------------------------------------------------------- device side
// A bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (all threads get the result).  `red` needs 33 doubles.
__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// gpu-scope acquire / release primitives for the grid barrier
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release_gpu(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch.  bar[0] counts arrivals, bar[1]
// is the generation.  Thread 0 of each block arrives with an acquire-release
// add (publishing the block's writes, which __syncthreads ordered before it);
// the last arrival resets the count and bumps the generation with a release;
// the others poll the generation with acquire loads.  Waits are bounded: past
// kWaitLimitNs, or when another block has raised *err, the waiter sets *err
// and returns false.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int *verr = err;
    const unsigned g = ld_acquire_gpu(bar + 1);
    const unsigned arrived = atom_add_acq_rel_gpu(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x * gridDim.y * gridDim.z - 1) {
      st_relaxed_gpu(bar, 0u);
      red_add_release_gpu(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_timer_ns();
      for (uint32_t spin = 0; ld_acquire_gpu(bar + 1) == g; ++spin) {
        if ((spin & 63u) == 63u) {
          if (*verr) { ok = 0; break; }
          if (global_timer_ns() - t0 > kWaitLimitNs) {
            atomicExch(err, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    if (*verr) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------ launchers
// Each returns TSVD_OK or an error; they only enqueue work on `stream`.
// ev0/ev1 (optional) are recorded on `stream` right around the Gram kernel.
tsvd_status launch_gram_simt(const float *A, int64_t rows, int64_t n, int64_t ld, double *G,
                             cudaStream_t stream, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
size_t gram_tc_scratch_bytes(int64_t rows, int64_t n, int precision);
// TMA map of a K-major tensor-core operand: n rows of Kp elements (TF32 in
// 32-bit words, or BF16), 1024-byte aligned base; box = one 128-byte swizzle
// row of K by 128 rows (64-byte aligned)
tsvd_status tc_make_map(CUtensorMap *map, const void *base, int64_t n, int64_t Kp, int precision);
// One task of the orthogonal batching (Sec. V-C): G[a][bs + b] += sum_r AJ[r][a] AI[r][b]
// for a < nJ, b < nI (panel J against panel I, both rows x n_* with stride ld);
// G is bs x 2 bs, row stride 2 bs.  Scratch: gram_tc_scratch_bytes(rows, 2 bs, precision).
tsvd_status launch_gram_tc_rect(const float *AJ, const float *AI, int64_t rows, int64_t bs, int64_t nJ, int64_t nI,
                                int64_t ld, double *G, int precision, void *scratch, size_t scratch_bytes,
                                cudaStream_t stream, bool reset_status);
// Gram of a transposed operand, G += X^T X with X[r][c] = A[c ld + r] (rows
// contraction indices, n outputs): a column block of a wide A, whose Gram is
// A A^T (Eq. 3).  Same storage of G as the row-major launchers.
tsvd_status launch_gram_simt_t(const float *A, int64_t rows, int64_t n, int64_t ld, double *G, cudaStream_t stream);
tsvd_status launch_gram_tc_t(const float *A, int64_t rows, int64_t n, int64_t ld, double *G, int precision,
                             void *scratch, size_t scratch_bytes, cudaStream_t stream, cudaEvent_t ev0 = nullptr,
                             cudaEvent_t ev1 = nullptr, bool reset_status = true, uint64_t wait_ns = 0);
// The same on CUDA cores (FP32): G[a][b] += sum_r AJ[r][a] AI[r][b], row stride ldg.
tsvd_status launch_gram_simt_rect(const float *AJ, const float *AI, int64_t rows, int64_t nJ, int64_t nI, int64_t ld,
                                  double *G, int64_t ldg, cudaStream_t stream);
// reset_status: zero the scratch's status word first (a caller that runs many
// chunks zeroes it once, so a timeout in any chunk stays visible).
// wait_ns: limit of the SYRK's pipeline waits, 0 = kWaitLimitNs (a shorter one
// only serves tests of the timeout path)
tsvd_status launch_gram_tc(const float *A, int64_t rows, int64_t n, int64_t ld, double *G,
                           int precision, void *scratch, size_t scratch_bytes, cudaStream_t stream,
                           cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, bool reset_status = true,
                           uint64_t wait_ns = 0);
// The two halves of launch_gram_tc: the prep (transpose, rounding, split) into
// the scratch, then the SYRK from it.
tsvd_status launch_gram_tc_prep(const float *A, int64_t rows, int64_t n, int64_t ld, int precision, void *scratch,
                                size_t scratch_bytes, cudaStream_t stream);
tsvd_status launch_gram_tc_syrk(int64_t rows, int64_t n, double *G, int precision, void *scratch,
                                size_t scratch_bytes, cudaStream_t stream, cudaEvent_t ev0 = nullptr,
                                cudaEvent_t ev1 = nullptr, bool reset_status = true, uint64_t wait_ns = 0);

// Tiled Gram operator (orthogonal batching): w_J += T v_I and, for an
// off-diagonal tile, w_I += T^T v_J (T: nJ x nI FP64, row stride ldt; a
// diagonal tile holds its upper triangle).  Then w = FP32(w64), ss += v . w64.
tsvd_status launch_tile_symv(const double *T, int64_t ldt, int64_t nJ, int64_t nI, const float *vJ, const float *vI,
                             double *wJ, double *wI, bool diag, cudaStream_t stream);
tsvd_status launch_tile_finish(int64_t n, const float *v, const double *w64, float *w, double *ss,
                               cudaStream_t stream);

// One triplet of the sparse power method (CSR on the device, whole matrix,
// rows m, columns n; l <= 32 earlier vectors in Vr, n x ldk row-major) in one
// cooperative launch of at most max_blocks blocks: buf0 holds v0 on entry,
// the iterate alternates between buf0 and buf1, w (n floats) is zero on entry
// and on exit; info as the explicit loop's (applications, status, done,
// stopping application).  part: csr_power_part_bytes(grid) bytes; bar / err:
// two zeroed words and a status word (a bounded barrier wait sets it).
size_t csr_power_part_bytes(int grid);
tsvd_status launch_csr_power(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci, const float *va,
                             const float *Vr, int64_t ldk, const double *sig2, int64_t l, float *buf0, float *buf1,
                             float *w, double *part, size_t part_bytes, unsigned *bar, int *err, double eps,
                             int max_iter, int iters_override, double rank_scale, int *info, double avg_nnz,
                             int max_blocks, cudaStream_t stream);

size_t power_scratch_bytes(int64_t n, int64_t l);
tsvd_status launch_power_dense(int64_t n, const float *G32, const double *G64, const double *V64,
                               const double *sigma2, int64_t l, double *x, double eps,
                               int max_iter, int iters_override, int sign_convention,
                               double *out_sigma2, int *info, void *scratch, size_t scratch_bytes,
                               cudaStream_t stream);
tsvd_status launch_power_dense_noalloc(int64_t n, const float *G32, const double *G64, const double *V64,
                                       const double *sigma2, int64_t l, double *x, double eps, int max_iter,
                                       int iters_override, int sign_convention, double *out_sigma2, int *info,
                                       cudaStream_t stream);
tsvd_status launch_symmetrize(int64_t n, double *G64, float *G32, cudaStream_t stream, bool full64 = false);
tsvd_status launch_gram_deflate(int64_t n, double *G64, float *G32, const double *v, const double *sigma2,
                                cudaStream_t stream);
tsvd_status launch_start_draws(uint64_t seed, int64_t l, int64_t n, double *x, cudaStream_t stream);
tsvd_status launch_philox_raw(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                              int64_t count, cudaStream_t stream);
tsvd_status launch_sigma_from_sigma2(const double *sig2, double *sigma, int64_t k,
                                     cudaStream_t stream);
tsvd_status launch_f64_to_f32(const double *src, float *dst, int64_t count, cudaStream_t stream);

// V[j][l] = sum_i A[i][j] U[i][l] / sigma_l for j < K (a column block of a wide
// A, d rows, stride ld); U d x k and V K x k column-major (ldu, ldv).
tsvd_status launch_left_trans(const float *A, int64_t K, int64_t d, int64_t ld, const float *U, int64_t ldu,
                              int64_t k, const double *sigma, float *V, int64_t ldv, cudaStream_t stream);
// address of the status word the TMA-fed left kernels raise on a bounded wait that gave up
tsvd_status left_status_word(int **p);
tsvd_status launch_left_dense(const float *A, int64_t rows, int64_t n, int64_t ld, const float *V,
                              int64_t ldv, int64_t k, const double *sigma, float *U, int64_t ldu,
                              cudaStream_t stream);

tsvd_status launch_csr_pair(int64_t rows, int64_t n, const int64_t *row_ptr,
                            const int32_t *col_idx, const float *values, const float *v, float *w,
                            double *ss, int scatter, double avg_nnz, cudaStream_t stream);
// Column-chunked form of the pair (see k_csr.cu): split points, then the two passes.
tsvd_status launch_csr_split(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx, int nch, int64_t cw,
                             int32_t *split, cudaStream_t stream);
tsvd_status launch_csr_chunk_y(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx, const float *values,
                               const int32_t *split, int nch, int c, const float *v, float *y, double avg_nnz,
                               cudaStream_t stream);
tsvd_status launch_csr_chunk_w(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx, const float *values,
                               const int32_t *split, int nch, int c, const float *y, float *w, double *ss, int scatter,
                               double avg_nnz, cudaStream_t stream);
tsvd_status launch_csr_left(int64_t rows, const int64_t *row_ptr, const int32_t *col_idx,
                            const float *values, const float *Vr, int64_t ldk, int64_t k,
                            const double *sigma, float *U, int64_t ldu, double avg_nnz,
                            cudaStream_t stream);

// Vector-level kernels of the streamed (CSR) power step; see k_vec.cu.
struct VecScratch {
  double *part;     // grid x kPartStride partial sums
  double *coef;     // deflation coefficients (k)
  double *scal;     // scalars: [0] ww, [1] vw, [2] vv, [3] xx, [4] 1/||w||, ...
  int *info;        // [0] iters, [1] status, [2] done flag, [3] reserved
  int grid;
};
constexpr int kVecPartStride = 40;
constexpr int kVecMaxCols = 32;  // deflation columns handled per chunk
size_t vec_scratch_bytes(int grid);
tsvd_status launch_vec_normalize_f64_to_f32(const double *x, float *v, int64_t n, VecScratch sc,
                                            cudaStream_t stream);
tsvd_status launch_vec_deflate_step(int64_t n, const float *Vr, int64_t ldk, const double *sig2,
                                    int64_t l, const float *v, float *w, float *vnext, double eps,
                                    int max_iter, int iters_override, double scale, VecScratch sc,
                                    int orth_only, cudaStream_t stream, int *ctr = nullptr);
tsvd_status launch_vec_store_column(int64_t n, const float *v, float *Vr, int64_t ldk, int64_t l,
                                    int sign_convention, VecScratch sc, cudaStream_t stream);

}  // namespace tsvd
