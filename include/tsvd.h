/*
 * tsvd.h - C ABI of a single-GPU truncated SVD by the deflated power method,
 * for NVIDIA GB300 (sm_103a).
 *
 * Method (arXiv 2208.08410, "Distributed Out-of-Memory SVD on CPU/GPU
 * Architectures"): Alg. 1 extracts the k leading singular triplets one at a
 * time; Alg. 2 finds each right singular vector by the power method on the
 * Gram matrix B = A^T A, stopping when |v0 . v1| >= 1 - eps; Sec. IV (Eq. 1-2)
 * replaces the explicit residual A - U S V^T by a deflated operator applied to
 * vectors; Sec. V-C batches row blocks of A from host memory through the GPU
 * (collinear batching) and overlaps the copies with compute on CUDA streams.
 *
 * This library computes, for A (m x n, m >= n):
 *   B  = sum over row blocks A_b^T A_b          (dense; CSR never forms B)
 *   for l = 0..k-1:
 *     v0 = x_l / ||x_l||,  x_l ~ N(0, 1)^n
 *     repeat  w = B v0 - sum_{j<l} sigma_j^2 v_j (v_j^T v0);  v1 = w / ||w||
 *     until   |v0 . v1| >= 1 - eps   (FP64), or a forced iteration count
 *     v_l = v1,  sigma_l = ||A v_l||  (= sqrt(v_l^T B v_l))
 *   U = A V diag(sigma)^-1            (one extra pass over A)
 *
 * Conventions for every entry point:
 *   - All sizes are element counts unless a name ends in _bytes.
 *   - Dense matrices are FP32 row-major with a row stride ld >= n (elements).
 *   - CSR matrices: row_ptr int64 (m+1 absolute offsets, row_ptr[0] == 0),
 *     col_idx int32 (nnz, each in [0, n)), values FP32 (nnz).
 *   - "device" pointers are CUDA device memory of the current device;
 *     "host" pointers are CPU memory (pinned memory is fastest; pageable
 *     memory works but is flagged in the report).
 *   - stream arguments are cudaStream_t values passed as void* (NULL means
 *     the legacy default stream).
 *   - No call aborts, traps or prints; every failure is a tsvd_status.
 *   - Memory passed in stays owned by the caller; the library never frees it.
 *     A plan owns only its own streams, events and small host arrays.
 */
#ifndef TSVD_H
#define TSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSVD_ABI_VERSION 1

#if defined(__GNUC__)
#define TSVD_API __attribute__((visibility("default")))
#else
#define TSVD_API
#endif

typedef enum {
  TSVD_OK = 0,
  TSVD_EINVAL = 1,       /* invalid argument, descriptor or CSR structure */
  TSVD_ENOMEM = 2,       /* host allocation failed */
  TSVD_EBUDGET = 3,      /* device budget / workspace too small for the plan */
  TSVD_ECUDA = 4,        /* a CUDA runtime call failed (see tsvd_last_cuda_error) */
  TSVD_ETIMEDOUT = 5,    /* a bounded device or host wait gave up */
  TSVD_ENOCONV = 6,      /* max_iter reached for some triplet; outputs written */
  TSVD_ERANK = 7,        /* B v0 vanished (rank(A) < k); outputs written */
  TSVD_EUNSUPPORTED = 8  /* valid request outside what this library implements */
} tsvd_status;

typedef enum { TSVD_DENSE_F32_ROWMAJOR = 0, TSVD_CSR_F32_I32_I64 = 1 } tsvd_kind;
typedef enum { TSVD_HOST = 0, TSVD_DEVICE = 1 } tsvd_location;

/* Arithmetic of the dense Gram accumulation G += A_b^T A_b (Sec. IV, Alg. 3).
 * The power iteration, deflation scalars, Rayleigh quotient and convergence
 * test are FP64 in every mode.  FP32: CUDA-core FMA.  TF32: tcgen05 tensor
 * cores on operands rounded to TF32 (nearest-even), FP32 accumulation.
 * TF32X3: each operand split a = hi + lo into two TF32 parts, products
 * hi*hi + hi*lo + lo*hi on tcgen05 (error close to FP32 inputs).
 * BF16X3: the same three-product split with two BF16 parts (hi = bf16(a),
 * mid = bf16(a - hi), both nearest-even; a - hi - mid is below 2^-16 |a|),
 * on tcgen05 kind::f16 at the BF16 rate (the paper's abstract runs the
 * products on tensor cores where the device has them).  The dropped mid*mid
 * term gives this mode a small downward bias on the diagonal (at most 2^-16
 * relative). */
typedef enum {
  TSVD_GRAM_FP32 = 0,
  TSVD_GRAM_TF32 = 1,
  TSVD_GRAM_TF32X3 = 2,
  TSVD_GRAM_BF16X3 = 3
} tsvd_gram_precision;

/* Matrix descriptor (caller-owned, read-only for the library). */
typedef struct {
  int32_t kind;             /* tsvd_kind */
  int32_t location;         /* tsvd_location of values / row_ptr / col_idx */
  int64_t m, n;             /* shape of A */
  int64_t ld;               /* dense: row stride in elements (>= n); CSR: ignored */
  const float *values;      /* dense: m*ld floats; CSR: nnz floats */
  const int64_t *row_ptr;   /* CSR: m+1 offsets; dense: NULL */
  const int32_t *col_idx;   /* CSR: nnz column indices; dense: NULL */
  int64_t nnz;              /* CSR: number of stored entries; dense: ignored */
} tsvd_matrix;

/* Options (initialise with tsvd_options_init, then override fields). */
typedef struct {
  size_t device_budget;          /* cap on the workspace in bytes (0 = none) */
  int64_t block_rows;            /* rows per streamed block (0 = planner picks) */
  int32_t n_buffers;             /* streamed blocks in flight, >= 2 (0 = 3) */
  int32_t precision;             /* tsvd_gram_precision, dense only */
  int32_t max_iter;              /* applications per triplet cap (0 = 10000) */
  int32_t sign_convention;       /* 1: largest-|entry| of each v_l made positive */
  const int32_t *iters_override; /* host, k counts: exactly that many applications
                                    per triplet, convergence test off; or NULL */
  const double *start_draws;     /* host, min(m,n) x k column-major N(0,1) draws used
                                    as x_l; NULL = the built-in Philox-4x32-10 stream */
  uint64_t seed;                 /* seed of the built-in start-vector stream */
  int32_t out_location;          /* tsvd_location of the U, sigma, V outputs */
  int32_t force_stream;          /* 1: stream host A even when it would fit */
  int32_t time_kernels;          /* 1: time each Gram kernel launch (compute stream)
                                    and each block copy (copy stream) with CUDA events
                                    (report.gram_kernel_ms, report.h2d_copy_ms) */
  int32_t power_kernel;          /* dense power phase (Alg. 1 loop over l, Alg. 2 per
                                    triplet): TSVD_POWER_AUTO, TSVD_POWER_GRID or
                                    TSVD_POWER_CLUSTER */
  int32_t gram_tile;             /* dense: width of the column panels of the orthogonal
                                    batching (a multiple of 256): the Gram matrix is
                                    formed as tiles A_J^T A_I (J <= I) and kept as FP64
                                    tiles on the device or, when they do not fit the
                                    budget, in page-locked host memory; 0 = only when
                                    the whole Gram matrix does not fit the budget */
  int32_t power_ctas;            /* CLUSTER: CTAs of the thread-block cluster (1, 2, 4
                                    or 8, reduced while a CTA would own no rows);
                                    0 = the planner's choice */
  int32_t wait_limit_ns;         /* limit in nanoseconds of the pipeline waits of the
                                    tensor-core Gram kernel (TF32, TF32X3, BF16X3) in
                                    the dense Gram pass; 0 = the default 2 s, < 0 =
                                    TSVD_EINVAL.  A limit shorter than a wait normally
                                    takes makes a correct kernel give up: it raises its
                                    status word, stops issuing, lets its own copies and
                                    MMAs complete, frees its tensor memory and returns,
                                    and tsvd_factor returns TSVD_ETIMEDOUT with
                                    TSVD_FLAG_TIMEOUT set.  It exists to test that path */
  int32_t csr_coop_blocks;       /* CSR in core, small operator: most blocks of the
                                    cooperative kernel that runs a whole triplet (0 =
                                    128, the fastest for a request alone; fewer let
                                    several requests share the GPU, as the server's
                                    sparse requests do with 64); < 0 = TSVD_EINVAL */
} tsvd_options;

/* Kernels of the dense power phase.  GRID: one cooperative launch per
 * triplet over up to one CTA per SM, a bounded grid-wide barrier per
 * application (any n).  CLUSTER: one launch for all k triplets on a single
 * thread-block cluster (up to 8 CTAs; the FP32 Gram rows in shared memory
 * when they fit), a cluster barrier per application; n <= 2048 and k <= 32,
 * otherwise tsvd_factor returns TSVD_EUNSUPPORTED.  AUTO takes CLUSTER
 * where it applies (it has the lower latency per application there). */
#define TSVD_POWER_AUTO 0
#define TSVD_POWER_GRID 1
#define TSVD_POWER_CLUSTER 2

/* Per-call report (all fields written by tsvd_factor). */
typedef struct {
  int32_t *iters;           /* caller array of k entries (applications per
                               triplet), or NULL */
  int32_t flags;            /* TSVD_FLAG_* bits */
  int32_t n_blocks;         /* streamed row blocks per pass over A */
  int32_t mode;             /* 0: A on device, 1: host A made resident, 2: streamed */
  int32_t gram_kernel_launches; /* Gram kernel launches (dense) or CSR pair launches
                                   (sparse) timed (time_kernels) */
  double gram_ms;           /* Gram pass (dense) wall time on the device clock */
  double power_ms;          /* all power iterations */
  double left_ms;           /* U pass */
  double total_ms;
  double h2d_bytes;         /* bytes copied host -> device */
  double d2h_bytes;         /* bytes copied device -> host */
  double gram_kernel_ms;    /* summed device time of those launches (time_kernels) */
  int64_t kernel_launches;  /* kernels launched by this call */
  int64_t applications;     /* total operator applications (sum of iters) */
  int32_t ring_slots;       /* row blocks the streaming ring holds (mode 2) */
  int32_t h2d_copies;       /* host -> device block copies timed (time_kernels) */
  double h2d_copy_ms;       /* summed duration of those copies on the copy stream */
  double h2d_copy_min_gbps; /* slowest single timed copy, 1e9 bytes per second */
  double h2d_copy_max_gbps; /* fastest single timed copy */
  int32_t csr_chunks;       /* CSR: column chunks of the two-pass operator (v and w
                               chunks that fit in L2), 0 = the fused single-pass
                               operator; dense: 0 */
  int32_t power_cluster;    /* dense: CTAs of the cluster power kernel, 0 = the
                               grid-wide cooperative kernel (and CSR) */
  int32_t gram_panels;      /* dense, orthogonal batching: column panels of A
                               (tasks = panels (panels + 1) / 2); 0 = one Gram */
  int32_t tiles_on_host;    /* orthogonal batching: 1 = the Gram tiles live in
                               page-locked host memory and every application
                               streams them in; 0 = they stay on the device */
} tsvd_report;

#define TSVD_FLAG_NOCONV 1        /* a triplet hit max_iter */
#define TSVD_FLAG_RANK 2          /* a triplet found B v0 == 0 */
#define TSVD_FLAG_NONMONOTONE 4   /* sigma not non-increasing in extraction order */
#define TSVD_FLAG_PAGEABLE 8      /* host input was not page-locked */
#define TSVD_FLAG_TIMEOUT 16      /* a bounded wait gave up */

typedef struct tsvd_plan_s *tsvd_plan_t;

/* Static description of a status code; never NULL. */
TSVD_API const char *tsvd_status_string(tsvd_status s);
/* Text of the last CUDA error or argument error recorded by this thread's
 * calls (or ""). */
TSVD_API const char *tsvd_last_cuda_error(void);
TSVD_API int32_t tsvd_abi_version(void);

TSVD_API void tsvd_options_init(tsvd_options *opt);

/*
 * tsvd_plan - validate A, k, eps and the options, choose how A reaches the
 * GPU (already on the device, copied once, or streamed in row blocks: the
 * paper's degree-0 / degree-1 out-of-memory cases, Sec. III) and lay out the
 * device workspace.  Pure host work: no CUDA call, no device memory.
 *
 *   out             receives a new plan (library-owned; free with tsvd_destroy)
 *   A               descriptor; for CSR host matrices the row_ptr is read
 *                   (validated, and used to size the streamed blocks)
 *   k               triplets wanted, 1..min(m,n), or -1 for min(m,n) (Alg. 1)
 *   eps             convergence threshold in (0,1) (ignored with iters_override)
 *   opt             options or NULL for defaults; arrays it points to are
 *                   copied into the plan
 *   workspace_bytes receives the device workspace size tsvd_factor needs
 *
 * Dense A with m < n takes Eq. 3: the Gram matrix is A A^T (m x m), formed
 * over column blocks of A (streamed from host memory as 2-D copies when A is
 * there), the power method finds the left vectors U, and one more pass over
 * A forms V = A^T U Sigma^-1 (Alg. 1).  start_draws then holds m x k
 * draws, and the sign convention applies to U.
 *
 * Errors: EINVAL (k out of range, eps not in (0,1), m or n <= 0, ld < n, bad
 * CSR: row_ptr not monotone, row_ptr[m] != nnz, a column outside [0,n)),
 * EUNSUPPORTED (CSR with m < n; dense min(m, n) > 32768; gram_tile with
 * m < n), EBUDGET (device_budget below the minimum workspace), ENOMEM.
 */
TSVD_API tsvd_status tsvd_plan(tsvd_plan_t *out, const tsvd_matrix *A, int64_t k, double eps,
                      const tsvd_options *opt, size_t *workspace_bytes);

/*
 * tsvd_factor - run the planned t-SVD.  Synchronous: returns when the outputs
 * are written.
 *
 *   plan       from tsvd_plan with the same A shape and kind
 *   A          the matrix (same descriptor as planned; values may change)
 *   workspace  device memory of at least workspace_bytes, 256-byte aligned
 *   stream     CUDA stream for the compute work (copies use the plan's own
 *              streams and are ordered with events)
 *   U          m x k FP32 column-major (host or device per opt.out_location),
 *              or NULL: for m >= n this skips the U pass; for m < n U holds
 *              the power method's vectors and NULL only skips their copy
 *   sigma      k FP64 singular values in extraction order (not sorted)
 *   V          n x k FP32 column-major (for m < n: the pass over A)
 *   report     optional
 *
 * Returns OK, ENOCONV / ERANK (outputs valid, flags in the report), or an
 * error (EINVAL, EBUDGET, ECUDA, ETIMEDOUT).
 */
TSVD_API tsvd_status tsvd_factor(tsvd_plan_t plan, const tsvd_matrix *A, void *workspace,
                        size_t workspace_bytes, void *stream, float *U, double *sigma,
                        float *V, tsvd_report *report);

/* The host -> device block copies of the plan's last tsvd_factor call, when
 * it ran with time_kernels (none otherwise), in issue order: for copy i,
 * first[i] is the block's first contraction index (a row of a tall dense or a
 * CSR A, a column of a wide A), bytes[i] its size and gbps[i] its rate in
 * 1e9 bytes per second between CUDA events on the copy stream.  The streamed
 * passes' rates per block show which host ranges copy slowly.  Up to `cap`
 * entries are written into each non-NULL array; *count gets the number of
 * copies recorded.  TSVD_EINVAL for a NULL plan or count or a negative cap. */
TSVD_API tsvd_status tsvd_plan_copy_log(tsvd_plan_t plan, int64_t *first, double *bytes, double *gbps,
                                        int64_t cap, int64_t *count);

/* Release a plan (NULL is accepted). */
TSVD_API void tsvd_destroy(tsvd_plan_t plan);

/* ------------------------------------------------------------------------ */
/* Step-level entry points (each one step of the method, device pointers).   */
/* ------------------------------------------------------------------------ */

/*
 * Dense Gram accumulation G += A_b^T A_b for one row block (Alg. 3 with
 * collinear row batching, Sec. V-C; B = X^T X of Alg. 2).
 *   dA      device, rows x n FP32 row-major, row stride ld
 *   dG      device, n x n FP64 row-major; the upper triangle (col >= row)
 *           receives the sums, the strict lower triangle is not touched
 *   precision  tsvd_gram_precision
 *   scratch    device scratch of tsvd_gram_scratch_bytes(rows, n, precision)
 *              bytes, 256-byte aligned (NULL allowed when that size is 0).
 *              Its first 4 bytes receive a status word once the kernels
 *              have run: 0, or nonzero when a bounded wait inside the
 *              tensor-core kernel gave up (its results are then invalid).
 * Errors: EINVAL (sizes, ld < n, misaligned scratch), EUNSUPPORTED (a tensor
 * precision on a device without tcgen05), ECUDA.
 */
TSVD_API size_t tsvd_gram_scratch_bytes(int64_t rows, int64_t n, int32_t precision);
TSVD_API tsvd_status tsvd_gram_accumulate(const float *dA, int64_t rows, int64_t n, int64_t ld, double *dG,
                                 int32_t precision, void *scratch, size_t scratch_bytes,
                                 void *stream);

/*
 * Fused CSR pair for one row block (Alg. 4 on one GPU):
 *   y_r = sum_p values[p] v[col_idx[p]]   for rows r of the block
 *   w[c] += values[p] * y_r               (FP32 atomics)
 *   *ss  += sum_r y_r^2                   (FP64)
 *   row_ptr  device, rows+1 absolute offsets; entry p of the block is at
 *            col_idx[p - row_ptr[0]], values[p - row_ptr[0]]
 *   v, w     device FP32 of length n;  ss device FP64 scalar
 *   scatter  0: only y and ss (used for sigma = ||A v||), 1: full pair
 */
TSVD_API tsvd_status tsvd_csr_gram_apply(int64_t rows, int64_t n, const int64_t *row_ptr,
                                const int32_t *col_idx, const float *values, const float *v,
                                float *w, double *ss, int32_t scatter, void *stream);

/*
 * Deflated power iteration for one triplet on a dense Gram matrix (the
 * iteration of Alg. 2 with the deflated operator of Eq. 2 in its Hotelling form), one
 * cooperative kernel that keeps the convergence loop on the device.
 *   n        order of G
 *   G32      device, n x n FP32 row-major: the Gram matrix already deflated
 *            by the earlier triplets, G - sum_{j<l} sigma_j^2 v_j v_j^T
 *            (tsvd_gram_symmetrize, then tsvd_gram_deflate once per triplet)
 *   G64      device, n x n FP64: the upper triangle of the same deflated
 *            matrix (FP64), for sigma_l^2 = v_l^T G v_l, formed as
 *            v_l^T G64 v_l + sum_{j<l} sigma_j^2 (v_j . v_l)^2
 *   V64      device, n x l FP64 column-major earlier vectors and
 *   sigma2   device, l FP64 earlier sigma^2 (the term above, and, when B v0
 *            vanishes, v_l = v0 made orthogonal to V64, sigma_l = 0); NULL if l == 0
 *   x        device, n FP64: in = start draw (not necessarily normalised),
 *            out = v_l (unit norm)
 *   eps, max_iter, iters_override (<= 0: use the convergence test)
 *   sign_convention  1: make the largest-|entry| positive
 *   out_sigma2  device FP64 scalar: sigma_l^2
 *   info     device int32[4]: {applications, status (0 ok, 1 noconv, 2 rank),
 *            timeout flag, 0}
 *   scratch  device, tsvd_power_scratch_bytes(n, l) bytes (zeroing not needed)
 */
TSVD_API size_t tsvd_power_scratch_bytes(int64_t n, int64_t l);
TSVD_API tsvd_status tsvd_power_dense(int64_t n, const float *G32, const double *G64, const double *V64,
                             const double *sigma2, int64_t l, double *x, double eps,
                             int32_t max_iter, int32_t iters_override, int32_t sign_convention,
                             double *out_sigma2, int32_t *info, void *scratch,
                             size_t scratch_bytes, void *stream);

/*
 * tsvd_power_dense_noalloc - the deflated power iteration of tsvd_power_dense
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; it exists for integration.  Some callers cannot call
 * cudaMalloc: their device memory belongs to another allocator (a
 * framework's caching pool, a process whose device memory is capped or fully
 * reserved up front), or they run where an allocation and the device
 * synchronisation it may imply are not allowed.  This entry point allocates
 * nothing: its scratch is one fixed-size array in the library's device
 * memory, held by every GPU that loads the library until the process exits.
 *
 * Arguments and outputs are those of tsvd_power_dense minus the scratch
 * pointer and size; the caller still passes all inputs and outputs.
 * Limits: n <= TSVD_NOALLOC_MAX_N and l <= TSVD_NOALLOC_MAX_L, otherwise
 * TSVD_EINVAL with a message in tsvd_last_cuda_error().
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, with that device current), and so does the
 * first call after the device's context was recreated (cudaDeviceReset): the
 * address is kept with the context it belongs to.  Make such a call before
 * any stream capture.  All calls share the one array, which keeps
 * the last call's contents (the call clears what must start at zero): calls
 * that overlap on the GPU, on any streams, race and give wrong results.
 */
#define TSVD_NOALLOC_MAX_N 16384
#define TSVD_NOALLOC_MAX_L 64
TSVD_API tsvd_status tsvd_power_dense_noalloc(int64_t n, const float *G32, const double *G64,
                                              const double *V64, const double *sigma2, int64_t l,
                                              double *x, double eps, int32_t max_iter,
                                              int32_t iters_override, int32_t sign_convention,
                                              double *out_sigma2, int32_t *info, void *stream);

/* Hotelling deflation of the Gram matrix by one triplet (the deflated
 * operator of Eq. 2 in Hotelling form), in FP64: on the upper triangle of
 * G64 (n x n row-major, entry (i, j) with j >= i) G64 -= sigma2[0] v v^T, then
 * G32 (n x n row-major FP32, both halves) = the FP32 rounding of the deflated
 * G64.  v device FP64 n, sigma2 device FP64 scalar.  Rounding the FP32 copy
 * from the deflated FP64 matrix keeps its error relative to the spectrum that
 * remains. */
TSVD_API tsvd_status tsvd_gram_deflate(int64_t n, double *G64, float *G32, const double *v, const double *sigma2,
                                       void *stream);

/* Fill G32 (n x n FP32, full) from the upper triangle of G64 (symmetrise). */
TSVD_API tsvd_status tsvd_gram_symmetrize(int64_t n, const double *G64, float *G32, void *stream);

/*
 * Start draw x ~ N(0,1)^n for triplet l (Alg. 2) from the Philox-4x32-10
 * stream keyed by splitmix64(seed) (Salmon et al., SC'11), Box-Muller in FP64:
 * counter (p mod 2^32, p div 2^32, l, 0x54535644) for pair p = i/2.
 *   x  device FP64, n entries
 */
TSVD_API tsvd_status tsvd_start_draws(uint64_t seed, int64_t l, int64_t n, double *x, void *stream);

/* Raw Philox-4x32-10 block function on the device, for checking the
 * generator: out[4*i .. 4*i+3] = philox(ctr[4*i..], key[2*i..]), count blocks.
 * ctr, key, out: device uint32 arrays. */
TSVD_API tsvd_status tsvd_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                               int64_t count, void *stream);

/*
 * Left vectors for one row block (Alg. 1): U_b = A_b V diag(sigma)^-1
 *   dA     device rows x n FP32 row-major (stride ld)
 *   V      device n x k FP32 column-major (stride ldv >= n)
 *   sigma  device k FP64; a zero sigma gives a zero column
 *   U      device, column-major with stride ldu >= rows: U[r + l*ldu]
 */
TSVD_API tsvd_status tsvd_left_vectors(const float *dA, int64_t rows, int64_t n, int64_t ld, const float *V,
                              int64_t ldv, int64_t k, const double *sigma, float *U, int64_t ldu,
                              void *stream);

/*
 * CSR row-block partition (Sec. V-C collinear batching), host only: blocks of
 * block_rows rows, the last one ragged.  block_start receives n_blocks+1 row
 * indices (caller array of at least ceil(m/block_rows)+1 entries); block
 * b covers rows [block_start[b], block_start[b+1]) and entries
 * [row_ptr[block_start[b]], row_ptr[block_start[b+1]]).  *max_block_nnz
 * receives the largest entry count of a block.
 */
TSVD_API tsvd_status tsvd_csr_partition(int64_t m, const int64_t *row_ptr, int64_t block_rows,
                               int64_t *block_start, int64_t *n_blocks, int64_t *max_block_nnz);

/* Page-locked host memory for A: an anonymous mapping aligned to the
 * transparent-huge-page size and advised MADV_HUGEPAGE (huge pages where the
 * host has them, base pages otherwise), zero-filled, then registered with
 * cudaHostRegister (portable: page-locked for every device).  With huge pages
 * the copy engines translate the range through a few hundred page-table
 * entries instead of millions, so row-block copies keep the link rate while
 * kernels run beside them.  From a quarter of a huge page up, the mapping is
 * rounded up to whole huge pages (at most one huge page more than asked), so
 * that its tail is not left on base pages.  *ptr is NULL on failure (TSVD_ENOMEM, or
 * TSVD_ECUDA when the registration fails).  Free with tsvd_host_free, which
 * accepts only pointers from tsvd_host_alloc (TSVD_EINVAL otherwise; NULL is
 * a no-op). */
TSVD_API tsvd_status tsvd_host_alloc(void **ptr, size_t bytes);
TSVD_API tsvd_status tsvd_host_free(void *ptr);

/* ------------------------------------------------------------------------ */
/* Serving: many t-SVD requests of different m, n, k with continuous         */
/* batching.  No counterpart in the paper (which factors one matrix); each   */
/* request runs the same method (Alg. 1/2, Hotelling deflation, FP64         */
/* Rayleigh quotient and convergence test; Eq. 3 when m < n).                */
/* ------------------------------------------------------------------------ */
typedef struct tsvd_server_s *tsvd_server_t;

typedef struct {
  size_t device_budget;   /* HBM the server allocates once and admits requests
                             into (0: 8 GiB) */
  int32_t max_inflight;   /* requests admitted at once (0: 4096) */
  int32_t n_streams;      /* waves in flight at once, one stream each (0: 8) */
  int32_t max_wave;       /* most requests one wave launches together (0: 64) */
  int32_t cluster_cap;    /* largest thread-block cluster of the power kernel
                             (1, 2, 4 or 8; 0: 8) */
  size_t host_staging;    /* page-locked host memory each request's results
                             are copied into from its device output region
                             before tsvd_server_wait hands them to the
                             caller (0: 2 GiB) */
  int32_t heavy_dim;      /* requests with min(m, n) above this run in waves
                             of their own ("heavy" lane): their power phase
                             reads a large Gram matrix per application and
                             can last long, and a wave's stream stays busy
                             until its last request is done, so light waves
                             (on the n_streams streams) are never held behind
                             them (0 or -1: one lane for all) */
  int32_t heavy_streams;  /* most streams the heavy lane opens, one more each
                             time heavy requests wait and none is idle
                             (0: 64 - n_streams; n_streams + heavy_streams
                             <= 64) */
  int32_t wave_graphs;    /* 1: each dense wave's kernels are captured and
                             launched as a CUDA graph (instantiated graphs
                             cached per stream by launch signature and updated
                             in place); 0 (default): launched directly on the
                             wave's stream.  Both run the same kernels on the
                             same descriptors, so results are bitwise equal */
  int32_t reserved[3];
} tsvd_server_options;

/* Per-request record (tsvd_server_wait / tsvd_server_poll). */
typedef struct {
  int32_t status;         /* TSVD_OK, TSVD_ENOCONV, TSVD_ERANK, or an error */
  int32_t flags;          /* TSVD_FLAG_* */
  int64_t applications;   /* operator applications over all triplets */
  double submit_s;        /* server clock (seconds since tsvd_server_create) */
  double admit_s;         /* admitted into the device budget */
  double launch_s;        /* its wave was launched */
  double done_s;          /* its wave's completion was observed */
  int32_t wave;           /* index of the wave it ran in */
  int32_t cluster;        /* CTAs of its power-kernel cluster */
} tsvd_request_info;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t waves;               /* waves launched */
  int64_t kernel_launches;     /* kernels the scheduler launched */
  int64_t peak_device_bytes;   /* high-water mark of the arena */
  double busy_s;               /* time with at least one wave in flight */
  int64_t graph_updates;       /* waves whose captured kernel graph updated the
                                  slot's instantiated graph in place */
  int64_t graph_instantiations;/* waves whose graph had a new shape and was
                                  instantiated */
  double wave_host_s;          /* scheduler time spent forming and launching waves
                                  (descriptors, copies, capture, graph update or
                                  instantiation, launch) */
  int64_t peak_streams_busy;   /* most streams with a wave in flight at once */
  double graph_host_s;         /* the part of wave_host_s spent capturing and updating
                                  or instantiating the waves' graphs (with graphs
                                  off: enqueuing the launches) */
} tsvd_server_stats;

TSVD_API tsvd_status tsvd_server_options_init(tsvd_server_options *opt);

/* Allocates the device arena (device_budget bytes, on the current device) and
 * starts the scheduler thread.  Errors: EINVAL (options), ENOMEM, ECUDA. */
TSVD_API tsvd_status tsvd_server_create(tsvd_server_t *server, const tsvd_server_options *opt);

/*
 * Queue one dense request A = U Sigma V^T (truncated to k).
 *   A        host, m x n FP32 row-major (row stride n); read by an
 *            asynchronous copy once the request is admitted, so it must stay
 *            valid and unchanged until the request completes.  Page-locked
 *            memory (tsvd_host_alloc) lets the copy overlap other work.
 *   U, sigma, V  host outputs: U m x k and V n x k column-major FP32, sigma k
 *            FP64; the kernels write the results into the request's device
 *            output region, the scheduler copies that to the server's
 *            page-locked staging, and tsvd_server_wait copies them here.
 *   k        1 <= k <= min(m, n), k <= 32;  min(m, n) <= 2048
 *   eps, max_iter, seed, sign_convention, iters_override  as for tsvd_plan /
 *            tsvd_options (start draws: the built-in Philox-4x32-10 stream of
 *            `seed`; iters_override: k forced application counts, or NULL)
 *   ticket   receives the request's id
 * Requests are admitted first in, first out as the device budget and
 * max_inflight allow.  Errors: EINVAL (arguments), EBUDGET (the request alone
 * exceeds the device budget), EUNSUPPORTED (min(m, n) > 2048 or k > 32).
 */
TSVD_API tsvd_status tsvd_server_submit(tsvd_server_t server, const float *A, int64_t m, int64_t n, int32_t k,
                                        double eps, int32_t max_iter, uint64_t seed, int32_t sign_convention,
                                        const int32_t *iters_override, float *U, double *sigma, float *V,
                                        uint64_t *ticket);

/*
 * tsvd_server_submit_csr - queue a sparse t-SVD (CSR, m >= n) with the same
 * arguments as tsvd_server_submit plus the CSR arrays (host memory: row_ptr
 * m+1 int64, col_idx nnz int32, values nnz FP32, read until completion).
 * Sparse requests do not join the dense waves: eight worker threads run them
 * one at a time each through tsvd_plan / tsvd_factor (the implicit operator
 * A^T (A v), Alg. 4), with the workspace taken from the server's device
 * budget (at most a quarter of it per request; beyond that the plan streams
 * A in row blocks) and the results written straight into U, sigma and V.
 * Dense waves keep running beside them.  Errors: EINVAL, EUNSUPPORTED (m < n).
 */
TSVD_API tsvd_status tsvd_server_submit_csr(tsvd_server_t server, const int64_t *row_ptr, const int32_t *col_idx,
                                            const float *values, int64_t m, int64_t n, int64_t nnz, int32_t k,
                                            double eps, int32_t max_iter, uint64_t seed, int32_t sign_convention,
                                            const int32_t *iters_override, float *U, double *sigma, float *V,
                                            uint64_t *ticket);

/* Block until the request completes or timeout_s passes (< 0: no limit),
 * then copy its results into the caller's U, sigma, V.  Returns the
 * request's status (TSVD_ETIMEDOUT on timeout) and fills *info.  A completed
 * request's record and staging are released by this call.  A request
 * completes as soon as its own cluster has finished (a flag the kernel sets),
 * not when the rest of its wave does. */
TSVD_API tsvd_status tsvd_server_wait(tsvd_server_t server, uint64_t ticket, double timeout_s, tsvd_request_info *info);

TSVD_API tsvd_status tsvd_server_get_stats(tsvd_server_t server, tsvd_server_stats *stats);

/* Message of the last failure inside the scheduler ("" if none). */
TSVD_API const char *tsvd_server_last_error(tsvd_server_t server);

/* Power-kernel cluster size the server uses for Gram dimension d. */
TSVD_API int32_t tsvd_server_cluster_for(tsvd_server_t server, int64_t d);

/* Set the power-kernel cluster size for the Gram dimensions of d's class
 * (d <= 64, 128, 256, 512, 1024, 2048): c in {1, 2, 4, 8}, at most the
 * server's cluster_cap, and reduced for small d as the kernel needs (every CTA
 * owns rows).  Applies to later submissions; a request's cluster still depends
 * on its own shape only.  EINVAL for other values. */
TSVD_API tsvd_status tsvd_server_set_cluster_for(tsvd_server_t server, int64_t d, int32_t c);

/*
 * Pick the power-kernel cluster size per Gram dimension by measurement: for
 * d in {64, 128, 256, 512, 1024, 2048} and each cluster size up to
 * cluster_cap, time `iters` iterations of one synthetic request alone, and
 * keep the size with the lowest single-request
 * time, a larger size only where it is more than 15 % faster: a request holds its CTAs,
 * memory and wave until it is done, so on a serving mix the fastest request
 * gives the highest capacity.  Then pick the Gram step's tile shape per size: for
 * d in {256, 512, 1024, 2048} it times the grouped tensor-core SYRK (128 x 256
 * tiles, 3xTF32) and the grouped CUDA-core SYRK (64 x 64 tiles, FP32) on
 * synthetic 8192 x d requests, enough to give both kernels work for every SM,
 * and sets the tensor-core threshold (tsvd_server_tc_min_d) to the smallest d
 * from which the tensor cores are faster at that size and every larger one
 * (INT64_MAX when they never are).  Call with no requests in flight.  Both
 * choices apply to later submissions; tsvd_server_cluster_for reads the first.
 */
TSVD_API tsvd_status tsvd_server_autotune(tsvd_server_t server, int32_t iters);

/*
 * Gram dimension d = min(m, n) from which a dense request forms its Gram
 * matrix on the tensor cores: a grouped, persistent tcgen05 SYRK over all
 * such requests of a wave (3xTF32: each FP32 value split into two TF32 parts,
 * three MMAs per product, FP32 accumulation in short TMEM segments carried
 * into FP64 every 512 rows).  Each 128 x 256 tile spans its request's whole
 * contraction range and writes its own entries without atomics, so a
 * request's result is bitwise the same alone and in any wave.  Smaller
 * requests use the CUDA-core SYRK.  Default 256 until tsvd_server_autotune
 * measures it; the setter overrides it for later submissions (d >= 1;
 * INT64_MAX: never).  The getter returns 0 for a NULL server.
 */
TSVD_API int64_t tsvd_server_tc_min_d(tsvd_server_t server);
/* The autotuner's Gram-step timings behind that choice: for d = 256, 512,
 * 1024, 2048 (4 entries each), milliseconds of the tensor-core and of the
 * CUDA-core grouped SYRK over `requests` synthetic 8192 x d requests (zeros
 * before tsvd_server_autotune or for a size the budget could not hold). */
TSVD_API tsvd_status tsvd_server_autotune_syrk_times(tsvd_server_t server, int64_t *d, double *ms_tensor,
                                                     double *ms_cuda, int32_t *requests);
TSVD_API tsvd_status tsvd_server_set_tc_min_d(tsvd_server_t server, int64_t d);

/* Stop the scheduler (requests still queued fail with TSVD_ECUDA) and free
 * the device arena.  NULL is accepted. */
TSVD_API void tsvd_server_destroy(tsvd_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* TSVD_H */
