// Host runtime of the tsvd C ABI: validation, the planner (device workspace
// layout, degree-0 / degree-1 out-of-memory mode, row-block sizes), the
// row-block streamer (page-locked host -> device ring on its own copy stream,
// event hand-off to the compute stream, Sec. V-C and the stream queue of
// Alg. 3), and the drivers of the three phases: Gram pass (dense), power
// phase (Alg. 1 loop over l, Alg. 2 per triplet) and the left-vector pass.
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "philox.cuh"
#include "serve.cuh"

namespace tsvd {

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;
static thread_local int64_t g_launches = 0;

void set_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
  g_err = buf;
}
void set_error_text(const std::string &s) { g_err = s; }

tsvd_status ensure_dynamic_smem(const void *func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> set;
  int dev = -1;
  TSVD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = set[std::make_pair(func, dev)];
  if (bytes <= cur) return TSVD_OK;
  TSVD_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return TSVD_OK;
}
void count_launch() { ++g_launches; }
void count_launches(int64_t n) { g_launches += n; }
int64_t launches_so_far() { return g_launches; }

// ---------------------------------------------------------------- page-locked host memory
static std::mutex g_pinned_mu;
static std::map<uintptr_t, size_t> g_pinned;  // start -> mapped length, for pinned_free

// Size of a transparent huge page (the PMD size the kernel reports), or 2 MiB.
static size_t thp_bytes() {
  static size_t cached = 0;
  if (!cached) {
    size_t v = 0;
    if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
      unsigned long long x = 0;
      if (fscanf(f, "%llu", &x) == 1) v = (size_t)x;
      fclose(f);
    }
    cached = (v >= 4096 && (v & (v - 1)) == 0) ? v : ((size_t)2 << 20);
  }
  return cached;
}

tsvd_status pinned_alloc(void **ptr, size_t bytes) {
  if (!ptr) return TSVD_EINVAL;
  *ptr = nullptr;
  if (bytes == 0) return TSVD_EINVAL;
  const size_t page = (size_t)sysconf(_SC_PAGESIZE);
  const size_t hp = std::max(thp_bytes(), page);
  if (bytes > SIZE_MAX - 2 * hp) return TSVD_EINVAL;
  size_t len = (bytes + page - 1) / page * page;
  // from a quarter of a huge page up, whole huge pages: the tail of a mapping
  // that ends inside a huge page stays on base pages, and those copy slowly
  // beside kernels on some hosts (every streamed pass pays for them again)
  if (hp > page && len >= hp / 4) len = (len + hp - 1) / hp * hp;
  // map one huge page more than needed so the start can be aligned, then trim
  void *raw = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) {
    set_error_text("tsvd_host_alloc: mmap failed");
    return TSVD_ENOMEM;
  }
  const uintptr_t r0 = reinterpret_cast<uintptr_t>(raw);
  const uintptr_t start = (r0 + hp - 1) / hp * hp;
  if (start > r0) munmap(raw, start - r0);
  const uintptr_t end = start + len, rend = r0 + len + hp;
  if (rend > end) munmap(reinterpret_cast<void *>(end), rend - end);
  unsigned char *p = reinterpret_cast<unsigned char *>(start);
  madvise(p, len, MADV_HUGEPAGE);  // advisory: base pages where huge ones are not available
  for (size_t o = 0; o < len; o += page) p[o] = 0;  // fault the pages in before pinning them
#ifndef MADV_COLLAPSE
#define MADV_COLLAPSE 25
#endif
  // ranges that faulted in as base pages (no free huge page at the time) are
  // collapsed into huge pages now, with compaction, where the kernel can;
  // an error (an older kernel, no memory to compact) leaves them as they are
  if (len >= hp) madvise(p, len, MADV_COLLAPSE);
  const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterPortable);
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaHostRegister", __FILE__, __LINE__);
    cudaGetLastError();
    munmap(p, len);
    return e == cudaErrorMemoryAllocation ? TSVD_ENOMEM : TSVD_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned[start] = len;
  }
  *ptr = p;
  return TSVD_OK;
}

tsvd_status pinned_free(void *ptr) {
  if (!ptr) return TSVD_OK;
  size_t len = 0;
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned.find(reinterpret_cast<uintptr_t>(ptr));
    if (it == g_pinned.end()) return TSVD_EINVAL;
    len = it->second;
    g_pinned.erase(it);
  }
  const cudaError_t e = cudaHostUnregister(ptr);
  munmap(ptr, len);
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaHostUnregister", __FILE__, __LINE__);
    cudaGetLastError();
    return TSVD_ECUDA;
  }
  return TSVD_OK;
}

tsvd_status device_info(DeviceInfo *out) {
  static thread_local DeviceInfo cache;
  int dev = -1;
  TSVD_CUDA(cudaGetDevice(&dev));
  if (cache.device != dev) {
    DeviceInfo d;
    d.device = dev;
    TSVD_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    TSVD_CUDA(cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    TSVD_CUDA(cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    int optin = 0;
    TSVD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    d.smem_optin = (size_t)optin;
    int l2 = 0;
    TSVD_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    d.l2_bytes = (size_t)l2;
    cache = d;
  }
  *out = cache;
  return TSVD_OK;
}

}  // namespace tsvd

using namespace tsvd;

// ---------------------------------------------------------------- plan
namespace {

enum Mode { MODE_DEVICE = 0, MODE_RESIDENT = 1, MODE_STREAM = 2 };

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = (size_t)round_up((int64_t)(off + bytes), 256);
    return o;
  }
};

}  // namespace

struct tsvd_plan_s {
  // problem
  int kind = 0, location = 0;
  int64_t m = 0, n = 0, ld = 0, nnz = 0, k = 0;
  double eps = 0.0;
  tsvd_options opt{};
  std::vector<int32_t> iters_override;
  std::vector<double> start_draws;
  // planning
  int mode = MODE_DEVICE;
  int64_t chunk_rows = 0, n_chunks = 0;
  int64_t gram_rows = 0;        // dense: rows per Gram launch (a block is cut into launches of this size)
  int64_t n_gram_launches = 0;  // dense: Gram launches per pass
  int n_buffers = 3;
  // CSR partition (rows) and per-block entry counts (host-located CSR)
  std::vector<int64_t> block_start;
  int64_t max_block_nnz = 0;
  double avg_nnz = 0.0;
  // workspace layout
  size_t ws = 0;
  size_t o_G64 = 0, o_G32 = 0, o_V64 = 0, o_V32 = 0, o_sig2 = 0, o_sigma = 0, o_info = 0;
  size_t o_pscr = 0, b_pscr = 0, o_gscr = 0, b_gscr = 0, o_ring = 0, b_slot = 0;
  size_t o_res = 0, o_ubuf = 0, b_ubuf = 0;
  size_t o_v = 0, o_vn = 0, o_w = 0, o_x64 = 0, o_Vr = 0, o_vsc = 0, o_flag = 0;
  // column-chunked CSR operator (v and w larger than what L2 holds)
  int csr_nch = 0;            // chunks (0: the fused single-pass kernel)
  int64_t csr_cw = 0;         // columns per chunk
  bool csr_sorted = true;     // every row's columns ascending (host CSR: checked at plan time)
  size_t o_csr_y = 0, o_csr_split = 0, b_split_slot = 0;
  int vec_grid = 0;
  // dense: the Gram's dimension d = min(m, n) and the contraction length K = max(m, n).
  // wide (m < n, Eq. 3): the Gram is A A^T, blocks are column blocks of A, the
  // power method finds U and the pass over A forms V = A^T U Sigma^-1
  bool wide = false;
  int64_t d = 0, K = 0;
  // orthogonal batching (dense; Sec. V-C, Alg. 3): the Gram matrix as FP64 tiles
  // B_JI = A_J^T A_I (J <= I) of tb-column panels, formed task by task
  bool tiled = false;
  int64_t tb = 0, n_panels = 0, n_tasks = 0, pan_rows = 0;
  bool tiles_host = false;   // tiles in page-locked host memory, streamed in every application
  size_t b_tile = 0, o_tiles = 0, o_Gt = 0, o_pan = 0, b_pan = 0, o_w64 = 0, o_Vc = 0;
  double *host_tiles = nullptr;  // n_tasks tiles of tb x tb (allocated on the first factorisation)
  // dense power phase on one thread-block cluster (n <= kSrvMaxDim, k <= kSrvMaxK)
  bool cluster_power = false;
  SrvReq srv_req{};  // host copy of the descriptor the cluster kernel reads (copied per call)
  // runtime objects (created on first factor, on the device current then)
  int device = -1;
  cudaStream_t copy_stream = nullptr, d2h_stream = nullptr;
  cudaStream_t copy_stream2 = nullptr;  // second half of every block copy (a second copy engine)
  // the explicit power loop's stream when it replays graphs (a capture cannot use the
  // legacy default stream a caller may pass), forked from and joined to the caller's
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_aux = nullptr;
  cudaEvent_t ev_csplit = nullptr, ev_cjoin = nullptr;
  std::vector<cudaEvent_t> ev_ready, ev_free;
  cudaEvent_t ev_u_ready[2] = {nullptr, nullptr}, ev_u_free[2] = {nullptr, nullptr};
  cudaEvent_t ev_t[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> ev_k;  // pairs around each timed Gram kernel
  std::vector<cudaEvent_t> ev_c;  // pairs around each timed block copy
  struct CopyRec {
    int64_t first;
    double bytes, gbps;
  };
  std::vector<CopyRec> copy_log;  // the timed block copies of the last tsvd_factor call
};

namespace {

tsvd_status validate_csr_host(const tsvd_matrix *A, bool *sorted) {
  const int64_t m = A->m, n = A->n, nnz = A->nnz;
  const int64_t *rp = A->row_ptr;
  if (rp[0] != 0 || rp[m] != nnz) return TSVD_EINVAL;
  for (int64_t r = 0; r < m; ++r)
    if (rp[r + 1] < rp[r]) return TSVD_EINVAL;
  const int32_t *ci = A->col_idx;
  for (int64_t p = 0; p < nnz; ++p)
    if (ci[p] < 0 || (int64_t)ci[p] >= n) return TSVD_EINVAL;
  bool srt = true;
  for (int64_t r = 0; r < m && srt; ++r)
    for (int64_t p = rp[r] + 1; p < rp[r + 1]; ++p)
      if (ci[p] < ci[p - 1]) {
        srt = false;
        break;
      }
  *sorted = srt;
  return TSVD_OK;
}

void partition_rows(int64_t m, int64_t block_rows, std::vector<int64_t> &starts) {
  starts.clear();
  for (int64_t r = 0; r < m; r += block_rows) starts.push_back(r);
  starts.push_back(m);
}

tsvd_status plan_dense_tiled(tsvd_plan_s *p);

tsvd_status plan_dense(tsvd_plan_s *p) {
  // in Gram terms: n = d (the Gram's dimension), m = K (the contraction length,
  // cut into blocks: rows of a tall A, columns of a wide one)
  const int64_t n = p->d, k = p->k, m = p->K;
  const int prec = p->opt.precision;
  if (p->opt.gram_tile > 0) return plan_dense_tiled(p);
  Carve c;
  p->o_G64 = c.take((size_t)n * n * 8);
  p->o_G32 = c.take((size_t)n * n * 4);
  p->o_V64 = c.take((size_t)n * k * 8);
  p->o_V32 = c.take((size_t)n * k * 4);
  p->o_sig2 = c.take((size_t)k * 8);
  p->o_sigma = c.take((size_t)k * 8);
  p->o_info = c.take((size_t)k * 4 * sizeof(int32_t));
  p->b_pscr = power_scratch_bytes(n, k);
  p->o_pscr = c.take(p->b_pscr);
  const size_t fixed = c.off;
  const bool host_a = p->location == TSVD_HOST;
  const bool host_u = p->opt.out_location == TSVD_HOST;
  const int R = p->n_buffers;
  // The Gram kernels run on sub-chunks of at most gram_target rows (the
  // in-core launch size, ~1 GiB of A): a larger streamed block is cut into
  // several launches, so the tensor-core scratch stays that size and the SYRK
  // keeps the K-slice working set it was tuned for.
  const int64_t gram_target = std::max<int64_t>(256, round_up(((int64_t)1 << 30) / (n * 4), 32));
  auto chunk_cost = [&](int64_t rows, int mode) -> size_t {
    size_t s = gram_tc_scratch_bytes(std::min(rows, gram_target), n, prec) + 256;
    if (mode == MODE_STREAM) s += (size_t)R * (size_t)round_up(rows * n * 4, 256);
    if (host_u) s += 2 * (size_t)round_up(rows * k * 4, 256);
    return s;
  };
  int64_t target = p->opt.block_rows > 0 ? p->opt.block_rows
                                         : std::max<int64_t>(256, ((int64_t)1 << 30) / (n * 4));
  target = std::min<int64_t>(round_up(target, 32), round_up(m, 32));
  const size_t budget = p->opt.device_budget;
  const size_t resident_bytes = (size_t)round_up(m * n * 4, 256);
  int mode = MODE_DEVICE;
  if (host_a) {
    mode = MODE_STREAM;
    if (!p->opt.force_stream) {
      if (budget == 0 || fixed + resident_bytes + chunk_cost(target, MODE_RESIDENT) <= budget)
        mode = MODE_RESIDENT;
    }
  }
  int64_t rows = target;
  if (budget) {
    while (rows > 32 && fixed + (mode == MODE_RESIDENT ? resident_bytes : 0) + chunk_cost(rows, mode) > budget)
      rows = round_up(rows / 2, 32);
    if (fixed + (mode == MODE_RESIDENT ? resident_bytes : 0) + chunk_cost(rows, mode) > budget) {
      // the whole Gram matrix does not fit: orthogonal batching
      return plan_dense_tiled(p);
    }
  }
  p->mode = mode;
  p->chunk_rows = rows;
  p->n_chunks = ceil_div(m, rows);
  p->gram_rows = std::min(rows, gram_target);
  p->n_gram_launches = 0;
  for (int64_t c = 0; c < p->n_chunks; ++c)
    p->n_gram_launches += ceil_div(std::min(rows, m - c * rows), p->gram_rows);
  p->b_gscr = gram_tc_scratch_bytes(p->gram_rows, n, prec);
  p->o_gscr = c.take(p->b_gscr + 256);
  if (mode == MODE_RESIDENT) p->o_res = c.take(resident_bytes);
  if (host_u) {
    p->b_ubuf = (size_t)round_up(rows * k * 4, 256);
    p->o_ubuf = c.take(2 * p->b_ubuf);
  }
  if (mode == MODE_STREAM) {
    // ring of row blocks, carved last: under a budget it takes every slot that
    // fits, so the blocks still resident after the Gram pass serve the U pass
    p->b_slot = (size_t)round_up(rows * n * 4, 256);
    int64_t slots = R;
    if (budget && budget > c.off + (size_t)R * p->b_slot) {
      const int64_t extra = (int64_t)((budget - c.off - (size_t)R * p->b_slot) / p->b_slot);
      slots = std::min<int64_t>(std::max<int64_t>(R, p->n_chunks), R + extra);
      slots = std::min<int64_t>(slots, 64);
    }
    p->n_buffers = (int)slots;
    p->o_ring = c.take(p->b_slot * slots);
  }
  p->ws = c.off;
  if (budget && p->ws > budget) return plan_dense_tiled(p);
  return TSVD_OK;
}

// Orthogonal batching: panels of tb columns, tasks (I, J) with J <= I (the
// symmetric task reuse: only B_JI = A_J^T A_I is formed, B_IJ is its
// transpose).  Workspace: the explicit power loop's vectors, the tiles (all
// of them when they fit, else a ring of n_buffers through which every
// application streams them from page-locked host memory), then one region
// used in turn by the Gram tasks (task tile, tensor-core scratch, panel ring
// for host A) and by the U pass (row-block ring for host A, U staging).
tsvd_status plan_dense_tiled(tsvd_plan_s *p) {
  if (p->wide) return TSVD_EUNSUPPORTED;  // column panels of a wide A: not built
  const int64_t n = p->n, k = p->k, m = p->m;
  const int prec = p->opt.precision;
  if (k + 4 > kVecPartStride) return TSVD_EUNSUPPORTED;
  const size_t budget = p->opt.device_budget;
  const bool host_a = p->location == TSVD_HOST;
  const bool host_u = p->opt.out_location == TSVD_HOST;
  const int R = std::max(2, p->n_buffers);
  p->n_buffers = R;
  p->tiled = true;
  p->cluster_power = false;
  p->o_G64 = p->o_G32 = p->o_V64 = p->o_pscr = p->o_res = 0;
  Carve c;
  p->o_v = c.take((size_t)n * 4);
  p->o_vn = c.take((size_t)n * 4);
  p->o_w = c.take((size_t)n * 4);
  p->o_x64 = c.take((size_t)n * 8);
  p->o_w64 = c.take((size_t)n * 8);
  p->o_Vr = c.take((size_t)n * k * 4);
  p->o_Vc = c.take((size_t)n * k * 4);
  p->o_sig2 = c.take((size_t)k * 8);
  p->o_sigma = c.take((size_t)k * 8);
  p->o_info = c.take((size_t)k * 4 * sizeof(int32_t));
  // 256-byte word region: [0] validation flag of a device CSR, [64] the operator's v^T G v
  // (FP64), [128] the triplet's application counter, [192] barrier words and [200] the
  // barrier status of the cooperative triplet loop
  p->o_flag = c.take(256);
  p->vec_grid = 1024;
  p->o_vsc = c.take(vec_scratch_bytes(p->vec_grid));
  const size_t fixed = c.off;
  auto al = [](size_t x) { return (size_t)round_up((int64_t)x, 256); };
  auto gram_area = [&](int64_t bs, int64_t rows) -> size_t {
    size_t g = al((size_t)bs * 2 * bs * 8);
    if (prec != TSVD_GRAM_FP32) g += gram_tc_scratch_bytes(rows, 2 * bs, prec) + 256;
    if (host_a) g += (size_t)R * al((size_t)rows * 2 * bs * 4);
    return g;
  };
  auto u_area = [&](int64_t rows) -> size_t {
    return (host_a ? (size_t)R * al((size_t)rows * n * 4) : 0) + (host_u ? 2 * al((size_t)rows * k * 4) : 0);
  };
  auto shrink = [&](int64_t target, const std::function<size_t(int64_t)> &need, size_t room) -> int64_t {
    int64_t rows = std::min<int64_t>(round_up(std::max<int64_t>(target, 32), 32), round_up(m, 32));
    while (rows > 32 && need(rows) > room) rows = round_up(rows / 2, 32);
    return need(rows) <= room ? rows : 0;
  };
  std::vector<int64_t> cands;
  if (p->opt.gram_tile > 0) {
    cands.push_back(p->opt.gram_tile);
  } else {
    for (int64_t bs = std::min<int64_t>(round_up(n, 256), 8192); bs >= 256; bs = bs / 2 / 256 * 256) {
      cands.push_back(bs);
      if (bs == 256) break;
    }
  }
  for (const int64_t bs : cands) {
    const int64_t nb = ceil_div(n, bs), tasks = nb * (nb + 1) / 2;
    const size_t bt = al((size_t)bs * bs * 8);
    for (int host_tiles = 0; host_tiles < 2; ++host_tiles) {
      const size_t tiles = host_tiles ? (size_t)R * bt : (size_t)tasks * bt;
      size_t room = SIZE_MAX;
      if (budget) {
        if (fixed + tiles >= budget) continue;
        room = budget - fixed - tiles;
      }
      const int64_t pr = shrink(std::max<int64_t>(256, ((int64_t)1 << 30) / (2 * bs * 4)),
                                [&](int64_t r) { return gram_area(bs, r); }, room);
      const int64_t ur = shrink(std::max<int64_t>(256, ((int64_t)1 << 30) / (n * 4)), u_area, room);
      if (!pr || !ur) continue;
      p->tb = bs;
      p->n_panels = nb;
      p->n_tasks = tasks;
      p->tiles_host = host_tiles != 0;
      p->b_tile = bt;
      p->pan_rows = std::min(pr, m);
      p->o_tiles = c.take(tiles);
      const size_t o_phase = c.take(std::max(gram_area(bs, p->pan_rows), u_area(ur)));
      // Gram tasks: task tile, tensor-core scratch, panel ring
      p->o_Gt = o_phase;
      size_t off = o_phase + al((size_t)bs * 2 * bs * 8);
      p->b_gscr = prec != TSVD_GRAM_FP32 ? gram_tc_scratch_bytes(p->pan_rows, 2 * bs, prec) : 0;
      p->o_gscr = off;
      if (prec != TSVD_GRAM_FP32) off += p->b_gscr + 256;
      p->b_pan = al((size_t)p->pan_rows * 2 * bs * 4);
      p->o_pan = off;
      // U pass: row-block ring (host A), then the U staging
      p->mode = host_a ? MODE_STREAM : MODE_DEVICE;
      p->chunk_rows = std::min(ur, m);
      p->n_chunks = ceil_div(m, p->chunk_rows);
      p->b_slot = host_a ? al((size_t)p->chunk_rows * n * 4) : 0;
      p->o_ring = o_phase;
      if (host_u) {
        p->b_ubuf = al((size_t)p->chunk_rows * k * 4);
        p->o_ubuf = o_phase + (host_a ? (size_t)R * p->b_slot : 0);
      }
      p->ws = c.off;
      return TSVD_OK;
    }
  }
  return TSVD_EBUDGET;
}

tsvd_status plan_csr(tsvd_plan_s *p, const tsvd_matrix *A) {
  const int64_t n = p->n, k = p->k, m = p->m;
  if (k + 4 > kVecPartStride) return TSVD_EUNSUPPORTED;
  p->avg_nnz = m > 0 ? (double)p->nnz / (double)m : 0.0;
  Carve c;
  p->o_v = c.take((size_t)n * 4);
  p->o_vn = c.take((size_t)n * 4);
  p->o_w = c.take((size_t)n * 4);
  p->o_x64 = c.take((size_t)n * 8);
  p->o_Vr = c.take((size_t)n * k * 4);
  p->o_sig2 = c.take((size_t)k * 8);
  p->o_sigma = c.take((size_t)k * 8);
  p->o_info = c.take((size_t)k * 4 * sizeof(int32_t));
  p->o_flag = c.take(256);
  p->vec_grid = 1024;
  p->o_vsc = c.take(vec_scratch_bytes(p->vec_grid));
  const size_t fixed = c.off;
  const bool host_a = p->location == TSVD_HOST;
  const bool host_u = p->opt.out_location == TSVD_HOST;
  const int R = p->n_buffers;
  int64_t rows = p->opt.block_rows > 0 ? p->opt.block_rows : std::min<int64_t>(m, (int64_t)1 << 20);
  rows = std::max<int64_t>(1, std::min<int64_t>(rows, m));
  const size_t budget = p->opt.device_budget;
  const size_t resident_bytes = (size_t)round_up((m + 1) * 8, 256) + 2 * (size_t)round_up(std::max<int64_t>(p->nnz, 1) * 4, 256);
  // v and w together beyond ~64 MB (half of L2): the column-chunked operator, with
  // chunks of at most ~40 MB of v (or w)
  if ((int64_t)n * 8 > ((int64_t)64 << 20)) {
    p->csr_nch = (int)std::min<int64_t>(8, std::max<int64_t>(2, ceil_div((int64_t)n * 4, (int64_t)40 << 20)));
    p->csr_cw = ceil_div(n, p->csr_nch);
  }
  const int nch = p->csr_nch;
  auto split_bytes = [&](int64_t r) -> size_t { return nch ? (size_t)round_up(r * (nch - 1) * 4, 256) : 0; };
  auto slot_bytes = [&](int64_t r, int64_t maxnnz) -> size_t {
    return (size_t)round_up((r + 1) * 8, 256) + 2 * (size_t)round_up(std::max<int64_t>(maxnnz, 1) * 4, 256) +
           split_bytes(r);
  };
  auto max_nnz_of = [&](int64_t r) -> int64_t {
    if (!host_a) return 0;
    int64_t mx = 0;
    for (int64_t s = 0; s < m; s += r) mx = std::max(mx, A->row_ptr[std::min(m, s + r)] - A->row_ptr[s]);
    return mx;
  };
  int mode = MODE_DEVICE;
  if (host_a) {
    mode = MODE_STREAM;
    const size_t ucost = host_u ? 2 * (size_t)round_up(rows * k * 4, 256) : 0;
    if (!p->opt.force_stream && (budget == 0 || fixed + resident_bytes + ucost <= budget)) mode = MODE_RESIDENT;
  }
  int64_t maxnnz = mode == MODE_STREAM ? max_nnz_of(rows) : 0;
  if (budget) {
    auto total = [&](int64_t r, int64_t mx) -> size_t {
      size_t s = fixed + (host_u ? 2 * (size_t)round_up(r * k * 4, 256) : 0);
      if (mode == MODE_STREAM) s += R * slot_bytes(r, mx) + (nch ? (size_t)round_up(r * 4, 256) : 0);
      if (mode == MODE_RESIDENT) s += resident_bytes;
      if (mode != MODE_STREAM && nch) s += (size_t)round_up(m * 4, 256) + split_bytes(m);
      return s;
    };
    while (rows > 1024 && total(rows, maxnnz) > budget) {
      rows = (rows + 1) / 2;
      if (mode == MODE_STREAM) maxnnz = max_nnz_of(rows);
    }
    if (total(rows, maxnnz) > budget) return TSVD_EBUDGET;
  }
  p->mode = mode;
  p->chunk_rows = rows;
  partition_rows(m, rows, p->block_start);
  p->n_chunks = (int64_t)p->block_start.size() - 1;
  p->max_block_nnz = maxnnz;
  if (mode == MODE_STREAM) {
    p->b_slot = slot_bytes(rows, maxnnz);
    p->b_split_slot = split_bytes(rows);
    p->o_ring = c.take(p->b_slot * R);
  }
  if (mode == MODE_RESIDENT) p->o_res = c.take(resident_bytes);
  if (host_u) {
    p->b_ubuf = (size_t)round_up(rows * k * 4, 256);
    p->o_ubuf = c.take(2 * p->b_ubuf);
  }
  if (nch) {
    // y of the rows a pass covers, and (in core) every row's split points
    p->o_csr_y = c.take((size_t)(mode == MODE_STREAM ? rows : m) * 4);
    if (mode != MODE_STREAM) p->o_csr_split = c.take(split_bytes(m));
  }
  p->ws = c.off;
  if (budget && p->ws > budget) return TSVD_EBUDGET;
  return TSVD_OK;
}

}  // namespace

extern "C" {

const char *tsvd_status_string(tsvd_status s) {
  switch (s) {
    case TSVD_OK: return "ok";
    case TSVD_EINVAL: return "invalid argument";
    case TSVD_ENOMEM: return "host allocation failed";
    case TSVD_EBUDGET: return "device budget or workspace too small";
    case TSVD_ECUDA: return "CUDA error";
    case TSVD_ETIMEDOUT: return "bounded wait timed out";
    case TSVD_ENOCONV: return "iteration cap reached before convergence";
    case TSVD_ERANK: return "matrix rank below k";
    case TSVD_EUNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

const char *tsvd_last_cuda_error(void) { return g_err.c_str(); }
int32_t tsvd_abi_version(void) { return TSVD_ABI_VERSION; }

void tsvd_options_init(tsvd_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof *opt);
  opt->n_buffers = 3;
  opt->precision = TSVD_GRAM_FP32;
  opt->max_iter = 10000;
  opt->out_location = TSVD_HOST;
}

tsvd_status tsvd_plan(tsvd_plan_t *out, const tsvd_matrix *A, int64_t k, double eps,
                      const tsvd_options *opt_in, size_t *workspace_bytes) {
  if (!out || !A || !workspace_bytes) return TSVD_EINVAL;
  *out = nullptr;
  *workspace_bytes = 0;
  tsvd_options opt;
  if (opt_in) opt = *opt_in; else tsvd_options_init(&opt);
  bool csr_sorted = true;
  if (A->kind != TSVD_DENSE_F32_ROWMAJOR && A->kind != TSVD_CSR_F32_I32_I64) return TSVD_EINVAL;
  if (A->location != TSVD_HOST && A->location != TSVD_DEVICE) return TSVD_EINVAL;
  if (A->m <= 0 || A->n <= 0) return TSVD_EINVAL;
  const int64_t mn = std::min(A->m, A->n);
  if (k == -1) k = mn;
  if (k < 1 || k > mn) return TSVD_EINVAL;
  if (!opt.iters_override && !(eps > 0.0 && eps < 1.0)) return TSVD_EINVAL;
  if (opt.n_buffers == 0) opt.n_buffers = 3;
  if (opt.n_buffers < 2 || opt.n_buffers > 64) return TSVD_EINVAL;
  if (opt.precision < TSVD_GRAM_FP32 || opt.precision > TSVD_GRAM_BF16X3) return TSVD_EINVAL;
  if (opt.max_iter <= 0) opt.max_iter = 10000;
  if (opt.out_location != TSVD_HOST && opt.out_location != TSVD_DEVICE) return TSVD_EINVAL;
  if (opt.block_rows < 0) return TSVD_EINVAL;
  if (opt.power_kernel < TSVD_POWER_AUTO || opt.power_kernel > TSVD_POWER_CLUSTER) return TSVD_EINVAL;
  if (opt.gram_tile < 0 || opt.gram_tile % 256 != 0) return TSVD_EINVAL;
  if (opt.power_ctas != 0 && opt.power_ctas != 1 && opt.power_ctas != 2 && opt.power_ctas != 4 &&
      opt.power_ctas != 8)
    return TSVD_EINVAL;
  if (opt.gram_tile > 0 && A->kind != TSVD_DENSE_F32_ROWMAJOR) return TSVD_EINVAL;
  if (opt.wait_limit_ns < 0 || opt.csr_coop_blocks < 0) return TSVD_EINVAL;
  const bool cluster_fits = A->kind == TSVD_DENSE_F32_ROWMAJOR && mn <= kSrvMaxDim && k <= kSrvMaxK;
  if (opt.power_kernel == TSVD_POWER_CLUSTER && !cluster_fits) {
    set_error_text("tsvd_plan: the cluster power kernel takes dense A with n <= " + std::to_string(kSrvMaxDim) +
                   " and k <= " + std::to_string(kSrvMaxK));
    return TSVD_EUNSUPPORTED;
  }
  if (A->kind == TSVD_DENSE_F32_ROWMAJOR) {
    if (!A->values || A->ld < A->n) return TSVD_EINVAL;
  } else {
    if (A->nnz < 0 || !A->row_ptr) return TSVD_EINVAL;
    if (A->nnz > 0 && (!A->col_idx || !A->values)) return TSVD_EINVAL;
    if (A->n > 0x7fffffffLL) return TSVD_EUNSUPPORTED;
    if (A->location == TSVD_HOST) TSVD_TRY(validate_csr_host(A, &csr_sorted));
  }
  // the CSR path applies A^T (A v) on R^n and needs m >= n; dense m < n takes Eq. 3
  if (A->kind == TSVD_CSR_F32_I32_I64 && A->m < A->n) return TSVD_EUNSUPPORTED;
  if (A->kind == TSVD_DENSE_F32_ROWMAJOR && A->n > 32768) return TSVD_EUNSUPPORTED;
  if (opt.iters_override) {
    for (int64_t l = 0; l < k; ++l)
      if (opt.iters_override[l] <= 0) return TSVD_EINVAL;
  }

  tsvd_plan_s *p = new (std::nothrow) tsvd_plan_s();
  if (!p) return TSVD_ENOMEM;
  try {
    p->kind = A->kind;
    p->location = A->location;
    p->csr_sorted = csr_sorted;
    p->m = A->m;
    p->n = A->n;
    p->ld = A->kind == TSVD_DENSE_F32_ROWMAJOR ? A->ld : 0;
    p->nnz = A->nnz;
    p->k = k;
    p->eps = eps;
    p->opt = opt;
    p->wide = A->kind == TSVD_DENSE_F32_ROWMAJOR && A->m < A->n;
    p->d = std::min(A->m, A->n);
    p->K = std::max(A->m, A->n);
    p->n_buffers = opt.n_buffers;
    if (opt.iters_override) p->iters_override.assign(opt.iters_override, opt.iters_override + k);
    if (opt.start_draws) p->start_draws.assign(opt.start_draws, opt.start_draws + (size_t)mn * k);
    p->opt.iters_override = nullptr;
    p->opt.start_draws = nullptr;
    p->cluster_power = A->kind == TSVD_DENSE_F32_ROWMAJOR &&
                       (opt.power_kernel == TSVD_POWER_CLUSTER ||
                        (opt.power_kernel == TSVD_POWER_AUTO && cluster_fits));
  } catch (...) {
    delete p;
    return TSVD_ENOMEM;
  }
  tsvd_status st = p->kind == TSVD_DENSE_F32_ROWMAJOR ? plan_dense(p) : plan_csr(p, A);
  if (st != TSVD_OK) {
    delete p;
    return st;
  }
  *workspace_bytes = p->ws;
  *out = p;
  return TSVD_OK;
}

void tsvd_destroy(tsvd_plan_t p) {
  if (!p) return;
  int cur = -1;
  if (p->device >= 0 && cudaGetDevice(&cur) == cudaSuccess) {
    if (cur != p->device) cudaSetDevice(p->device);
    for (auto e : p->ev_ready) cudaEventDestroy(e);
    for (auto e : p->ev_free) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
      if (p->ev_u_ready[i]) cudaEventDestroy(p->ev_u_ready[i]);
      if (p->ev_u_free[i]) cudaEventDestroy(p->ev_u_free[i]);
    }
    for (auto e : p->ev_t)
      if (e) cudaEventDestroy(e);
    for (auto e : p->ev_k) cudaEventDestroy(e);
    for (auto e : p->ev_c) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->copy_stream2) cudaStreamDestroy(p->copy_stream2);
    if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
    if (p->ev_aux) cudaEventDestroy(p->ev_aux);
    if (p->ev_csplit) cudaEventDestroy(p->ev_csplit);
    if (p->ev_cjoin) cudaEventDestroy(p->ev_cjoin);
    if (p->d2h_stream) cudaStreamDestroy(p->d2h_stream);
    if (p->host_tiles) pinned_free(p->host_tiles);
    if (cur != p->device) cudaSetDevice(cur);
  }
  delete p;
}

}  // extern "C"

// ---------------------------------------------------------------- factor
namespace {

tsvd_status ensure_runtime(tsvd_plan_s *p) {
  int dev = -1;
  TSVD_CUDA(cudaGetDevice(&dev));
  if (p->device == dev) return TSVD_OK;
  if (p->device >= 0) return TSVD_EINVAL;  // a plan serves one device
  p->device = dev;
  TSVD_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
  TSVD_CUDA(cudaStreamCreateWithFlags(&p->copy_stream2, cudaStreamNonBlocking));
  TSVD_CUDA(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
  TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_aux, cudaEventDisableTiming));
  TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_csplit, cudaEventDisableTiming));
  TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_cjoin, cudaEventDisableTiming));
  TSVD_CUDA(cudaStreamCreateWithFlags(&p->d2h_stream, cudaStreamNonBlocking));
  p->ev_ready.resize(p->n_buffers, nullptr);
  p->ev_free.resize(p->n_buffers, nullptr);
  for (int i = 0; i < p->n_buffers; ++i) {
    TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_ready[i], cudaEventDisableTiming));
    TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_free[i], cudaEventDisableTiming));
  }
  for (int i = 0; i < 2; ++i) {
    TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_u_ready[i], cudaEventDisableTiming));
    TSVD_CUDA(cudaEventCreateWithFlags(&p->ev_u_free[i], cudaEventDisableTiming));
  }
  for (int i = 0; i < 4; ++i) TSVD_CUDA(cudaEventCreate(&p->ev_t[i]));
  return TSVD_OK;
}

struct Run {
  tsvd_plan_s *p;
  const tsvd_matrix *A;
  unsigned char *ws;
  cudaStream_t cs;
  double h2d = 0.0, d2h = 0.0;
  int64_t chunk_seq = 0;  // ring position, continues across passes
  int32_t left_err = 0;   // the left kernels' status word after the pass (read back on the stream)
  int64_t copies = 0;     // timed block copies recorded so far
  std::vector<double> copy_bytes;  // bytes of each timed copy
  std::vector<int64_t> copy_first; // first contraction index (row, or column of a wide A) of each timed copy
  double kernel_ms = 0.0;          // timed operator kernels (CSR pair)
  int64_t kernel_launches = 0;
  bool chunked = false;            // this factorisation uses the column-chunked CSR operator
};

// Events around a block copy on the copy stream (only with time_kernels).
tsvd_status copy_event(Run &r, bool start) {
  tsvd_plan_s *p = r.p;
  if (!p->opt.time_kernels) return TSVD_OK;
  const size_t idx = (size_t)(2 * r.copies + (start ? 0 : 1));
  while (p->ev_c.size() <= idx) {
    cudaEvent_t e;
    TSVD_CUDA(cudaEventCreate(&e));
    p->ev_c.push_back(e);
  }
  TSVD_CUDA(cudaEventRecord(p->ev_c[idx], p->copy_stream));
  if (!start) ++r.copies;
  return TSVD_OK;
}

tsvd_status copy_time_ms(Run &r, double *ms, double *min_gbps, double *max_gbps) {
  *ms = 0.0;
  *min_gbps = 0.0;
  *max_gbps = 0.0;
  for (int64_t c = 0; c < r.copies; ++c) {
    float t = 0.f;
    TSVD_CUDA(cudaEventElapsedTime(&t, r.p->ev_c[2 * c], r.p->ev_c[2 * c + 1]));
    *ms += t;
    if (t > 0.f) {
      const double g = r.copy_bytes[(size_t)c] / ((double)t * 1e6);
      if (c == 0 || g < *min_gbps) *min_gbps = g;
      if (g > *max_gbps) *max_gbps = g;
    }
  }
  return TSVD_OK;
}

// Bring dense block [r0, r0+rows) of the contraction index to the device (rows
// of a tall A; columns of a wide A, all m rows of them); returns the pointer /
// stride to use on the compute stream.  The slot is released by release_slot().
tsvd_status acquire_dense(Run &r, int64_t r0, int64_t rows, const float **out, int64_t *ldo, int *slot,
                          bool resident_fill) {
  tsvd_plan_s *p = r.p;
  const tsvd_matrix *A = r.A;
  const bool wide = p->wide;
  *slot = -1;
  if (p->mode == MODE_DEVICE) {
    *out = wide ? A->values + r0 : A->values + r0 * A->ld;
    *ldo = A->ld;
    return TSVD_OK;
  }
  // destination and its row stride: the resident copy of A (m x n, stride n), or a ring slot
  // (a tall block: rows x n, stride n; a wide block: m x rows, stride chunk_rows)
  float *dst;
  int64_t ldd;
  if (p->mode == MODE_RESIDENT) {
    float *res = reinterpret_cast<float *>(r.ws + p->o_res);
    dst = wide ? res + r0 : res + r0 * p->n;
    ldd = p->n;
    *out = dst;
    *ldo = ldd;
    if (!resident_fill) return TSVD_OK;
  } else {
    const int s = (int)(r.chunk_seq++ % p->n_buffers);
    *slot = s;
    dst = reinterpret_cast<float *>(r.ws + p->o_ring + p->b_slot * s);
    ldd = wide ? p->chunk_rows : p->n;
    TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_free[s], 0));
    *out = dst;
    *ldo = ldd;
  }
  // copy height x width floats: a tall block is rows x n, a wide block m x rows
  const int64_t height = wide ? p->m : rows, width = wide ? rows : p->n;
  const float *src = wide ? A->values + r0 : A->values + r0 * A->ld;
  TSVD_TRY(copy_event(r, true));
  // the block in two halves on two copy streams: host memory that a single copy
  // drains slowly (seen on some hosts for parts of a large pinned allocation)
  // gets two copy engines; the halves join on the first stream
  const int64_t h0 = height / 2, h1 = height - h0;
  TSVD_CUDA(cudaEventRecord(p->ev_csplit, p->copy_stream));
  TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream2, p->ev_csplit, 0));
  for (int half = 0; half < 2; ++half) {
    const int64_t rr0 = half ? h0 : 0, rr = half ? h1 : h0;
    if (rr == 0) continue;
    cudaStream_t cst = half ? p->copy_stream2 : p->copy_stream;
    if (A->ld == width && ldd == width) {
      TSVD_CUDA(cudaMemcpyAsync(dst + rr0 * ldd, src + rr0 * A->ld, (size_t)rr * width * 4, cudaMemcpyHostToDevice,
                                cst));
    } else {
      TSVD_CUDA(cudaMemcpy2DAsync(dst + rr0 * ldd, (size_t)ldd * 4, src + rr0 * A->ld, (size_t)A->ld * 4,
                                  (size_t)width * 4, (size_t)rr, cudaMemcpyHostToDevice, cst));
    }
  }
  TSVD_CUDA(cudaEventRecord(p->ev_cjoin, p->copy_stream2));
  TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_cjoin, 0));
  TSVD_TRY(copy_event(r, false));
  if (p->opt.time_kernels) {
    r.copy_bytes.push_back((double)height * width * 4);
    r.copy_first.push_back(r0);
  }
  r.h2d += (double)height * width * 4;
  const int ev = *slot >= 0 ? *slot : 0;
  TSVD_CUDA(cudaEventRecord(p->ev_ready[ev], p->copy_stream));
  TSVD_CUDA(cudaStreamWaitEvent(r.cs, p->ev_ready[ev], 0));
  return TSVD_OK;
}

tsvd_status release_slot(Run &r, int slot) {
  if (slot >= 0) TSVD_CUDA(cudaEventRecord(r.p->ev_free[slot], r.cs));
  return TSVD_OK;
}

tsvd_status gram_dispatch(const float *A, int64_t rows, int64_t n, int64_t ld, double *G, int prec,
                          void *scr, size_t scr_bytes, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                          cudaEvent_t ev1 = nullptr, bool reset_status = true, bool trans = false,
                          uint64_t wait_ns = 0) {
  if (trans) {
    // a column block of a wide A: X[r][c] = A[c ld + r], Gram X^T X (Eq. 3)
    if (prec == TSVD_GRAM_FP32) {
      if (ev0) TSVD_CUDA(cudaEventRecord(ev0, s));
      TSVD_TRY(launch_gram_simt_t(A, rows, n, ld, G, s));
      if (ev1) TSVD_CUDA(cudaEventRecord(ev1, s));
      return TSVD_OK;
    }
    return launch_gram_tc_t(A, rows, n, ld, G, prec, scr, scr_bytes, s, ev0, ev1, reset_status, wait_ns);
  }
  if (prec == TSVD_GRAM_FP32) return launch_gram_simt(A, rows, n, ld, G, s, ev0, ev1);
  return launch_gram_tc(A, rows, n, ld, G, prec, scr, scr_bytes, s, ev0, ev1, reset_status, wait_ns);
}

// The other factor, one pass over A (Alg. 1): OUT = A P
// Sigma^-1 for a tall A (P = V, OUT = U) or A^T P Sigma^-1 for a wide A
// (P = U from A A^T, OUT = V); P is d x k and OUT is K x k, both column-major.
tsvd_status left_pass_dense(Run &r, const float *P32, const double *sigma, float *OUT) {
  tsvd_plan_s *p = r.p;
  const bool host_u = p->opt.out_location == TSVD_HOST;
  const int64_t d = p->d, K = p->K, k = p->k;
  // In the streamed mode the last n_buffers blocks of the Gram pass are
  // still in the ring (block c in slot c % n_buffers): use them first, then
  // stream the others through the slots they free.
  // (Not after an orthogonally batched Gram: its ring held column panels.)
  const int64_t nc = p->n_chunks;
  const bool reuse = p->mode == MODE_STREAM && !p->tiled;
  int *lst = nullptr;
  TSVD_TRY(left_status_word(&lst));
  TSVD_CUDA(cudaMemsetAsync(lst, 0, 4, r.cs));
  const int64_t first_res = reuse ? std::max<int64_t>(0, nc - p->n_buffers) : nc;
  auto kernel = [&](const float *Ab, int64_t rows, int64_t ldb, float *dst, int64_t ldo) -> tsvd_status {
    if (p->wide) return launch_left_trans(Ab, rows, d, ldb, P32, d, k, sigma, dst, ldo, r.cs);
    return launch_left_dense(Ab, rows, d, ldb, P32, d, k, sigma, dst, ldo, r.cs);
  };
  for (int64_t idx = 0; idx < nc; ++idx) {
    const int64_t c = reuse ? (idx < nc - first_res ? first_res + idx : idx - (nc - first_res)) : idx;
    const int64_t r0 = c * p->chunk_rows, rows = std::min(p->chunk_rows, K - r0);
    const float *Ab;
    int64_t ldb;
    int slot;
    if (reuse && c >= first_res) {
      slot = (int)(c % p->n_buffers);
      Ab = reinterpret_cast<const float *>(r.ws + p->o_ring + p->b_slot * slot);
      ldb = p->wide ? p->chunk_rows : p->n;
    } else {
      TSVD_TRY(acquire_dense(r, r0, rows, &Ab, &ldb, &slot, false));
    }
    if (!host_u) {
      TSVD_TRY(kernel(Ab, rows, ldb, OUT + r0, K));
      TSVD_TRY(release_slot(r, slot));
    } else {
      const int b = (int)(idx & 1);
      float *ub = reinterpret_cast<float *>(r.ws + p->o_ubuf + p->b_ubuf * b);
      TSVD_CUDA(cudaStreamWaitEvent(r.cs, p->ev_u_free[b], 0));
      TSVD_TRY(kernel(Ab, rows, ldb, ub, rows));
      TSVD_TRY(release_slot(r, slot));
      TSVD_CUDA(cudaEventRecord(p->ev_u_ready[b], r.cs));
      TSVD_CUDA(cudaStreamWaitEvent(p->d2h_stream, p->ev_u_ready[b], 0));
      TSVD_CUDA(cudaMemcpy2DAsync(OUT + r0, (size_t)K * 4, ub, (size_t)rows * 4, (size_t)rows * 4, (size_t)k,
                                  cudaMemcpyDeviceToHost, p->d2h_stream));
      r.d2h += (double)rows * k * 4;
      TSVD_CUDA(cudaEventRecord(p->ev_u_free[b], p->d2h_stream));
    }
  }
  TSVD_CUDA(cudaMemcpyAsync(&r.left_err, lst, 4, cudaMemcpyDeviceToHost, r.cs));
  return TSVD_OK;
}

// Power phase of a dense plan on one thread-block cluster: all k triplets in
// one launch (Alg. 1 loop over l, Alg. 2 per triplet, Hotelling deflation of
// the full FP64 G64 and its FP32 copy row by row), writing V64, V32, sig2,
// sigma and info.  The descriptor, the forced counts and the completion word
// sit at the start of the power scratch, which the grid kernel would use.
tsvd_status power_cluster_dense(Run &r, double *G64, float *G32, double *V64, float *V32, double *sig2,
                                double *sigma, int32_t *info, void *pscr) {
  tsvd_plan_s *p = r.p;
  const int64_t n = p->d, k = p->k;  // the Gram's dimension
  unsigned char *base = static_cast<unsigned char *>(pscr);
  SrvReq *dq = reinterpret_cast<SrvReq *>(base);
  int32_t *d_iters = reinterpret_cast<int32_t *>(base + round_up(sizeof(SrvReq), 256));
  uint32_t *d_flag = reinterpret_cast<uint32_t *>(base + round_up(sizeof(SrvReq), 256) + 256);
  static_assert(kSrvMaxK * 4 <= 256, "forced counts fit their slot");
  if ((size_t)round_up(sizeof(SrvReq), 256) + 512 > p->b_pscr) return TSVD_EINVAL;

  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  const size_t static_bytes = 24 * 1024;  // the kernel's static shared arrays, rounded up
  const size_t cap = di.smem_optin > static_bytes ? di.smem_optin - static_bytes : 0;
  const int C = srv_clamp_cluster(n, p->opt.power_ctas > 0 ? p->opt.power_ctas : 8);
  const int resident = srv_power_smem(n, C, 1) <= cap ? 1 : 0;
  const size_t smem = srv_power_smem(n, C, resident);
  if (smem > cap) return TSVD_EUNSUPPORTED;

  if (!p->start_draws.empty()) {
    // the kernel reads x_l from column l of V64 before the triplet overwrites it
    TSVD_CUDA(cudaMemcpyAsync(V64, p->start_draws.data(), (size_t)n * k * 8, cudaMemcpyHostToDevice, r.cs));
    r.h2d += (double)n * k * 8;
  }
  if (!p->iters_override.empty())
    TSVD_CUDA(cudaMemcpyAsync(d_iters, p->iters_override.data(), (size_t)k * 4, cudaMemcpyHostToDevice, r.cs));
  SrvReq &q = p->srv_req;
  q = SrvReq{};
  q.A = nullptr;  // the other factor is the left pass's
  q.m = p->K;  // the kernel reads d = n of a tall descriptor; the other factor is not formed here
  q.n = n;
  q.trans = 0;
  q.k = (int32_t)k;
  q.G64 = G64;
  q.G32 = G32;
  q.V64 = V64;
  q.sig2 = sig2;
  q.info = info;
  q.vout = V32;
  q.eps = p->eps;
  q.max_iter = p->opt.max_iter;
  q.sign_convention = p->opt.sign_convention;
  q.iters_override = p->iters_override.empty() ? nullptr : d_iters;
  const uint64_t key = splitmix64(p->opt.seed);
  q.key0 = (uint32_t)key;
  q.key1 = (uint32_t)(key >> 32);
  q.cluster = C;
  q.resident = resident;
  q.oU = nullptr;
  q.oV = V32;  // the epilogue's copy of the power vectors lands on itself
  q.oS = sigma;
  q.oInfo = info;
  q.flag = d_flag;
  q.ticket = 1;
  q.no_other = 1;
  q.x_start = p->start_draws.empty() ? nullptr : V64;
  if (!srv_req_complete(q)) return TSVD_EINVAL;
  // pageable source: the copy is staged before the call returns; the plan
  // keeps the host copy alive anyway
  TSVD_CUDA(cudaMemcpyAsync(dq, &q, sizeof(SrvReq), cudaMemcpyHostToDevice, r.cs));
  return launch_srv_power(dq, 1, C, smem, r.cs);
}

tsvd_status factor_dense(Run &r, float *U, double *sigma_out, float *V_out, tsvd_report *rep) {
  tsvd_plan_s *p = r.p;
  const int64_t n = p->d, k = p->k;  // the Gram's dimension (n for a tall A, m for a wide one)
  // the power method's vectors and the other factor (Alg. 1)
  float *P_out = p->wide ? U : V_out;
  float *O_out = p->wide ? V_out : U;
  unsigned char *ws = r.ws;
  double *G64 = reinterpret_cast<double *>(ws + p->o_G64);
  float *G32 = reinterpret_cast<float *>(ws + p->o_G32);
  double *V64 = reinterpret_cast<double *>(ws + p->o_V64);
  float *V32 = reinterpret_cast<float *>(ws + p->o_V32);
  double *sig2 = reinterpret_cast<double *>(ws + p->o_sig2);
  double *sigma = reinterpret_cast<double *>(ws + p->o_sigma);
  int32_t *info = reinterpret_cast<int32_t *>(ws + p->o_info);
  void *pscr = ws + p->o_pscr;
  void *gscr = ws + p->o_gscr;

  const bool timed = p->opt.time_kernels != 0;
  if (timed && (int64_t)p->ev_k.size() < 2 * p->n_gram_launches) {
    const size_t have = p->ev_k.size();
    p->ev_k.resize(2 * p->n_gram_launches, nullptr);
    for (size_t i = have; i < p->ev_k.size(); ++i) TSVD_CUDA(cudaEventCreate(&p->ev_k[i]));
  }
  TSVD_CUDA(cudaEventRecord(p->ev_t[0], r.cs));
  // ---- Gram pass: B = sum_b A_b^T A_b
  TSVD_CUDA(cudaMemsetAsync(G64, 0, (size_t)n * n * 8, r.cs));
  // status word of the tensor-core scratch, zeroed once for the whole pass
  // (the 256-byte aligned scratch starts with its status word)
  if (p->opt.precision != TSVD_GRAM_FP32) TSVD_CUDA(cudaMemsetAsync(gscr, 0, 4, r.cs));
  int64_t gl = 0;  // Gram launches so far
  for (int64_t c = 0; c < p->n_chunks; ++c) {
    const int64_t r0 = c * p->chunk_rows, rows = std::min(p->chunk_rows, p->K - r0);
    const float *Ab;
    int64_t ldb;
    int slot;
    TSVD_TRY(acquire_dense(r, r0, rows, &Ab, &ldb, &slot, true));
    // the block in launches of gram_rows contraction indices (rows of a tall
    // block, columns of a wide one)
    for (int64_t s0 = 0; s0 < rows; s0 += p->gram_rows, ++gl) {
      const int64_t sr = std::min(p->gram_rows, rows - s0);
      const float *As = p->wide ? Ab + s0 : Ab + s0 * ldb;
      TSVD_TRY(gram_dispatch(As, sr, n, ldb, G64, p->opt.precision, gscr, p->b_gscr, r.cs,
                             timed ? p->ev_k[2 * gl] : nullptr, timed ? p->ev_k[2 * gl + 1] : nullptr, false,
                             p->wide, (uint64_t)p->opt.wait_limit_ns));
    }
    TSVD_TRY(release_slot(r, slot));
  }
  int32_t gram_err = 0;
  if (p->opt.precision != TSVD_GRAM_FP32)
    TSVD_CUDA(cudaMemcpyAsync(&gram_err, gscr, 4, cudaMemcpyDeviceToHost, r.cs));
  // the cluster kernel reads and deflates full rows of G64: mirror its lower triangle too
  TSVD_TRY(launch_symmetrize(n, G64, G32, r.cs, p->cluster_power));
  TSVD_CUDA(cudaEventRecord(p->ev_t[1], r.cs));

  // ---- power phase: Alg. 1 loop over l, Alg. 2 per triplet (on the device)
  TSVD_CUDA(cudaMemsetAsync(info, 0, (size_t)k * 4 * sizeof(int32_t), r.cs));
  if (p->cluster_power) {
    TSVD_TRY(power_cluster_dense(r, G64, G32, V64, V32, sig2, sigma, info, pscr));
  }
  for (int64_t l = 0; l < k && !p->cluster_power; ++l) {
    double *x = V64 + l * n;
    if (!p->start_draws.empty()) {
      TSVD_CUDA(cudaMemcpyAsync(x, p->start_draws.data() + l * n, (size_t)n * 8, cudaMemcpyHostToDevice, r.cs));
      r.h2d += (double)n * 8;
    } else {
      TSVD_TRY(launch_start_draws(p->opt.seed, l, n, x, r.cs));
    }
    const int ovr = p->iters_override.empty() ? 0 : p->iters_override[l];
    TSVD_TRY(launch_power_dense(n, G32, G64, l ? V64 : nullptr, l ? sig2 : nullptr, l, x, p->eps,
                                p->opt.max_iter, ovr, p->opt.sign_convention, sig2 + l, info + 4 * l,
                                pscr, p->b_pscr, r.cs));
    // Hotelling deflation of the FP32 Gram copy for the next triplet
    if (l + 1 < k) TSVD_TRY(launch_gram_deflate(n, G64, G32, x, sig2 + l, r.cs));
  }
  if (!p->cluster_power) {
    TSVD_TRY(launch_sigma_from_sigma2(sig2, sigma, k, r.cs));
    TSVD_TRY(launch_f64_to_f32(V64, V32, n * k, r.cs));
  }
  TSVD_CUDA(cudaEventRecord(p->ev_t[2], r.cs));

  // ---- the other factor: U = A V diag(sigma)^-1, or V = A^T U diag(sigma)^-1 for a wide A
  // (a tall A skips it when U is NULL; a wide A always forms V)
  if (O_out) TSVD_TRY(left_pass_dense(r, V32, sigma, O_out));
  TSVD_CUDA(cudaEventRecord(p->ev_t[3], r.cs));

  // ---- outputs
  const cudaMemcpyKind kind = p->opt.out_location == TSVD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  TSVD_CUDA(cudaMemcpyAsync(sigma_out, sigma, (size_t)k * 8, kind, r.cs));
  if (P_out) TSVD_CUDA(cudaMemcpyAsync(P_out, V32, (size_t)n * k * 4, kind, r.cs));
  if (kind == cudaMemcpyDeviceToHost) r.d2h += (double)k * 8 + (P_out ? (double)n * k * 4 : 0.0);
  std::vector<int32_t> hinfo((size_t)k * 4);
  TSVD_CUDA(cudaMemcpyAsync(hinfo.data(), info, hinfo.size() * 4, cudaMemcpyDeviceToHost, r.cs));
  TSVD_CUDA(cudaStreamSynchronize(r.cs));
  TSVD_CUDA(cudaStreamSynchronize(p->d2h_stream));
  TSVD_CUDA(cudaStreamSynchronize(p->copy_stream));

  float t01 = 0, t12 = 0, t23 = 0;
  TSVD_CUDA(cudaEventElapsedTime(&t01, p->ev_t[0], p->ev_t[1]));
  TSVD_CUDA(cudaEventElapsedTime(&t12, p->ev_t[1], p->ev_t[2]));
  TSVD_CUDA(cudaEventElapsedTime(&t23, p->ev_t[2], p->ev_t[3]));
  if (timed && rep) {
    double sum = 0.0;
    for (int64_t c = 0; c < p->n_gram_launches; ++c) {
      float t = 0.f;
      TSVD_CUDA(cudaEventElapsedTime(&t, p->ev_k[2 * c], p->ev_k[2 * c + 1]));
      sum += t;
    }
    rep->gram_kernel_ms = sum;
    rep->gram_kernel_launches = (int32_t)p->n_gram_launches;
  }
  int flags = 0;
  int64_t apps = 0;
  if (gram_err || r.left_err) flags |= TSVD_FLAG_TIMEOUT;
  for (int64_t l = 0; l < k; ++l) {
    if (hinfo[4 * l + 2]) flags |= TSVD_FLAG_TIMEOUT;
    if (hinfo[4 * l + 1] == 1) flags |= TSVD_FLAG_NOCONV;
    if (hinfo[4 * l + 1] == 2) flags |= TSVD_FLAG_RANK;
    apps += hinfo[4 * l];
    if (rep && rep->iters) rep->iters[l] = hinfo[4 * l];
  }
  if (rep) {
    rep->gram_ms = t01;
    rep->power_ms = t12;
    rep->left_ms = t23;
    rep->total_ms = (double)t01 + t12 + t23;
    rep->applications = apps;
  }
  // sigma order check
  if (p->opt.out_location == TSVD_HOST) {
    for (int64_t l = 1; l < k; ++l)
      if (sigma_out[l] > sigma_out[l - 1]) flags |= TSVD_FLAG_NONMONOTONE;
  }
  if (rep) rep->flags |= flags;
  if (flags & TSVD_FLAG_TIMEOUT) return TSVD_ETIMEDOUT;
  if (flags & TSVD_FLAG_RANK) return TSVD_ERANK;
  if (flags & TSVD_FLAG_NOCONV) return TSVD_ENOCONV;
  return TSVD_OK;
}

// ---------------------------------------------------------------- CSR
struct CsrBlock {
  const int64_t *rp;
  const int32_t *ci;
  const float *va;
  int64_t rows;
  int slot;
  int32_t *split;  // streamed blocks: the slot's split-point buffer (chunked operator)
};

// flag bit 0: invalid structure; bit 1: some row's columns are not ascending
__global__ void csr_validate_kernel(int64_t m, int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                                    int *flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += (int64_t)gridDim.x * blockDim.x) {
    if (i == 0 && rp[0] != 0) atomicOr(flag, 1);
    if (i == m && rp[m] != nnz) atomicOr(flag, 1);
    if (i < m && rp[i + 1] < rp[i]) atomicOr(flag, 1);
    if (i < m && rp[i] >= 0 && rp[i + 1] <= nnz) {
      for (int64_t p = rp[i] + 1; p < rp[i + 1]; ++p)
        if (ci[p] < ci[p - 1]) {
          atomicOr(flag, 2);
          break;
        }
    }
  }
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    if (ci[p] < 0 || (int64_t)ci[p] >= n) atomicOr(flag, 1);
}

tsvd_status acquire_csr(Run &r, int64_t b, const std::vector<int64_t> &bnd_nnz, CsrBlock *out) {
  tsvd_plan_s *p = r.p;
  const tsvd_matrix *A = r.A;
  const int64_t s0 = p->block_start[b], s1 = p->block_start[b + 1];
  const int64_t e0 = bnd_nnz[b], e1 = bnd_nnz[b + 1];
  out->rows = s1 - s0;
  out->slot = -1;
  out->split = nullptr;
  if (p->mode == MODE_DEVICE) {
    out->rp = A->row_ptr + s0;
    out->ci = A->col_idx + e0;
    out->va = A->values + e0;
    return TSVD_OK;
  }
  if (p->mode == MODE_RESIDENT) {
    const int64_t *rp = reinterpret_cast<const int64_t *>(r.ws + p->o_res);
    const int32_t *ci = reinterpret_cast<const int32_t *>(r.ws + p->o_res + round_up((p->m + 1) * 8, 256));
    const float *va = reinterpret_cast<const float *>(r.ws + p->o_res + round_up((p->m + 1) * 8, 256) +
                                                      round_up(std::max<int64_t>(p->nnz, 1) * 4, 256));
    out->rp = rp + s0;
    out->ci = ci + e0;
    out->va = va + e0;
    return TSVD_OK;
  }
  const int s = (int)(r.chunk_seq++ % p->n_buffers);
  out->slot = s;
  unsigned char *base = r.ws + p->o_ring + p->b_slot * s;
  int64_t *rp = reinterpret_cast<int64_t *>(base);
  int32_t *ci = reinterpret_cast<int32_t *>(base + round_up((p->chunk_rows + 1) * 8, 256));
  float *va = reinterpret_cast<float *>(base + round_up((p->chunk_rows + 1) * 8, 256) +
                                        round_up(std::max<int64_t>(p->max_block_nnz, 1) * 4, 256));
  if (p->b_split_slot)
    out->split = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(va) +
                                             round_up(std::max<int64_t>(p->max_block_nnz, 1) * 4, 256));
  TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_free[s], 0));
  TSVD_TRY(copy_event(r, true));
  TSVD_CUDA(cudaMemcpyAsync(rp, A->row_ptr + s0, (size_t)(out->rows + 1) * 8, cudaMemcpyHostToDevice, p->copy_stream));
  if (e1 > e0) {
    // column indices and values on two copy streams, joined on the first
    TSVD_CUDA(cudaEventRecord(p->ev_csplit, p->copy_stream));
    TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream2, p->ev_csplit, 0));
    TSVD_CUDA(cudaMemcpyAsync(ci, A->col_idx + e0, (size_t)(e1 - e0) * 4, cudaMemcpyHostToDevice, p->copy_stream));
    TSVD_CUDA(cudaMemcpyAsync(va, A->values + e0, (size_t)(e1 - e0) * 4, cudaMemcpyHostToDevice, p->copy_stream2));
    TSVD_CUDA(cudaEventRecord(p->ev_cjoin, p->copy_stream2));
    TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_cjoin, 0));
  }
  TSVD_TRY(copy_event(r, false));
  const double bytes = (double)(out->rows + 1) * 8 + (double)(e1 - e0) * 8;
  if (p->opt.time_kernels) {
    r.copy_bytes.push_back(bytes);
    r.copy_first.push_back(s0);
  }
  r.h2d += bytes;
  TSVD_CUDA(cudaEventRecord(p->ev_ready[s], p->copy_stream));
  TSVD_CUDA(cudaStreamWaitEvent(r.cs, p->ev_ready[s], 0));
  out->rp = rp;
  out->ci = ci;
  out->va = va;
  return TSVD_OK;
}

// one application w += A^T (A v), ss += ||A v||^2 over all row blocks; with
// time_kernels each block's kernels are bracketed by events (read back by
// csr_kernel_time once the stream has been synchronised)
tsvd_status csr_apply(Run &r, const std::vector<int64_t> &bnd, const float *v, float *w, double *ss, int scatter) {
  tsvd_plan_s *p = r.p;
  const bool timed = p->opt.time_kernels != 0;
  if (r.chunked) {
    const int nch = p->csr_nch;
    float *y = reinterpret_cast<float *>(r.ws + p->o_csr_y);
    if (p->mode != MODE_STREAM) {
      // in core: chunk-major over every block, so each chunk of v (then of w) stays in L2
      const int32_t *split = reinterpret_cast<const int32_t *>(r.ws + p->o_csr_split);
      if (timed) TSVD_CUDA(cudaEventRecord(p->ev_k[0], r.cs));
      for (int pass = 0; pass < 2; ++pass) {
        // without the scatter (||A v||^2 only) the second pass is one sweep over y (chunk 0)
        const int nc = (pass == 1 && !scatter) ? 1 : nch;
        for (int c = 0; c < nc; ++c)
          for (int64_t b = 0; b < p->n_chunks; ++b) {
            CsrBlock blk;
            TSVD_TRY(acquire_csr(r, b, bnd, &blk));
            const int64_t r0 = p->block_start[b];
            if (pass == 0)
              TSVD_TRY(launch_csr_chunk_y(blk.rows, blk.rp, blk.ci, blk.va, split + r0 * (nch - 1), nch, c, v, y + r0,
                                          p->avg_nnz, r.cs));
            else
              TSVD_TRY(launch_csr_chunk_w(blk.rows, blk.rp, blk.ci, blk.va, split + r0 * (nch - 1), nch, c, y + r0, w,
                                          ss, scatter, p->avg_nnz, r.cs));
          }
      }
      if (timed) TSVD_CUDA(cudaEventRecord(p->ev_k[1], r.cs));
      return TSVD_OK;
    }
    for (int64_t b = 0; b < p->n_chunks; ++b) {
      CsrBlock blk;
      TSVD_TRY(acquire_csr(r, b, bnd, &blk));
      if (timed) TSVD_CUDA(cudaEventRecord(p->ev_k[2 * b], r.cs));
      TSVD_TRY(launch_csr_split(blk.rows, blk.rp, blk.ci, nch, p->csr_cw, blk.split, r.cs));
      for (int c = 0; c < nch; ++c)
        TSVD_TRY(launch_csr_chunk_y(blk.rows, blk.rp, blk.ci, blk.va, blk.split, nch, c, v, y, p->avg_nnz, r.cs));
      for (int c = 0; c < (scatter ? nch : 1); ++c)
        TSVD_TRY(launch_csr_chunk_w(blk.rows, blk.rp, blk.ci, blk.va, blk.split, nch, c, y, w, ss, scatter,
                                    p->avg_nnz, r.cs));
      if (timed) TSVD_CUDA(cudaEventRecord(p->ev_k[2 * b + 1], r.cs));
      TSVD_TRY(release_slot(r, blk.slot));
    }
    return TSVD_OK;
  }
  for (int64_t b = 0; b < p->n_chunks; ++b) {
    CsrBlock blk;
    TSVD_TRY(acquire_csr(r, b, bnd, &blk));
    if (timed) TSVD_CUDA(cudaEventRecord(p->ev_k[2 * b], r.cs));
    TSVD_TRY(launch_csr_pair(blk.rows, p->n, blk.rp, blk.ci, blk.va, v, w, ss, scatter, p->avg_nnz, r.cs));
    if (timed) TSVD_CUDA(cudaEventRecord(p->ev_k[2 * b + 1], r.cs));
    TSVD_TRY(release_slot(r, blk.slot));
  }
  return TSVD_OK;
}

// adds the durations of the last csr_apply's kernels (the stream must have been synchronised)
tsvd_status csr_kernel_time(Run &r) {
  tsvd_plan_s *p = r.p;
  if (!p->opt.time_kernels) return TSVD_OK;
  const int64_t pairs = (r.chunked && p->mode != MODE_STREAM) ? 1 : p->n_chunks;
  for (int64_t b = 0; b < pairs; ++b) {
    float t = 0.f;
    TSVD_CUDA(cudaEventElapsedTime(&t, p->ev_k[2 * b], p->ev_k[2 * b + 1]));
    r.kernel_ms += t;
    ++r.kernel_launches;
  }
  return TSVD_OK;
}

// Vectors of the power loop with an explicit operator (CSR, tiled Gram).
struct ExplicitLoop {
  float *v, *vn, *w;  // iterate, next iterate, operator output (n each)
  double *x64;        // FP64 start draws (n)
  double *ss;         // the operator's v^T G v (sigma pass)
  float *Vr;          // the vectors found so far, n x k row-major (ld k)
  float *Vcol;        // optional n x k column-major copy (ld n), or null
  double *sig2;       // k
  int32_t *info;      // 4 k
  VecScratch sc;
  int32_t *ctr;       // the current triplet's application counter (device)
};

// Alg. 1 loop over l with Alg. 2 per triplet, the operator B v applied
// explicitly (w = A^T A v or w = G v) and Hotelling's correction
// w -= V (sigma^2 . V^T v) (Eq. 2) in the vector kernels; the convergence
// test runs on the device and the host reads its decision after every
// application.  sigma_l^2 = v_l^T A^T A v_l from one more application.
// `batch` applications are queued per host round trip: an application that
// finds the triplet already stopped by an earlier one in the same batch
// changes nothing (the decision and the next-iterate kernels test the stop
// word against a device counter), so the trajectory is the same as with one
// round trip per application; the queued operator applications still run
// (they only write scratch), so batching is for cheap operators.  With
// `graph`, two consecutive applications (v -> v', v' -> v) are captured once
// per triplet into a CUDA graph and replayed, one launch instead of about a
// dozen per application; the operator must then be capturable (no host
// waits, no work on other streams).
// A whole triplet's loop in one launch: (buf0 = v0, buf1, l, forced count, rank scale, info)
using TripletLoop = std::function<tsvd_status(float *, float *, int64_t, int, double, int32_t *)>;

tsvd_status explicit_power_on(Run &r, ExplicitLoop &L,
                              const std::function<tsvd_status(const float *, float *, double *, int)> &apply,
                              const std::function<tsvd_status()> &after_sync, float *V_out, int *flags_out,
                              int64_t *apps_out, tsvd_report *rep, int batch, bool graph, const TripletLoop *coop);

tsvd_status explicit_power(Run &r, ExplicitLoop &L,
                           const std::function<tsvd_status(const float *, float *, double *, int)> &apply,
                           const std::function<tsvd_status()> &after_sync, float *V_out, int *flags_out,
                           int64_t *apps_out, tsvd_report *rep, int batch = 1, bool graph = false,
                           const TripletLoop *coop = nullptr) {
  if (!graph && !coop)
    return explicit_power_on(r, L, apply, after_sync, V_out, flags_out, apps_out, rep, batch, false, nullptr);
  // a capture cannot use the legacy default stream: then the loop runs on the plan's own
  // stream, ordered after and before the caller's work (any other stream is used as it is)
  tsvd_plan_s *p = r.p;
  cudaStream_t caller = r.cs;
  if (caller != nullptr && caller != cudaStreamLegacy && caller != cudaStreamPerThread)
    return explicit_power_on(r, L, apply, after_sync, V_out, flags_out, apps_out, rep, batch, graph, coop);
  TSVD_CUDA(cudaEventRecord(p->ev_aux, caller));
  TSVD_CUDA(cudaStreamWaitEvent(p->aux_stream, p->ev_aux, 0));
  r.cs = p->aux_stream;
  const tsvd_status st = explicit_power_on(r, L, apply, after_sync, V_out, flags_out, apps_out, rep, batch, graph, coop);
  r.cs = caller;
  TSVD_CUDA(cudaEventRecord(p->ev_aux, p->aux_stream));
  TSVD_CUDA(cudaStreamWaitEvent(caller, p->ev_aux, 0));
  return st;
}

tsvd_status explicit_power_on(Run &r, ExplicitLoop &L,
                              const std::function<tsvd_status(const float *, float *, double *, int)> &apply,
                              const std::function<tsvd_status()> &after_sync, float *V_out, int *flags_out,
                              int64_t *apps_out, tsvd_report *rep, int batch, bool graph, const TripletLoop *coop) {
  tsvd_plan_s *p = r.p;
  const int64_t n = p->n, k = p->k;
  float *v = L.v, *vn = L.vn;
  VecScratch sc = L.sc;
  std::vector<double> hsig2((size_t)k, 0.0);
  TSVD_CUDA(cudaMemsetAsync(L.info, 0, (size_t)k * 16, r.cs));
  int flags = 0;
  int64_t apps = 0;
  const bool host_out = p->opt.out_location == TSVD_HOST;
  for (int64_t l = 0; l < k; ++l) {
    // start vector v0 = x / ||x||
    if (!p->start_draws.empty()) {
      TSVD_CUDA(cudaMemcpyAsync(L.x64, p->start_draws.data() + l * n, (size_t)n * 8, cudaMemcpyHostToDevice, r.cs));
      r.h2d += (double)n * 8;
    } else {
      TSVD_TRY(launch_start_draws(p->opt.seed, l, n, L.x64, r.cs));
    }
    sc.info = L.info + 4 * l;
    TSVD_TRY(launch_vec_normalize_f64_to_f32(L.x64, v, n, sc, r.cs));
    const double rank_scale = l == 0 ? 1.0 : hsig2[0];
    const int ovr = p->iters_override.empty() ? 0 : p->iters_override[l];
    int32_t h[4] = {0, 0, 0, 0};
    // application e (1-based) reads buf[(e - 1) & 1] and writes buf[e & 1]
    float *buf[2] = {v, vn};
    TSVD_CUDA(cudaMemsetAsync(L.ctr, 0, 4, r.cs));
    // (the operator's v^T G v accumulates into L.ss here unread; the sigma pass clears it first)
    auto one = [&](const float *in, float *out) -> tsvd_status {
      TSVD_CUDA(cudaMemsetAsync(L.w, 0, (size_t)n * 4, r.cs));
      TSVD_TRY(apply(in, L.w, L.ss, 1));
      return launch_vec_deflate_step(n, L.Vr, k, L.sig2, l, in, L.w, out, p->eps, p->opt.max_iter, ovr, rank_scale,
                                     sc, 0, r.cs, L.ctr);
    };
    cudaGraphExec_t ge = nullptr;
    int64_t nodes = 0;
    if (coop) {
      // the whole loop of this triplet in one cooperative launch
      TSVD_TRY((*coop)(buf[0], buf[1], l, ovr, rank_scale, sc.info));
      TSVD_CUDA(cudaMemcpyAsync(h, sc.info, 16, cudaMemcpyDeviceToHost, r.cs));
      TSVD_CUDA(cudaStreamSynchronize(r.cs));
      TSVD_TRY(after_sync());
      if (h[3] == 0) return TSVD_ETIMEDOUT;  // a bounded barrier wait gave up before the triplet stopped
    }
    if (graph && !coop) {
      // the pair v -> v', v' -> v as one graph (the same for every pair of the triplet)
      const int64_t c0 = launches_so_far();
      TSVD_CUDA(cudaStreamBeginCapture(r.cs, cudaStreamCaptureModeThreadLocal));
      tsvd_status cst = one(buf[0], buf[1]);
      if (cst == TSVD_OK) cst = one(buf[1], buf[0]);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(r.cs, &g);
      if (cst != TSVD_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        if (cst != TSVD_OK) return cst;
        TSVD_CUDA(ce);
      }
      const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      TSVD_CUDA(ie);
      nodes = launches_so_far() - c0;
      count_launches(-nodes);  // counted again per replay
    }
    const int per_sync = std::max(batch, 1);
    int64_t e = 0;
    tsvd_status lst = TSVD_OK;
    for (; !coop;) {
      if (ge) {
        for (int b = 0; b < per_sync; b += 2) {
          const cudaError_t le = cudaGraphLaunch(ge, r.cs);
          if (le != cudaSuccess) {
            (void)cudaGetLastError();
            set_cuda_error(le, "cudaGraphLaunch", __FILE__, __LINE__);
            lst = TSVD_ECUDA;
            break;
          }
          count_launches(nodes);
          e += 2;
        }
      } else {
        for (int b = 0; b < per_sync && lst == TSVD_OK; ++b) {
          ++e;
          lst = one(buf[(e - 1) & 1], buf[e & 1]);
        }
      }
      if (lst == TSVD_OK && cudaMemcpyAsync(h, sc.info, 16, cudaMemcpyDeviceToHost, r.cs) != cudaSuccess) {
        (void)cudaGetLastError();
        lst = TSVD_ECUDA;
      }
      if (lst == TSVD_OK) {
        const cudaError_t se = cudaStreamSynchronize(r.cs);
        if (se != cudaSuccess) {
          (void)cudaGetLastError();
          set_cuda_error(se, "cudaStreamSynchronize", __FILE__, __LINE__);
          lst = TSVD_ECUDA;
        }
      }
      if (lst == TSVD_OK) lst = after_sync();
      if (lst != TSVD_OK || h[3] != 0) break;  // stopped at application h[3]: converged, forced count, or rank
    }
    if (ge) cudaGraphExecDestroy(ge);
    TSVD_TRY(lst);
    // rank: keep v0 of the stopping application; otherwise its output
    const int64_t stop = h[3];
    v = h[1] == 2 ? buf[(stop - 1) & 1] : buf[stop & 1];
    vn = v == buf[0] ? buf[1] : buf[0];
    if (h[1] == 2) {
      // v := v0 orthogonalised against earlier vectors, twice; sigma_l = 0
      for (int pass = 0; pass < 2; ++pass) {
        TSVD_TRY(launch_vec_deflate_step(n, L.Vr, k, L.sig2, l, v, L.w, vn, p->eps, p->opt.max_iter, ovr, rank_scale,
                                         sc, 1, r.cs));
        std::swap(v, vn);
      }
      TSVD_CUDA(cudaMemsetAsync(L.sig2 + l, 0, 8, r.cs));
      flags |= TSVD_FLAG_RANK;
    } else {
      // sigma_l^2 = ||A v_l||^2 (Alg. 1)
      TSVD_CUDA(cudaMemsetAsync(L.ss, 0, 8, r.cs));
      TSVD_TRY(apply(v, L.w, L.ss, 0));
      TSVD_CUDA(cudaMemcpyAsync(L.sig2 + l, L.ss, 8, cudaMemcpyDeviceToDevice, r.cs));
      if (h[1] == 1) flags |= TSVD_FLAG_NOCONV;
    }
    TSVD_TRY(launch_vec_store_column(n, v, L.Vr, k, l, p->opt.sign_convention, sc, r.cs));
    if (L.Vcol) TSVD_CUDA(cudaMemcpyAsync(L.Vcol + l * n, v, (size_t)n * 4, cudaMemcpyDeviceToDevice, r.cs));
    TSVD_CUDA(cudaMemcpyAsync(V_out + l * n, v, (size_t)n * 4,
                              host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, r.cs));
    if (host_out) r.d2h += (double)n * 4;
    TSVD_CUDA(cudaMemcpyAsync(&hsig2[l], L.sig2 + l, 8, cudaMemcpyDeviceToHost, r.cs));
    TSVD_CUDA(cudaStreamSynchronize(r.cs));
    if (h[1] != 2) TSVD_TRY(after_sync());
    apps += h[0];
    if (rep && rep->iters) rep->iters[l] = h[0];
  }
  *flags_out |= flags;
  *apps_out += apps;
  return TSVD_OK;
}

// Dense t-SVD with an orthogonally batched Gram (Sec. V-C, Fig. 2c-d, Alg. 3):
// every task (I, J), J <= I, streams the row range of panels J and I (device
// pointers into A, or page-locked host rows copied into the panel ring) and
// accumulates B_JI = A_J^T A_I in FP64 (triangular SYRK for J == I,
// rectangular otherwise); the tile then goes to the device tile array or to
// page-locked host memory.  The power phase applies G through the tiles
// (explicit Hotelling correction, as for CSR), then U = A V Sigma^-1 over
// row blocks.
tsvd_status factor_dense_tiled(Run &r, float *U, double *sigma_out, float *V_out, tsvd_report *rep) {
  tsvd_plan_s *p = r.p;
  const tsvd_matrix *A = r.A;
  const int64_t n = p->n, k = p->k, m = p->m, bs = p->tb, nb = p->n_panels;
  const int prec = p->opt.precision;
  const bool host_a = p->location == TSVD_HOST;
  unsigned char *ws = r.ws;
  float *v = reinterpret_cast<float *>(ws + p->o_v);
  float *vn = reinterpret_cast<float *>(ws + p->o_vn);
  float *w = reinterpret_cast<float *>(ws + p->o_w);
  double *x64 = reinterpret_cast<double *>(ws + p->o_x64);
  double *w64 = reinterpret_cast<double *>(ws + p->o_w64);
  float *Vr = reinterpret_cast<float *>(ws + p->o_Vr);
  float *Vc = reinterpret_cast<float *>(ws + p->o_Vc);
  double *sig2 = reinterpret_cast<double *>(ws + p->o_sig2);
  double *sigma = reinterpret_cast<double *>(ws + p->o_sigma);
  int32_t *info = reinterpret_cast<int32_t *>(ws + p->o_info);
  double *ss = reinterpret_cast<double *>(ws + p->o_flag + 64);
  double *Gt = reinterpret_cast<double *>(ws + p->o_Gt);
  void *tscr = ws + p->o_gscr;
  double *dtiles = reinterpret_cast<double *>(ws + p->o_tiles);
  const int64_t tstride = (int64_t)(p->b_tile / 8);  // doubles per device tile slot
  VecScratch sc;
  sc.part = reinterpret_cast<double *>(ws + p->o_vsc);
  sc.coef = sc.part + (size_t)p->vec_grid * kVecPartStride;
  sc.scal = sc.coef + 64 * 2;
  sc.grid = p->vec_grid;
  auto width = [&](int64_t P) { return std::min(bs, n - P * bs); };
  if (p->tiles_host && !p->host_tiles)
    TSVD_TRY(pinned_alloc(reinterpret_cast<void **>(&p->host_tiles), (size_t)p->n_tasks * bs * bs * 8));

  TSVD_CUDA(cudaEventRecord(p->ev_t[0], r.cs));
  // ---- Gram, task by task
  if (prec != TSVD_GRAM_FP32) TSVD_CUDA(cudaMemsetAsync(tscr, 0, 4, r.cs));
  for (int64_t I = 0; I < nb; ++I) {
    for (int64_t J = 0; J <= I; ++J) {
      const int64_t nI = width(I), nJ = width(J);
      const bool diag = I == J;
      TSVD_CUDA(cudaMemsetAsync(Gt, 0, (size_t)bs * 2 * bs * 8, r.cs));
      for (int64_t r0 = 0; r0 < m; r0 += p->pan_rows) {
        const int64_t rows = std::min(p->pan_rows, m - r0);
        const float *AJ, *AI;
        int64_t ld;
        int slot = -1;
        if (!host_a) {
          AJ = A->values + r0 * A->ld + J * bs;
          AI = A->values + r0 * A->ld + I * bs;
          ld = A->ld;
        } else {
          slot = (int)(r.chunk_seq++ % p->n_buffers);
          float *dst = reinterpret_cast<float *>(ws + p->o_pan + p->b_pan * slot);
          TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_free[slot], 0));
          TSVD_TRY(copy_event(r, true));
          TSVD_CUDA(cudaEventRecord(p->ev_csplit, p->copy_stream));
          TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream2, p->ev_csplit, 0));
          const float *src = A->values + r0 * A->ld;
          TSVD_CUDA(cudaMemcpy2DAsync(dst, (size_t)2 * bs * 4, src + J * bs, (size_t)A->ld * 4, (size_t)nJ * 4,
                                      (size_t)rows, cudaMemcpyHostToDevice, p->copy_stream));
          if (!diag)
            TSVD_CUDA(cudaMemcpy2DAsync(dst + bs, (size_t)2 * bs * 4, src + I * bs, (size_t)A->ld * 4,
                                        (size_t)nI * 4, (size_t)rows, cudaMemcpyHostToDevice, p->copy_stream2));
          TSVD_CUDA(cudaEventRecord(p->ev_cjoin, p->copy_stream2));
          TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_cjoin, 0));
          TSVD_TRY(copy_event(r, false));
          const double bytes = (double)rows * (nJ + (diag ? 0 : nI)) * 4;
          if (p->opt.time_kernels) {
            r.copy_bytes.push_back(bytes);
            r.copy_first.push_back(r0);
          }
          r.h2d += bytes;
          TSVD_CUDA(cudaEventRecord(p->ev_ready[slot], p->copy_stream));
          TSVD_CUDA(cudaStreamWaitEvent(r.cs, p->ev_ready[slot], 0));
          AJ = dst;
          AI = diag ? dst : dst + bs;
          ld = 2 * bs;
        }
        if (diag)
          TSVD_TRY(gram_dispatch(AI, rows, nI, ld, Gt, prec, tscr, p->b_gscr, r.cs, nullptr, nullptr, false));
        else if (prec == TSVD_GRAM_FP32)
          TSVD_TRY(launch_gram_simt_rect(AJ, AI, rows, nJ, nI, ld, Gt + bs, 2 * bs, r.cs));
        else
          TSVD_TRY(launch_gram_tc_rect(AJ, AI, rows, bs, nJ, nI, ld, Gt, prec, tscr, p->b_gscr, r.cs, false));
        TSVD_TRY(release_slot(r, slot));
      }
      // the task's tile: nJ rows of nI, row stride bs
      const int64_t t = I * (I + 1) / 2 + J;
      const double *src = diag ? Gt : Gt + bs;
      const size_t spitch = (size_t)(diag ? nI : 2 * bs) * 8;
      if (p->tiles_host) {
        TSVD_CUDA(cudaMemcpy2DAsync(p->host_tiles + t * bs * bs, (size_t)bs * 8, src, spitch, (size_t)nI * 8,
                                    (size_t)nJ, cudaMemcpyDeviceToHost, r.cs));
        r.d2h += (double)nI * nJ * 8;
      } else {
        TSVD_CUDA(cudaMemcpy2DAsync(dtiles + t * tstride, (size_t)bs * 8, src, spitch, (size_t)nI * 8, (size_t)nJ,
                                    cudaMemcpyDeviceToDevice, r.cs));
      }
    }
  }
  int32_t gram_err = 0;
  if (prec != TSVD_GRAM_FP32) TSVD_CUDA(cudaMemcpyAsync(&gram_err, tscr, 4, cudaMemcpyDeviceToHost, r.cs));
  TSVD_CUDA(cudaEventRecord(p->ev_t[1], r.cs));

  // ---- power phase: w = G v through the tiles
  int64_t tseq = 0;
  auto apply = [&](const float *vv, float *ww, double *s2, int) -> tsvd_status {
    TSVD_CUDA(cudaMemsetAsync(w64, 0, (size_t)n * 8, r.cs));
    for (int64_t I = 0; I < nb; ++I) {
      for (int64_t J = 0; J <= I; ++J) {
        const int64_t nI = width(I), nJ = width(J), t = I * (I + 1) / 2 + J;
        const double *T = dtiles + t * tstride;
        int slot = -1;
        if (p->tiles_host) {
          slot = (int)(tseq++ % p->n_buffers);
          double *dst = dtiles + slot * tstride;
          TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_free[slot], 0));
          TSVD_CUDA(cudaMemcpy2DAsync(dst, (size_t)bs * 8, p->host_tiles + t * bs * bs, (size_t)bs * 8,
                                      (size_t)nI * 8, (size_t)nJ, cudaMemcpyHostToDevice, p->copy_stream));
          r.h2d += (double)nI * nJ * 8;
          TSVD_CUDA(cudaEventRecord(p->ev_ready[slot], p->copy_stream));
          TSVD_CUDA(cudaStreamWaitEvent(r.cs, p->ev_ready[slot], 0));
          T = dst;
        }
        TSVD_TRY(launch_tile_symv(T, bs, nJ, nI, vv + J * bs, vv + I * bs, w64 + J * bs, w64 + I * bs, I == J, r.cs));
        TSVD_TRY(release_slot(r, slot));
      }
    }
    return launch_tile_finish(n, vv, w64, ww, s2, r.cs);
  };
  ExplicitLoop L{v, vn, w, x64, ss, Vr, Vc, sig2, info, sc, reinterpret_cast<int32_t *>(ws + p->o_flag) + 32};
  int flags = 0;
  int64_t apps = 0;
  TSVD_TRY(explicit_power(r, L, apply, []() { return TSVD_OK; }, V_out, &flags, &apps, rep));
  TSVD_TRY(launch_sigma_from_sigma2(sig2, sigma, k, r.cs));
  TSVD_CUDA(cudaEventRecord(p->ev_t[2], r.cs));

  // ---- left vectors: U = A V Sigma^-1 over row blocks (their ring reuses the Gram region)
  if (U) {
    TSVD_CUDA(cudaEventRecord(p->ev_csplit, r.cs));
    TSVD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_csplit, 0));
    TSVD_TRY(left_pass_dense(r, Vc, sigma, U));
  }
  TSVD_CUDA(cudaEventRecord(p->ev_t[3], r.cs));
  const bool host_out = p->opt.out_location == TSVD_HOST;
  TSVD_CUDA(cudaMemcpyAsync(sigma_out, sigma, (size_t)k * 8, host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            r.cs));
  if (host_out) r.d2h += (double)k * 8;
  TSVD_CUDA(cudaStreamSynchronize(r.cs));
  TSVD_CUDA(cudaStreamSynchronize(p->d2h_stream));
  TSVD_CUDA(cudaStreamSynchronize(p->copy_stream));
  float t01 = 0, t12 = 0, t23 = 0;
  TSVD_CUDA(cudaEventElapsedTime(&t01, p->ev_t[0], p->ev_t[1]));
  TSVD_CUDA(cudaEventElapsedTime(&t12, p->ev_t[1], p->ev_t[2]));
  TSVD_CUDA(cudaEventElapsedTime(&t23, p->ev_t[2], p->ev_t[3]));
  if (gram_err || r.left_err) flags |= TSVD_FLAG_TIMEOUT;
  if (host_out) {
    for (int64_t l = 1; l < k; ++l)
      if (sigma_out[l] > sigma_out[l - 1]) flags |= TSVD_FLAG_NONMONOTONE;
  }
  if (rep) {
    rep->gram_ms = t01;
    rep->power_ms = t12;
    rep->left_ms = t23;
    rep->total_ms = (double)t01 + t12 + t23;
    rep->applications = apps;
    rep->flags |= flags;
    rep->gram_panels = (int32_t)nb;
    rep->tiles_on_host = p->tiles_host ? 1 : 0;
  }
  if (flags & TSVD_FLAG_TIMEOUT) return TSVD_ETIMEDOUT;
  if (flags & TSVD_FLAG_RANK) return TSVD_ERANK;
  if (flags & TSVD_FLAG_NOCONV) return TSVD_ENOCONV;
  return TSVD_OK;
}

tsvd_status factor_csr(Run &r, float *U, double *sigma_out, float *V_out, tsvd_report *rep) {
  tsvd_plan_s *p = r.p;
  const tsvd_matrix *A = r.A;
  const int64_t n = p->n, k = p->k, m = p->m;
  unsigned char *ws = r.ws;
  float *v = reinterpret_cast<float *>(ws + p->o_v);
  float *vn = reinterpret_cast<float *>(ws + p->o_vn);
  float *w = reinterpret_cast<float *>(ws + p->o_w);
  double *x64 = reinterpret_cast<double *>(ws + p->o_x64);
  float *Vr = reinterpret_cast<float *>(ws + p->o_Vr);
  double *sig2 = reinterpret_cast<double *>(ws + p->o_sig2);
  double *sigma = reinterpret_cast<double *>(ws + p->o_sigma);
  int32_t *info = reinterpret_cast<int32_t *>(ws + p->o_info);
  int32_t *flag = reinterpret_cast<int32_t *>(ws + p->o_flag);
  double *ss = reinterpret_cast<double *>(ws + p->o_flag + 64);
  VecScratch sc;
  sc.part = reinterpret_cast<double *>(ws + p->o_vsc);
  sc.coef = sc.part + (size_t)p->vec_grid * kVecPartStride;
  sc.scal = sc.coef + 64 * 2;
  sc.grid = p->vec_grid;

  if (p->opt.time_kernels && (int64_t)p->ev_k.size() < 2 * p->n_chunks) {
    const size_t have = p->ev_k.size();
    p->ev_k.resize(2 * p->n_chunks, nullptr);
    for (size_t i = have; i < p->ev_k.size(); ++i) TSVD_CUDA(cudaEventCreate(&p->ev_k[i]));
  }
  TSVD_CUDA(cudaEventRecord(p->ev_t[0], r.cs));
  // entry offsets at block boundaries
  std::vector<int64_t> bnd(p->n_chunks + 1);
  if (p->location == TSVD_HOST) {
    for (int64_t b = 0; b <= p->n_chunks; ++b) bnd[b] = A->row_ptr[p->block_start[b]];
    r.chunked = p->csr_nch > 0 && p->csr_sorted;
  } else {
    // device CSR: validate on the device, then read the boundary offsets
    TSVD_CUDA(cudaMemsetAsync(flag, 0, 4, r.cs));
    csr_validate_kernel<<<1024, 256, 0, r.cs>>>(m, n, p->nnz, A->row_ptr, A->col_idx, flag);
    TSVD_LAUNCHED();
    int hflag = 0;
    TSVD_CUDA(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, r.cs));
    for (int64_t b = 0; b <= p->n_chunks; ++b)
      TSVD_CUDA(cudaMemcpyAsync(&bnd[b], A->row_ptr + p->block_start[b], 8, cudaMemcpyDeviceToHost, r.cs));
    TSVD_CUDA(cudaStreamSynchronize(r.cs));
    if (hflag & 1) return TSVD_EINVAL;
    r.chunked = p->csr_nch > 0 && !(hflag & 2);
  }
  if (p->mode == MODE_RESIDENT) {
    unsigned char *base = ws + p->o_res;
    const size_t orp = 0, oci = round_up((m + 1) * 8, 256), ova = oci + round_up(std::max<int64_t>(p->nnz, 1) * 4, 256);
    TSVD_CUDA(cudaMemcpyAsync(base + orp, A->row_ptr, (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, r.cs));
    if (p->nnz) {
      TSVD_CUDA(cudaMemcpyAsync(base + oci, A->col_idx, (size_t)p->nnz * 4, cudaMemcpyHostToDevice, r.cs));
      TSVD_CUDA(cudaMemcpyAsync(base + ova, A->values, (size_t)p->nnz * 4, cudaMemcpyHostToDevice, r.cs));
    }
    r.h2d += (double)(m + 1) * 8 + (double)p->nnz * 8;
  }
  if (r.chunked && p->mode != MODE_STREAM) {
    // in core: every row's chunk split points, once per factorisation
    const int64_t *rp_all = p->mode == MODE_DEVICE ? A->row_ptr : reinterpret_cast<const int64_t *>(ws + p->o_res);
    const int32_t *ci_all = p->mode == MODE_DEVICE
                                ? A->col_idx
                                : reinterpret_cast<const int32_t *>(ws + p->o_res + round_up((m + 1) * 8, 256));
    TSVD_TRY(launch_csr_split(m, rp_all, ci_all, p->csr_nch, p->csr_cw,
                              reinterpret_cast<int32_t *>(ws + p->o_csr_split), r.cs));
  }
  TSVD_CUDA(cudaEventRecord(p->ev_t[1], r.cs));

  ExplicitLoop L{v, vn, w, x64, ss, Vr, nullptr, sig2, info, sc, flag + 32};
  int flags = 0;
  int64_t apps = 0;
  const bool host_out = p->opt.out_location == TSVD_HOST;
  // small operators: 16 applications per host round trip (the round trip dominates them),
  // replayed from a CUDA graph when A is on the device (the streamed operator waits on
  // copies); large ones, or per-application kernel timing: one at a time
  const bool small = !p->opt.time_kernels && p->nnz < ((int64_t)1 << 25);
  const int batch = small ? 16 : 1;
  const bool graph = small && p->mode != MODE_STREAM;
  // small, in core, single-pass operator, at most 32 earlier vectors: the whole loop of a
  // triplet in one cooperative launch (k_csr_power.cu)
  const bool coop = graph && !r.chunked && k <= 33;
  const int64_t *rp_all = p->mode == MODE_DEVICE ? A->row_ptr : reinterpret_cast<const int64_t *>(ws + p->o_res);
  const int32_t *ci_all = p->mode == MODE_DEVICE
                              ? A->col_idx
                              : reinterpret_cast<const int32_t *>(ws + p->o_res + round_up((m + 1) * 8, 256));
  const float *va_all = p->mode == MODE_DEVICE
                            ? A->values
                            : reinterpret_cast<const float *>(ws + p->o_res + round_up((m + 1) * 8, 256) +
                                                              round_up(std::max<int64_t>(p->nnz, 1) * 4, 256));
  TripletLoop coop_fn = [&](float *b0, float *b1, int64_t l, int ovr, double rank_scale,
                            int32_t *info_l) -> tsvd_status {
    unsigned *bar = reinterpret_cast<unsigned *>(flag + 48);  // bytes 192..199 of the flag region
    int *err = flag + 50;                                     // bytes 200..203
    TSVD_CUDA(cudaMemsetAsync(bar, 0, 16, r.cs));
    TSVD_CUDA(cudaMemsetAsync(w, 0, (size_t)n * 4, r.cs));
    return launch_csr_power(m, n, rp_all, ci_all, va_all, Vr, k, sig2, l, b0, b1, w, sc.part,
                            (size_t)sc.grid * kVecPartStride * sizeof(double), bar, err, p->eps, p->opt.max_iter,
                            ovr, rank_scale, info_l, p->avg_nnz,
                            p->opt.csr_coop_blocks > 0 ? p->opt.csr_coop_blocks : 128, r.cs);
  };
  TSVD_TRY(explicit_power(
      r, L, [&](const float *vv, float *ww, double *s2, int scatter) { return csr_apply(r, bnd, vv, ww, s2, scatter); },
      [&]() { return csr_kernel_time(r); }, V_out, &flags, &apps, rep, batch, graph, coop ? &coop_fn : nullptr));
  TSVD_TRY(launch_sigma_from_sigma2(sig2, sigma, k, r.cs));
  TSVD_CUDA(cudaEventRecord(p->ev_t[2], r.cs));
  if (U) {
    for (int64_t b = 0; b < p->n_chunks; ++b) {
      CsrBlock blk;
      TSVD_TRY(acquire_csr(r, b, bnd, &blk));
      const int64_t r0 = p->block_start[b];
      if (!host_out) {
        TSVD_TRY(launch_csr_left(blk.rows, blk.rp, blk.ci, blk.va, Vr, k, k, sigma, U + r0, m, p->avg_nnz, r.cs));
        TSVD_TRY(release_slot(r, blk.slot));
      } else {
        const int bb = (int)(b & 1);
        float *ub = reinterpret_cast<float *>(ws + p->o_ubuf + p->b_ubuf * bb);
        TSVD_CUDA(cudaStreamWaitEvent(r.cs, p->ev_u_free[bb], 0));
        TSVD_TRY(launch_csr_left(blk.rows, blk.rp, blk.ci, blk.va, Vr, k, k, sigma, ub, blk.rows, p->avg_nnz, r.cs));
        TSVD_TRY(release_slot(r, blk.slot));
        TSVD_CUDA(cudaEventRecord(p->ev_u_ready[bb], r.cs));
        TSVD_CUDA(cudaStreamWaitEvent(p->d2h_stream, p->ev_u_ready[bb], 0));
        TSVD_CUDA(cudaMemcpy2DAsync(U + r0, (size_t)m * 4, ub, (size_t)blk.rows * 4, (size_t)blk.rows * 4,
                                    (size_t)k, cudaMemcpyDeviceToHost, p->d2h_stream));
        r.d2h += (double)blk.rows * k * 4;
        TSVD_CUDA(cudaEventRecord(p->ev_u_free[bb], p->d2h_stream));
      }
    }
  }
  TSVD_CUDA(cudaEventRecord(p->ev_t[3], r.cs));
  TSVD_CUDA(cudaMemcpyAsync(sigma_out, sigma, (size_t)k * 8, host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            r.cs));
  TSVD_CUDA(cudaStreamSynchronize(r.cs));
  TSVD_CUDA(cudaStreamSynchronize(p->d2h_stream));
  TSVD_CUDA(cudaStreamSynchronize(p->copy_stream));
  float t01 = 0, t12 = 0, t23 = 0;
  TSVD_CUDA(cudaEventElapsedTime(&t01, p->ev_t[0], p->ev_t[1]));
  TSVD_CUDA(cudaEventElapsedTime(&t12, p->ev_t[1], p->ev_t[2]));
  TSVD_CUDA(cudaEventElapsedTime(&t23, p->ev_t[2], p->ev_t[3]));
  if (host_out) {
    for (int64_t l = 1; l < k; ++l)
      if (sigma_out[l] > sigma_out[l - 1]) flags |= TSVD_FLAG_NONMONOTONE;
  }
  if (rep) {
    rep->gram_ms = t01;
    rep->power_ms = t12;
    rep->left_ms = t23;
    rep->total_ms = (double)t01 + t12 + t23;
    rep->applications = apps;
    rep->flags |= flags;
    rep->gram_kernel_ms = r.kernel_ms;
    rep->gram_kernel_launches = (int32_t)r.kernel_launches;
  }
  if (flags & TSVD_FLAG_RANK) return TSVD_ERANK;
  if (flags & TSVD_FLAG_NOCONV) return TSVD_ENOCONV;
  return TSVD_OK;
}

}  // namespace

extern "C" {

tsvd_status tsvd_factor(tsvd_plan_t plan, const tsvd_matrix *A, void *workspace, size_t workspace_bytes,
                        void *stream, float *U, double *sigma, float *V, tsvd_report *report) {
  if (!plan || !A || !sigma || !V) return TSVD_EINVAL;
  tsvd_plan_s *p = plan;
  if (A->kind != p->kind || A->location != p->location || A->m != p->m || A->n != p->n) return TSVD_EINVAL;
  if (p->kind == TSVD_DENSE_F32_ROWMAJOR && (!A->values || A->ld != p->ld)) return TSVD_EINVAL;
  if (p->kind == TSVD_CSR_F32_I32_I64 && (A->nnz != p->nnz || !A->row_ptr)) return TSVD_EINVAL;
  if (!workspace || workspace_bytes < p->ws) return TSVD_EBUDGET;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return TSVD_EINVAL;
  TSVD_TRY(ensure_runtime(p));
  const int64_t l0 = launches_so_far();
  Run r;
  r.p = p;
  r.A = A;
  r.ws = static_cast<unsigned char *>(workspace);
  r.cs = static_cast<cudaStream_t>(stream);
  int flags = 0;
  if (p->location == TSVD_HOST) {
    cudaPointerAttributes at;
    const void *probe = p->kind == TSVD_DENSE_F32_ROWMAJOR ? (const void *)A->values : (const void *)A->row_ptr;
    if (cudaPointerGetAttributes(&at, probe) != cudaSuccess || at.type == cudaMemoryTypeUnregistered) {
      cudaGetLastError();
      flags |= TSVD_FLAG_PAGEABLE;
    }
  }
  if (report) {
    int32_t *it = report->iters;
    memset(report, 0, sizeof *report);
    report->iters = it;
    report->flags = flags;
    report->mode = p->mode;
    report->n_blocks = (int32_t)p->n_chunks;
    report->ring_slots = p->mode == MODE_STREAM ? p->n_buffers : 0;
  }
  tsvd_status st = p->kind != TSVD_DENSE_F32_ROWMAJOR ? factor_csr(r, U, sigma, V, report)
                   : p->tiled                          ? factor_dense_tiled(r, U, sigma, V, report)
                                                       : factor_dense(r, U, sigma, V, report);
  if (report) {
    report->h2d_bytes = r.h2d;
    report->d2h_bytes = r.d2h;
    report->csr_chunks = (p->kind == TSVD_CSR_F32_I32_I64 && r.chunked) ? p->csr_nch : 0;
    report->power_cluster = (p->kind == TSVD_DENSE_F32_ROWMAJOR && p->cluster_power) ? p->srv_req.cluster : 0;
    report->kernel_launches = launches_so_far() - l0;
    if (st == TSVD_OK || st == TSVD_ENOCONV || st == TSVD_ERANK) {
      double ms = 0.0, gmin = 0.0, gmax = 0.0;
      if (copy_time_ms(r, &ms, &gmin, &gmax) == TSVD_OK) {
        report->h2d_copy_ms = ms;
        report->h2d_copies = (int32_t)r.copies;
        report->h2d_copy_min_gbps = gmin;
        report->h2d_copy_max_gbps = gmax;
      }
    }
  }
  // the copy log of this call (time_kernels): block, bytes, rate
  p->copy_log.clear();
  if (p->opt.time_kernels && (st == TSVD_OK || st == TSVD_ENOCONV || st == TSVD_ERANK)) {
    for (int64_t c = 0; c < r.copies && c < (int64_t)r.copy_bytes.size(); ++c) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p->ev_c[2 * c], p->ev_c[2 * c + 1]) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      p->copy_log.push_back({c < (int64_t)r.copy_first.size() ? r.copy_first[(size_t)c] : -1,
                             r.copy_bytes[(size_t)c], t > 0.f ? r.copy_bytes[(size_t)c] / ((double)t * 1e6) : 0.0});
    }
  }
  return st;
}

tsvd_status tsvd_plan_copy_log(tsvd_plan_t p, int64_t *first, double *bytes, double *gbps, int64_t cap,
                               int64_t *count) {
  if (!p || !count || cap < 0) return TSVD_EINVAL;
  const int64_t nrec = (int64_t)p->copy_log.size();
  *count = nrec;
  for (int64_t i = 0; i < nrec && i < cap; ++i) {
    if (first) first[i] = p->copy_log[(size_t)i].first;
    if (bytes) bytes[i] = p->copy_log[(size_t)i].bytes;
    if (gbps) gbps[i] = p->copy_log[(size_t)i].gbps;
  }
  return TSVD_OK;
}

// ---------------------------------------------------------------- step entry points
size_t tsvd_gram_scratch_bytes(int64_t rows, int64_t n, int32_t precision) {
  if (rows <= 0 || n <= 0) return 0;
  if (precision == TSVD_GRAM_FP32) return 0;
  return gram_tc_scratch_bytes(rows, n, precision);
}

tsvd_status tsvd_gram_accumulate(const float *dA, int64_t rows, int64_t n, int64_t ld, double *dG,
                                 int32_t precision, void *scratch, size_t scratch_bytes, void *stream) {
  if (rows < 0 || n <= 0 || ld < n || !dG || (rows > 0 && !dA)) return TSVD_EINVAL;
  if (precision < TSVD_GRAM_FP32 || precision > TSVD_GRAM_BF16X3) return TSVD_EINVAL;
  if (precision != TSVD_GRAM_FP32) {
    if (scratch_bytes < gram_tc_scratch_bytes(rows, n, precision)) return TSVD_EINVAL;
    if (scratch && (reinterpret_cast<uintptr_t>(scratch) & 255) != 0) return TSVD_EINVAL;
  }
  return gram_dispatch(dA, rows, n, ld, dG, precision, scratch, scratch_bytes, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_csr_gram_apply(int64_t rows, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                const float *values, const float *v, float *w, double *ss, int32_t scatter,
                                void *stream) {
  if (rows < 0 || n <= 0 || !row_ptr || !v || !ss || (scatter && !w)) return TSVD_EINVAL;
  if (rows == 0) return TSVD_OK;
  // mean row length from the block's first and last offsets
  int64_t e[2];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TSVD_CUDA(cudaMemcpyAsync(&e[0], row_ptr, 8, cudaMemcpyDeviceToHost, s));
  TSVD_CUDA(cudaMemcpyAsync(&e[1], row_ptr + rows, 8, cudaMemcpyDeviceToHost, s));
  TSVD_CUDA(cudaStreamSynchronize(s));
  const double avg = (double)(e[1] - e[0]) / (double)rows;
  return launch_csr_pair(rows, n, row_ptr, col_idx, values, v, w, ss, scatter, avg, s);
}

size_t tsvd_power_scratch_bytes(int64_t n, int64_t l) { return power_scratch_bytes(n, l); }

tsvd_status tsvd_power_dense(int64_t n, const float *G32, const double *G64, const double *V64,
                             const double *sigma2, int64_t l, double *x, double eps, int32_t max_iter,
                             int32_t iters_override, int32_t sign_convention, double *out_sigma2, int32_t *info,
                             void *scratch, size_t scratch_bytes, void *stream) {
  if (iters_override <= 0 && !(eps > 0.0 && eps < 1.0)) return TSVD_EINVAL;
  return launch_power_dense(n, G32, G64, V64, sigma2, l, x, eps, max_iter, iters_override, sign_convention,
                            out_sigma2, info, scratch, scratch_bytes, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_power_dense_noalloc(int64_t n, const float *G32, const double *G64, const double *V64,
                                     const double *sigma2, int64_t l, double *x, double eps, int32_t max_iter,
                                     int32_t iters_override, int32_t sign_convention, double *out_sigma2,
                                     int32_t *info, void *stream) {
  if (iters_override <= 0 && !(eps > 0.0 && eps < 1.0)) return TSVD_EINVAL;
  return launch_power_dense_noalloc(n, G32, G64, V64, sigma2, l, x, eps, max_iter, iters_override,
                                    sign_convention, out_sigma2, info, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_gram_deflate(int64_t n, double *G64, float *G32, const double *v, const double *sigma2,
                              void *stream) {
  if (n <= 0 || !G64 || !G32 || !v || !sigma2) return TSVD_EINVAL;
  return launch_gram_deflate(n, G64, G32, v, sigma2, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_gram_symmetrize(int64_t n, const double *G64, float *G32, void *stream) {
  if (n <= 0 || !G64 || !G32) return TSVD_EINVAL;
  // G64 is only read when the FP64 lower triangle is not mirrored
  return launch_symmetrize(n, const_cast<double *>(G64), G32, static_cast<cudaStream_t>(stream), false);
}

tsvd_status tsvd_start_draws(uint64_t seed, int64_t l, int64_t n, double *x, void *stream) {
  if (n <= 0 || l < 0 || !x) return TSVD_EINVAL;
  return launch_start_draws(seed, l, n, x, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count,
                               void *stream) {
  if (count < 0 || (count > 0 && (!ctr || !key || !out))) return TSVD_EINVAL;
  return launch_philox_raw(ctr, key, out, count, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_left_vectors(const float *dA, int64_t rows, int64_t n, int64_t ld, const float *V, int64_t ldv,
                              int64_t k, const double *sigma, float *U, int64_t ldu, void *stream) {
  if (rows < 0 || n <= 0 || k <= 0 || ld < n || ldv < n || ldu < rows || !V || !sigma || !U ||
      (rows > 0 && !dA))
    return TSVD_EINVAL;
  return launch_left_dense(dA, rows, n, ld, V, ldv, k, sigma, U, ldu, static_cast<cudaStream_t>(stream));
}

tsvd_status tsvd_csr_partition(int64_t m, const int64_t *row_ptr, int64_t block_rows, int64_t *block_start,
                               int64_t *n_blocks, int64_t *max_block_nnz) {
  if (m <= 0 || !row_ptr || block_rows <= 0 || !block_start || !n_blocks) return TSVD_EINVAL;
  int64_t nb = 0, mx = 0;
  for (int64_t r = 0; r < m; r += block_rows) {
    block_start[nb++] = r;
    const int64_t r1 = std::min(m, r + block_rows);
    mx = std::max(mx, row_ptr[r1] - row_ptr[r]);
  }
  block_start[nb] = m;
  *n_blocks = nb;
  if (max_block_nnz) *max_block_nnz = mx;
  return TSVD_OK;
}

tsvd_status tsvd_host_alloc(void **ptr, size_t bytes) { return pinned_alloc(ptr, bytes); }

tsvd_status tsvd_host_free(void *ptr) { return pinned_free(ptr); }

}  // extern "C"
