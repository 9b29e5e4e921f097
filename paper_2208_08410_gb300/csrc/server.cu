// t-SVD server: continuous batching of many small requests on one GPU.
//
// The server owns two arenas allocated once: the device budget (each admitted
// request's A, Gram matrices, vectors, scalars and results) and a page-locked
// staging area (each request's results on the host), plus a device array of
// completion flags with a page-locked mirror.  Requests are admitted first in,
// first out while both arenas and the in-flight limit allow.  Admitted
// requests are launched in waves: a wave takes up to `max_wave` of them,
// copies their matrices in and runs the grouped launches of serve.cuh over all
// of them on one of `n_streams` streams.  Each request's cluster writes its
// results into device memory and then stores the request's ticket into its
// flag word.  The scheduler copies the flag array to the host on a stream of
// its own as often as it can; for every flag that shows its ticket it copies
// the request's results to the staging (one copy) and completes the request
// when that copy has finished, releasing its device memory.  So a request
// completes as soon as its own cluster is done, not when its wave is; the
// wave's event only releases its descriptors and its stream.  Waves on
// different streams overlap on the device, so requests that arrive while
// others run are admitted as memory frees up and start without waiting.
// Requests with a large Gram dimension (above `heavy_dim`) form waves of their
// own on streams opened on demand (up to `heavy_streams`): their power phase
// can last long, and a stream stays busy until its wave's last request is
// done, so light waves, which turn over quickly, never queue behind them, and
// heavy ones never wait for a heavy stream while memory admits them.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "philox.cuh"
#include "serve.cuh"

namespace tsvd {
namespace {

constexpr size_t kAlign = 256;
inline size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over one allocation (device memory, or the page-locked
// host staging area the results are copied into); free ranges are kept by
// offset and merged with their neighbours on release.
class Arena {
 public:
  unsigned char *base = nullptr;   // device memory, or page-locked host memory
  bool host = false;
  size_t size = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes

  tsvd_status init(size_t bytes, bool on_host) {
    bytes = bytes & ~(kAlign - 1);
    host = on_host;
    if (!on_host) {
      if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        set_error_text("server: cudaMalloc of the device budget failed");
        return TSVD_ENOMEM;
      }
    } else {
      if (pinned_alloc(reinterpret_cast<void **>(&base), bytes) != TSVD_OK) {
        base = nullptr;
        set_error_text("server: page-locked allocation of the staging area failed");
        return TSVD_ENOMEM;
      }
    }
    size = bytes;
    free_[0] = bytes;
    return TSVD_OK;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = al(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, o = it->first + bytes;
        free_.erase(it);
        if (rest) free_[o] = rest;
        used += bytes;
        peak = std::max(peak, used);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al(std::max<size_t>(bytes, 1));
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  void destroy() {
    if (base) {
      if (host)
        pinned_free(base);
      else
        cudaFree(base);
    }
    base = nullptr;
  }
};

struct Request {
  uint64_t id = 0;
  const float *A = nullptr;
  int64_t m = 0, n = 0;
  int32_t k = 0;
  double eps = 0.0;
  int32_t max_iter = 0;
  uint64_t seed = 0;
  int32_t sign = 0;
  float *U = nullptr;
  double *sigma = nullptr;
  float *V = nullptr;
  std::vector<int32_t> iters;   // forced applications per triplet (empty: convergence test)
  // a CSR request (host arrays, read until completion); runs on a sparse worker
  bool csr = false;
  const int64_t *row_ptr = nullptr;
  const int32_t *col_idx = nullptr;
  int64_t nnz = 0;
  size_t off = 0, bytes = 0;    // device arena region
  size_t soff = 0, sbytes = 0;  // staging region
  size_t out_off = 0;           // results within the device region (same layout as the staging)
  int32_t slot = -1;            // index of the request's completion flag
  cudaEvent_t copied = nullptr; // results copied to the staging
  bool admitted = false;
  SrvReq dq{};
  bool done = false;
  tsvd_request_info rec{};
  // Gram on the tensor cores (grouped 3xTF32 SYRK): the K-major operand pair in the device region
  bool tc = false;
  bool heavy = false;  // runs in the heavy lane
  int64_t Kp = 0;
  float *At_hi = nullptr, *At_lo = nullptr;
};
using ReqPtr = std::shared_ptr<Request>;

// results of one request (device output region and host staging alike): info, sigma, U, V
size_t staging_bytes(int64_t m, int64_t n, int64_t k) {
  return al(k * 16) + al(k * 8) + al(m * k * 4) + al(n * k * 4);
}
// contraction length of a request padded to a stage of the tensor-core SYRK
int64_t tc_kp(int64_t m, int64_t n) { return round_up(std::max(m, n), (int64_t)kSrvTcKStage); }

// device region of one request: A, G64, G32, V64, sig2, info, vout, forced iteration counts,
// the tensor-core operand pair (tc), results
size_t request_bytes(int64_t m, int64_t n, int64_t k, bool tc = false) {
  const int64_t d = std::min(m, n);
  const size_t op = tc ? 2 * al((size_t)d * tc_kp(m, n) * 4) : 0;
  return al(m * n * 4) + al(d * d * 8) + al(d * d * 4) + al(d * k * 8) + al(k * 8) + al(k * 16) + al(d * k * 4) +
         al(k * 4) + op + staging_bytes(m, n, k);
}

void carve(Request &r, unsigned char *p) {
  const int64_t m = r.m, n = r.n, k = r.k;
  const int64_t d = std::min(m, n);
  SrvReq &q = r.dq;
  q.A = reinterpret_cast<const float *>(p);
  p += al(m * n * 4);
  q.G64 = reinterpret_cast<double *>(p);
  p += al(d * d * 8);
  q.G32 = reinterpret_cast<float *>(p);
  p += al(d * d * 4);
  q.V64 = reinterpret_cast<double *>(p);
  p += al(d * k * 8);
  q.sig2 = reinterpret_cast<double *>(p);
  p += al(k * 8);
  q.info = reinterpret_cast<int32_t *>(p);
  p += al(k * 16);
  q.vout = reinterpret_cast<float *>(p);
  p += al(d * k * 4);
  q.iters_override = r.iters.empty() ? nullptr : reinterpret_cast<const int32_t *>(p);
  p += al(k * 4);
  if (r.tc) {
    r.Kp = tc_kp(m, n);
    r.At_hi = reinterpret_cast<float *>(p);
    p += al((size_t)d * r.Kp * 4);
    r.At_lo = reinterpret_cast<float *>(p);
    p += al((size_t)d * r.Kp * 4);
  }
  unsigned char *o = p;
  r.out_off = (size_t)(o - reinterpret_cast<unsigned char *>(const_cast<float *>(q.A)));
  q.oInfo = reinterpret_cast<int32_t *>(o);
  o += al(k * 16);
  q.oS = reinterpret_cast<double *>(o);
  o += al(k * 8);
  q.oU = reinterpret_cast<float *>(o);
  o += al(m * k * 4);
  q.oV = reinterpret_cast<float *>(o);
  q.m = m;
  q.n = n;
  q.trans = m < n ? 1 : 0;  // Eq. 3: the left vectors from A A^T when m < n
  q.k = (int32_t)k;
  q.eps = r.eps;
  q.max_iter = r.max_iter;
  q.sign_convention = r.sign;
  const uint64_t key = splitmix64(r.seed);
  q.key0 = (uint32_t)key;
  q.key1 = (uint32_t)(key >> 32);
}

struct Slot {  // one stream and the page-locked descriptors of the wave it runs
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned char *stage = nullptr;
  size_t stage_cap = 0;
  // stages outgrown by a larger wave, freed with the server: freeing page-locked memory
  // waits for the whole device, which would stall the scheduler behind every wave in flight
  std::vector<unsigned char *> stage_old;
  bool busy = false;
  std::vector<ReqPtr> reqs;
  size_t dev_off = 0, dev_bytes = 0;  // descriptor arrays in the device arena
  int64_t wave = 0;
  // the kernel part of its waves as instantiated graphs, one per launch signature (see
  // launch_wave), the least recently used replaced when kSlotGraphs are held
  struct Graph {
    std::vector<int32_t> shape;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
  };
  std::vector<Graph> graphs;
  uint64_t uses = 0;
};
constexpr size_t kSlotGraphs = 8;


}  // namespace
}  // namespace tsvd

struct tsvd_server_s {
  tsvd_server_options opt{};
  int device = 0;
  tsvd::Arena arena, staging;
  std::deque<tsvd::Slot> slots;  // the first n_streams take light waves; heavy ones are added on demand
  // completion flags: one word per in-flight request (device), its page-locked mirror,
  // the stream and event of the copy that refreshes the mirror, the free flag words
  uint32_t *dflags = nullptr, *hflags = nullptr;
  cudaStream_t poll_stream = nullptr, out_stream = nullptr;
  cudaEvent_t poll_done = nullptr;
  bool poll_inflight = false;
  std::vector<int32_t> free_flags;
  std::vector<cudaEvent_t> event_pool;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<tsvd::ReqPtr> pending;                  // submitted, not admitted
  std::deque<tsvd::ReqPtr> admitted;                 // in the arenas, not launched (light lane)
  std::deque<tsvd::ReqPtr> admitted_heavy;           // the same, heavy lane (min(m, n) > heavy_dim)
  std::list<tsvd::ReqPtr> running;                   // launched, flag not seen yet
  std::list<tsvd::ReqPtr> copying;                   // flag seen, results on their way to the staging
  std::unordered_map<uint64_t, tsvd::ReqPtr> table;  // every request not yet waited for
  uint64_t next_id = 1;
  int64_t inflight = 0;                              // admitted and not completed
  bool stop = false;
  std::thread thr;
  std::deque<tsvd::ReqPtr> csr_pending;              // sparse requests, run by the sparse workers
  std::vector<std::thread> csr_workers;
  std::condition_variable cv_csr;
  int csr_large_running = 0;                         // large sparse requests on the device now
  std::chrono::steady_clock::time_point t0;
  tsvd_server_stats stats{};
  std::string err;
  int32_t cluster_table[6] = {1, 2, 4, 8, 8, 8};     // d <= 64, 128, 256, 512, 1024, 2048
  // requests with d >= tc_min_d form their Gram matrix on the tensor cores (128 x 256 tiles,
  // 3xTF32), the others on the CUDA cores (64 x 64 tiles, FP32); set by the autotuner
  std::atomic<int64_t> tc_min_d{256};
  double syrk_ms_tc[4] = {0, 0, 0, 0}, syrk_ms_cc[4] = {0, 0, 0, 0};  // the autotuner's timings (d = 256 .. 2048)
  int32_t syrk_nreq[4] = {0, 0, 0, 0};
  double busy_since = -1.0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace tsvd {
namespace {

int bucket_of(int64_t d) {
  int b = 0;
  for (int64_t lim = 64; b < 5 && d > lim; lim *= 2) ++b;
  return b;
}

int clamp_cluster(int64_t d, int c) { return srv_clamp_cluster(d, c); }

int cluster_for(const tsvd_server_s *s, int64_t d) {
  return clamp_cluster(d, std::min(s->cluster_table[bucket_of(d)], s->opt.cluster_cap));
}

size_t power_smem_budget() {
  DeviceInfo di;
  if (device_info(&di) != TSVD_OK) return 48 * 1024;
  const size_t static_bytes = 24 * 1024;  // the power kernel's static shared arrays, rounded up
  return di.smem_optin > static_bytes ? di.smem_optin - static_bytes : 0;
}


// The tensor-core part of a wave: for every request with the tc flag, its
// operand descriptor, prep strips, finish tiles and SYRK units (longest
// contraction first, so the tail of the persistent launch is short) and its two
// tensor maps; laid out in one block of `bytes` (offsets from the block's start).
struct TcWave {
  std::vector<SrvTcReq> tcs;
  std::vector<int64_t> prep_start{0}, fin_start{0};
  std::vector<SrvTcUnit> units;
  std::vector<CUtensorMap> maps;
  size_t o_ps = 0, o_fs = 0, o_units = 0, o_maps = 0, bytes = 0;
};

tsvd_status build_tc_wave(const std::vector<ReqPtr> &rs, TcWave *w) {
  std::vector<int64_t> unit_cost;
  for (size_t i = 0; i < rs.size(); ++i) {
    const Request &r = *rs[i];
    if (!r.tc) continue;
    SrvTcReq c{};
    c.req = (int32_t)i;
    c.d = std::min(r.m, r.n);
    c.K = std::max(r.m, r.n);
    c.Kp = r.Kp;
    c.hi = r.At_hi;
    c.lo = r.At_lo;
    c.G64 = r.dq.G64;
    c.G32 = r.dq.G32;
    const int32_t t = (int32_t)w->tcs.size();
    const int64_t nb = ceil_div(c.d, (int64_t)kSrvTcTM);
    for (int64_t bi = 0; bi < nb; ++bi)
      for (int64_t bj = 0; bj <= bi / 2; ++bj) {  // 256-row block bj with bj 256 <= bi 128 + 127
        w->units.push_back({t, (int32_t)bi, (int32_t)bj, 0});
        unit_cost.push_back(c.Kp);
      }
    w->prep_start.push_back(w->prep_start.back() + srv_tc_prep_strips(c.d, c.Kp));
    w->fin_start.push_back(w->fin_start.back() + srv_tc_finish_tiles(c.d));
    w->tcs.push_back(c);
  }
  std::vector<size_t> idx(w->units.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return unit_cost[a] > unit_cost[b]; });
  std::vector<SrvTcUnit> u2(w->units.size());
  for (size_t i = 0; i < idx.size(); ++i) u2[i] = w->units[idx[i]];
  w->units.swap(u2);
  const size_t ntc = w->tcs.size();
  w->maps.resize(2 * ntc);
  for (size_t t = 0; t < ntc; ++t) {
    TSVD_TRY(tc_make_map(&w->maps[2 * t], w->tcs[t].hi, w->tcs[t].d, w->tcs[t].Kp, TSVD_GRAM_TF32X3));
    TSVD_TRY(tc_make_map(&w->maps[2 * t + 1], w->tcs[t].lo, w->tcs[t].d, w->tcs[t].Kp, TSVD_GRAM_TF32X3));
  }
  w->o_ps = al(ntc * sizeof(SrvTcReq));
  w->o_fs = w->o_ps + al((ntc + 1) * 8);
  w->o_units = w->o_fs + al((ntc + 1) * 8);
  w->o_maps = w->o_units + al(w->units.size() * sizeof(SrvTcUnit));  // 256-byte aligned (maps need 64)
  w->bytes = w->o_maps + al(2 * ntc * sizeof(CUtensorMap));
  return TSVD_OK;
}

void stage_tc_wave(const TcWave &w, unsigned char *p) {
  const size_t ntc = w.tcs.size();
  if (!ntc) return;
  std::memcpy(p, w.tcs.data(), ntc * sizeof(SrvTcReq));
  std::memcpy(p + w.o_ps, w.prep_start.data(), (ntc + 1) * 8);
  std::memcpy(p + w.o_fs, w.fin_start.data(), (ntc + 1) * 8);
  std::memcpy(p + w.o_units, w.units.data(), w.units.size() * sizeof(SrvTcUnit));
  std::memcpy(p + w.o_maps, w.maps.data(), 2 * ntc * sizeof(CUtensorMap));
}

// `dev`: the device copy of the block stage_tc_wave filled
tsvd_status launch_tc_wave(const TcWave &w, const SrvReq *dreq, unsigned char *dev, int32_t *derr, cudaStream_t st) {
  return launch_srv_syrk_tc(dreq, reinterpret_cast<const SrvTcReq *>(dev), (int)w.tcs.size(),
                            reinterpret_cast<const int64_t *>(dev + w.o_ps), w.prep_start.back(),
                            reinterpret_cast<const int64_t *>(dev + w.o_fs), w.fin_start.back(),
                            reinterpret_cast<const CUtensorMap *>(dev + w.o_maps),
                            reinterpret_cast<const SrvTcUnit *>(dev + w.o_units), (int)w.units.size(), derr, st);
}

// Build and enqueue one wave on slot `s` (scheduler thread, lock not held).
tsvd_status launch_wave(tsvd_server_s *sv, Slot &s) {
  std::vector<ReqPtr> &rs = s.reqs;
  s.dev_bytes = 0;  // nothing of this wave in the arena yet
  const size_t smem_cap = power_smem_budget();
  for (auto &r : rs) {
    const int64_t d = std::min(r->m, r->n);
    r->dq.cluster = cluster_for(sv, d);
    r->dq.resident = srv_power_smem(d, r->dq.cluster, 1) <= smem_cap ? 1 : 0;
  }
  // requests of one power launch share the cluster size and residency: sort by them
  std::stable_sort(rs.begin(), rs.end(), [](const ReqPtr &a, const ReqPtr &b) {
    return std::make_pair(a->dq.cluster, a->dq.resident) < std::make_pair(b->dq.cluster, b->dq.resident);
  });
  std::vector<SrvTile> tiles;
  std::vector<int64_t> tile_cost;
  for (size_t i = 0; i < rs.size(); ++i) {
    const Request &r = *rs[i];
    if (r.tc) continue;  // its Gram matrix comes from the tensor-core SYRK
    const int64_t d = std::min(r.m, r.n), K = std::max(r.m, r.n);
    const int T = (int)ceil_div(d, kSrvTile);
    for (int ti = 0; ti < T; ++ti)
      for (int tj = 0; tj <= ti; ++tj) {
        tiles.push_back({(int32_t)i, ti, tj, 0});
        tile_cost.push_back(K);
      }
  }
  {  // longest tiles first, so the tail of the launch is short
    std::vector<size_t> idx(tiles.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return tile_cost[a] > tile_cost[b]; });
    std::vector<SrvTile> t2(tiles.size());
    for (size_t i = 0; i < idx.size(); ++i) t2[i] = tiles[idx[i]];
    tiles.swap(t2);
  }
  TcWave tw;
  TSVD_TRY(build_tc_wave(rs, &tw));
  const size_t ntc = tw.tcs.size();
  const size_t b_req = al(rs.size() * sizeof(SrvReq)), b_tiles = al(tiles.size() * sizeof(SrvTile));
  const size_t o_tc = b_req + b_tiles, o_err = o_tc + tw.bytes;
  const size_t need = o_err + al(4);
  if (need > s.stage_cap) {
    // grow geometrically from 1 MB, so a slot reallocates a few times at most
    const size_t cap = std::max({need, 2 * s.stage_cap, (size_t)1 << 20});
    unsigned char *p = nullptr;
    TSVD_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&p), cap, cudaHostAllocPortable));
    if (s.stage) s.stage_old.push_back(s.stage);
    s.stage = p;
    s.stage_cap = cap;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->arena.alloc(need, &s.dev_off)) {
      set_error_text("server: no arena room for the wave descriptors");
      return TSVD_ENOMEM;
    }
  }
  s.dev_bytes = need;
  unsigned char *dev = sv->arena.base + s.dev_off;
  int32_t *derr = reinterpret_cast<int32_t *>(dev + o_err);
  SrvReq *hreq = reinterpret_cast<SrvReq *>(s.stage);
  for (size_t i = 0; i < rs.size(); ++i) {
    rs[i]->dq.gram_err = rs[i]->tc ? derr : nullptr;
    if (!srv_req_complete(rs[i]->dq) || (rs[i]->tc && (!rs[i]->At_hi || !rs[i]->At_lo))) {
      set_error_text("server: request descriptor with an unset pointer");
      return TSVD_EINVAL;
    }
    hreq[i] = rs[i]->dq;
  }
  std::memcpy(s.stage + b_req, tiles.data(), tiles.size() * sizeof(SrvTile));
  stage_tc_wave(tw, s.stage + o_tc);
  cudaStream_t st = s.stream;
  for (auto &r : rs) {
    TSVD_CUDA(cudaMemcpyAsync(const_cast<float *>(r->dq.A), r->A, (size_t)r->m * r->n * 4, cudaMemcpyHostToDevice, st));
    if (r->dq.iters_override)
      TSVD_CUDA(cudaMemcpyAsync(const_cast<int32_t *>(r->dq.iters_override), r->iters.data(), r->iters.size() * 4,
                                cudaMemcpyHostToDevice, st));
  }
  // the kernel part of the wave is captured into a CUDA graph: the descriptor copy, the
  // grouped SYRK (tensor-core prep / SYRK / finish, then the CUDA-core tiles) and one power
  // launch per (cluster, residency) run of the sorted requests.  Waves of the same shape
  // (the same launches with other sizes and pointers) update the slot's instantiated graph in
  // place; a new shape instantiates it again.
  const SrvReq *dreq = reinterpret_cast<const SrvReq *>(dev);
  const auto g0 = std::chrono::steady_clock::now();
  auto graph_time = [&]() {
    const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count();
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stats.graph_host_s += t;
  };
  if (!sv->opt.wave_graphs) {
    TSVD_CUDA(cudaMemcpyAsync(dev, s.stage, need, cudaMemcpyHostToDevice, st));
    TSVD_TRY(launch_tc_wave(tw, dreq, dev + o_tc, derr, st));
    TSVD_TRY(launch_srv_syrk(dreq, reinterpret_cast<const SrvTile *>(dev + b_req), (int)tiles.size(), st));
    for (size_t i = 0; i < rs.size();) {
      size_t j = i, smem = 0;
      while (j < rs.size() && rs[j]->dq.cluster == rs[i]->dq.cluster && rs[j]->dq.resident == rs[i]->dq.resident) {
        smem = std::max(smem, srv_power_smem(std::min(rs[j]->m, rs[j]->n), rs[j]->dq.cluster, rs[j]->dq.resident));
        ++j;
      }
      TSVD_TRY(launch_srv_power(dreq + i, (int)(j - i), rs[i]->dq.cluster, smem, st));
      i = j;
    }
    graph_time();
    TSVD_CUDA(cudaEventRecord(s.done, st));
    return TSVD_OK;
  }
  TSVD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  auto enqueue = [&]() -> tsvd_status {
    TSVD_CUDA(cudaMemcpyAsync(dev, s.stage, need, cudaMemcpyHostToDevice, st));
    TSVD_TRY(launch_tc_wave(tw, dreq, dev + o_tc, derr, st));
    TSVD_TRY(launch_srv_syrk(dreq, reinterpret_cast<const SrvTile *>(dev + b_req), (int)tiles.size(), st));
    for (size_t i = 0; i < rs.size();) {
      size_t j = i, smem = 0;
      while (j < rs.size() && rs[j]->dq.cluster == rs[i]->dq.cluster && rs[j]->dq.resident == rs[i]->dq.resident) {
        smem = std::max(smem, srv_power_smem(std::min(rs[j]->m, rs[j]->n), rs[j]->dq.cluster, rs[j]->dq.resident));
        ++j;
      }
      TSVD_TRY(launch_srv_power(dreq + i, (int)(j - i), rs[i]->dq.cluster, smem, st));
      i = j;
    }
    return TSVD_OK;
  };
  const tsvd_status est = enqueue();
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);  // always ends the capture, also after a failure
  if (est != TSVD_OK) {
    if (g) cudaGraphDestroy(g);
    return est;
  }
  TSVD_CUDA(ce);
  // The launch signature: which SYRK launches there are and the (cluster, residency) of
  // every power launch.  The instantiated graph is updated in place only for a wave with
  // the same signature, so every node keeps its kernel and its launch attributes (the
  // power kernel's cluster size is one) and only sizes and pointers change.
  std::vector<int32_t> shape = {ntc > 0 ? 1 : 0, tiles.empty() ? 0 : 1};
  for (size_t i = 0; i < rs.size();) {
    size_t j = i;
    while (j < rs.size() && rs[j]->dq.cluster == rs[i]->dq.cluster && rs[j]->dq.resident == rs[i]->dq.resident) ++j;
    shape.push_back(rs[i]->dq.cluster * 2 + rs[i]->dq.resident);
    i = j;
  }
  size_t gi = s.graphs.size();
  for (size_t x = 0; x < s.graphs.size(); ++x)
    if (s.graphs[x].shape == shape) gi = x;
  bool updated = false;
  if (gi < s.graphs.size()) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(s.graphs[gi].exec, g, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(s.graphs[gi].exec);
      s.graphs[gi].exec = nullptr;
    }
  } else if (s.graphs.size() < kSlotGraphs) {
    s.graphs.emplace_back();
  } else {
    gi = 0;  // the least recently used signature makes room
    for (size_t x = 1; x < s.graphs.size(); ++x)
      if (s.graphs[x].used < s.graphs[gi].used) gi = x;
    cudaGraphExecDestroy(s.graphs[gi].exec);
    s.graphs[gi].exec = nullptr;
  }
  Slot::Graph &ge = s.graphs[gi];
  ge.shape = shape;
  if (!updated) {
    const cudaError_t ie = cudaGraphInstantiate(&ge.exec, g, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(g);
      ge.exec = nullptr;
      s.graphs.erase(s.graphs.begin() + (std::ptrdiff_t)gi);
      TSVD_CUDA(ie);
    }
  }
  ge.used = ++s.uses;
  cudaGraphDestroy(g);
  graph_time();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    ++(updated ? sv->stats.graph_updates : sv->stats.graph_instantiations);
  }
  TSVD_CUDA(cudaGraphLaunch(ge.exec, st));
  TSVD_CUDA(cudaEventRecord(s.done, st));
  return TSVD_OK;
}

// Complete one request (lock held): status and flags from its staged info.
void complete(tsvd_server_s *sv, const ReqPtr &r, tsvd_status st) {
  int flags = 0, status = st;
  int64_t apps = 0;
  if (st == TSVD_OK) {
    std::atomic_thread_fence(std::memory_order_acquire);
    const unsigned char *sp = sv->staging.base + r->soff;
    const int32_t *info = reinterpret_cast<const int32_t *>(sp);
    const double *sg = reinterpret_cast<const double *>(sp + al(r->k * 16));
    for (int l = 0; l < r->k; ++l) {
      apps += info[4 * l];
      if (info[4 * l + 1] == 1) flags |= TSVD_FLAG_NOCONV;
      if (info[4 * l + 1] == 2) flags |= TSVD_FLAG_RANK;
      if (info[4 * l + 2]) flags |= TSVD_FLAG_TIMEOUT;
    }
    for (int l = 1; l < r->k; ++l)
      if (sg[l] > sg[l - 1]) flags |= TSVD_FLAG_NONMONOTONE;
    status = (flags & TSVD_FLAG_TIMEOUT) ? TSVD_ETIMEDOUT
             : (flags & TSVD_FLAG_RANK)  ? TSVD_ERANK
             : (flags & TSVD_FLAG_NOCONV) ? TSVD_ENOCONV
                                          : TSVD_OK;
  }
  r->rec.status = status;
  r->rec.flags = flags;
  r->rec.applications = apps;
  r->rec.done_s = sv->now();
  r->done = true;
  sv->arena.release(r->off, r->bytes);
  if (r->slot >= 0) sv->free_flags.push_back(r->slot);
  r->slot = -1;
  if (r->copied) sv->event_pool.push_back(r->copied);
  r->copied = nullptr;
  --sv->inflight;
  if (status == TSVD_OK || status == TSVD_ENOCONV || status == TSVD_ERANK)
    ++sv->stats.completed;
  else
    ++sv->stats.failed;
}

void retire_slot(tsvd_server_s *sv, Slot &s) {
  if (s.dev_bytes) sv->arena.release(s.dev_off, s.dev_bytes);
  s.dev_bytes = 0;
  s.reqs.clear();
  s.busy = false;
}

void scheduler(tsvd_server_s *sv) {
  cudaSetDevice(sv->device);
  const int64_t l0 = launches_so_far();
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    bool progressed = false;
    // the flag mirror: requests whose cluster stored its ticket get their results copied out
    if (sv->poll_inflight) {
      const cudaError_t q = cudaEventQuery(sv->poll_done);
      if (q != cudaErrorNotReady) {
        sv->poll_inflight = false;
        if (q != cudaSuccess) sv->err = std::string("server: flag copy failed: ") + cudaGetErrorString(q);
        for (auto it = sv->running.begin(); q == cudaSuccess && it != sv->running.end();) {
          Request &r = **it;
          if (reinterpret_cast<volatile uint32_t *>(sv->hflags)[r.slot] == r.dq.ticket) {
            if (sv->event_pool.empty()) {
              cudaEvent_t e;
              if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
              sv->event_pool.push_back(e);
            }
            r.copied = sv->event_pool.back();
            sv->event_pool.pop_back();
            const size_t ob = staging_bytes(r.m, r.n, r.k);
            cudaMemcpyAsync(sv->staging.base + r.soff, reinterpret_cast<const unsigned char *>(r.dq.A) + r.out_off, ob,
                            cudaMemcpyDeviceToHost, sv->out_stream);
            cudaEventRecord(r.copied, sv->out_stream);
            sv->copying.push_back(*it);
            it = sv->running.erase(it);
            progressed = true;
          } else {
            ++it;
          }
        }
      }
    }
    if (!sv->poll_inflight && !sv->running.empty()) {
      cudaMemcpyAsync(sv->hflags, sv->dflags, (size_t)sv->opt.max_inflight * 4, cudaMemcpyDeviceToHost,
                      sv->poll_stream);
      cudaEventRecord(sv->poll_done, sv->poll_stream);
      sv->poll_inflight = true;
    }
    // results in the staging: the request is complete
    for (auto it = sv->copying.begin(); it != sv->copying.end();) {
      const cudaError_t q = cudaEventQuery((*it)->copied);
      if (q == cudaErrorNotReady) {
        ++it;
        continue;
      }
      complete(sv, *it, q == cudaSuccess ? TSVD_OK : TSVD_ECUDA);
      it = sv->copying.erase(it);
      progressed = true;
    }
    // finished waves release their descriptors; a failed wave fails what it has not completed
    for (auto &s : sv->slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        sv->err = std::string("server: wave failed: ") + cudaGetErrorString(q);
        for (auto &r : s.reqs) {
          if (r->done) continue;
          sv->running.remove(r);
          sv->copying.remove(r);
          complete(sv, r, TSVD_ECUDA);
        }
      }
      retire_slot(sv, s);
      progressed = true;
    }
    if (progressed) sv->cv_done.notify_all();
    // admission, first in first out
    while (!sv->pending.empty() && sv->inflight < sv->opt.max_inflight) {
      ReqPtr r = sv->pending.front();
      size_t off = 0, soff = 0;
      if (!sv->arena.alloc(r->bytes, &off)) break;
      if (!sv->staging.alloc(r->sbytes, &soff)) {
        sv->arena.release(off, r->bytes);
        break;
      }
      if (sv->free_flags.empty()) {
        sv->arena.release(off, r->bytes);
        sv->staging.release(soff, r->sbytes);
        break;
      }
      sv->pending.pop_front();
      r->off = off;
      r->soff = soff;
      r->admitted = true;
      r->slot = sv->free_flags.back();
      sv->free_flags.pop_back();
      carve(*r, sv->arena.base + off);
      r->dq.flag = sv->dflags + r->slot;
      r->dq.ticket = (uint32_t)(r->id & 0x7fffffffu) | 0x80000000u;  // never 0, the flags' initial value
      r->rec.admit_s = sv->now();
      ++sv->inflight;
      (r->heavy ? sv->admitted_heavy : sv->admitted).push_back(r);
      progressed = true;
    }
    // waves
    // heavy requests waiting and no idle heavy stream: open one more, up to heavy_streams
    if (!sv->admitted_heavy.empty()) {
      bool idle = false;
      for (size_t si = (size_t)sv->opt.n_streams; si < sv->slots.size(); ++si) idle |= !sv->slots[si].busy;
      if (!idle && (int)sv->slots.size() < sv->opt.n_streams + sv->opt.heavy_streams) {
        Slot ns;
        if (cudaStreamCreateWithFlags(&ns.stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&ns.done, cudaEventDisableTiming) == cudaSuccess) {
          sv->slots.push_back(ns);
        } else {
          cudaGetLastError();
          if (ns.stream) cudaStreamDestroy(ns.stream);
        }
      }
    }
    for (size_t si = 0; si < sv->slots.size(); ++si) {
      Slot &s = sv->slots[si];
      // the first n_streams streams take light requests only, the heavy streams heavy ones
      // only, so a light wave never waits behind a heavy request's long power phase
      std::deque<ReqPtr> &q = si < (size_t)sv->opt.n_streams ? sv->admitted : sv->admitted_heavy;
      if (s.busy || q.empty()) continue;
      const size_t take = std::min(q.size(), (size_t)sv->opt.max_wave);
      s.reqs.assign(q.begin(), q.begin() + take);
      q.erase(q.begin(), q.begin() + take);
      s.busy = true;
      s.wave = sv->stats.waves++;
      const double t = sv->now();
      for (auto &r : s.reqs) {
        r->rec.launch_s = t;
        r->rec.wave = (int32_t)s.wave;
      }
      {
        int64_t nb = 0;
        for (auto &o : sv->slots) nb += o.busy ? 1 : 0;
        sv->stats.peak_streams_busy = std::max(sv->stats.peak_streams_busy, nb);
      }
      lk.unlock();
      const auto h0 = std::chrono::steady_clock::now();
      const tsvd_status st = launch_wave(sv, s);
      const double hs = std::chrono::duration<double>(std::chrono::steady_clock::now() - h0).count();
      lk.lock();
      sv->stats.wave_host_s += hs;
      for (auto &r : s.reqs) {
        r->rec.cluster = r->dq.cluster;
        if (st == TSVD_OK) sv->running.push_back(r);
      }
      if (st != TSVD_OK) {
        sv->err = std::string("server: launching a wave failed: ") + tsvd_last_cuda_error();
        lk.unlock();
        cudaStreamSynchronize(s.stream);
        lk.lock();
        for (auto &r : s.reqs) complete(sv, r, st);
        retire_slot(sv, s);
        sv->cv_done.notify_all();
      }
      progressed = true;
    }
    sv->stats.kernel_launches = launches_so_far() - l0;
    sv->stats.peak_device_bytes = (int64_t)sv->arena.peak;
    bool any_busy = !sv->running.empty() || !sv->copying.empty() || sv->poll_inflight;
    for (auto &s : sv->slots) any_busy |= s.busy;
    const double t = sv->now();
    if (any_busy && sv->busy_since < 0) sv->busy_since = t;
    if (!any_busy && sv->busy_since >= 0) {
      sv->stats.busy_s += t - sv->busy_since;
      sv->busy_since = -1.0;
    }
    if (sv->stop && !any_busy) break;
    if (!progressed) {
      if (any_busy)
        sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

__global__ void fill_uniform_kernel(float *a, int64_t count, uint32_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), seed, 0x41554e45u};
    philox10(c, 0x12345678u, seed);
    a[i] = (float)((double)c[0] * 0x1.0p-31 - 1.0);
  }
}

// Time the power kernel on `nreq` synthetic d x d requests with cluster c
// (`iters` applications per triplet, k = 2).  Returns milliseconds.
tsvd_status time_power(tsvd_server_s *sv, int64_t d, int c, int nreq, int iters, cudaStream_t st, cudaEvent_t e0,
                       cudaEvent_t e1, double *ms_out) {
  const int k = 2;
  const size_t per = request_bytes(d, d, k);
  const int T = (int)ceil_div(d, kSrvTile);
  const size_t ntiles = (size_t)nreq * T * (T + 1) / 2;
  const size_t need = per * nreq + al(nreq * sizeof(SrvReq)) + al(ntiles * sizeof(SrvTile)) + al(nreq * 4);
  size_t off = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->arena.alloc(need, &off)) return TSVD_EBUDGET;
  }
  const size_t smem_cap = power_smem_budget();
  const int resident = srv_power_smem(d, c, 1) <= smem_cap ? 1 : 0;
  unsigned char *base = sv->arena.base + off;
  SrvReq *dreq = reinterpret_cast<SrvReq *>(base + per * nreq);
  SrvTile *dtiles = reinterpret_cast<SrvTile *>(base + per * nreq + al(nreq * sizeof(SrvReq)));
  uint32_t *dflags = reinterpret_cast<uint32_t *>(base + per * nreq + al(nreq * sizeof(SrvReq)) +
                                                  al(ntiles * sizeof(SrvTile)));
  std::vector<SrvReq> reqs(nreq);
  std::vector<SrvTile> tiles;
  tsvd_status ls = TSVD_OK;
  for (int i = 0; i < nreq && ls == TSVD_OK; ++i) {
    Request r;
    r.m = d;
    r.n = d;
    r.k = k;
    r.eps = 1e-300;  // never met: every triplet runs exactly max_iter applications
    r.max_iter = iters;
    r.seed = (uint64_t)i;
    carve(r, base + per * i);
    r.dq.cluster = c;
    r.dq.resident = resident;
    r.dq.flag = dflags + i;
    r.dq.ticket = 1u;
    if (!srv_req_complete(r.dq)) ls = TSVD_EINVAL;
    reqs[i] = r.dq;
    fill_uniform_kernel<<<64, 256, 0, st>>>(const_cast<float *>(r.dq.A), d * d, (uint32_t)i);
    if (cudaGetLastError() != cudaSuccess) ls = TSVD_ECUDA;
    for (int ti = 0; ti < T; ++ti)
      for (int tj = 0; tj <= ti; ++tj) tiles.push_back({i, ti, tj, 0});
  }
  if (ls == TSVD_OK && cudaMemcpyAsync(dreq, reqs.data(), nreq * sizeof(SrvReq), cudaMemcpyHostToDevice, st) != cudaSuccess)
    ls = TSVD_ECUDA;
  if (ls == TSVD_OK &&
      cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(SrvTile), cudaMemcpyHostToDevice, st) != cudaSuccess)
    ls = TSVD_ECUDA;
  if (ls == TSVD_OK) ls = launch_srv_syrk(dreq, dtiles, (int)tiles.size(), st);
  const size_t smem = srv_power_smem(d, c, resident);
  if (ls == TSVD_OK) ls = launch_srv_power(dreq, nreq, c, smem, st);  // warm-up
  if (ls == TSVD_OK && cudaEventRecord(e0, st) != cudaSuccess) ls = TSVD_ECUDA;
  if (ls == TSVD_OK) ls = launch_srv_power(dreq, nreq, c, smem, st);
  if (ls == TSVD_OK && cudaEventRecord(e1, st) != cudaSuccess) ls = TSVD_ECUDA;
  float ms = 0.f;
  if (ls == TSVD_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    ls = TSVD_ECUDA;
  cudaStreamSynchronize(st);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->arena.release(off, need);
  }
  *ms_out = ms;
  return ls;
}

// Time the grouped Gram step on `nreq` synthetic tall requests of K x d, on the
// tensor cores (tc) or on the CUDA cores: a warm-up launch sequence, then one
// timed.  Milliseconds of the timed one.
tsvd_status time_syrk(tsvd_server_s *sv, int64_t d, int64_t K, int nreq, bool tc, cudaStream_t st, cudaEvent_t e0,
                      cudaEvent_t e1, double *ms_out) {
  const int k = 2;
  const size_t per = al(request_bytes(K, d, k, tc));
  size_t off = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->arena.alloc(per * nreq, &off)) return TSVD_EBUDGET;
  }
  unsigned char *base = sv->arena.base + off;
  std::vector<ReqPtr> rs(nreq);
  tsvd_status ls = TSVD_OK;
  for (int i = 0; i < nreq && ls == TSVD_OK; ++i) {
    rs[i] = std::make_shared<Request>();
    Request &r = *rs[i];
    r.m = K;
    r.n = d;
    r.k = k;
    r.eps = 0.5;
    r.max_iter = 1;
    r.tc = tc;
    carve(r, base + per * i);
    fill_uniform_kernel<<<64, 256, 0, st>>>(const_cast<float *>(r.dq.A), K * d, (uint32_t)i);
    if (cudaGetLastError() != cudaSuccess) ls = TSVD_ECUDA;
  }
  std::vector<SrvTile> tiles;
  TcWave tw;
  if (ls == TSVD_OK && tc) ls = build_tc_wave(rs, &tw);
  if (!tc) {
    const int T = (int)ceil_div(d, kSrvTile);
    for (int i = 0; i < nreq; ++i)
      for (int ti = 0; ti < T; ++ti)
        for (int tj = 0; tj <= ti; ++tj) tiles.push_back({i, ti, tj, 0});
  }
  const size_t o_tiles = al(nreq * sizeof(SrvReq)), o_tc = o_tiles + al(tiles.size() * sizeof(SrvTile));
  const size_t o_err = o_tc + tw.bytes, need = o_err + al(4);
  size_t doff = 0;
  bool have_d = false;
  if (ls == TSVD_OK) {
    std::lock_guard<std::mutex> lk(sv->mu);
    have_d = sv->arena.alloc(need, &doff);
    if (!have_d) ls = TSVD_EBUDGET;
  }
  std::vector<unsigned char> stage(need, 0);
  unsigned char *dev = have_d ? sv->arena.base + doff : nullptr;
  if (ls == TSVD_OK) {
    for (int i = 0; i < nreq; ++i) {
      rs[i]->dq.gram_err = tc ? reinterpret_cast<int32_t *>(dev + o_err) : nullptr;
      reinterpret_cast<SrvReq *>(stage.data())[i] = rs[i]->dq;
    }
    std::memcpy(stage.data() + o_tiles, tiles.data(), tiles.size() * sizeof(SrvTile));
    stage_tc_wave(tw, stage.data() + o_tc);
    if (cudaMemcpyAsync(dev, stage.data(), need, cudaMemcpyHostToDevice, st) != cudaSuccess) ls = TSVD_ECUDA;
  }
  auto run = [&]() -> tsvd_status {
    const SrvReq *dreq = reinterpret_cast<const SrvReq *>(dev);
    if (tc) return launch_tc_wave(tw, dreq, dev + o_tc, reinterpret_cast<int32_t *>(dev + o_err), st);
    return launch_srv_syrk(dreq, reinterpret_cast<const SrvTile *>(dev + o_tiles), (int)tiles.size(), st);
  };
  if (ls == TSVD_OK) ls = run();  // warm-up
  if (ls == TSVD_OK && cudaEventRecord(e0, st) != cudaSuccess) ls = TSVD_ECUDA;
  if (ls == TSVD_OK) ls = run();
  if (ls == TSVD_OK && cudaEventRecord(e1, st) != cudaSuccess) ls = TSVD_ECUDA;
  float ms = 0.f;
  if (ls == TSVD_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    ls = TSVD_ECUDA;
  cudaStreamSynchronize(st);  // the copy of `stage` and every launch are done before it is freed
  int32_t herr = 0;
  if (ls == TSVD_OK && tc && cudaMemcpy(&herr, dev + o_err, 4, cudaMemcpyDeviceToHost) == cudaSuccess && herr)
    ls = TSVD_ETIMEDOUT;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->arena.release(off, per * nreq);
    if (have_d) sv->arena.release(doff, need);
  }
  *ms_out = ms;
  return ls;
}

// Sparse requests with at least this many stored entries run one operator
// application per host round trip (the plan's explicit loop), with kernels
// over every SM; smaller ones run each triplet in one cooperative launch.
constexpr int64_t kLargeCsrNnz = (int64_t)1 << 25;
// large sparse requests on the device at once
constexpr int kLargeCsrConcurrent = 2;

// A sparse request runs through the plan API on a stream of its worker: the
// workspace comes from the server's device arena (first fit; the worker waits
// while the arena is full), the outputs go straight into the caller's
// buffers, and the request completes when tsvd_factor returns.  Dense waves
// keep running on their own streams meanwhile.
void csr_worker(tsvd_server_s *sv) {
  cudaSetDevice(sv->device);
  // small requests take the highest stream priority: their cooperative launches wait for
  // whole SMs, and the block scheduler then serves them before the dense waves' pending
  // blocks.  Large requests (seconds of back-to-back launches over every SM) take the
  // default priority and run at most kLargeCsrConcurrent at a time, so that the dense
  // waves keep their share of the SMs instead of queueing behind them.
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t st_hi = nullptr, st_lo = nullptr;
  if (cudaStreamCreateWithPriority(&st_hi, cudaStreamNonBlocking, hi) != cudaSuccess) return;
  if (cudaStreamCreateWithPriority(&st_lo, cudaStreamNonBlocking, lo) != cudaSuccess) {
    cudaStreamDestroy(st_hi);
    return;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    sv->cv_csr.wait(lk, [&] { return sv->stop || !sv->csr_pending.empty(); });
    if (sv->csr_pending.empty()) break;  // stop, nothing left
    ReqPtr r = sv->csr_pending.front();
    sv->csr_pending.pop_front();
    const bool large = r->nnz >= kLargeCsrNnz;
    if (large) {
      // a stopping server still runs what was submitted (the destructor waits for it)
      sv->cv_csr.wait(lk, [&] { return sv->csr_large_running < kLargeCsrConcurrent; });
      ++sv->csr_large_running;
    }
    cudaStream_t st = large ? st_lo : st_hi;
    r->rec.admit_s = sv->now();
    lk.unlock();
    tsvd_matrix A{};
    A.kind = TSVD_CSR_F32_I32_I64;
    A.location = TSVD_HOST;
    A.m = r->m;
    A.n = r->n;
    A.values = r->A;
    A.row_ptr = r->row_ptr;
    A.col_idx = r->col_idx;
    A.nnz = r->nnz;
    tsvd_options opt;
    tsvd_options_init(&opt);
    opt.max_iter = r->max_iter;
    opt.seed = r->seed;
    opt.sign_convention = r->sign;
    opt.iters_override = r->iters.empty() ? nullptr : r->iters.data();
    opt.out_location = TSVD_HOST;
    // a smaller cooperative grid than a lone request takes (128), so that several sparse
    // requests and the dense waves share the GPU: measured on the serving mix, 64 blocks
    // gave 163 solves/s against 139 and dense p99 75 ms against 222 ms at 0.9x capacity
    opt.csr_coop_blocks = 64;
    // at most a quarter of the arena per sparse request (the plan streams A beyond that)
    opt.device_budget = std::max<size_t>(sv->arena.size / 4, (size_t)64 << 20);
    tsvd_plan_t plan = nullptr;
    size_t ws_bytes = 0;
    tsvd_status st_r = tsvd_plan(&plan, &A, r->k, r->iters.empty() ? r->eps : 0.5, &opt, &ws_bytes);
    size_t off = 0;
    bool have = false;
    if (st_r == TSVD_OK) {
      lk.lock();
      const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(600);
      while (!(have = sv->arena.alloc(std::max<size_t>(ws_bytes, 256), &off)) && !sv->stop) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
      }
      lk.unlock();
      if (!have) st_r = TSVD_EBUDGET;
    }
    tsvd_report rep{};
    std::vector<int32_t> its((size_t)r->k, 0);
    rep.iters = its.data();
    if (st_r == TSVD_OK) {
      r->rec.launch_s = sv->now();
      st_r = tsvd_factor(plan, &A, sv->arena.base + off, ws_bytes, st, r->U, r->sigma, r->V, &rep);
    }
    if (plan) tsvd_destroy(plan);
    lk.lock();
    if (large) {
      --sv->csr_large_running;
      sv->cv_csr.notify_all();
    }
    if (have) sv->arena.release(off, std::max<size_t>(ws_bytes, 256));
    if (st_r != TSVD_OK && st_r != TSVD_ENOCONV && st_r != TSVD_ERANK)
      sv->err = std::string("server: sparse request failed: ") + tsvd_status_string(st_r) + " " + tsvd_last_cuda_error();
    r->rec.status = st_r;
    r->rec.flags = rep.flags;
    r->rec.applications = rep.applications;
    r->rec.done_s = sv->now();
    r->rec.cluster = 0;
    r->rec.wave = -1;
    r->done = true;
    --sv->inflight;
    if (st_r == TSVD_OK || st_r == TSVD_ENOCONV || st_r == TSVD_ERANK)
      ++sv->stats.completed;
    else
      ++sv->stats.failed;
    sv->cv_done.notify_all();
  }
  lk.unlock();
  for (cudaStream_t st : {st_hi, st_lo}) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

}  // namespace
}  // namespace tsvd

using namespace tsvd;

extern "C" {

tsvd_status tsvd_server_options_init(tsvd_server_options *opt) {
  if (!opt) return TSVD_EINVAL;
  std::memset(opt, 0, sizeof *opt);
  opt->device_budget = (size_t)8 << 30;
  opt->max_inflight = 4096;
  opt->n_streams = 8;
  opt->max_wave = 64;
  opt->cluster_cap = 8;
  opt->host_staging = (size_t)2 << 30;
  return TSVD_OK;
}

tsvd_status tsvd_server_create(tsvd_server_t *out, const tsvd_server_options *opt_in) {
  if (!out) return TSVD_EINVAL;
  *out = nullptr;
  tsvd_server_options opt;
  tsvd_server_options_init(&opt);
  if (opt_in) {
    const tsvd_server_options d = opt;
    opt = *opt_in;
    if (!opt.device_budget) opt.device_budget = d.device_budget;
    if (!opt.max_inflight) opt.max_inflight = d.max_inflight;
    if (!opt.n_streams) opt.n_streams = d.n_streams;
    if (!opt.max_wave) opt.max_wave = d.max_wave;
    if (!opt.cluster_cap) opt.cluster_cap = d.cluster_cap;
    if (!opt.host_staging) opt.host_staging = d.host_staging;
  }
  if (opt.max_inflight < 1 || opt.n_streams < 1 || opt.n_streams > 64 || opt.max_wave < 1 ||
      (opt.cluster_cap != 1 && opt.cluster_cap != 2 && opt.cluster_cap != 4 && opt.cluster_cap != 8))
    return TSVD_EINVAL;
  if (opt.heavy_dim == 0) opt.heavy_dim = -1;  // one lane unless asked for
  if (opt.heavy_streams == 0) opt.heavy_streams = 64 - opt.n_streams;
  if (opt.heavy_dim < -1 || opt.heavy_streams < 0 || opt.n_streams + opt.heavy_streams > 64) return TSVD_EINVAL;
  if (opt.heavy_dim >= 0 && opt.heavy_streams == 0) return TSVD_EINVAL;  // a heavy lane needs a stream
  auto *sv = new tsvd_server_s();
  sv->opt = opt;
  sv->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&sv->device);
  tsvd_status st = sv->arena.init(opt.device_budget, false);
  if (st == TSVD_OK) st = sv->staging.init(opt.host_staging, true);
  if (st != TSVD_OK) {
    sv->arena.destroy();
    sv->staging.destroy();
    delete sv;
    return st;
  }
  {
    const size_t fb = (size_t)opt.max_inflight * 4;
    if (cudaMalloc(&sv->dflags, fb) != cudaSuccess || cudaMemset(sv->dflags, 0, fb) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&sv->hflags), fb, cudaHostAllocPortable) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->poll_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->out_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->poll_done, cudaEventDisableTiming) != cudaSuccess) {
      set_cuda_error(cudaGetLastError(), "server flags", __FILE__, __LINE__);
      tsvd_server_destroy(sv);
      return TSVD_ECUDA;
    }
    for (int32_t i = opt.max_inflight - 1; i >= 0; --i) sv->free_flags.push_back(i);
  }
  sv->slots.resize(opt.n_streams);
  for (auto &s : sv->slots) {
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
      set_cuda_error(cudaGetLastError(), "server streams", __FILE__, __LINE__);
      tsvd_server_destroy(sv);
      return TSVD_ECUDA;
    }
  }
  sv->thr = std::thread(scheduler, sv);
  for (int i = 0; i < 8; ++i) sv->csr_workers.emplace_back(csr_worker, sv);
  *out = sv;
  return TSVD_OK;
}

tsvd_status tsvd_server_submit(tsvd_server_t sv, const float *A, int64_t m, int64_t n, int32_t k, double eps,
                               int32_t max_iter, uint64_t seed, int32_t sign_convention, const int32_t *iters_override,
                               float *U, double *sigma, float *V, uint64_t *ticket) {
  if (!sv || !A || !U || !sigma || !V || !ticket || m <= 0 || n <= 0) return TSVD_EINVAL;
  const int64_t d = std::min(m, n);
  if (k < 1 || k > d) return TSVD_EINVAL;
  if (!iters_override && !(eps > 0.0 && eps < 1.0)) return TSVD_EINVAL;
  if (iters_override)
    for (int32_t l = 0; l < k; ++l)
      if (iters_override[l] < 1) return TSVD_EINVAL;
  if (d > kSrvMaxDim || k > kSrvMaxK) return TSVD_EUNSUPPORTED;
  auto r = std::make_shared<Request>();
  r->A = A;
  r->m = m;
  r->n = n;
  r->k = k;
  r->eps = eps;
  r->max_iter = max_iter > 0 ? max_iter : 10000;
  r->seed = seed;
  r->sign = sign_convention ? 1 : 0;
  r->U = U;
  r->sigma = sigma;
  r->V = V;
  if (iters_override) r->iters.assign(iters_override, iters_override + k);
  r->tc = d >= sv->tc_min_d.load();
  r->heavy = sv->opt.heavy_dim >= 0 && d > sv->opt.heavy_dim;
  r->bytes = request_bytes(m, n, k, r->tc);
  r->sbytes = staging_bytes(m, n, k);
  if (al(r->bytes) > sv->arena.size || al(r->sbytes) > sv->staging.size) return TSVD_EBUDGET;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return TSVD_EINVAL;
    r->id = sv->next_id++;
    r->rec.submit_s = sv->now();
    sv->table[r->id] = r;
    sv->pending.push_back(r);
    ++sv->stats.submitted;
    *ticket = r->id;
  }
  sv->cv_work.notify_one();
  return TSVD_OK;
}

tsvd_status tsvd_server_submit_csr(tsvd_server_t sv, const int64_t *row_ptr, const int32_t *col_idx,
                                   const float *values, int64_t m, int64_t n, int64_t nnz, int32_t k, double eps,
                                   int32_t max_iter, uint64_t seed, int32_t sign_convention,
                                   const int32_t *iters_override, float *U, double *sigma, float *V,
                                   uint64_t *ticket) {
  if (!sv || !row_ptr || !U || !sigma || !V || !ticket || m <= 0 || n <= 0 || nnz < 0) return TSVD_EINVAL;
  if (nnz > 0 && (!col_idx || !values)) return TSVD_EINVAL;
  if (k < 1 || k > std::min(m, n)) return TSVD_EINVAL;
  if (m < n) return TSVD_EUNSUPPORTED;  // the sparse path applies A^T (A v) on R^n
  if (!iters_override && !(eps > 0.0 && eps < 1.0)) return TSVD_EINVAL;
  if (iters_override)
    for (int32_t l = 0; l < k; ++l)
      if (iters_override[l] < 1) return TSVD_EINVAL;
  auto r = std::make_shared<Request>();
  r->csr = true;
  r->A = values;
  r->row_ptr = row_ptr;
  r->col_idx = col_idx;
  r->nnz = nnz;
  r->m = m;
  r->n = n;
  r->k = k;
  r->eps = eps;
  r->max_iter = max_iter > 0 ? max_iter : 10000;
  r->seed = seed;
  r->sign = sign_convention ? 1 : 0;
  r->U = U;
  r->sigma = sigma;
  r->V = V;
  if (iters_override) r->iters.assign(iters_override, iters_override + k);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return TSVD_EINVAL;
    r->id = sv->next_id++;
    r->rec.submit_s = sv->now();
    sv->table[r->id] = r;
    sv->csr_pending.push_back(r);
    ++sv->inflight;
    ++sv->stats.submitted;
    *ticket = r->id;
  }
  sv->cv_csr.notify_all();  // a worker may be parked on the large-request limit
  return TSVD_OK;
}

tsvd_status tsvd_server_wait(tsvd_server_t sv, uint64_t ticket, double timeout_s, tsvd_request_info *info) {
  if (!sv) return TSVD_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->table.find(ticket);
  if (it == sv->table.end()) return TSVD_EINVAL;
  ReqPtr r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_s < 0) {
    sv->cv_done.wait(lk, pred);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return TSVD_ETIMEDOUT;
  }
  sv->table.erase(ticket);
  const bool staged = r->admitted;
  lk.unlock();
  if (staged) {
    // results from the staging into the caller's buffers (the kernel has finished with them)
    const tsvd_status s = (tsvd_status)r->rec.status;
    if (s == TSVD_OK || s == TSVD_ENOCONV || s == TSVD_ERANK) {
      const unsigned char *sp = sv->staging.base + r->soff + al(r->k * 16);
      std::memcpy(r->sigma, sp, (size_t)r->k * 8);
      sp += al(r->k * 8);
      std::memcpy(r->U, sp, (size_t)r->m * r->k * 4);
      sp += al(r->m * r->k * 4);
      std::memcpy(r->V, sp, (size_t)r->n * r->k * 4);
    }
    lk.lock();
    sv->staging.release(r->soff, r->sbytes);
    lk.unlock();
  }
  if (info) *info = r->rec;
  return (tsvd_status)r->rec.status;
}

tsvd_status tsvd_server_get_stats(tsvd_server_t sv, tsvd_server_stats *stats) {
  if (!sv || !stats) return TSVD_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *stats = sv->stats;
  if (sv->busy_since >= 0) stats->busy_s += sv->now() - sv->busy_since;
  return TSVD_OK;
}

const char *tsvd_server_last_error(tsvd_server_t sv) { return sv ? sv->err.c_str() : ""; }

int64_t tsvd_server_tc_min_d(tsvd_server_t sv) { return sv ? sv->tc_min_d.load() : 0; }

tsvd_status tsvd_server_autotune_syrk_times(tsvd_server_t sv, int64_t *d, double *ms_tensor, double *ms_cuda,
                                            int32_t *requests) {
  if (!sv || !d || !ms_tensor || !ms_cuda || !requests) return TSVD_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  for (int b = 0; b < 4; ++b) {
    d[b] = (int64_t)256 << b;
    ms_tensor[b] = sv->syrk_ms_tc[b];
    ms_cuda[b] = sv->syrk_ms_cc[b];
    requests[b] = sv->syrk_nreq[b];
  }
  return TSVD_OK;
}

tsvd_status tsvd_server_set_tc_min_d(tsvd_server_t sv, int64_t d) {
  if (!sv || d < 1) return TSVD_EINVAL;
  sv->tc_min_d.store(d);
  return TSVD_OK;
}

int32_t tsvd_server_cluster_for(tsvd_server_t sv, int64_t d) {
  if (!sv || d <= 0) return 0;
  std::lock_guard<std::mutex> lk(sv->mu);
  return cluster_for(sv, d);
}

tsvd_status tsvd_server_set_cluster_for(tsvd_server_t sv, int64_t d, int32_t c) {
  if (!sv || d <= 0 || d > kSrvMaxDim || (c != 1 && c != 2 && c != 4 && c != 8) || c > sv->opt.cluster_cap)
    return TSVD_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->cluster_table[bucket_of(d)] = c;
  return TSVD_OK;
}

tsvd_status tsvd_server_autotune(tsvd_server_t sv, int32_t iters) {
  if (!sv || iters < 1) return TSVD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->inflight || !sv->pending.empty()) return TSVD_EINVAL;
  }
  DeviceInfo di;
  TSVD_TRY(device_info(&di));
  cudaStream_t st = nullptr;
  TSVD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  TSVD_CUDA(cudaEventCreate(&e0));
  TSVD_CUDA(cudaEventCreate(&e1));
  const int64_t dims[6] = {64, 128, 256, 512, 1024, 2048};
  tsvd_status result = TSVD_OK;
  for (int b = 0; b < 6 && result == TSVD_OK; ++b) {
    const int64_t d = dims[b];
    // per cluster size: the time of one request alone
    std::vector<int> cs;
    std::vector<double> lat;
    for (int c = 1; c <= sv->opt.cluster_cap; c *= 2) {
      if (clamp_cluster(d, c) != c) break;
      double ms1 = 0.0;
      result = time_power(sv, d, c, 1, iters, st, e0, e1, &ms1);
      if (result != TSVD_OK) break;
      cs.push_back(c);
      lat.push_back(ms1);
    }
    if (result != TSVD_OK || cs.empty()) break;
    // the fastest lone request, a larger cluster taken only where it cuts the time by more
    // than 15 %.  On the serving mix a request holds its CTAs, its arena memory and its
    // wave's stream until it is done, so the fastest request frees them soonest: measured
    // on 10,000 dense requests, the largest clusters d allows gave 1,403 solves/s against
    // 1,238 for the table that maximised whole-GPU throughput per size (and 937 / 452 with
    // clusters capped at 4 / 2 CTAs), and p99 0.33 s against 0.79 s at 0.9x capacity.  For
    // small d a larger cluster saves little time for many more CTAs: a 5 % rule put 8-CTA
    // clusters on d = 128 and gave p99 0.57 s at 0.9x capacity
    double best_lat = lat[0];
    int best_c = cs[0];
    for (size_t i = 1; i < cs.size(); ++i)
      if (lat[i] < 0.85 * best_lat) {
        best_lat = lat[i];
        best_c = cs[i];
      }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->cluster_table[b] = best_c;
  }
  // the Gram step's tile shape per size: 128 x 256 tensor-core tiles (3xTF32) against
  // 64 x 64 CUDA-core tiles (FP32), on as many K = 8192 requests as give both kernels
  // work for every SM (within half of the arena); tensor cores from the smallest d at
  // which they are faster there and at every larger size
  if (result == TSVD_OK && di.cc_major == 10) {
    const int64_t tdims[4] = {256, 512, 1024, 2048};
    bool tc_wins[4] = {false, false, false, false};
    const int64_t K = 8192;
    for (int b = 0; b < 4 && result == TSVD_OK; ++b) {
      const int64_t d = tdims[b];
      const size_t per = al(request_bytes(K, d, 2, true));
      const int64_t want = std::max<int64_t>(1, ceil_div(2 * (int64_t)di.sms, srv_tc_tiles(d)));
      const int nreq = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)(sv->arena.size / 2 / per) / 2));
      double ms_tc = 0.0, ms_cc = 0.0;
      result = time_syrk(sv, d, K, nreq, true, st, e0, e1, &ms_tc);
      if (result == TSVD_OK) result = time_syrk(sv, d, K, nreq, false, st, e0, e1, &ms_cc);
      if (result == TSVD_OK) {
        tc_wins[b] = ms_tc < ms_cc;
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->syrk_ms_tc[b] = ms_tc;
        sv->syrk_ms_cc[b] = ms_cc;
        sv->syrk_nreq[b] = nreq;
      }
      if (result == TSVD_EBUDGET) result = TSVD_OK;  // a budget too small for the size: keep the default
    }
    if (result == TSVD_OK) {
      int64_t from = INT64_MAX;
      for (int b = 3; b >= 0 && tc_wins[b]; --b) from = tdims[b];
      sv->tc_min_d.store(from);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return result;
}

void tsvd_server_destroy(tsvd_server_t sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (auto &r : sv->pending) {
      r->rec.status = TSVD_ECUDA;
      r->done = true;
    }
    sv->pending.clear();
    for (auto &r : sv->csr_pending) {
      r->rec.status = TSVD_ECUDA;
      r->done = true;
      --sv->inflight;
    }
    sv->csr_pending.clear();
  }
  sv->cv_work.notify_all();
  sv->cv_csr.notify_all();
  for (auto &t : sv->csr_workers)
    if (t.joinable()) t.join();
  if (sv->thr.joinable()) sv->thr.join();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto *qq : {&sv->admitted, &sv->admitted_heavy}) {
      for (auto &r : *qq) {
        r->rec.status = TSVD_ECUDA;
        r->done = true;
      }
      qq->clear();
    }
  }
  sv->cv_done.notify_all();
  for (auto &s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    for (auto &x : s.graphs)
      if (x.exec) cudaGraphExecDestroy(x.exec);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stage) cudaFreeHost(s.stage);
    for (unsigned char *p : s.stage_old) cudaFreeHost(p);
  }
  for (cudaStream_t st : {sv->poll_stream, sv->out_stream})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  if (sv->poll_done) cudaEventDestroy(sv->poll_done);
  for (auto e : sv->event_pool) cudaEventDestroy(e);
  if (sv->dflags) cudaFree(sv->dflags);
  if (sv->hflags) cudaFreeHost(sv->hflags);
  sv->arena.destroy();
  sv->staging.destroy();
  delete sv;
}

}  // extern "C"
