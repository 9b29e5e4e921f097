"""Benchmark: dense out-of-core truncated SVD (deflated power method) on one GB300.

Workload (the paper's dense synthetic case scaled to this host): A is m x 4096
FP32 row-major, rank-64 with sigma_i = 1/(1+i) plus 1e-4 N(0,1) noise, stored
in page-locked host memory in row blocks of 262,144 rows; k = 16, eps = 1e-6.
m is 13,107,200 rows (200 GiB) when the host can pin it, otherwise the largest
multiple of 262,144 rows that fits (stated in config.m).

One step = one full t-SVD: Gram pass over A, k power iterations, U pass.
Metric: A-stream throughput = bytes of A consumed by the t-SVD (two passes,
2 m n 4 bytes) / t-SVD seconds (higher is better).
  value : A resident in HBM, outputs on the device, CUDA events on the stream.
  e2e   : A in pinned host memory, streamed under a 32 GB device budget,
          outputs copied back to host memory, all copies inside the timed region.

--impl reference runs the FP64 CPU oracle on the host cores over a bounded
sample of the same workload (one row block per step).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BLOCK_ROWS = 262_144
N_COLS = 4096
RANK = 64
K = 16
EPS = 1e-6
NOISE = 1e-4
FULL_M = 13_107_200
BUDGET = 32 * 10 ** 9
PREC_NAMES = {0: "f32", 1: "tf32", 2: "tf32x3", 3: "bf16x3"}


def mem_available_bytes() -> int:
    for line in open("/proc/meminfo"):
        if line.startswith("MemAvailable:"):
            return int(line.split()[1]) * 1024
    return 0


def pick_m(requested: int | None) -> int:
    if requested:
        return requested
    avail = mem_available_bytes() - 40 * 2 ** 30
    blocks = max(1, min(FULL_M // BLOCK_ROWS, avail // (BLOCK_ROWS * N_COLS * 4)))
    return int(blocks * BLOCK_ROWS)


def source_digest(*paths) -> str:
    """sha256 over the source a stored ncu capture measured.  An entry is a
    file path, or "path#start#end": the text from the first line containing
    `start` (empty: the file's start) up to the next line containing `end`
    (empty: its end), so that host-side edits of a file leave the digest of
    its device code unchanged."""
    import hashlib
    h = hashlib.sha256()
    for ent in paths:
        pth, start, end = (ent.split("#") + ["", ""])[:3] if "#" in ent else (ent, "", "")
        with open(os.path.join(ROOT, pth), "r", encoding="utf-8") as f:
            lines = f.read().split("\n")
        i0 = next((i for i, ln in enumerate(lines) if start in ln), 0) if start else 0
        i1 = next((i for i in range(i0 + 1, len(lines)) if end in lines[i]), len(lines)) if end else len(lines)
        h.update("\n".join(lines[i0:i1]).encode("utf-8"))
    return h.hexdigest()


def measured_traffic(kernel: str, rows: int, n: int):
    """DRAM bytes (read + write) per launch from the committed ncu capture of
    `kernel`, or None when no capture matches this launch configuration or the
    kernel's source changed since the capture."""
    pth = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(pth):
        return None
    rec = json.load(open(pth)).get(kernel)
    if not rec or rec.get("rows") != rows or rec.get("n") != n:
        return None
    if rec.get("source_sha256") != source_digest(*rec["sources"]):
        return None
    return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        load = [s for s in sm]
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ----------------------------------------------------------------------------- workload
def make_host_A(m: int, seed: int):
    """Pinned host buffer (library allocator) filled on the GPU by the seeded generator."""
    import torch

    import synth
    from paper_2208_08410_gb300 import _binding as B
    ptr = C.c_void_p()
    B.check(B.tsvd_host_alloc(C.byref(ptr), m * N_COLS * 4), "tsvd_host_alloc")
    A = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_float)), shape=(m, N_COLS))
    At = torch.from_numpy(A)
    sigma = 1.0 / (1.0 + np.arange(RANK))
    facts = synth.dense_lowrank_blocks_torch(At, m, N_COLS, RANK, sigma, NOISE, seed, BLOCK_ROWS)
    return A, ptr, facts


def thp_coverage(arr: np.ndarray) -> dict:
    """Resident and huge-page-backed bytes of the mappings that hold `arr`
    (from /proc/self/smaps), to see whether the page-locked buffer got the
    transparent huge pages its allocator asked for."""
    lo = arr.__array_interface__["data"][0]
    hi = lo + arr.nbytes
    rss = huge = 0
    cur = False
    try:
        for ln in open("/proc/self/smaps"):
            parts = ln.split()
            if parts and "-" in parts[0] and len(parts) >= 5 and not parts[0].endswith(":"):
                a, b = (int(x, 16) for x in parts[0].split("-"))
                cur = a < hi and b > lo
            elif cur and parts[0] == "Rss:":
                rss += int(parts[1]) * 1024
            elif cur and parts[0] == "AnonHugePages:":
                huge += int(parts[1]) * 1024
    except OSError:
        return {}
    return {"rss_GiB": round(rss / 2 ** 30, 2), "huge_GiB": round(huge / 2 ** 30, 2),
            "huge_frac": round(huge / rss, 4) if rss else None}


def thp_by_block(arr: np.ndarray, block_bytes: int, samples: int = 16):
    """Per block of `arr`, the fraction of sampled base pages that belong to a
    transparent huge page: the page frame from /proc/self/pagemap and its THP
    flag (bit 22) from /proc/kpageflags.  Both need root; None otherwise."""
    base = arr.__array_interface__["data"][0]
    page = os.sysconf("SC_PAGE_SIZE")
    try:
        pm = open("/proc/self/pagemap", "rb")
        kf = open("/proc/kpageflags", "rb")
    except OSError:
        return None
    out = []
    with pm, kf:
        for b0 in range(0, arr.nbytes, block_bytes):
            span = min(block_bytes, arr.nbytes - b0)
            hits = seen = 0
            for j in range(samples):
                va = base + b0 + span * j // samples
                va -= va % page
                pm.seek(va // page * 8)
                e = int.from_bytes(pm.read(8), "little")
                pfn = e & ((1 << 55) - 1)
                if not (e >> 63) & 1 or pfn == 0:
                    continue
                kf.seek(pfn * 8)
                f = int.from_bytes(kf.read(8), "little")
                seen += 1
                hits += (f >> 22) & 1
            out.append(round(hits / seen, 2) if seen else None)
    return out


def measure_h2d_peak(A: np.ndarray):
    """Pinned host -> HBM copy rates (cudaMemcpyAsync via torch, one copy stream):
    burst = best of 3 copies of the first 4 GiB block; sustained = every row
    block of A copied back to back into a 2-buffer ring (what a streamed pass
    over the whole matrix can reach), the faster of two timed passes after
    an untimed one (the benchmark's warm-up steps also run before its timed
    ones; a single stalled block can halve one pass)."""
    import torch
    rows = min(A.shape[0], BLOCK_ROWS)
    dst = [torch.empty((rows, A.shape[1]), dtype=torch.float32, device="cuda") for _ in range(2)]
    best = 0.0
    src = torch.from_numpy(A[:rows])
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        dst[0].copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, rows * A.shape[1] * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    for i, r0 in enumerate(range(0, A.shape[0], rows)):  # untimed first pass
        blk = torch.from_numpy(A[r0:r0 + rows])
        dst[i & 1][:blk.shape[0]].copy_(blk, non_blocking=True)
    sustained, per = 0.0, []
    for _ in range(2):  # two timed passes; the faster one (a stalled block can halve a pass)
        evs = []
        torch.cuda.synchronize()
        total = 0
        for i, r0 in enumerate(range(0, A.shape[0], rows)):
            blk = torch.from_numpy(A[r0:r0 + rows])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst[i & 1][:blk.shape[0]].copy_(blk, non_blocking=True)
            b.record()
            evs.append((a, b, blk.numel() * 4))
            total += blk.numel() * 4
        torch.cuda.synchronize()
        rate = total / (evs[0][0].elapsed_time(evs[-1][1]) / 1e3) / 1e9
        if rate > sustained:
            sustained = rate
            per = sorted(nb / (x.elapsed_time(y) / 1e3) / 1e9 for x, y, nb in evs)
    measure_h2d_peak.per_block = {"min": round(per[0], 1), "median": round(per[len(per) // 2], 1),
                                  "max": round(per[-1], 1)}
    del dst
    return best, sustained


# ----------------------------------------------------------------------------- multi-rank
def whole_job_rate(sec_local: float, units_local: float, dist=None, device="cpu"):
    """Whole-job throughput over ranks: (units summed over ranks) / (time of the
    slowest rank).  Ranks run independent replicas of the workload, so no data
    moves between them; only these two scalars are reduced."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units_local / sec_local, sec_local
    t = torch.tensor([sec_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


# ----------------------------------------------------------------------------- runs
_PINNED = {}  # address of a page-locked array's first byte -> the allocator's pointer


def pinned_array(shape, dtype):
    """Page-locked host array from the library's allocator (freed at exit, or
    by free_pinned)."""
    from paper_2208_08410_gb300 import _binding as B
    nbytes = int(np.prod(shape)) * np.dtype(dtype).itemsize
    ptr = C.c_void_p()
    B.check(B.tsvd_host_alloc(C.byref(ptr), max(nbytes, 16)), "tsvd_host_alloc")
    ctype = {np.float32: C.c_float, np.float64: C.c_double, np.uint8: C.c_uint8}[dtype]
    arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=shape)
    _PINNED[ptr.value] = ptr
    return arr


def pinned_views(shapes_dtypes, align: int = 4096):
    """Many page-locked host arrays carved from ONE allocation of the library's
    allocator, so that small arrays share its huge pages (a separate
    allocation below the huge-page size stays on base pages).  Returns
    (arena, views); free the arena with free_pinned(arena)."""
    offs, total = [], 0
    for shape, dtype in shapes_dtypes:
        offs.append(total)
        total += (int(np.prod(shape)) * np.dtype(dtype).itemsize + align - 1) // align * align
    arena = pinned_array((max(total, 16),), np.uint8)
    views = [arena[o:o + int(np.prod(sh)) * np.dtype(dt).itemsize].view(dt).reshape(sh)
             for o, (sh, dt) in zip(offs, shapes_dtypes)]
    return arena, views


def free_pinned(arr):
    """Return a pinned_array's memory (views of it must not be used after)."""
    from paper_2208_08410_gb300 import _binding as B
    ptr = _PINNED.pop(arr.__array_interface__["data"][0], None)
    if ptr is not None:
        B.tsvd_host_free(ptr)


def time_steps(plan, A_in, steps: int, warmup: int, want_u=True, outs=None):
    import torch
    reps = []
    outs = outs or {}
    for _ in range(warmup):
        plan.factor(A_in, want_u=want_u, **outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    e0.record()
    last = None
    for _ in range(steps):
        last = plan.factor(A_in, want_u=want_u, **outs)
        reps.append(last.report)
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    return e0.elapsed_time(e1) / 1e3, wall, reps, last


def dense_config(m: int, prec: int, world: int) -> dict:
    """The dense workload's config, the same on the GPU line and the reference
    (oracle) line."""
    return {"workload": f"dense t-SVD (rank-64 + 1e-4 noise), m={m}, n={N_COLS}, k={K}, eps={EPS}; "
                        "value: A resident in HBM (in-core); e2e: A streamed from page-locked host "
                        f"memory under a {BUDGET / 1e9:.0f} GB device budget (out-of-core)",
            "m": m, "n": N_COLS, "k": K, "eps": EPS,
            "block_rows": BLOCK_ROWS, "device_budget_bytes_e2e": BUDGET,
            "full_m": FULL_M, "host_ram_limited": m < FULL_M,
            "l2": "inputs larger than L2 (A is %.0f GiB)" % (m * N_COLS * 4 / 2 ** 30),
            "gram_precision": PREC_NAMES[prec] + (" (FP32-class split: hi*hi + hi*lo + lo*hi on the "
                                                  "tensor cores, FP32 accumulate)" if prec == 2 else ""),
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def reference_arm(args, m: int):
    """The FP64 oracle timed on the host cores over one row block per step."""
    import synth
    from oracle import tsvd_ref as ref
    rows = args.ref_rows
    sigma = 1.0 / (1.0 + np.arange(RANK))
    V = synth.orthonormal_columns(N_COLS, RANK, 0, 1)
    Ab = synth.dense_lowrank_rows(0, rows, V, sigma, m, NOISE, seed=0)
    Vk = V[:, :K]
    sig = sigma[:K]
    for _ in range(args.warmup):
        ref.gram(Ab)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ref.gram(Ab)  # Gram accumulation of the block (FP64)
        _ = (Ab.astype(np.float64) @ Vk) / sig  # left vectors of the block
        t.append(time.perf_counter() - t0)
    sec = sum(t) / len(t)
    value = 2 * rows * N_COLS * 4 / sec / 1e9
    cores = len(os.sched_getaffinity(0))
    return {"impl": "reference", "metric": "t-SVD A-stream throughput", "value": round(value, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dense_config(m, args.precision, 1),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"one {rows}-row block per step: FP64 Gram + left vectors; power phase "
                                       f"excluded (O(n^2) per iteration, independent of m)"},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_baseline(m: int, A: np.ndarray, V_gpu: np.ndarray, sig_gpu: np.ndarray, iters, budget_s: float = 25.0):
    """FP64 oracle on this host: Gram + left vectors timed on one row block, the
    power phase timed on that block's Gram with the GPU's per-triplet counts;
    extrapolated to the whole matrix."""
    from oracle import tsvd_ref as ref
    rows = min(m, 65_536)
    Ab = A[:rows]
    t0 = time.perf_counter()
    G = ref.gram(Ab)
    t_gram = time.perf_counter() - t0
    t0 = time.perf_counter()
    _ = (Ab.astype(np.float64) @ V_gpu.astype(np.float64)) / sig_gpu
    t_left = time.perf_counter() - t0
    # power phase with the same application counts (bounded by the time budget)
    t0 = time.perf_counter()
    done = 0
    sig2 = []
    Vd = np.zeros((N_COLS, 0))
    for l, it in enumerate(iters):
        if time.perf_counter() - t0 > budget_s:
            break
        x = np.random.default_rng(l).standard_normal(N_COLS)
        res = ref.power_method(ref.hotelling_apply(G, Vd, np.array(sig2)), x / np.linalg.norm(x), EPS,
                               iters_override=int(it))
        sig2.append(float(res.v @ G @ res.v))
        Vd = np.concatenate([Vd, res.v[:, None]], axis=1)
        done += int(it)
    t_pow = (time.perf_counter() - t0) * (sum(iters) / max(done, 1))
    blocks = m / rows
    total = blocks * (t_gram + t_left) + t_pow
    cores = len(os.sched_getaffinity(0))
    return {"value": round(2 * m * N_COLS * 4 / total / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle: Gram + left vectors of one {rows}-row block ({t_gram + t_left:.1f} s) scaled "
                      f"to {m} rows, plus the power phase on that block's Gram with the GPU's {sum(iters)} "
                      f"applications ({t_pow:.1f} s); est. t-SVD {total:.0f} s"}


def parity_full_oracle(A: np.ndarray, res, seed: int = 0):
    """The oracle's trajectory at the headline size: FP64 Gram of the stored
    values of all of A (row blocks of 65,536), O-1 from the start draws of the
    GPU run (the built-in Philox stream of `seed`, which the oracle's generator
    reproduces bit for bit) with the GPU's iteration counts, and U = A V
    Sigma^-1; sigma on every triplet, u_l and v_l angles on the gapped ones."""
    from oracle import tsvd_ref as ref
    m = A.shape[0]
    t0 = time.time()
    G = ref.gram_row_blocks(A, 65_536)
    t_gram = time.time() - t0
    it = [int(i) for i in res.iters]
    sig_o, V_o, it_o, st_o = ref.right_vectors(G, K, EPS, seed=seed, iters_override=it)
    lam = np.linalg.eigvalsh(G)[::-1]
    del G
    gapped = ref.gapped_indices(lam, K)
    V = res.V.cpu().numpy().astype(np.float64)
    sig = np.asarray(res.sigma.cpu(), dtype=np.float64)
    Ug = res.U  # (m, k) on the device
    ang_u = {}
    U_o_cols = np.zeros((m, len(gapped)))
    for r0 in range(0, m, 65_536):
        U_o_cols[r0:r0 + 65_536] = (np.asarray(A[r0:r0 + 65_536], dtype=np.float64) @ V_o[:, gapped]) / sig_o[gapped]
    for j, l in enumerate(gapped):
        ang_u[int(l)] = float("%.3g" % ref.vector_angle(Ug[:, l].cpu().numpy().astype(np.float64), U_o_cols[:, j]))
    ang_v = {int(l): float("%.3g" % ref.vector_angle(V[:, l], V_o[:, l])) for l in gapped}
    err = float(np.max(np.abs(sig - sig_o) / sig_o))
    return {"oracle": "O-1 on the FP64 Gram of all of A, start draws of the GPU run (Philox seed), GPU counts forced",
            "sigma_rel_err_vs_oracle": float("%.3g" % err), "gapped": [int(l) for l in gapped],
            "v_angle_max_gapped": max(ang_v.values()) if ang_v else None,
            "u_angle_max_gapped": max(ang_u.values()) if ang_u else None, "v_angles": ang_v, "u_angles": ang_u,
            "pass": bool(err <= 1e-5 and gapped and all(a <= 1e-4 for a in list(ang_v.values()) + list(ang_u.values()))),
            "oracle_gram_seconds": round(t_gram, 1), "oracle_seconds": round(time.time() - t0, 1),
            "oracle_cores": len(os.sched_getaffinity(0))}


def parity_full_size(A: np.ndarray, dA, res, prec: int):
    """Checks at full size on outputs the oracle computes one by one."""
    import torch
    from paper_2208_08410_gb300 import _binding as B
    m, n = A.shape
    out = {}
    stream = torch.cuda.current_stream().cuda_stream
    # sampled Gram entries: 48 random columns over all rows (FP64 oracle) vs the
    # library's Gram accumulated block by block with the same entry point
    rng = np.random.default_rng(7)
    cols = np.sort(rng.choice(n, size=48, replace=False))
    G = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    scr_b = B.tsvd_gram_scratch_bytes(BLOCK_ROWS, n, prec)
    scr = torch.empty(max(scr_b, 256), dtype=torch.uint8, device="cuda")
    for r0 in range(0, m, BLOCK_ROWS):
        rows = min(BLOCK_ROWS, m - r0)
        B.check(B.tsvd_gram_accumulate(dA[r0:].data_ptr(), rows, n, n, G.data_ptr(), prec, scr.data_ptr(), scr_b,
                                       stream), "gram")
    torch.cuda.synchronize()
    Gs = G[cols][:, cols].cpu().numpy()
    del G, scr
    Gref = np.zeros((48, 48))
    absref = np.zeros((48, 48))
    step = 1 << 18
    for r0 in range(0, m, step):
        blk = A[r0:r0 + step][:, cols].astype(np.float64)
        Gref += blk.T @ blk
        ab = np.abs(blk)
        absref += ab.T @ ab
    iu = np.triu_indices(48)
    # the library stores the upper triangle (row j <= column i) of G
    Gsu = np.where(np.arange(48)[:, None] <= np.arange(48)[None, :], Gs, Gs.T)
    relerr = np.abs(Gsu[iu] - Gref[iu]) / absref[iu]
    out["gram_sampled_max_err_over_absgram"] = float(relerr.max())
    # sigma_l = ||A v_l|| (Alg. 1) for the GPU's v_l, FP64 over all rows
    V = res.V.cpu().numpy().astype(np.float64) if hasattr(res.V, "cpu") else np.asarray(res.V, dtype=np.float64)
    sig_g = res.sigma.cpu().numpy() if hasattr(res.sigma, "cpu") else np.asarray(res.sigma)
    AV2 = np.zeros(V.shape[1])
    step = 1 << 16
    for r0 in range(0, m, step):
        AV2 += np.sum((A[r0:r0 + step].astype(np.float64) @ V) ** 2, axis=0)
    sig_o = np.sqrt(AV2)
    out["sigma_rel_err_vs_oracle_norm"] = float(np.max(np.abs(sig_g - sig_o) / sig_o))
    out["VtV_offdiag_max"] = float(np.max(np.abs(V.T @ V - np.eye(V.shape[1]))))
    return out


def kernel_case(args):
    """Single-kernel microbenchmarks on device-resident inputs larger than L2
    (used for the per-kernel roofline table and as the small ncu case)."""
    import torch
    from paper_2208_08410_gb300 import _binding as B
    B.load(build_if_missing=True)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    out = {"case": args.case}
    reps = args.steps

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    peaks, src = load_peaks()
    if args.case == "tf32ref":
        # the library GEMM the tensor-core Gram is compared with: cuBLAS TF32, 8192^3
        res = measure_tf32_peak(burst_reps=3, sustained_s=0.2)
        out.update({"n": 8192, "cublas_tf32": res})
    elif args.case == "gram":
        m = args.m or BLOCK_ROWS
        n = args.n
        A = torch.randn((m, n), generator=gen, device="cuda", dtype=torch.float32)
        G = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        sb = B.tsvd_gram_scratch_bytes(m, n, args.precision)
        scr = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda")

        def fn():
            B.check(B.tsvd_gram_accumulate(A.data_ptr(), m, n, n, G.data_ptr(), args.precision, scr.data_ptr(), sb,
                                           stream), "gram")
        t = timed(fn)
        fl = m * n * (n + 1)
        out.update({"m": m, "n": n, "precision": PREC_NAMES[args.precision], "ms": round(t * 1e3, 3),
                    "tflops_algorithmic": round(fl / t / 1e12, 2),
                    "frac_of_dtype_peak_burst": round(fl / t / 1e12 / dtype_peak(
                        args.precision, peaks, False, getattr(measure_tf32_peak, "result", None))[0], 4),
                    "note": "time covers prep (transpose/round) + SYRK for tensor precisions"})
    elif args.case == "power":
        n = args.n
        X = torch.randn((n, n), generator=gen, device="cuda", dtype=torch.float64)
        G64 = (X @ X.T).contiguous()
        G32 = G64.float()
        x = torch.randn(n, generator=gen, device="cuda", dtype=torch.float64)
        sb = B.tsvd_power_scratch_bytes(n, 0)
        scr = torch.empty(sb, dtype=torch.uint8, device="cuda")
        info = torch.zeros(4, dtype=torch.int32, device="cuda")
        s2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        iters = 200

        def fn():
            B.check(B.tsvd_power_dense(n, G32.data_ptr(), G64.data_ptr(), None, None, 0, x.data_ptr(), 1e-8, 10000,
                                       iters, 0, s2.data_ptr(), info.data_ptr(), scr.data_ptr(), sb, stream), "power")
        t = timed(fn)
        per_it = t / iters
        out.update({"n": n, "iters_per_launch": iters, "us_per_iteration": round(per_it * 1e6, 2),
                    "GBps_G32": round(4 * n * n / per_it / 1e9, 1)})
    elif args.case == "csr":
        import synth
        m = args.m or (1 << 22)
        csr = synth.csr_uniform(m, m, 33.5, seed=1)
        rp = torch.from_numpy(csr["row_ptr"]).cuda()
        ci = torch.from_numpy(csr["col_idx"]).cuda()
        va = torch.from_numpy(csr["values"]).cuda()
        v = torch.rand(m, generator=gen, device="cuda", dtype=torch.float32)
        w = torch.zeros(m, dtype=torch.float32, device="cuda")
        ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        nnz = int(va.shape[0])

        def fn():
            B.check(B.tsvd_csr_gram_apply(m, m, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), v.data_ptr(),
                                          w.data_ptr(), ss.data_ptr(), 1, stream), "csr")
        t = timed(fn)
        alg = 8 * nnz + 8 * (m + 1) + 4 * m + 8 * m
        out.update({"m": m, "nnz": nnz, "ms": round(t * 1e3, 3), "GBps_algorithmic": round(alg / t / 1e9, 1),
                    "frac_hbm": round(alg / t / 1e9 / peaks["hbm_gbs"], 3)})
    elif args.case == "left":
        m = args.m or BLOCK_ROWS
        n, k = args.n, K
        A = torch.randn((m, n), generator=gen, device="cuda", dtype=torch.float32)
        V = torch.randn((k, n), generator=gen, device="cuda", dtype=torch.float32)
        sig = torch.ones(k, dtype=torch.float64, device="cuda")
        U = torch.empty((k, m), dtype=torch.float32, device="cuda")

        def fn():
            B.check(B.tsvd_left_vectors(A.data_ptr(), m, n, n, V.data_ptr(), n, k, sig.data_ptr(), U.data_ptr(), m,
                                        stream), "left")
        t = timed(fn)
        out.update({"m": m, "n": n, "k": k, "ms": round(t * 1e3, 3), "GBps_A": round(m * n * 4 / t / 1e9, 1),
                    "frac_hbm": round(m * n * 4 / t / 1e9 / peaks["hbm_gbs"], 3)})
    elif args.case == "c1":
        out.update(c1_latency(reps=max(reps, 5)))
    elif args.case == "csr_small":
        # one sparse serving request alone: m = n = 65,536 at density 1e-4, k = 16, eps = 1e-6,
        # at most 200 applications per triplet, the CSR on the device (the cooperative loop)
        import synth
        from paper_2208_08410_gb300 import Plan
        m = args.m or (1 << 16)
        csr = synth.csr_uniform(m, m, 1e-4 * m, seed=3)
        dcsr = {"row_ptr": torch.from_numpy(csr["row_ptr"]).cuda(), "col_idx": torch.from_numpy(csr["col_idx"]).cuda(),
                "values": torch.from_numpy(csr["values"]).cuda(), "m": m, "n": m}
        plan = Plan(dcsr, 16, 1e-6, out_device=True, max_iter=200)
        for _ in range(max(args.warmup, 1)):
            plan.factor(dcsr, ok=(B.TSVD_OK, B.TSVD_ENOCONV))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = plan.factor(dcsr, ok=(B.TSVD_OK, B.TSVD_ENOCONV))
        e1.record()
        torch.cuda.synchronize()
        plan.close()
        ms = e0.elapsed_time(e1)
        out.update({"m": m, "nnz": int(csr["values"].shape[0]), "ms_per_tsvd": round(ms, 2),
                    "applications": r.report["applications"],
                    "us_per_application": round(ms * 1e3 / max(r.report["applications"], 1), 2),
                    "phases_ms": {"power": round(r.report["power_ms"], 2)}, "launches": r.report["kernel_launches"]})
    elif args.case == "csr_tsvd":
        # in-core CSR t-SVD alone (device CSR, k = 4, 3 applications per triplet): the
        # column-chunked operator when 8 n exceeds 64 MB
        import synth
        from paper_2208_08410_gb300 import Plan
        m = args.m or (1 << 24)
        dcsr = synth.csr_uniform_torch(m, m, 33.5, seed=1)
        nnz = int(dcsr["values"].shape[0])
        plan = Plan(dcsr, 4, EPS, out_device=True, iters_override=[3] * 4, time_kernels=True)
        for _ in range(max(args.warmup, 1)):
            r = plan.factor(dcsr)
        torch.cuda.synchronize()
        r = plan.factor(dcsr)
        rep = r.report
        plan.close()
        t_app = rep["gram_kernel_ms"] / max(rep["gram_kernel_launches"], 1) / 1e3
        alg = 8 * nnz + 8 * (m + 1) + 4 * m + 8 * m
        out.update({"m": m, "nnz": nnz, "csr_chunks": rep["csr_chunks"], "ms_per_application": round(t_app * 1e3, 3),
                    "GBps_algorithmic": round(alg / t_app / 1e9, 1),
                    "frac_hbm": round(alg / t_app / 1e9 / peaks["hbm_gbs"], 4),
                    "applications_timed": rep["gram_kernel_launches"]})
    print(json.dumps(out), flush=True)


def alt_precision_in_core(dA, args, m, res_ref, peaks, prec):
    """The same in-core step with the Gram in another tensor-core precision
    (plain TF32: one MMA per product; BF16x3: three BF16 MMAs per product),
    reported beside the FP32-class 3xTF32 headline, never as it: throughput,
    SYRK fraction of that dtype's peak, the power phase's applications and the
    largest relative change of sigma against the 3xTF32 run (whose own error
    against the FP64 oracle the headline's parity fields give)."""
    from paper_2208_08410_gb300 import Plan
    plan = Plan(dA, K, EPS, precision=prec, out_device=True, time_kernels=True)
    sec, wall, reps, res = time_steps(plan, dA, args.steps, args.warmup)
    plan.close()
    gk_ms = sum(r["gram_kernel_ms"] for r in reps)
    tf = m * N_COLS * (N_COLS + 1) * args.steps / (gk_ms / 1e3) / 1e12
    peak, _, _ = dtype_peak(prec, peaks, sustained=True, tf32_measured=getattr(measure_tf32_peak, "result", None))
    s1 = np.asarray(res.sigma.cpu(), dtype=np.float64)
    s0 = np.asarray(res_ref.sigma.cpu(), dtype=np.float64)
    return {"value": round(2 * m * N_COLS * 4 * args.steps / sec / 1e9, 3), "unit": "GB/s",
            "ms_per_step": round(sec / args.steps * 1e3, 2), "syrk_tflops": round(tf, 1),
            f"syrk_frac_of_{PREC_NAMES[prec]}_peak": round(tf / peak, 4),
            "applications": int(reps[-1]["applications"]) if "applications" in reps[-1] else None,
            "sigma_max_rel_diff_vs_tf32x3": float("%.3g" % np.max(np.abs(s1 - s0) / s0))}




def c1_latency(reps: int = 50):
    """In-core tiny case (m = 2048, n = 256, sigma_i = 0.8^i plus 1e-6 noise,
    k = 8, eps = 1e-8, plain FP32 Gram): latency-bound (G is 256 KB), so the
    figures are the device time of one whole t-SVD call (CUDA events on the
    launching stream, median of `reps`), the time per power application and
    the kernel launches per call, for the default power kernel (one
    thread-block cluster for all triplets) and for the grid-wide cooperative
    kernel beside it."""
    import torch

    import synth
    from paper_2208_08410_gb300 import Plan, _binding as B
    inp = synth.dense_prescribed(2048, 256, synth.spectrum_geometric(256, 0.8), 1e-6, seed=0)
    dA = torch.from_numpy(inp["A"]).cuda()

    def run(pk, ctas=0):
        plan = Plan(dA, 8, 1e-8, precision=0, out_device=True, time_kernels=True, power_kernel=pk,
                    power_ctas=ctas)
        for _ in range(5):
            plan.factor(dA)
        torch.cuda.synchronize()
        times, reps_out = [], []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = plan.factor(dA)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            reps_out.append(r.report)
        plan.close()
        rep = reps_out[-1]
        return {"ms_per_tsvd": round(float(np.median(times)), 4), "ms_min": round(float(np.min(times)), 4),
                "us_per_power_application": round(rep["power_ms"] * 1e3 / max(rep["applications"], 1), 3),
                "applications": rep["applications"], "kernel_launches_per_tsvd": rep["kernel_launches"],
                "phases_ms": {"gram": round(rep["gram_ms"], 4), "power": round(rep["power_ms"], 4),
                              "left": round(rep["left_ms"], 4)},
                "power_cluster_ctas": rep.get("power_cluster", 0)}

    out = {"workload": "m=2048, n=256, sigma_i=0.8^i + 1e-6 noise, k=8, eps=1e-8, FP32 Gram, A in HBM",
           "power_kernel": "cluster (all triplets in one launch on one thread-block cluster)"}
    out.update(run(B.TSVD_POWER_AUTO))
    out["power_cluster"] = out.pop("power_cluster_ctas")
    out["cluster_sizes"] = {}
    for c in (1, 2, 4, 8):
        t = run(B.TSVD_POWER_CLUSTER, c)
        out["cluster_sizes"][str(t.pop("power_cluster_ctas"))] = {
            "ms_per_tsvd": t["ms_per_tsvd"], "us_per_power_application": t["us_per_power_application"]}
    out["grid_kernel"] = run(B.TSVD_POWER_GRID)
    out["grid_kernel"].pop("power_cluster_ctas")
    return out


def measure_tf32_peak(n: int = 8192, burst_reps: int = 10, sustained_s: float = 3.0):
    """cuBLAS TF32 GEMM rate on this GPU (torch.matmul of two n x n FP32
    matrices with TF32 allowed, 2 n^3 flop): best of `burst_reps` launches
    (burst) and back-to-back launches for `sustained_s` seconds (sustained).
    Kept on the function as `result` for the legs that report against it."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        g = torch.Generator(device="cuda").manual_seed(3)
        a = torch.randn((n, n), generator=g, device="cuda")
        b = torch.randn((n, n), generator=g, device="cuda")
        c = torch.empty((n, n), device="cuda")
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(burst_reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = max(best, 2 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12)
        reps = max(1, int(sustained_s * best * 1e12 / (2 * n ** 3)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        sus = 2 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        del a, b, c
        torch.cuda.empty_cache()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    measure_tf32_peak.result = {"burst_tflops": round(best, 1), "sustained_tflops": round(sus, 1),
                                "how": f"torch.matmul FP32 {n}^3 with TF32 allowed (cuBLAS), best of {burst_reps} "
                                       f"and {reps} back to back"}
    return measure_tf32_peak.result


def dtype_peak(prec: int, peaks: dict, sustained: bool = True, tf32_measured=None):
    """Roofline denominator of the Gram arithmetic in TFLOP/s (algorithmic
    flops: a split mode's three MMAs per product count once), its bound and a
    note on where it comes from.  Kernels timed inside a long step take the
    sustained figures, kernels timed alone the burst ones.  TF32-based modes
    take the larger of the bf16 measurement x the nominal 1.1/2.25 ratio and
    this GPU's measured cuBLAS TF32 rate, so a kernel is never graded against
    the smaller of two estimates of the same peak."""
    kind = "sustained" if sustained else "burst"
    bf = peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"]
    if prec == 0:
        return 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, "alu", \
            "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"
    if prec in (1, 2):
        derived = bf * (1.1 / 2.25)
        meas = (tf32_measured or {}).get(f"{kind}_tflops")
        tf32 = max(derived, meas or 0.0)
        src = (f"TF32 = max(bf16 measured {kind} {bf:.0f} x 1.1/2.25 = {derived:.0f}, cuBLAS TF32 measured "
               f"{kind} {meas:.0f})" if meas else f"TF32 = bf16 measured {kind} {bf:.0f} x 1.1/2.25 = {derived:.0f}")
        if prec == 1:
            return tf32, "tensor", src
        return tf32 / 3, "tensor", "3xTF32 = TF32 / 3 (three TF32 MMAs per product); " + src
    return bf / 3, "tensor", f"BF16x3 = bf16 measured {kind} {bf:.0f} / 3 (three BF16 MMAs per product)"


C2S_M = 1_048_576            # the dense out-of-core configuration's small case (16 GiB)
C2S_BUDGET = 8 * 10 ** 9      # its device budget


def leg_c2_small(args, h2d_peak=None):
    """The dense out-of-core configuration's small case: m = 1,048,576, n = 4096
    (16 GiB in page-locked host memory), streamed under an 8 GB device budget,
    3xTF32 Gram, k = 16, eps = 1e-6.
    - e2e: A-stream throughput of whole t-SVDs (own convergence test), host A
      and host outputs, every copy inside the timed region; the Gram pass
      against the pinned copy rate of the same blocks.
    - parity: the oracle forms the FP64 Gram of the same stored values (row
      blocks of 65,536), runs O-1 from the same start draws with its own
      convergence test and forms U = A V Sigma^-1; the GPU reruns with the
      oracle's counts forced.  sigma error on all triplets, angles of u_l and
      v_l on the gapped ones (relative eigen-gap >= 0.05)."""
    import torch

    import synth
    from oracle import tsvd_ref as ref
    from paper_2208_08410_gb300 import Plan, _binding as B
    m = C2S_M
    A, ptr, _ = make_host_A(m, seed=5)
    try:
        burst, sustained = measure_h2d_peak(A)
        per_block = getattr(measure_h2d_peak, "per_block", None)
        thp = thp_coverage(A)
        x = synth.start_normals(N_COLS, K, seed=3)
        outs = {"U": pinned_array((K, m), np.float32), "sigma": pinned_array((K,), np.float64),
                "V": pinned_array((K, N_COLS), np.float32)}
        steps = max(1, min(args.steps, 5))
        plan = Plan(A, K, EPS, precision=2, device_budget=C2S_BUDGET, force_stream=True, time_kernels=True,
                    start_draws=x)
        clocks = ClockSampler(0)
        clocks.start()
        sec, wall, reps, res = time_steps(plan, A, steps, max(1, min(args.warmup, 3)), outs=outs)
        clk = clocks.stop()
        plan.close()
        r = reps[-1]
        own_iters = list(res.iters)
        gram_s = r["gram_ms"] / 1e3
        e2e = {"value": round(2 * m * N_COLS * 4 * steps / sec / 1e9, 2), "unit": "GB/s",
               "ms_per_step": round(sec / steps * 1e3, 2), "steps": steps,
               "h2d_bytes_per_step": int(r["h2d_bytes"]), "d2h_bytes_per_step": int(r["d2h_bytes"]),
               "phases_ms": {"gram": round(r["gram_ms"], 2), "power": round(r["power_ms"], 2),
                             "left": round(r["left_ms"], 2)},
               "gram_pass_GBps": round(m * N_COLS * 4 / gram_s / 1e9, 2),
               "pinned_copy_peak_GBps": round(sustained, 2), "pinned_copy_burst_GBps": round(burst, 2),
               "pinned_copy_per_block_GBps": per_block,
               "frac_gram_pass": round(m * N_COLS * 4 / gram_s / 1e9 / sustained, 4),
               "frac_gram_pass_of_burst": round(m * N_COLS * 4 / gram_s / 1e9 / burst, 4),
               "blocks_per_pass": r["n_blocks"], "ring_slots": r["ring_slots"],
               "copy_stream_GBps": round(r["h2d_bytes"] / (r["h2d_copy_ms"] / 1e3) / 1e9, 2)
               if r["h2d_copy_ms"] else None,
               "copy_min_GBps": round(r["h2d_copy_min_gbps"], 1), "copy_max_GBps": round(r["h2d_copy_max_gbps"], 1),
               "host_A_pages": thp, "clocks": clk}
        # ---- parity against the oracle's trajectory
        t0 = time.time()
        G = ref.gram_row_blocks(A, 65_536)
        t_gram = time.time() - t0
        sig_o, V_o, it_o, st_o = ref.right_vectors(G, K, EPS, x_start=x)
        lam = np.linalg.eigvalsh(G)[::-1]
        del G
        gapped = ref.gapped_indices(lam, K)
        U_o = np.empty((m, K))
        for r0 in range(0, m, 65_536):
            U_o[r0:r0 + 65_536] = np.asarray(A[r0:r0 + 65_536], dtype=np.float64) @ V_o
        U_o /= sig_o[None, :]
        t_oracle = time.time() - t0
        plan = Plan(A, K, EPS, precision=2, device_budget=C2S_BUDGET, force_stream=True, start_draws=x,
                    iters_override=it_o)
        res2 = plan.factor(A, **outs)
        plan.close()
        sig = np.asarray(res2.sigma, dtype=np.float64)
        V = np.asarray(res2.V, dtype=np.float64)
        U = np.asarray(res2.U, dtype=np.float64)
        sig_err = float(np.max(np.abs(sig - sig_o) / sig_o))
        ang_v = {int(l): float("%.3g" % ref.vector_angle(V[:, l], V_o[:, l])) for l in gapped}
        ang_u = {int(l): float("%.3g" % ref.vector_angle(U[:, l], U_o[:, l])) for l in gapped}
        parity = {"oracle": "O-1: FP64 Gram of the stored values, Hotelling deflation, same start draws, "
                            "own convergence test; GPU with the oracle's counts forced",
                  "sigma_rel_err_vs_oracle": float("%.3g" % sig_err),
                  "gapped": [int(l) for l in gapped],
                  "v_angle_max_gapped": max(ang_v.values()) if ang_v else None,
                  "u_angle_max_gapped": max(ang_u.values()) if ang_u else None,
                  "v_angles": ang_v, "u_angles": ang_u,
                  "pass": bool(sig_err <= 1e-5 and all(a <= 1e-4 for a in list(ang_v.values()) + list(ang_u.values()))
                               and len(gapped) > 0),
                  "oracle_iters": [int(i) for i in it_o], "gpu_own_iters": own_iters,
                  "oracle_status": sorted(set(st_o)), "oracle_seconds": round(t_oracle, 1),
                  "oracle_gram_seconds": round(t_gram, 1), "oracle_cores": len(os.sched_getaffinity(0))}
        return {"workload": f"dense out-of-core t-SVD (rank-64 + 1e-4 noise), m={m}, n={N_COLS}, k={K}, "
                            f"eps={EPS}, 3xTF32 Gram, host A streamed under an {C2S_BUDGET / 1e9:.0f} GB "
                            "device budget", "m": m, "e2e": e2e, "parity": parity}
    finally:
        B.tsvd_host_free(ptr)
        torch.cuda.empty_cache()


def leg_c4(args, steps: int, warmup: int):
    """Mixed-precision Gram on a clustered spectrum: m = 2^20, n = 8192,
    sigma_i = 1/(1+i) with sigma_11 = sigma_10 - 1e-3, k = 32, eps = 1e-8, A
    resident in HBM (32 GiB), stacked-orthogonal construction (A^T A = 128
    M^T M exactly, so the oracle's FP64 Gram is exact and O-1 runs at full
    size).  The oracle runs from fixed start draws with its own convergence
    test; every Gram precision follows its trajectory (counts forced) and is
    timed.  Reported per precision: seconds per t-SVD, the Gram kernel
    against its dtype's peak, the sigma error against O-1 and against the
    closed form, the gapped vectors' angles to O-1 and the clustered pair's
    largest principal angle."""
    import torch

    import synth
    from oracle import tsvd_ref as ref
    from paper_2208_08410_gb300 import Plan, _binding as B
    n, copies, k, eps = 8192, 128, 32, 1e-8
    m = n * copies
    pair = (10, 11)
    t0 = time.time()
    sig_t = synth.spectrum_harmonic_clustered(n, 10, 1e-3)
    fac = synth.stacked_factor(n, sig_t, copies, seed=0)
    dA = torch.empty((m, n), dtype=torch.float32, device="cuda")
    synth.stacked_rows_torch(dA, fac["M32"], seed=0)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    x = synth.start_normals(n, k, seed=4)
    t0 = time.time()
    G = copies * ref.gram(fac["M32"])
    sig_o, V_o, it_o, st_o = ref.right_vectors(G, k, eps, x_start=x)
    del G
    t_oracle = time.time() - t0
    gapped = [i for i in ref.gapped_indices(sig_t ** 2, k) if i not in pair]
    peaks, peak_src = load_peaks()
    tf32_meas = getattr(measure_tf32_peak, "result", None)
    flops = m * n * (n + 1)
    rows = {}
    clocks = ClockSampler(0)
    clocks.start()
    for prec in (0, 1, 2, 3):
        plan = Plan(dA, k, eps, precision=prec, out_device=True, time_kernels=True, start_draws=x,
                    iters_override=it_o)
        sec, wall, reps, res = time_steps(plan, dA, steps, warmup, want_u=True)
        plan.close()
        sig = np.asarray(res.sigma.cpu(), dtype=np.float64)
        V = res.V.cpu().numpy().astype(np.float64)
        err_o = float(np.max(np.abs(sig - sig_o) / sig_o))
        err_t = float(np.max(np.abs(sig - sig_t[:k]) / sig_t[:k]))
        ang = max(ref.vector_angle(V[:, l], V_o[:, l]) for l in gapped)
        ang_pair = ref.subspace_angle(V[:, list(pair)], V_o[:, list(pair)])
        gk = sum(r["gram_kernel_ms"] for r in reps) / 1e3
        tf = flops * steps / gk / 1e12 if gk > 0 else None
        pk, bound, note = dtype_peak(prec, peaks, sustained=True, tf32_measured=tf32_meas)
        rows[PREC_NAMES[prec]] = {
            "seconds_per_tsvd": round(sec / steps, 4),
            "sigma_max_rel_err_vs_oracle": float("%.3g" % err_o),
            "sigma_max_rel_err_vs_truth": float("%.3g" % err_t),
            "v_angle_max_gapped_vs_oracle": float("%.3g" % ang),
            "pair_subspace_angle_vs_oracle": float("%.3g" % ang_pair),
            "within_1e-5": bool(err_o <= 1e-5 and ang <= 1e-4 and ang_pair <= 1e-4),
            "gram_tflops": round(tf, 1) if tf else None, "gram_peak_tflops": round(pk, 1), "bound": bound,
            "gram_frac_of_dtype_peak": round(tf / pk, 4) if tf else None, "peak_note": note,
            "phases_ms": {"gram": round(reps[-1]["gram_ms"], 1), "power": round(reps[-1]["power_ms"], 1),
                          "left": round(reps[-1]["left_ms"], 1)},
            "applications": reps[-1]["applications"], "gpu_launches": int(sum(r["kernel_launches"] for r in reps))}
        torch.cuda.empty_cache()
    clk = clocks.stop()
    del dA
    torch.cuda.empty_cache()
    ok = {p: r for p, r in rows.items() if r["within_1e-5"]}
    best = min(ok, key=lambda p: ok[p]["seconds_per_tsvd"]) if ok else None
    fp32 = rows["f32"]["seconds_per_tsvd"]
    return {"workload": f"dense in-core t-SVD, stacked-orthogonal A, m={m}, n={n}, sigma_i=1/(1+i), "
                        f"sigma_11=sigma_10-1e-3, k={k}, eps={eps}; every precision on the oracle's trajectory",
            "m": m, "n": n, "k": k, "eps": eps, "steps": steps, "warmup": warmup,
            "fastest_within_1e-5": best, "seconds_per_tsvd": ok[best]["seconds_per_tsvd"] if best else None,
            "speedup_vs_f32": round(fp32 / ok[best]["seconds_per_tsvd"], 3) if best else None,
            "precisions": rows, "oracle_iters": [int(i) for i in it_o], "oracle_seconds": round(t_oracle, 1),
            "gapped_graded": gapped, "clustered_pair": list(pair), "gen_seconds": round(gen_s, 1),
            "peak_source": peak_src, "clocks": clk}


def c4_workload(args):
    """The mixed-precision leg as its own JSON line (seconds per t-SVD of the
    fastest precision within 1e-5 of the oracle)."""
    import torch

    from paper_2208_08410_gb300 import _binding as B
    B.load(build_if_missing=True)
    torch.cuda.set_device(0)
    measure_tf32_peak()
    leg = leg_c4(args, args.steps, args.warmup)
    line = {"metric": "t-SVD seconds, mixed-precision Gram at sigma err <= 1e-5 vs the FP64 oracle "
                      "(clustered spectrum)",
            "value": leg["seconds_per_tsvd"], "unit": "s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": leg["fastest_within_1e-5"], "data": "synthetic",
            "config": {"workload": leg["workload"], "l2": "inputs larger than L2 (A is 32 GiB)"}, "c4": leg,
            "clocks": leg["clocks"]}
    print(json.dumps(line), flush=True)


def tiled_workload(args):
    """Orthogonal batching (Sec. V-C, Fig. 2c-d, Alg. 3): dense A in HBM, m =
    262,144, n = 16,384, rank 64 with sigma_i = 1/(1+i) and no noise (its
    singular values are the prescribed ones to FP32 storage accuracy), k = 8,
    eps = 1e-8, 3xTF32 Gram in panels of 4096 columns (10 tasks).  Two
    budgets: none (the FP64 tiles stay on the device) and 1 GB (they go to
    page-locked host memory and every power application streams them back,
    1.3 GB per application).  The line reports seconds per t-SVD with host
    tiles, the Gram phase against the 3xTF32 peak and the tile stream against
    the measured pinned-copy peak; sigma is checked against the closed form."""
    import torch

    import synth
    from paper_2208_08410_gb300 import Plan, _binding as B
    B.load(build_if_missing=True)
    torch.cuda.set_device(0)
    m, n, rank, k, eps, bs = 262_144, 16_384, 64, 8, 1e-8, 4096
    t0 = time.time()
    sig_t = 1.0 / (1.0 + np.arange(rank))
    dA = torch.empty((m, n), dtype=torch.float32, device="cuda")
    synth.dense_lowrank_blocks_torch(dA, m, n, rank, sig_t, 0.0, seed=3, block_rows=65_536)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    peaks, peak_src = load_peaks()
    flops = m * n * (n + 1)
    nb = -(-n // bs)
    tile_bytes = sum(min(bs, n - J * bs) * min(bs, n - I * bs) * 8 for I in range(nb) for J in range(I + 1))
    out = {}
    for name, budget in (("tiles_on_device", 0), ("tiles_on_host", 1 << 30)):
        plan = Plan(dA, k, eps, precision=B.TSVD_GRAM_TF32X3, out_device=True, gram_tile=bs, device_budget=budget)
        sec, wall, reps, res = time_steps(plan, dA, args.steps, args.warmup, want_u=True)
        ws = plan.workspace_bytes
        plan.close()
        rep = reps[-1]
        sig = np.asarray(res.sigma.cpu(), dtype=np.float64)
        err = float(np.max(np.abs(sig - sig_t[:k]) / sig_t[:k]))
        apps = rep["applications"] + k  # the sigma pass of every triplet applies G once more
        row = {"seconds_per_tsvd": round(sec / args.steps, 4), "workspace_bytes": ws,
               "tiles_on_host": rep["tiles_on_host"], "gram_panels": rep["gram_panels"],
               "gram_tflops": round(flops / (rep["gram_ms"] / 1e3) / 1e12, 1),
               "ms_per_application": round(rep["power_ms"] / apps, 3), "applications": apps,
               "phases_ms": {"gram": round(rep["gram_ms"], 1), "power": round(rep["power_ms"], 1),
                             "left": round(rep["left_ms"], 1)},
               "sigma_max_rel_err_vs_truth": float("%.3g" % err),
               "gpu_launches": int(sum(r["kernel_launches"] for r in reps))}
        if rep["tiles_on_host"]:
            gbps = tile_bytes / (rep["power_ms"] / apps / 1e3) / 1e9
            row["tile_stream_GBps"] = round(gbps, 1)
        out[name] = row
        torch.cuda.empty_cache()
    pk = dtype_peak(B.TSVD_GRAM_TF32X3, peaks, sustained=True,
                    tf32_measured=getattr(measure_tf32_peak, "result", None))[0]
    h = out["tiles_on_host"]
    # the pinned-copy peak for tile-sized copies: best of 5 copies of one tile
    tile_h = pinned_array((bs, bs), np.float64)
    tile_h[:] = 1.0
    tile_d = torch.empty((bs, bs), dtype=torch.float64, device="cuda")
    h2d_peak = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        tile_d.copy_(torch.from_numpy(tile_h), non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        h2d_peak = max(h2d_peak, bs * bs * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    line = {"metric": "t-SVD seconds, orthogonally batched Gram with its tiles in host memory",
            "value": h["seconds_per_tsvd"], "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"dense in-core A m={m}, n={n}, rank {rank}, sigma_i=1/(1+i), no noise, k={k}, "
                                   f"eps={eps}, 3xTF32 Gram, panels of {bs} columns ({nb * (nb + 1) // 2} tasks)",
                       "m": m, "n": n, "k": k, "gram_tile": bs, "tile_bytes_per_application": tile_bytes,
                       "l2": "inputs larger than L2 (A is 16 GiB)"},
            "roofline": {"bound": "h2d", "achieved": h.get("tile_stream_GBps"), "peak": round(h2d_peak, 1),
                         "unit": "GB/s", "frac": round(h["tile_stream_GBps"] / h2d_peak, 4)
                         if h.get("tile_stream_GBps") else None, "traffic": None,
                         "kernel": "power phase: FP64 tiles streamed host -> device per application",
                         "peak_source": "measured here: best of 5 pinned copies of one tile"},
            "gram_frac_of_3xtf32_peak": round(h["gram_tflops"] / pk, 4), "budgets": out,
            "gen_seconds": round(gen_s, 1), "peak_source": peak_src}
    print(json.dumps(line), flush=True)


ENVELOPE = 0.1  # sigma_i / sigma_0 down to which an FP32-accumulated Gram resolves sigma to 1e-5
SP_EPS, SP_MAX_ITER = 1e-6, 200  # sparse serving requests: the out-of-core CSR config's eps, capped applications


def serve_workload(args):
    """The serving leg as its own JSON line."""
    import torch

    from paper_2208_08410_gb300 import _binding as B
    B.load(build_if_missing=True)
    torch.cuda.set_device(0)
    print(json.dumps(leg_serve(args, args.requests)), flush=True)


def leg_serve(args, n_req: int):
    """Serving: 10,000 dense t-SVD requests with Poisson arrivals at 2,000 req/s
    drawn from a pool of 512 matrices (m log-uniform in [512, 65536], n
    log-uniform in [64, 2048], sigma_i = rho^i with rho ~ U(0.5, 0.95), exact
    rank where rho^i >= 1e-12), k ~ U{4..32} (capped by min(m, n)), eps = 1e-8,
    each request with its own start seed.  Latency = completion - submission
    on the server's clock.  A second pass submits every request at once
    (capacity, solves/s); the plain per-request path (one tsvd_factor call at a
    time, FP32 Gram) runs on a sample of the same requests as the baseline.
    sigma is checked against the closed form rho^i for every request."""
    import queue
    import threading

    import torch

    import synth
    from paper_2208_08410_gb300 import Plan, Server, _binding as B
    n_pool, rate, eps = args.pool, args.rate, 1e-8
    t0 = time.time()
    shapes = synth.serving_shapes(n_pool, seed=11)
    # the whole pool in one page-locked arena (huge pages for the small matrices too)
    arena, pool = pinned_views([((sh["m"], sh["n"]), np.float32) for sh in shapes])
    for i, sh in enumerate(shapes):
        synth.serving_matrix_torch(sh, seed=i, out=pool[i])
    torch.cuda.empty_cache()
    gen_s = time.time() - t0
    # sparse requests (a share of the mix): square CSR, m = n log-uniform, density 1e-4
    n_sp_pool = (args.serve_sparse_pool or max(4, n_pool // 8)) if args.csr_share > 0 else 0
    sp_lo, sp_hi = (int(x) for x in args.serve_sparse_log2.split(","))
    sp_shapes = synth.serving_sparse_shapes(n_sp_pool, seed=13, dim_range=(1 << sp_lo, 1 << sp_hi))
    if sp_hi <= 16:
        sp_host = [synth.csr_uniform(sh["m"], sh["n"], sh["nnz_per_row"], seed=500 + i)
                   for i, sh in enumerate(sp_shapes)]
    else:  # up to 2^20 x 2^20 at density 1e-4 (1.1e8 entries): drawn on the GPU
        sp_host = []
        for i, sh in enumerate(sp_shapes):
            t = synth.csr_uniform_torch(sh["m"], sh["n"], sh["nnz_per_row"], seed=500 + i)
            sp_host.append({"row_ptr": t["row_ptr"].cpu().numpy(), "col_idx": t["col_idx"].cpu().numpy(),
                            "values": t["values"].cpu().numpy(), "m": sh["m"], "n": sh["n"]})
            del t
        torch.cuda.empty_cache()
    # the sparse pool, too, in one page-locked arena
    keys = ("row_ptr", "col_idx", "values")
    sp_arena, sp_views = pinned_views([(c[key].shape, c[key].dtype.type) for c in sp_host for key in keys])
    sp_pool = []
    for j, c in enumerate(sp_host):
        d = {"m": c["m"], "n": c["n"]}
        for q, key in enumerate(keys):
            v = sp_views[3 * j + q]
            v[...] = c[key]
            d[key] = v
        sp_pool.append(d)
    del sp_host
    g = np.random.default_rng(12)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n_req))
    picks = g.integers(0, n_pool, n_req)
    ks = np.array([min(int(k), min(shapes[p]["m"], shapes[p]["n"]), shapes[p]["rank"])
                   for p, k in zip(picks, g.integers(4, 33, n_req))])
    is_sp = g.random(n_req) < args.csr_share if n_sp_pool else np.zeros(n_req, dtype=bool)
    sp_picks = g.integers(0, max(n_sp_pool, 1), n_req)
    for i in np.nonzero(is_sp)[0]:
        ks[i] = min(int(g.integers(4, 33)), sp_shapes[sp_picks[i]]["m"])
    # output slots: one pool sized for the dense shapes, a smaller one for the sparse shapes
    # (a 2^20-row sparse slot holds 268 MB of U and V, so those are capped at 8 GiB in all)
    m_max, n_max = max(sh["m"] for sh in shapes), max(sh["n"] for sh in shapes)
    slots = 768
    outU = pinned_array((slots, 32 * m_max), np.float32)
    outV = pinned_array((slots, 32 * n_max), np.float32)
    outS = pinned_array((slots, 32), np.float64)
    sp_m = max([sh["m"] for sh in sp_shapes], default=1)
    sp_n = max([sh["n"] for sh in sp_shapes], default=1)
    sp_slots = max(4, min(128, (8 << 30) // (32 * (sp_m + sp_n) * 4))) if n_sp_pool else 1
    outUs = pinned_array((sp_slots, 32 * sp_m), np.float32)
    outVs = pinned_array((sp_slots, 32 * sp_n), np.float32)
    outSs = pinned_array((sp_slots, 32), np.float64)

    def run(server, arr):  # arr: arrival times in seconds, or None to submit everything at once
        free, free_sp = queue.Queue(), queue.Queue()
        for sl in range(slots):
            free.put(sl)
        for sl in range(sp_slots):
            free_sp.put(sl)
        recs = queue.Queue()
        errs = np.zeros(n_req)      # every triplet
        errs_env = np.zeros(n_req)  # triplets with sigma_i >= 0.1 sigma_0
        lat = np.zeros(n_req)
        serv = np.zeros(n_req)     # launch -> completion (the request's time on the GPU, shared)
        apps = np.zeros(n_req)
        done_t = np.zeros(n_req)
        sub_t = np.zeros(n_req)
        status = np.zeros(n_req, dtype=np.int64)

        # several collectors, each waiting on the next submitted ticket, so one slow request
        # holds back one collector (and one output slot), not every completion behind it
        n_coll = 8

        def collector():
            while True:
                item = recs.get()
                if item is None:
                    return
                i, t, sl = item
                st, info = server.wait(t, 600.0)
                p, k = picks[i], ks[i]
                if not is_sp[i]:
                    sig = outS[sl, :k].copy()
                    truth = shapes[p]["rho"] ** np.arange(k)
                    rel = np.abs(sig - truth) / truth
                    errs[i] = float(np.max(rel))
                    env = truth >= ENVELOPE
                    errs_env[i] = float(np.max(rel[env])) if env.any() else 0.0
                lat[i] = info["done_s"] - info["submit_s"]
                serv[i] = info["done_s"] - info["launch_s"]
                apps[i] = info["applications"]
                done_t[i], sub_t[i], status[i] = info["done_s"], info["submit_s"], st
                (free_sp if is_sp[i] else free).put(sl)
        ths = [threading.Thread(target=collector) for _ in range(n_coll)]
        for th in ths:
            th.start()
        start = time.perf_counter()
        for i in range(n_req):
            if arr is not None:
                delay = start + arr[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            sl = (free_sp if is_sp[i] else free).get()
            k = int(ks[i])
            if is_sp[i]:
                csr = sp_pool[sp_picks[i]]
                m, n = csr["m"], csr["n"]
                t = server.submit_csr(csr, k, SP_EPS, outUs[sl, :m * k], outSs[sl, :k], outVs[sl, :n * k],
                                      max_iter=SP_MAX_ITER, seed=i)
            else:
                p = picks[i]
                m, n = shapes[p]["m"], shapes[p]["n"]
                t = server.submit(pool[p], k, eps, outU[sl, :m * k], outS[sl, :k], outV[sl, :n * k], seed=i)
            recs.put((i, t, sl))
        for _ in range(n_coll):
            recs.put(None)
        for th in ths:
            th.join()
        span = float(done_t.max() - sub_t.min())
        dims = np.array([min(shapes[p]["m"], shapes[p]["n"]) for p in picks])
        by_dim = {}
        sparse = None
        if is_sp.any():
            sp = is_sp
            sparse = {"requests": int(sp.sum()), "p50_ms": round(float(np.percentile(lat[sp], 50)) * 1e3, 2),
                      "p99_ms": round(float(np.percentile(lat[sp], 99)) * 1e3, 2),
                      "mean_service_ms": round(float(serv[sp].mean()) * 1e3, 2),
                      "mean_applications": round(float(apps[sp].mean()), 1),
                      "status_counts": {B.STATUS_NAMES[int(c)]: int((status[sp] == c).sum())
                                        for c in np.unique(status[sp])}}
        for lo, hi in ((0, 64), (64, 128), (128, 256), (256, 512), (512, 1024), (1024, 2048)):
            sel = (dims > lo) & (dims <= hi) & ~is_sp
            if sel.any():
                by_dim[f"d<={hi}"] = {"requests": int(sel.sum()),
                                      "mean_service_ms": round(float(serv[sel].mean()) * 1e3, 2),
                                      "p99_service_ms": round(float(np.percentile(serv[sel], 99)) * 1e3, 2),
                                      "mean_applications": round(float(apps[sel].mean()), 1)}
        dn = ~is_sp

        def pct(x, q):
            return round(float(np.percentile(x, q)) * 1e3, 3) if x.size else None

        def mx(x):
            return float("%.3g" % x.max()) if x.size else None
        return {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "dense_p50_ms": pct(lat[dn], 50), "dense_p99_ms": pct(lat[dn], 99),
                "mean_ms": round(float(lat.mean()) * 1e3, 3), "solves_per_s": round(n_req / span, 1),
                "span_s": round(span, 3),
                "sigma_max_rel_err_in_envelope": mx(errs_env[dn]),
                "frac_requests_sigma_err_le_1e-5_in_envelope": float(np.mean(errs_env[dn] <= 1e-5)) if dn.any() else None,
                "sigma_max_rel_err_all_triplets": mx(errs[dn]),
                "frac_requests_sigma_err_le_1e-5_all_triplets": float(np.mean(errs[dn] <= 1e-5)) if dn.any() else None,
                "sparse": sparse,
                "status_counts": {B.STATUS_NAMES[int(c)]: int((status == c).sum()) for c in np.unique(status)},
                "by_dim": by_dim}

    server = Server(device_budget=args.serve_budget << 30, n_streams=args.serve_streams, max_wave=args.serve_max_wave,
                    heavy_dim=args.serve_heavy_dim, heavy_streams=args.serve_heavy_streams,
                    wave_graphs=bool(args.serve_graphs), cluster_cap=args.serve_cluster_cap)
    server.autotune(iters=30)
    if args.serve_cluster_table:  # a fixed table instead of the autotuner's (d <= 64 .. 2048)
        for d, c in zip((64, 128, 256, 512, 1024, 2048), (int(x) for x in args.serve_cluster_table.split(","))):
            server.set_cluster_for(d, c)
    table = {d: server.cluster_for(d) for d in (64, 128, 256, 512, 1024, 2048)}
    tc_from = server.tc_min_d()
    syrk_times = server.autotune_syrk_times()
    s0 = server.stats()
    clocks = ClockSampler(0)
    clocks.start()
    timed = run(server, arrivals)
    s1 = server.stats()
    capacity = run(server, None)
    s2 = server.stats()
    # the same requests once more, Poisson arrivals at 0.9 x the measured capacity: latency of
    # a loaded server that keeps up (the offered 2,000 req/s is above capacity, so there the
    # percentiles measure the queue)
    rate_fit = 0.9 * capacity["solves_per_s"]
    at_fit = run(server, np.cumsum(np.random.default_rng(14).exponential(1.0 / rate_fit, n_req)))
    at_fit = {"rate": round(rate_fit, 1), **{key: at_fit[key] for key in
              ("p50_ms", "p99_ms", "dense_p50_ms", "dense_p99_ms", "solves_per_s", "sparse",
               "sigma_max_rel_err_in_envelope", "frac_requests_sigma_err_le_1e-5_in_envelope")}}
    clk = clocks.stop()
    server.close()
    # baseline: the per-request path, one request at a time, FP32 Gram, same requests
    # (the per-request path takes m >= n only, so the sample skips wide requests)
    tb, n_tall = 0.0, 0
    # the same mix of requests, dense (both shapes) and sparse, one plan per request
    for i in range(min(args.baseline_requests, n_req)):
        k = int(ks[i])
        torch.cuda.synchronize()
        ts = time.perf_counter()
        if is_sp[i]:
            csr = sp_pool[sp_picks[i]]
            m, n = csr["m"], csr["n"]
            plan = Plan(csr, k, SP_EPS, max_iter=SP_MAX_ITER, seed=i)
            plan.factor(csr, U=outUs[0, :m * k], sigma=outSs[0, :k], V=outVs[0, :n * k], ok=(B.TSVD_OK, B.TSVD_ENOCONV))
        else:
            p = picks[i]
            m, n = shapes[p]["m"], shapes[p]["n"]
            plan = Plan(pool[p], k, eps, seed=i)
            plan.factor(pool[p], U=outU[0, :m * k], sigma=outS[0, :k], V=outV[0, :n * k])
        plan.close()
        torch.cuda.synchronize()
        tb += time.perf_counter() - ts
        n_tall += 1
    base_rate = n_tall / tb if tb > 0 else None
    launches = s2["kernel_launches"] - s0["kernel_launches"]
    line = {"metric": "serve p50/p99 latency (2,000 req/s Poisson), sigma err <= 1e-5 inside the FP32-Gram envelope",
            "value": timed["p99_ms"], "unit": "ms", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n_req} t-SVD requests, Poisson {rate} req/s; dense from a pool of {n_pool}: "
                                   "m logU[512,65536], n logU[64,2048], sigma_i=rho^i, rho~U(0.5,0.95), "
                                   f"k~U{{4..32}}, eps=1e-8; {args.csr_share:.0%} CSR from a pool of {n_sp_pool}: "
                                   f"m=n logU[2^{sp_lo},2^{sp_hi}], density 1e-4, eps={SP_EPS}, max_iter {SP_MAX_ITER}",
                       "requests": n_req, "sparse_requests": int(is_sp.sum()), "rate": rate, "pool": n_pool,
                       "sparse_output_slots": sp_slots if n_sp_pool else 0,
                       "pool_bytes": int(sum(a.nbytes for a in pool)), "device_budget_gib": args.serve_budget},
            "accuracy_scope": f"sigma graded against the closed form rho^i on the triplets with rho^i >= {ENVELOPE} "
                              "(an FP32-accumulated Gram moves lambda_i by ~1e-7 lambda_0, i.e. sigma_i by "
                              "~5e-8 / (sigma_i/sigma_0)^2 relative; smaller sigma_i are reported, not graded)",
            "latency": timed, "capacity": capacity, "latency_at_0.9_capacity": at_fit, "cluster_table": table,
            "syrk_tensor_cores_from_d": tc_from if tc_from < (1 << 62) else None,
            "syrk_autotune_ms_tensor_cuda_requests": syrk_times,
            "baseline_per_request": {"solves_per_s": round(base_rate, 1) if base_rate else None,
                                     "requests": n_tall, "path": "tsvd_plan/tsvd_factor per request (the first "
                                                                 "requests of the same mix, dense and sparse), FP32 "
                                                                 "Gram, pinned host A, one at a time"},
            "speedup_capacity_vs_per_request": round(capacity["solves_per_s"] / base_rate, 2) if base_rate else None,
            "server": {"streams": args.serve_streams, "max_wave": args.serve_max_wave,
                       "wave_graphs": bool(args.serve_graphs), "cluster_cap": args.serve_cluster_cap or None,
                       "heavy_dim": args.serve_heavy_dim if args.serve_heavy_dim > 0 else None,
                       "heavy_streams": args.serve_heavy_streams or "auto",
                       "busy_s": round(s2.get("busy_s", 0.0) - s0.get("busy_s", 0.0), 3),
                       "wave_host_s": round(s2.get("wave_host_s", 0.0) - s0.get("wave_host_s", 0.0), 3),
                       "wave_host_ms_per_wave": round(1e3 * (s2.get("wave_host_s", 0.0) - s0.get("wave_host_s", 0.0))
                                                      / max(s2["waves"] - s0["waves"], 1), 3),
                       "graph_host_s": round(s2.get("graph_host_s", 0.0) - s0.get("graph_host_s", 0.0), 3),
                       "peak_streams_busy": s2.get("peak_streams_busy")},
            "waves": s2["waves"] - s0["waves"], "gpu_launches": launches,
            "wave_graphs": {"updated_in_place": s2["graph_updates"] - s0["graph_updates"],
                            "instantiated": s2["graph_instantiations"] - s0["graph_instantiations"]},
            "peak_device_bytes": s2["peak_device_bytes"], "gen_seconds": round(gen_s, 1), "clocks": clk}
    del pool, sp_pool, sp_views
    for a in (arena, sp_arena, outU, outV, outS, outUs, outVs, outSs):
        free_pinned(a)
    torch.cuda.empty_cache()
    return line


def measure_l2_read(nbytes: int = 64 << 20, reps: int = 200) -> float:
    """L2 read rate (GB/s): a torch reduction over an FP32 buffer that fits in
    L2 (64 MB of the 129 MB), read `reps` times back to back after a warm-up,
    CUDA events around the loop."""
    import torch
    x = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    for _ in range(5):
        x.sum()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        x.sum()
    e1.record()
    e1.synchronize()
    return nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def csr_pair_checks(dcsr, host, m, nnz, peaks, peak_src, args, with_cpu=True):
    """Full-size measurements of the fused CSR pair (one operator application
    w = A^T (A v), ||A v||^2) on the device-resident matrix:
    - roofline: average duration of tsvd_csr_gram_apply over the whole matrix
      (CUDA events on the launching stream) against HBM with the algorithmic
      bytes 8 nnz + 8 (m+1) + 4n (v) + 8n (w read + written);
    - cpu_baseline: the oracle's time for sampled row blocks, scaled to one
      application of the whole matrix."""
    import torch

    from paper_2208_08410_gb300 import _binding as B
    stream = torch.cuda.current_stream().cuda_stream
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    v = torch.rand(m, generator=gen, device="cuda", dtype=torch.float32)
    w = torch.zeros(m, dtype=torch.float32, device="cuda")
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    rp, ci, va = dcsr["row_ptr"], dcsr["col_idx"], dcsr["values"]

    def apply_all():
        B.check(B.tsvd_csr_gram_apply(m, m, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), v.data_ptr(),
                                      w.data_ptr(), ss.data_ptr(), 1, stream), "tsvd_csr_gram_apply")
    for _ in range(3):
        apply_all()
    reps = 10
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        apply_all()
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    alg = 8 * nnz + 8 * (m + 1) + 4 * m + 8 * m
    roofline = {"bound": "hbm", "achieved": round(alg / t / 1e9, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(alg / t / 1e9 / peaks["hbm_gbs"], 4),
                "traffic": measured_traffic("csr_pair_kernel", m, m), "kernel": "csr_pair_kernel (fused CSR pair)",
                "ms_per_application": round(t * 1e3, 3), "algorithmic_bytes": alg,
                "peak_source": f"{peak_src} copy bandwidth"}
    cpu = None
    if with_cpu:
        from oracle.csr_c import csr_gram_apply as oracle_apply
        vh = v.cpu().numpy().astype(np.float64)
        bl = 1 << 20
        t0 = time.time()
        rows_done = 0
        sample = []
        for b in range(0, m, bl * 8):
            oracle_apply(host["row_ptr"], host["col_idx"], host["values"], vh, r0=b, r1=min(m, b + bl))
            rows_done += min(m, b + bl) - b
            sample.append(b)
            if time.time() - t0 > 15.0:
                break
        sec = (time.time() - t0) * m / rows_done
        cpu = {"value": round(alg / sec / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle FP64 C operator on {len(sample)} row blocks of {bl} rows "
                         f"({rows_done} of {m} rows), scaled to one application",
               "seconds_per_application": round(sec, 2)}
    return roofline, cpu


def csr_oom_sweep(host, m, nnz, args):
    """Single-GPU analogue of the paper's out-of-memory sweep (Sec. VI-B,
    Fig. 4): the streamed CSR t-SVD timed over the number of row blocks n_b
    (block rows 2^19 .. 2^21) and the ring depth q_s (2 .. 4 buffers), with the
    device footprint of each plan.  k = 4 and 3 applications per triplet keep
    the sweep short; every point reads the whole matrix 4*3 + 4 + 1 times."""
    import torch

    from paper_2208_08410_gb300 import Plan
    k, iters = 4, 3
    out = []
    for br in (1 << 19, 1 << 20, 1 << 21):
        for nb in (2, 3, 4):
            plan = Plan(host, k, EPS, iters_override=[iters] * k, block_rows=br, n_buffers=nb,
                        device_budget=16 * 10 ** 9, force_stream=True, time_kernels=True)
            sec, wall, reps, res = time_steps(plan, host, 2, 1)
            r = reps[-1]
            out.append({"block_rows": br, "n_blocks": r["n_blocks"], "n_buffers": nb,
                        "workspace_bytes": plan.workspace_bytes, "seconds_per_tsvd": round(sec / 2, 3),
                        "h2d_GBps": round(r["h2d_bytes"] / (sec / 2) / 1e9, 1)})
            plan.close()
            torch.cuda.empty_cache()
    return {"k": k, "applications_per_triplet": iters, "points": out}


def csr_workload(args):
    """The sparse out-of-core leg as its own JSON line (plus the out-of-memory
    sweep with --sweep)."""
    import torch

    from paper_2208_08410_gb300 import _binding as B
    B.load(build_if_missing=True)
    torch.cuda.set_device(0)
    print(json.dumps(leg_c3(args, args.steps, args.warmup, with_cpu=not args.no_cpu, sweep=args.sweep)),
          flush=True)


def leg_c3(args, steps: int, warmup: int, with_cpu: bool = False, sweep: bool = False, h2d_peak=None,
           m: int = 0):
    """Sparse out-of-core t-SVD: m = n = 2^25 (default), ~33.5 entries per row
    at uniform random positions, U(0,1) values, row blocks of 2^20 rows under a
    4 GB device budget, k = 16.  A-stream throughput = CSR bytes consumed per
    step (every operator application, the sigma passes and the U pass read the
    whole matrix) / step seconds.  The number of applications per triplet is
    fixed with --csr-iters (the paper's out-of-memory runs fix it at 100) to
    bound the run time.  value: CSR resident in HBM; e2e: CSR streamed from
    page-locked host memory, against the pinned copy rate (h2d_peak)."""
    import torch

    import synth
    from paper_2208_08410_gb300 import Plan, _binding as B
    m = m or args.m or (1 << 25)
    k = K
    t0 = time.time()
    dcsr = synth.csr_uniform_torch(m, m, 33.5, seed=1)
    nnz = int(dcsr["values"].shape[0])
    csr_bytes = 8 * (m + 1) + 8 * nnz
    # pinned host copy for the streamed run
    hrp = pinned_array((m + 1,), np.float64).view(np.int64)
    hvals = pinned_array((nnz,), np.float32)
    hci = pinned_array((nnz,), np.float32).view(np.int32)
    hrp[:] = dcsr["row_ptr"].cpu().numpy()
    hci[:] = dcsr["col_idx"].cpu().numpy()
    hvals[:] = dcsr["values"].cpu().numpy()
    host = {"row_ptr": hrp, "col_idx": hci, "values": hvals, "m": m, "n": m}
    gen_s = time.time() - t0
    iters = [args.csr_iters] * k
    peaks, peak_src = load_peaks()
    roofline, cpu = csr_pair_checks(dcsr, host, m, nnz, peaks, peak_src, args, with_cpu)
    clocks = ClockSampler(0)
    clocks.start()
    plan_d = Plan(dcsr, k, EPS, out_device=True, iters_override=iters, time_kernels=True)
    sec, wall, reps, res = time_steps(plan_d, dcsr, steps, warmup)
    apps = reps[-1]["applications"]
    passes = apps + k + 1  # applications, one sigma pass per triplet, the U pass
    value = csr_bytes * passes * steps / sec / 1e9
    # the operator the in-core t-SVD runs (column-chunked two-pass when v and w outgrow L2):
    # CUDA events around every application on the launching stream
    nch = reps[-1]["csr_chunks"]
    if nch and reps[-1]["gram_kernel_launches"]:
        t_app = reps[-1]["gram_kernel_ms"] / reps[-1]["gram_kernel_launches"] / 1e3
        alg = roofline["algorithmic_bytes"]
        fused = {k2: roofline[k2] for k2 in ("achieved", "frac", "traffic", "ms_per_application")}
        # L2 sectors: pass 1 gathers v (one 32-byte sector per entry) and streams the entries (8 B
        # each), pass 2 streams them again and adds into w (one 32-byte sector per atomic)
        l2_bytes = 80 * nnz + 16 * (m + 1)
        l2_peak = measure_l2_read()
        roofline["l2_sectors"] = {"bound": "l2", "achieved": round(l2_bytes / t_app / 1e9, 1),
                                  "peak": round(l2_peak, 1), "unit": "GB/s",
                                  "frac": round(l2_bytes / t_app / 1e9 / l2_peak, 4),
                                  "sector_bytes_per_application": l2_bytes,
                                  "peak_source": "measured L2 read rate: torch reduction over an L2-resident 64 MB "
                                                 "buffer"}
        roofline.update({"achieved": round(alg / t_app / 1e9, 1), "frac": round(alg / t_app / 1e9 / peaks["hbm_gbs"], 4),
                         "traffic": measured_traffic("csr_chunk_y_kernel+csr_chunk_w_kernel", m, m),
                         "kernel": f"column-chunked CSR operator ({nch} chunks: csr_chunk_y + csr_chunk_w)",
                         "ms_per_application": round(t_app * 1e3, 3),
                         "applications_timed": reps[-1]["gram_kernel_launches"],
                         "fused_pair_kernel": fused})
    plan_d.close()
    del plan_d
    torch.cuda.empty_cache()
    plan_h = Plan(host, k, EPS, iters_override=iters, device_budget=4 * 10 ** 9, block_rows=1 << 20,
                  force_stream=True, time_kernels=True)
    nst = max(1, min(steps, args.e2e_steps or steps))
    sec_e, wall_e, reps_e, res_e = time_steps(plan_h, host, nst, warmup)
    e2e = csr_bytes * passes * nst / sec_e / 1e9
    plan_h.close()
    clk = clocks.stop()
    if h2d_peak is None:
        blk = torch.from_numpy(hvals[:1 << 26])
        dst = torch.empty_like(blk, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 0.0
        for _ in range(3):
            e0.record()
            dst.copy_(blk, non_blocking=True)
            e1.record()
            e1.synchronize()
            best = max(best, blk.numel() * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
        h2d_peak = best
        del dst
    sweep = csr_oom_sweep(host, m, nnz, args) if sweep else None
    line = {"metric": "t-SVD A-stream throughput (CSR)", "value": round(value, 2), "unit": "GB/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": round(sec / steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"sparse CSR t-SVD, m=n={m}, ~33.5 nnz/row ({nnz} nnz), k={k}, "
                                   f"{args.csr_iters} applications per triplet", "m": m, "nnz": nnz,
                       "csr_bytes": csr_bytes, "k": k, "block_rows_e2e": 1 << 20,
                       "device_budget_bytes_e2e": 4 * 10 ** 9},
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "ms_per_step": round(sec_e / nst * 1e3, 1),
                    "steps": nst, "pinned_copy_peak_GBps": round(h2d_peak, 2),
                    "host_values_pages": thp_coverage(hvals), "host_col_idx_pages": thp_coverage(hci),
                    "host_row_ptr_pages": thp_coverage(hrp),
                    "frac_of_pinned_copy": round(e2e / h2d_peak, 4),
                    "h2d_bytes_per_step": int(reps_e[-1]["h2d_bytes"]),
                    "d2h_bytes_per_step": int(reps_e[-1]["d2h_bytes"]),
                    "blocks_per_pass": reps_e[-1]["n_blocks"],
                    "copy_stream_GBps": round(reps_e[-1]["h2d_bytes"] / (reps_e[-1]["h2d_copy_ms"] / 1e3) / 1e9, 2)
                    if reps_e[-1]["h2d_copy_ms"] else None,
                    "copy_min_GBps": round(reps_e[-1]["h2d_copy_min_gbps"], 1),
                    "copy_max_GBps": round(reps_e[-1]["h2d_copy_max_gbps"], 1),
                    "pair_kernel_ms_per_step": round(reps_e[-1]["gram_kernel_ms"], 1),
                    "pair_kernel_launches_per_step": reps_e[-1]["gram_kernel_launches"]},
            "roofline": roofline, "cpu_baseline": cpu, "oom_sweep": sweep,
            "sigma": [round(float(x), 6) for x in res.sigma.cpu().numpy()], "gen_seconds": round(gen_s, 1),
            "gpu_launches": int(sum(r["kernel_launches"] for r in reps)), "clocks": clk}
    for a in (hrp, hci, hvals):
        free_pinned(a)
    del dcsr
    torch.cuda.empty_cache()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=0, help="rows (default: largest multiple of 262,144 that fits)")
    ap.add_argument("--precision", type=int, default=2,
                    help="Gram arithmetic: 0 FP32 CUDA cores, 1 TF32, 2 3xTF32 (FP32-class, default), 3 BF16x3")
    ap.add_argument("--ref-rows", type=int, default=65_536)
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0)
    ap.add_argument("--case", default="",
                    choices=["", "gram", "power", "csr", "left", "c1", "csr_tsvd", "csr_small", "tf32ref"],
                    help="single-kernel microbenchmark instead of the t-SVD step")
    ap.add_argument("--n", type=int, default=N_COLS)
    ap.add_argument("--workload", default="dense", choices=["dense", "csr", "c4", "serve", "tiled"])
    ap.add_argument("--pool", type=int, default=512)
    ap.add_argument("--requests", type=int, default=10_000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--serve-budget", type=int, default=128, help="server device budget, GiB")
    ap.add_argument("--baseline-requests", type=int, default=200)
    ap.add_argument("--csr-share", type=float, default=0.1, help="serving: fraction of sparse requests")
    ap.add_argument("--csr-iters", type=int, default=10)
    ap.add_argument("--sweep", action="store_true", help="CSR: out-of-memory sweep over n_b and q_s")
    ap.add_argument("--legs", default="c2_small,c4,c3_streamed,serve",
                    help="dense workload: further configurations run after the headline and reported as keys of "
                         "the same line (comma list, empty for none)")
    ap.add_argument("--legs-budget-s", type=float, default=1500.0,
                    help="skip the remaining legs once the run has taken this long")
    ap.add_argument("--serve-requests-leg", type=int, default=10_000, help="requests of the serving leg")
    ap.add_argument("--e2e-block-rows", type=int, default=BLOCK_ROWS, help="rows per streamed block (e2e)")
    ap.add_argument("--full-oracle", action="store_true",
                    help="dense: the oracle's trajectory over all of A (FP64 Gram on the host, ~5 min on 16 cores)")
    ap.add_argument("--serve-streams", type=int, default=8, help="serving: waves in flight (streams)")
    ap.add_argument("--serve-graphs", type=int, default=0, help="serving: 1 launches each wave as a CUDA graph")
    ap.add_argument("--serve-cluster-table", default="",
                    help="serving: power-kernel cluster sizes for d <= 64,128,256,512,1024,2048 (default: autotuned)")
    ap.add_argument("--serve-cluster-cap", type=int, default=0,
                    help="serving: most CTAs per power-kernel cluster (0: the server's default, 8)")
    ap.add_argument("--serve-max-wave", type=int, default=256, help="serving: requests per wave")
    ap.add_argument("--serve-heavy-dim", type=int, default=0, help="serving: heavy lane above this d (0: none)")
    ap.add_argument("--serve-sparse-pool", type=int, default=0, help="serving: distinct sparse matrices (0: pool/8)")
    ap.add_argument("--serve-sparse-log2", default="14,16",
                    help="serving: sparse requests m = n log-uniform in [2^a, 2^b] (the config allows up to 2^20)")
    ap.add_argument("--serve-heavy-streams", type=int, default=0, help="serving: streams of the heavy lane (0: auto)")
    args = ap.parse_args()
    if args.case:
        kernel_case(args)
        return
    if args.workload == "csr" and args.impl != "reference":
        csr_workload(args)
        return
    if args.workload == "c4" and args.impl != "reference":
        c4_workload(args)
        return
    if args.workload == "tiled" and args.impl != "reference":
        tiled_workload(args)
        return
    if args.workload == "serve" and args.impl != "reference":
        serve_workload(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        m = pick_m(args.m)
        print(json.dumps(reference_arm(args, m)), flush=True)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2208_08410_gb300 import Plan, _binding as B
    B.load(build_if_missing=True)
    t_run = time.time()

    m = pick_m(args.m)
    t0 = time.time()
    A, hptr, facts = make_host_A(m, seed=rank)
    gen_s = time.time() - t0
    thp_A = thp_coverage(A)
    h2d_burst, h2d_peak = measure_h2d_peak(A)
    dA = torch.empty((m, N_COLS), dtype=torch.float32, device="cuda")
    for r0 in range(0, m, BLOCK_ROWS):
        dA[r0:r0 + BLOCK_ROWS].copy_(torch.from_numpy(A[r0:r0 + BLOCK_ROWS]), non_blocking=True)
    torch.cuda.synchronize()

    prec = args.precision
    peaks, peak_src = load_peaks()
    tf32_meas = measure_tf32_peak()
    # ---------------- value: A in HBM
    plan_dev = Plan(dA, K, EPS, precision=prec, out_device=True, time_kernels=True)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    sec, wall, reps, res_dev = time_steps(plan_dev, dA, args.steps, args.warmup)
    clk = clocks.stop()
    bytes_per_step = 2 * m * N_COLS * 4
    rate, sec = whole_job_rate(sec, bytes_per_step * args.steps, dist, "cuda")
    step_s = sec / args.steps
    value = rate / 1e9
    launches = int(sum(r["kernel_launches"] for r in reps))
    gk_ms = sum(r["gram_kernel_ms"] for r in reps)
    gk_n = sum(r["gram_kernel_launches"] for r in reps)
    flops_per_step = m * N_COLS * (N_COLS + 1)
    achieved_tf = flops_per_step * args.steps / (gk_ms / 1e3) / 1e12 if gk_ms > 0 else None
    peak, bound, peak_note = dtype_peak(prec, peaks, sustained=True, tf32_measured=tf32_meas)
    roof = {"bound": bound, "peak_note": peak_note}
    chunk_rows = int(round(m / max(gk_n / max(args.steps, 1), 1)))
    kname = {0: "syrk_simt_kernel", 1: "syrk_tc_kernel<TF32>", 2: "syrk_tc_kernel<TF32X3>",
             3: "syrk_tc_kernel<BF16X3>"}[prec]
    roofline = {"bound": roof["bound"], "achieved": round(achieved_tf, 2) if achieved_tf else None,
                "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved_tf / peak, 4) if achieved_tf else None,
                "traffic": measured_traffic(kname, chunk_rows, N_COLS),
                "kernel": "Gram accumulation (SYRK)", "launches_per_step": gk_n / max(args.steps, 1),
                "algorithmic_flops_per_step": flops_per_step, "peak_source": peak_src + "; " + roof["peak_note"]}
    plan_dev.close()
    del plan_dev
    torch.cuda.empty_cache()
    alt = alt_bf = None
    if prec == 2:
        alt = alt_precision_in_core(dA, args, m, res_dev, peaks, 1)
        torch.cuda.empty_cache()
        alt_bf = alt_precision_in_core(dA, args, m, res_dev, peaks, 3)
        torch.cuda.empty_cache()
    small = c1_latency() if rank == 0 else None

    # ---------------- e2e: pinned host A, streamed, outputs to host
    e2e_steps = args.e2e_steps or min(args.steps, 10)
    plan_host = Plan(A, K, EPS, precision=prec, device_budget=BUDGET, block_rows=args.e2e_block_rows,
                     force_stream=True, time_kernels=True)
    outs = {"U": pinned_array((K, m), np.float32), "sigma": pinned_array((K,), np.float64),
            "V": pinned_array((K, N_COLS), np.float32)}
    clocks_e = ClockSampler(local)
    clocks_e.start()
    sec_e, wall_e, reps_e, res_host = time_steps(plan_host, A, e2e_steps, args.warmup, outs=outs)
    clk_e = clocks_e.stop()
    _, lb, lg = plan_host.copy_log()
    nb_gram = reps_e[-1]["n_blocks"]
    rate_e, sec_e = whole_job_rate(sec_e, bytes_per_step * e2e_steps, dist, "cuda")
    e2e_step = sec_e / e2e_steps
    h2d_b = reps_e[-1]["h2d_bytes"]
    d2h_b = reps_e[-1]["d2h_bytes"]
    gram_pass_s = reps_e[-1]["gram_ms"] / 1e3
    e2e = {"value": round(rate_e / 1e9, 3), "unit": "GB/s",
           "h2d_bytes_per_step": int(h2d_b), "d2h_bytes_per_step": int(d2h_b),
           "ms_per_step": round(e2e_step * 1e3, 2),
           "phases_ms": {"gram": round(reps_e[-1]["gram_ms"], 2), "power": round(reps_e[-1]["power_ms"], 2),
                         "left": round(reps_e[-1]["left_ms"], 2)},
           "h2d": {"gram_pass_GBps": round(m * N_COLS * 4 / gram_pass_s / 1e9, 2),
                   "pinned_copy_peak_GBps": round(h2d_peak, 2),
                   "pinned_copy_burst_GBps": round(h2d_burst, 2),
                   "pinned_copy_per_block_GBps": getattr(measure_h2d_peak, "per_block", None),
                   "peak_note": "peak = sustained pinned copy of every row block of A back to back",
                   "frac_gram_pass": round(m * N_COLS * 4 / gram_pass_s / 1e9 / h2d_peak, 4),
                   "frac_gram_pass_of_burst": round(m * N_COLS * 4 / gram_pass_s / 1e9 / h2d_burst, 4),
                   "blocks_per_pass": reps_e[-1]["n_blocks"], "ring_slots": reps_e[-1]["ring_slots"],
                   "block_copies_per_step": reps_e[-1]["h2d_copies"],
                   "copy_stream_GBps": round(reps_e[-1]["h2d_bytes"] / (reps_e[-1]["h2d_copy_ms"] / 1e3) / 1e9, 2)
                   if reps_e[-1]["h2d_copy_ms"] else None,
                   "copy_min_GBps": round(reps_e[-1]["h2d_copy_min_gbps"], 1),
                   "copy_max_GBps": round(reps_e[-1]["h2d_copy_max_gbps"], 1),
                   "host_A_pages": thp_A,
                   "gram_pass_block_GBps": [round(float(x), 1) for x in lg[:nb_gram]],
                   "u_pass_block_GBps": [round(float(x), 1) for x in lg[nb_gram:]],
                   "block_huge_page_frac": thp_by_block(A, args.e2e_block_rows * N_COLS * 4)},
           "gram_kernels": {"syrk_ms_per_step": round(reps_e[-1]["gram_kernel_ms"], 2),
                            "launches_per_step": reps_e[-1]["gram_kernel_launches"],
                            "syrk_tflops": round(m * N_COLS * (N_COLS + 1) / (reps_e[-1]["gram_kernel_ms"] / 1e3)
                                                 / 1e12, 1) if reps_e[-1]["gram_kernel_ms"] else None},
           "clocks": clk_e}
    launches_e = int(sum(r["kernel_launches"] for r in reps_e))
    plan_host.close()
    for a in outs.values():
        free_pinned(a)
    del res_host

    parity = None
    if not args.no_parity and rank == 0:
        parity = parity_full_size(A, dA, res_dev, prec)
    full_oracle = None
    if args.full_oracle and rank == 0:
        full_oracle = parity_full_oracle(A, res_dev, seed=0)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        sig = np.asarray(res_dev.sigma.cpu().numpy())
        Vg = res_dev.V.cpu().numpy()
        cpu = cpu_baseline(m, A, Vg, sig, res_dev.iters)

    del dA
    torch.cuda.empty_cache()
    B.tsvd_host_free(hptr)
    hptr = None
    del A
    legs = {}
    if rank == 0 and world == 1:
        steps_leg, warm_leg = max(1, min(args.steps, 3)), max(1, min(args.warmup, 2))
        runners = {"c2_small": lambda: leg_c2_small(args),
                   "c4": lambda: leg_c4(args, steps_leg, warm_leg),
                   "c3_streamed": lambda: leg_c3(args, steps_leg, 1, with_cpu=False, h2d_peak=h2d_peak,
                                                 m=1 << 25),
                   "serve": lambda: leg_serve(args, args.serve_requests_leg)}
        for name in [x for x in args.legs.split(",") if x]:
            if name not in runners:
                legs[name] = {"error": "unknown leg"}
                continue
            if time.time() - t_run > args.legs_budget_s:
                legs[name] = {"skipped": f"run time above {args.legs_budget_s:.0f} s before this leg"}
                continue
            t_leg = time.time()
            try:
                legs[name] = runners[name]()
            except Exception as e:  # a leg's failure is reported in the line, not fatal to it
                legs[name] = {"error": repr(e)[:400]}
            legs[name]["leg_seconds"] = round(time.time() - t_leg, 1)
            torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": "t-SVD A-stream throughput", "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 2),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": PREC_NAMES[prec], "data": "synthetic",
                "config": dense_config(m, prec, world),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "tf32_in_core": alt, "bf16x3_in_core": alt_bf,
                "c1_latency": small,
                "gpu_launches": launches, "gpu_launches_e2e": launches_e,
                "phases_ms": {"gram": round(reps[-1]["gram_ms"], 2), "power": round(reps[-1]["power_ms"], 2),
                              "left": round(reps[-1]["left_ms"], 2), "applications": reps[-1]["applications"]},
                "iters": res_dev.iters, "sigma": [round(float(s), 8) for s in np.asarray(res_dev.sigma.cpu())],
                "parity": parity, "parity_oracle_full_size": full_oracle,
                "gen_seconds": round(gen_s, 1), "tf32_cublas_peak": tf32_meas,
                "run_seconds": round(time.time() - t_run, 1)}
        line.update(legs)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
