"""Single-GPU (GB300, sm_103a) truncated SVD by the deflated power method of
arXiv 2208.08410, behind a C ABI (include/tsvd.h).

`tsvd(A, k, eps, ...)` plans and runs one factorisation.  A may be a NumPy
array (host memory; pinned buffers stream fastest), a CUDA torch tensor
(device-resident A), or a CSR dict {row_ptr, col_idx, values, m, n} of either.
PyTorch is used only to allocate the device workspace and pick the stream;
every step of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _binding as B

__all__ = ["tsvd", "TSVDResult", "Plan", "B"]


@dataclass
class TSVDResult:
    U: object
    sigma: object
    V: object
    iters: list
    status: int
    report: dict


def _ptr(a):
    """Data pointer of a NumPy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def make_matrix(A):
    """Build a tsvd_matrix descriptor (and the list of objects to keep alive)."""
    m = B.tsvd_matrix()
    keep = []
    if isinstance(A, dict):
        rp, ci, va = A["row_ptr"], A["col_idx"], A["values"]
        dev = _is_device(rp)
        if not dev:
            rp = np.ascontiguousarray(rp, dtype=np.int64)
            ci = np.ascontiguousarray(ci, dtype=np.int32)
            va = np.ascontiguousarray(va, dtype=np.float32)
        keep += [rp, ci, va]
        m.kind = B.TSVD_CSR_F32_I32_I64
        m.location = B.TSVD_DEVICE if dev else B.TSVD_HOST
        m.m, m.n = int(A["m"]), int(A["n"])
        m.ld = 0
        m.values, m.row_ptr, m.col_idx = _ptr(va), _ptr(rp), _ptr(ci)
        m.nnz = int(va.shape[0])
    else:
        dev = _is_device(A)
        if not dev:
            if not (isinstance(A, np.ndarray) and A.dtype == np.float32 and A.strides[1] == 4):
                A = np.ascontiguousarray(A, dtype=np.float32)
            ld = A.strides[0] // 4
        else:
            import torch
            assert A.dtype == torch.float32 and A.stride(1) == 1
            ld = A.stride(0)
        keep.append(A)
        m.kind = B.TSVD_DENSE_F32_ROWMAJOR
        m.location = B.TSVD_DEVICE if dev else B.TSVD_HOST
        m.m, m.n = int(A.shape[0]), int(A.shape[1])
        m.ld = int(ld)
        m.values = _ptr(A)
    return m, keep


class Plan:
    """A tsvd plan plus its device workspace (torch-allocated).

    The keyword options map one to one onto `tsvd_options` in include/tsvd.h:
    precision (TSVD_GRAM_FP32 / TF32 / TF32X3 / BF16X3), device_budget (bytes,
    0 = none), block_rows and n_buffers (the streamed ring), max_iter,
    iters_override (k forced application counts), start_draws (min(m, n) x k
    N(0,1) draws instead of the built-in Philox stream), seed, out_device
    (outputs in device memory), sign_convention, force_stream, time_kernels,
    power_kernel (TSVD_POWER_AUTO / GRID / CLUSTER), gram_tile (orthogonal
    batching panel width), power_ctas (cluster size of the cluster kernel) and
    wait_limit_ns (limit of the tensor-core Gram kernel's waits, for testing the
    timeout path; 0 = 2 s).
    `factor()` runs the t-SVD; `close()` releases the plan."""

    def __init__(self, A, k: int, eps: float, *, precision: int = B.TSVD_GRAM_FP32, device_budget: int = 0,
                 block_rows: int = 0, n_buffers: int = 3, max_iter: int = 10000, iters_override=None,
                 start_draws=None, seed: int = 0, out_device: bool = False, sign_convention: bool = False,
                 force_stream: bool = False, time_kernels: bool = False, power_kernel: int = B.TSVD_POWER_AUTO,
                 gram_tile: int = 0, power_ctas: int = 0, wait_limit_ns: int = 0):
        import torch
        self.lib = B.load()
        self.mat, self._keep = make_matrix(A)
        opt = B.tsvd_options()
        self.lib.tsvd_options_init(C.byref(opt))
        opt.device_budget = int(device_budget)
        opt.block_rows = int(block_rows)
        opt.n_buffers = int(n_buffers)
        opt.precision = int(precision)
        opt.max_iter = int(max_iter)
        opt.sign_convention = int(bool(sign_convention))
        opt.seed = int(seed)
        opt.out_location = B.TSVD_DEVICE if out_device else B.TSVD_HOST
        opt.force_stream = int(bool(force_stream))
        opt.time_kernels = int(bool(time_kernels))
        opt.power_kernel = int(power_kernel)
        opt.gram_tile = int(gram_tile)
        opt.power_ctas = int(power_ctas)
        opt.wait_limit_ns = int(wait_limit_ns)
        mn = min(self.mat.m, self.mat.n)
        self.k = mn if k == -1 else int(k)
        if iters_override is not None:
            self._ovr = np.ascontiguousarray(iters_override, dtype=np.int32)
            opt.iters_override = self._ovr.ctypes.data
        if start_draws is not None:
            self._sd = np.asfortranarray(start_draws, dtype=np.float64)
            opt.start_draws = self._sd.ctypes.data
        self.opt = opt
        h = C.c_void_p()
        ws = C.c_size_t()
        B.check(self.lib.tsvd_plan(C.byref(h), C.byref(self.mat), int(k), float(eps), C.byref(opt), C.byref(ws)),
                "tsvd_plan")
        self.handle = h
        self.workspace_bytes = int(ws.value)
        self.out_device = out_device
        self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device="cuda")

    def factor(self, A=None, U=None, sigma=None, V=None, want_u: bool = True, ok=(B.TSVD_OK,)):
        import torch
        if A is not None:
            self.mat, self._keep = make_matrix(A)
        m, n, k = self.mat.m, self.mat.n, self.k
        if self.out_device:
            if U is None and want_u:
                U = torch.empty((k, m), dtype=torch.float32, device="cuda")
            if sigma is None:
                sigma = torch.empty(k, dtype=torch.float64, device="cuda")
            if V is None:
                V = torch.empty((k, n), dtype=torch.float32, device="cuda")
        else:
            if U is None and want_u:
                U = np.empty((k, m), dtype=np.float32)
            if sigma is None:
                sigma = np.empty(k, dtype=np.float64)
            if V is None:
                V = np.empty((k, n), dtype=np.float32)
        iters = np.zeros(k, dtype=np.int32)
        rep = B.tsvd_report()
        rep.iters = iters.ctypes.data
        stream = torch.cuda.current_stream().cuda_stream
        st = self.lib.tsvd_factor(self.handle, C.byref(self.mat), self.workspace.data_ptr(), self.workspace_bytes,
                                  stream, _ptr(U) if want_u else None, _ptr(sigma), _ptr(V), C.byref(rep))
        B.check(st, "tsvd_factor", ok=ok)
        report = {f: getattr(rep, f) for f, _ in B.tsvd_report._fields_ if f != "iters"}
        # U and V are stored column-major (m x k / n x k): expose them as (rows, k) views
        Uo = U.T if U is not None else None
        return TSVDResult(Uo, sigma, V.T, iters.tolist(), st, report)

    def copy_log(self):
        """(first, bytes, GB/s) of each timed block copy of the last factor()
        call (time_kernels=True), from tsvd_plan_copy_log."""
        cnt = C.c_int64()
        B.check(self.lib.tsvd_plan_copy_log(self.handle, None, None, None, 0, C.byref(cnt)), "tsvd_plan_copy_log")
        n = int(cnt.value)
        first = np.zeros(n, dtype=np.int64)
        nb = np.zeros(n, dtype=np.float64)
        g = np.zeros(n, dtype=np.float64)
        B.check(self.lib.tsvd_plan_copy_log(self.handle, first.ctypes.data, nb.ctypes.data, g.ctypes.data, n,
                                            C.byref(cnt)), "tsvd_plan_copy_log")
        return first, nb, g

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tsvd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tsvd(A, k: int, eps: float, **kw) -> TSVDResult:
    """Plan and run one truncated SVD; see Plan for the keyword options."""
    ok = kw.pop("ok", (B.TSVD_OK,))
    want_u = kw.pop("want_u", True)
    p = Plan(A, k, eps, **kw)
    try:
        return p.factor(want_u=want_u, ok=ok)
    finally:
        p.close()


class Server:
    """A t-SVD server (continuous batching of many requests on one GPU); see
    tsvd_server_* in include/tsvd.h.  Inputs and outputs are host arrays the
    caller keeps alive until the request completes (page-locked ones, e.g. from
    tsvd_host_alloc, let the copies overlap other work)."""

    def __init__(self, device_budget: int = 8 << 30, max_inflight: int = 0, n_streams: int = 0,
                 max_wave: int = 0, cluster_cap: int = 0, heavy_dim: int = 0, heavy_streams: int = 0,
                 wave_graphs: bool = False):
        import torch
        torch.cuda.init()
        self.lib = B.load()
        opt = B.tsvd_server_options()
        self.lib.tsvd_server_options_init(C.byref(opt))
        opt.device_budget = int(device_budget)
        opt.max_inflight = int(max_inflight)
        opt.n_streams = int(n_streams)
        opt.max_wave = int(max_wave)
        opt.cluster_cap = int(cluster_cap)
        opt.heavy_dim = int(heavy_dim)
        opt.heavy_streams = int(heavy_streams)
        opt.wave_graphs = 1 if wave_graphs else 0
        h = C.c_void_p()
        B.check(self.lib.tsvd_server_create(C.byref(h), C.byref(opt)), "tsvd_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, A, k: int, eps: float, U, sigma, V, max_iter: int = 10000, seed: int = 0,
               sign_convention: bool = False, iters_override=None) -> int:
        m, n = A.shape
        t = C.c_uint64()
        ovr = None
        if iters_override is not None:
            ovr = np.ascontiguousarray(iters_override, dtype=np.int32)
        B.check(self.lib.tsvd_server_submit(self.handle, _ptr(A), m, n, int(k), float(eps), int(max_iter), int(seed),
                                            int(bool(sign_convention)), _ptr(ovr), _ptr(U), _ptr(sigma), _ptr(V),
                                            C.byref(t)),
                "tsvd_server_submit")
        self._keep[t.value] = (A, U, sigma, V)
        return t.value

    def submit_csr(self, csr: dict, k: int, eps: float, U, sigma, V, max_iter: int = 10000, seed: int = 0,
                   sign_convention: bool = False, iters_override=None) -> int:
        """A sparse request: csr = {"row_ptr", "col_idx", "values", "m", "n"} in host memory, kept
        alive until the request completes."""
        rp, ci, va = csr["row_ptr"], csr["col_idx"], csr["values"]
        m, n = int(csr["m"]), int(csr["n"])
        t = C.c_uint64()
        ovr = None
        if iters_override is not None:
            ovr = np.ascontiguousarray(iters_override, dtype=np.int32)
        B.check(self.lib.tsvd_server_submit_csr(self.handle, _ptr(rp), _ptr(ci), _ptr(va), m, n, int(va.shape[0]),
                                                int(k), float(eps), int(max_iter), int(seed),
                                                int(bool(sign_convention)), _ptr(ovr), _ptr(U), _ptr(sigma), _ptr(V),
                                                C.byref(t)),
                "tsvd_server_submit_csr")
        self._keep[t.value] = (csr, U, sigma, V, ovr)
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        info = B.tsvd_request_info()
        st = self.lib.tsvd_server_wait(self.handle, int(ticket), float(timeout_s), C.byref(info))
        if st != B.TSVD_ETIMEDOUT:
            self._keep.pop(ticket, None)
        return st, {f: getattr(info, f) for f, _ in B.tsvd_request_info._fields_}

    def stats(self) -> dict:
        s = B.tsvd_server_stats()
        B.check(self.lib.tsvd_server_get_stats(self.handle, C.byref(s)), "tsvd_server_get_stats")
        return {f: getattr(s, f) for f, _ in B.tsvd_server_stats._fields_}

    def cluster_for(self, d: int) -> int:
        return int(self.lib.tsvd_server_cluster_for(self.handle, int(d)))

    def set_cluster_for(self, d: int, c: int):
        B.check(self.lib.tsvd_server_set_cluster_for(self.handle, int(d), int(c)), "tsvd_server_set_cluster_for")

    def tc_min_d(self) -> int:
        """Gram dimension from which requests use the tensor-core SYRK."""
        return int(self.lib.tsvd_server_tc_min_d(self.handle))

    def autotune_syrk_times(self) -> dict:
        """{d: (ms tensor cores, ms CUDA cores, requests)} of the last autotune."""
        d = np.zeros(4, dtype=np.int64)
        a = np.zeros(4)
        b = np.zeros(4)
        n = np.zeros(4, dtype=np.int32)
        B.check(self.lib.tsvd_server_autotune_syrk_times(self.handle, d.ctypes.data, a.ctypes.data, b.ctypes.data,
                                                          n.ctypes.data), "tsvd_server_autotune_syrk_times")
        return {int(d[i]): (round(float(a[i]), 3), round(float(b[i]), 3), int(n[i])) for i in range(4)}

    def set_tc_min_d(self, d: int):
        B.check(self.lib.tsvd_server_set_tc_min_d(self.handle, int(d)), "tsvd_server_set_tc_min_d")

    def autotune(self, iters: int = 50):
        B.check(self.lib.tsvd_server_autotune(self.handle, int(iters)), "tsvd_server_autotune")

    def last_error(self) -> str:
        return self.lib.tsvd_server_last_error(self.handle).decode()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tsvd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
