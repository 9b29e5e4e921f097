"""ctypes binding of the tsvd C ABI (include/tsvd.h), argument marshalling only.

Every function keeps the C name; all compute happens in the CUDA library.
If the compiled library is missing the loader raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

TSVD_OK, TSVD_EINVAL, TSVD_ENOMEM, TSVD_EBUDGET, TSVD_ECUDA = 0, 1, 2, 3, 4
TSVD_ETIMEDOUT, TSVD_ENOCONV, TSVD_ERANK, TSVD_EUNSUPPORTED = 5, 6, 7, 8
TSVD_DENSE_F32_ROWMAJOR, TSVD_CSR_F32_I32_I64 = 0, 1
TSVD_HOST, TSVD_DEVICE = 0, 1
TSVD_GRAM_FP32, TSVD_GRAM_TF32, TSVD_GRAM_TF32X3, TSVD_GRAM_BF16X3 = 0, 1, 2, 3
TSVD_POWER_AUTO, TSVD_POWER_GRID, TSVD_POWER_CLUSTER = 0, 1, 2
TSVD_NOALLOC_MAX_N, TSVD_NOALLOC_MAX_L = 16384, 64
TSVD_FLAG_NOCONV, TSVD_FLAG_RANK, TSVD_FLAG_NONMONOTONE, TSVD_FLAG_PAGEABLE, TSVD_FLAG_TIMEOUT = 1, 2, 4, 8, 16

STATUS_NAMES = {0: "TSVD_OK", 1: "TSVD_EINVAL", 2: "TSVD_ENOMEM", 3: "TSVD_EBUDGET", 4: "TSVD_ECUDA",
                5: "TSVD_ETIMEDOUT", 6: "TSVD_ENOCONV", 7: "TSVD_ERANK", 8: "TSVD_EUNSUPPORTED"}


class tsvd_matrix(C.Structure):
    _fields_ = [("kind", C.c_int32), ("location", C.c_int32), ("m", C.c_int64), ("n", C.c_int64),
                ("ld", C.c_int64), ("values", C.c_void_p), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("nnz", C.c_int64)]


class tsvd_options(C.Structure):
    _fields_ = [("device_budget", C.c_size_t), ("block_rows", C.c_int64), ("n_buffers", C.c_int32),
                ("precision", C.c_int32), ("max_iter", C.c_int32), ("sign_convention", C.c_int32),
                ("iters_override", C.c_void_p), ("start_draws", C.c_void_p), ("seed", C.c_uint64),
                ("out_location", C.c_int32), ("force_stream", C.c_int32), ("time_kernels", C.c_int32),
                ("power_kernel", C.c_int32), ("gram_tile", C.c_int32),
                ("power_ctas", C.c_int32), ("wait_limit_ns", C.c_int32), ("csr_coop_blocks", C.c_int32)]


class tsvd_report(C.Structure):
    _fields_ = [("iters", C.c_void_p), ("flags", C.c_int32), ("n_blocks", C.c_int32), ("mode", C.c_int32),
                ("gram_kernel_launches", C.c_int32), ("gram_ms", C.c_double), ("power_ms", C.c_double),
                ("left_ms", C.c_double), ("total_ms", C.c_double), ("h2d_bytes", C.c_double),
                ("d2h_bytes", C.c_double), ("gram_kernel_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("applications", C.c_int64), ("ring_slots", C.c_int32), ("h2d_copies", C.c_int32),
                ("h2d_copy_ms", C.c_double), ("h2d_copy_min_gbps", C.c_double),
                ("h2d_copy_max_gbps", C.c_double), ("csr_chunks", C.c_int32), ("power_cluster", C.c_int32),
                ("gram_panels", C.c_int32), ("tiles_on_host", C.c_int32)]


class tsvd_server_options(C.Structure):
    _fields_ = [("device_budget", C.c_size_t), ("max_inflight", C.c_int32), ("n_streams", C.c_int32),
                ("max_wave", C.c_int32), ("cluster_cap", C.c_int32), ("host_staging", C.c_size_t),
                ("heavy_dim", C.c_int32), ("heavy_streams", C.c_int32), ("wave_graphs", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class tsvd_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("flags", C.c_int32), ("applications", C.c_int64),
                ("submit_s", C.c_double), ("admit_s", C.c_double), ("launch_s", C.c_double),
                ("done_s", C.c_double), ("wave", C.c_int32), ("cluster", C.c_int32)]


class tsvd_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("waves", C.c_int64), ("kernel_launches", C.c_int64), ("peak_device_bytes", C.c_int64),
                ("busy_s", C.c_double), ("graph_updates", C.c_int64),
                ("graph_instantiations", C.c_int64), ("wave_host_s", C.c_double),
                ("peak_streams_busy", C.c_int64), ("graph_host_s", C.c_double)]


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_D = C.c_double
_SZ = C.c_size_t

# name -> (restype, argtypes); the list mirrors include/tsvd.h
SIGNATURES = {
    "tsvd_status_string": (C.c_char_p, [C.c_int]),
    "tsvd_last_cuda_error": (C.c_char_p, []),
    "tsvd_abi_version": (_I32, []),
    "tsvd_options_init": (None, [C.POINTER(tsvd_options)]),
    "tsvd_plan": (C.c_int, [C.POINTER(_P), C.POINTER(tsvd_matrix), _I64, _D, C.POINTER(tsvd_options),
                            C.POINTER(_SZ)]),
    "tsvd_factor": (C.c_int, [_P, C.POINTER(tsvd_matrix), _P, _SZ, _P, _P, _P, _P, C.POINTER(tsvd_report)]),
    "tsvd_destroy": (None, [_P]),
    "tsvd_gram_scratch_bytes": (_SZ, [_I64, _I64, _I32]),
    "tsvd_gram_accumulate": (C.c_int, [_P, _I64, _I64, _I64, _P, _I32, _P, _SZ, _P]),
    "tsvd_csr_gram_apply": (C.c_int, [_I64, _I64, _P, _P, _P, _P, _P, _P, _I32, _P]),
    "tsvd_power_scratch_bytes": (_SZ, [_I64, _I64]),
    "tsvd_power_dense": (C.c_int, [_I64, _P, _P, _P, _P, _I64, _P, _D, _I32, _I32, _I32, _P, _P, _P, _SZ, _P]),
    "tsvd_power_dense_noalloc": (C.c_int, [_I64, _P, _P, _P, _P, _I64, _P, _D, _I32, _I32, _I32, _P, _P, _P]),
    "tsvd_gram_symmetrize": (C.c_int, [_I64, _P, _P, _P]),
    "tsvd_gram_deflate": (C.c_int, [_I64, _P, _P, _P, _P, _P]),
    "tsvd_start_draws": (C.c_int, [C.c_uint64, _I64, _I64, _P, _P]),
    "tsvd_philox4x32_10": (C.c_int, [_P, _P, _P, _I64, _P]),
    "tsvd_left_vectors": (C.c_int, [_P, _I64, _I64, _I64, _P, _I64, _I64, _P, _P, _I64, _P]),
    "tsvd_csr_partition": (C.c_int, [_I64, _P, _I64, _P, C.POINTER(_I64), C.POINTER(_I64)]),
    "tsvd_host_alloc": (C.c_int, [C.POINTER(_P), _SZ]),
    "tsvd_host_free": (C.c_int, [_P]),
    "tsvd_plan_copy_log": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "tsvd_server_options_init": (C.c_int, [C.POINTER(tsvd_server_options)]),
    "tsvd_server_create": (C.c_int, [C.POINTER(_P), C.POINTER(tsvd_server_options)]),
    "tsvd_server_submit": (C.c_int, [_P, _P, _I64, _I64, _I32, _D, _I32, C.c_uint64, _I32, _P, _P, _P, _P,
                                     C.POINTER(C.c_uint64)]),
    "tsvd_server_submit_csr": (C.c_int, [_P, _P, _P, _P, _I64, _I64, _I64, _I32, _D, _I32, C.c_uint64, _I32, _P,
                                         _P, _P, _P, C.POINTER(C.c_uint64)]),
    "tsvd_server_wait": (C.c_int, [_P, C.c_uint64, _D, C.POINTER(tsvd_request_info)]),
    "tsvd_server_get_stats": (C.c_int, [_P, C.POINTER(tsvd_server_stats)]),
    "tsvd_server_last_error": (C.c_char_p, [_P]),
    "tsvd_server_cluster_for": (_I32, [_P, _I64]),
    "tsvd_server_set_cluster_for": (_I32, [_P, _I64, _I32]),
    "tsvd_server_tc_min_d": (C.c_int64, [_P]),
    "tsvd_server_set_tc_min_d": (C.c_int, [_P, C.c_int64]),
    "tsvd_server_autotune_syrk_times": (C.c_int, [_P, _P, _P, _P, _P]),
    "tsvd_server_autotune": (C.c_int, [_P, _I32]),
    "tsvd_server_destroy": (None, [_P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the compiled library (building it in-tree when missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"tsvd CUDA library not built: {path} is missing")
        path = _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TSVDError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.tsvd_status_string(status).decode()
        cuda = lib.tsvd_last_cuda_error().decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})" + (f" [{cuda}]" if cuda else ""))
        self.status = status


def check(status: int, where: str, ok=(TSVD_OK,)) -> int:
    if status not in ok:
        raise TSVDError(status, where)
    return status


def _wrap(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


# module-level functions with the C names
for _name in SIGNATURES:
    globals()[_name] = _wrap(_name)
