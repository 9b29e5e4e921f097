"""Host-side checks of the C ABI: the library loads without a GPU, exports
every symbol the header declares, validates its inputs in tsvd_plan (pure
host work), sizes the device workspace under a budget, and partitions CSR
row blocks exactly.  No compute call runs here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
from paper_2208_08410_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if path.endswith(".h"):
            text = open(os.path.join(ROOT, "include", path)).read()
            names += re.findall(r"TSVD_API[^;(]*?\b(tsvd_\w+)\s*\(", text)
    return names


def test_library_exports_every_declared_symbol(lib):
    names = header_symbols()
    assert len(names) >= 19
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in B.SIGNATURES, f"binding lacks {nm}"


def test_status_strings(lib):
    for s in range(9):
        assert lib.tsvd_status_string(s)
    assert lib.tsvd_status_string(99) == b"unknown status"
    assert lib.tsvd_abi_version() == 1


def _plan(A_desc, k, eps, opt=None):
    h = C.c_void_p()
    ws = C.c_size_t()
    st = B.tsvd_plan(C.byref(h), C.byref(A_desc), k, eps, C.byref(opt) if opt is not None else None, C.byref(ws))
    if st == B.TSVD_OK:
        B.tsvd_destroy(h)
    return st, ws.value


def _dense_desc(m, n, ld=None, arr=None):
    d = B.tsvd_matrix()
    d.kind, d.location, d.m, d.n, d.ld = B.TSVD_DENSE_F32_ROWMAJOR, B.TSVD_HOST, m, n, ld or n
    if arr is None:
        arr = np.zeros((m, ld or n), dtype=np.float32)
    d.values = arr.ctypes.data
    return d, arr


def _opts(**kw):
    o = B.tsvd_options()
    B.tsvd_options_init(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_plan_validation_dense(lib):
    d, keep = _dense_desc(100, 20)
    assert _plan(d, 5, 1e-6)[0] == B.TSVD_OK
    assert _plan(d, -1, 1e-6)[0] == B.TSVD_OK  # k = min(m, n)
    assert _plan(d, 0, 1e-6)[0] == B.TSVD_EINVAL
    assert _plan(d, 21, 1e-6)[0] == B.TSVD_EINVAL
    assert _plan(d, 5, 0.0)[0] == B.TSVD_EINVAL
    assert _plan(d, 5, 1.0)[0] == B.TSVD_EINVAL
    ovr = np.array([3, 3, 3, 3, 3], dtype=np.int32)
    assert _plan(d, 5, 0.0, _opts(iters_override=ovr.ctypes.data))[0] == B.TSVD_OK
    bad = np.array([3, 0, 3, 3, 3], dtype=np.int32)
    assert _plan(d, 5, 1e-6, _opts(iters_override=bad.ctypes.data))[0] == B.TSVD_EINVAL
    assert _plan(d, 5, 1e-6, _opts(precision=7))[0] == B.TSVD_EINVAL
    assert _plan(d, 5, 1e-6, _opts(precision=4))[0] == B.TSVD_EINVAL
    for prec in (B.TSVD_GRAM_FP32, B.TSVD_GRAM_TF32, B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_BF16X3):
        assert _plan(d, 5, 1e-6, _opts(precision=prec))[0] == B.TSVD_OK
    assert _plan(d, 5, 1e-6, _opts(n_buffers=1))[0] == B.TSVD_EINVAL
    d2, keep2 = _dense_desc(100, 20)
    d2.ld = 10
    assert _plan(d2, 5, 1e-6)[0] == B.TSVD_EINVAL
    wide, keep3 = _dense_desc(20, 100)
    assert _plan(wide, 5, 1e-6)[0] == B.TSVD_OK  # m < n: Eq. 3
    assert _plan(wide, 21, 1e-6)[0] == B.TSVD_EINVAL  # k <= min(m, n)
    assert _plan(wide, 5, 1e-6, _opts(gram_tile=256))[0] == B.TSVD_EUNSUPPORTED  # no column panels of a wide A
    d3, keep4 = _dense_desc(100, 20)
    d3.m = 0
    assert _plan(d3, 1, 1e-6)[0] == B.TSVD_EINVAL
    # power-phase kernel choice
    for pk in (B.TSVD_POWER_AUTO, B.TSVD_POWER_GRID, B.TSVD_POWER_CLUSTER):
        assert _plan(d, 5, 1e-6, _opts(power_kernel=pk))[0] == B.TSVD_OK
    assert _plan(d, 5, 1e-6, _opts(power_kernel=3))[0] == B.TSVD_EINVAL
    assert _plan(d, 5, 1e-6, _opts(power_kernel=-1))[0] == B.TSVD_EINVAL
    for c in (0, 1, 2, 4, 8):
        assert _plan(d, 5, 1e-6, _opts(power_ctas=c))[0] == B.TSVD_OK
    for c in (-1, 3, 16):
        assert _plan(d, 5, 1e-6, _opts(power_ctas=c))[0] == B.TSVD_EINVAL
    # the test-only limit of the tensor-core Gram kernel's waits
    assert _plan(d, 5, 1e-6, _opts(wait_limit_ns=1))[0] == B.TSVD_OK
    assert _plan(d, 5, 1e-6, _opts(wait_limit_ns=-1))[0] == B.TSVD_EINVAL
    assert _plan(d, 5, 1e-6, _opts(csr_coop_blocks=64))[0] == B.TSVD_OK
    assert _plan(d, 5, 1e-6, _opts(csr_coop_blocks=-1))[0] == B.TSVD_EINVAL
    big, keep5 = _dense_desc(8, 2049, arr=np.zeros((1, 1), dtype=np.float32))
    big.m = 4096  # plan reads no values
    assert _plan(big, 4, 1e-6, _opts(power_kernel=B.TSVD_POWER_CLUSTER))[0] == B.TSVD_EUNSUPPORTED
    assert _plan(big, 4, 1e-6, _opts(power_kernel=B.TSVD_POWER_AUTO))[0] == B.TSVD_OK
    tall, keep6 = _dense_desc(200, 64)
    assert _plan(tall, 33, 1e-6, _opts(power_kernel=B.TSVD_POWER_CLUSTER))[0] == B.TSVD_EUNSUPPORTED
    assert _plan(tall, 32, 1e-6, _opts(power_kernel=B.TSVD_POWER_CLUSTER))[0] == B.TSVD_OK


def test_plan_orthogonal_batching(lib):
    """Orthogonal batching: forced by gram_tile (a multiple of 256), or taken
    when the whole Gram matrix does not fit the budget; the workspace stays
    within the budget."""
    d, keep = _dense_desc(6000, 1000)
    assert _plan(d, 8, 1e-6, _opts(gram_tile=256))[0] == B.TSVD_OK
    assert _plan(d, 8, 1e-6, _opts(gram_tile=512, precision=B.TSVD_GRAM_TF32X3))[0] == B.TSVD_OK
    for bad in (100, 255, -256):
        assert _plan(d, 8, 1e-6, _opts(gram_tile=bad))[0] == B.TSVD_EINVAL
    # n = 4096: G64 + G32 alone are 201 MB; 64 MB forces the tiles, 2 MB is too little for anything
    big, keep2 = _dense_desc(8, 4096, arr=np.zeros((1, 1), dtype=np.float32))
    big.m = 100000
    st, ws = _plan(big, 16, 1e-6, _opts(device_budget=64 << 20))
    assert st == B.TSVD_OK and ws <= 64 << 20
    st, ws = _plan(big, 16, 1e-6, _opts(device_budget=64 << 20, precision=B.TSVD_GRAM_BF16X3))
    assert st == B.TSVD_OK and ws <= 64 << 20
    assert _plan(big, 16, 1e-6, _opts(device_budget=2 << 20))[0] == B.TSVD_EBUDGET
    # CSR takes no column panels
    c = B.tsvd_matrix()
    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    va = np.ones(2, dtype=np.float32)
    c.kind, c.location, c.m, c.n, c.nnz = B.TSVD_CSR_F32_I32_I64, B.TSVD_HOST, 2, 2, 2
    c.values, c.row_ptr, c.col_idx = va.ctypes.data, rp.ctypes.data, ci.ctypes.data
    assert _plan(c, 1, 1e-6, _opts(gram_tile=256))[0] == B.TSVD_EINVAL


def test_plan_budget_and_streaming_layout(lib):
    m, n, k = 1 << 16, 512, 8
    d, keep = _dense_desc(m, n)
    st, ws_res = _plan(d, k, 1e-6)
    assert st == B.TSVD_OK and ws_res >= m * n * 4  # resident: A copied once
    st, ws_cap = _plan(d, k, 1e-6, _opts(device_budget=48 << 20))
    assert st == B.TSVD_OK and ws_cap <= 48 << 20  # streamed under the cap
    st, _ = _plan(d, k, 1e-6, _opts(device_budget=1 << 20))
    assert st == B.TSVD_EBUDGET


def test_memory_model_avoids_the_residual(lib):
    # Sec. III worked example scaled down: a sparse A whose dense residual
    # would be huge plans a workspace of O(n k + nnz), never O(m n).
    csr = synth.csr_uniform(1 << 17, 1 << 17, 4.0, seed=0)
    d = B.tsvd_matrix()
    d.kind, d.location, d.m, d.n = B.TSVD_CSR_F32_I32_I64, B.TSVD_HOST, csr["m"], csr["n"]
    d.row_ptr, d.col_idx, d.values = (csr["row_ptr"].ctypes.data, csr["col_idx"].ctypes.data,
                                      csr["values"].ctypes.data)
    d.nnz = csr["values"].shape[0]
    st, ws = _plan(d, 8, 1e-6)
    assert st == B.TSVD_OK
    dense_residual = csr["m"] * csr["n"] * 4
    assert ws < dense_residual / 1000
    assert ws < 64 * (csr["n"] * 8 + d.nnz * 8)


def _csr_desc(csr):
    d = B.tsvd_matrix()
    d.kind, d.location, d.m, d.n = B.TSVD_CSR_F32_I32_I64, B.TSVD_HOST, csr["m"], csr["n"]
    d.row_ptr, d.col_idx, d.values = (csr["row_ptr"].ctypes.data, csr["col_idx"].ctypes.data,
                                      csr["values"].ctypes.data)
    d.nnz = csr["values"].shape[0]
    return d


def test_plan_rejects_invalid_csr(lib):
    csr = synth.csr_uniform(500, 300, 5.0, seed=1)
    assert _plan(_csr_desc(csr), 4, 1e-6)[0] == B.TSVD_OK
    bad = dict(csr)
    bad["col_idx"] = csr["col_idx"].copy()
    bad["col_idx"][17] = 300  # out of range
    assert _plan(_csr_desc(bad), 4, 1e-6)[0] == B.TSVD_EINVAL
    bad = dict(csr)
    bad["row_ptr"] = csr["row_ptr"].copy()
    bad["row_ptr"][10], bad["row_ptr"][11] = bad["row_ptr"][11] + 1, bad["row_ptr"][10]  # non-monotone
    assert _plan(_csr_desc(bad), 4, 1e-6)[0] == B.TSVD_EINVAL
    bad = dict(csr)
    d = _csr_desc(bad)
    d.nnz = d.nnz - 1  # row_ptr[m] != nnz
    assert _plan(d, 4, 1e-6)[0] == B.TSVD_EINVAL


@pytest.mark.parametrize("block_rows", [1, 7, 128, 1000, 4096])
def test_csr_partition_is_bit_exact(lib, block_rows):
    csr = synth.csr_uniform(3001, 2000, 9.0, seed=2)
    m = csr["m"]
    rp = csr["row_ptr"]
    starts = np.zeros(m // block_rows + 2, dtype=np.int64)
    nb = C.c_int64()
    mx = C.c_int64()
    assert B.tsvd_csr_partition(m, rp.ctypes.data, block_rows, starts.ctypes.data, C.byref(nb), C.byref(mx)) == 0
    nb = nb.value
    starts = starts[:nb + 1]
    assert starts[0] == 0 and starts[-1] == m and np.all(np.diff(starts) > 0)
    assert np.all(np.diff(starts)[:-1] == block_rows)
    # concatenating the blocks reproduces the arrays byte for byte
    cols, vals, rebased = [], [], []
    biggest = 0
    for b in range(nb):
        r0, r1 = starts[b], starts[b + 1]
        e0, e1 = rp[r0], rp[r1]
        cols.append(csr["col_idx"][e0:e1])
        vals.append(csr["values"][e0:e1])
        brp = rp[r0:r1 + 1] - rp[r0]
        assert np.array_equal(brp, rp[r0:r1 + 1] - e0)  # block_row_ptr[i] = row_ptr[r0+i] - row_ptr[r0]
        rebased.append(brp[:-1] + e0)
        biggest = max(biggest, e1 - e0)
    assert np.concatenate(cols).tobytes() == csr["col_idx"].tobytes()
    assert np.concatenate(vals).tobytes() == csr["values"].tobytes()
    assert np.array_equal(np.concatenate(rebased + [rp[-1:]]), rp)
    assert mx.value == biggest


def test_loader_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2208_08410_gb300 import build as bld
    monkeypatch.setattr(bld, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        B.load(build_if_missing=False)


def test_gram_scratch_sizes(lib):
    """Tensor-core scratch: a status word, then one (TF32) or two parts of the
    K-major copy At (n x Kp); Kp is rows rounded up to a stage of 128 bytes of
    K (32 FP32 or 64 BF16 rows); each part is 1024-byte aligned."""
    rows, n = 1000, 300

    def up(x, q):
        return -(-x // q) * q
    assert B.tsvd_gram_scratch_bytes(rows, n, B.TSVD_GRAM_FP32) == 0
    assert B.tsvd_gram_scratch_bytes(rows, n, B.TSVD_GRAM_TF32) == 2048 + up(n * up(rows, 32) * 4, 1024)
    assert B.tsvd_gram_scratch_bytes(rows, n, B.TSVD_GRAM_TF32X3) == 2048 + 2 * up(n * up(rows, 32) * 4, 1024)
    assert B.tsvd_gram_scratch_bytes(rows, n, B.TSVD_GRAM_BF16X3) == 2048 + 2 * up(n * up(rows, 64) * 2, 1024)
    assert B.tsvd_gram_scratch_bytes(0, n, B.TSVD_GRAM_BF16X3) == 0


def test_server_options_validation(lib):
    """Option checks happen before any device call, so they run without a GPU."""
    opt = B.tsvd_server_options()
    assert B.tsvd_server_options_init(C.byref(opt)) == B.TSVD_OK
    assert opt.max_inflight > 0 and opt.n_streams > 0 and opt.max_wave > 0 and opt.cluster_cap == 8
    h = C.c_void_p()
    for field, bad in (("cluster_cap", 3), ("n_streams", 65), ("max_wave", -1), ("max_inflight", -5)):
        o = B.tsvd_server_options()
        B.tsvd_server_options_init(C.byref(o))
        setattr(o, field, bad)
        assert B.tsvd_server_create(C.byref(h), C.byref(o)) == B.TSVD_EINVAL, field
    assert B.tsvd_server_submit(None, None, 10, 10, 1, 1e-6, 10, 0, 0, None, None, None, None, None) == B.TSVD_EINVAL
    assert B.tsvd_server_cluster_for(None, 100) == 0


def test_binding_constants_match_the_header():
    """Every #define and enum value the binding copies from include/tsvd.h
    has the header's value (the no-allocation limits, flags, kernel choices,
    status codes), so a change to the header cannot drift from Python."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "tsvd.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(TSVD_\w+)\s+(-?\d+)\b", hdr)}
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(TSVD_\w+)\s*=\s*(-?\d+)", hdr)}
    named = dict(defines, **enums)
    checked = 0
    for name, value in named.items():
        if hasattr(B, name):
            assert getattr(B, name) == value, name
            checked += 1
    for must in ("TSVD_NOALLOC_MAX_N", "TSVD_NOALLOC_MAX_L", "TSVD_FLAG_TIMEOUT", "TSVD_POWER_CLUSTER",
                 "TSVD_ETIMEDOUT", "TSVD_GRAM_BF16X3"):
        assert must in named and hasattr(B, must), must
    assert checked >= 20, checked



def test_copy_log_arguments():
    """tsvd_plan_copy_log: a fresh plan has recorded no copies; NULL plan or
    count and a negative capacity are TSVD_EINVAL."""
    d, keep = _dense_desc(100, 20)
    h = C.c_void_p()
    ws = C.c_size_t()
    assert B.tsvd_plan(C.byref(h), C.byref(d), 5, 1e-6, None, C.byref(ws)) == B.TSVD_OK
    lib = B.load()
    try:
        cnt = C.c_int64(-1)
        assert lib.tsvd_plan_copy_log(h, None, None, None, 0, C.byref(cnt)) == B.TSVD_OK and cnt.value == 0
        assert lib.tsvd_plan_copy_log(h, None, None, None, -1, C.byref(cnt)) == B.TSVD_EINVAL
        assert lib.tsvd_plan_copy_log(h, None, None, None, 0, None) == B.TSVD_EINVAL
        assert lib.tsvd_plan_copy_log(None, None, None, None, 0, C.byref(cnt)) == B.TSVD_EINVAL
    finally:
        lib.tsvd_destroy(h)


def _header_structs(hdr):
    """name -> [(field, C type, is pointer, count)] for every typedef struct
    with a body in the header (comments stripped; one declaration may name
    several fields; arrays carry their length)."""
    import re
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(\w+);", hdr, re.S):
        body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            mm = re.match(r"(?:const\s+)?(\w+)\s*(\**)\s*(.+)$", decl)
            assert mm, decl
            ctype, stars, names = mm.group(1), mm.group(2), mm.group(3)
            for nm in names.split(","):
                nm = nm.strip()
                ptr = bool(stars) or nm.startswith("*")
                nm = nm.lstrip("* ")
                count = 1
                arr = re.match(r"(\w+)\s*\[(\d+)\]$", nm)
                if arr:
                    nm, count = arr.group(1), int(arr.group(2))
                fields.append((nm, ctype, ptr, count))
        out[m.group(2)] = fields
    return out


def test_binding_structs_match_the_header():
    """Every struct the binding mirrors has the header's fields, in the
    header's order, each of the header's size (pointers 8 bytes, the fixed-
    width integers and double by their width), and the same total size, so a
    field added to or moved in include/tsvd.h cannot shift the ones after it
    on the Python side."""
    import ctypes as C
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "tsvd.h")).read()
    size = {"int32_t": 4, "uint32_t": 4, "int64_t": 8, "uint64_t": 8, "double": 8, "size_t": 8, "float": 4}
    structs = _header_structs(hdr)
    checked = 0
    for name, fields in structs.items():
        cls = getattr(B, name, None)
        if cls is None:
            continue
        py = cls._fields_
        assert [f[0] for f in py] == [f[0] for f in fields], name
        offset = 0
        for (fname, ftype), (hname, ctype, ptr, count) in zip(py, fields):
            want = (8 if ptr else size[ctype]) * count
            assert C.sizeof(ftype) == want, (name, fname, C.sizeof(ftype), want)
            align = 8 if ptr else size[ctype]
            offset = (offset + align - 1) // align * align + want
        assert C.sizeof(cls) == (offset + 7) // 8 * 8, name
        checked += 1
    assert checked >= 6, sorted(structs)
