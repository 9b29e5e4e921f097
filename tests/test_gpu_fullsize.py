"""Parity at full size, in the launch configurations the benchmark times.

Mixed precision: m = 2^20, n = 8192 stacked-orthogonal A with a harmonic
spectrum and the clustered pair sigma_10 - sigma_11 = 1e-3, k = 32,
eps = 1e-8, A resident on the device, every Gram precision.  Its Gram is
exactly 128 M^T M (the generator's identity), so here the oracle runs the
whole method at full size and the GPU follows its trajectory.

Dense: m x 4096 FP32 (13,107,200 rows when the device holds them, else the
largest multiple of 262,144 that fits), rank 64 with sigma_i = 1/(1+i) plus
1e-4 N(0,1) noise, k = 16, eps = 1e-6, A resident on the device, Gram in
3xTF32.  Sparse: m = n = 2^25 CSR with ~33.5 entries per row, k = 16,
streamed from pinned host memory in row blocks of 2^20 rows under a 4 GB
device budget, 10 operator applications per triplet.

At these sizes the oracle cannot run the whole method, so the checks are on
outputs it computes one by one, in FP64 on the host:
- sampled Gram entries (48 columns over all rows) against the oracle's Gram of
  those columns;
- sigma_l = ||A v_l|| (Alg. 1) for the library's v_l;
- rows of U against (A v_l)_r / sigma_l;
- one CSR row block's operator application (w and ||A_b v||^2) against the C
  oracle, every entry of w;
- the CSR row-block partition, bit-exact.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import tsvd_ref as ref
from oracle.csr_c import csr_gram_apply as oracle_csr_apply
from paper_2208_08410_gb300 import Plan, _binding as B
from clustered_checks import check_clustered

pytestmark = pytest.mark.gpu

N = 4096
RANK = 64
K = 16
EPS = 1e-6
BLOCK_ROWS = 262_144
FULL_M = 13_107_200


def _dense_rows() -> int:
    free, _ = torch.cuda.mem_get_info()
    blocks = (free - 48 * 2 ** 30) // (BLOCK_ROWS * N * 4)
    return int(max(1, min(FULL_M // BLOCK_ROWS, blocks)) * BLOCK_ROWS)


def _pinned(count: int, dtype):
    ptr = C.c_void_p()
    nbytes = max(count * np.dtype(dtype).itemsize, 16)
    B.check(B.tsvd_host_alloc(C.byref(ptr), nbytes), "tsvd_host_alloc")
    ctype = {np.float32: C.c_float, np.int32: C.c_int32, np.int64: C.c_int64}[dtype]
    return ptr, np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,))


def test_dense_full_size_in_core():
    B.load()
    m = _dense_rows()
    dA = torch.empty((m, N), dtype=torch.float32, device="cuda")
    sigma_p = 1.0 / (1.0 + np.arange(RANK))
    synth.dense_lowrank_blocks_torch(dA, m, N, RANK, sigma_p, 1e-4, seed=0, block_rows=BLOCK_ROWS)
    torch.cuda.empty_cache()

    plan = Plan(dA, K, EPS, precision=B.TSVD_GRAM_TF32X3, out_device=True)
    res = plan.factor(dA)
    torch.cuda.synchronize()
    assert res.status == B.TSVD_OK and res.report["flags"] == 0, res.report
    chunk = -(-m // res.report["n_blocks"])  # rows per Gram launch in this plan
    plan.close()
    del plan
    torch.cuda.empty_cache()

    # ---- sampled Gram entries, accumulated chunk by chunk like the plan
    rng = np.random.default_rng(11)
    cols = np.sort(rng.choice(N, size=48, replace=False))
    G = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    sb = B.tsvd_gram_scratch_bytes(chunk, N, B.TSVD_GRAM_TF32X3)
    scr = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for r0 in range(0, m, chunk):
        rows = min(chunk, m - r0)
        B.check(B.tsvd_gram_accumulate(dA[r0:].data_ptr(), rows, N, N, G.data_ptr(), B.TSVD_GRAM_TF32X3,
                                       scr.data_ptr(), sb, stream), "tsvd_gram_accumulate")
    torch.cuda.synchronize()
    assert int(scr[:4].view(torch.int32).item()) == 0
    Gs = G[torch.as_tensor(cols, device="cuda")][:, torch.as_tensor(cols, device="cuda")].cpu().numpy()
    del G, scr
    torch.cuda.empty_cache()
    Ac = dA[:, torch.as_tensor(cols, device="cuda")].cpu().numpy().astype(np.float64)
    Gref = ref.gram(Ac)
    absG = np.abs(Ac).T @ np.abs(Ac)
    del Ac
    # The library keeps the upper triangle (row j <= column i).  3xTF32 split
    # error 3 * 2^-22; each TMEM segment (2 stages of 32 rows, 3 MMAs of K = 8
    # per 8 rows) chains at most 24 truncating FP32 additions; segment sums are
    # added with round-to-nearest in registers, at most chunk/64 + 1 of them;
    # work units are summed in FP64.
    e = 3 * 2.0 ** -22 + 24 * 2.0 ** -23 + (chunk // 64 + 1) * 2.0 ** -24
    iu = np.triu_indices(48)
    Gu = np.where(np.arange(48)[:, None] <= np.arange(48)[None, :], Gs, Gs.T)
    ratio = np.abs(Gu[iu] - Gref[iu]) / (e * absG[iu])
    assert float(ratio.max()) <= 1.0, float(ratio.max())

    # ---- sigma_l = ||A v_l|| and sampled rows of U, FP64 over all rows
    V = res.V.cpu().numpy().astype(np.float64)  # n x k
    sig = res.sigma.cpu().numpy()
    U = res.U  # (m, k) view on the device
    sample = np.sort(rng.choice(m, size=4096, replace=False))
    AV2 = np.zeros(K)
    u_ref = np.zeros((sample.size, K))
    u_bound = np.zeros((sample.size, K))
    absV = np.abs(V)
    for r0 in range(0, m, BLOCK_ROWS):
        r1 = min(m, r0 + BLOCK_ROWS)
        blk = dA[r0:r1].cpu().numpy().astype(np.float64)
        AVb = blk @ V
        AV2 += np.sum(AVb ** 2, axis=0)
        sel = (sample >= r0) & (sample < r1)
        if sel.any():
            rows = sample[sel] - r0
            u_ref[sel] = AVb[rows]
            u_bound[sel] = np.abs(blk[rows]) @ absV
        del blk, AVb
    sig_ref = np.sqrt(AV2)
    rel = np.abs(sig - sig_ref) / sig_ref
    assert float(rel.max()) <= 1e-5, rel
    Ug = U[torch.as_tensor(sample, device="cuda")].cpu().numpy().astype(np.float64)
    # U = A V / sigma with FP32 dot products of length n, scaled by the library's sigma
    u_exp = u_ref / sig[None, :]
    bound = (N + 2) * 2.0 ** -24 * u_bound / sig[None, :] + 2.0 ** -23 * np.abs(u_exp) + 1e-30
    assert np.all(np.abs(Ug - u_exp) <= bound), float(np.max(np.abs(Ug - u_exp) / bound))
    del dA, res, U
    torch.cuda.empty_cache()


C2S_M = 1_048_576          # the out-of-core configuration's small case: 16 GiB of FP32
C2S_BUDGET = 8_000_000_000  # device budget that forces streaming


def test_c2_small_streamed_follows_oracle():
    """The dense out-of-core configuration at m = 1,048,576, n = 4096: A (16 GiB)
    in page-locked host memory, streamed in row blocks under an 8 GB device
    budget, Gram in 3xTF32, k = 16, eps = 1e-6.  The oracle forms the FP64 Gram
    of the same stored values block by block (Alg. 2 B = X^T X over row
    batches, Sec. V-C), runs O-1 (Alg. 1/2, Hotelling deflation) from the same
    start draws with its own convergence test, and forms U = A V Sigma^-1;
    the GPU follows with the oracle's iteration counts forced.  sigma within
    1e-5 on every triplet; u_l and v_l within 1e-4 on the gapped triplets."""
    B.load()
    m = C2S_M
    ptr, flat = _pinned(m * N, np.float32)
    try:
        A = flat.reshape(m, N)
        sigma_p = 1.0 / (1.0 + np.arange(RANK))
        synth.dense_lowrank_blocks_torch(torch.from_numpy(A), m, N, RANK, sigma_p, 1e-4, seed=2,
                                         block_rows=BLOCK_ROWS)
        x = synth.start_normals(N, K, seed=3)
        G = ref.gram_row_blocks(A, 65536)
        sig_o, V_o, it_o, st_o = ref.right_vectors(G, K, EPS, x_start=x)
        assert all(s == "ok" for s in st_o), st_o
        lam = np.linalg.eigvalsh(G)[::-1]
        del G
        # noise Gram ~ m 1e-8 I = 0.0105 I: the relative gaps fall below 0.05 near i = 12
        gapped = ref.gapped_indices(lam, K)
        assert gapped[:11] == list(range(11)), gapped
        U_o = np.empty((m, K))
        for r0 in range(0, m, 65536):
            U_o[r0:r0 + 65536] = np.asarray(A[r0:r0 + 65536], dtype=np.float64) @ V_o
        U_o /= sig_o[None, :]

        plan = Plan(A, K, EPS, precision=B.TSVD_GRAM_TF32X3, device_budget=C2S_BUDGET, force_stream=True,
                    start_draws=x, iters_override=it_o)
        try:
            res = plan.factor()
        finally:
            plan.close()
        assert res.status == B.TSVD_OK and res.report["flags"] == 0, res.report
        assert res.report["mode"] == 2 and res.report["n_blocks"] >= 2, res.report
        assert res.iters == it_o
        rel = np.abs(np.asarray(res.sigma) - sig_o) / sig_o
        assert float(rel.max()) <= 1e-5, rel
        V = np.asarray(res.V, dtype=np.float64)
        U = np.asarray(res.U, dtype=np.float64)
        for l in gapped:
            assert ref.vector_angle(V[:, l], V_o[:, l]) <= 1e-4, (l, ref.vector_angle(V[:, l], V_o[:, l]))
            assert ref.vector_angle(U[:, l], U_o[:, l]) <= 1e-4, (l, ref.vector_angle(U[:, l], U_o[:, l]))
    finally:
        B.tsvd_host_free(ptr)


def test_csr_full_size_streamed():
    B.load()
    m = 1 << 25
    dcsr = synth.csr_uniform_torch(m, m, 33.5, seed=1)
    nnz = int(dcsr["values"].shape[0])
    p_rp, rp = _pinned(m + 1, np.int64)
    p_ci, ci = _pinned(nnz, np.int32)
    p_va, va = _pinned(nnz, np.float32)
    try:
        rp[:] = dcsr["row_ptr"].cpu().numpy()
        ci[:] = dcsr["col_idx"].cpu().numpy()
        va[:] = dcsr["values"].cpu().numpy()
        host = {"row_ptr": rp, "col_idx": ci, "values": va, "m": m, "n": m}

        # ---- partition into 2^20-row blocks, bit-exact
        bl = 1 << 20
        nb = -(-m // bl)
        starts = np.zeros(nb + 1, dtype=np.int64)
        nbo = C.c_int64()
        mx = C.c_int64()
        B.check(B.tsvd_csr_partition(m, rp.ctypes.data, bl, starts.ctypes.data, C.byref(nbo), C.byref(mx)),
                "tsvd_csr_partition")
        expect = np.minimum(np.arange(nb + 1, dtype=np.int64) * bl, m)
        assert nbo.value == nb and np.array_equal(starts, expect)
        assert mx.value == int(np.max(rp[expect[1:]] - rp[expect[:-1]]))

        # ---- one row block's application against the C oracle, all of w
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        v = torch.rand(m, generator=gen, device="cuda", dtype=torch.float32)
        w = torch.zeros(m, dtype=torch.float32, device="cuda")
        ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        r0 = (m // 2) // bl * bl
        r1 = r0 + bl
        p0 = int(rp[r0])
        drp, dci, dva = dcsr["row_ptr"], dcsr["col_idx"], dcsr["values"]
        B.check(B.tsvd_csr_gram_apply(r1 - r0, m, drp[r0:].data_ptr(), dci[p0:].data_ptr(), dva[p0:].data_ptr(),
                                      v.data_ptr(), w.data_ptr(), ss.data_ptr(), 1,
                                      torch.cuda.current_stream().cuda_stream), "tsvd_csr_gram_apply")
        torch.cuda.synchronize()
        vh = v.cpu().numpy().astype(np.float64)
        w_ref, ss_ref = oracle_csr_apply(rp, ci, va, vh, r0=r0, r1=r1)
        wd = w.cpu().numpy().astype(np.float64)
        # all values and v are positive, so |A|^T |A| |v| is the oracle's w itself.
        # y_r: FP32 sum of len_r products (<= len_r + 1 roundings); w_c: one product
        # and one atomic addition per entry of column c in the block.
        p1 = int(rp[r1])
        maxlen = int(np.max(np.diff(rp[r0:r1 + 1])))
        cnt = np.bincount(ci[p0:p1], minlength=m)
        bound = (maxlen + 1 + 2 * cnt + 2) * 2.0 ** -24 * w_ref + 1e-30
        assert np.all(np.abs(wd - w_ref) <= bound), float(np.max(np.abs(wd - w_ref) / bound))
        assert abs(float(ss.item()) - ss_ref) <= 1e-5 * ss_ref
        del dcsr, drp, dci, dva, v, w
        torch.cuda.empty_cache()

        # ---- the streamed t-SVD; sigma_l = ||A v_l|| and u_l = A v_l / sigma_l
        plan = Plan(host, K, EPS, iters_override=[10] * K, device_budget=4 * 10 ** 9, block_rows=bl,
                    force_stream=True)
        res = plan.factor(host)
        assert res.report["mode"] == 2 and res.report["n_blocks"] == nb
        plan.close()
        rows_of = ref.csr_row_index(rp)
        lens = np.diff(rp).astype(np.float64)
        for l in (0, K - 1):
            vl = res.V[:, l].astype(np.float64)
            y = ref.csr_matvec(rp, ci, va, vl, rows_of=rows_of)
            s_ref = float(np.sqrt(np.dot(y, y)))
            assert abs(res.sigma[l] - s_ref) <= 1e-5 * s_ref, (l, res.sigma[l], s_ref)
            absy = ref.csr_matvec(rp, ci, np.abs(va), np.abs(vl), rows_of=rows_of)
            u_exp = y / res.sigma[l]
            ub = (lens + 2) * 2.0 ** -24 * absy / res.sigma[l] + 2.0 ** -23 * np.abs(u_exp) + 1e-30
            ug = res.U[:, l].astype(np.float64)
            assert np.all(np.abs(ug - u_exp) <= ub), (l, float(np.max(np.abs(ug - u_exp) / ub)))
            del y, absy, u_exp, ub
    finally:
        for p in (p_rp, p_ci, p_va):
            B.tsvd_host_free(p)


C4_N, C4_COPIES, C4_K, C4_EPS = 8192, 128, 32, 1e-8


@pytest.fixture(scope="module")
def c4():
    sig_t = synth.spectrum_harmonic_clustered(C4_N, 10, 1e-3)
    fac = synth.stacked_factor(C4_N, sig_t, C4_COPIES, seed=0)
    G = C4_COPIES * ref.gram(fac["M32"])  # = A^T A of the stacked matrix, FP64
    x = synth.start_normals(C4_N, C4_K, seed=3)
    sig_o, V_o, it_o, st_o = ref.right_vectors(G, C4_K, C4_EPS, x_start=x)
    assert all(st == "ok" for st in st_o)
    del G
    dA = torch.empty((C4_N * C4_COPIES, C4_N), dtype=torch.float32, device="cuda")
    synth.stacked_rows_torch(dA, fac["M32"], seed=0)
    yield {"sig_t": sig_t, "x": x, "sig_o": sig_o, "V_o": V_o, "it_o": it_o, "A": dA}
    del dA
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [B.TSVD_GRAM_FP32, B.TSVD_GRAM_TF32, B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_BF16X3])
def test_clustered_spectrum_full_size(c4, prec):
    B.load()
    dA = c4["A"]
    r = Plan(dA, C4_K, C4_EPS, start_draws=c4["x"], iters_override=c4["it_o"], precision=prec,
             out_device=True).factor(dA)
    assert r.iters == c4["it_o"]
    sig = r.sigma.cpu().numpy()
    V = r.V.cpu().numpy()
    r.sigma, r.V = sig, V
    check_clustered(r, c4["sig_o"], c4["V_o"], C4_K, prec, c4["sig_t"])
    # rows of U against (A_r v_l) / sigma_l in FP64
    rng = np.random.default_rng(prec)
    rows = np.sort(rng.choice(dA.shape[0], size=1024, replace=False))
    Ar = dA[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    Vd = V.astype(np.float64)
    u_exp = (Ar @ Vd) / sig[None, :]
    bound = (C4_N + 2) * 2.0 ** -24 * (np.abs(Ar) @ np.abs(Vd)) / sig[None, :] + 2.0 ** -23 * np.abs(u_exp)
    Ug = r.U[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Ug - u_exp) <= bound + 1e-30)
