"""GPU parity: every step of the CUDA path against the FP64 oracle on the
same seeded inputs, called through the C ABI.

Tolerances are derived from the arithmetic:
  * Gram (FP32 CUDA cores): each slice sums at most K products in FP32 before
    the FP64 add, so |dG_ij| <= (K+2) u32 (|A|^T |A|)_ij  (u32 = 2^-24).
  * Power iteration on G32 = fp32(G) with FP32 products and FP64 sums: the
    iterate follows the oracle's to ~1e-6; sigma^2 comes from FP64 G.
  * Whole t-SVD: sigma relative error <= 1e-5 and angle <= 1e-4 for gapped
    triplets (relative eigen-gap >= 0.05), compared on the same trajectory
    (same start draws, the oracle's iteration counts forced).
"""
import ctypes as C
import math
import os

import numpy as np
import pytest

import synth
from oracle import philox
from oracle import tsvd_ref as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2208_08410_gb300 import _binding as B  # noqa: E402
from paper_2208_08410_gb300 import tsvd  # noqa: E402
from clustered_checks import check_clustered  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U32 = 2.0 ** -24


def S():
    return torch.cuda.current_stream().cuda_stream


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.load()


# ---------------------------------------------------------------- a7 start vectors
def test_philox_matches_known_answers_and_oracle():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    rng = np.random.default_rng(0)
    extra = rng.integers(0, 2 ** 32, size=(1000, 6), dtype=np.uint64)
    ctr = np.array([r[0:4] for r in rows] + extra[:, :4].tolist(), dtype=np.uint32)
    key = np.array([r[4:6] for r in rows] + extra[:, 4:6].tolist(), dtype=np.uint32)
    d_ctr, d_key = dev(ctr.view(np.int32)), dev(key.view(np.int32))
    d_out = torch.empty_like(d_ctr)
    assert B.tsvd_philox4x32_10(d_ctr.data_ptr(), d_key.data_ptr(), d_out.data_ptr(), ctr.shape[0], S()) == 0
    got = d_out.cpu().numpy().view(np.uint32)
    assert [list(map(int, g)) for g in got[:3]] == [r[6:10] for r in rows]
    want = philox.philox4x32_10(ctr, key)
    assert np.array_equal(got, want)  # bit-exact


@pytest.mark.parametrize("n", [1, 2, 257, 100001])
def test_start_draws_match_oracle(n):
    for seed, l in [(0, 0), (12345, 7)]:
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        assert B.tsvd_start_draws(seed, l, n, x.data_ptr(), S()) == 0
        want = philox.start_normals(seed, l, n)
        assert np.max(np.abs(x.cpu().numpy() - want)) < 1e-13


# ---------------------------------------------------------------- a2 Gram
@pytest.mark.parametrize("rows,n,ld", [(1000, 256, 256), (777, 130, 130), (64, 5, 5), (5000, 300, 300),
                                       (300, 129, 133), (1, 17, 17), (0, 40, 40)])
def test_gram_fp32_matches_oracle(rows, n, ld):
    rng = np.random.default_rng(rows + n)
    Afull = rng.standard_normal((max(rows, 1), ld)).astype(np.float32)[:rows]
    A = Afull[:, :n]
    sentinel = -7.25
    G = np.triu(np.zeros((n, n))) + np.tril(np.full((n, n), sentinel), -1)
    dG = dev(G)
    dA = dev(Afull) if rows else torch.empty(1, dtype=torch.float32, device="cuda")
    assert B.tsvd_gram_accumulate(dA.data_ptr(), rows, n, ld, dG.data_ptr(), B.TSVD_GRAM_FP32, None, 0, S()) == 0
    # accumulate a second time: G must double (+= semantics)
    assert B.tsvd_gram_accumulate(dA.data_ptr(), rows, n, ld, dG.data_ptr(), B.TSVD_GRAM_FP32, None, 0, S()) == 0
    got = dG.cpu().numpy()
    ref_G = 2.0 * ref.gram(A)
    absA = np.abs(A.astype(np.float64))
    bound = 2.0 * (rows + 2) * U32 * (absA.T @ absA) + 1e-300
    iu = np.triu_indices(n)
    err = np.abs(got[iu] - ref_G[iu])
    assert np.all(err <= bound[iu])
    il = np.tril_indices(n, -1)
    assert np.all(got[il] == sentinel)  # strict lower triangle untouched
    if rows >= 100:
        rel = err / np.maximum(bound[iu] / ((rows + 2) * U32), 1e-300)
        assert np.sqrt(np.mean(rel ** 2)) < 8 * math.sqrt(rows) * U32


def test_symmetrize_is_exact():
    rng = np.random.default_rng(3)
    n = 301
    G = rng.standard_normal((n, n))
    G = G + G.T
    dG = dev(np.triu(G))
    d32 = torch.empty((n, n), dtype=torch.float32, device="cuda")
    assert B.tsvd_gram_symmetrize(n, dG.data_ptr(), d32.data_ptr(), S()) == 0
    assert np.array_equal(d32.cpu().numpy(), G.astype(np.float32))


# ---------------------------------------------------------------- a4/a5 power step
def _power_case(n=256, m=2048, l=3, seed=0):
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=seed)
    Gf = ref.gram(inp["A"])
    prior = ref.tsvd_dense(inp["A"], l, 1e-12, x_start=synth.start_normals(n, l, seed=9), B=Gf)
    return Gf, prior


@pytest.mark.parametrize("l", [0, 3])
def test_power_dense_follows_oracle(l):
    n = 256
    Gf, prior = _power_case(n=n, l=max(l, 1))
    V = prior.V[:, :l]
    s2 = prior.sigma[:l] ** 2
    x = synth.start_normals(n, 1, seed=21)[:, 0]
    v0 = x / np.linalg.norm(x)
    res = ref.power_method(ref.hotelling_apply(Gf, V, s2), v0, 1e-8)
    dG64, dG32 = dev(Gf), dev(Gf.astype(np.float32))
    dV = dev(np.asfortranarray(V).T.copy()) if l else None  # column-major n x l == row-major l x n
    ds2 = dev(s2) if l else None
    for j in range(l):  # Hotelling deflation in FP64, FP32 copy rounded from it, one triplet at a time
        assert B.tsvd_gram_deflate(n, dG64.data_ptr(), dG32.data_ptr(), dV[j].data_ptr(), ds2[j:].data_ptr(),
                                   S()) == 0
    if l:
        want = Gf - V @ np.diag(s2) @ V.T
        got64 = dG64.cpu().numpy()
        iu = np.triu_indices(n)
        # l FP64 fused multiply-adds per entry
        assert np.max(np.abs(got64[iu] - want[iu])) <= 4 * l * 2.0 ** -53 * np.max(np.abs(Gf))
        il = np.tril_indices(n, -1)
        assert np.array_equal(got64[il], Gf[il])  # the strict lower triangle is not touched
        got32 = dG32.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got32 - want) - 2.0 ** -24 * np.abs(want)) <= 8 * l * 2.0 ** -53 * np.max(np.abs(Gf))
    scratch_b = B.tsvd_power_scratch_bytes(n, l)
    scr = torch.empty(scratch_b, dtype=torch.uint8, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    out_s2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for override in (res.iters, 0):
        dx = dev(x)
        st = B.tsvd_power_dense(n, dG32.data_ptr(), dG64.data_ptr(), dV.data_ptr() if l else None,
                                ds2.data_ptr() if l else None, l, dx.data_ptr(), 1e-8, 10000, override, 0,
                                out_s2.data_ptr(), info.data_ptr(), scr.data_ptr(), scratch_b, S())
        assert st == 0
        torch.cuda.synchronize()
        got = dx.cpu().numpy()
        inf = info.cpu().numpy()
        assert inf[1] == 0 and inf[2] == 0
        if override:
            assert inf[0] == res.iters
        else:
            assert abs(int(inf[0]) - res.iters) <= 1
        assert abs(np.linalg.norm(got) - 1.0) < 1e-12
        assert ref.vector_angle(got, res.v) < 1e-5
        s2_ref = float(res.v @ Gf @ res.v)  # sigma_l^2 = v^T G v with the undeflated G
        assert abs(out_s2.item() - s2_ref) / s2_ref < 1e-6


def test_power_dense_rank_deficient():
    n = 64
    G = np.zeros((n, n))
    dG64, dG32 = dev(G), dev(G.astype(np.float32))
    scr_b = B.tsvd_power_scratch_bytes(n, 0)
    scr = torch.empty(scr_b, dtype=torch.uint8, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    out_s2 = torch.ones(1, dtype=torch.float64, device="cuda")
    x = synth.start_normals(n, 1, seed=2)[:, 0]
    dx = dev(x)
    assert B.tsvd_power_dense(n, dG32.data_ptr(), dG64.data_ptr(), None, None, 0, dx.data_ptr(), 1e-8, 100, 0, 0,
                              out_s2.data_ptr(), info.data_ptr(), scr.data_ptr(), scr_b, S()) == 0
    inf = info.cpu().numpy()
    assert inf[1] == 2 and out_s2.item() == 0.0
    assert ref.vector_angle(dx.cpu().numpy(), x) < 1e-12


# ---------------------------------------------------------------- a6 left vectors
@pytest.mark.parametrize("rows,n,k", [(1000, 300, 20), (37, 64, 3), (513, 256, 16)])
def test_left_vectors_match_oracle(rows, n, k):
    _check_left(rows, n, k)


@pytest.mark.parametrize("form", ["mma", "mma_ws", "mma_ws5", "simt8", "simt4"])
@pytest.mark.parametrize("rows,n,k", [(1000, 300, 20), (4133, 1000, 16), (20000, 4096, 7), (70000, 160, 16)])
def test_left_vectors_every_kernel_form(form, rows, n, k, monkeypatch):
    """The TMA-fed forms: tensor cores with a block barrier per chunk or a
    producer warp and per-stage mbarriers (3xTF32 with the TF32 part rounded by
    integer add and mask and the low part truncated by the tensor core: at
    most ~2.5 * 2^-21 per product, inside the FP32 bound (n + 2) 2^-24 for
    the n >= 64 that takes this path), CUDA cores with 8 or 4 rows
    per warp (TSVD_LEFT_MMA, TSVD_LEFT_RW): many tiles per block, a ragged
    last tile and chunk, k below and above one sweep of 16."""
    monkeypatch.setenv("TSVD_LEFT_MMA", {"mma": "1", "mma_ws": "2", "mma_ws5": "2"}.get(form, "0"))
    monkeypatch.setenv("TSVD_LEFT_STAGES", "5" if form == "mma_ws5" else "4")
    monkeypatch.setenv("TSVD_LEFT_RW", "4" if form == "simt4" else "8")
    _check_left(rows, n, k)


def _check_left(rows, n, k):
    rng = np.random.default_rng(rows)
    A = rng.standard_normal((rows, n)).astype(np.float32)
    V = rng.standard_normal((n, k)).astype(np.float32)
    sig = rng.uniform(0.5, 2.0, size=k)
    sig[k // 2] = 0.0  # a zero sigma gives a zero column
    dA, dV, ds = dev(A), dev(np.asfortranarray(V).T.copy()), dev(sig)
    ldu = rows + 5
    dU = torch.full((k, ldu), 3.0, dtype=torch.float32, device="cuda")
    assert B.tsvd_left_vectors(dA.data_ptr(), rows, n, n, dV.data_ptr(), n, k, ds.data_ptr(), dU.data_ptr(), ldu,
                               S()) == 0
    got = dU.cpu().numpy()[:, :rows].T
    want = (A.astype(np.float64) @ V.astype(np.float64))
    scale = np.abs(A.astype(np.float64)) @ np.abs(V.astype(np.float64))
    for l in range(k):
        if sig[l] == 0:
            assert np.all(got[:, l] == 0)
        else:
            assert np.all(np.abs(got[:, l] - want[:, l] / sig[l]) <= (n + 2) * U32 * scale[:, l] / sig[l] + 1e-30)
    assert np.all(dU.cpu().numpy()[:, rows:] == 3.0)  # padding rows untouched


# ---------------------------------------------------------------- a3 CSR pair
def _csr_with_edge_rows(m, n, seed):
    csr = synth.csr_uniform(m, n, 12.0, seed=seed)
    rows = []
    rp, ci, va = csr["row_ptr"], csr["col_idx"], csr["values"]
    rng = np.random.default_rng(seed)
    for r in range(m):
        c, v = ci[rp[r]:rp[r + 1]], va[rp[r]:rp[r + 1]]
        if r == 3:
            c, v = c[:0], v[:0]                      # empty row
        elif r == 4:
            c, v = c[:1], v[:1]                      # one entry
        elif r == 5:
            c = np.arange(n, dtype=np.int32)         # dense row
            v = rng.random(n, dtype=np.float32)
        elif r == 6:
            p = rng.permutation(c.shape[0])          # unsorted columns
            c, v = c[p], v[p]
        rows.append((c, v))
    rp2 = np.zeros(m + 1, dtype=np.int64)
    rp2[1:] = np.cumsum([c.shape[0] for c, _ in rows])
    return {"row_ptr": rp2, "col_idx": np.concatenate([c for c, _ in rows]).astype(np.int32),
            "values": np.concatenate([v for _, v in rows]).astype(np.float32), "m": m, "n": n}


@pytest.mark.parametrize("scatter", [1, 0])
def test_csr_pair_matches_oracle(scatter):
    m, n = 5000, 3000
    csr = _csr_with_edge_rows(m, n, 7)
    rp, ci, va = csr["row_ptr"], csr["col_idx"], csr["values"]
    v = np.random.default_rng(1).standard_normal(n).astype(np.float32)
    # a middle block: rows [1000, 3500), pointers offset to its first entry
    r0, r1 = 1000, 3500
    for (a, b) in [(0, m), (r0, r1)]:
        e0 = rp[a]
        d_rp = dev(rp[a:b + 1])
        d_ci = dev(ci[e0:rp[b]])
        d_va = dev(va[e0:rp[b]])
        d_v = dev(v)
        d_w = torch.full((n,), 0.5, dtype=torch.float32, device="cuda")
        d_ss = torch.full((1,), 0.25, dtype=torch.float64, device="cuda")
        assert B.tsvd_csr_gram_apply(b - a, n, d_rp.data_ptr(), d_ci.data_ptr(), d_va.data_ptr(), d_v.data_ptr(),
                                     d_w.data_ptr(), d_ss.data_ptr(), scatter, S()) == 0
        torch.cuda.synchronize()
        sub_rp = rp[a:b + 1] - e0
        y = ref.csr_matvec(sub_rp, ci[e0:rp[b]], va[e0:rp[b]], v.astype(np.float64))
        w_ref = ref.csr_rmatvec(sub_rp, ci[e0:rp[b]], va[e0:rp[b]], y, n)
        ss_ref = float(y @ y)
        assert abs(d_ss.item() - 0.25 - ss_ref) <= 1e-5 * ss_ref
        w = d_w.cpu().numpy().astype(np.float64)
        if scatter:
            absy = np.abs(ref.csr_matvec(sub_rp, ci[e0:rp[b]], np.abs(va[e0:rp[b]]), np.abs(v.astype(np.float64))))
            scale = ref.csr_rmatvec(sub_rp, ci[e0:rp[b]], np.abs(va[e0:rp[b]]), absy, n)
            assert np.all(np.abs(w - 0.5 - w_ref) <= 64 * U32 * (scale + 0.5) + 1e-30)
        else:
            assert np.all(w == 0.5)


# ---------------------------------------------------------------- whole t-SVD
def _gapped(sig, k):
    lam = sig ** 2
    return ref.gapped_indices(lam, k)


def _all_gapped(o, k):
    """The graded triplets of a geometric spectrum rho^i (rho <= 0.93 here):
    every relative eigen-gap is 1 - rho^2 >= 0.13 and the 1e-6 noise moves it
    by far less, so all k must be graded; an empty or short set would make the
    vector checks vacuous."""
    g = ref.gapped_indices(o.sigma ** 2, k)
    assert g == list(range(k)), g
    return g


def _compare(res, o, k, angle_tol=1e-4, sig_tol=1e-5, gapped=None):
    sig = np.asarray(res.sigma)
    assert np.max(np.abs(sig - o.sigma) / o.sigma) <= sig_tol, (sig, o.sigma)
    idx = gapped if gapped is not None else range(k)
    for l in idx:
        assert ref.vector_angle(np.asarray(res.V[:, l]), o.V[:, l]) <= angle_tol, l
        assert ref.vector_angle(np.asarray(res.U[:, l]), o.U[:, l]) <= angle_tol, l


@pytest.mark.parametrize("pk", [B.TSVD_POWER_GRID, B.TSVD_POWER_CLUSTER])
@pytest.mark.parametrize("mode", ["device", "resident", "stream"])
def test_tsvd_c1_matches_oracle(mode, pk):
    m, n, k, eps = 2048, 256, 8, 1e-8
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=0)
    A = inp["A"]
    x = synth.start_normals(n, k, seed=1)
    o = ref.tsvd_dense(A, k, eps, x_start=x)
    gapped = _gapped(np.linalg.svd(A.astype(np.float64), compute_uv=False), k)
    assert gapped == list(range(k))
    kw = {}
    if mode == "device":
        Ain = torch.from_numpy(A).cuda()
    else:
        Ain = A
        if mode == "stream":
            kw = dict(force_stream=True, block_rows=300, n_buffers=2)
    kw["power_kernel"] = pk
    # same trajectory: the oracle's iteration counts forced
    r = tsvd(Ain, k, eps, start_draws=x, iters_override=o.iters, **kw)
    assert r.iters == o.iters
    _compare(r, o, k, gapped=gapped)
    # own convergence test
    r2 = tsvd(Ain, k, eps, start_draws=x, **kw)
    assert all(abs(a - b) <= 1 for a, b in zip(r2.iters, o.iters))
    assert np.max(np.abs(r2.sigma - o.sigma) / o.sigma) <= 1e-5
    # orthonormality as far as eps allows (A6: theta ~ sqrt(2 eps) r / (1 - r)),
    # and the same departure from it as the oracle's factors
    V = np.asarray(r.V, dtype=np.float64)
    U = np.asarray(r.U, dtype=np.float64)
    assert np.allclose(V.T @ V, np.eye(k), atol=3e-3)
    assert np.allclose(V.T @ V, o.V.T @ o.V, atol=1e-5)
    assert np.allclose(U.T @ U, o.U.T @ o.U, atol=1e-4)


# m, n, k, rho: odd n (scalar row loads), n not a multiple of 4, n = 512 with k = 32 (rows of the
# FP32 Gram resident in shared memory), n = 2048 (rows read from L2), n = 1000.  sigma_{k-1}/sigma_0
# stays above 0.1: the FP32-accumulated Gram's error, relative to lambda_0, is ~1e-7 on these shapes,
# so sigma_{k-1} moves by ~1e-7 / (2 (sigma_{k-1}/sigma_0)^2), and 1e-5 needs the ratio well above 0.07
POWER_CASES = [(3000, 5, 5, 0.6), (2000, 130, 12, 0.82), (4096, 512, 32, 0.93), (6000, 2048, 8, 0.75),
               (1024, 1000, 16, 0.87)]


@pytest.mark.parametrize("pk", [B.TSVD_POWER_GRID, B.TSVD_POWER_CLUSTER])
@pytest.mark.parametrize("m,n,k,rho", POWER_CASES)
def test_tsvd_power_kernels_match_oracle(pk, m, n, k, rho):
    """Both kernels of the dense power phase follow the oracle's trajectory
    (forced counts, caller start draws, sign convention)."""
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, rho), 1e-7, seed=n)
    x = synth.start_normals(n, k, seed=2)
    o = ref.tsvd_dense(inp["A"], k, 1e-10, x_start=x, sign_convention=True)
    r = tsvd(torch.from_numpy(inp["A"]).cuda(), k, 1e-10, start_draws=x, iters_override=o.iters,
             sign_convention=True, power_kernel=pk)
    assert r.iters == o.iters
    _compare(r, o, k, gapped=_all_gapped(o, k))
    # the sign convention fixes the vectors themselves, not only their span
    for l in _all_gapped(o, k):
        assert np.max(np.abs(np.asarray(r.V[:, l], dtype=np.float64) - o.V[:, l])) < 1e-4


@pytest.mark.parametrize("ctas", [1, 2, 4])
@pytest.mark.parametrize("n", [256, 520])
def test_tsvd_cluster_sizes_follow_oracle(ctas, n):
    """The cluster kernel on 1, 2 or 4 CTAs (Gram rows resident in shared
    memory or read from L2) follows the oracle's trajectory."""
    m, k = 3000, 12
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.82), 1e-7, seed=n + ctas)
    x = synth.start_normals(n, k, seed=3)
    o = ref.tsvd_dense(inp["A"], k, 1e-10, x_start=x, sign_convention=True)
    r = tsvd(torch.from_numpy(inp["A"]).cuda(), k, 1e-10, start_draws=x, iters_override=o.iters,
             sign_convention=True, power_kernel=B.TSVD_POWER_CLUSTER, power_ctas=ctas)
    assert r.report["power_cluster"] == ctas
    assert r.iters == o.iters
    _compare(r, o, k, gapped=_all_gapped(o, k))


@pytest.mark.parametrize("pk", [B.TSVD_POWER_GRID, B.TSVD_POWER_CLUSTER])
@pytest.mark.parametrize("e", [-40, 30])
def test_tsvd_power_kernels_scale_invariant(pk, e):
    """sigma(2^e A) = 2^e sigma(A) and the same vectors: Alg. 2 is invariant
    under scaling A, and the power kernels keep their FP32 sums inside range
    for Gram diagonals from ~1e-24 to ~1e18 (the oracle's trajectory forced)."""
    m, n, k = 2048, 256, 8
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=4)
    x = synth.start_normals(n, k, seed=5)
    o = ref.tsvd_dense(inp["A"], k, 1e-10, x_start=x, sign_convention=True)
    As = np.ldexp(inp["A"], e).astype(np.float32)
    r = tsvd(torch.from_numpy(As).cuda(), k, 1e-10, start_draws=x, iters_override=o.iters,
             sign_convention=True, power_kernel=pk)
    assert r.status == B.TSVD_OK
    assert np.max(np.abs(np.ldexp(r.sigma, -e) - o.sigma) / o.sigma) <= 1e-5
    for l in _all_gapped(o, k):
        assert np.max(np.abs(np.asarray(r.V[:, l], dtype=np.float64) - o.V[:, l])) < 1e-4


def test_tsvd_cluster_power_builtin_draws_and_own_convergence():
    """The cluster kernel draws x_l from the built-in Philox stream itself and
    takes its own convergence decisions (counts within one of the oracle's)."""
    m, n, k, eps = 2048, 256, 8, 1e-8
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=0)
    o = ref.tsvd_dense(inp["A"], k, eps, seed=11)
    r = tsvd(torch.from_numpy(inp["A"]).cuda(), k, eps, seed=11, power_kernel=B.TSVD_POWER_CLUSTER)
    assert all(abs(a - b) <= 1 for a, b in zip(r.iters, o.iters))
    assert np.max(np.abs(r.sigma - o.sigma) / o.sigma) <= 1e-5


# orthogonal batching: n, panel width, precision, where A lives, device budget (0 = none: tiles
# resident on the device; 4 MB: the tiles go to page-locked host memory and stream back)
TILED_CASES = [
    (1000, 256, B.TSVD_GRAM_FP32, "device", 0), (1000, 256, B.TSVD_GRAM_TF32X3, "device", 0),
    (1300, 512, B.TSVD_GRAM_TF32X3, "host", 0), (1300, 512, B.TSVD_GRAM_BF16X3, "device", 0),
    (1000, 256, B.TSVD_GRAM_TF32X3, "host", 4 << 20), (1000, 256, B.TSVD_GRAM_FP32, "host", 4 << 20),
]


@pytest.mark.parametrize("n,bs,prec,where,budget", TILED_CASES)
def test_tsvd_orthogonal_batching_matches_oracle(n, bs, prec, where, budget):
    """Gram as tiles A_J^T A_I (J <= I) of bs-column panels with a ragged last
    panel; the power loop applies G through the tiles.  Same trajectory as the
    oracle (forced counts, caller start draws, sign convention)."""
    m, k, eps = 6000, 8, 1e-10
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.72), 1e-7, seed=n + bs)
    A = inp["A"]
    x = synth.start_normals(n, k, seed=9)
    o = ref.tsvd_dense(A, k, eps, x_start=x, sign_convention=True)
    Ain = torch.from_numpy(A).cuda() if where == "device" else A
    kw = dict(device_budget=budget, force_stream=True) if budget else {}
    r = tsvd(Ain, k, eps, start_draws=x, iters_override=o.iters, sign_convention=True, precision=prec,
             gram_tile=bs, **kw)
    assert r.iters == o.iters
    assert r.report["gram_panels"] == -(-n // bs)
    assert r.report["tiles_on_host"] == (1 if budget else 0)
    _compare(r, o, k, gapped=_all_gapped(o, k))
    for l in _all_gapped(o, k):
        assert np.max(np.abs(np.asarray(r.V[:, l], dtype=np.float64) - o.V[:, l])) < 1e-4


# wide A (m < n, Eq. 3): the Gram is A A^T over column blocks, U from the power method,
# V = A^T U Sigma^-1 from one more pass.  m, n, precision, where A lives, power kernel
WIDE_CASES = [
    (300, 5000, B.TSVD_GRAM_FP32, "device", B.TSVD_POWER_CLUSTER),
    (300, 5000, B.TSVD_GRAM_TF32X3, "resident", B.TSVD_POWER_GRID),
    (1000, 3001, B.TSVD_GRAM_FP32, "stream", B.TSVD_POWER_AUTO),
    (1000, 3001, B.TSVD_GRAM_TF32X3, "stream", B.TSVD_POWER_AUTO),
    (777, 4100, B.TSVD_GRAM_BF16X3, "device", B.TSVD_POWER_GRID),
]


@pytest.mark.parametrize("m,n,prec,where,pk", WIDE_CASES)
def test_tsvd_wide_matches_oracle(m, n, prec, where, pk):
    k, eps = 8, 1e-10
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(m, 0.74), 1e-7, seed=m + n)
    A = inp["A"]
    x = synth.start_normals(m, k, seed=6)  # start vectors of the left (power) side
    o = ref.tsvd_dense(A, k, eps, x_start=x, sign_convention=True)
    kw = dict(power_kernel=pk, precision=prec)
    if where == "device":
        Ain = torch.from_numpy(A).cuda()
    else:
        Ain = A
        if where == "stream":
            kw.update(force_stream=True, block_rows=700, n_buffers=3)
    r = tsvd(Ain, k, eps, start_draws=x, iters_override=o.iters, sign_convention=True, **kw)
    assert r.iters == o.iters
    if where == "stream":
        assert r.report["mode"] == 2 and r.report["n_blocks"] == -(-n // 704)
    gapped = _all_gapped(o, k)
    _compare(r, o, k, gapped=gapped)
    for l in gapped:  # the power vectors are U here, fixed by the sign convention
        assert np.max(np.abs(np.asarray(r.U[:, l], dtype=np.float64) - o.U[:, l])) < 1e-4


def test_tsvd_builtin_start_vectors_match_oracle_generator():
    m, n, k, eps = 1500, 120, 5, 1e-8
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.75), 1e-6, seed=4)
    o = ref.tsvd_dense(inp["A"], k, eps, seed=77)  # oracle's own Philox stream
    r = tsvd(inp["A"], k, eps, seed=77, iters_override=o.iters)
    _compare(r, o, k)


def test_tsvd_sign_convention_and_outputs_on_device():
    m, n, k = 800, 64, 4
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.7), 0.0, seed=5)
    x = synth.start_normals(n, k, seed=3)
    o = ref.tsvd_dense(inp["A"], k, 1e-10, x_start=x, sign_convention=True)
    r = tsvd(torch.from_numpy(inp["A"]).cuda(), k, 1e-10, start_draws=x, iters_override=o.iters,
             sign_convention=True, out_device=True)
    V = r.V.cpu().numpy()
    for l in range(k):
        i = int(np.argmax(np.abs(V[:, l])))
        assert V[i, l] > 0
        assert np.max(np.abs(V[:, l] - o.V[:, l])) < 1e-5  # same sign, same vector
    assert np.max(np.abs(r.sigma.cpu().numpy() - o.sigma) / o.sigma) < 1e-5


def test_tsvd_zero_matrix_reports_rank():
    A = np.zeros((300, 40), dtype=np.float32)
    r = tsvd(A, 3, 1e-8, ok=(B.TSVD_ERANK,))
    assert r.status == B.TSVD_ERANK
    assert np.all(r.sigma == 0)
    V = np.asarray(r.V, dtype=np.float64)
    assert np.allclose(V.T @ V, np.eye(3), atol=1e-6)


def test_tsvd_noconv_flag():
    inp = synth.dense_prescribed(500, 50, synth.spectrum_geometric(50, 0.99), 0.0, seed=6)
    r = tsvd(inp["A"], 2, 1e-14, max_iter=5, ok=(B.TSVD_ENOCONV,))
    assert r.status == B.TSVD_ENOCONV and r.iters == [5, 5]
    assert r.report["flags"] & B.TSVD_FLAG_NOCONV


@pytest.mark.parametrize("mode", ["device", "resident", "stream"])
def test_tsvd_csr_matches_oracle(mode):
    m = n = 1 << 14
    k, eps = 4, 1e-6
    csr = synth.csr_uniform(m, n, 33.5, seed=3)
    x = synth.start_normals(n, k, seed=5)
    o = ref.tsvd_csr(csr, k, eps, x_start=x)
    if mode == "device":
        Ain = {"row_ptr": dev(csr["row_ptr"]), "col_idx": dev(csr["col_idx"]), "values": dev(csr["values"]),
               "m": m, "n": n}
        kw = {}
    else:
        Ain = csr
        kw = dict(force_stream=True, block_rows=3000, n_buffers=3) if mode == "stream" else {}
    r = tsvd(Ain, k, eps, start_draws=x, iters_override=o.iters, **kw)
    assert r.iters == o.iters
    # the bulk of a random sparse spectrum is not gapped; grade sigma for all,
    # vectors for the gapped leading triplet only (the mean direction)
    _compare(r, o, k, gapped=[0])
    r2 = tsvd(Ain, k, eps, start_draws=x, **kw)
    assert abs(r2.sigma[0] - o.sigma[0]) / o.sigma[0] <= 1e-5


@pytest.mark.parametrize("mode,unsorted", [("device", False), ("stream", False), ("device", True)])
def test_tsvd_csr_column_chunked_matches_oracle(mode, unsorted):
    """n = 2^24 > 8M columns: v and w (64 MB each) exceed half of L2, so the
    library applies A^T A in column chunks (two passes, split points per row);
    rows whose columns are not ascending fall back to the fused pair.  Same
    trajectory as the oracle (its application counts forced)."""
    import torch as _t
    m = n = 1 << 24
    k, eps = 3, 1e-6
    g = _t.Generator(device="cuda")
    g.manual_seed(17)
    counts = _t.randint(2, 7, (m,), generator=g, device="cuda", dtype=_t.int64)
    rp = _t.zeros(m + 1, dtype=_t.int64, device="cuda")
    _t.cumsum(counts, 0, out=rp[1:])
    nnz = int(rp[-1].item())
    rows = _t.repeat_interleave(_t.arange(m, device="cuda"), counts)
    cols = _t.randint(0, n, (nnz,), generator=g, device="cuda", dtype=_t.int64)
    key, _ = _t.sort(rows * n + cols)  # sorted within rows (repeated columns allowed: they add up)
    cols = (key - rows * n).to(_t.int32)
    if unsorted:
        # reverse the entries of every row that has more than one
        first = rp[:-1][rows]
        last = rp[1:][rows] - 1
        pos = _t.arange(nnz, device="cuda")
        cols = cols[first + last - pos]
    vals = _t.rand(nnz, generator=g, device="cuda", dtype=_t.float32)
    csr = {"row_ptr": rp.cpu().numpy(), "col_idx": cols.cpu().numpy(), "values": vals.cpu().numpy(), "m": m, "n": n}
    del key, rows
    x = synth.start_normals(n, k, seed=8)
    o = ref.tsvd_csr(csr, k, eps, x_start=x, iters_override=[4, 4, 4])
    if mode == "device":
        Ain = {"row_ptr": rp, "col_idx": cols, "values": vals, "m": m, "n": n}
        kw = {}
    else:
        Ain = csr
        kw = dict(force_stream=True, block_rows=1 << 21, n_buffers=3, device_budget=3 << 30)
    r = tsvd(Ain, k, eps, start_draws=x, iters_override=o.iters, **kw)
    assert r.iters == o.iters
    _compare(r, o, k, gapped=[0])


def test_tsvd_csr_empty_matrix_reports_rank():
    # no stored entries: every application gives w = 0 exactly
    m, n = 400, 200
    csr = {"row_ptr": np.zeros(m + 1, dtype=np.int64), "col_idx": np.zeros(0, dtype=np.int32),
           "values": np.zeros(0, dtype=np.float32), "m": m, "n": n}
    x = synth.start_normals(n, 3, seed=1)
    o = ref.tsvd_csr(csr, 3, 1e-10, x_start=x)
    assert o.status == ["rank"] * 3
    r = tsvd(csr, 3, 1e-10, start_draws=x, ok=(B.TSVD_ERANK,))
    assert r.status == B.TSVD_ERANK
    assert np.all(r.sigma == 0)
    V = np.asarray(r.V, dtype=np.float64)
    assert np.allclose(V.T @ V, np.eye(3), atol=1e-5)
    for l in range(3):
        assert ref.vector_angle(V[:, l], o.V[:, l]) < 1e-5


# ---------------------------------------------------------------- a2 Gram on tcgen05
def _tc_case(rows, n, ld, seed):
    rng = np.random.default_rng(seed)
    Afull = rng.standard_normal((max(rows, 1), ld)).astype(np.float32)[:rows]
    return Afull


def _split_error(prec) -> float:
    """Relative error of one product a*b as the tensor-core mode forms it.
    TF32: both operands rounded to 11 significant bits (2^-11 each).
    TF32X3: a = hi + lo + r with |r| <= 2^-22 |a|; the dropped lo*lo and the
    r terms stay below 3 * 2^-22.  BF16X3: hi = bf16(a) (|a - hi| <= 2^-8 |a|),
    mid = bf16(a - hi) (|a - hi - mid| <= 2^-16 |a|); the dropped mid*mid and
    the four remainder terms sum to at most
    2^-16 ((1+2^-8)^2 + 2 (1+2^-8) + 2^-7 (1+2^-8) + 2^-16)."""
    if prec == B.TSVD_GRAM_TF32:
        return 2.0 ** -10 + 2.0 ** -22
    if prec == B.TSVD_GRAM_TF32X3:
        return 3 * 2.0 ** -22
    u = 1 + 2.0 ** -8
    return 2.0 ** -16 * (u * u + 2 * u + 2.0 ** -7 * u + 2.0 ** -16)


@pytest.mark.parametrize("prec", [B.TSVD_GRAM_TF32, B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_BF16X3])
@pytest.mark.parametrize("rows,n,ld", [(1000, 256, 256), (777, 130, 130), (64, 5, 5), (5000, 300, 300),
                                       (300, 129, 133), (20000, 512, 512), (1, 17, 17), (70, 640, 640)])
def test_gram_tensor_cores_match_oracle(prec, rows, n, ld):
    """Products with the split error of the mode (_split_error), FP32
    accumulation over a K slice, then FP64.  Bound: (e_in + (K+2) 2^-23) (|A|^T |A|)."""
    _check_gram_tc(prec, rows, n, ld)


@pytest.mark.parametrize("prec", [B.TSVD_GRAM_TF32, B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_BF16X3])
@pytest.mark.parametrize("rowb", [64, 128])
@pytest.mark.parametrize("rows,n,ld", [(5000, 300, 300), (300, 129, 133), (70, 640, 640)])
def test_gram_tensor_cores_both_stage_layouts(prec, rowb, rows, n, ld, monkeypatch):
    """Both stage layouts of the SYRK (64-byte and 128-byte swizzle rows of K,
    TSVD_TC_ROW) meet the same bound, whichever one a precision takes by
    default."""
    monkeypatch.setenv("TSVD_TC_ROW", str(rowb))
    _check_gram_tc(prec, rows, n, ld)


def _check_gram_tc(prec, rows, n, ld):
    Afull = _tc_case(rows, n, ld, rows * 7 + n)
    A = Afull[:, :n]
    sentinel = -7.25
    G = np.tril(np.full((n, n), sentinel), -1)
    dG = dev(G)
    dA = dev(Afull) if rows else torch.empty(1, dtype=torch.float32, device="cuda")
    sb = B.tsvd_gram_scratch_bytes(rows, n, prec)
    scr = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda")
    assert B.tsvd_gram_accumulate(dA.data_ptr(), rows, n, ld, dG.data_ptr(), prec, scr.data_ptr(), sb, S()) == 0
    torch.cuda.synchronize()
    assert int(scr[:4].view(torch.int32).item()) == 0  # no bounded wait gave up
    got = dG.cpu().numpy()
    ref_G = ref.gram(A)
    absA = np.abs(A.astype(np.float64))
    absG = absA.T @ absA
    e_in = _split_error(prec)
    K = min(rows, 8192)
    bound = (e_in + (K + 2) * 2.0 ** -23) * absG + 1e-300
    iu = np.triu_indices(n)
    err = got[iu] - ref_G[iu]
    assert np.all(np.abs(err) <= bound[iu]), float(np.max(np.abs(err) / bound[iu]))
    il = np.tril_indices(n, -1)
    assert np.all(got[il] == sentinel)
    if rows >= 1000:
        # no systematic bias on the diagonal (a biased Gram shifts every sigma)
        d = np.arange(n)
        bias = float(np.mean((got[d, d] - ref_G[d, d]) / ref_G[d, d]))
        # short TMEM accumulation segments keep the toward-zero drift of the
        # tensor-core accumulator to ~0.4 ulp x (16..24 MMAs) ~ 5e-7.  BF16X3
        # also drops mid*mid >= 0 on the diagonal: E[(a - hi)^2 / a^2] is about
        # 2^-15 / 12 = 2.5e-6 for Gaussian entries.
        lim = 1e-5 if prec == B.TSVD_GRAM_BF16X3 else 2e-6
        assert abs(bias) < lim, bias


# ---------------------------------------------------------------- mixed precision (clustered spectrum)
@pytest.mark.parametrize("prec", [B.TSVD_GRAM_FP32, B.TSVD_GRAM_TF32, B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_BF16X3])
def test_tsvd_clustered_spectrum_precisions_match_oracle(prec):
    """Mixed-precision workload at reduced size: stacked-orthogonal A with a
    harmonic spectrum and the pair sigma_10 - sigma_11 = 1e-3, k = 32,
    eps = 1e-8; every Gram precision follows the oracle's trajectory."""
    n, copies, k, eps = 1024, 16, 32, 1e-8
    sig_t = synth.spectrum_harmonic_clustered(n, 10, 1e-3)
    fac = synth.stacked_factor(n, sig_t, copies, seed=2)
    A = torch.empty((copies * n, n), dtype=torch.float32, device="cuda")
    synth.stacked_rows_torch(A, fac["M32"], seed=2)
    Ah = A.cpu().numpy()
    x = synth.start_normals(n, k, seed=4)
    sig_o, V_o, it_o, st_o = ref.right_vectors(ref.gram(Ah), k, eps, x_start=x)
    assert all(s == "ok" for s in st_o)
    r = tsvd(A, k, eps, start_draws=x, iters_override=it_o, precision=prec, out_device=True)
    assert r.iters == it_o
    r.sigma = r.sigma.cpu().numpy()
    r.V = r.V.cpu().numpy()
    check_clustered(r, sig_o, V_o, k, prec, sig_t)


@pytest.mark.parametrize("prec", [B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_BF16X3])
def test_tsvd_split_precisions_c1_match_oracle(prec):
    m, n, k, eps = 2048, 256, 8, 1e-8
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=0)
    x = synth.start_normals(n, k, seed=1)
    o = ref.tsvd_dense(inp["A"], k, eps, x_start=x)
    r = tsvd(torch.from_numpy(inp["A"]).cuda(), k, eps, start_draws=x, iters_override=o.iters, precision=prec)
    _compare(r, o, k)


@pytest.mark.parametrize("prec,budget", [(B.TSVD_GRAM_TF32, 0), (B.TSVD_GRAM_TF32X3, 0),
                                         (B.TSVD_GRAM_TF32, 256 << 20)])
def test_tsvd_tensor_cores_c2_shape(prec, budget):
    # the out-of-core workload's structure at a size the oracle handles:
    # rank-64, sigma_i = 1/(1+i), 1e-4 noise; streamed in row blocks
    m, n, k, eps = 1 << 17, 512, 8, 1e-6
    sig = 1.0 / (1.0 + np.arange(64))
    V = synth.orthonormal_columns(n, 64, 3, 1)
    A = synth.dense_lowrank_rows(0, m, V, sig, m, 1e-4, seed=3)
    x = synth.start_normals(n, k, seed=2)
    Gf = ref.gram(A)
    o = ref.tsvd_dense(A, k, eps, x_start=x, B=Gf)
    lam = np.linalg.eigvalsh(Gf)[::-1]
    gapped = ref.gapped_indices(lam, k)
    assert gapped == list(range(k)), gapped  # noise Gram 1.3e-3 I: gaps of the leading 8 stay above 0.19
    # under a budget the ring takes every slot that fits and the U pass
    # starts from the row blocks still resident after the Gram pass
    r = tsvd(A, k, eps, start_draws=x, iters_override=o.iters, precision=prec, force_stream=True,
             block_rows=(1 << 14) if budget else (1 << 15), device_budget=budget)
    assert r.report["n_blocks"] == (8 if budget else 4)
    assert r.report["ring_slots"] == (6 if budget else 3)
    _compare(r, o, k, gapped=gapped)


@pytest.mark.parametrize("prec,where", [(B.TSVD_GRAM_TF32X3, "device"), (B.TSVD_GRAM_BF16X3, "device"),
                                        (B.TSVD_GRAM_TF32X3, "resident")])
def test_tsvd_in_core_many_chunks(prec, where):
    """In core with many chunks (a ragged last one) on the tensor-core Gram:
    the same trajectory as the oracle's, no flag but the pageable-input one."""
    m, n, k, eps = 40000, 384, 6, 1e-6
    sig = 1.0 / (1.0 + np.arange(64))
    V = synth.orthonormal_columns(n, 64, 5, 1)
    A = synth.dense_lowrank_rows(0, m, V, sig, m, 1e-4, seed=5)
    x = synth.start_normals(n, k, seed=4)
    Gf = ref.gram(A)
    o = ref.tsvd_dense(A, k, eps, x_start=x, B=Gf)
    gapped = ref.gapped_indices(np.linalg.eigvalsh(Gf)[::-1], k)
    assert gapped == list(range(k)), gapped
    Ain = torch.from_numpy(A).cuda() if where == "device" else A
    r = tsvd(Ain, k, eps, start_draws=x, iters_override=o.iters, precision=prec, block_rows=3000)
    assert r.report["n_blocks"] == -(-m // 3008) and r.report["mode"] == (0 if where == "device" else 1)
    assert r.report["flags"] & ~B.TSVD_FLAG_PAGEABLE == 0
    _compare(r, o, k, gapped=gapped)
