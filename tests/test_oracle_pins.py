"""Pins for the FP64 oracle: each test ties it to something other than itself
(published known-answer vectors, closed forms, LAPACK, brute-force Jacobi,
algebraic identities, invariants), so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import jacobi, philox
from oracle import tsvd_ref as ref
from oracle import csr_c

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator pins
def _kat_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32))
        assert [int(x) for x in got] == out


def test_splitmix64_reference_outputs():
    # SplitMix64 sequence from state 0 (Steele et al. 2014; the generator
    # advances its state by the golden gamma before each output)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = []
    state = 0
    for _ in range(3):
        got.append(philox.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    assert got == want


def test_box_muller_is_standard_normal():
    from scipy import stats
    x = philox.start_normals(seed=7, l=3, n=400_001)
    assert x.shape == (400_001,)
    n = x.shape[0]
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # pairs are independent: correlation of even and odd draws ~ 0
    assert abs(np.corrcoef(x[0:-1:2], x[1::2])[0, 1]) < 5 / math.sqrt(n / 2)


def test_start_vector_streams_differ_and_repeat():
    a = philox.start_normals(1, 0, 1001)
    b = philox.start_normals(1, 1, 1001)
    c = philox.start_normals(2, 0, 1001)
    assert np.array_equal(a, philox.start_normals(1, 0, 1001))
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # prefix property: the first draws do not depend on n
    assert np.array_equal(philox.start_normals(1, 0, 10), a[:10])


# ---------------------------------------------------------------- Gram pins
def test_gram_matches_loops_and_exact_integers():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((13, 5)).astype(np.float32)
    assert np.allclose(ref.gram(A), ref.gram_plain(A), rtol=1e-14, atol=1e-14)
    # integer matrix: every product and sum is exact in FP64
    Ai = rng.integers(-50, 50, size=(37, 9)).astype(np.float32)
    exact = np.zeros((9, 9), dtype=np.int64)
    Aii = Ai.astype(np.int64)
    for i in range(9):
        for j in range(9):
            exact[i, j] = int(np.sum(Aii[:, i] * Aii[:, j]))
    assert np.array_equal(ref.gram(Ai), exact.astype(np.float64))
    # a transposed operand (A A^T) has the wrong shape and values
    assert ref.gram(Ai).shape == (9, 9)


@pytest.mark.parametrize("block", [1, 7, 64, 1000])
def test_gram_row_blocks_equals_gram(block):
    rng = np.random.default_rng(1)
    A = rng.integers(-9, 9, size=(130, 11)).astype(np.float32)
    assert np.array_equal(ref.gram_row_blocks(A, block), ref.gram(A))


# ---------------------------------------------------------------- power-method pins
def test_diagonal_matrix_gives_canonical_vectors():
    d = np.array([3.0, -7.0, 0.5, 5.0, 1.5, 2.0])
    A = np.zeros((10, 6))
    A[np.arange(6), np.arange(6)] = d
    r = ref.tsvd_dense(A, 6, 1e-15, seed=3)
    order = np.argsort(-np.abs(d))
    assert np.allclose(r.sigma, np.abs(d)[order], rtol=1e-12)
    for l, idx in enumerate(order):
        e = np.zeros(6); e[idx] = 1.0
        assert ref.vector_angle(r.V[:, l], e) < 1e-6


def test_rank_one_converges_immediately():
    rng = np.random.default_rng(2)
    u = rng.standard_normal(50); u /= np.linalg.norm(u)
    v = rng.standard_normal(20); v /= np.linalg.norm(v)
    A = 3.25 * np.outer(u, v)
    r = ref.tsvd_dense(A, 1, 1e-12, seed=0)
    assert r.iters[0] == 2  # first application lands on v, second confirms it
    assert abs(r.sigma[0] - 3.25) < 1e-13
    assert ref.vector_angle(r.V[:, 0], v) < 1e-12
    assert ref.vector_angle(r.U[:, 0], u) < 1e-12


def test_prescribed_spectrum_closed_form():
    # noise-free A = U diag(0.8^i) V^T in FP64: the sigma_i are known exactly
    sig = synth.spectrum_geometric(64, 0.8)
    U = synth.orthonormal_columns(256, 64, 11, 0)
    V = synth.orthonormal_columns(64, 64, 11, 1)
    A = (U * sig) @ V.T
    r = ref.tsvd_dense(A, 8, 1e-15, seed=5)
    assert np.max(np.abs(r.sigma - sig[:8]) / sig[:8]) < 1e-9
    for l in range(8):
        assert ref.vector_angle(r.V[:, l], V[:, l]) < 1e-5
        assert ref.vector_angle(r.U[:, l], U[:, l]) < 1e-5


def test_against_lapack_on_c1_shape():
    inp = synth.dense_prescribed(2048, 256, synth.spectrum_geometric(256, 0.8), 1e-6, seed=0)
    A = inp["A"]
    r = ref.tsvd_dense(A, 8, 1e-15, seed=0)
    Ut, st, Vt = np.linalg.svd(A.astype(np.float64), full_matrices=False)
    assert np.max(np.abs(r.sigma - st[:8]) / st[:8]) < 1e-10
    for l in range(8):
        assert ref.vector_angle(r.V[:, l], Vt[l]) < 1e-6
        assert ref.vector_angle(r.U[:, l], Ut[:, l]) < 1e-6


def test_against_brute_force_jacobi():
    rng = np.random.default_rng(4)
    for (m, n) in [(40, 12), (64, 16), (9, 9)]:
        A = rng.standard_normal((m, n))
        Uj, sj, Vj = jacobi.jacobi_svd(A)
        # Jacobi itself reproduces A and is orthonormal
        assert np.allclose((Uj * sj) @ Vj.T, A, atol=1e-12)
        assert np.allclose(Vj.T @ Vj, np.eye(n), atol=1e-12)
        k = min(6, n)
        r = ref.tsvd_dense(A, k, 1e-15, seed=1, max_iter=200000)
        assert np.max(np.abs(r.sigma - sj[:k]) / sj[:k]) < 1e-8
        for l in range(k):
            gap = min(sj[l - 1] ** 2 - sj[l] ** 2 if l else np.inf, sj[l] ** 2 - sj[l + 1] ** 2)
            if gap / sj[l] ** 2 > 0.05:
                assert ref.vector_angle(r.V[:, l], Vj[:, l]) < 1e-5


def test_eckart_young_and_orthonormality():
    inp = synth.dense_prescribed(300, 40, synth.spectrum_geometric(40, 0.7), 0.0, seed=9)
    A = inp["A"].astype(np.float64)
    k = 6
    r = ref.tsvd_dense(A, k, 1e-15, seed=2)
    s_all = np.linalg.svd(A, compute_uv=False)
    res = ref.frobenius_residual_sq(A, r.U, r.sigma, r.V)
    assert abs(res - np.sum(s_all[k:] ** 2)) < 1e-8 * np.sum(s_all ** 2)
    # eps = 1e-15 leaves each vector ~sqrt(2 eps) r / (1 - r) ~ 5e-8 from the truth
    assert np.allclose(r.V.T @ r.V, np.eye(k), atol=1e-6)
    assert np.allclose(r.U.T @ r.U, np.eye(k), atol=1e-6)


def test_wide_matrix_is_transpose_of_tall():
    inp = synth.dense_prescribed(120, 30, synth.spectrum_geometric(30, 0.75), 0.0, seed=4)
    A = inp["A"].astype(np.float64)
    x = synth.start_normals(30, 5, seed=8)
    tall = ref.tsvd_dense(A, 5, 1e-14, x_start=x)
    wide = ref.tsvd_dense(A.T, 5, 1e-14, x_start=x)
    assert np.allclose(tall.sigma, wide.sigma, rtol=1e-12)
    for l in range(5):
        assert ref.vector_angle(tall.V[:, l], wide.U[:, l]) < 1e-12
        assert ref.vector_angle(tall.U[:, l], wide.V[:, l]) < 1e-12


def test_zero_matrix_reports_rank_deficiency():
    A = np.zeros((20, 6))
    r = ref.tsvd_dense(A, 3, 1e-8, seed=0)
    assert np.all(r.sigma == 0) and r.status == ["rank"] * 3
    assert np.allclose(r.V.T @ r.V, np.eye(3), atol=1e-12)


def test_iters_override_runs_exact_counts():
    inp = synth.dense_prescribed(200, 30, synth.spectrum_geometric(30, 0.9), 0.0, seed=6)
    r = ref.tsvd_dense(inp["A"], 4, 1e-8, seed=0, iters_override=[3, 1, 7, 2])
    assert r.iters == [3, 1, 7, 2]


def test_convergence_rule_matches_definition():
    # the stopping iterate is the first with |v0.v1| >= 1 - eps
    inp = synth.dense_prescribed(200, 30, synth.spectrum_geometric(30, 0.9), 0.0, seed=6)
    B = ref.gram(inp["A"])
    v0 = philox.start_normals(0, 0, 30)
    v0 = v0 / np.linalg.norm(v0)
    res = ref.power_method(lambda v: B @ v, v0, 1e-6, record=True)
    assert res.cos_hist[-1] >= 1 - 1e-6
    assert all(c < 1 - 1e-6 for c in res.cos_hist[:-1])
    assert len(res.cos_hist) == res.iters


# ---------------------------------------------------------------- Eq. 1-3, Alg. 4
def _eq_inputs(m, n, k, seed, orth="U"):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, n))
    if orth == "U":
        U = np.linalg.qr(rng.standard_normal((m, k)))[0]
        V = rng.standard_normal((n, k))
    else:
        U = rng.standard_normal((m, k))
        V = np.linalg.qr(rng.standard_normal((n, k)))[0]
    S = rng.uniform(0.5, 2.0, size=k)
    v0 = rng.standard_normal(n if orth == "U" else m)
    return X, U, S, V, v0


def test_eq1_equals_explicit_residual_gram():
    X, U, S, V, _ = _eq_inputs(50, 12, 4, 0)
    Xp = X - (U * S) @ V.T
    assert np.allclose(ref.eq1_gram(X, U, S, V), Xp.T @ Xp, rtol=1e-12, atol=1e-11)


def test_eq2_equals_explicit_residual_product():
    X, U, S, V, v0 = _eq_inputs(60, 15, 5, 1)
    Xp = X - (U * S) @ V.T
    assert np.allclose(ref.eq2_apply(X, U, S, V, v0), Xp.T @ (Xp @ v0), rtol=1e-12, atol=1e-11)


def test_eq3_equals_explicit_residual_product():
    X, U, S, V, u0 = _eq_inputs(14, 55, 4, 2, orth="V")
    Xp = X - (U * S) @ V.T
    assert np.allclose(ref.eq3_apply(X, U, S, V, u0), Xp @ (Xp.T @ u0), rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("n_b,N", [(1, 1), (4, 1), (3, 5), (5, 2)])
def test_alg4_corrected_equals_eq2(n_b, N):
    X, U, S, V, v0 = _eq_inputs(47, 19, 4, 3)
    assert np.allclose(ref.dist_compute_v0(X, U, S, V, v0, n_b, N), ref.eq2_apply(X, U, S, V, v0),
                       rtol=1e-12, atol=1e-11)


def test_hotelling_equals_eq2_for_exact_vectors():
    # with exact singular triplets, Eq. 2 and the Hotelling form coincide
    inp = synth.dense_prescribed(80, 20, synth.spectrum_geometric(20, 0.8), 0.0, seed=5)
    A = inp["A"].astype(np.float64)
    Ut, st, Vt = np.linalg.svd(A, full_matrices=False)
    k = 4
    U, S, V = Ut[:, :k], st[:k], Vt[:k].T
    v0 = np.random.default_rng(0).standard_normal(20)
    hot = ref.hotelling_apply(ref.gram(A), V, S ** 2)(v0)
    assert np.allclose(hot, ref.eq2_apply(A, U, S, V, v0), rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- O-1 vs O-2
def test_hotelling_oracle_agrees_with_literal_algorithm():
    inp = synth.dense_prescribed(512, 64, synth.spectrum_geometric(64, 0.8), 1e-6, seed=1)
    A = inp["A"]
    x = synth.start_normals(64, 6, seed=3)
    o1 = ref.tsvd_dense(A, 6, 1e-12, x_start=x)
    o2 = ref.tsvd_literal(A, 6, 1e-12, x_start=x)
    assert np.max(np.abs(o1.sigma - o2.sigma) / o2.sigma) < 1e-8
    for l in range(6):
        assert ref.vector_angle(o1.V[:, l], o2.V[:, l]) < 1e-4


# ---------------------------------------------------------------- CSR oracle
def test_csr_operators_match_dense():
    rng = np.random.default_rng(5)
    D = rng.standard_normal((40, 25)) * (rng.random((40, 25)) < 0.2)
    D[3] = 0.0  # an empty row
    D = D.astype(np.float32)
    csr = synth.csr_from_dense(D)
    v = rng.standard_normal(25)
    y = ref.csr_matvec(csr["row_ptr"], csr["col_idx"], csr["values"], v)
    assert np.allclose(y, D.astype(np.float64) @ v, rtol=1e-13, atol=1e-13)
    w = ref.csr_rmatvec(csr["row_ptr"], csr["col_idx"], csr["values"], y, 25)
    assert np.allclose(w, D.astype(np.float64).T @ y, rtol=1e-13, atol=1e-13)
    wc, ss = csr_c.csr_gram_apply(csr["row_ptr"], csr["col_idx"], csr["values"], v)
    assert np.allclose(wc, w, rtol=1e-13, atol=1e-13) and abs(ss - y @ y) < 1e-11


def test_csr_oracle_equals_dense_oracle():
    csr = synth.csr_uniform(300, 120, 6.0, seed=2)
    D = np.zeros((300, 120), dtype=np.float32)
    rows = ref.csr_row_index(csr["row_ptr"])
    D[rows, csr["col_idx"]] = csr["values"]
    x = synth.start_normals(120, 4, seed=1)
    a = ref.tsvd_csr(csr, 4, 1e-10, x_start=x)
    b = ref.tsvd_dense(D, 4, 1e-10, x_start=x)
    assert a.iters == b.iters
    assert np.allclose(a.sigma, b.sigma, rtol=1e-12)
    for l in range(4):
        assert ref.vector_angle(a.V[:, l], b.V[:, l]) < 1e-9


def test_csr_generator_structure():
    csr = synth.csr_uniform(2000, 5000, 7.5, seed=3)
    rp, ci = csr["row_ptr"], csr["col_idx"]
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == ci.shape[0]
    assert ci.dtype == np.int32 and rp.dtype == np.int64 and csr["values"].dtype == np.float32
    for r in range(0, 2000, 37):
        seg = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(seg) > 0)  # sorted, no duplicates
    assert abs(np.diff(rp).mean() - 7.5) < 0.5
    assert np.all((csr["values"] >= 0) & (csr["values"] < 1))


# ---------------------------------------------------------------- grading helpers
# The parity tests grade a singular vector only when its eigenvalue is gapped
# (relative gap >= 0.05 to both neighbours) and grade a clustered pair as a
# 2-D subspace by its largest principal angle.  These pins tie the helpers
# that make those decisions to closed forms.
def _planes(theta, phi, n=7, perm=None, signs=None):
    """span(e0, e1) and span(cos(phi) e0 + sin(phi) e2, cos(theta) e1 + sin(theta) e3):
    principal angles phi and theta, built from exact entries (row permutations
    and sign flips keep them exact)."""
    a = np.zeros((n, 2))
    a[0, 0] = a[1, 1] = 1.0
    b = np.zeros((n, 2))
    b[0, 0], b[2, 0] = math.cos(phi), math.sin(phi)
    b[1, 1], b[3, 1] = math.cos(theta), math.sin(theta)
    if perm is not None:
        a, b = a[perm], b[perm]
    if signs is not None:
        a, b = a * signs[:, None], b * signs[:, None]
    return a, b


def _grading_pins_hold():
    """True when both grading helpers agree with their closed forms."""
    ok = True
    rng = np.random.default_rng(3)
    for theta in (1e-6, 1e-3, 0.5):
        for perm, signs in ((None, None), (rng.permutation(7), rng.choice([-1.0, 1.0], 7))):
            a, b = _planes(theta, theta / 3, perm=perm, signs=signs)
            for x, y in ((a, b), (b, a)):
                ok &= abs(ref.subspace_angle(x, y) - theta) <= 1e-12 * theta
    # the same span in another basis (an in-plane rotation) has angle zero
    a, _ = _planes(0.1, 0.05)
    c, s_ = math.cos(0.7), math.sin(0.7)
    ok &= ref.subspace_angle(a, a @ np.array([[c, -s_], [s_, c]])) <= 1e-15
    # a one-dimensional span is the vector angle
    ok &= abs(ref.subspace_angle(a[:, 0], _planes(1e-6, 1e-6)[1][:, 0]) - 1e-6) <= 1e-18
    # hand-built spectrum: i = 1 is 0.0449 / 0.9 = 0.0499 under the bar on its right,
    # i = 2 is 0.0449 / 0.8551 = 0.0525 over it on its left, i = 3 and 4 are 0.0199 apart,
    # i = 5 has its right neighbour (beyond k = 6) only 1e-4 below it, i = 0 has no left one
    lam = np.array([1.0, 0.9, 0.8551, 0.5, 0.4801, 0.3, 0.2999, 0.1])
    ok &= ref.gapped_indices(lam, 6) == [0, 2]
    ok &= ref.gapped_indices(lam, 8) == [0, 2, 7]
    lam2 = np.array([4.0, 2.0, 1.0, 0.0])  # a zero eigenvalue is never graded
    ok &= ref.gapped_indices(lam2, 4) == [0, 1, 2]
    ok &= ref.gapped_indices(lam2, 3, rel_gap=0.6) == [2]  # relative gaps 0.5, 0.5, 1.0
    return bool(ok)


def test_subspace_angle_closed_forms():
    """Largest principal angle of two planes built at a known angle (1e-6,
    1e-3, 0.5) to 1e-12 relative; zero for the same span in a rotated basis."""
    assert _grading_pins_hold()


def test_vector_angle_closed_forms():
    e0, e1 = np.eye(5)[0], np.eye(5)[1]
    for theta in (1e-7, 1e-4, 0.3, 1.2):
        b = math.cos(theta) * e0 + math.sin(theta) * e1
        assert abs(ref.vector_angle(e0, b) - theta) <= 1e-12 * theta
        assert abs(ref.vector_angle(e0, -3.0 * b) - theta) <= 1e-12 * theta  # sign and scale free
    assert ref.vector_angle(e0, e1) == pytest.approx(math.pi / 2, rel=1e-15)


def test_gapped_indices_hand_built_spectrum():
    lam = np.array([1.0, 0.9, 0.8551, 0.5, 0.4801, 0.3, 0.2999, 0.1])
    # relative gaps min(left, right) / lam_i: 0.1, 0.0499, 0.0525, 0.0398, 0.0414, 3.3e-4, 3.3e-4, 1.999
    assert ref.gapped_indices(lam, 6) == [0, 2]
    assert ref.gapped_indices(lam, 8) == [0, 2, 7]
    assert ref.gapped_indices(lam, 3, rel_gap=0.0) == [0, 1, 2]
    # a geometric spectrum rho^(2i): every gap is 1 - rho^2
    assert ref.gapped_indices(0.97 ** (2 * np.arange(10.0)), 9) == list(range(9))  # 0.0591
    assert ref.gapped_indices(0.98 ** (2 * np.arange(10.0)), 9) == []  # 0.0396
    assert ref.gapped_indices(np.array([4.0, 2.0, 1.0, 0.0]), 4) == [0, 1, 2]


# ---------------------------------------------------------------- planted mistakes
def _pins_hold():
    """Run a compact set of pins; returns True when all hold."""
    inp = synth.dense_prescribed(256, 48, synth.spectrum_geometric(48, 0.8), 0.0, seed=11)
    A = inp["A"].astype(np.float64)
    r = ref.tsvd_dense(A, 5, 1e-14, seed=5)
    st = np.linalg.svd(A, compute_uv=False)
    ok_sigma = np.max(np.abs(r.sigma - st[:5]) / st[:5]) < 1e-8
    ok_orth = np.allclose(r.V.T @ r.V, np.eye(5), atol=1e-6)
    ok_u = np.allclose(r.U.T @ r.U, np.eye(5), atol=1e-6)
    # square, non-symmetric input: right vectors against LAPACK
    sq = synth.dense_prescribed(40, 40, synth.spectrum_geometric(40, 0.7), 0.0, seed=12)["A"]
    sq = sq.astype(np.float64)
    rs = ref.tsvd_dense(sq, 3, 1e-14, seed=1)
    _, _, Vt = np.linalg.svd(sq)
    ok_v = all(ref.vector_angle(rs.V[:, l], Vt[l]) < 1e-5 for l in range(3))
    return bool(ok_sigma and ok_orth and ok_u and ok_v)


def test_pins_catch_planted_mistakes(monkeypatch):
    assert _pins_hold()

    def flipped(B, V, sigma2):  # wrong sign on the deflation term
        def apply(v):
            w = B @ v
            if V.shape[1]:
                w = w + V @ (sigma2 * (V.T @ v))
            return w
        return apply

    def dropped(B, V, sigma2):  # deflation term dropped
        return lambda v: B @ v

    def shifted(B, V, sigma2):  # wrong index: sigma_{j+1} paired with v_j
        def apply(v):
            w = B @ v
            if V.shape[1]:
                s = np.roll(sigma2, -1)
                w = w - V @ (s * (V.T @ v))
            return w
        return apply

    for bad in (flipped, dropped, shifted):
        monkeypatch.setattr(ref, "hotelling_apply", bad)
        assert not _pins_hold(), bad.__name__
    monkeypatch.undo()

    # transposed operand in the Gram: A A^T instead of A^T A
    def gram_t(M):
        M = np.asarray(M, dtype=np.float64)
        return M @ M.T if M.shape[0] == M.shape[1] else M.T @ M
    monkeypatch.setattr(ref, "gram", gram_t)
    assert not _pins_hold()
    monkeypatch.undo()

    # grading helpers: each plausible slip must break a closed form
    assert _grading_pins_hold()
    true_angle = ref.subspace_angle

    def smallest_angle(a, b):  # cos from the largest singular value: the smallest principal angle
        qa, _ = np.linalg.qr(np.atleast_2d(np.asarray(a, float).T).T)
        qb, _ = np.linalg.qr(np.atleast_2d(np.asarray(b, float).T).T)
        return math.acos(min(1.0, np.linalg.svd(qa.T @ qb, compute_uv=False).max()))

    def acos_form(a, b):  # the cosine alone: half the digits lost at tiny angles
        qa, _ = np.linalg.qr(np.atleast_2d(np.asarray(a, float).T).T)
        qb, _ = np.linalg.qr(np.atleast_2d(np.asarray(b, float).T).T)
        return math.acos(min(1.0, np.linalg.svd(qa.T @ qb, compute_uv=False).min()))

    for bad in (smallest_angle, acos_form, lambda a, b: true_angle(a, b[:, ::-1] if b.ndim > 1 else b) / 2):
        monkeypatch.setattr(ref, "subspace_angle", bad)
        assert not _grading_pins_hold()
    monkeypatch.undo()

    def right_only(lam, k, rel_gap=0.05):  # left neighbour ignored
        return [i for i in range(k) if lam[i] > 0 and
                ((lam[i] - lam[i + 1]) if i + 1 < len(lam) else np.inf) / lam[i] >= rel_gap]

    def absolute_gap(lam, k, rel_gap=0.05):  # gap not divided by lam_i
        out = []
        for i in range(k):
            le = lam[i - 1] - lam[i] if i > 0 else np.inf
            ri = lam[i] - lam[i + 1] if i + 1 < len(lam) else np.inf
            if lam[i] > 0 and min(le, ri) >= rel_gap:
                out.append(i)
        return out

    def truncated(lam, k, rel_gap=0.05):  # neighbours beyond k ignored
        return true_gapped(np.asarray(lam)[:k], k, rel_gap)

    def over_previous(lam, k, rel_gap=0.05):  # divided by lam_{i-1} instead of lam_i
        out = []
        for i in range(k):
            le = lam[i - 1] - lam[i] if i > 0 else np.inf
            ri = lam[i] - lam[i + 1] if i + 1 < len(lam) else np.inf
            if lam[i] > 0 and min(le, ri) / lam[max(i - 1, 0)] >= rel_gap:
                out.append(i)
        return out

    true_gapped = ref.gapped_indices
    for bad in (right_only, absolute_gap, truncated, over_previous):
        monkeypatch.setattr(ref, "gapped_indices", bad)
        assert not _grading_pins_hold(), bad.__name__


def test_stacked_workload_identities():
    """The stacked dense workload: A^T A = copies * M^T M exactly (row
    permutations and signs), singular values = the prescribed sigma up to the
    FP32 rounding of M, right singular vectors = the generator's V."""
    torch = pytest.importorskip("torch")
    n, copies = 48, 6
    sig = synth.spectrum_harmonic_clustered(n, 10, 1e-3)
    fac = synth.stacked_factor(n, sig, copies, seed=5)
    A = torch.empty((copies * n, n), dtype=torch.float32)
    synth.stacked_rows_torch(A, fac["M32"], seed=5)
    A = A.numpy()
    G = ref.gram(A)
    Gs = copies * ref.gram(fac["M32"])
    assert np.allclose(G, Gs, rtol=0, atol=1e-14 * np.abs(Gs).max())
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    # FP32 rounding of M: |dM| <= 2^-24 |M| per entry
    assert np.max(np.abs(s - sig)) <= 2.0 ** -24 * np.sqrt(copies) * np.linalg.norm(np.abs(fac["M32"]), 2) * 4
    lam, Q = np.linalg.eigh(G)
    for i in (0, 5, 20):
        assert ref.vector_angle(Q[:, n - 1 - i], fac["V"][:, i]) < 1e-5
    # every block is a signed row permutation of M
    for b in range(copies):
        blk = np.abs(A[b * n:(b + 1) * n])
        assert np.array_equal(np.sort(blk, axis=0), np.sort(np.abs(fac["M32"]), axis=0))
