"""FP64 CPU oracle for the truncated SVD by the deflated power method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this module: only the tests, the smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA library.

Paper: "Distributed Out-of-Memory SVD on CPU/GPU Architectures" (2208.08410).
Notation follows the paper: A is m x n, X the (deflated) matrix, B the Gram
matrix, v0/v1 successive iterates, sigma the singular values, U and V the left
and right singular vectors, eps the convergence threshold, l the triplet index.

Contents, each citing the passage it restates:
  gram, gram_row_blocks, gram_plain    B = A^T A                 (Alg. 2, Sec. IV, Sec. V-C)
  power_method                         Alg. 2's while-loop       (Alg. 2)
  tsvd_dense                           O-1: Hotelling deflation  (Alg. 1; Eq. 2 with U = A V S^-1)
  tsvd_csr                             O-1 on a CSR matrix       (Alg. 1, Alg. 4 operator)
  tsvd_literal                         Alg. 1 + Alg. 2 verbatim with the explicit residual
  eq1_gram, eq2_apply, eq3_apply       Eq. 1, Eq. 2, Eq. 3
  dist_compute_v0                      Alg. 4 (typos corrected, see below)
  csr_matvec, csr_rmatvec              y = A v, w = A^T y (Alg. 4)
  gapped_indices, subspace_angle,      the grading rule of the parity tests: a triplet is graded
  vector_angle                         when its relative eigen-gap is >= 0.05 to both neighbours,
                                       a cluster by its largest principal angle

Every function is pinned by tests/test_oracle_pins.py against something other
than itself (closed forms, published known answers, LAPACK, brute force,
identities); none is "parity unpinned".

Readings of the paper taken here (each also listed in the design notes):
  * m >= n takes the right-vector branch (Alg. 4 uses m >= n; Alg. 1 says m > n).
  * Deflation for the primary oracle is the Hotelling form
        v1 = (B - V S^2 V^T) v0,   B = A^T A,
    which Eq. 2 reduces to when u_j = A v_j / sigma_j and the v_j are exact
    eigenvectors of B; tsvd_literal keeps the paper's explicit residual.
  * The convergence test |v0 . v1| >= 1 - eps is evaluated in FP64; an
    iteration cap max_iter stops a non-converging loop; iters_override forces
    a fixed number of applications per triplet (the paper's benchmark mode
    with the convergence test disabled, Sec. V-E).
  * sigma_l = ||A v_l|| (Alg. 1).  For dense A this is computed as
    sqrt(v_l^T B v_l), the same quantity.
  * Start vectors: x ~ N(0,1) of length min(m, n), one fresh draw per l, then
    x / ||x||; the draws are passed in (x_start) or taken from the Philox
    generator in oracle.philox.
  * A zero (or underflowing) B v0 means rank(A) < l: sigma_l = 0 and the
    returned vector is v0 made orthogonal to the earlier ones; status 'rank'.
  * Alg. 4 corrections: the batch sum forming X v0 runs over the n_b
    batches; the projection V^T v0 multiplies by V_j^T; the deflation term
    is Sigma^2 V^T v0; the last term of the update is (V Sigma^2 V^T v0)_j
    (as printed it repeats the third term).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox

RANK_TINY = 1e-30  # ||B v0|| below RANK_TINY * sigma_1^2 counts as zero (rank < l)


# ----------------------------------------------------------------------------
# Gram matrix B = A^T A  (Alg. 2: "B = X^T @ X"; Sec. IV, Sec. V-C)
# ----------------------------------------------------------------------------
def gram(A: np.ndarray) -> np.ndarray:
    """B = A^T A in FP64 from the stored values (library matmul as one step)."""
    A64 = np.asarray(A, dtype=np.float64)
    return A64.T @ A64


def gram_row_blocks(A: np.ndarray, block_rows: int) -> np.ndarray:
    """B = sum_b A_b^T A_b over contiguous row blocks (collinear batching, Sec. V-C)."""
    m, n = A.shape
    B = np.zeros((n, n), dtype=np.float64)
    for r0 in range(0, m, block_rows):
        Ab = np.asarray(A[r0:r0 + block_rows], dtype=np.float64)
        B += Ab.T @ Ab
    return B


def gram_plain(A: np.ndarray) -> np.ndarray:
    """B_ij = sum_r A_ri A_rj written out with loops (tiny inputs only)."""
    A64 = np.asarray(A, dtype=np.float64)
    m, n = A64.shape
    B = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(n):
            s = 0.0
            for r in range(m):
                s += A64[r, i] * A64[r, j]
            B[i, j] = s
    return B


# ----------------------------------------------------------------------------
# Alg. 2 inner loop
# ----------------------------------------------------------------------------
@dataclass
class PowerResult:
    v: np.ndarray
    iters: int
    status: str  # "ok" | "noconv" | "rank"
    cos_hist: list = field(default_factory=list)


def power_method(apply_B, v0: np.ndarray, eps: float, max_iter: int = 10000,
                 iters_override: int | None = None, scale: float = 1.0,
                 record: bool = False) -> PowerResult:
    """Alg. 2: v1 = B v0; v1 /= ||v1||; stop when |v0 . v1| >= 1 - eps.

    With iters_override the loop runs exactly that many applications and the
    test is skipped (convergence disabled).  `scale` is the magnitude used for
    the rank-deficiency check (sigma_1^2 of the matrix).
    """
    v0 = np.asarray(v0, dtype=np.float64)
    it = 0
    hist = []
    while True:
        w = apply_B(v0)
        it += 1
        nw = math.sqrt(float(w @ w))
        if not nw > RANK_TINY * max(scale, 1e-300):
            return PowerResult(v0, it, "rank", hist)
        v1 = w / nw
        c = abs(float(v0 @ v1))
        if record:
            hist.append(c)
        if iters_override is not None:
            if it >= iters_override:
                return PowerResult(v1, it, "ok", hist)
        else:
            if c >= 1.0 - eps:
                return PowerResult(v1, it, "ok", hist)
            if it >= max_iter:
                return PowerResult(v1, it, "noconv", hist)
        v0 = v1


def _normalise(x: np.ndarray) -> np.ndarray:
    """Alg. 2: x / ||x||."""
    x = np.asarray(x, dtype=np.float64)
    return x / math.sqrt(float(x @ x))


def _start(l: int, length: int, x_start, seed: int) -> np.ndarray:
    if x_start is not None:
        return _normalise(np.asarray(x_start)[:, l])
    return _normalise(philox.start_normals(seed, l, length))


def _orth_against(v: np.ndarray, V: np.ndarray) -> np.ndarray:
    if V.shape[1]:
        v = v - V @ (V.T @ v)
        v = v - V @ (V.T @ v)
    nv = math.sqrt(float(v @ v))
    return v / nv if nv > 0 else v


def _sign_fix(v: np.ndarray) -> float:
    """+1 or -1 so that the largest-magnitude entry (lowest index on ties) is positive."""
    i = int(np.argmax(np.abs(v)))
    return -1.0 if v[i] < 0 else 1.0


# ----------------------------------------------------------------------------
# O-1: Alg. 1 with Hotelling deflation, dense
# ----------------------------------------------------------------------------
@dataclass
class TSVDResult:
    U: np.ndarray
    sigma: np.ndarray
    V: np.ndarray
    iters: list
    status: list


def hotelling_apply(B: np.ndarray, V: np.ndarray, sigma2: np.ndarray):
    """v -> B v - V diag(sigma2) V^T v  (Eq. 2 with u_j = A v_j / sigma_j, exact v_j)."""
    def apply(v):
        w = B @ v
        if V.shape[1]:
            c = V.T @ v
            w = w - V @ (sigma2 * c)
        return w
    return apply


def tsvd_dense(A: np.ndarray, k: int, eps: float, x_start=None, seed: int = 0,
               max_iter: int = 10000, iters_override=None, sign_convention: bool = False,
               B: np.ndarray | None = None) -> TSVDResult:
    """Alg. 1 for dense A (m >= n: right vectors from B = A^T A; m < n: left
    vectors from B = A A^T, Eq. 3), deflating B in Hotelling form.

    x_start: optional (min(m,n) x k) start draws; iters_override: optional
    per-triplet application counts.  B may be passed in when already formed.
    """
    A64 = np.asarray(A, dtype=np.float64)
    m, n = A64.shape
    if k == -1:
        k = min(m, n)  # Alg. 1
    right = m >= n
    M = A64 if right else A64.T  # Eq. 3 is Eq. 2 applied to A^T
    if B is None:
        B = gram(M)
    sig, W, iters, status = right_vectors(B, k, eps, x_start, seed, max_iter, iters_override, sign_convention)
    # Alg. 1: the other factor from A and sigma (U for a tall A, V for a wide one)
    with np.errstate(divide="ignore", invalid="ignore"):
        other = (M @ W) / np.where(sig > 0, sig, np.inf)[None, :]
    if right:
        return TSVDResult(other, sig, W, iters, status)
    return TSVDResult(W, sig, other, iters, status)


def right_vectors(B: np.ndarray, k: int, eps: float, x_start=None, seed: int = 0, max_iter: int = 10000,
                  iters_override=None, sign_convention: bool = False):
    """The loop of Alg. 1 over l on a formed Gram matrix B (FP64): Alg. 2 for
    each triplet with B deflated in Hotelling form, sigma_l = sqrt(v_l^T B v_l).
    Returns (sigma, V, iters, status)."""
    d = B.shape[0]
    W = np.zeros((d, 0))
    sig = np.zeros(k)
    iters, status = [], []
    scale = None
    for l in range(k):
        v0 = _start(l, d, x_start, seed)
        it_l = None if iters_override is None else int(iters_override[l])
        res = power_method(hotelling_apply(B, W, sig[:l] ** 2), v0, eps, max_iter, it_l,
                           scale=1.0 if scale is None else scale)
        v = res.v
        if res.status == "rank":
            v = _orth_against(v0, W)
            s = 0.0
        else:
            s = math.sqrt(max(float(v @ (B @ v)), 0.0))  # sigma_l = ||M v_l|| (Alg. 1)
        if sign_convention:
            v = v * _sign_fix(v)
        if scale is None:
            scale = s * s
        sig[l] = s
        W = np.concatenate([W, v[:, None]], axis=1)
        iters.append(res.iters)
        status.append(res.status)
    return sig, W, iters, status


# ----------------------------------------------------------------------------
# CSR operators (Alg. 4 on one device: y = X v0, w = X^T y)
# ----------------------------------------------------------------------------
def csr_row_index(row_ptr: np.ndarray) -> np.ndarray:
    m = row_ptr.shape[0] - 1
    return np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))


def csr_matvec(row_ptr, col_idx, values, v, rows_of=None) -> np.ndarray:
    """y_r = sum_{p in row r} values_p * v[col_p], FP64."""
    m = row_ptr.shape[0] - 1
    if rows_of is None:
        rows_of = csr_row_index(row_ptr)
    prod = values.astype(np.float64) * np.asarray(v, dtype=np.float64)[col_idx]
    return np.bincount(rows_of, weights=prod, minlength=m)


def csr_rmatvec(row_ptr, col_idx, values, y, n: int, rows_of=None) -> np.ndarray:
    """w_c = sum_{p: col_p = c} values_p * y[row_p], FP64."""
    if rows_of is None:
        rows_of = csr_row_index(row_ptr)
    prod = values.astype(np.float64) * np.asarray(y, dtype=np.float64)[rows_of]
    return np.bincount(col_idx, weights=prod, minlength=n)


def tsvd_csr(csr: dict, k: int, eps: float, x_start=None, seed: int = 0, max_iter: int = 10000,
             iters_override=None, sign_convention: bool = False) -> TSVDResult:
    """Alg. 1 for a CSR matrix with m >= n, never forming B: each application
    is w = A^T (A v0) - V diag(sigma^2) V^T v0 (the Alg. 4 operator in the
    Hotelling form), and sigma_l = ||A v_l|| (Alg. 1)."""
    row_ptr, col_idx, values = csr["row_ptr"], csr["col_idx"], csr["values"]
    m, n = csr["m"], csr["n"]
    assert m >= n, "the CSR oracle covers the m >= n branch"
    if k == -1:
        k = min(m, n)
    rows_of = csr_row_index(row_ptr)
    W = np.zeros((n, 0))
    sig = np.zeros(k)
    iters, status = [], []
    scale = None
    for l in range(k):
        v0 = _start(l, n, x_start, seed)
        s2 = sig[:l] ** 2
        Wl = W

        def apply(v, Wl=Wl, s2=s2):
            w = csr_rmatvec(row_ptr, col_idx, values, csr_matvec(row_ptr, col_idx, values, v, rows_of),
                            n, rows_of)
            if Wl.shape[1]:
                w = w - Wl @ (s2 * (Wl.T @ v))
            return w
        it_l = None if iters_override is None else int(iters_override[l])
        res = power_method(apply, v0, eps, max_iter, it_l, scale=1.0 if scale is None else scale)
        v = res.v
        if res.status == "rank":
            v = _orth_against(v0, W)
            s = 0.0
        else:
            y = csr_matvec(row_ptr, col_idx, values, v, rows_of)
            s = math.sqrt(float(y @ y))
        if sign_convention:
            v = v * _sign_fix(v)
        if scale is None:
            scale = s * s
        sig[l] = s
        W = np.concatenate([W, v[:, None]], axis=1)
        iters.append(res.iters)
        status.append(res.status)
    AV = np.stack([csr_matvec(row_ptr, col_idx, values, W[:, j], rows_of) for j in range(k)], axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        U = AV / np.where(sig > 0, sig, np.inf)[None, :]
    return TSVDResult(U, sig, W, iters, status)


# ----------------------------------------------------------------------------
# O-2: Alg. 1 and Alg. 2 as printed, with the explicit residual
# ----------------------------------------------------------------------------
def tsvd_literal(A: np.ndarray, k: int, eps: float, x_start=None, seed: int = 0,
                 max_iter: int = 10000, iters_override=None) -> TSVDResult:
    """Alg. 1: for each l, X = A - U[:l] diag(sigma[:l]) V[:l]^T (l.7-9),
    v_l = SVD_1D(X) with B = X^T X (Alg. 2), u_l = A v_l, sigma_l = ||u_l||,
    u_l /= sigma_l (l.11-13); the m < n branch swaps the roles (l.15-17)."""
    A64 = np.asarray(A, dtype=np.float64)
    m, n = A64.shape
    if k == -1:
        k = min(m, n)
    U = np.zeros((m, 0))
    V = np.zeros((n, 0))
    sig = np.zeros(0)
    iters, status = [], []
    for l in range(k):
        X = A64 - (U * sig[None, :]) @ V.T
        if m >= n:
            B = X.T @ X
            v0 = _start(l, n, x_start, seed)
            it_l = None if iters_override is None else int(iters_override[l])
            res = power_method(lambda v: B @ v, v0, eps, max_iter, it_l)
            v = res.v
            u = A64 @ v
            s = math.sqrt(float(u @ u))
            u = u / s
        else:
            B = X @ X.T
            u0 = _start(l, m, x_start, seed)
            it_l = None if iters_override is None else int(iters_override[l])
            res = power_method(lambda v: B @ v, u0, eps, max_iter, it_l)
            u = res.v
            v = A64.T @ u
            s = math.sqrt(float(v @ v))
            v = v / s
        U = np.concatenate([U, u[:, None]], axis=1)
        V = np.concatenate([V, v[:, None]], axis=1)
        sig = np.append(sig, s)
        iters.append(res.iters)
        status.append(res.status)
    return TSVDResult(U, sig, V, iters, status)


# ----------------------------------------------------------------------------
# Eq. 1-3 and Alg. 4, for the algebraic identity checks
# ----------------------------------------------------------------------------
def eq1_gram(X, U, S, V):
    """Eq. 1: X'^T X' = X^T X - V S U^T X - X^T U S V^T + V S^2 V^T  (needs U^T U = I)."""
    X = np.asarray(X, dtype=np.float64)
    Sm = np.diag(S)
    return X.T @ X - V @ Sm.T @ U.T @ X - X.T @ U @ Sm @ V.T + V @ (Sm @ Sm) @ V.T


def eq2_apply(X, U, S, V, v0):
    """Eq. 2, evaluated right to left (matrix-vector products only), m > n."""
    X = np.asarray(X, dtype=np.float64)
    Xv0 = X @ v0
    t1 = X.T @ Xv0
    t2 = V @ (S * (U.T @ Xv0))
    t3 = X.T @ (U @ (S * (V.T @ v0)))
    t4 = V @ (S * S * (V.T @ v0))
    return t1 - t2 - t3 + t4


def eq3_apply(X, U, S, V, v0):
    """Eq. 3 (m < n): X X^T v0 - U S V^T X^T v0 - X V S U^T v0 + U S^2 U^T v0."""
    X = np.asarray(X, dtype=np.float64)
    Xtv0 = X.T @ v0
    t1 = X @ Xtv0
    t2 = U @ (S * (V.T @ Xtv0))
    t3 = X @ (V @ (S * (U.T @ v0)))
    t4 = U @ (S * S * (U.T @ v0))
    return t1 - t2 - t3 + t4


def dist_compute_v0(X, U, S, V, v0, n_b: int, N: int):
    """Alg. 4 (m >= n) with its typos corrected: X split into N row partitions
    (one per GPU, index i) and n_b column batches (index j); U follows the row
    partition, V and v0 the column batches.  Returns v1 = Eq. 2's right side."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    rows = np.array_split(np.arange(m), N)
    cols = np.array_split(np.arange(n), n_b)
    # (X v0)_i = sum_j X_ij (v0)_j
    Xv0 = [sum(X[np.ix_(ri, cj)] @ v0[cj] for cj in cols) for ri in rows]
    # (X^T X v0)_j = sum_i X_ij^T (X v0)_i   (all-reduce over i)
    XtXv0 = [sum(X[np.ix_(ri, cj)].T @ Xv0[a] for a, ri in enumerate(rows)) for cj in cols]
    # U^T X v0 = sum_i U_i^T (X v0)_i        (all-reduce over i)
    UtXv0 = sum(U[ri].T @ Xv0[a] for a, ri in enumerate(rows))
    # (V S^T U^T X v0)_j
    VSUtXv0 = [V[cj] @ (S * UtXv0) for cj in cols]
    # V^T v0 = sum_j V_j^T (v0)_j, then S V^T v0
    SVtv0 = S * sum(V[cj].T @ v0[cj] for cj in cols)
    # (X^T U S V^T v0)_j = sum_i X_ij^T (U S V^T v0)_i
    USVtv0 = [U[ri] @ SVtv0 for ri in rows]
    XtUSVtv0 = [sum(X[np.ix_(ri, cj)].T @ USVtv0[a] for a, ri in enumerate(rows)) for cj in cols]
    # (V S^2 V^T v0)_j (the corrected deflation term)
    VS2Vtv0 = [V[cj] @ (S * SVtv0) for cj in cols]
    # the update with its corrected last term
    out = np.empty(n)
    for b, cj in enumerate(cols):
        out[cj] = XtXv0[b] - VSUtXv0[b] - XtUSVtv0[b] + VS2Vtv0[b]
    return out


# ----------------------------------------------------------------------------
# Checks used by the tests (closed forms, invariants)
# ----------------------------------------------------------------------------
def subspace_angle(a: np.ndarray, b: np.ndarray) -> float:
    """Largest principal angle between span(a) and span(b), both of the same
    dimension (columns).  With Qa, Qb orthonormal bases, sin of the angle is
    the 2-norm of the part of Qb outside span(a), ||Qb - Qa Qa^T Qb||_2, and
    its cos the smallest singular value of Qa^T Qb; atan2 of the pair keeps
    full relative accuracy at tiny angles, where acos of the cosine alone
    loses about half the digits (Bjorck & Golub 1973; Knyazev & Argentati
    2002 for the sine form)."""
    a = np.atleast_2d(np.asarray(a, dtype=np.float64).T).T
    b = np.atleast_2d(np.asarray(b, dtype=np.float64).T).T
    qa, _ = np.linalg.qr(a)
    qb, _ = np.linalg.qr(b)
    c = float(np.linalg.svd(qa.T @ qb, compute_uv=False).min())
    s = float(np.linalg.norm(qb - qa @ (qa.T @ qb), 2))
    return float(math.atan2(s, c))


def vector_angle(a: np.ndarray, b: np.ndarray) -> float:
    """Sign-invariant angle between two vectors, accurate for tiny angles."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    a = a / np.linalg.norm(a); b = b / np.linalg.norm(b)
    if a @ b < 0:
        b = -b
    return float(2.0 * math.asin(min(1.0, np.linalg.norm(a - b) / 2.0)))


def frobenius_residual_sq(A, U, sigma, V) -> float:
    """||A - U diag(sigma) V^T||_F^2 in FP64 (small inputs)."""
    A64 = np.asarray(A, dtype=np.float64)
    R = A64 - (U * sigma[None, :]) @ V.T
    return float(np.sum(R * R))


def gapped_indices(lam: np.ndarray, k: int, rel_gap: float = 0.05) -> list:
    """Indices i < k whose eigenvalue lam_i has relative gap >= rel_gap to both neighbours."""
    out = []
    for i in range(k):
        left = lam[i - 1] - lam[i] if i > 0 else np.inf
        right = lam[i] - lam[i + 1] if i + 1 < lam.shape[0] else np.inf
        if lam[i] > 0 and min(left, right) / lam[i] >= rel_gap:
            out.append(i)
    return out
