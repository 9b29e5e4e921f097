"""Seeded synthetic inputs for the truncated-SVD workloads.

This module only draws random numbers and lays them out; it contains none of
the method's arithmetic (no Gram products, no power iterations, no deflation).
Both the FP64 oracle and the GPU library consume the arrays it returns, so the
two sides always see byte-identical inputs.

Workload shapes follow the paper's synthetic experiments (Sec. V-D, the dense
and sparse scaling matrices and the out-of-memory sparse run): dense FP32
matrices with a prescribed spectrum plus Gaussian noise, and CSR matrices with
uniformly random column positions and U(0,1) values.  The paper uses no public
dataset; these generators stand in for its randomly generated matrices.

Two back ends exist for the dense generator:
  * NumPy (CPU), used by the tests and by every size the oracle can handle;
  * PyTorch on a CUDA device (``dense_lowrank_blocks_torch``), used only to
    fill very large pinned host buffers quickly.  It is seeded as well, but it
    draws from torch's device generator, so its values differ from the NumPy
    back end for the same seed.  The oracle checks such runs on the host
    buffer that was actually produced, never on a regeneration.
"""
from __future__ import annotations

import math
import numpy as np

__all__ = [
    "orthonormal_columns",
    "dense_prescribed",
    "spectrum_geometric",
    "spectrum_harmonic",
    "spectrum_harmonic_clustered",
    "dense_lowrank_rows",
    "csr_uniform",
    "csr_from_dense",
    "start_normals",
    "dense_lowrank_blocks_torch",
    "csr_uniform_torch",
    "stacked_factor",
    "stacked_rows_torch",
    "serving_shapes",
    "serving_matrix_torch",
]


def _rng(seed: int, *stream: int) -> np.random.Generator:
    """Independent Philox stream per (seed, *stream) tuple."""
    ss = np.random.SeedSequence([int(seed) & 0xFFFFFFFF, *[int(s) & 0xFFFFFFFF for s in stream]])
    return np.random.Generator(np.random.Philox(ss))


def orthonormal_columns(rows: int, cols: int, seed: int, stream: int = 0) -> np.ndarray:
    """Q factor of a seeded Gaussian rows x cols matrix (FP64), rows >= cols."""
    g = _rng(seed, 101, stream).standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    # fix the sign so that the factor is a deterministic function of the seed
    q *= np.sign(np.diag(r))[None, :]
    return q


def spectrum_geometric(count: int, rho: float) -> np.ndarray:
    """sigma_i = rho**i, i = 0..count-1 (0-based: sigma_0 = 1)."""
    return rho ** np.arange(count, dtype=np.float64)


def spectrum_harmonic(count: int) -> np.ndarray:
    """sigma_i = 1/(1+i), i = 0..count-1."""
    return 1.0 / (1.0 + np.arange(count, dtype=np.float64))


def spectrum_harmonic_clustered(count: int, i0: int = 10, gap: float = 1e-3) -> np.ndarray:
    """Harmonic spectrum whose pair (i0, i0+1) is pulled to an absolute gap."""
    s = spectrum_harmonic(count)
    s[i0 + 1] = s[i0] - gap
    return s


def dense_prescribed(m: int, n: int, sigma: np.ndarray, noise: float, seed: int) -> dict:
    """A = U diag(sigma) V^T + noise * N(0,1), built in FP64, stored as FP32.

    U (m x r) and V (n x r) have orthonormal columns (QR of seeded Gaussians),
    r = len(sigma) <= min(m, n).  Returns the FP32 matrix (row-major) together
    with the FP64 construction factors.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    assert r <= min(m, n)
    U = orthonormal_columns(m, r, seed, 0)
    V = orthonormal_columns(n, r, seed, 1)
    A = (U * sigma[None, :]) @ V.T
    if noise:
        A += noise * _rng(seed, 202).standard_normal((m, n))
    return {"A": np.ascontiguousarray(A, dtype=np.float32), "U": U, "V": V, "sigma": sigma}


def dense_lowrank_rows(r0: int, r1: int, V: np.ndarray, sigma: np.ndarray, m_total: int,
                       noise: float, seed: int) -> np.ndarray:
    """Rows [r0, r1) of a rank-r matrix with a roughly prescribed spectrum.

    Row i is (g_i / sqrt(m_total)) diag(sigma) V^T + noise * e_i, where g_i is a
    seeded standard-normal r-vector drawn from a stream keyed on the row block,
    so that any block can be regenerated on its own.  The left factor is only
    approximately orthonormal (deviation ~ sqrt(r / m_total)); the singular
    values of the result are therefore taken from the data, never from sigma.
    """
    rows = r1 - r0
    r = sigma.shape[0]
    g = _rng(seed, 303, r0).standard_normal((rows, r)) / math.sqrt(m_total)
    A = (g * sigma[None, :]) @ V.T
    if noise:
        A += noise * _rng(seed, 404, r0).standard_normal((rows, V.shape[0]))
    return np.ascontiguousarray(A, dtype=np.float32)


def csr_uniform(m: int, n: int, nnz_per_row: float, seed: int, values: str = "uniform") -> dict:
    """Random CSR matrix: per-row nnz ~ Poisson(nnz_per_row) (capped at n),
    columns uniform without replacement and sorted, values U(0,1) in FP32.

    row_ptr is int64, col_idx int32, values float32 (the layout the library
    consumes).  Poisson(n*delta) approximates Binomial(n, delta) for the
    paper's densities.
    """
    rng = _rng(seed, 505)
    counts = np.minimum(rng.poisson(nnz_per_row, size=m), n).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    cols = np.empty(nnz, dtype=np.int64)
    # draw with replacement, then redraw rows that happen to repeat a column
    cols[:] = rng.integers(0, n, size=nnz)
    rows_of = np.repeat(np.arange(m, dtype=np.int64), counts)
    key = rows_of * n + cols
    key.sort()
    dup = np.nonzero(key[1:] == key[:-1])[0]
    if dup.size:
        bad_rows = np.unique(key[dup + 1] // n)
        for rr in bad_rows:
            a, b = row_ptr[rr], row_ptr[rr + 1]
            key[a:b] = rr * n + np.sort(rng.choice(n, size=b - a, replace=False))
    col_idx = (key - rows_of * n).astype(np.int32)
    if values == "uniform":
        vals = rng.random(nnz, dtype=np.float32)
    elif values == "normal":
        vals = rng.standard_normal(nnz).astype(np.float32)
    else:
        raise ValueError(values)
    return {"row_ptr": row_ptr, "col_idx": col_idx, "values": vals, "m": m, "n": n}


def csr_from_dense(A: np.ndarray) -> dict:
    """Exact CSR image of a dense FP32 matrix (zeros dropped, columns sorted)."""
    A = np.asarray(A, dtype=np.float32)
    m, n = A.shape
    mask = A != 0
    counts = mask.sum(axis=1).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    r, c = np.nonzero(mask)
    return {"row_ptr": row_ptr, "col_idx": c.astype(np.int32), "values": A[r, c].astype(np.float32),
            "m": m, "n": n}


def start_normals(n: int, k: int, seed: int) -> np.ndarray:
    """k seeded standard-normal start draws of length n, FP64, column-major (n x k).

    These are the N(0, 1) samples the power method starts from; passing them
    to both sides makes the GPU path and the oracle follow one trajectory.
    """
    x = _rng(seed, 606).standard_normal((k, n))
    return np.asfortranarray(x.T)


def dense_lowrank_blocks_torch(out_host, m: int, n: int, rank: int, sigma: np.ndarray, noise: float,
                               seed: int, block_rows: int, device="cuda"):
    """Fill an FP32 buffer (m x n row-major; pinned host memory or a device
    tensor) with the rank-r plus noise workload, generating each row block on
    the GPU with torch.

    Left factor: seeded Gaussian (m x r) made orthonormal by two rounds of
    Cholesky QR over the whole height (the Gaussian stays on the device, 4 B
    per entry).  Right factor: QR of a seeded Gaussian (n x r).  Each row
    block is then U_b diag(sigma) V^T + noise * N(0,1), copied to the host.
    Returns the FP64 factors on the host for reference.
    """
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 1000003 + 17)
    Ug = torch.randn((m, rank), generator=gen, device=dev, dtype=torch.float32)
    for _ in range(2):  # CholeskyQR2: U <- U R^{-1}, twice, FP64 Gram (small factorisations on the host)
        W = torch.zeros((rank, rank), dtype=torch.float64, device=dev)
        for r0 in range(0, m, block_rows):
            Ub = Ug[r0:r0 + block_rows].double()
            W += Ub.T @ Ub
        R = np.linalg.cholesky(W.cpu().numpy()).T  # upper
        Rinv = torch.as_tensor(np.linalg.inv(R), device=dev)
        for r0 in range(0, m, block_rows):
            Ug[r0:r0 + block_rows] = (Ug[r0:r0 + block_rows].double() @ Rinv).float()
    gv = torch.Generator(device=dev)
    gv.manual_seed(int(seed) * 1000003 + 29)
    Vg = torch.randn((n, rank), generator=gv, device=dev, dtype=torch.float64).cpu().numpy()
    Vq_np, Vr_np = np.linalg.qr(Vg)
    Vq_np = Vq_np * np.sign(np.diag(Vr_np))[None, :]
    Vq = torch.as_tensor(Vq_np, device=dev)
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=dev)
    SVt = (sig[:, None] * Vq.T).float()  # r x n
    gn = torch.Generator(device=dev)
    gn.manual_seed(int(seed) * 1000003 + 41)
    buf = torch.empty((block_rows, n), dtype=torch.float32, device=dev)
    for r0 in range(0, m, block_rows):
        r1 = min(m, r0 + block_rows)
        b = buf[: r1 - r0]
        torch.randn(b.shape, generator=gn, device=dev, dtype=torch.float32, out=b)
        b.mul_(noise)
        b.addmm_(Ug[r0:r1], SVt)
        out_host[r0:r1].copy_(b, non_blocking=False)
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)
    return {"V": Vq_np, "sigma": np.asarray(sigma, dtype=np.float64)}


def csr_uniform_torch(m: int, n: int, nnz_per_row: float, seed: int, device="cuda"):
    """CSR matrix like csr_uniform, drawn on the GPU with torch (for sizes
    where the NumPy generator is too slow): per-row nnz ~ Poisson(nnz_per_row),
    columns uniform without replacement and sorted (rows that drew a repeated
    column redraw it until none repeat), values U(0,1) FP32.  Returns torch
    tensors on `device` (row_ptr int64, col_idx int32, values float32)."""
    import torch
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed) * 7919 + 3)
    rate = torch.full((m,), float(nnz_per_row), dtype=torch.float32, device=dev)
    counts = torch.poisson(rate, generator=g).to(torch.int64).clamp_(max=n)
    row_ptr = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    torch.cumsum(counts, 0, out=row_ptr[1:])
    nnz = int(row_ptr[-1].item())
    rows = torch.repeat_interleave(torch.arange(m, device=dev, dtype=torch.int64), counts)
    cols = torch.randint(0, n, (nnz,), generator=g, device=dev, dtype=torch.int64)
    for _ in range(64):
        key = rows * n + cols
        key, _ = torch.sort(key)
        cols = key - rows * n  # rows is already non-decreasing, so it stays aligned
        dup = torch.zeros(nnz, dtype=torch.bool, device=dev)
        if nnz > 1:
            dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum().item())
        if nd == 0:
            break
        cols[dup] = torch.randint(0, n, (nd,), generator=g, device=dev, dtype=torch.int64)
        del key
    vals = torch.rand(nnz, generator=g, device=dev, dtype=torch.float32)
    return {"row_ptr": row_ptr, "col_idx": cols.to(torch.int32), "values": vals, "m": m, "n": n}


def stacked_factor(n: int, sigma: np.ndarray, copies: int, seed: int) -> dict:
    """Generator matrix of the stacked-orthogonal dense workload (copies * n rows).

    A = stack_b (S_b P_b) M with M = fl32(W diag(sigma) V^T / sqrt(copies)),
    W and V the Q factors of two seeded n x n Gaussians, P_b a random row
    permutation and S_b random signs per block (drawn by stacked_rows_torch).
    U = stack_b S_b P_b W / sqrt(copies) has orthonormal columns exactly
    (sum_b W^T P_b^T S_b S_b P_b W / copies = I), so the singular values of A
    are sigma up to the FP32 rounding of M, its right singular vectors are the
    columns of V, and A^T A = copies * M^T M exactly (a row permutation and
    signs leave each block's Gram M^T M unchanged).  Returns M (FP32), V, sigma.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    W = orthonormal_columns(n, n, seed, stream=7)
    V = orthonormal_columns(n, n, seed, stream=8)
    M = (W * sigma[None, :]) @ V.T
    M *= 1.0 / math.sqrt(copies)
    return {"M32": M.astype(np.float32), "V": V, "sigma": sigma, "copies": int(copies)}


def stacked_rows_torch(out, M32: np.ndarray, seed: int):
    """Fill `out` (a torch FP32 tensor of copies * n rows and n columns, on any
    device) with the stacked workload of stacked_factor: rows [b n, (b+1) n)
    are M32 with its rows permuted and signs flipped at random (torch
    generator of out's device, seeded)."""
    import torch
    n = M32.shape[0]
    m = out.shape[0]
    if m % n or out.shape[1] != n:
        raise ValueError("out must have a multiple of n rows and n columns")
    dev = out.device
    Md = torch.as_tensor(np.ascontiguousarray(M32), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed) * 1000003 + 53)
    for b in range(m // n):
        perm = torch.randperm(n, generator=g, device=dev)
        sgn = torch.randint(0, 2, (n,), generator=g, device=dev).to(torch.float32).mul_(2.0).sub_(1.0)
        torch.mul(Md[perm], sgn[:, None], out=out[b * n:(b + 1) * n])
    return out


def serving_shapes(count: int, seed: int, m_range=(512, 65536), n_range=(64, 2048), rho_range=(0.5, 0.95),
                   tail: float = 1e-12) -> list:
    """Shapes of the serving pool: m and n log-uniform in their ranges, a
    geometric spectrum sigma_i = rho^i with rho uniform, truncated to the
    rank where rho^i < tail (and to min(m, n))."""
    g = _rng(seed, 707)
    out = []
    for _ in range(count):
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        rho = float(g.uniform(*rho_range))
        r = min(min(m, n), int(math.ceil(math.log(tail) / math.log(rho))))
        out.append({"m": m, "n": n, "rho": rho, "rank": r})
    return out


def serving_sparse_shapes(count: int, seed: int, dim_range=(1 << 14, 1 << 16), density: float = 1e-4) -> list:
    """Square sparse requests of the serving mix: m = n log-uniform in
    dim_range, density as given (entries per row = density * n)."""
    g = _rng(seed, 708)
    out = []
    for _ in range(count):
        m = int(round(math.exp(g.uniform(math.log(dim_range[0]), math.log(dim_range[1])))))
        out.append({"m": m, "n": m, "nnz_per_row": density * m})
    return out


def serving_matrix_torch(shape: dict, seed: int, out=None, device="cuda"):
    """A = Q1 diag(rho^i) Q2^T (exact rank r, no noise) for one pool entry:
    Q1 (m x r) and Q2 (n x r) the Q factors of seeded Gaussians, formed on
    the GPU in FP64 and rounded to FP32 once.  Written into `out` (an m x n
    FP32 array or tensor) when given.  The singular values are rho^i, i < r,
    up to that rounding."""
    import torch
    m, n, r, rho = shape["m"], shape["n"], shape["rank"], shape["rho"]
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed) * 1000003 + 97)

    def orth(rows):
        # CholeskyQR2 (two rounds): the r x r Cholesky factor and its inverse on
        # the host, the tall products on the GPU (no device LAPACK needed)
        q = torch.randn((rows, r), generator=g, device=dev, dtype=torch.float64)
        for _ in range(2):
            R = np.linalg.cholesky((q.T @ q).cpu().numpy()).T
            q = q @ torch.as_tensor(np.linalg.inv(R), device=dev)
        return q
    q1 = orth(m)
    q2 = orth(n)
    sig = torch.as_tensor(rho ** np.arange(r, dtype=np.float64), device=dev)
    A = ((q1 * sig[None, :]) @ q2.T).to(torch.float32)
    if out is not None:
        if isinstance(out, np.ndarray):
            out[:] = A.cpu().numpy()
        else:
            out.copy_(A)
        return out
    return A
