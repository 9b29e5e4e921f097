"""Brute-force one-sided Jacobi SVD (Hestenes), for tiny matrices.

TEST INFRASTRUCTURE ONLY: part of the FP64 oracle, used to pin it.  Textbook
method (Hestenes 1958; Golub & Van Loan, "Matrix Computations", one-sided
Jacobi): rotate column pairs of W = A until every pair is orthogonal; then the
column norms are the singular values, the normalised columns the left vectors
and the accumulated rotations the right vectors.  Independent of the power
method, so it checks the oracle's results from outside.
"""
from __future__ import annotations

import math
import numpy as np


def jacobi_svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = float(W[:, p] @ W[:, p])
                beta = float(W[:, q] @ W[:, q])
                gamma = float(W[:, p] @ W[:, q])
                if gamma == 0.0 or abs(gamma) <= tol * math.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                wp, wq = W[:, p].copy(), W[:, q].copy()
                W[:, p] = c * wp - s * wq
                W[:, q] = s * wp + c * wq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if not rotated:
            break
    sigma = np.sqrt(np.sum(W * W, axis=0))
    order = np.argsort(-sigma, kind="stable")
    sigma = sigma[order]
    V = V[:, order]
    W = W[:, order]
    U = np.zeros_like(W)
    nz = sigma > 0
    U[:, nz] = W[:, nz] / sigma[nz][None, :]
    return U, sigma, V
