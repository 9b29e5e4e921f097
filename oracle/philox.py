"""Philox-4x32-10 counter-based generator and the start-vector draw, in NumPy.

TEST INFRASTRUCTURE ONLY: part of the FP64 oracle.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this package.

The generator follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2): a 4 x 32-bit
counter and a 2 x 32-bit key, ten rounds; each round multiplies words 0 and 2
by fixed odd constants, keeps the 64-bit products' high and low halves, and
mixes the high halves with the other two words and the round key; the key is
bumped by two Weyl constants between rounds.

The start vector of the power method (Algorithm 2: x ~ N(0, 1) of length
min(m, n), then x / ||x||) is drawn from it with the Box-Muller transform in
FP64.  Counter layout used by both this oracle and the CUDA library:
    counter = (p mod 2^32, p div 2^32, l, 0x54535644), p = pair index i // 2
    key     = (lo32(s), hi32(s)), s = splitmix64(seed)
    u1 = ((x0 << 32 | x1) >> 11 + 1) * 2^-53     in (0, 1]
    u2 = ((x2 << 32 | x3) >> 11) * 2^-53         in [0, 1)
    x[2p]   = sqrt(-2 ln u1) cos(2 pi u2)
    x[2p+1] = sqrt(-2 ln u1) sin(2 pi u2)
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
TSVD_TAG = 0x54535644  # "TSVD" in ASCII, fourth counter word
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr: (..., 4) uint32, key: (2,) or (..., 2) uint32 -> (..., 4) uint32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    key = np.asarray(key, dtype=np.uint32)
    k0 = np.broadcast_to(key[..., 0], c[0].shape).astype(np.uint64)
    k1 = np.broadcast_to(key[..., 1], c[0].shape).astype(np.uint64)
    for rnd in range(10):
        if rnd:  # key schedule: Weyl increments modulo 2^32
            k0 = (k0 + np.uint64(PHILOX_W0)) & MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & MASK32
        p0 = PHILOX_M0 * c[0]  # exact: both factors < 2^32
        p1 = PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA'14): one output for state x."""
    z = (int(x) + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def philox_words(seed: int, l: int, pairs: int) -> np.ndarray:
    """Raw generator output for pair indices 0..pairs-1 of vector l: (pairs, 4) uint32."""
    s = splitmix64(seed)
    key = np.array([s & 0xFFFFFFFF, s >> 32], dtype=np.uint32)
    p = np.arange(pairs, dtype=np.uint64)
    ctr = np.empty((pairs, 4), dtype=np.uint32)
    ctr[:, 0] = (p & MASK32).astype(np.uint32)
    ctr[:, 1] = (p >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(l & 0xFFFFFFFF)
    ctr[:, 3] = np.uint32(TSVD_TAG)
    return philox4x32_10(ctr, key)


def start_normals(seed: int, l: int, n: int) -> np.ndarray:
    """x ~ N(0, 1)^n for vector index l (0-based), FP64, Box-Muller."""
    pairs = (n + 1) // 2
    w = philox_words(seed, l, pairs).astype(np.uint64)
    a = (w[:, 0] << np.uint64(32)) | w[:, 1]
    b = (w[:, 2] << np.uint64(32)) | w[:, 3]
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (b >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    x = np.empty(2 * pairs, dtype=np.float64)
    x[0::2] = rad * np.cos(ang)
    x[1::2] = rad * np.sin(ang)
    return x[:n]
