"""The t-SVD server (continuous batching) against the oracle, through the C ABI.

Every request runs the same method as tsvd_factor (Alg. 1/2 with Hotelling
deflation; Eq. 3 when m < n) with the built-in Philox start draws of its seed,
which the oracle draws too.  Parity is graded on the same trajectory: the
oracle runs first and its application counts are forced on the server
(iters_override), as for tsvd_factor.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import tsvd_ref as ref
from paper_2208_08410_gb300 import Server, _binding as B

pytestmark = pytest.mark.gpu


def _pinned(shape, dtype):
    ptr = C.c_void_p()
    nbytes = max(int(np.prod(shape)) * np.dtype(dtype).itemsize, 16)
    B.check(B.tsvd_host_alloc(C.byref(ptr), nbytes), "tsvd_host_alloc")
    ctype = {np.float32: C.c_float, np.float64: C.c_double}[dtype]
    return ptr, np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=shape)


class Pool:
    """Page-locked inputs and outputs of a set of requests."""

    def __init__(self):
        self.ptrs = []

    def arr(self, shape, dtype):
        p, a = _pinned(shape, dtype)
        self.ptrs.append(p)
        return a

    def close(self):
        for p in self.ptrs:
            B.tsvd_host_free(p)


def _request(pool, m, n, rho, seed, noise=1e-7):
    d = min(m, n)
    sig = synth.spectrum_geometric(d, rho)
    A = synth.dense_prescribed(max(m, n), d, sig, noise, seed=seed)["A"]
    A = A if m >= n else np.ascontiguousarray(A.T)
    hA = pool.arr((m, n), np.float32)
    hA[:] = A
    return hA


def _outputs(pool, m, n, k):
    return pool.arr((k, m), np.float32), pool.arr((k,), np.float64), pool.arr((k, n), np.float32)


# m, n, k, rho: sigma_{k-1} / sigma_0 = rho^(k-1) stays above ~0.04, inside the envelope where an
# FP32-accumulated Gram and FP32 iterate resolve sigma to 1e-5.  The other factor (U = A V / sigma
# for tall requests) carries V's error along the larger triplets amplified by sigma_0 / sigma_l, so
# its 1e-4 angle needs the same margin (at sigma_16 / sigma_0 = 0.028 a 70 x 70 request's u_16 was
# 2.3e-4 off while v_16 passed)
CASES = [
    (3000, 64, 8, 0.7), (512, 200, 12, 0.8), (4096, 700, 16, 0.85), (300, 1000, 10, 0.75),
    (2048, 2048, 6, 0.6), (9000, 130, 32, 0.9), (70, 70, 12, 0.8), (1500, 5, 5, 0.5),
]


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("tc_min_d", [256, 64, 1 << 62])
def test_server_mixed_wave_matches_oracle(tc_min_d, graphs):
    """A wave of tall and wide requests of many sizes follows the oracle's
    trajectory.  The tensor-core threshold puts the Gram step of requests with
    d >= 256 (the default), of every request with d >= 64, or of none on the
    grouped tcgen05 SYRK; the others take the CUDA-core SYRK.  The waves are
    launched directly (the default) or as CUDA graphs."""
    B.load()
    pool = Pool()
    sv = Server(device_budget=4 << 30, n_streams=2, wave_graphs=graphs)
    sv.set_tc_min_d(tc_min_d)
    assert sv.tc_min_d() == tc_min_d
    try:
        eps = 1e-10
        jobs = []
        for i, (m, n, k, rho) in enumerate(CASES):
            A = _request(pool, m, n, rho, seed=100 + i)
            U, s, V = _outputs(pool, m, n, k)
            o = ref.tsvd_dense(A, k, eps, seed=7 + i)
            t = sv.submit(A, k, eps, U, s, V, seed=7 + i, iters_override=o.iters)
            jobs.append((t, A, k, U, s, V, o))
        for t, A, k, U, s, V, o in jobs:
            st, info = sv.wait(t, 120.0)
            assert st == B.TSVD_OK, (st, sv.last_error())
            assert np.max(np.abs(s - o.sigma) / o.sigma) <= 1e-5
            assert info["applications"] == sum(o.iters)
            m, n = A.shape
            gapped = ref.gapped_indices(o.sigma ** 2, k)
            assert gapped == list(range(k)), gapped  # geometric, rho <= 0.9: every gap >= 0.19
            # U is m x k and V is n x k, column-major (stored as k rows)
            for l in gapped:
                assert ref.vector_angle(V[l].astype(np.float64), o.V[:, l]) <= 1e-4, (m, n, l)
                assert ref.vector_angle(U[l].astype(np.float64), o.U[:, l]) <= 1e-4, (m, n, l)
        stats = sv.stats()
        assert stats["completed"] == len(CASES) and stats["failed"] == 0
        assert stats["kernel_launches"] >= 3
        if graphs:  # every wave ran as a CUDA graph: updated in place or instantiated
            assert stats["graph_updates"] + stats["graph_instantiations"] == stats["waves"] >= 1
        else:
            assert stats["graph_updates"] + stats["graph_instantiations"] == 0 and stats["waves"] >= 1
    finally:
        sv.close()
        pool.close()


def test_server_result_alone_equals_result_in_the_mix():
    """Grouped kernels take no atomics and a request's cluster size depends on
    its own shape only, so its outputs are bitwise the same in any wave.  The
    request runs alone in a directly launched wave and in the mix in waves
    launched as CUDA graphs, so this also shows both launch forms agree."""
    B.load()
    pool = Pool()
    m, n, k = 2500, 300, 10
    A = _request(pool, m, n, 0.8, seed=5)
    alone = _outputs(pool, m, n, k)
    sv = Server(device_budget=2 << 30)
    try:
        assert sv.tc_min_d() <= n  # this request's Gram step runs on the tensor-core SYRK
        st, _ = sv.wait(sv.submit(A, k, 1e-9, *alone, seed=3), 60.0)
        assert st == B.TSVD_OK
    finally:
        sv.close()
    sv = Server(device_budget=4 << 30, n_streams=3, max_wave=16, wave_graphs=True)
    mix = _outputs(pool, m, n, k)
    tickets = []
    try:
        rng = np.random.default_rng(0)
        for i in range(40):
            mm, nn = int(rng.integers(64, 3000)), int(rng.integers(64, 900))
            kk = int(rng.integers(1, min(mm, nn, 32) + 1))
            Ai = _request(pool, mm, nn, float(rng.uniform(0.5, 0.9)), seed=1000 + i)
            tickets.append(sv.submit(Ai, kk, 1e-9, *_outputs(pool, mm, nn, kk), seed=i))
            if i == 17:
                t_mix = sv.submit(A, k, 1e-9, *mix, seed=3)
        for t in tickets:
            st, _ = sv.wait(t, 120.0)
            assert st in (B.TSVD_OK, B.TSVD_ENOCONV)
        st, info = sv.wait(t_mix, 120.0)
        assert st == B.TSVD_OK
        for a, b in zip(alone, mix):
            assert np.array_equal(a, b)
        st2 = sv.stats()
        assert st2["waves"] >= 2 and st2["graph_updates"] + st2["graph_instantiations"] == st2["waves"]
    finally:
        sv.close()
        pool.close()


def test_server_set_cluster_for():
    """A fixed cluster size per class of Gram dimension: invalid sizes are
    rejected, a valid one is what later requests of that class run with, and
    the result still follows the oracle's trajectory."""
    B.load()
    pool = Pool()
    sv = Server(device_budget=2 << 30)
    try:
        for bad_d, bad_c in ((0, 2), (4096, 2), (512, 3), (512, 16)):
            assert sv.lib.tsvd_server_set_cluster_for(sv.handle, bad_d, bad_c) == B.TSVD_EINVAL
        sv.set_cluster_for(700, 2)
        assert sv.cluster_for(1000) == 2 and sv.cluster_for(600) == 2
        m, n, k = 3000, 700, 6
        A = _request(pool, m, n, 0.8, seed=41)
        U, s, V = _outputs(pool, m, n, k)
        o = ref.tsvd_dense(A, k, 1e-10, seed=9)
        st, info = sv.wait(sv.submit(A, k, 1e-10, U, s, V, seed=9, iters_override=o.iters), 60.0)
        assert st == B.TSVD_OK and info["cluster"] == 2
        assert np.max(np.abs(s - o.sigma) / o.sigma) <= 1e-5
        for l in range(k):
            assert ref.vector_angle(V[l].astype(np.float64), o.V[:, l]) <= 1e-4
    finally:
        sv.close()
        pool.close()


def test_server_zero_matrix_reports_rank():
    B.load()
    pool = Pool()
    sv = Server(device_budget=1 << 30)
    try:
        A = pool.arr((100, 40), np.float32)
        A[:] = 0.0
        U, s, V = _outputs(pool, 100, 40, 3)
        st, info = sv.wait(sv.submit(A, 3, 1e-8, U, s, V), 30.0)
        assert st == B.TSVD_ERANK and info["flags"] & B.TSVD_FLAG_RANK
        assert np.all(s == 0.0)
        Vd = V.astype(np.float64)
        assert np.allclose(Vd @ Vd.T, np.eye(3), atol=1e-6)  # orthonormal fallback vectors
    finally:
        sv.close()
        pool.close()


def test_server_autotune_table():
    B.load()
    sv = Server(device_budget=6 << 30)
    try:
        sv.autotune(iters=20)
        for d in (64, 128, 256, 512, 1024, 2048):
            c = sv.cluster_for(d)
            assert c in (1, 2, 4, 8)
        # the Gram step's tile shape: tensor cores from one of the timed sizes on, or never
        assert sv.tc_min_d() in (256, 512, 1024, 2048, (1 << 63) - 1)
    finally:
        sv.close()


def test_server_sparse_requests_beside_dense_ones():
    """CSR requests run on the server's sparse workers (plan API, workspace from
    the server's budget) while dense waves run; each follows the oracle's
    trajectory (forced counts, the seed's Philox start draws)."""
    B.load()
    pool = Pool()
    sv = Server(device_budget=4 << 30, n_streams=2)
    try:
        sparse = []
        for i, (m, n, per_row, k) in enumerate([(4000, 3000, 20.0, 5), (6000, 6000, 8.0, 4), (2500, 700, 40.0, 6)]):
            csr = synth.csr_uniform(m, n, per_row, seed=50 + i)
            o = ref.tsvd_csr(csr, k, 1e-6, seed=9 + i)
            U = pool.arr((k, m), np.float32)
            s_ = pool.arr((k,), np.float64)
            V = pool.arr((k, n), np.float32)
            t = sv.submit_csr(csr, k, 1e-6, U, s_, V, seed=9 + i, iters_override=o.iters)
            sparse.append((t, csr, k, U, s_, V, o))
        dense = []
        for i, (m, n, k, rho) in enumerate(CASES[:4]):
            A = _request(pool, m, n, rho, seed=300 + i)
            U, s_, V = _outputs(pool, m, n, k)
            o = ref.tsvd_dense(A, k, 1e-10, seed=40 + i)
            dense.append((sv.submit(A, k, 1e-10, U, s_, V, seed=40 + i, iters_override=o.iters), k, s_, o))
        for t, csr, k, U, s_, V, o in sparse:
            st, info = sv.wait(t, 300.0)
            assert st == B.TSVD_OK, (st, sv.last_error())
            assert info["applications"] == sum(o.iters)
            assert np.max(np.abs(s_ - o.sigma) / o.sigma) <= 1e-5
            gapped = ref.gapped_indices(o.sigma ** 2, k)
            assert gapped and gapped[0] == 0, gapped  # the leading (Perron) triplet of a positive A is gapped
            for l in gapped:
                assert ref.vector_angle(V[l].astype(np.float64), o.V[:, l]) <= 1e-4
                assert ref.vector_angle(U[l].astype(np.float64), o.U[:, l]) <= 1e-4
        for t, k, s_, o in dense:
            st, _ = sv.wait(t, 120.0)
            assert st == B.TSVD_OK and np.max(np.abs(s_ - o.sigma) / o.sigma) <= 1e-5
        assert sv.stats()["completed"] == len(sparse) + len(dense)
    finally:
        sv.close()
        pool.close()
