"""The no-allocation power iteration (tsvd_power_dense_noalloc).

Some callers cannot call cudaMalloc (their device memory is owned by another
allocator, or an allocation is not allowed where they run); this entry point
keeps its scratch in a fixed array inside the library instead.  The test
calls it through the C ABI twice in a row and checks each result against the
allocating entry point tsvd_power_dense on the same inputs, within the
tolerance the power-step parity test uses.  It lives in its own file so that
pytest collects it last, and it builds every input itself, so it passes both
alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import tsvd_ref as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2208_08410_gb300 import _binding as B  # noqa: E402


def _inputs(n=256, l=3):
    inp = synth.dense_prescribed(2048, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=0)
    G = ref.gram(inp["A"])
    prior = ref.tsvd_dense(inp["A"], l, 1e-12, x_start=synth.start_normals(n, l, seed=9), B=G)
    x = synth.start_normals(n, 1, seed=21)[:, 0]
    return G, prior.V[:, :l], prior.sigma[:l] ** 2, x


def _run(fn_name, n, l, dG32, dG64, dV, ds2, x, override, scratch=None):
    stream = torch.cuda.current_stream().cuda_stream
    dx = torch.from_numpy(x.copy()).cuda()
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    s2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    common = (n, dG32.data_ptr(), dG64.data_ptr(), dV.data_ptr(), ds2.data_ptr(), l, dx.data_ptr(), 1e-8, 10000,
              override, 0, s2.data_ptr(), info.data_ptr())
    if fn_name == "tsvd_power_dense":
        st = B.tsvd_power_dense(*common, scratch.data_ptr(), scratch.numel(), stream)
    else:
        st = B.tsvd_power_dense_noalloc(*common, stream)
    assert st == B.TSVD_OK, B.load().tsvd_last_cuda_error()
    torch.cuda.synchronize()
    return dx.cpu().numpy(), s2.item(), info.cpu().numpy()


def test_noalloc_power_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    n, l = 256, 3
    G, V, s2, x = _inputs(n, l)
    dG64 = torch.from_numpy(G).cuda()
    dG32 = torch.from_numpy(G.astype(np.float32)).cuda()
    dV = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()  # column-major n x l
    ds2 = torch.from_numpy(s2).cuda()
    scratch = torch.empty(B.tsvd_power_scratch_bytes(n, l), dtype=torch.uint8, device="cuda")
    for override in (0, 25):
        want_v, want_s2, want_info = _run("tsvd_power_dense", n, l, dG32, dG64, dV, ds2, x, override, scratch)
        for _ in range(2):  # two calls in a row share the static scratch
            v, got_s2, info = _run("tsvd_power_dense_noalloc", n, l, dG32, dG64, dV, ds2, x, override)
            assert info[0] == want_info[0] and info[1] == want_info[1] == 0 and info[2] == 0
            assert ref.vector_angle(v, want_v) < 1e-5
            assert abs(got_s2 - want_s2) <= 1e-6 * want_s2


def test_noalloc_power_at_its_size_limit():
    """The largest problem the fixed array accepts (n = TSVD_NOALLOC_MAX_N,
    l = TSVD_NOALLOC_MAX_L earlier vectors; the launch needs the array's whole
    size and more than 48 KB of dynamic shared memory): the same result as the
    allocating entry point with its own scratch, twice in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    n, l, r = B.TSVD_NOALLOC_MAX_N, B.TSVD_NOALLOC_MAX_L, B.TSVD_NOALLOC_MAX_L + 16
    rng = np.random.default_rng(5)
    W, _ = np.linalg.qr(rng.standard_normal((n, r)))  # seeded orthonormal basis of a rank-r Gram matrix
    lam = 0.9 ** np.arange(r)
    dW = torch.from_numpy(W).cuda()
    dG64 = (dW * torch.from_numpy(lam).cuda()) @ dW.T  # G = W diag(lam) W^T, 2 GiB in FP64
    dG32 = dG64.float()
    dV = torch.from_numpy(np.ascontiguousarray(W[:, :l].T)).cuda()  # the l earlier vectors, column-major
    ds2 = torch.from_numpy(lam[:l].copy()).cuda()
    x = rng.standard_normal(n)
    scratch = torch.empty(B.tsvd_power_scratch_bytes(n, l), dtype=torch.uint8, device="cuda")
    want_v, want_s2, want_info = _run("tsvd_power_dense", n, l, dG32, dG64, dV, ds2, x, 30, scratch)
    assert want_info[0] == 30 and want_info[2] == 0
    for _ in range(2):
        v, got_s2, info = _run("tsvd_power_dense_noalloc", n, l, dG32, dG64, dV, ds2, x, 30)
        assert info[0] == 30 and info[2] == 0
        assert ref.vector_angle(v, want_v) < 1e-5
        assert abs(got_s2 - want_s2) <= 1e-6 * want_s2
    del dG64, dG32, dW, scratch
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load()
    n = B.TSVD_NOALLOC_MAX_N + 1
    st = B.tsvd_power_dense_noalloc(n, None, None, None, None, 0, None, 1e-8, 100, 0, 0, None, None, None)
    assert st == B.TSVD_EINVAL
    assert b"16384" in lib.tsvd_last_cuda_error()
    st = B.tsvd_power_dense_noalloc(64, None, None, None, None, B.TSVD_NOALLOC_MAX_L + 1, None, 1e-8, 100, 0, 0,
                                    None, None, None)
    assert st == B.TSVD_EINVAL
