"""The timeout path of the tensor-core Gram kernel on the GPU.

Every wait of the library's kernels is bounded: when one gives up, the kernel
raises its status word, stops issuing work, lets its own TMA loads and MMAs
complete, frees its tensor memory and returns, and tsvd_factor reports
TSVD_ETIMEDOUT.  Here a correct kernel is made to give up by the test-only
option wait_limit_ns (a 1 ns limit on its pipeline waits, shorter than any TMA
load takes); nothing is broken on purpose and no wait is left unbounded.
"""
import numpy as np
import pytest

import synth
from oracle import tsvd_ref as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2208_08410_gb300 import Plan, tsvd  # noqa: E402
from paper_2208_08410_gb300 import _binding as B  # noqa: E402


@pytest.mark.parametrize("prec", [B.TSVD_GRAM_TF32X3, B.TSVD_GRAM_TF32])
def test_gram_wait_limit_gives_etimedout_and_leaves_the_device_usable(prec):
    B.load()
    # one row block of the in-core workload's shape: 65,536 x 4096 (the SYRK's full launch)
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn((65536, 4096), generator=g, device="cuda", dtype=torch.float32)
    p = Plan(A, 1, 1e-6, precision=prec, out_device=True, max_iter=20, wait_limit_ns=1)
    try:
        r = p.factor(ok=(B.TSVD_ETIMEDOUT,))
    finally:
        p.close()
    assert r.status == B.TSVD_ETIMEDOUT
    assert r.report["flags"] & B.TSVD_FLAG_TIMEOUT
    torch.cuda.synchronize()  # no fault: the context is intact
    del A
    # every CTA of the next launches allocates tensor memory again: the same
    # kernel without the limit follows the oracle on the small dense workload
    m, n, k, eps = 2048, 256, 8, 1e-8
    inp = synth.dense_prescribed(m, n, synth.spectrum_geometric(n, 0.8), 1e-6, seed=0)
    x = synth.start_normals(n, k, seed=1)
    o = ref.tsvd_dense(inp["A"], k, eps, x_start=x)
    r2 = tsvd(torch.from_numpy(inp["A"]).cuda(), k, eps, start_draws=x, iters_override=o.iters,
              precision=B.TSVD_GRAM_TF32X3)
    assert r2.status == B.TSVD_OK and r2.report["flags"] == 0
    assert np.max(np.abs(r2.sigma - o.sigma) / o.sigma) <= 1e-5
    gapped = ref.gapped_indices(o.sigma ** 2, k)
    assert gapped == list(range(k))
    for l in gapped:
        assert ref.vector_angle(np.asarray(r2.V[:, l]), o.V[:, l]) <= 1e-4

