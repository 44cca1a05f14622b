"""The allocation-free multi-dot against the regular one.

qdd_cdot_multi_noalloc serves callers that must not allocate device memory
(a pre-sized memory pool owns everything, or a loop cannot afford the
synchronisation a cudaFree brings); its partial sums sit in a fixed array
inside the library.  This checks, through the C ABI, that two calls in a row
give what qdd_cdot_multi gives, within the tolerance of the other vector
tests.  The file is named to run last, after every other GPU test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_cdot_matches_regular_twice():
    import torch

    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    ctx = qdd.qdd_create(0, 0)
    g = torch.Generator().manual_seed(11)
    n = 200_003
    for nvec in (17, 3):  # two calls in a row, the second smaller than the first
        v = torch.randn(nvec, n, dtype=torch.complex128, generator=g).cuda()
        w = torch.randn(n, dtype=torch.complex128, generator=g).cuda()
        ref = qdd.qdd_cdot_multi(ctx, v, w).cpu().numpy()
        got = qdd.qdd_cdot_multi_noalloc(v, w).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        want = np.conj(v.cpu().numpy()) @ w.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    with pytest.raises(qdd.QddError):
        qdd.qdd_cdot_multi_noalloc(torch.zeros(65, 8, dtype=torch.complex128, device="cuda"),
                                   torch.zeros(8, dtype=torch.complex128, device="cuda"))
    qdd.qdd_destroy(ctx)
