"""bilu_apply_noalloc, the preconditioner application for callers that cannot allocate device
memory (during CUDA graph capture, under a fixed memory pool or another framework's allocator,
in loops that must not allocate).  Its scratch is a fixed device array shared by all calls.

Collected last on purpose, so that a run stopping at the first failure has run every other
test; it also passes alone in a fresh process (it creates everything it uses).
"""
import numpy as np
import pytest

import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_apply_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A = W.convdiff_upwind((16, 16, 16), seed=2)
    ctx = B.bilu_create(0)
    try:
        B.bilu_analyze(ctx, A.n, A.rowptr, A.colind, A.val, B.bilu_params_default(fixed_block=16, max_block=64))
        B.bilu_factor(ctx, 1e-2)
        rng = np.random.default_rng(3)
        for _ in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
            r = torch.from_numpy(rng.standard_normal(A.n)).cuda()
            z_ref = torch.empty_like(r)
            z_na = torch.full_like(r, np.nan)
            B.bilu_apply(ctx, r, z_ref)
            B.bilu_apply_noalloc(ctx, r, z_na)
            torch.cuda.synchronize()
            zr, zn = z_ref.cpu().numpy(), z_na.cpu().numpy()
            assert np.all(np.isfinite(zn))
            assert np.abs(zn - zr).max() <= 1e-11 * np.abs(zr).max()  # as the apply parity test
        with pytest.raises(B.BiluError) as e:
            B.bilu_apply_noalloc(ctx, np.zeros(A.n), np.zeros(A.n))
        assert e.value.status == B.BILU_ERR_ARG
    finally:
        B.bilu_destroy(ctx)
