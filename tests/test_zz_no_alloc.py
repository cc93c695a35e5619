"""bilu_apply_noalloc, the preconditioner application for callers that cannot allocate device
memory when they apply it (programs whose device memory belongs to a fixed pool or to another
framework's allocator, loops that must not enter the allocator).  Its scratch is a fixed
device array shared by all calls.

Collected last on purpose, so that a run stopping at the first failure has run every other
test; it also passes alone in a fresh process (it creates everything it uses).
"""
import numpy as np
import pytest

import oracle as O
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("blk", [16, 48, 64])
def test_noalloc_apply_matches_apply_on_two_calls_in_a_row(torch, blk):
    """Blocks of 16 (one lane per row), 48 and 64 (rows past lane 32): two calls in a row agree
    with bilu_apply and with the oracle's block substitution on the oracle's factor."""
    A = W.convdiff_upwind((16, 16, 16), seed=2)
    ctx = B.bilu_create(0)
    try:
        B.bilu_analyze(ctx, A.n, A.rowptr, A.colind, A.val, B.bilu_params_default(fixed_block=blk, max_block=64))
        B.bilu_factor(ctx, 1e-2)
        Fo = O.bilu_factor(A, O.partition_fixed(A.n, blk), 1e-2)
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
            zo = O.bilu_apply(Fo, r.cpu().numpy())
            assert np.abs(zn - zo).max() <= 1e-10 * np.abs(zo).max()
        Fo.free()
        with pytest.raises(B.BiluError) as e:
            B.bilu_apply_noalloc(ctx, np.zeros(A.n), np.zeros(A.n))
        assert e.value.status == B.BILU_ERR_ARG
    finally:
        B.bilu_destroy(ctx)


def test_noalloc_apply_allocates_nothing_and_reports_a_timeout_as_nan(torch):
    """Free device memory does not move over repeated calls; a wait that runs out (a flag that
    nothing sets, test hook) leaves z all NaN, and the next call is correct again."""
    A = W.convdiff_upwind((12, 12, 12), seed=4)
    ctx = B.bilu_create(0)
    try:
        B.bilu_analyze(ctx, A.n, A.rowptr, A.colind, A.val, B.bilu_params_default(fixed_block=12, max_block=64))
        B.bilu_factor(ctx, 1e-2)
        r = torch.from_numpy(np.random.default_rng(5).standard_normal(A.n)).cuda()
        z_ref = torch.empty_like(r)
        z = torch.empty_like(r)
        B.bilu_apply(ctx, r, z_ref)
        B.bilu_apply_noalloc(ctx, r, z)  # first call on the device: the scratch address lookup
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            B.bilu_apply_noalloc(ctx, r, z)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        B.bilu_debug_set(ctx, B.BILU_DEBUG_SPIN_LIMIT, 20000)
        B.bilu_debug_set(ctx, B.BILU_DEBUG_EXTRA_CTA, 1)
        try:
            B.bilu_apply_noalloc(ctx, r, z)
            torch.cuda.synchronize()
        finally:
            B.bilu_debug_set(ctx, B.BILU_DEBUG_EXTRA_CTA, 0)
            B.bilu_debug_set(ctx, B.BILU_DEBUG_SPIN_LIMIT, 0)
        assert torch.isnan(z).all()
        B.bilu_apply_noalloc(ctx, r, z)
        torch.cuda.synchronize()
        assert torch.equal(torch.isfinite(z), torch.ones_like(z, dtype=torch.bool))
        assert (z - z_ref).abs().max().item() <= 1e-11 * z_ref.abs().max().item()
    finally:
        B.bilu_destroy(ctx)
