"""GPU parity of progressive aggregation (Sec. 3.5) against the oracle, which merges inside
its factorization loop.

Bar: the same merged partition (void blocks included), the same kept rows and columns of
every merged block, values of L, U-breve, D and P to relative 1e-10 per block, the
preconditioner applied to a vector to relative 1e-10, and the GMRES(30) iteration count of
the unmerged factor.
"""
import numpy as np
import pytest

import oracle as O
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W
from tests.gpu_helpers import compare_factors, gpu_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.bilu_create(0)
    yield c
    B.bilu_destroy(c)


def _case(name):
    if name == "cd2d_32 scalar blocks":
        w = W.cd2d_32()
        return w, np.arange(w.A.n + 1, dtype=np.int32)
    if name == "cd3d 10^3 scalar blocks":
        w = W.cd3d(side=10, seed=1, block=4)
        return w, np.arange(w.A.n + 1, dtype=np.int32)
    if name == "elasticity 6^3 node blocks":
        w = W.elasticity3d(side=6, seed=2, block=24)
        return w, np.arange(0, w.A.n + 1, 3, dtype=np.int32)
    if name == "elasticity 6^3 ILU(1,tau) blocks":
        w = W.elasticity3d(side=6, seed=2, block=24)
        return w, O.partition_ilu1t(w.A, 1e-2, 64)
    raise KeyError(name)


CASES = ["cd2d_32 scalar blocks", "cd3d 10^3 scalar blocks", "elasticity 6^3 node blocks",
         "elasticity 6^3 ILU(1,tau) blocks"]


def _apply(ctx, r):
    import torch
    rt = torch.from_numpy(r).cuda()
    z = torch.empty_like(rt)
    B.bilu_apply(ctx, rt, z)  # on the context's stream
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("amax", [64, 8])
def test_aggregated_factor_matches_oracle(ctx, name, amax):
    w, bs = _case(name)
    p = B.bilu_params_default(aggregate_max=amax)
    g = gpu_factor(ctx, w.A, 1e-2, p, bstart=bs)
    Fo = O.bilu_factor(w.A, bs, 1e-2, agg_max=amax)
    assert g.stats.agg_merges == Fo.merges > 0, name
    assert np.array_equal(g.bstart, Fo.bstart)
    assert g.stats.agg_max_bsize == int(np.diff(Fo.bstart).max()) <= amax
    rep = compare_factors(Fo, g, rtol=1e-10)
    print(f"{name}, at most {amax}: {Fo.merges} merges, {rep}")
    r = np.random.default_rng(5).standard_normal(w.A.n)
    zg, zo = _apply(ctx, r), O.bilu_apply(Fo, r)
    assert np.abs(zg - zo).max() <= 1e-10 * np.abs(zo).max()


@pytest.mark.parametrize("name", CASES[:3])
def test_aggregation_keeps_the_operator_and_the_iterations(ctx, name):
    """The merged factor is the same preconditioner: its application equals the unmerged
    one's (to rounding) and GMRES(30) takes the same number of steps."""
    import torch
    w, bs = _case(name)
    c2 = B.bilu_create(0)
    try:
        gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(aggregate_max=64), bstart=bs, export=False)
        gpu_factor(c2, w.A, 1e-2, B.bilu_params_default(), bstart=bs, export=False)
        assert B.bilu_stats(ctx).agg_merges > 0 and B.bilu_stats(c2).agg_merges == 0
        r = np.random.default_rng(6).standard_normal(w.A.n)
        z1, z0 = _apply(ctx, r), _apply(c2, r)
        assert np.abs(z1 - z0).max() <= 1e-11 * np.abs(z0).max()
        b = torch.from_numpy(w.b).cuda()
        x1, x0 = torch.zeros_like(b), torch.zeros_like(b)
        i1 = B.gmres_solve(ctx, b, x1, 1e-8, 30, 5000)
        i0 = B.gmres_solve(c2, b, x0, 1e-8, 30, 5000)
        assert i1.iters == i0.iters and i1.relres_true <= 1e-8
    finally:
        B.bilu_destroy(c2)


def test_aggregation_after_the_tree_schedule(ctx):
    """Merges are taken on the finished factor, so the tree schedule (same factor, bit for
    bit, as the chain on the same ordering) gives the same merged factor, bit for bit."""
    w, bs = _case("elasticity 6^3 node blocks")
    A = w.A
    perm, bnd, _ = B.bilu_nd_order(A.n, A.rowptr, A.colind, bs)
    A2 = W.CSR(A.n, *B.bilu_permute_csr(A.n, A.rowptr, A.colind, A.val, perm))
    gc = gpu_factor(ctx, A2, 1e-2, B.bilu_params_default(aggregate_max=64, schedule=B.BILU_SCHED_CHAIN), bstart=bnd)
    c2 = B.bilu_create(0)
    try:
        gt = gpu_factor(c2, A2, 1e-2, B.bilu_params_default(aggregate_max=64, schedule=B.BILU_SCHED_TREE,
                                                            group_ctas=4), bstart=bnd)
    finally:
        B.bilu_destroy(c2)
    assert gc.stats.agg_merges > 0
    for k in ("bstart", "Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(gc, k), getattr(gt, k)), k
    Fo = O.bilu_factor(A2, bnd, 1e-2, agg_max=64)
    assert np.array_equal(gc.bstart, Fo.bstart)
    compare_factors(Fo, gc, rtol=1e-10)


@pytest.mark.parametrize("prec,tol", [(B.BILU_PREC_FP32, 1e-4), (B.BILU_PREC_BF16, 3e-2)])
def test_aggregation_with_reduced_precision_storage(ctx, prec, tol):
    """FP32 / BF16 storage: the merged values are formed in FP64 from the stored ones and
    rounded once, so the merged preconditioner agrees with the unmerged one of the same
    precision to the storage rounding (and to the sweeps' FP32 arithmetic), and GMRES needs at
    most one more step."""
    import torch
    w, bs = _case("elasticity 6^3 node blocks")
    c2 = B.bilu_create(0)
    try:
        gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(aggregate_max=64, precision=prec), bstart=bs, export=False)
        gpu_factor(c2, w.A, 1e-2, B.bilu_params_default(precision=prec), bstart=bs, export=False)
        assert B.bilu_stats(ctx).agg_merges > 0
        r = np.random.default_rng(7).standard_normal(w.A.n)
        z1, z0 = _apply(ctx, r), _apply(c2, r)
        assert np.abs(z1 - z0).max() <= tol * np.abs(z0).max()
        b = torch.from_numpy(w.b).cuda()
        x1, x0 = torch.zeros_like(b), torch.zeros_like(b)
        i1 = B.gmres_solve(ctx, b, x1, 1e-8, 30, 5000)
        i0 = B.gmres_solve(c2, b, x0, 1e-8, 30, 5000)
        assert abs(i1.iters - i0.iters) <= 1 and i1.relres_true <= 1e-8
    finally:
        B.bilu_destroy(c2)


def test_aggregation_off_and_fixed_blocks_of_64_leave_the_factor_alone(ctx):
    """aggregate_max 0, or blocks that cannot merge (two blocks of 64 exceed the cap): the
    factor is exported as computed."""
    w = W.cd3d(side=12, seed=3, block=12)
    bs = O.partition_fixed(w.A.n, 64)
    g0 = gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(), bstart=bs)
    g1 = gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(aggregate_max=64), bstart=bs)
    assert g1.stats.agg_merges == 0
    for k in ("bstart", "Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(g0, k), getattr(g1, k)), k


def test_aggregate_max_is_validated(ctx):
    w, bs = _case("cd2d_32 scalar blocks")
    for bad in (1, -3, 65):
        with pytest.raises(B.BiluError) as ei:
            gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(aggregate_max=bad), bstart=bs, export=False)
        assert ei.value.status == B.BILU_ERR_ARG


def test_no_alloc_apply_reads_the_merged_blocks(ctx):
    import torch
    w, bs = _case("cd2d_32 scalar blocks")
    gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(aggregate_max=64), bstart=bs, export=False)
    assert B.bilu_stats(ctx).agg_merges > 0
    r = torch.from_numpy(np.random.default_rng(8).standard_normal(w.A.n)).cuda()
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    B.bilu_apply(ctx, r, z1)
    B.bilu_apply_noalloc(ctx, r, z2)
    torch.cuda.synchronize()
    assert torch.allclose(z1, z2, rtol=1e-11, atol=1e-13)
