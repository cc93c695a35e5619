"""GPU tests of the tree schedule: groups of CTAs factor independent subtrees of the block
elimination tree side by side (every block that updates block K lies in K's subtree, so K runs
once its children are done; Sec. 3.3 reorders the matrix so that the tree has independent
subtrees), and the trunk of single-child blocks at the top runs on the whole GPU.

Bar: the same factor, bit for bit, as the chain schedule on the same ordering (each block sees
the same inputs and its producers in the same order), hence the oracle's kept sets and values
to the FP64 parity bar and its GMRES(30) iteration count."""
import json
import os

import numpy as np
import pytest

from oracle import block_check as BC
import oracle as O
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W
from tests.gpu_helpers import compare_factors, gpu_factor

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "computed")


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.bilu_create(0)
    yield c
    B.bilu_debug_set(c, B.BILU_DEBUG_NO_TRUNK, 0)
    B.bilu_destroy(c)


def nd_workload(w, blk):
    """w after the block nested dissection of its fixed blocks of blk (library host analysis)."""
    bs = np.append(np.arange(0, w.A.n, blk), w.A.n).astype(np.int32)
    perm, nbs, _ = B.bilu_nd_order(w.A.n, w.A.rowptr, w.A.colind, bs)
    A = W.CSR(w.A.n, *B.bilu_permute_csr(w.A.n, w.A.rowptr, w.A.colind, w.A.val, perm))
    return A, w.b[perm], nbs


def params(schedule, G=0, **kw):
    return B.bilu_params_default(max_block=64, schedule=schedule, group_ctas=G, **kw)


def same_factor(g1, g2):
    for k in ("bstart", "Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        a, b = getattr(g1, k), getattr(g2, k)
        assert a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8)), k
    for k in ("kept_rows", "kept_cols", "cand_rows", "cand_cols", "flop_upd_l", "flop_upd_u", "flop_scale",
              "flop_norm", "nperturb", "skipped_rows", "skipped_cols", "bound_drops"):
        assert getattr(g1.stats, k) == getattr(g2.stats, k), k


@pytest.mark.parametrize("side,blk,G,trunk", [(12, 12, 4, True), (16, 16, 1, False), (16, 16, 8, True),
                                              (20, 20, 2, False), (16, 8, 19, True), (24, 24, 8, False),
                                              (24, 24, 38, True),
                                              # group sizes that do not divide the grid: the CTAs
                                              # past the last group join only the trunk
                                              (16, 16, 12, True), (20, 20, 5, True), (24, 24, 24, False),
                                              (16, 16, 100, True)])
def test_tree_equals_chain_bitwise(ctx, side, blk, G, trunk):
    A, b, bs = nd_workload(W.cd3d(side=side, seed=1, block=blk), blk)
    gc = gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_CHAIN), bstart=bs)
    B.bilu_debug_set(ctx, B.BILU_DEBUG_NO_TRUNK, 0 if trunk else 1)
    try:
        gt = gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_TREE, G), bstart=bs)
    finally:
        B.bilu_debug_set(ctx, B.BILU_DEBUG_NO_TRUNK, 0)
    assert gt.status == B.BILU_OK
    s = gt.stats
    assert s.schedule == B.BILU_SCHED_TREE and s.group_ctas == G and s.tree_height < s.nblocks
    same_factor(gc, gt)


@pytest.mark.parametrize("side,blk", [(16, 16), (24, 24), (20, 40)])
def test_tree_nd_parity_with_oracle(ctx, side, blk):
    """Kept sets and values against the oracle on the dissection order; GMRES(30) takes the
    oracle's iteration count."""
    import torch
    A, b, bs = nd_workload(W.cd3d(side=side, seed=1, block=blk), blk)
    g = gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_TREE, 4), bstart=bs)
    Fo = O.bilu_factor(A, bs, 1e-2)
    compare_factors(Fo, g, A=A, tau=1e-2)
    ro = O.gmres(A, Fo, b, tol=1e-8, restart=30)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    info = B.gmres_solve(ctx, bt, x, 1e-8, 30, 10000)
    assert info.iters == ro.iters
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-6 * max(1.0, np.abs(ro.x).max())
    Fo.free()


def test_tree_natural_order_is_one_trunk(ctx):
    """In natural order the block elimination tree of a banded matrix is a chain: the whole
    factorization is the trunk, on the whole GPU, and equals the chain schedule."""
    w = W.cd3d(side=12, seed=1, block=12)
    gc = gpu_factor(ctx, w.A, 1e-2, params(B.BILU_SCHED_CHAIN, fixed_block=12))
    gt = gpu_factor(ctx, w.A, 1e-2, params(B.BILU_SCHED_TREE, 8, fixed_block=12))
    assert gt.stats.tree_trunk == gt.stats.nblocks == gt.stats.tree_height
    same_factor(gc, gt)


@pytest.mark.parametrize("prec,skip", [(B.BILU_PREC_FP32, B.BILU_SKIP_NONE), (B.BILU_PREC_BF16, B.BILU_SKIP_NONE),
                                       (B.BILU_PREC_FP64, B.BILU_SKIP_BOUND), (B.BILU_PREC_FP32, B.BILU_SKIP_BOUND)])
def test_tree_precisions_and_bound_skip_equal_chain(ctx, prec, skip):
    A, b, bs = nd_workload(W.cd3d(side=16, seed=1, block=16), 16)
    gc = gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_CHAIN, precision=prec, skip=skip), bstart=bs)
    gt = gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_TREE, 4, precision=prec, skip=skip), bstart=bs)
    same_factor(gc, gt)
    if skip == B.BILU_SKIP_BOUND:
        assert gt.stats.skipped_rows + gt.stats.skipped_cols > 0


def test_tree_vector_stencil_and_random_partition(ctx):
    """Elasticity (3 unknowns per node, blocks of 24) after dissection, and a random matrix
    with ragged blocks in its own (tree-shaped or not) order: tree equals chain."""
    A, b, bs = nd_workload(W.elasticity3d(side=6, seed=2, block=24), 24)
    same_factor(gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_CHAIN), bstart=bs),
                gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_TREE, 2), bstart=bs))
    rng = np.random.default_rng(7)
    A2 = W.random_diag_dominant(300, 0.02, 57, dominance=1.1)
    cuts = np.sort(rng.choice(np.arange(1, 300), size=40, replace=False))
    bs2 = np.concatenate([[0], cuts, [300]]).astype(np.int32)
    bs2 = bs2[np.concatenate([[True], np.diff(bs2) > 0])]
    same_factor(gpu_factor(ctx, A2, 1e-3, params(B.BILU_SCHED_CHAIN), bstart=bs2),
                gpu_factor(ctx, A2, 1e-3, params(B.BILU_SCHED_TREE, 3), bstart=bs2))


def test_tree_reruns_from_minimal_storage(ctx):
    """Pools and producer lists that start minimal: the tree schedule grows them, runs again
    and ends with the same factor."""
    A, b, bs = nd_workload(W.cd3d(side=12, seed=1, block=12), 12)
    ref = gpu_factor(ctx, A, 1e-2, params(B.BILU_SCHED_CHAIN), bstart=bs)
    c2 = B.bilu_create(0)
    try:
        B.bilu_debug_set(c2, B.BILU_DEBUG_SMALL_POOLS, 1)
        g = gpu_factor(c2, A, 1e-2, params(B.BILU_SCHED_TREE, 4), bstart=bs)
        assert g.stats.pool_retries > 0
        same_factor(ref, g)
    finally:
        B.bilu_debug_set(c2, B.BILU_DEBUG_SMALL_POOLS, 0)
        B.bilu_destroy(c2)


def test_tree_bounded_wait_timeout_leaves_context_usable(ctx):
    """Every group barrier waits for one CTA that never arrives: the bounded waits give up,
    bilu_factor returns BILU_ERR_TIMEOUT, and the next factorization on the context works."""
    A, b, bs = nd_workload(W.cd3d(side=12, seed=1, block=12), 12)
    B.bilu_analyze_partition(ctx, A.n, A.rowptr, A.colind, A.val, bs, params(B.BILU_SCHED_TREE, 4))
    B.bilu_debug_set(ctx, B.BILU_DEBUG_SPIN_LIMIT, 20000)
    B.bilu_debug_set(ctx, B.BILU_DEBUG_EXTRA_CTA, 1)
    try:
        with pytest.raises(B.BiluError) as e:
            B.bilu_factor(ctx, 1e-2)
        assert e.value.status == B.BILU_ERR_TIMEOUT
    finally:
        B.bilu_debug_set(ctx, B.BILU_DEBUG_EXTRA_CTA, 0)
        B.bilu_debug_set(ctx, B.BILU_DEBUG_SPIN_LIMIT, 0)
    assert B.bilu_factor(ctx, 1e-2) == B.BILU_OK


def test_tree_rejects_learned_skip_and_bad_arguments(ctx):
    w = W.cd3d(side=8, seed=1, block=8)
    with pytest.raises(B.BiluError):
        B.bilu_analyze(ctx, w.A.n, w.A.rowptr, w.A.colind, w.A.val, params(5, fixed_block=8))
    with pytest.raises(B.BiluError):
        B.bilu_analyze(ctx, w.A.n, w.A.rowptr, w.A.colind, w.A.val, params(B.BILU_SCHED_TREE, 100000, fixed_block=8))
    c2 = B.bilu_create(0)
    try:
        B.bilu_analyze(c2, w.A.n, w.A.rowptr, w.A.colind, w.A.val,
                       params(B.BILU_SCHED_TREE, 4, fixed_block=8, skip=B.BILU_SKIP_LEARNED))
        model = np.zeros(B.BILU_MLP_PARAMS, np.float32)
        model[B.BILU_MLP_FEATURES:2 * B.BILU_MLP_FEATURES] = 1.0  # unit std: a valid model
        B.bilu_set_skip_model(c2, model, 0.0)
        with pytest.raises(B.BiluError) as e:
            B.bilu_factor(c2, 1e-2)
        assert e.value.status == B.BILU_ERR_ARG
        B.bilu_analyze(c2, w.A.n, w.A.rowptr, w.A.colind, w.A.val, params(B.BILU_SCHED_TREE, 4, fixed_block=8))
        B.bilu_record_samples(c2, 1000, 0.5, 1)
        with pytest.raises(B.BiluError) as e:
            B.bilu_factor(c2, 1e-2)
        assert e.value.status == B.BILU_ERR_ARG
        B.bilu_record_samples(c2, 0, 0.0, 0)
        assert B.bilu_factor(c2, 1e-2) == B.BILU_OK
    finally:
        B.bilu_destroy(c2)


def test_cd3d64_nd_tree_full_size(ctx):
    """The benchmark matrix after block nested dissection, tree schedule in the launch
    configuration bench.py times: sampled blocks against the oracle's single step from the
    GPU's own earlier blocks, the oracle's kept counts and GMRES(30) iteration count (written
    by tests/golden/computed/make_cd3d64_nd.py), the solution's true residual."""
    import torch
    ref = json.load(open(os.path.join(GOLDEN, "cd3d64_nd.json")))
    w = W.cd3d(side=64, seed=1, block=64)
    A, b, bs = nd_workload(w, 64)
    g = gpu_factor(ctx, A, w.droptol, params(B.BILU_SCHED_TREE, 0), bstart=bs)
    s = g.stats
    assert s.nblocks == ref["nblocks"] and s.tree_height == ref["tree_height"]
    assert (s.kept_rows, s.kept_cols) == (ref["kept_rows"], ref["kept_cols"])
    E = {k: getattr(g, k) for k in ("bstart", "Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk")}
    blocks = BC._blocks(E)
    nb = s.nblocks
    rng = np.random.default_rng(1)
    sample = sorted(set([0, 1, nb // 2, nb - 65, nb - 2, nb - 1] + list(rng.integers(0, nb, 8))))
    flips = 0
    for K in sample:
        f, err = BC.compare_block(A, E, K, w.droptol, rtol=1e-10, blocks=blocks)
        flips += f
    assert flips == 0
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    info = B.gmres_solve(ctx, bt, x, 1e-8, 30, 10000)
    assert info.iters == ref["gmres_iters"]
    r = b - A.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
