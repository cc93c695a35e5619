"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bar: identical partitions and kept row / column sets, values of L, U-breve, D_K and P_K to
relative 1e-10 per block (the FP64 tolerance the method's target states), identical
GMRES(30) iteration counts to relative residual 1e-8.
"""
import numpy as np
import pytest

import oracle as O
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W
from tests import test_golden as TG
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


def _fixed(b, mx=64):
    return B.bilu_params_default(blocking=B.BILU_BLOCKING_FIXED, fixed_block=b, max_block=mx)


def _oracle(A, bstart, tau):
    return O.bilu_factor(A, bstart, tau)


def test_partition_fixed_and_ilu1t_match_oracle(ctx):
    A = W.convdiff_upwind((10, 10, 10), seed=3)
    g = gpu_factor(ctx, A, 1e-2, _fixed(7), export=False)
    assert np.array_equal(g.bstart, O.partition_fixed(A.n, 7))
    p = B.bilu_params_default(blocking=B.BILU_BLOCKING_ILU1T, max_block=16, tau_analyze=1e-2)
    g = gpu_factor(ctx, A, 1e-2, p, export=False)
    assert np.array_equal(g.bstart, O.partition_ilu1t(A, 1e-2, 16))
    Ad = np.eye(50) * 100.0
    Ad[10:40, 0] = 1.0
    Ad[14:44, 1] = 1.0
    A2 = W.from_dense(Ad)
    p = B.bilu_params_default(blocking=B.BILU_BLOCKING_ILU1T, max_block=64, tau_analyze=1e-3)
    g = gpu_factor(ctx, A2, 1e-2, p, export=False)
    assert np.array_equal(g.bstart, O.partition_ilu1t(A2, 1e-3, 64))


@pytest.mark.parametrize("blk", [1, 4, 32])
def test_factor_parity_cd2d(ctx, blk):
    w = W.cd2d_32()
    g = gpu_factor(ctx, w.A, 1e-2, _fixed(blk))
    o = _oracle(w.A, g.bstart, 1e-2)
    rep = compare_factors(o, g, A=w.A, tau=1e-2)
    assert rep.blocks == len(g.bstart) - 1


@pytest.mark.parametrize("seed,maxb,tau", [(0, 8, 1e-2), (1, 3, 1e-3), (2, 16, 5e-2), (3, 64, 0.0)])
def test_factor_parity_random(ctx, seed, maxb, tau):
    A = W.random_diag_dominant(300, 0.02, 50 + seed, dominance=1.1)
    p = B.bilu_params_default(blocking=B.BILU_BLOCKING_ILU1T, max_block=maxb, tau_analyze=1e-2)
    g = gpu_factor(ctx, A, tau, p)
    o = _oracle(A, g.bstart, tau)
    compare_factors(o, g, A=A, tau=tau)


@pytest.mark.parametrize("side,blk", [(12, 12), (16, 16), (16, 64), (20, 40)])
def test_factor_parity_cd3d(ctx, side, blk):
    A = W.convdiff_upwind((side, side, side), seed=1)
    g = gpu_factor(ctx, A, 1e-2, _fixed(blk))
    o = _oracle(A, g.bstart, 1e-2)
    compare_factors(o, g, A=A, tau=1e-2)


@pytest.mark.parametrize("kind,side,blk", [("elasticity", 6, 63), ("elasticity", 8, 24), ("laplace27x4", 6, 64),
                                           ("laplace27x4", 7, 32)])
def test_factor_parity_vector_stencils(ctx, kind, side, blk):
    """The mixed-precision and learned-skip configurations' matrices (3 and 4 coupled unknowns
    per node, 27-point couplings) at small sizes: FP64 factor against the oracle."""
    if kind == "elasticity":
        w = W.elasticity3d(side=side, seed=2, block=blk)
    else:
        w = W.laplace27_4dof(side=side, seed=3, block=blk)
    g = gpu_factor(ctx, w.A, w.droptol, _fixed(blk))
    compare_factors(_oracle(w.A, g.bstart, w.droptol), g, A=w.A, tau=w.droptol)


def test_factor_is_deterministic(ctx):
    A = W.convdiff_upwind((16, 16, 16), seed=5)
    g1 = gpu_factor(ctx, A, 1e-2, _fixed(32))
    g2 = gpu_factor(ctx, A, 1e-2, _fixed(32))
    for f in ("Lrow", "Lval", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(g1, f), getattr(g2, f)), f


def test_apply_parity(ctx):
    import torch
    A = W.convdiff_upwind((16, 16, 16), seed=2)
    g = gpu_factor(ctx, A, 1e-2, _fixed(16))
    o = _oracle(A, g.bstart, 1e-2)
    rng = np.random.default_rng(0)
    for _ in range(3):
        r = rng.standard_normal(A.n)
        zo = O.bilu_apply(o, r)
        rt = torch.from_numpy(r).cuda()
        zt = torch.empty_like(rt)
        B.bilu_apply(ctx, rt, zt)
        torch.cuda.synchronize()
        zg = zt.cpu().numpy()
        assert np.abs(zg - zo).max() <= 1e-11 * np.abs(zo).max()
    # host vectors through the same entry point
    zh = np.zeros(A.n)
    B.bilu_apply(ctx, r, zh)
    assert np.abs(zh - zo).max() <= 1e-11 * np.abs(zo).max()


@pytest.mark.parametrize("case", ["cd2d", "cd3d16", "cd3d24"])
def test_gmres_parity(ctx, case):
    import torch
    if case == "cd2d":
        w = W.cd2d_32()
        A, b, blk = w.A, w.b, 32
    else:
        side = 16 if case == "cd3d16" else 24
        A = W.convdiff_upwind((side,) * 3, seed=1)
        b, blk = W.rhs_ones(A), side
    g = gpu_factor(ctx, A, 1e-2, _fixed(blk), export=False)
    o = _oracle(A, g.bstart, 1e-2)
    ro = O.gmres(A, o, b, tol=1e-8, restart=30)
    bt = torch.from_numpy(b).cuda()
    xt = torch.zeros_like(bt)
    info = B.gmres_solve(ctx, bt, xt, 1e-8, 30, 10000)
    assert info.status == B.BILU_OK
    assert info.iters == ro.iters, (info.iters, ro.iters)
    assert info.relres_true <= 1e-8
    x = xt.cpu().numpy()
    assert np.abs(x - ro.x).max() <= 1e-6 * np.abs(ro.x).max()
    # host vectors
    xh = np.zeros(A.n)
    info2 = B.gmres_solve(ctx, b, xh, 1e-8, 30, 10000)
    assert info2.iters == ro.iters and np.array_equal(xh, x)


def test_singular_block_status(ctx):
    Ad = np.array([[2.0, 0.0, 1.0], [1.0, 0.0, 5.0], [0.5, 1.0, 4.0]])
    A = W.from_dense(Ad)
    p = B.bilu_params_default(blocking=B.BILU_BLOCKING_FIXED, fixed_block=2, max_block=2)
    g = gpu_factor(ctx, A, 0.0, p)
    assert g.status == B.BILU_PERTURBED
    o = O.bilu_factor(A, np.array([0, 2, 3], np.int32), 0.0)
    compare_factors(o, g)
    p.perturb = 0
    with pytest.raises(B.BiluError) as e:
        gpu_factor(ctx, A, 0.0, p)
    assert e.value.status == B.BILU_ERR_SINGULAR
    # [[1,1],[1,1]]: breakdown at pivot 2, perturbed at the diagonal
    A2 = W.from_dense(np.array([[1.0, 1.0], [1.0, 1.0]]))
    g2 = gpu_factor(ctx, A2, 0.0, B.bilu_params_default(fixed_block=2, max_block=2))
    o2 = O.bilu_factor(A2, np.array([0, 2], np.int32), 0.0)
    compare_factors(o2, g2)
    # a zero row in the pivot block; a breakdown whose diagonal entry is within a factor of two
    # of the column's largest (perturbed at the diagonal) or not (perturbed at the largest)
    for Ad3, bs3 in ((np.array([[2.0, 1.0, 0.5], [0.0, 0.0, 3.0], [1.0, 0.5, 4.0]]), [0, 2, 3]),
                     (np.array([[1.0, 2.0], [0.75, 1.5]]), [0, 2]),
                     (np.array([[1.0, 2.0], [0.25, 0.5]]), [0, 2])):
        A3 = W.from_dense(Ad3)
        g3 = gpu_factor(ctx, A3, 0.0, B.bilu_params_default(blocking=B.BILU_BLOCKING_FIXED, fixed_block=2, max_block=2))
        assert g3.status == B.BILU_PERTURBED
        compare_factors(O.bilu_factor(A3, np.array(bs3, np.int32), 0.0), g3)


@pytest.mark.parametrize("name", TG.factor_fixtures())
def test_gpu_matches_worked_example(ctx, name):
    """The hand-derived worked examples of tests/golden, factored by the library."""
    g = TG.load(name)
    A = W.from_dense(TG.frac(g["A"]))
    b = int(np.diff(g["bstart"]).max())
    G = gpu_factor(ctx, A, TG.frac(g["tau"]), _fixed(b))
    assert G.status == B.BILU_OK and list(G.bstart) == g["bstart"]
    TG.check_factor(g, G, rtol=1e-14)


def test_cosine_blocking_end_to_end(ctx):
    """Sec. 3.2 then Sec. 2.2 / Sec. 4: a Q1 elasticity matrix (3 unknowns per node) in a
    random ordering; the library's cosine blocking finds the node blocks, the permuted matrix
    is factored with that partition (bilu_analyze_partition), and factor and GMRES(30) match
    the oracle on the same matrix and partition."""
    w = W.elasticity3d(side=5, seed=2, block=63)
    scramble = np.random.default_rng(11).permutation(w.A.n).astype(np.int32)
    A1 = W.CSR(w.A.n, *B.bilu_permute_csr(w.A.n, w.A.rowptr, w.A.colind, w.A.val, scramble))
    perm, bs = B.bilu_cosine_blocking(A1.n, A1.rowptr, A1.colind, 0.8, 64)
    assert np.diff(bs).max() == 3 and (np.diff(bs) == 3).sum() >= 50
    A2 = W.CSR(A1.n, *B.bilu_permute_csr(A1.n, A1.rowptr, A1.colind, A1.val, perm))
    g = gpu_factor(ctx, A2, w.droptol, bstart=bs)
    assert np.array_equal(g.bstart, bs)
    o = _oracle(A2, bs, w.droptol)
    compare_factors(o, g, A=A2, tau=w.droptol)
    b = W.rhs_ones(A2)
    ro = O.gmres(A2, o, b, tol=1e-8, restart=30)
    x = np.zeros(A2.n)
    info = B.gmres_solve(ctx, b, x, 1e-8, 30, 10000)
    assert info.status == B.BILU_OK and info.iters == ro.iters, (info.iters, ro.iters)
    assert np.abs(x - ro.x).max() <= 1e-6 * np.abs(ro.x).max()


def test_cosine_blocks_merged_by_ilu1t_end_to_end(ctx):
    """Sec. 3.2 then Sec. 3.4: the cosine blocks of a scrambled elasticity matrix, merged whole
    by the ILU(1,tau) growth rule inside bilu_analyze_partition (BILU_BLOCKING_ILU1T); the
    partition equals the oracle's, and factor and GMRES(30) match the oracle on it."""
    w = W.elasticity3d(side=5, seed=2, block=63)
    scramble = np.random.default_rng(11).permutation(w.A.n).astype(np.int32)
    A1 = W.CSR(w.A.n, *B.bilu_permute_csr(w.A.n, w.A.rowptr, w.A.colind, w.A.val, scramble))
    perm, groups = B.bilu_cosine_blocking(A1.n, A1.rowptr, A1.colind, 0.8, 64)
    A2 = W.CSR(A1.n, *B.bilu_permute_csr(A1.n, A1.rowptr, A1.colind, A1.val, perm))
    p = B.bilu_params_default(blocking=B.BILU_BLOCKING_ILU1T, max_block=63, tau_analyze=1e-2)
    g = gpu_factor(ctx, A2, w.droptol, p, bstart=groups)
    want = O.partition_ilu1t_groups(A2, 1e-2, 63, groups)
    assert np.array_equal(g.bstart, want) and len(want) < len(groups)
    o = _oracle(A2, want, w.droptol)
    compare_factors(o, g, A=A2, tau=w.droptol)
    b = W.rhs_ones(A2)
    ro = O.gmres(A2, o, b, tol=1e-8, restart=30)
    x = np.zeros(A2.n)
    info = B.gmres_solve(ctx, b, x, 1e-8, 30, 10000)
    assert info.status == B.BILU_OK and info.iters == ro.iters, (info.iters, ro.iters)


def test_matching_and_scaling_end_to_end(ctx):
    """Sec. 3.1 then Sec. 2.2 / Sec. 4: a convection-diffusion matrix with its rows in a random
    order (zeros on the diagonal; the oracle's factor of it fails as singular) is matched and
    scaled on the host, A^ = D_l A D_r Pi; the library factors A^ and solves A^ y = D_l b like
    the oracle, and x = D_r Pi y solves A x = b."""
    A0 = W.convdiff_upwind((8, 8, 8), seed=2)
    rows = np.random.default_rng(5).permutation(A0.n).astype(np.int32)
    A = W.CSR(A0.n, *B.bilu_scale_permute_csr(A0.n, A0.rowptr, A0.colind, A0.val, rowperm=rows))
    sigma, dl, dr = B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
    Ah = W.CSR(A.n, *B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, None, sigma, dl, dr))
    g = gpu_factor(ctx, Ah, 1e-2, _fixed(8))
    assert g.status == B.BILU_OK
    o = _oracle(Ah, g.bstart, 1e-2)
    compare_factors(o, g, A=Ah, tau=1e-2)
    b = np.random.default_rng(1).standard_normal(A.n)
    ro = O.gmres(Ah, o, dl * b, tol=1e-8, restart=30)
    y = np.zeros(A.n)
    info = B.gmres_solve(ctx, dl * b, y, 1e-8, 30, 10000)
    assert info.status == B.BILU_OK and info.iters == ro.iters, (info.iters, ro.iters)
    x = np.zeros(A.n)
    x[sigma] = dr[sigma] * y
    assert np.linalg.norm(O.spmv(A, x) - b) <= 1e-7 * np.linalg.norm(b)


def test_analyze_partition_rejects_invalid_partitions(ctx):
    A = W.convdiff_upwind((4, 4, 4), seed=1)
    for bs in ([0, 10, 10, 64], [0, 70], [1, 64], [0, 32]):
        with pytest.raises(B.BiluError) as e:
            B.bilu_analyze_partition(ctx, A.n, A.rowptr, A.colind, A.val, np.array(bs, np.int32))
        assert e.value.status == B.BILU_ERR_ARG


def test_bounded_wait_timeout_leaves_context_usable(ctx):
    A = W.convdiff_upwind((8, 8, 8), seed=1)
    B.bilu_debug_set(ctx, B.BILU_DEBUG_SPIN_LIMIT, 20000)
    B.bilu_debug_set(ctx, B.BILU_DEBUG_EXTRA_CTA, 1)
    try:
        with pytest.raises(B.BiluError) as e:
            gpu_factor(ctx, A, 1e-2, _fixed(8), export=False)
        assert e.value.status == B.BILU_ERR_TIMEOUT
    finally:
        B.bilu_debug_set(ctx, B.BILU_DEBUG_EXTRA_CTA, 0)
        B.bilu_debug_set(ctx, B.BILU_DEBUG_SPIN_LIMIT, 0)
    g = gpu_factor(ctx, A, 1e-2, _fixed(8))
    compare_factors(O.bilu_factor(A, g.bstart, 1e-2), g, A=A, tau=1e-2)


def test_argument_and_state_errors(ctx):
    c = B.bilu_create(0)
    try:
        with pytest.raises(B.BiluError) as e:
            B.bilu_factor(c, 1e-2)
        assert e.value.status == B.BILU_ERR_STATE
        A = W.convdiff_upwind((4, 4, 4), seed=1)
        bad = A.val.copy()
        bad[3] = np.nan
        with pytest.raises(B.BiluError) as e:
            B.bilu_analyze(c, A.n, A.rowptr, A.colind, bad)
        assert e.value.status == B.BILU_ERR_ARG
        ci = A.colind.copy()
        ci[1], ci[2] = ci[2], ci[1]
        with pytest.raises(B.BiluError) as e:
            B.bilu_analyze(c, A.n, A.rowptr, ci, A.val)
        assert e.value.status == B.BILU_ERR_ARG
        with pytest.raises(B.BiluError) as e:
            B.bilu_analyze(c, A.n, A.rowptr, A.colind, A.val, B.bilu_params_default(fixed_block=65, max_block=65))
        assert e.value.status == B.BILU_ERR_ARG
        B.bilu_analyze(c, A.n, A.rowptr, A.colind, A.val)
        with pytest.raises(B.BiluError) as e:
            B.bilu_factor(c, -1.0)
        assert e.value.status == B.BILU_ERR_ARG
    finally:
        B.bilu_destroy(c)


def test_empty_matrix(ctx):
    c = B.bilu_create(0)
    try:
        B.bilu_analyze(c, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
        assert B.bilu_factor(c, 1e-2) == B.BILU_OK
        info = B.gmres_solve(c, np.zeros(0), np.zeros(0))
        assert info.iters == 0
    finally:
        B.bilu_destroy(c)


@pytest.mark.parametrize("case", ["diagonal", "drop_all", "n1"])
def test_degenerate_factors(ctx, case):
    """Degenerate cases of the method: a diagonal matrix (no candidate anywhere, ragged
    blocks), tau so large that every candidate is dropped (the preconditioner is block
    Jacobi), and n = 1.  Factor and GMRES(30) against the oracle."""
    if case == "diagonal":
        A = W.from_dense(np.diag(np.random.default_rng(3).uniform(1.0, 5.0, 100)))
        tau, blk = 1e-2, 7
    elif case == "drop_all":
        A = W.convdiff_upwind((8, 8, 8), seed=2)
        tau, blk = 1e300, 8
    else:
        A = W.from_dense(np.array([[3.0]]))
        tau, blk = 1e-2, 1
    g = gpu_factor(ctx, A, tau, _fixed(blk))
    o = _oracle(A, g.bstart, tau)
    assert g.Lrow.size == 0 and g.Ucol.size == 0 and o.Lrow.size == 0 and o.Ucol.size == 0
    compare_factors(o, g)
    b = W.rhs_ones(A)
    ro = O.gmres(A, o, b, tol=1e-8, restart=30)
    x = np.zeros(A.n)
    info = B.gmres_solve(ctx, b, x, 1e-8, 30, 10000)
    assert info.status == B.BILU_OK and info.iters == ro.iters, (info.iters, ro.iters)
    assert np.abs(x - ro.x).max() <= 1e-6 * np.abs(ro.x).max()


def test_algorithmic_flop_counters_match_oracle(ctx):
    """The factor kernel counts its algorithmic work on the device; the integer counts
    equal the oracle's (same candidate sets, same update shapes).  Candidates that the norm
    bound of the scaling phase drops are not scaled: their 2 b^2 flops are the difference."""
    A = W.convdiff_upwind((16, 16, 16), seed=1)
    g = gpu_factor(ctx, A, 1e-2, _fixed(32), export=False)
    o = _oracle(A, g.bstart, 1e-2)
    c, s = o.counters, g.stats
    assert s.flop_upd_l == c["flop_upd_L"] and s.flop_upd_u == c["flop_upd_U"]
    assert s.bound_drops > 0
    assert s.flop_scale + 2 * 32 * 32 * s.bound_drops == c["flop_scale"] and s.flop_norm == c["flop_norm"]
    assert s.cand_rows == c["cand_rows"] and s.cand_cols == c["cand_cols"]
    total = sum(c[k] for k in ("flop_upd_L", "flop_upd_U", "flop_getrf", "flop_inv", "flop_scale", "flop_norm"))
    assert abs(s.flops_factor + 2 * 32 * 32 * s.bound_drops - total) <= 1e-9 * total


def test_newton_reciprocal_within_one_ulp_of_ieee(ctx):
    """The kernels replace FP64 divisions on critical paths by a Newton-Raphson reciprocal;
    it must stay within one ulp of CUDA's IEEE quotient."""
    B.bilu_debug_set(ctx, B.BILU_DEBUG_SELFTEST_RECIP, 1 << 20)


@pytest.mark.parametrize("side,blk", [(16, 16), (20, 40), (24, 64)])
def test_norm_bound_skip_gives_identical_factor(ctx, side, blk):
    """BILU_SKIP_BOUND skips the products of candidate rows / columns that the triangle
    inequality proves dropped (||l_i|| <= ||T_L[i,:]|| ||D_K||_F <= tau); the factor is the
    same bit for bit, and the skip does fire on these stencils."""
    A = W.convdiff_upwind((side, side, side), seed=1)
    g0 = gpu_factor(ctx, A, 1e-2, _fixed(blk))
    p = _fixed(blk)
    p.skip = B.BILU_SKIP_BOUND
    g1 = gpu_factor(ctx, A, 1e-2, p)
    for f in ("Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(g0, f), getattr(g1, f)), f
    assert g1.stats.skipped_rows + g1.stats.skipped_cols > 0
    assert g1.stats.flop_upd_l + g1.stats.flop_upd_u < g0.stats.flop_upd_l + g0.stats.flop_upd_u
    compare_factors(_oracle(A, g1.bstart, 1e-2), g1, A=A, tau=1e-2)


def test_batched_factor_and_gmres_match_one_by_one(ctx):
    """Several uneven matrices factored in one launch (groups of CTAs, work queue) give the
    same factors, bit for bit, as one-by-one factorizations -- on the first call (group size
    from the count), the second (candidates timed), the third (tuned size) and with forced
    group sizes of 1 and 3 CTAs -- and the batched GMRES (one graph, a branch per system) the
    same iteration counts and solutions."""
    import torch
    ws = W.cd_batch(count=6, seed0=100, n_lo=300, n_hi=3000, block=16)
    ctxs = [B.bilu_create(0) for _ in ws]
    B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_POISON, 1)  # an unwritten value shows as NaN
    try:
        for c, w in zip(ctxs, ws):
            B.bilu_analyze(c, w.A.n, w.A.rowptr, w.A.colind, w.A.val,
                           B.bilu_params_default(fixed_block=w.fixed_block, max_block=64))
        singles, xsingle, ref = [], [], []
        for w in ws:
            g1 = gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(fixed_block=w.fixed_block, max_block=64))
            ref.append(g1)
            bt = torch.from_numpy(w.b).cuda()
            x1 = torch.zeros_like(bt)
            singles.append(B.gmres_solve(ctx, bt, x1, 1e-8, 30, 10000).iters)
            xsingle.append(x1.cpu().numpy())

        def check_factors(tag):
            for c, w, g1 in zip(ctxs, ws, ref):
                s = B.bilu_stats(c)
                arrs = dict(Lptr=np.zeros(s.nblocks + 1, np.int64), Lrow=np.zeros(s.kept_rows, np.int32),
                            Lval=np.zeros(s.nnz_l), Uptr=np.zeros(s.nblocks + 1, np.int64),
                            Ucol=np.zeros(s.kept_cols, np.int32), Uval=np.zeros(s.nnz_u),
                            Dinv=np.zeros(s.nnz_d), Pblk=np.zeros(s.nnz_d))
                B.bilu_export(c, **arrs)
                for k, v in arrs.items():
                    assert np.array_equal(v, getattr(g1, k)), (tag, w.name, k)

        for call in range(3):
            B.bilu_factor_batch(ctxs, 1e-2)
            check_factors(f"call {call}")
        try:
            for G in (1, 3):
                B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_BATCH_GROUP, G)
                B.bilu_factor_batch(ctxs, 1e-2)
                check_factors(f"G={G}")
        finally:
            B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_BATCH_GROUP, 0)
        # from minimal storage: every matrix is re-run (inside the batch launch) with grown
        # pools and producer lists, the factors are still the same
        small = [B.bilu_create(0) for _ in ws]
        try:
            B.bilu_debug_set(small[0], B.BILU_DEBUG_SMALL_POOLS, 1)
            for c, w in zip(small, ws):
                B.bilu_analyze(c, w.A.n, w.A.rowptr, w.A.colind, w.A.val,
                               B.bilu_params_default(fixed_block=w.fixed_block, max_block=64))
            B.bilu_factor_batch(small, 1e-2)
            assert all(B.bilu_stats(c).pool_retries > 0 for c in small)
            ctxs, kept = small, ctxs
            check_factors("small pools")
            ctxs = kept
        finally:
            B.bilu_debug_set(small[0], B.BILU_DEBUG_SMALL_POOLS, 0)
            for c in small:
                B.bilu_destroy(c)
        bs = [torch.from_numpy(w.b).cuda() for w in ws]
        for rep in range(2):
            xs = [torch.zeros_like(v) for v in bs]
            infos = B.gmres_solve_batch(ctxs, bs, xs, 1e-8, 30, 10000)
            assert [i.iters for i in infos] == singles
            assert all(i.relres_true <= 1e-8 for i in infos)
            for x, x1 in zip(xs, xsingle):  # same kernels, same order: the same solution
                assert np.array_equal(x.cpu().numpy(), x1)
    finally:
        B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_POISON, 0)
        for c in ctxs:
            B.bilu_destroy(c)


@pytest.mark.parametrize("G,cap", [(1, 0), (2, 0), (5, 0), (5, 4), (2, 8)])
def test_batched_small_groups_large_blocks(ctx, G, cap):
    """Groups with fewer CTAs than half a block's columns (the inverse D_K = P_K^{-1} then
    takes several columns per CTA and several rounds), and update tiles capped at fewer
    candidate rows (cap; 0: the tuned cap): same factors as one by one, with every value
    array filled with NaN before each run."""
    ws = W.cd_batch(count=3, seed0=200, n_lo=1500, n_hi=4000, block=48)
    ctxs = [B.bilu_create(0) for _ in ws]
    B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_POISON, 1)
    B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_BATCH_GROUP, G)
    B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_BATCH_TRCAP, cap)
    try:
        for c, w in zip(ctxs, ws):
            B.bilu_analyze(c, w.A.n, w.A.rowptr, w.A.colind, w.A.val,
                           B.bilu_params_default(fixed_block=w.fixed_block, max_block=64))
        B.bilu_factor_batch(ctxs, 1e-2)
        for c, w in zip(ctxs, ws):
            g1 = gpu_factor(ctx, w.A, 1e-2, B.bilu_params_default(fixed_block=w.fixed_block, max_block=64))
            s = B.bilu_stats(c)
            assert s.nblocks == len(g1.bstart) - 1
            arrs = dict(Lptr=np.zeros(s.nblocks + 1, np.int64), Lrow=np.zeros(s.kept_rows, np.int32),
                        Lval=np.zeros(s.nnz_l), Uptr=np.zeros(s.nblocks + 1, np.int64),
                        Ucol=np.zeros(s.kept_cols, np.int32), Uval=np.zeros(s.nnz_u),
                        Dinv=np.zeros(s.nnz_d), Pblk=np.zeros(s.nnz_d))
            B.bilu_export(c, **arrs)
            for k, v in arrs.items():
                assert np.array_equal(v, getattr(g1, k)), (w.name, k)
    finally:
        B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_BATCH_GROUP, 0)
        B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_BATCH_TRCAP, 0)
        B.bilu_debug_set(ctxs[0], B.BILU_DEBUG_POISON, 0)
        for c in ctxs:
            B.bilu_destroy(c)


def test_factor_rerun_from_minimal_storage(ctx):
    """A factorization that starts from minimal pools and producer lists runs again with
    grown storage until it fits, and ends with the same factor, bit for bit."""
    A = W.cd3d(side=12, seed=3, block=12).A
    p = B.bilu_params_default(fixed_block=12, max_block=64)
    ref = gpu_factor(ctx, A, 1e-2, p)
    c = B.bilu_create(0)
    try:
        B.bilu_debug_set(c, B.BILU_DEBUG_SMALL_POOLS, 1)
        g = gpu_factor(c, A, 1e-2, p)
        assert B.bilu_stats(c).pool_retries >= 2
    finally:
        B.bilu_debug_set(c, B.BILU_DEBUG_SMALL_POOLS, 0)
        B.bilu_destroy(c)
    for k in ("Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(g, k), getattr(ref, k)), k
