"""The BF16 update tiles on the tensor cores (tcgen05 MMA, BF16 operands, FP32 accumulation
in tensor memory) against the same factorization with the update tiles on the FP32 units.

Both sum the same exact BF16 products in FP32, in different orders, so the stored BF16 values
differ by at most a few units in their last place, and a drop decision may flip only for a
candidate whose norm lies within that rounding of tau.  The step parity of the BF16 factor
against the FP64 oracle (tests/test_gpu_mixed.py) runs on the tensor path as well."""
import numpy as np
import pytest

import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W
from tests.gpu_helpers import _vptr, gpu_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.bilu_create(0)
    yield c
    B.bilu_destroy(c)


def _factor(ctx, w, tensor, sched=B.BILU_SCHED_CHAIN, bs=None):
    B.bilu_debug_set(ctx, B.BILU_DEBUG_NO_TENSOR, 0 if tensor else 1)
    try:
        p = B.bilu_params_default(fixed_block=w.fixed_block, max_block=64, precision=B.BILU_PREC_BF16, schedule=sched)
        return gpu_factor(ctx, w.A, w.droptol, p, bstart=bs)
    finally:
        B.bilu_debug_set(ctx, B.BILU_DEBUG_NO_TENSOR, 0)


def _iters(ctx, w):
    import torch
    b = torch.from_numpy(w.b).cuda()
    x = torch.zeros_like(b)
    info = B.gmres_solve(ctx, b, x, 1e-8, 30, 10000)
    assert info.relres_true <= 1e-8
    return info.iters


@pytest.mark.parametrize("case", ["cd3d16", "elasticity6"])
def test_tensor_tiles_agree_with_fp32_unit_tiles(ctx, case):
    w = W.cd3d(side=16, seed=1, block=32) if case == "cd3d16" else W.elasticity3d(side=6, seed=2, block=24)
    gt = _factor(ctx, w, True)
    it_t = _iters(ctx, w)
    gf = _factor(ctx, w, False)
    it_f = _iters(ctx, w)
    # the same algorithmic work
    assert gt.stats.flop_upd_l == gf.stats.flop_upd_l and gt.stats.flop_upd_u == gf.stats.flop_upd_u
    nb = len(gt.bstart) - 1
    differ, worst = 0, 0.0
    for K in range(nb):
        b = int(gt.bstart[K + 1] - gt.bstart[K])
        same = (np.array_equal(gt.Lrow[gt.Lptr[K]:gt.Lptr[K + 1]], gf.Lrow[gf.Lptr[K]:gf.Lptr[K + 1]]) and
                np.array_equal(gt.Ucol[gt.Uptr[K]:gt.Uptr[K + 1]], gf.Ucol[gf.Uptr[K]:gf.Uptr[K + 1]]))
        if not same:
            differ += 1
            break  # the later blocks follow different patterns
        for (pa, pb, va, vb, vp) in ((gt.Lptr, gf.Lptr, gt.Lval, gf.Lval, _vptr(gt.Lptr, gt.bstart)),
                                     (gt.Uptr, gf.Uptr, gt.Uval, gf.Uval, _vptr(gt.Uptr, gt.bstart))):
            a, c = va[vp[K]:vp[K + 1]], vb[vp[K]:vp[K + 1]]
            if a.size:
                a2, c2 = a.reshape(-1, b), c.reshape(-1, b)
                worst = max(worst, float((np.abs(a2 - c2).max(axis=1) / np.abs(c2).max(axis=1)).max()))
    print(f"{case}: kept sets of all {nb} blocks equal: {differ == 0}; worst row difference {worst:.2e}; "
          f"GMRES {it_t} (tensor) / {it_f} (FP32 units)")
    # BF16 stores 8 significant bits: rows agree to a few units of 2^-8 relative to the row
    assert worst <= 4 * 2.0 ** -8
    assert abs(it_t - it_f) <= max(1, it_f // 10)


def test_tensor_tiles_same_factor_on_every_schedule(ctx):
    """The tile a row falls in does not change its MMA sums (the contraction of one output runs
    over its own k only), so the chain and tree schedules give the same BF16 factor bit for bit."""
    w = W.cd3d(side=16, seed=1, block=32)
    n = w.A.n
    perm, bnd, _ = B.bilu_nd_order(n, w.A.rowptr, w.A.colind, np.append(np.arange(0, n, 32), n).astype(np.int32))
    A2 = W.CSR(n, *B.bilu_permute_csr(n, w.A.rowptr, w.A.colind, w.A.val, perm))
    import dataclasses
    w2 = dataclasses.replace(w, A=A2)
    gc = _factor(ctx, w2, True, B.BILU_SCHED_CHAIN, bnd)
    gt = _factor(ctx, w2, True, B.BILU_SCHED_TREE, bnd)
    for k in ("Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(gc, k), getattr(gt, k)), k


@pytest.mark.parametrize("prec,tol", [(B.BILU_PREC_FP32, 1e-5), (B.BILU_PREC_BF16, 2e-2)])
def test_reduced_precision_sweeps_against_a_dense_solve(ctx, prec, tol):
    """The sweeps of a reduced-precision factor run in FP32 arithmetic: z = M^{-1} r agrees with
    a dense FP64 solve with M = L U-breve assembled from the exported (widened) factor.  The
    backward sweep multiplies by D_K U-breve_K as the factor stored it, rounded to the storage
    format, so the two agree to that rounding (FP32: 2^-24, BF16: 2^-8) amplified by M's
    conditioning, plus FP32 arithmetic."""
    import torch
    w = W.cd3d(side=12, seed=2, block=24)
    g = gpu_factor(ctx, w.A, w.droptol, B.bilu_params_default(fixed_block=24, max_block=64, precision=prec))
    n = w.A.n
    Ld, Ud = np.eye(n), np.zeros((n, n))
    for K in range(len(g.bstart) - 1):
        s0, s1 = int(g.bstart[K]), int(g.bstart[K + 1])
        rows, Lv = g.L_block(K)
        Ld[rows, s0:s1] = Lv
        cols, Uv = g.U_block(K)
        Ud[s0:s1, s0:s1] = g.P_block(K)
        Ud[s0:s1, cols] = Uv.T
    M = Ld @ Ud
    r = np.random.default_rng(9).standard_normal(n)
    zref = np.linalg.solve(M, r)
    rt = torch.from_numpy(r).cuda()
    z = torch.empty_like(rt)
    B.bilu_apply(ctx, rt, z)
    torch.cuda.synchronize()
    zg = z.cpu().numpy()
    err = np.abs(zg - zref).max() / np.abs(zref).max()
    print(f"precision {prec}: sweeps against the dense FP64 solve {err:.2e}")
    assert err <= tol


def test_tensor_tiles_in_the_batched_launch(ctx):
    """The batched launch (groups of CTAs over a queue of matrices) runs the BF16 tiles on the
    tensor cores too: each matrix's factor equals its one-by-one BF16 factor bit for bit (a
    row's MMA sums do not depend on the tile or the group it falls in)."""
    ws = W.cd_batch(count=3, seed0=300, n_lo=1500, n_hi=4000, block=32)
    ctxs = [B.bilu_create(0) for _ in ws]
    try:
        p = lambda w: B.bilu_params_default(fixed_block=w.fixed_block, max_block=64, precision=B.BILU_PREC_BF16)
        for c, w in zip(ctxs, ws):
            B.bilu_analyze(c, w.A.n, w.A.rowptr, w.A.colind, w.A.val, p(w))
        B.bilu_factor_batch(ctxs, 1e-2)
        for c, w in zip(ctxs, ws):
            g1 = gpu_factor(ctx, w.A, 1e-2, p(w))
            s = B.bilu_stats(c)
            arrs = dict(Lptr=np.zeros(s.nblocks + 1, np.int64), Lrow=np.zeros(s.kept_rows, np.int32),
                        Lval=np.zeros(s.nnz_l), Uptr=np.zeros(s.nblocks + 1, np.int64),
                        Ucol=np.zeros(s.kept_cols, np.int32), Uval=np.zeros(s.nnz_u),
                        Dinv=np.zeros(s.nnz_d), Pblk=np.zeros(s.nnz_d))
            B.bilu_export(c, **arrs)
            for k, v in arrs.items():
                assert np.array_equal(v, getattr(g1, k)), (w.name, k)
    finally:
        for c in ctxs:
            B.bilu_destroy(c)
