"""GPU parity at the benchmark's full sizes, on sampled outputs: blocks of the factorization
recomputed by the oracle's single-step checker from the GPU's own earlier blocks, and the true
residual of the GMRES solution.  The 64^3 case runs in the launch configuration bench.py times
(one persistent cooperative launch over all SMs); the batch case is the 64-system workload."""
import numpy as np
import pytest

from oracle import block_check as BC
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W
from tests.gpu_helpers import gpu_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.bilu_create(0)
    yield c
    B.bilu_destroy(c)


def _exp(g):
    return {"bstart": g.bstart, "Lptr": g.Lptr, "Lrow": g.Lrow, "Lval": g.Lval, "Uptr": g.Uptr, "Ucol": g.Ucol,
            "Uval": g.Uval, "Dinv": g.Dinv, "Pblk": g.Pblk}


def _residual(A, b, x):
    return float(np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b))


def test_cd3d64_sampled_blocks_and_solution(ctx):
    """64^3 upwind convection-diffusion, blocks of 64 (the benchmark workload)."""
    import torch
    w = W.cd3d(side=64, seed=1, block=64)
    g = gpu_factor(ctx, w.A, w.droptol, B.bilu_params_default(fixed_block=64, max_block=64))
    E = _exp(g)
    blocks = BC._blocks(E)
    nb = len(g.bstart) - 1
    rng = np.random.default_rng(0)
    sample = sorted(set([0, 1, 2, 63, 64, 65, nb // 2, nb - 2, nb - 1] + list(rng.integers(0, nb, 6))))
    flips = 0
    for K in sample:
        f, err = BC.compare_block(w.A, E, K, w.droptol, rtol=1e-10, blocks=blocks)
        flips += f
    assert flips == 0
    bt = torch.from_numpy(w.b).cuda()
    x = torch.zeros_like(bt)
    info = B.gmres_solve(ctx, bt, x, 1e-8, 30, 10000)
    assert info.iters == 24  # the oracle's count on this matrix (bench.py's CPU baseline)
    assert _residual(w.A, w.b, x.cpu().numpy()) <= 1e-8


def test_laplace27x4_64_sampled_blocks_and_solution(ctx):
    """The learned skip's evaluation matrix at full size, plain FP64 (the method without the
    skip): Q1 27-point operator on 64^3 nodes with 4 coupled unknowns per node, n = 1,048,576,
    blocks of 64, natural order.  Sampled blocks against the oracle's single-step checker, and
    the GMRES solution's true residual."""
    import torch
    w = W.laplace27_4dof(side=64, seed=3, block=64)
    g = gpu_factor(ctx, w.A, w.droptol, B.bilu_params_default(fixed_block=64, max_block=64))
    E = _exp(g)
    blocks = BC._blocks(E)
    nb = len(g.bstart) - 1
    flips = 0
    for K in (0, 1, 2, 255, 256, nb // 2, nb - 2, nb - 1):
        f, err = BC.compare_block(w.A, E, K, w.droptol, rtol=1e-10, blocks=blocks)
        flips += f
    assert flips == 0
    bt = torch.from_numpy(w.b).cuda()
    x = torch.zeros_like(bt)
    info = B.gmres_solve(ctx, bt, x, 1e-8, 30, 10000)
    assert _residual(w.A, w.b, x.cpu().numpy()) <= 1e-8
    print(f"laplace27x4 64^3: {nb} blocks, GMRES {info.iters} iterations")


@pytest.mark.parametrize("prec,u_store", [(B.BILU_PREC_FP32, BC.U_FP32), (B.BILU_PREC_BF16, BC.U_BF16)])
def test_cd3d64_mixed_precision_sampled_blocks(ctx, prec, u_store):
    """FP32 updates (or BF16 storage) at full size: every sampled block equals the FP64 step
    recomputed from the GPU's own earlier blocks within twice the first-order error bound of a
    step in that arithmetic (oracle/block_check.py, step_bounds); drop decisions differ only
    within twice the norm's bound of the threshold."""
    w = W.cd3d(side=64, seed=1, block=64)
    g = gpu_factor(ctx, w.A, w.droptol, B.bilu_params_default(fixed_block=64, max_block=64, precision=prec))
    E = _exp(g)
    blocks = BC._blocks(E)
    nb = len(g.bstart) - 1
    for K in (0, 1, 64, nb // 2, nb - 1):
        BC.compare_block_bounded(w.A, E, K, w.droptol, BC.U_FP32, BC.U_FP32, u_store, blocks=blocks)


def test_batch64_sampled_blocks(ctx):
    """The 64-system batch (one launch, FP32 updates): sampled blocks of the largest 2D and 3D
    systems against the FP64 step from their own earlier blocks (within twice the FP32 step's
    error bound), all systems solved to 1e-8."""
    import torch
    ws = W.cd_batch(count=64, seed0=100)
    ctxs = [B.bilu_create(0) for _ in ws]
    try:
        for c, w in zip(ctxs, ws):
            B.bilu_analyze(c, w.A.n, w.A.rowptr, w.A.colind, w.A.val,
                           B.bilu_params_default(fixed_block=w.fixed_block, max_block=64, precision=B.BILU_PREC_FP32))
        B.bilu_factor_batch(ctxs, 1e-2)
        big2 = max((k for k in range(64) if "cd2d" in ws[k].name), key=lambda k: ws[k].A.n)
        big3 = max((k for k in range(64) if "cd3d" in ws[k].name), key=lambda k: ws[k].A.n)
        for k in (big2, big3):
            c, w = ctxs[k], ws[k]
            s = B.bilu_stats(c)
            bs = np.zeros(s.nblocks + 1, np.int32)
            B.bilu_get_partition(c, bs)
            E = {"bstart": bs, "Lptr": np.zeros(s.nblocks + 1, np.int64), "Lrow": np.zeros(s.kept_rows, np.int32),
                 "Lval": np.zeros(s.nnz_l), "Uptr": np.zeros(s.nblocks + 1, np.int64),
                 "Ucol": np.zeros(s.kept_cols, np.int32), "Uval": np.zeros(s.nnz_u), "Dinv": np.zeros(s.nnz_d),
                 "Pblk": np.zeros(s.nnz_d)}
            B.bilu_export(c, E["Lptr"], E["Lrow"], E["Lval"], E["Uptr"], E["Ucol"], E["Uval"], E["Dinv"], E["Pblk"])
            blocks = BC._blocks(E)
            nb = s.nblocks
            for K in (0, 1, nb // 3, nb // 2, nb - 1):
                BC.compare_block_bounded(w.A, E, K, w.droptol, BC.U_FP32, BC.U_FP32, BC.U_FP32, blocks=blocks)
        bs_ = [torch.from_numpy(w.b).cuda() for w in ws]
        xs = [torch.zeros_like(v) for v in bs_]
        infos = B.gmres_solve_batch(ctxs, bs_, xs, 1e-8, 30, 10000)
        for w, x, i in zip(ws, xs, infos):
            assert i.relres_true <= 1e-8
            assert _residual(w.A, w.b, x.cpu().numpy()) <= 1.5e-8
    finally:
        for c in ctxs:
            B.bilu_destroy(c)
