"""GPU parity of the mixed-precision factorization (FP32 updates and scaling; BF16 storage
with FP32 accumulation; pivot LU, inverse, drop norms and GMRES in FP64).

Bar (step parity): every checked block K of the GPU factor equals the FP64 step recomputed by
the oracle's block checker from the GPU's own earlier blocks, within twice the first-order
componentwise error bound of a step carried out in that arithmetic (oracle/block_check.py,
step_bounds: summation bounds gamma_m sum|terms| for the FP32 accumulation, D_K = P_K^{-1}
perturbed by -D dP D, FP32 scaling, rounding of the stored value).  A drop decision may
differ from the FP64 step's only for a candidate whose norm lies within twice its error bound
of tau; those flips are counted.  GMRES(30) reaches 1e-8 within 10 % (+1) of the FP64
iteration count.  The error of the whole factor against the FP64 oracle (which also holds the
earlier blocks' rounding) is reported."""
import numpy as np
import pytest

from oracle import block_check as BC
import oracle as O
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W
from tests.gpu_helpers import _vptr, gpu_factor

pytestmark = pytest.mark.gpu

PREC = {"fp32": (B.BILU_PREC_FP32, BC.U_FP32), "bf16": (B.BILU_PREC_BF16, BC.U_BF16)}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.bilu_create(0)
    yield c
    B.bilu_destroy(c)


def _exp(g):
    return {k: getattr(g, k) for k in ("bstart", "Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk")}


def _iters(ctx, b):
    import torch
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    info = B.gmres_solve(ctx, bt, x, 1e-8, 30, 10000)
    assert info.status == B.BILU_OK and info.relres_true <= 1e-8
    return info.iters


def _check_blocks(A, g, Ks, tau, u_store):
    E = _exp(g)
    blocks = BC._blocks(E)
    flips, worst, ncand = 0, [], 0
    for K in Ks:
        f, w, nc = BC.compare_block_bounded(A, E, K, tau, BC.U_FP32, BC.U_FP32, u_store, blocks=blocks)
        flips += f
        ncand += nc
        worst.append(w)
    return flips, np.array(worst), ncand


def _vs_fp64_oracle(Fo, g):
    """Largest relative error of L / U-breve rows (columns) against the FP64 oracle over the
    blocks whose kept sets agree, and how many blocks' kept sets differ."""
    oLv, oUv, gLv, gUv = Fo.Lvptr(), Fo.Uvptr(), _vptr(g.Lptr, g.bstart), _vptr(g.Uptr, g.bstart)
    err, differ = 0.0, 0
    for K in range(len(Fo.bstart) - 1):
        b = int(Fo.bstart[K + 1] - Fo.bstart[K])
        ro, rg = Fo.Lrow[Fo.Lptr[K]:Fo.Lptr[K + 1]], g.Lrow[g.Lptr[K]:g.Lptr[K + 1]]
        co, cg = Fo.Ucol[Fo.Uptr[K]:Fo.Uptr[K + 1]], g.Ucol[g.Uptr[K]:g.Uptr[K + 1]]
        if not (np.array_equal(ro, rg) and np.array_equal(co, cg)):
            differ += 1
            continue
        for a, bb in ((Fo.Lval[oLv[K]:oLv[K + 1]], g.Lval[gLv[K]:gLv[K + 1]]),
                      (Fo.Uval[oUv[K]:oUv[K + 1]], g.Uval[gUv[K]:gUv[K + 1]])):
            if a.size:
                a2, b2 = a.reshape(-1, b), bb.reshape(-1, b)
                err = max(err, float((np.abs(a2 - b2).max(axis=1) / np.abs(a2).max(axis=1)).max()))
    return err, differ


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("case", ["cd3d14", "elasticity6"])
def test_mixed_precision_step_parity_every_block(ctx, prec, case):
    if case == "cd3d14":
        A = W.convdiff_upwind((14, 14, 14), seed=1)
        blk = 14
    else:
        A = W.elasticity3d(side=6, seed=2, block=24).A
        blk = 24
    b = W.rhs_ones(A)
    code, us = PREC[prec]
    g64 = gpu_factor(ctx, A, 1e-2, B.bilu_params_default(fixed_block=blk, max_block=64), export=False)
    it64 = _iters(ctx, b)
    g = gpu_factor(ctx, A, 1e-2, B.bilu_params_default(fixed_block=blk, max_block=64, precision=code))
    it = _iters(ctx, b)
    nb = len(g.bstart) - 1
    flips, worst, ncand = _check_blocks(A, g, range(nb), 1e-2, us)
    Fo = O.bilu_factor(A, g.bstart, 1e-2)
    err, differ = _vs_fp64_oracle(Fo, g)
    Fo.free()
    print(f"{case} {prec}: {nb} blocks, {ncand} candidates, {flips} drop decisions within the window; "
          f"error / bound median {np.median(worst):.2e} max {worst.max():.2e}; vs FP64 oracle: "
          f"max row error {err:.2e}, {differ} blocks with other kept sets; GMRES {it} vs {it64}")
    assert it <= 1.1 * it64 + 1, (it, it64)
    assert flips <= 0.01 * ncand


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_elasticity48_mixed_precision_sampled_blocks(ctx, prec):
    """The mixed-precision configuration at full size: Q1 elasticity on 48^3 interior nodes
    (n = 331,776, blocks of 63), sampled blocks against the bounded FP64 step, GMRES(30) within
    10 % of the FP64 iterations."""
    w = W.elasticity3d(side=48, seed=2, block=63)
    code, us = PREC[prec]
    gpu_factor(ctx, w.A, w.droptol, B.bilu_params_default(fixed_block=63, max_block=64), export=False)
    it64 = _iters(ctx, w.b)
    g = gpu_factor(ctx, w.A, w.droptol, B.bilu_params_default(fixed_block=63, max_block=64, precision=code))
    it = _iters(ctx, w.b)
    nb = len(g.bstart) - 1
    rng = np.random.default_rng(5)
    Ks = sorted(set([0, 1, 2, nb // 3, nb // 2, nb - 2, nb - 1] + list(rng.integers(0, nb, 5))))
    flips, worst, ncand = _check_blocks(w.A, g, Ks, w.droptol, us)
    print(f"elasticity 48^3 {prec}: blocks {Ks}: {ncand} candidates, {flips} flips in the window, error / bound "
          f"max {worst.max():.2e}; GMRES {it} vs FP64 {it64}")
    assert it <= 1.1 * it64 + 1, (it, it64)
