"""Pins of the single-block-step checker (oracle/block_check.py, numpy + LAPACK) against the
full C oracle (an independent implementation): recomputing every block of the C oracle's own
factor from its earlier blocks reproduces it, and a planted change is detected."""
import numpy as np
import pytest

import oracle as O
from oracle import block_check as BC
from paper_1908_10169_gb300 import workloads as W


def _export(F):
    return {"bstart": F.bstart, "Lptr": F.Lptr, "Lrow": F.Lrow, "Lval": F.Lval, "Uptr": F.Uptr,
            "Ucol": F.Ucol, "Uval": F.Uval, "Dinv": F.Dinv, "Pblk": F.Pblk}


@pytest.mark.parametrize("case", ["cd2d", "cd3d", "random"])
def test_block_step_reproduces_the_c_oracle(case):
    if case == "cd2d":
        w = W.cd2d_32()
        A, bs, tau = w.A, np.arange(0, w.A.n + 1, 32), w.droptol
    elif case == "cd3d":
        w = W.cd3d(side=8, seed=3, block=16)
        A, bs, tau = w.A, np.arange(0, w.A.n + 1, 16), w.droptol
    else:
        A = W.random_diag_dominant(150, 0.05, seed=4)
        bs, tau = np.array([0, 7, 20, 41, 64, 90, 97, 120, 150]), 3e-2
    F = O.bilu_factor(A, bs, tau)
    E = _export(F)
    blocks = BC._blocks(E)
    worst = 0.0
    for K in range(len(bs) - 1):
        flips, err = BC.compare_block(A, E, K, tau, rtol=1e-12, blocks=blocks)
        assert flips == 0
        worst = max(worst, err)
    assert worst < 1e-12


def test_block_check_detects_a_changed_value():
    w = W.cd3d(side=8, seed=3, block=16)
    bs = np.arange(0, w.A.n + 1, 16)
    F = O.bilu_factor(w.A, bs, w.droptol)
    E = _export(F)
    K = 5
    b = 16
    # perturb one stored value of block K's L part
    lo = int(F.Lptr[K]) * b
    E["Lval"] = E["Lval"].copy()
    E["Lval"][lo + 3] += 1e-8 * np.abs(E["Lval"][lo:lo + b]).max()  # relative change 1e-8 of the row
    with pytest.raises(AssertionError):
        BC.compare_block(w.A, E, K, w.droptol)


def test_block_check_rejects_a_flip_far_from_tau():
    """A kept row of L removed from the factor (its norm far above tau) is a drop decision
    that differs for a reason other than rounding: the checker raises."""
    w = W.cd3d(side=8, seed=3, block=16)
    bs = np.arange(0, w.A.n + 1, 16)
    F = O.bilu_factor(w.A, bs, w.droptol)
    E = _export(F)
    K, b = 5, 16
    p = int(F.Lptr[K])
    lo = p * b
    assert np.linalg.norm(F.Lval[lo:lo + b]) > 10 * w.droptol
    E["Lrow"] = np.delete(F.Lrow, p)
    E["Lval"] = np.delete(F.Lval, np.arange(lo, lo + b))
    E["Lptr"] = F.Lptr.copy()
    E["Lptr"][K + 1:] -= 1
    with pytest.raises(AssertionError, match="drop decision"):
        BC.compare_block(w.A, E, K, w.droptol)


# ---- error bounds of a reduced-precision block step (mixed-precision parity, a9) ----------

def _to_bf16(x):
    """Round to BF16 (nearest, ties to even) through FP32, as __float2bfloat16((float)v)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32)).view(np.uint32)
    r = ((f.astype(np.uint64) + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _dense_factor(F, n):
    """Dense copies of the blocks' kept L rows and U-breve columns of an exported factor."""
    bs = np.asarray(F["bstart"])
    Ls, Us = [], []
    for lr, L, uc, U in BC._blocks(F):
        Ld = np.zeros((n, L.shape[1]))
        Ld[lr] = L
        Ud = np.zeros((U.shape[1], n))
        Ud[:, uc] = U.T
        Ls.append(Ld)
        Us.append(Ud)
    return bs, Ls, Us


def _emulated_step(A, F, K, store):
    """Block step K in emulated reduced precision (numpy FP32; dense, small n): T = A - sum_J
    L_J U-breve_J accumulated in FP32 one producer at a time, P and D = P^{-1} in FP64, l_i =
    T_i fl32(D) in FP32, stored through `store` (FP32 or BF16 rounding)."""
    n = A.n
    Ad = np.zeros((n, n))
    for i in range(n):
        Ad[i, A.colind[A.rowptr[i]:A.rowptr[i + 1]]] = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    bs, Ls, Us = _dense_factor(F, n)
    s0, s1 = int(bs[K]), int(bs[K + 1])
    T = Ad[:, s0:s1].astype(np.float32)
    TU = Ad[s0:s1, :].astype(np.float32)
    for J in range(K):
        T = (T - (Ls[J].astype(np.float32) @ Us[J][:, s0:s1].astype(np.float32))).astype(np.float32)
        TU = (TU - (Ls[J][s0:s1].astype(np.float32) @ Us[J].astype(np.float32))).astype(np.float32)
    P = T[s0:s1].astype(np.float64)
    D = np.linalg.inv(P)
    Lc = (T @ D.astype(np.float32)).astype(np.float32).astype(np.float64)
    return store(Lc), P, D, store(TU.astype(np.float64))


@pytest.mark.parametrize("case", ["cd3d6", "random", "graded", "underflow"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_step_bounds_cover_an_emulated_reduced_precision_step(case, prec):
    """The first-order bounds of step_bounds hold for a step carried out in emulated FP32
    arithmetic (BF16 storage: the inputs are BF16 values and the outputs are rounded to BF16),
    on every block of three problems, one with pivot blocks graded over six decades."""
    if case == "cd3d6":
        A = W.convdiff_upwind((6, 6, 6), seed=4)
        bs = O.partition_fixed(A.n, 6)
    elif case == "random":
        A = W.random_diag_dominant(120, 0.05, 9, dominance=1.05)
        bs = O.partition_fixed(A.n, 8)
    elif case == "underflow":
        # entries of the inverse and of the products far below FP32's smallest normal number
        rng = np.random.default_rng(5)
        M = np.diag(10.0 ** rng.uniform(0, 2, 64)) + np.diag(-1e-30 * rng.random(63), 1) \
            + np.diag(-1e-25 * rng.random(63), -1)
        M[40:, :8] = 1e-38 * rng.standard_normal((24, 8))
        A = W.from_dense(M)
        bs = O.partition_fixed(A.n, 8)
    else:
        rng = np.random.default_rng(3)
        d = 10.0 ** rng.uniform(-3, 3, 96)
        M = np.diag(d) + 0.3 * rng.standard_normal((96, 96)) * np.sqrt(np.outer(d, d)) * (rng.random((96, 96)) < 0.08)
        A = W.from_dense(M)
        bs = O.partition_fixed(A.n, 12)
    Fo = O.bilu_factor(A, bs, 1e-3)
    F = _export(Fo)
    Fo.free()
    store = (lambda x: x.astype(np.float32).astype(np.float64)) if prec == "fp32" else _to_bf16
    if prec == "bf16":  # a BF16 factor's earlier blocks are BF16 values
        F = dict(F, Lval=_to_bf16(F["Lval"]), Uval=_to_bf16(F["Uval"]))
    us = BC.U_FP32 if prec == "fp32" else BC.U_BF16
    worst = []
    for K in range(len(bs) - 1):
        R = BC.block_step(A, F, K, 1e-3, magnitudes=True)
        Bd = BC.step_bounds(R, BC.U_FP32, BC.U_FP32, us)
        Lc, P, D, TU = _emulated_step(A, F, K, store)
        assert np.all(np.abs(P - R.P) <= Bd.P)
        assert np.all(np.abs(D - R.D) <= Bd.D)
        if len(R.lcand):
            exact = R.TL @ R.D
            err = np.abs(Lc[R.lcand] - exact)
            assert np.all(err <= Bd.Lstore), (K, float((err / np.maximum(Bd.Lstore, 1e-300)).max()))
            worst.append(float((err / np.maximum(Bd.Lstore, 1e-300)).max()))
            # the emulation's norm is of the stored values: the window plus the storage rounding
            nerr = np.abs(np.sqrt(np.sum(Lc[R.lcand] ** 2, axis=1)) - R.lnorm)
            assert np.all(nerr <= np.sqrt(np.sum(Bd.Lstore ** 2, axis=1)))
        if len(R.ucand):
            err = np.abs(TU[:, R.ucand].T - R.TU)
            assert np.all(err <= Bd.U)
    assert max(worst) > 0.0  # the emulation does round


def test_step_bounds_vanish_with_the_unit_roundoffs():
    A = W.convdiff_upwind((6, 6, 6), seed=4)
    bs = O.partition_fixed(A.n, 6)
    Fo = O.bilu_factor(A, bs, 1e-3)
    F = _export(Fo)
    Fo.free()
    R = BC.block_step(A, F, 20, 1e-3, magnitudes=True)
    B1 = BC.step_bounds(R, BC.U_FP32, BC.U_FP32, BC.U_FP32)
    B2 = BC.step_bounds(R, BC.U_FP32 / 2, BC.U_FP32 / 2, BC.U_FP32 / 2)
    B0 = BC._step_bounds(R, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    # without reduced-precision rounding only the FP64 rounding of the inversions is left
    assert np.all(B0.P == 0)
    assert np.all(B0.Lstore <= 1e-11 * np.abs(R.TL @ R.D).max()) and np.all(B0.D <= 1e-11 * np.abs(R.D).max())
    assert np.allclose(B2.Lstore, B1.Lstore / 2, rtol=1e-3) and np.allclose(B2.P, B1.P / 2, rtol=1e-12)
    # relative to the values the bound is small: the check is not vacuous
    rel = B1.Lstore / np.maximum(np.abs(R.TL @ R.D), 1e-300)
    assert np.median(rel[np.abs(R.TL @ R.D) > 1e-8]) < 1e-4


def test_compare_block_bounded_detects_a_planted_error():
    """An FP32-rounded factor passes; one value moved by 20 times its bound fails."""
    A = W.convdiff_upwind((6, 6, 6), seed=4)
    bs = O.partition_fixed(A.n, 6)
    Fo = O.bilu_factor(A, bs, 1e-3)
    F = _export(Fo)
    Fo.free()
    F32 = dict(F, Lval=F["Lval"].astype(np.float32).astype(np.float64),
               Uval=F["Uval"].astype(np.float32).astype(np.float64))
    blocks = BC._blocks(F32)
    for K in (3, 17, 30):
        flips, worst, ncand = BC.compare_block_bounded(A, F32, K, 1e-3, BC.U_FP32, BC.U_FP32, BC.U_FP32, blocks=blocks)
        assert flips == 0 and worst <= 1.0
    K = 17
    R = BC.block_step(A, F32, K, 1e-3, blocks, magnitudes=True)
    Bd = BC.step_bounds(R, BC.U_FP32, BC.U_FP32, BC.U_FP32)
    lr = blocks[K][0]
    assert len(lr) > 0
    k = int(np.searchsorted(R.lcand, lr[0]))
    vp = int(np.sum(np.diff(F32["Lptr"])[:K] * np.diff(bs)[:K]))
    bad = F32["Lval"].copy()
    bad[vp] += 20 * Bd.Lstore[k, 0] + 1e-300
    Fb = dict(F32, Lval=bad)
    with pytest.raises(AssertionError):
        BC.compare_block_bounded(A, Fb, K, 1e-3, BC.U_FP32, BC.U_FP32, BC.U_FP32)
