"""One block step of the Crout BILU recomputed from a given factor's earlier blocks.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): used by the tests to check sampled
blocks of factorizations too large for the full oracle.

Step K of the block Crout factorization (Algorithm 1 with blocks, Sec. 2.2) reads only A and
the final values of blocks J < K.  Given those values (taken from the factor under test), this
module performs step K in plain FP64 numpy, in the paper's order:
  1. T_L = A[i, B_K] for rows i >= s_{K-1} with a stored entry, T_U = A[B_K, j] for j >= s_K;
  2. for every earlier J in increasing order: T_L[i, c] -= L_J[i, :] U-breve_J[:, c] over J's
     kept rows i >= s_{K-1} and kept columns c in B_K; T_U[r, j] -= L_J[r, :] U-breve_J[:, j]
     over J's kept rows r in B_K and kept columns j >= s_K;
  3. P_K = T_L[B_K, B_K], D_K = P_K^{-1} (partial-pivot LU, LAPACK);
  4. l_i = T_L[i, :] D_K for candidate rows i >= s_K, kept iff ||l_i||_2 > tau;
  5. u^_j = D_K T_U[:, j] for candidate columns, kept iff ||u^_j||_2 > tau; U-breve stores T_U.
The result is compared with the factor's own block K.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla


@dataclasses.dataclass
class BlockResult:
    Lrow: np.ndarray    # kept rows (sorted)
    Lval: np.ndarray    # len(Lrow) x b
    Ucol: np.ndarray
    Uval: np.ndarray    # len(Ucol) x b (columns of U-breve)
    P: np.ndarray       # b x b
    D: np.ndarray       # b x b
    lnorm: np.ndarray   # ||l_i|| of every candidate row (sorted by row)
    lcand: np.ndarray
    unorm: np.ndarray
    ucand: np.ndarray
    # with magnitudes=True: |A| + sum_J |L_J| |U-breve_J| per entry of the candidate rows
    # (same order as lcand), of the pivot rows, and of the candidate columns (ucand order); the
    # number of product terms that enter one entry at most (sum of b_J over the producers)
    SL: np.ndarray = None
    SP: np.ndarray = None
    SU: np.ndarray = None
    TL: np.ndarray = None   # T_L rows of the candidates (before scaling)
    TU: np.ndarray = None   # T_U columns of the candidates
    nterms: int = 0


def _blocks(F):
    """Per block: (kept rows, L values b_J-wide, kept cols, U-breve values)."""
    bs = np.asarray(F["bstart"], dtype=np.int64)
    nb = len(bs) - 1
    out = []
    lv = uv = 0
    for J in range(nb):
        bJ = int(bs[J + 1] - bs[J])
        lr = np.asarray(F["Lrow"][F["Lptr"][J]:F["Lptr"][J + 1]], dtype=np.int64)
        uc = np.asarray(F["Ucol"][F["Uptr"][J]:F["Uptr"][J + 1]], dtype=np.int64)
        L = np.asarray(F["Lval"][lv:lv + len(lr) * bJ]).reshape(len(lr), bJ)
        U = np.asarray(F["Uval"][uv:uv + len(uc) * bJ]).reshape(len(uc), bJ)
        lv += len(lr) * bJ
        uv += len(uc) * bJ
        out.append((lr, L, uc, U))
    return out


def block_step(A, F: dict, K: int, tau: float, blocks=None, magnitudes: bool = False) -> BlockResult:
    """Step K from A and the factor F's blocks J < K.  F holds numpy arrays bstart, Lptr,
    Lrow, Lval, Uptr, Ucol, Uval (the export layout of the library and the oracle).  With
    magnitudes=True the same loops also sum the magnitudes of every term (for error bounds)."""
    bs = np.asarray(F["bstart"], dtype=np.int64)
    s0, s1 = int(bs[K]), int(bs[K + 1])
    b = s1 - s0
    blocks = blocks if blocks is not None else _blocks(F)
    rp, ci, va = A.rowptr, A.colind, A.val
    # 1. load A: rows i >= s0 of the block column, columns j >= s1 of the block row
    TL, TU = {}, {}
    ML, MU = {}, {}  # magnitudes (magnitudes=True)
    nterms = 0
    # block column of A via the rows that have entries in [s0, s1): scan CSR rows >= s0
    sel = np.nonzero((ci >= s0) & (ci < s1))[0]
    rows_of = np.searchsorted(rp, sel, side="right") - 1
    for e, i in zip(sel, rows_of):
        if i >= s0:
            TL.setdefault(int(i), np.zeros(b))[int(ci[e]) - s0] = va[e]
            if magnitudes:
                ML.setdefault(int(i), np.zeros(b))[int(ci[e]) - s0] = abs(va[e])
    for r in range(s0, s1):
        TL.setdefault(r, np.zeros(b))  # the pivot rows always exist
        if magnitudes:
            ML.setdefault(r, np.zeros(b))
        for e in range(rp[r], rp[r + 1]):
            j = int(ci[e])
            if j >= s1:
                TU.setdefault(j, np.zeros(b))[r - s0] = va[e]
                if magnitudes:
                    MU.setdefault(j, np.zeros(b))[r - s0] = abs(va[e])
    # 2. updates from earlier blocks in increasing J
    for J in range(K):
        lr, L, uc, U = blocks[J]
        # L side: kept columns of U-breve_J inside B_K, kept rows of L_J at or after s0
        qs, qe = np.searchsorted(uc, s0), np.searchsorted(uc, s1)
        ps = np.searchsorted(lr, s0)
        hit = False
        if qe > qs and len(lr) > ps:
            hit = True
            upd = L[ps:] @ U[qs:qe].T
            mag = np.abs(L[ps:]) @ np.abs(U[qs:qe]).T if magnitudes else None
            for a, i in enumerate(lr[ps:]):
                t = TL.setdefault(int(i), np.zeros(b))
                t[uc[qs:qe] - s0] -= upd[a]
                if magnitudes:
                    ML.setdefault(int(i), np.zeros(b))[uc[qs:qe] - s0] += mag[a]
        # U side: kept rows of L_J inside B_K, kept columns of U-breve_J at or after s1
        ps2, pe2 = np.searchsorted(lr, s0), np.searchsorted(lr, s1)
        qs2 = np.searchsorted(uc, s1)
        if pe2 > ps2 and len(uc) > qs2:
            hit = True
            upd = L[ps2:pe2] @ U[qs2:].T  # rows r in B_K x columns j
            mag = np.abs(L[ps2:pe2]) @ np.abs(U[qs2:]).T if magnitudes else None
            for a, j in enumerate(uc[qs2:]):
                t = TU.setdefault(int(j), np.zeros(b))
                t[lr[ps2:pe2] - s0] -= upd[:, a]
                if magnitudes:
                    MU.setdefault(int(j), np.zeros(b))[lr[ps2:pe2] - s0] += mag[:, a]
        if hit:
            nterms += L.shape[1]
    # 3. pivot block and its inverse
    P = np.array([TL[r] for r in range(s0, s1)])
    D = sla.lu_solve(sla.lu_factor(P), np.eye(b))
    # 4./5. scaled candidates and the drop test
    lcand = np.array(sorted(i for i in TL if i >= s1), dtype=np.int64)
    ucand = np.array(sorted(TU), dtype=np.int64)
    Lc = np.array([TL[i] for i in lcand]).reshape(-1, b) @ D if len(lcand) else np.zeros((0, b))
    Uc = np.array([TU[j] for j in ucand]).reshape(-1, b) if len(ucand) else np.zeros((0, b))
    uh = (D @ Uc.T).T if len(ucand) else np.zeros((0, b))
    ln = np.sqrt(np.sum(Lc * Lc, axis=1))
    un = np.sqrt(np.sum(uh * uh, axis=1))
    keepL, keepU = ln > tau, un > tau
    R = BlockResult(lcand[keepL], Lc[keepL], ucand[keepU], Uc[keepU], P, D, ln, lcand, un, ucand)
    if magnitudes:
        R.SL = np.array([ML[i] for i in lcand]).reshape(-1, b)
        R.SP = np.array([ML[r] for r in range(s0, s1)])
        R.SU = np.array([MU.get(int(j), np.zeros(b)) for j in ucand]).reshape(-1, b)
        R.TL = np.array([TL[i] for i in lcand]).reshape(-1, b)
        R.TU = Uc
        R.nterms = nterms
    return R


# Unit roundoffs of the arithmetic and storage formats of the reduced-precision factor
# (a9): FP32 has a 24-bit significand (u = 2^-24), BF16 an 8-bit one (u = 2^-8).
U_FP32 = 2.0 ** -24
U_BF16 = 2.0 ** -8
U_FP64 = 2.0 ** -53
# Gradual underflow adds an absolute error of at most half the smallest subnormal to a rounded
# result: FP32 2^-150 (subnormals down to 2^-149), BF16 2^-134 (8-bit significand, the FP32
# exponent range: subnormals down to 2^-133), FP64 2^-1075.
ETA = {U_FP32: 2.0 ** -150, U_BF16: 2.0 ** -134, U_FP64: 2.0 ** -1075}


def gamma(n: int, u: float) -> float:
    """gamma_n = n u / (1 - n u): a sum of n rounded terms (any order) is off by at most
    gamma_n times the sum of their magnitudes (the standard forward error bound of floating-
    point summation and dot products)."""
    return n * u / (1.0 - n * u)


@dataclasses.dataclass
class StepBounds:
    L: np.ndarray       # per candidate row (lcand order) and column: bound of |l_i - l_i^exact|
    Lstore: np.ndarray  # the same, plus the rounding of the stored value
    U: np.ndarray       # per candidate column (ucand order): bound of the stored U-breve column
    P: np.ndarray       # bound of |P_K - P_K^exact|
    D: np.ndarray       # bound of |D_K - D_K^exact|, first order in the error of P_K
    lnorm: np.ndarray   # bound of | ||l_i|| - ||l_i^exact|| | (the drop test's window)
    unorm: np.ndarray   # bound of | ||u^_j|| - ||u^_j^exact|| |


def step_bounds(R: BlockResult, u_acc: float, u_scale: float, u_store: float) -> StepBounds:
    """(see below)"""
    return _step_bounds(R, u_acc, u_scale, u_store, ETA.get(u_acc, 0.0), ETA.get(u_scale, 0.0),
                        ETA.get(u_store, 0.0))


def _step_bounds(R: BlockResult, u_acc: float, u_scale: float, u_store: float, eta_acc: float, eta_scale: float,
                 eta_store: float) -> StepBounds:
    """First-order componentwise bounds of the error of one block step computed with reduced
    precision, against the same step in exact arithmetic on the same inputs (A and the earlier
    blocks' stored values), for a step that (a) accumulates every entry of T_L / T_U -- A's
    value and the products of the producers, at most nterms of them, plus the 3 additions of
    the pivot rows' partial sums -- with unit roundoff u_acc, (b) inverts P_K (= the pivot rows
    of T_L) in FP64, (c) forms l_i = T_L[i,:] D_K and u^_j = D_K T_U[:,j] from D_K rounded to
    u_scale with sums of b_K terms rounded to u_scale, and (d) stores l_i and U-breve columns
    rounded to u_store.  With S = |A| + sum |L_J| |U-breve_J| (the magnitudes, from the step):
      |dT| <= gamma_m S,  m = nterms + 4                      (summation bound)
      |dD| <= |D| (|dP| + 2 gamma_4b(u_FP64) Pi |L^||U^|) |D|  (dD = -D dP D + O(dP^2), and
              the FP64 rounding of both inversions: the backward error of an inverse through
              the LU factors P = Pi L^ U^ is within gamma_3b |L^||U^|)
      |dl_i| <= |dT_i| |D| + |T_i| |dD| + (u_scale + gamma_b(u_scale)) |T_i| |D|
      stored: + u_store |l_i|;  U-breve_j: gamma_m S_j + u_store |T_U[:,j]|
      | ||l_i|| - ||l_i^exact|| | <= || bound of dl_i ||_2 (the triangle inequality),
    each with the absolute underflow terms of its format (ETA): m eta_acc per accumulated entry,
    eta_scale (sum_k |T_ik| + b) per scaled entry (D_K rounded, b products and sums), eta_store
    per stored value."""
    b = R.P.shape[0]
    m = R.nterms + 4
    gm = gamma(m, u_acc)
    gb = gamma(b, u_scale) + u_scale
    aD = np.abs(R.D)
    dP = gm * R.SP + m * eta_acc
    Pm, Lf, Uf = sla.lu(R.P)
    dD = aD @ (dP + 2.0 * gamma(4 * b, U_FP64) * (Pm @ (np.abs(Lf) @ np.abs(Uf)))) @ aD
    if len(R.lcand):
        aT = np.abs(R.TL)
        dl = (gm * R.SL + m * eta_acc) @ aD + aT @ dD + gb * (aT @ aD)
        dl += eta_scale * (aT.sum(axis=1, keepdims=True) + b)
    else:
        dl = np.zeros((0, b))
    if len(R.ucand):
        aU = np.abs(R.TU)
        dU = gm * R.SU + m * eta_acc
        du = (aD @ dU.T + dD @ aU.T + gb * (aD @ aU.T)).T
        du += eta_scale * (aU.sum(axis=1, keepdims=True) + b)
    else:
        dU = du = np.zeros((0, b))
    Lc = R.TL @ R.D if len(R.lcand) else np.zeros((0, b))
    return StepBounds(L=dl, Lstore=dl + u_store * np.abs(Lc) + eta_store,
                      U=dU + u_store * np.abs(R.TU) + eta_store if len(R.ucand) else dU,
                      P=dP, D=dD, lnorm=np.sqrt(np.sum(dl * dl, axis=1)), unorm=np.sqrt(np.sum(du * du, axis=1)))


def compare_block_bounded(A, F: dict, K: int, tau: float, u_acc: float, u_scale: float, u_store: float,
                          blocks=None, safety: float = 2.0):
    """Block K of a reduced-precision factor F against the exact step from F's own earlier
    blocks, within safety x the bounds of step_bounds (an AssertionError otherwise): values of
    the kept rows / columns present on both sides, P_K and D_K elementwise; a drop decision may differ only where the exact norm lies
    within safety x its bound of tau.  Returns (flips, worst error / bound ratio, candidates)."""
    blocks = blocks if blocks is not None else _blocks(F)
    R = block_step(A, F, K, tau, blocks, magnitudes=True)
    Bd = step_bounds(R, u_acc, u_scale, u_store)
    lr, L, uc, U = blocks[K]
    flips, worst = 0, 0.0
    for got, want, cand, nrm, win in ((lr, R.Lrow, R.lcand, R.lnorm, Bd.lnorm), (uc, R.Ucol, R.ucand, R.unorm, Bd.unorm)):
        for idx in np.setxor1d(got, want):
            k = np.searchsorted(cand, idx)
            assert k < len(cand) and cand[k] == idx, f"block {K}: index {idx} is not a candidate"
            assert abs(nrm[k] - tau) <= safety * win[k] + 1e-15 * tau, \
                f"block {K}: drop decision of {idx} differs, norm {nrm[k]:.6e}, window {safety * win[k]:.3e}"
            flips += 1
    for got_idx, got_val, want_idx, want_val, bound, cand in ((lr, L, R.Lrow, R.Lval, Bd.Lstore, R.lcand),
                                                              (uc, U, R.Ucol, R.Uval, Bd.U, R.ucand)):
        common, ia, ib = np.intersect1d(got_idx, want_idx, return_indices=True)
        if len(common):
            bnd = bound[np.searchsorted(cand, common)]
            err = np.abs(got_val[ia] - want_val[ib])
            ratio = err / np.maximum(safety * bnd, 1e-300)
            worst = max(worst, float(ratio.max()))
            assert np.all(err <= safety * bnd), f"block {K}: value error {float(err.max()):.3e} exceeds its bound"
    bs = np.asarray(F["bstart"], dtype=np.int64)
    b = int(bs[K + 1] - bs[K])
    dp = int(np.sum(np.diff(bs[:K + 1]) ** 2))
    Dg = np.asarray(F["Dinv"][dp:dp + b * b]).reshape(b, b)
    Pg = np.asarray(F["Pblk"][dp:dp + b * b]).reshape(b, b)
    for got, want, bound in ((Pg, R.P, safety * Bd.P), (Dg, R.D, safety * Bd.D)):
        err = np.abs(got - want)
        worst = max(worst, float((err / np.maximum(bound, 1e-300)).max()))
        assert np.all(err <= bound), f"block {K}: P / D error {float(err.max()):.3e} exceeds its bound"
    return flips, worst, len(R.lcand) + len(R.ucand)


def compare_block(A, F: dict, K: int, tau: float, rtol: float = 1e-10, blocks=None, flip_rtol: float = 1e-12):
    """Recompute block K and compare with F's block K.  Returns (flips, max_rel_err): flips =
    candidates whose drop decision differs, allowed only within flip_rtol relative of tau (an
    AssertionError is raised otherwise, or when a value differs by more than rtol)."""
    blocks = blocks if blocks is not None else _blocks(F)
    R = block_step(A, F, K, tau, blocks)
    lr, L, uc, U = blocks[K]
    flips = 0
    for got, want, cand, nrm in ((lr, R.Lrow, R.lcand, R.lnorm), (uc, R.Ucol, R.ucand, R.unorm)):
        diff = np.setxor1d(got, want)
        for idx in diff:
            k = np.searchsorted(cand, idx)
            assert k < len(cand) and cand[k] == idx, f"block {K}: index {idx} is not a candidate"
            assert abs(nrm[k] - tau) <= flip_rtol * tau, f"block {K}: drop decision of {idx} differs, norm {nrm[k]}"
            flips += 1
    err = 0.0
    for got_idx, got_val, want_idx, want_val in ((lr, L, R.Lrow, R.Lval), (uc, U, R.Ucol, R.Uval)):
        common, ia, ib = np.intersect1d(got_idx, want_idx, return_indices=True)
        if len(common):
            g, w = got_val[ia], want_val[ib]
            scale = np.maximum(np.abs(w).max(axis=1, keepdims=True), 1e-300)
            err = max(err, float(np.max(np.abs(g - w) / scale)))
    bs = np.asarray(F["bstart"], dtype=np.int64)
    b = int(bs[K + 1] - bs[K])
    dp = int(np.sum(np.diff(bs[:K + 1]) ** 2))
    Dg = np.asarray(F["Dinv"][dp:dp + b * b]).reshape(b, b)
    Pg = np.asarray(F["Pblk"][dp:dp + b * b]).reshape(b, b)
    err = max(err, float(np.max(np.abs(Pg - R.P)) / max(np.abs(R.P).max(), 1e-300)))
    err = max(err, float(np.max(np.abs(Dg - R.D)) / max(np.abs(R.D).max(), 1e-300)))
    assert err <= rtol, f"block {K}: relative error {err:.3e} > {rtol:g}"
    return flips, err
