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


def block_step(A, F: dict, K: int, tau: float, blocks=None) -> BlockResult:
    """Step K from A and the factor F's blocks J < K.  F holds numpy arrays bstart, Lptr,
    Lrow, Lval, Uptr, Ucol, Uval (the export layout of the library and the oracle)."""
    bs = np.asarray(F["bstart"], dtype=np.int64)
    s0, s1 = int(bs[K]), int(bs[K + 1])
    b = s1 - s0
    blocks = blocks if blocks is not None else _blocks(F)
    rp, ci, va = A.rowptr, A.colind, A.val
    # 1. load A: rows i >= s0 of the block column, columns j >= s1 of the block row
    TL, TU = {}, {}
    # block column of A via the rows that have entries in [s0, s1): scan CSR rows >= s0
    sel = np.nonzero((ci >= s0) & (ci < s1))[0]
    rows_of = np.searchsorted(rp, sel, side="right") - 1
    for e, i in zip(sel, rows_of):
        if i >= s0:
            TL.setdefault(int(i), np.zeros(b))[int(ci[e]) - s0] = va[e]
    for r in range(s0, s1):
        TL.setdefault(r, np.zeros(b))  # the pivot rows always exist
        for e in range(rp[r], rp[r + 1]):
            j = int(ci[e])
            if j >= s1:
                TU.setdefault(j, np.zeros(b))[r - s0] = va[e]
    # 2. updates from earlier blocks in increasing J
    for J in range(K):
        lr, L, uc, U = blocks[J]
        # L side: kept columns of U-breve_J inside B_K, kept rows of L_J at or after s0
        qs, qe = np.searchsorted(uc, s0), np.searchsorted(uc, s1)
        ps = np.searchsorted(lr, s0)
        if qe > qs and len(lr) > ps:
            upd = L[ps:] @ U[qs:qe].T
            for a, i in enumerate(lr[ps:]):
                t = TL.setdefault(int(i), np.zeros(b))
                t[uc[qs:qe] - s0] -= upd[a]
        # U side: kept rows of L_J inside B_K, kept columns of U-breve_J at or after s1
        ps2, pe2 = np.searchsorted(lr, s0), np.searchsorted(lr, s1)
        qs2 = np.searchsorted(uc, s1)
        if pe2 > ps2 and len(uc) > qs2:
            upd = L[ps2:pe2] @ U[qs2:].T  # rows r in B_K x columns j
            for a, j in enumerate(uc[qs2:]):
                t = TU.setdefault(int(j), np.zeros(b))
                t[lr[ps2:pe2] - s0] -= upd[:, a]
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
    return BlockResult(lcand[keepL], Lc[keepL], ucand[keepU], Uc[keepU], P, D, ln, lcand, un, ucand)


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
