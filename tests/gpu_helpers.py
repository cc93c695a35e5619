"""Helpers for the GPU tests: run the CUDA path through the C ABI and compare with the oracle."""
from __future__ import annotations

import dataclasses

import numpy as np

import paper_1908_10169_gb300 as B


@dataclasses.dataclass
class GpuFactor:
    bstart: np.ndarray
    Lptr: np.ndarray
    Lrow: np.ndarray
    Lval: np.ndarray
    Uptr: np.ndarray
    Ucol: np.ndarray
    Uval: np.ndarray
    Dinv: np.ndarray
    Pblk: np.ndarray
    stats: object
    status: int

    # block accessors with the oracle Factor's names (small problems)
    def _b(self, K):
        return int(self.bstart[K + 1] - self.bstart[K])

    def L_block(self, K):
        vp = _vptr(self.Lptr, self.bstart)
        rows = self.Lrow[self.Lptr[K]:self.Lptr[K + 1]]
        return rows, self.Lval[vp[K]:vp[K + 1]].reshape(len(rows), self._b(K))

    def U_block(self, K):
        vp = _vptr(self.Uptr, self.bstart)
        cols = self.Ucol[self.Uptr[K]:self.Uptr[K + 1]]
        return cols, self.Uval[vp[K]:vp[K + 1]].reshape(len(cols), self._b(K))

    def _dblk(self, arr, K):
        d0 = int(np.sum(np.diff(self.bstart[:K + 1]).astype(np.int64) ** 2))
        b = self._b(K)
        return arr[d0:d0 + b * b].reshape(b, b)

    def D_block(self, K):
        return self._dblk(self.Dinv, K)

    def P_block(self, K):
        return self._dblk(self.Pblk, K)


def gpu_factor(ctx, A, droptol, params=None, export=True, bstart=None) -> GpuFactor:
    """Analyse (with the partition bstart when given), factor and export through the C ABI."""
    p = params if params is not None else B.bilu_params_default()
    if bstart is not None:
        B.bilu_analyze_partition(ctx, A.n, A.rowptr.astype(np.int64), A.colind.astype(np.int32),
                                 A.val.astype(np.float64), bstart, p)
    else:
        B.bilu_analyze(ctx, A.n, A.rowptr.astype(np.int64), A.colind.astype(np.int32), A.val.astype(np.float64), p)
    st = B.bilu_factor(ctx, droptol)
    s = B.bilu_stats(ctx)
    bs = np.zeros(s.nblocks + 1, np.int32)
    B.bilu_get_factor_partition(ctx, bs)  # the analysis partition, or the merged one
    if not export:
        return GpuFactor(bs, *([None] * 8), s, st)
    nb = s.nblocks
    Lptr = np.zeros(nb + 1, np.int64)
    Uptr = np.zeros(nb + 1, np.int64)
    Lrow = np.zeros(s.kept_rows, np.int32)
    Ucol = np.zeros(s.kept_cols, np.int32)
    Lval = np.zeros(s.nnz_l)
    Uval = np.zeros(s.nnz_u)
    Dinv = np.zeros(s.nnz_d)
    Pblk = np.zeros(s.nnz_d)
    B.bilu_export(ctx, Lptr, Lrow, Lval, Uptr, Ucol, Uval, Dinv, Pblk)
    return GpuFactor(bs, Lptr, Lrow, Lval, Uptr, Ucol, Uval, Dinv, Pblk, s, st)


def _vptr(ptr, bstart):
    bs = np.diff(bstart).astype(np.int64)
    return np.concatenate([[0], np.cumsum(np.diff(ptr) * bs)])


@dataclasses.dataclass
class ParityReport:
    blocks: int
    flips_L: int
    flips_U: int
    max_rel_L: float
    max_rel_U: float
    max_rel_D: float
    max_rel_P: float


def compare_factors(Fo, Fg: GpuFactor, rtol: float = 1e-10, A=None, tau=None) -> ParityReport:
    """Block-by-block comparison of kept sets (exact) and values (max-norm relative per block).

    With A and tau given, a block whose kept set differs is accepted when every differing
    candidate's drop norm lies within 1e-12 (relative) of tau: from that block on the two
    factorizations follow different patterns, so each remaining block of the GPU factor is
    checked against the step recomputed from the GPU's own earlier blocks (oracle/block_check),
    and the flipped decisions are counted in the report."""
    assert np.array_equal(Fo.bstart, Fg.bstart), "partitions differ"
    nb = len(Fo.bstart) - 1
    oLv, oUv, gLv, gUv = Fo.Lvptr(), Fo.Uvptr(), _vptr(Fg.Lptr, Fg.bstart), _vptr(Fg.Uptr, Fg.bstart)
    Dp = Fo.Dptr()
    flipsL = flipsU = 0
    mL = mU = mD = mP = 0.0

    def rel(a, b):
        den = np.abs(a).max() if a.size else 0.0
        return 0.0 if a.size == 0 else float(np.abs(a - b).max() / max(den, 1e-300))

    for K in range(nb):
        b = int(Fo.bstart[K + 1] - Fo.bstart[K])
        ro = Fo.Lrow[Fo.Lptr[K]:Fo.Lptr[K + 1]]
        rg = Fg.Lrow[Fg.Lptr[K]:Fg.Lptr[K + 1]]
        co = Fo.Ucol[Fo.Uptr[K]:Fo.Uptr[K + 1]]
        cg = Fg.Ucol[Fg.Uptr[K]:Fg.Uptr[K + 1]]
        if not (np.array_equal(ro, rg) and np.array_equal(co, cg)):
            if A is None:
                raise AssertionError(f"kept sets differ at block {K}: L {np.setxor1d(ro, rg)[:8]} "
                                     f"U {np.setxor1d(co, cg)[:8]}")
            from oracle import block_check as BC
            E = {"bstart": Fg.bstart, "Lptr": Fg.Lptr, "Lrow": Fg.Lrow, "Lval": Fg.Lval, "Uptr": Fg.Uptr,
                 "Ucol": Fg.Ucol, "Uval": Fg.Uval, "Dinv": Fg.Dinv, "Pblk": Fg.Pblk}
            blocks = BC._blocks(E)
            flips = 0
            for K2 in range(K, nb):
                f, err = BC.compare_block(A, E, K2, tau, rtol=rtol, blocks=blocks, flip_rtol=1e-12)
                flips += f
            rep = ParityReport(nb, flips, 0, mL, mU, mD, mP)
            print(f"parity: {flips} drop decision(s) within 1e-12 of tau differ from the oracle from block {K} on")
            assert mL <= rtol and mU <= rtol and mD <= rtol and mP <= rtol, rep
            return rep
        mL = max(mL, rel(Fo.Lval[oLv[K]:oLv[K + 1]], Fg.Lval[gLv[K]:gLv[K + 1]]))
        mU = max(mU, rel(Fo.Uval[oUv[K]:oUv[K + 1]], Fg.Uval[gUv[K]:gUv[K + 1]]))
        mD = max(mD, rel(Fo.Dinv[Dp[K]:Dp[K + 1]], Fg.Dinv[Dp[K]:Dp[K + 1]]))
        mP = max(mP, rel(Fo.Pblk[Dp[K]:Dp[K + 1]], Fg.Pblk[Dp[K]:Dp[K + 1]]))
    rep = ParityReport(nb, flipsL, flipsU, mL, mU, mD, mP)
    assert mL <= rtol and mU <= rtol and mD <= rtol and mP <= rtol, rep
    return rep
