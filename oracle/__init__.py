"""Python access to the FP64 CPU oracle (plain C, ``bilu_oracle.c``).

TEST INFRASTRUCTURE ONLY: the slow, obviously correct reference the CUDA path is
checked against.  Only the test suite, the smoke check and the benchmark's CPU
baseline may import this package.  It never imports the product package and the
product never imports it.

Paper: Bollhoefer, Schenk, Verbosio, "High Performance Block Incomplete LU
Factorization", arXiv:1908.10169 (Algorithm 1, Sec. 2.2, Sec. 3.4, Sec. 3.6, Sec. 4).

The other modules of this package are plain Python / numpy references of the remaining
parts: ``mwm_oracle`` (matching + scaling, Sec. 3.1), ``cosine_oracle`` (cosine blocking,
Sec. 3.2), ``nd_oracle`` (block nested dissection and elimination tree, Sec. 3.3),
``block_check`` (one block step of Sec. 2.2 from a given factor) and ``skip_oracle`` (the
learned skip's features and classifier).
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bilu_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

C_NAMES = ["flop_upd_L", "flop_upd_U", "flop_getrf", "flop_inv", "flop_scale", "flop_norm",
           "cand_rows", "cand_cols", "panel_read_bytes", "npairs_L", "npairs_U", "nperturb"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no vectorisation flags beyond -O2)."""
    hdr = os.path.join(_HERE, "bilu_oracle.h")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(hdr)):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(build())
        P = ct.c_void_p
        i64, i32, f64 = ct.c_int64, ct.c_int32, ct.c_double
        L.orc_partition_fixed.argtypes = [i64, i32, P]
        L.orc_partition_fixed.restype = i32
        L.orc_partition_ilu1t.argtypes = [i64, P, P, P, f64, i32, P]
        L.orc_partition_ilu1t.restype = i32
        L.orc_partition_ilu1t_groups.argtypes = [i64, P, P, P, f64, i32, i32, P, P]
        L.orc_partition_ilu1t_groups.restype = i32
        L.orc_bilu_factor.argtypes = [i64, P, P, P, i32, P, f64, i32, f64, f64, ct.POINTER(P)]
        L.orc_bilu_factor.restype = i32
        L.orc_bilu_factor_agg.argtypes = [i64, P, P, P, i32, P, f64, i32, f64, f64, i32, ct.POINTER(P)]
        L.orc_bilu_factor_agg.restype = i32
        L.orc_agg_rule.argtypes = [i64] * 10
        L.orc_agg_rule.restype = i32
        L.orc_factor_bstart.argtypes = [P, P]
        L.orc_factor_sizes.argtypes = [P, P]
        L.orc_factor_export.argtypes = [P] * 11
        L.orc_factor_counters.argtypes = [P, P]
        L.orc_factor_free.argtypes = [P]
        L.orc_bilu_apply.argtypes = [P, P, P]
        L.orc_spmv.argtypes = [i64, P, P, P, P, P]
        L.orc_gmres.argtypes = [i64, P, P, P, P, P, P, f64, i32, i32, ct.POINTER(i32),
                                ct.POINTER(f64), P]
        L.orc_gmres.restype = i32
        L.orc_bildl_factor.argtypes = [i64, P, P, P, i32, P, f64, i32, f64, f64, ct.POINTER(P)]
        L.orc_bildl_factor.restype = i32
        L.orc_sqmr.argtypes = [i64, P, P, P, P, P, P, f64, i32, ct.POINTER(i32), ct.POINTER(f64), P]
        L.orc_sqmr.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _csr_args(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, va


def partition_fixed(n: int, b: int) -> np.ndarray:
    out = np.zeros(n // b + 2, dtype=np.int32)
    nb = lib().orc_partition_fixed(n, b, _p(out))
    return out[: nb + 1].copy()


def partition_ilu1t(A, tau: float, max_block: int) -> np.ndarray:
    rp, ci, va = _csr_args(A)
    out = np.zeros(A.n + 1, dtype=np.int32)
    nb = lib().orc_partition_ilu1t(A.n, _p(rp), _p(ci), _p(va), tau, max_block, _p(out))
    if nb < 0:
        raise ValueError("orc_partition_ilu1t failed")
    return out[: nb + 1].copy()


def partition_ilu1t_groups(A, tau: float, max_block: int, gstart) -> np.ndarray:
    """Sec. 3.4 growth rule with whole groups of columns (e.g. cosine blocks) as the unit."""
    rp, ci, va = _csr_args(A)
    gs = np.ascontiguousarray(gstart, dtype=np.int32)
    out = np.zeros(A.n + 1, dtype=np.int32)
    nb = lib().orc_partition_ilu1t_groups(A.n, _p(rp), _p(ci), _p(va), tau, max_block, len(gs) - 1, _p(gs),
                                          _p(out))
    if nb < 0:
        raise ValueError("orc_partition_ilu1t_groups failed")
    return out[: nb + 1].copy()


@dataclasses.dataclass
class Factor:
    """The oracle's factor, exported into plain arrays (layout in bilu_oracle.h)."""
    bstart: np.ndarray
    Lptr: np.ndarray
    Lrow: np.ndarray
    Lval: np.ndarray
    Uptr: np.ndarray
    Ucol: np.ndarray
    Uval: np.ndarray
    Dinv: np.ndarray
    Pblk: np.ndarray
    LUblk: np.ndarray
    piv: np.ndarray
    counters: dict
    status: int
    handle: object = None
    merges: int = 0  # progressive aggregation: blocks merged into their successor (void blocks)

    @property
    def nb(self) -> int:
        return len(self.bstart) - 1

    def bsize(self, K: int) -> int:
        return int(self.bstart[K + 1] - self.bstart[K])

    def Lvptr(self) -> np.ndarray:
        bs = np.diff(self.bstart).astype(np.int64)
        return np.concatenate([[0], np.cumsum(np.diff(self.Lptr) * bs)])

    def Uvptr(self) -> np.ndarray:
        bs = np.diff(self.bstart).astype(np.int64)
        return np.concatenate([[0], np.cumsum(np.diff(self.Uptr) * bs)])

    def Dptr(self) -> np.ndarray:
        bs = np.diff(self.bstart).astype(np.int64)
        return np.concatenate([[0], np.cumsum(bs * bs)])

    def L_block(self, K):
        b = self.bsize(K)
        rows = self.Lrow[self.Lptr[K]:self.Lptr[K + 1]]
        v = self.Lval[self.Lvptr()[K]:self.Lvptr()[K + 1]].reshape(len(rows), b)
        return rows, v

    def U_block(self, K):
        b = self.bsize(K)
        cols = self.Ucol[self.Uptr[K]:self.Uptr[K + 1]]
        v = self.Uval[self.Uvptr()[K]:self.Uvptr()[K + 1]].reshape(len(cols), b)
        return cols, v

    def D_block(self, K):
        b = self.bsize(K)
        d = self.Dptr()
        return self.Dinv[d[K]:d[K + 1]].reshape(b, b)

    def P_block(self, K):
        b = self.bsize(K)
        d = self.Dptr()
        return self.Pblk[d[K]:d[K + 1]].reshape(b, b)

    def LU_block(self, K):
        b = self.bsize(K)
        d = self.Dptr()
        return self.LUblk[d[K]:d[K + 1]].reshape(b, b), self.piv[self.bstart[K]:self.bstart[K + 1]]

    def nnz_L(self) -> int:
        return int(self.Lval.size)

    def nnz_U(self) -> int:
        return int(self.Uval.size)

    def dense_L(self) -> np.ndarray:
        """Unit block lower triangular L (dense; small problems only)."""
        n = int(self.bstart[-1])
        Ld = np.eye(n)
        for K in range(self.nb):
            rows, v = self.L_block(K)
            s0, s1 = self.bstart[K], self.bstart[K + 1]
            Ld[rows, s0:s1] = v
        return Ld

    def dense_Ubreve(self) -> np.ndarray:
        """Block upper U-breve: P_K on the diagonal, kept columns to the right."""
        n = int(self.bstart[-1])
        Ud = np.zeros((n, n))
        for K in range(self.nb):
            s0, s1 = self.bstart[K], self.bstart[K + 1]
            Ud[s0:s1, s0:s1] = self.P_block(K)
            cols, v = self.U_block(K)
            Ud[s0:s1, cols] = v.T
        return Ud

    def free(self):
        if self.handle is not None:
            lib().orc_factor_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def bilu_factor(A, bstart: np.ndarray, droptol: float, perturb: bool = True,
                pert_tau: float = 1e-2, pert_rho: float = 1e-1, keep_handle: bool = True,
                agg_max: int = 0) -> Factor:
    """Crout BILU (Sec. 2.2), with progressive aggregation of blocks up to agg_max columns
    when agg_max > 0 (Sec. 3.5; the factor's bstart then has void blocks).  Raises on
    argument errors and singular blocks."""
    return _factor(A, bstart, droptol, perturb, pert_tau, pert_rho, keep_handle, agg_max, False)


def bildl_factor(A, bstart: np.ndarray, droptol: float, perturb: bool = True,
                 pert_tau: float = 1e-2, pert_rho: float = 1e-1, keep_handle: bool = True) -> Factor:
    """BILDL, the incomplete block L D L^T of a symmetric A (Sec. 4.2), in the BILU layout:
    column i of U-breve is the unnormalised row of L's row i.  Raises ValueError when A is
    not symmetric."""
    return _factor(A, bstart, droptol, perturb, pert_tau, pert_rho, keep_handle, 0, True)


def _factor(A, bstart, droptol, perturb, pert_tau, pert_rho, keep_handle, agg_max, sym) -> Factor:
    L = lib()
    rp, ci, va = _csr_args(A)
    bs = np.ascontiguousarray(bstart, dtype=np.int32)
    h = ct.c_void_p()
    if sym:
        st = L.orc_bildl_factor(A.n, _p(rp), _p(ci), _p(va), len(bs) - 1, _p(bs), droptol,
                                int(perturb), pert_tau, pert_rho, ct.byref(h))
        if st == -1:
            raise ValueError("BILDL needs a symmetric matrix and a valid partition")
    else:
        st = L.orc_bilu_factor_agg(A.n, _p(rp), _p(ci), _p(va), len(bs) - 1, _p(bs), droptol,
                                   int(perturb), pert_tau, pert_rho, int(agg_max), ct.byref(h))
    if st < 0:
        raise RuntimeError(f"oracle factor failed with status {st}")
    sizes = np.zeros(8, dtype=np.int64)
    L.orc_factor_sizes(h, _p(sizes))
    nb = len(bs) - 1
    bs = np.zeros(nb + 1, np.int32)
    L.orc_factor_bstart(h, _p(bs))
    Lptr = np.zeros(nb + 1, np.int64)
    Uptr = np.zeros(nb + 1, np.int64)
    Lrow = np.zeros(sizes[0], np.int32)
    Ucol = np.zeros(sizes[1], np.int32)
    Lval = np.zeros(sizes[2])
    Uval = np.zeros(sizes[3])
    Dinv = np.zeros(sizes[4])
    Pblk = np.zeros(sizes[4])
    LUblk = np.zeros(sizes[4])
    piv = np.zeros(A.n, np.int32)
    L.orc_factor_export(h, _p(Lptr), _p(Lrow), _p(Lval), _p(Uptr), _p(Ucol), _p(Uval),
                        _p(Dinv), _p(Pblk), _p(LUblk), _p(piv))
    c = np.zeros(16)
    L.orc_factor_counters(h, _p(c))
    counters = {k: float(c[i]) for i, k in enumerate(C_NAMES)}
    F = Factor(bs.copy(), Lptr, Lrow, Lval, Uptr, Ucol, Uval, Dinv, Pblk, LUblk, piv, counters, st,
               h if keep_handle else None, int(sizes[7]))
    if not keep_handle:
        L.orc_factor_free(h)
    return F


def agg_rule(p, q, r, s, rp, sp, t, tp, u, v) -> bool:
    """The Sec. 3.5 merge test on the counts it names (see bilu_oracle.c)."""
    return bool(lib().orc_agg_rule(p, q, r, s, rp, sp, t, tp, u, v))


def bilu_apply(F: Factor, r: np.ndarray) -> np.ndarray:
    """z = M^{-1} r, M = L D^{-1} U (block forward / backward substitution)."""
    assert F.handle is not None
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.zeros_like(r)
    lib().orc_bilu_apply(F.handle, _p(r), _p(z))
    return z


def spmv(A, x: np.ndarray) -> np.ndarray:
    rp, ci, va = _csr_args(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.n)
    lib().orc_spmv(A.n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    relres: float
    status: int
    hist: np.ndarray


def gmres(A, F: Factor | None, b: np.ndarray, tol: float = 1e-8, restart: int = 30,
          maxit: int = 10000, x0: np.ndarray | None = None) -> GmresResult:
    """Right-preconditioned restarted GMRES(restart), MGS + Givens (Sec. 4 setup)."""
    rp, ci, va = _csr_args(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
    it = ct.c_int32()
    rr = ct.c_double()
    hist = np.zeros(maxit + 1)
    st = lib().orc_gmres(A.n, _p(rp), _p(ci), _p(va), None if F is None else F.handle, _p(b),
                         _p(x), tol, restart, maxit, ct.byref(it), ct.byref(rr), _p(hist))
    return GmresResult(x, it.value, rr.value, st, hist[: it.value + 1].copy())


@dataclasses.dataclass
class SqmrResult:
    x: np.ndarray
    iters: int
    berr: float
    status: int
    hist: np.ndarray


def sqmr(A, F: Factor | None, b: np.ndarray, tol: float = 1e-6, maxit: int = 10000,
         x0: np.ndarray | None = None) -> SqmrResult:
    """Simplified QMR with the symmetric preconditioner F (None: none), stopped on the
    normwise backward error (Sec. 4.2).  status: 0 converged, 1 maxit, 3 breakdown."""
    rp, ci, va = _csr_args(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
    it = ct.c_int32()
    be = ct.c_double()
    hist = np.zeros(maxit + 1)
    st = lib().orc_sqmr(A.n, _p(rp), _p(ci), _p(va), None if F is None else F.handle, _p(b),
                        _p(x), tol, maxit, ct.byref(it), ct.byref(be), _p(hist))
    return SqmrResult(x, it.value, be.value, st, hist[: it.value + 1].copy())
