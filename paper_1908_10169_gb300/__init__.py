"""Python binding of the GB300 block incomplete LU library (libbilu.so).

Thin ctypes marshalling of the C ABI declared in include/bilu.h: the functions keep the
C names and take numpy arrays or torch tensors (host or CUDA) for the pointer arguments.
Every numerical step runs in the library's CUDA kernels; there is no CPU fallback, and
loading fails loudly when the compiled library is missing (run ``build.build()``).

Method: Bollhoefer, Schenk, Verbosio, "High Performance Block Incomplete LU
Factorization", arXiv:1908.10169 (Crout-type BILU, Sec. 2.2; GMRES(30), Sec. 4).
"""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbilu.so")

BILU_OK, BILU_NOT_CONVERGED, BILU_PERTURBED = 0, 1, 2
BILU_ERR_ARG, BILU_ERR_OOM, BILU_ERR_CUDA, BILU_ERR_SINGULAR, BILU_ERR_TIMEOUT, BILU_ERR_STATE = -1, -2, -3, -4, -5, -6
BILU_BLOCKING_FIXED, BILU_BLOCKING_ILU1T = 0, 1
BILU_PREC_FP64, BILU_PREC_FP32, BILU_PREC_BF16 = 0, 1, 2
BILU_SKIP_NONE, BILU_SKIP_BOUND, BILU_SKIP_LEARNED = 0, 1, 2
BILU_SCHED_CHAIN, BILU_SCHED_TREE = 0, 1
(BILU_DEBUG_EXTRA_CTA, BILU_DEBUG_SPIN_LIMIT, BILU_DEBUG_SELFTEST_RECIP, BILU_DEBUG_BATCH_GROUP,
 BILU_DEBUG_SMALL_POOLS, BILU_DEBUG_POISON, BILU_DEBUG_NO_TRUNK, BILU_DEBUG_TRACE,
 BILU_DEBUG_BATCH_TRCAP, BILU_DEBUG_NO_TENSOR) = 1, 2, 3, 4, 5, 6, 7, 8, 9, 10
BILU_MAX_BLOCK = 64

# every extern "C" symbol that include/bilu.h declares
EXPORTED = ["bilu_params_default", "bilu_create", "bilu_analyze", "bilu_factor", "bilu_apply",
            "gmres_solve", "sqmr_solve", "bilu_stats", "bilu_get_partition", "bilu_get_factor_partition", "bilu_export",
            "bilu_last_error",
            "bilu_debug_set", "bilu_apply_noalloc", "bilu_factor_batch", "gmres_solve_batch",
            "bilu_record_samples", "bilu_get_samples", "bilu_mlp_train", "bilu_mlp_forward", "bilu_mlp_grad",
            "bilu_set_skip_model", "bilu_cosine_blocking", "bilu_partition_ilu1t", "bilu_mwm", "bilu_sym_mwm", "bilu_cosine_blocking_units", "bilu_scale_permute_csr",
            "bilu_nd_order", "bilu_block_etree",
            "bilu_permute_csr",
            "bilu_analyze_partition",
            "bilu_destroy"]

# learned skip classifier (layout of the model array: mean[F] std[F] W1[64][F] b1[64] W2[64][64]
# b2[64] w3[64] b3)
BILU_MLP_FEATURES = 12
BILU_MLP_HIDDEN = 64
BILU_MLP_PARAMS = 2 * 12 + 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1


class bilu_params(ct.Structure):
    _fields_ = [("blocking", ct.c_int32), ("max_block", ct.c_int32), ("fixed_block", ct.c_int32),
                ("tau_analyze", ct.c_double), ("perturb", ct.c_int32), ("pert_tau", ct.c_double),
                ("pert_rho", ct.c_double), ("precision", ct.c_int32), ("skip", ct.c_int32),
                ("schedule", ct.c_int32), ("group_ctas", ct.c_int32), ("aggregate_max", ct.c_int32),
                ("symmetric", ct.c_int32)]


class sqmr_info(ct.Structure):
    _fields_ = [("iters", ct.c_int32), ("breakdown", ct.c_int32), ("backward_error", ct.c_double),
                ("relres_true", ct.c_double), ("t_solve_ms", ct.c_double)]


class gmres_info(ct.Structure):
    _fields_ = [("iters", ct.c_int32), ("restarts", ct.c_int32), ("relres_true", ct.c_double),
                ("relres_est", ct.c_double), ("t_solve_ms", ct.c_double)]


class bilu_stats_t(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("nnz_a", ct.c_int64), ("nblocks", ct.c_int32), ("max_bsize", ct.c_int32),
                ("avg_bsize", ct.c_double), ("std_bsize", ct.c_double), ("nnz_l", ct.c_int64),
                ("nnz_u", ct.c_int64), ("nnz_d", ct.c_int64), ("kept_rows", ct.c_int64),
                ("kept_cols", ct.c_int64), ("cand_rows", ct.c_int64), ("cand_cols", ct.c_int64),
                ("nperturb", ct.c_int64), ("flops_factor", ct.c_double), ("flop_upd_l", ct.c_int64),
                ("flop_upd_u", ct.c_int64), ("flop_scale", ct.c_int64), ("flop_norm", ct.c_int64),
                ("t_analyze_ms", ct.c_double),
                ("t_factor_ms", ct.c_double), ("pool_retries", ct.c_int32),
                ("kernel_launches", ct.c_int64), ("phase_ms", ct.c_double * 8),
                ("skipped_rows", ct.c_int64), ("skipped_cols", ct.c_int64), ("schedule", ct.c_int32),
                ("tree_height", ct.c_int32), ("tree_trunk", ct.c_int32), ("group_ctas", ct.c_int32),
                ("idle_ms", ct.c_double), ("bound_drops", ct.c_int64), ("agg_merges", ct.c_int32),
                ("agg_max_bsize", ct.c_int32), ("t_aggregate_ms", ct.c_double)]


class bilu_mlp_train_cfg(ct.Structure):
    _fields_ = [("epochs", ct.c_int32), ("batch", ct.c_int32), ("lr", ct.c_float), ("seed", ct.c_uint64)]


class BiluError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bilu status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded library; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1908_10169_gb300.build.build()")
        L = ct.CDLL(LIB_PATH)
        P, i32, i64, f64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
        sig = {
            "bilu_params_default": ([ct.POINTER(bilu_params)], i32),
            "bilu_create": ([ct.POINTER(P), ct.c_int, P], i32),
            "bilu_analyze": ([P, i64, P, P, P, i32, ct.POINTER(bilu_params)], i32),
            "bilu_factor": ([P, f64], i32),
            "bilu_apply": ([P, P, P], i32),
            "gmres_solve": ([P, P, P, f64, i32, i32, ct.POINTER(gmres_info)], i32),
            "sqmr_solve": ([P, P, P, f64, i32, ct.POINTER(sqmr_info)], i32),
            "bilu_stats": ([P, ct.POINTER(bilu_stats_t)], i32),
            "bilu_get_partition": ([P, P], i32),
            "bilu_get_factor_partition": ([P, P], i32),
            "bilu_export": ([P] * 9, i32),
            "bilu_last_error": ([P], ct.c_char_p),
            "bilu_debug_set": ([P, i32, i64], i32),
            "bilu_apply_noalloc": ([P, P, P], i32),
            "bilu_factor_batch": ([P, i32, f64], i32),
            "gmres_solve_batch": ([P, i32, P, P, f64, i32, i32, P], i32),
            "bilu_record_samples": ([P, i64, f64, ct.c_uint64], i32),
            "bilu_get_samples": ([P, P, P, P, i64, ct.POINTER(i64)], i32),
            "bilu_mlp_train": ([P, P, P, i64, ct.POINTER(bilu_mlp_train_cfg), P, ct.POINTER(f64)], i32),
            "bilu_mlp_forward": ([P, P, P, i64, P], i32),
            "bilu_mlp_grad": ([P, P, P, P, i64, P], i32),
            "bilu_set_skip_model": ([P, P, f64], i32),
            "bilu_cosine_blocking": ([i64, P, P, f64, i32, P, P, ct.POINTER(i32)], i32),
            "bilu_permute_csr": ([i64, P, P, P, P, P, P, P], i32),
            "bilu_partition_ilu1t": ([i64, P, P, P, f64, i32, i32, P, P, ct.POINTER(i32)], i32),
            "bilu_mwm": ([i64, P, P, P, P, P, P], i32),
            "bilu_sym_mwm": ([i64, P, P, P, P, P, P, P], i32),
            "bilu_cosine_blocking_units": ([i64, P, P, f64, i32, i32, P, P, P, P], i32),
            "bilu_nd_order": ([i64, P, P, i32, P, i32, P, P, P], i32),
            "bilu_block_etree": ([i64, P, P, i32, P, P, ct.POINTER(i32)], i32),
            "bilu_scale_permute_csr": ([i64, P, P, P, P, P, P, P, P, P, P], i32),
            "bilu_analyze_partition": ([P, i64, P, P, P, i32, ct.POINTER(bilu_params), i32, P], i32),
            "bilu_destroy": ([P], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ct.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ct.c_void_p)


def _size_of(a, dtype: str, name: str) -> int:
    """Element count of a numpy array or torch tensor of exactly `dtype` (e.g. "float64"),
    C-contiguous; raises TypeError / ValueError otherwise (no silent conversion: the C side
    reads the memory as that type)."""
    if hasattr(a, "data_ptr"):
        got = str(a.dtype).replace("torch.", "")
        if got != dtype:
            raise TypeError(f"{name}: tensor of {got}, expected {dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        return int(a.numel())
    if not hasattr(a, "dtype") or not hasattr(a, "flags"):
        raise TypeError(f"{name}: expected a numpy array or a torch tensor, got {type(a).__name__}")
    if str(a.dtype) != dtype:
        raise TypeError(f"{name}: array of {a.dtype}, expected {dtype}")
    if not a.flags.c_contiguous:
        raise ValueError(f"{name}: array must be C-contiguous")
    return int(a.size)


def _buf(a, dtype: str, count: int | None, name: str, allow_none: bool = False):
    """Pointer of `a` after checking its type and that it holds at least `count` elements
    (count None: not known here).  None passes as NULL where the C call accepts NULL."""
    if a is None:
        if allow_none or count == 0:
            return None
        raise ValueError(f"{name} is None")
    size = _size_of(a, dtype, name)
    if count is not None and size < count:
        raise ValueError(f"{name}: {size} elements, the call needs {count}")
    return _ptr(a)


def _item(a, i: int) -> int:
    """a[i] of a numpy array or a (host or device) torch tensor as a Python int."""
    v = a[i]
    return int(v.item()) if hasattr(v, "item") else int(v)


# the size n of each context's last analysis through this binding (vector length checks)
_CTX_N: dict = {}


def _ctx_key(ctx):
    return ctx.value if hasattr(ctx, "value") else ctx


def _csr(n: int, rowptr, colind, val):
    if n < 0:
        raise ValueError("n < 0")
    prp = _buf(rowptr, "int64", n + 1, "rowptr")
    nnz = _item(rowptr, n)
    if nnz < 0:
        raise ValueError("rowptr[n] < 0")
    return prp, _buf(colind, "int32", nnz, "colind"), _buf(val, "float64", nnz, "val")


def _check(ctx, st: int, allow=(BILU_OK,)):
    if st in allow or st > 0 and BILU_PERTURBED in allow:
        return st
    if st < 0 or st not in allow:
        msg = lib().bilu_last_error(ctx).decode()  # ctx None: this thread's context-free calls
        raise BiluError(st, msg)
    return st


def bilu_params_default(**overrides) -> bilu_params:
    """The library defaults (bilu_params_default), with the given fields overridden."""
    p = bilu_params()
    lib().bilu_params_default(ct.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def bilu_create(device: int = 0, stream=None):
    """Context on `device`; `stream` is a torch.cuda.Stream, a raw cudaStream_t, or None."""
    h = ct.c_void_p()
    raw = None
    if stream is not None:
        raw = ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    st = lib().bilu_create(ct.byref(h), device, raw)
    if st != BILU_OK:
        raise BiluError(st, "bilu_create failed")
    return h


def bilu_destroy(ctx):
    """Releases the context and its device memory."""
    _CTX_N.pop(_ctx_key(ctx), None)
    lib().bilu_destroy(ctx)


def bilu_last_error(ctx) -> str:
    """The last error message of ctx (None: this thread's context-free calls)."""
    return lib().bilu_last_error(ctx).decode()


def bilu_analyze(ctx, n: int, rowptr, colind, val, params: bilu_params | None = None):
    """rowptr int64[n+1], colind int32[nnz], val float64[nnz]; numpy / CPU tensors or CUDA tensors."""
    on_dev = int(bool(getattr(val, "is_cuda", False)))
    prp, pci, pva = _csr(n, rowptr, colind, val)
    p = params if params is not None else bilu_params_default()
    st = lib().bilu_analyze(ctx, n, prp, pci, pva, on_dev, ct.byref(p))
    _check(ctx, st)
    _CTX_N[_ctx_key(ctx)] = n
    return st


def bilu_analyze_partition(ctx, n: int, rowptr, colind, val, bstart, params: bilu_params | None = None):
    """bilu_analyze with the caller's block partition bstart (int32[nblocks + 1], host)."""
    import numpy as np
    on_dev = int(bool(getattr(val, "is_cuda", False)))
    prp, pci, pva = _csr(n, rowptr, colind, val)
    p = params if params is not None else bilu_params_default()
    bs = np.ascontiguousarray(bstart, dtype=np.int32)
    if bs.size < 1:
        raise ValueError("bstart needs at least one entry")
    st = lib().bilu_analyze_partition(ctx, n, prp, pci, pva, on_dev, ct.byref(p), len(bs) - 1, _ptr(bs))
    _check(ctx, st)
    _CTX_N[_ctx_key(ctx)] = n
    return st


def bilu_cosine_blocking(n: int, rowptr, colind, tau: float = 0.8, max_block: int = BILU_MAX_BLOCK):
    """Sec. 3.2 cosine blocking on the host: returns (perm int32[n], bstart int32[nblocks + 1])."""
    import numpy as np
    if n < 0:
        raise ValueError("n < 0")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    if rp.size < n + 1:
        raise ValueError("rowptr needs n + 1 entries")
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    if ci.size < (int(rp[n]) if n > 0 else 0):
        raise ValueError("colind shorter than rowptr[n]")
    perm = np.zeros(max(n, 1), np.int32)
    bs = np.zeros(n + 1, np.int32)
    nb = ct.c_int32(0)
    st = lib().bilu_cosine_blocking(n, _ptr(rp), _ptr(ci), tau, max_block, _ptr(perm), _ptr(bs), ct.byref(nb))
    _check(None, st)
    return perm[:n].copy(), bs[:nb.value + 1].copy()


def bilu_partition_ilu1t(n: int, rowptr, colind, val, tau: float = 1e-2, max_block: int = BILU_MAX_BLOCK,
                         groups=None):
    """Sec. 3.4 partition on the host, column by column or over the given group starts."""
    import numpy as np
    if n < 0:
        raise ValueError("n < 0")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    if rp.size < n + 1:
        raise ValueError("rowptr needs n + 1 entries")
    nnz = int(rp[n]) if n > 0 else 0
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    if ci.size < nnz or va.size < nnz:
        raise ValueError("colind / val shorter than rowptr[n]")
    gs = None if groups is None else np.ascontiguousarray(groups, dtype=np.int32)
    if gs is not None and gs.size < 1:
        raise ValueError("groups needs at least one entry")
    bs = np.zeros(n + 1, np.int32)
    nb = ct.c_int32(0)
    st = lib().bilu_partition_ilu1t(n, _ptr(rp), _ptr(ci), _ptr(va), tau, max_block,
                                    -1 if gs is None else len(gs) - 1, _ptr(gs), _ptr(bs), ct.byref(nb))
    _check(None, st)
    return bs[:nb.value + 1].copy()


def _host_csr(n: int, rowptr, colind, val):
    """Host CSR arrays of the C types, checked against n and rowptr[n] (context-free calls)."""
    import numpy as np
    if n < 0:
        raise ValueError("n < 0")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    if rp.size < n + 1:
        raise ValueError("rowptr needs n + 1 entries")
    nnz = int(rp[n]) if n > 0 else 0
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    if ci.size < nnz or va.size < nnz:
        raise ValueError("colind / val shorter than rowptr[n]")
    return rp, ci, va, nnz


def bilu_mwm(n: int, rowptr, colind, val):
    """Sec. 3.1 maximum weight matching with scaling on the host: (sigma, dl, dr)."""
    import numpy as np
    rp, ci, va, _ = _host_csr(n, rowptr, colind, val)
    sigma = np.zeros(max(n, 1), np.int32)
    dl = np.zeros(max(n, 1))
    dr = np.zeros(max(n, 1))
    _check(None, lib().bilu_mwm(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(sigma), _ptr(dl), _ptr(dr)))
    return sigma[:n].copy(), dl[:n].copy(), dr[:n].copy()


def bilu_cosine_blocking_units(n: int, rowptr, colind, ustart, tau: float = 0.8, max_block: int = 64):
    """Sec. 4.2 cosine blocking of the pattern compressed by the units ustart (whole units per
    block, at most max_block indices): (perm, bstart) over the indices of A."""
    import numpy as np
    if n < 0:
        raise ValueError("n < 0")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    if rp.size < n + 1:
        raise ValueError("rowptr needs n + 1 entries")
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    if ci.size < (int(rp[n]) if n > 0 else 0):
        raise ValueError("colind shorter than rowptr[n]")
    us = np.ascontiguousarray(ustart, dtype=np.int32)
    if us.size < 1:
        raise ValueError("ustart needs at least one entry")
    perm = np.zeros(max(n, 1), np.int32)
    bs = np.zeros(n + 1, np.int32)
    nb = ct.c_int32(0)
    _check(None, lib().bilu_cosine_blocking_units(n, _ptr(rp), _ptr(ci), tau, max_block, len(us) - 1, _ptr(us),
                                                  _ptr(perm), _ptr(bs), ct.byref(nb)))
    return perm[:n].copy(), bs[: nb.value + 1].copy()


def bilu_sym_mwm(n: int, rowptr, colind, val):
    """Sec. 4.2 symmetrised matching of a symmetric A on the host: (perm, ds, ustart), the
    symmetric permutation, the symmetric scaling (by original index) and the 1 x 1 / 2 x 2
    pivot units in the new order."""
    import numpy as np
    rp, ci, va, _ = _host_csr(n, rowptr, colind, val)
    perm = np.zeros(max(n, 1), np.int32)
    ds = np.zeros(max(n, 1))
    ustart = np.zeros(n + 1, np.int32)
    nu = ct.c_int32(0)
    _check(None, lib().bilu_sym_mwm(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(perm), _ptr(ds), _ptr(ustart), ct.byref(nu)))
    return perm[:n].copy(), ds[:n].copy(), ustart[: nu.value + 1].copy()


def bilu_scale_permute_csr(n: int, rowptr, colind, val, rowperm=None, colperm=None, dl=None, dr=None):
    """B[k, l] = A[r_k, c_l] (dl[r_k] dr[c_l]) on the host: returns (rowptr, colind, val)."""
    import numpy as np
    rp, ci, va, nnz = _host_csr(n, rowptr, colind, val)

    def opt(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        if a.size < n:
            raise ValueError("permutations and scalings need n entries")
        return a
    rpm, cpm = opt(rowperm, np.int32), opt(colperm, np.int32)
    sl, sr = opt(dl, np.float64), opt(dr, np.float64)
    orp = np.zeros(n + 1, np.int64)
    oci = np.zeros(max(nnz, 1), np.int32)
    ova = np.zeros(max(nnz, 1), np.float64)
    _check(None, lib().bilu_scale_permute_csr(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(rpm), _ptr(cpm), _ptr(sl),
                                              _ptr(sr), _ptr(orp), _ptr(oci), _ptr(ova)))
    return orp, oci[:nnz].copy(), ova[:nnz].copy()


def _host_pattern(n: int, rowptr, colind, bstart):
    """Host pattern arrays (rowptr, colind) and a partition of the C types, length-checked."""
    import numpy as np
    if n < 0:
        raise ValueError("n < 0")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    if rp.size < n + 1:
        raise ValueError("rowptr needs n + 1 entries")
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    if ci.size < (int(rp[n]) if n > 0 else 0):
        raise ValueError("colind shorter than rowptr[n]")
    bs = np.ascontiguousarray(bstart, dtype=np.int32)
    if bs.size < 1:
        raise ValueError("bstart needs at least one entry")
    return rp, ci, bs


def bilu_nd_order(n: int, rowptr, colind, bstart, leaf: int = 1):
    """Sec. 3.3 block nested dissection on the host: (perm, bstart_out, block_order)."""
    import numpy as np
    rp, ci, bs = _host_pattern(n, rowptr, colind, bstart)
    nb = len(bs) - 1
    perm = np.zeros(max(n, 1), np.int32)
    bso = np.zeros(nb + 1, np.int32)
    order = np.zeros(max(nb, 1), np.int32)
    _check(None, lib().bilu_nd_order(n, _ptr(rp), _ptr(ci), nb, _ptr(bs), leaf, _ptr(perm), _ptr(bso), _ptr(order)))
    return perm[:n].copy(), bso, order[:nb].copy()


def bilu_block_etree(n: int, rowptr, colind, bstart):
    """Block elimination tree on the host: (parent, height)."""
    import numpy as np
    rp, ci, bs = _host_pattern(n, rowptr, colind, bstart)
    nb = len(bs) - 1
    parent = np.zeros(max(nb, 1), np.int32)
    h = ct.c_int32(0)
    _check(None, lib().bilu_block_etree(n, _ptr(rp), _ptr(ci), nb, _ptr(bs), _ptr(parent), ct.byref(h)))
    return parent[:nb].copy(), h.value


def bilu_permute_csr(n: int, rowptr, colind, val, perm):
    """Q^T A Q on the host: returns (rowptr int64[n+1], colind int32[nnz], val float64[nnz])."""
    import numpy as np
    if n < 0:
        raise ValueError("n < 0")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    if rp.size < n + 1 or pm.size < n:
        raise ValueError("rowptr needs n + 1 entries and perm n")
    nnz = int(rp[n]) if n > 0 else 0
    if ci.size < nnz or va.size < nnz:
        raise ValueError("colind / val shorter than rowptr[n]")
    orp = np.zeros(n + 1, np.int64)
    oci = np.zeros(max(nnz, 1), np.int32)
    ova = np.zeros(max(nnz, 1), np.float64)
    st = lib().bilu_permute_csr(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(pm), _ptr(orp), _ptr(oci), _ptr(ova))
    _check(None, st)
    return orp, oci[:nnz].copy(), ova[:nnz].copy()


def bilu_factor(ctx, droptol: float) -> int:
    """Numeric block Crout ILU (Algorithm 1 with blocks, Sec. 2.2); returns BILU_OK or BILU_PERTURBED."""
    st = lib().bilu_factor(ctx, droptol)
    return _check(ctx, st, (BILU_OK, BILU_PERTURBED))


def _vec(ctx, v, name):
    return _buf(v, "float64", _CTX_N.get(_ctx_key(ctx)), name)


def bilu_apply(ctx, r, z) -> int:
    """z = M^{-1} r (float64, n entries each, host or device; r and z distinct)."""
    st = lib().bilu_apply(ctx, _vec(ctx, r, "r"), _vec(ctx, z, "z"))
    return _check(ctx, st)


def bilu_apply_noalloc(ctx, r, z) -> int:
    """bilu_apply for callers that cannot allocate: device vectors only, fixed scratch."""
    st = lib().bilu_apply_noalloc(ctx, _vec(ctx, r, "r"), _vec(ctx, z, "z"))
    return _check(ctx, st)


def gmres_solve(ctx, b, x, tol: float = 1e-8, restart: int = 30, maxit: int = 10000) -> gmres_info:
    """Right-preconditioned GMRES(restart) (Sec. 4); x holds x0 on entry.  The info carries the status."""
    info = gmres_info()
    st = lib().gmres_solve(ctx, _vec(ctx, b, "b"), _vec(ctx, x, "x"), tol, restart, maxit, ct.byref(info))
    _check(ctx, st, (BILU_OK, BILU_NOT_CONVERGED))
    info.status = st
    return info


def sqmr_solve(ctx, b, x, tol: float = 1e-6, maxit: int = 10000) -> sqmr_info:
    """Simplified QMR preconditioned with the context's factor (Sec. 4.2; the symmetric variant
    BILDL gives a symmetric preconditioner), stopped on the normwise backward error; x holds
    x0 on entry.  The info carries the status."""
    info = sqmr_info()
    st = lib().sqmr_solve(ctx, _vec(ctx, b, "b"), _vec(ctx, x, "x"), tol, maxit, ct.byref(info))
    _check(ctx, st, (BILU_OK, BILU_NOT_CONVERGED))
    info.status = st
    return info


def bilu_factor_batch(ctxs, droptol: float) -> int:
    """Factor the analysed matrices of several contexts in one persistent launch."""
    arr = (ct.c_void_p * len(ctxs))(*[c.value if hasattr(c, "value") else c for c in ctxs])
    st = lib().bilu_factor_batch(arr, len(ctxs), droptol)
    return _check(ctxs[0], st, (BILU_OK, BILU_PERTURBED))


def gmres_solve_batch(ctxs, bs, xs, tol: float = 1e-8, restart: int = 30, maxit: int = 10000):
    """GMRES on every system of a batch; returns the gmres_info of each system."""
    n = len(ctxs)
    arr = (ct.c_void_p * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    if len(bs) != n or len(xs) != n:
        raise ValueError("one b and one x per context")
    pb = (ct.c_void_p * n)(*[_vec(c, v, "b").value for c, v in zip(ctxs, bs)])
    px = (ct.c_void_p * n)(*[_vec(c, v, "x").value for c, v in zip(ctxs, xs)])
    infos = (gmres_info * n)()
    st = lib().gmres_solve_batch(arr, n, pb, px, tol, restart, maxit, infos)
    _check(ctxs[0], st, (BILU_OK, BILU_NOT_CONVERGED))
    return list(infos)


def bilu_stats(ctx) -> bilu_stats_t:
    """Statistics of the last analysis / factorization."""
    s = bilu_stats_t()
    _check(ctx, lib().bilu_stats(ctx, ct.byref(s)))
    return s


def bilu_get_partition(ctx, out):
    """Copies the block starts into out (int32, nblocks + 1)."""
    s = bilu_stats(ctx)
    return _check(ctx, lib().bilu_get_partition(ctx, _buf(out, "int32", s.nblocks + 1, "bstart")))


def bilu_get_factor_partition(ctx, out):
    """Copies the factor's block starts (after any merges; void blocks repeat a start) into out
    (int32, nblocks + 1)."""
    s = bilu_stats(ctx)
    return _check(ctx, lib().bilu_get_factor_partition(ctx, _buf(out, "int32", s.nblocks + 1, "bstart")))


def bilu_export(ctx, Lptr=None, Lrow=None, Lval=None, Uptr=None, Ucol=None, Uval=None, Dinv=None, Pblk=None):
    """Copies the factor into host arrays sized from bilu_stats (any may be None)."""
    s = bilu_stats(ctx)
    nb1 = s.nblocks + 1
    args = [_buf(Lptr, "int64", nb1, "Lptr", True), _buf(Lrow, "int32", s.kept_rows, "Lrow", True),
            _buf(Lval, "float64", s.nnz_l, "Lval", True), _buf(Uptr, "int64", nb1, "Uptr", True),
            _buf(Ucol, "int32", s.kept_cols, "Ucol", True), _buf(Uval, "float64", s.nnz_u, "Uval", True),
            _buf(Dinv, "float64", s.nnz_d, "Dinv", True), _buf(Pblk, "float64", s.nnz_d, "Pblk", True)]
    return _check(ctx, lib().bilu_export(ctx, *args))


def bilu_debug_set(ctx, what: int, value: int):
    """Test hooks of the failure paths (BILU_DEBUG_*); not for production use."""
    return _check(ctx, lib().bilu_debug_set(ctx, what, value))


# ---- learned skip --------------------------------------------------------------------------

def bilu_record_samples(ctx, capacity: int, rate: float = 1.0, seed: int = 0):
    """Record (features, label) samples of the candidates in the following factorizations."""
    return _check(ctx, lib().bilu_record_samples(ctx, capacity, rate, seed))


def bilu_get_samples(ctx, x=None, y=None, tags=None, cap: int = 0) -> int:
    """Copies up to cap samples into x (cap x F float32), y (cap float32), tags (cap int64 or
    None); returns the number of samples held."""
    cnt = ct.c_int64()
    px = _buf(x, "float32", cap * BILU_MLP_FEATURES, "x")
    py = _buf(y, "float32", cap, "y")
    pt = _buf(tags, "int64", cap, "tags", allow_none=True)
    _check(ctx, lib().bilu_get_samples(ctx, px, py, pt, cap, ct.byref(cnt)))
    return cnt.value


def bilu_mlp_train(ctx, x, y, epochs: int = 4, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Trains the classifier on n samples (x n x F float32, y n float32); returns (model, loss)."""
    import numpy as np
    n = int(y.shape[0])
    px, py = _buf(x, "float32", n * BILU_MLP_FEATURES, "x"), _buf(y, "float32", n, "y")
    cfg = bilu_mlp_train_cfg(epochs, batch, lr, seed)
    model = np.zeros(BILU_MLP_PARAMS, np.float32)
    loss = ct.c_double()
    _check(ctx, lib().bilu_mlp_train(ctx, px, py, n, ct.byref(cfg), _ptr(model), ct.byref(loss)))
    return model, loss.value


def bilu_mlp_forward(ctx, model, x, logits):
    """Logits of the samples x (n x 12 float32) into logits (n float32)."""
    n = int(logits.shape[0])
    return _check(ctx, lib().bilu_mlp_forward(ctx, _buf(model, "float32", BILU_MLP_PARAMS, "model"),
                                              _buf(x, "float32", n * BILU_MLP_FEATURES, "x"), n,
                                              _buf(logits, "float32", n, "logits")))


def bilu_mlp_grad(ctx, model, x, y):
    """Gradient of the mean cross-entropy with respect to the model (float32, BILU_MLP_PARAMS)."""
    import numpy as np
    n = int(y.shape[0])
    g = np.zeros(BILU_MLP_PARAMS, np.float32)
    _check(ctx, lib().bilu_mlp_grad(ctx, _buf(model, "float32", BILU_MLP_PARAMS, "model"),
                                    _buf(x, "float32", n * BILU_MLP_FEATURES, "x"), _buf(y, "float32", n, "y"),
                                    n, _ptr(g)))
    return g


def bilu_set_skip_model(ctx, model, logit_hi: float):
    """Installs the classifier for BILU_SKIP_LEARNED: candidates with logit >= logit_hi are skipped."""
    return _check(ctx, lib().bilu_set_skip_model(ctx, _buf(model, "float32", BILU_MLP_PARAMS, "model"), logit_hi))
