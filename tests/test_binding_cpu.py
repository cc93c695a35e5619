"""The Python binding's argument checks (CPU): arrays of the wrong type, layout or length are
refused in Python, before the library reads them as its C types."""
import ctypes as ct

import numpy as np
import pytest

import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W


def test_buffer_checks_numpy():
    a = np.zeros(10)
    assert B._buf(a, "float64", 10, "a") is not None
    with pytest.raises(TypeError, match="float32"):
        B._buf(a.astype(np.float32), "float64", 10, "a")
    with pytest.raises(ValueError, match="needs 11"):
        B._buf(a, "float64", 11, "a")
    with pytest.raises(ValueError, match="contiguous"):
        B._buf(np.zeros((4, 4))[:, 1], "float64", 4, "a")
    with pytest.raises(TypeError, match="numpy array or a torch tensor"):
        B._buf([0.0] * 10, "float64", 10, "a")
    assert B._buf(None, "float64", 0, "a") is None
    assert B._buf(None, "float64", 5, "a", allow_none=True) is None
    with pytest.raises(ValueError, match="None"):
        B._buf(None, "float64", 5, "a")


def test_buffer_checks_torch():
    torch = pytest.importorskip("torch")
    t = torch.zeros(8, dtype=torch.float64)
    assert B._buf(t, "float64", 8, "t").value == t.data_ptr()
    with pytest.raises(TypeError, match="int32"):
        B._buf(t.to(torch.int32), "float64", 8, "t")
    with pytest.raises(ValueError, match="contiguous"):
        B._buf(torch.zeros(4, 4, dtype=torch.float64).t(), "float64", 16, "t")
    assert B._item(torch.tensor([3, 7], dtype=torch.int64), 1) == 7


def test_analyze_refuses_wrong_index_types_before_the_library():
    A = W.convdiff_upwind((3, 3, 3), seed=1)
    with pytest.raises(TypeError, match="rowptr"):
        B.bilu_analyze(None, A.n, A.rowptr.astype(np.int32), A.colind, A.val)
    with pytest.raises(TypeError, match="colind"):
        B.bilu_analyze(None, A.n, A.rowptr, A.colind.astype(np.int64), A.val)
    with pytest.raises(ValueError, match="val"):
        B.bilu_analyze(None, A.n, A.rowptr, A.colind, A.val[:-1])
    with pytest.raises(ValueError, match="rowptr"):
        B.bilu_analyze_partition(None, A.n + 1, A.rowptr, A.colind, A.val, [0, A.n + 1])


def test_vectors_checked_against_the_analysed_size():
    key = 0x5eed
    B._CTX_N[key] = 10
    try:
        with pytest.raises(ValueError, match="needs 10"):
            B.bilu_apply(ct.c_void_p(key), np.zeros(5), np.zeros(10))
        with pytest.raises(TypeError, match="float32"):
            B.gmres_solve(ct.c_void_p(key), np.zeros(10, np.float32), np.zeros(10))
    finally:
        B._CTX_N.pop(key, None)


def test_host_only_calls_check_lengths():
    A = W.convdiff_upwind((3, 3, 3), seed=1)
    with pytest.raises(ValueError, match="rowptr"):
        B.bilu_cosine_blocking(A.n + 5, A.rowptr, A.colind)
    with pytest.raises(ValueError):
        B.bilu_permute_csr(A.n, A.rowptr, A.colind, A.val, np.arange(A.n - 1))
