"""The library's host-side maximum weight matching with scaling (Sec. 3.1) and the general
scale-and-permute transform, against the oracle and scipy on the CPU (host code: no context,
no device).  Several matchings can be optimal, so the optimal cost is compared and the rest is
checked for validity: a perfect matching, |a^_ij| <= 1, |a^_ii| = 1."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1908_10169_gb300 as B
from oracle import mwm_oracle as M
from paper_1908_10169_gb300 import workloads as W
from tests.test_mwm_oracle import random_matchable


def _cases():
    for s in range(8):
        yield f"random{s}", random_matchable(5 + 9 * s, 0.1 + 0.02 * s, 200 + s)[0]
    A = W.convdiff_upwind((5, 5, 5), seed=1)
    yield "convdiff", A
    rows = np.random.default_rng(4).permutation(A.n).astype(np.int32)
    yield "convdiff_rows_scrambled", W.CSR(A.n, *B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, rowperm=rows))
    yield "elasticity", W.elasticity3d(side=3, seed=2, block=63).A


CASES = dict(_cases())


@pytest.mark.parametrize("name", sorted(CASES))
def test_library_matching_is_optimal_and_scales(name):
    A = CASES[name]
    sigma, dl, dr = B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
    so, dlo, dro, u, v, total = M.mwm(A)
    C, _ = M.costs(A)
    assert sorted(sigma) == list(range(A.n))
    assert abs(sum(C[i, sigma[i]] for i in range(A.n)) - total) <= 1e-11 * max(1.0, abs(total))
    Ah = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n)).toarray()
    Ah = dl[:, None] * Ah * dr[None, :]
    assert np.all(np.abs(Ah) <= 1 + 1e-12)
    assert np.allclose(np.abs(Ah[np.arange(A.n), sigma]), 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", sorted(CASES))
def test_transform_matches_scipy(name):
    A = CASES[name]
    rng = np.random.default_rng(len(name))
    rp_, cp_ = rng.permutation(A.n).astype(np.int32), rng.permutation(A.n).astype(np.int32)
    dl, dr = rng.uniform(0.5, 2.0, A.n), rng.uniform(0.5, 2.0, A.n)
    D = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    for rows, cols, l, r in ((rp_, cp_, dl, dr), (None, cp_, dl, None), (rp_, rp_, None, None)):
        got = B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, rows, cols, l, r)
        M_ = D.multiply(l[:, None]) if l is not None else D
        M_ = sp.csr_matrix(M_.multiply(r[None, :])) if r is not None else sp.csr_matrix(M_)
        M_ = M_[rows if rows is not None else np.arange(A.n)][:, cols if cols is not None else np.arange(A.n)].tocsr()
        M_.sort_indices()
        assert np.array_equal(got[0], M_.indptr) and np.array_equal(got[1], M_.indices)
        assert np.allclose(got[2], M_.data, rtol=1e-15, atol=0)


def test_matching_solves_the_scrambled_system():
    """Rows of a convection-diffusion matrix in a random order have zeros on the diagonal; the
    matching puts the original diagonal back (the unique optimum), so A^ y = D_l b solved
    exactly gives x with A x = b."""
    A = CASES["convdiff_rows_scrambled"]
    sigma, dl, dr = B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
    Ahat = W.CSR(A.n, *B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, None, sigma, dl, dr))
    Hd = sp.csr_matrix((Ahat.val, Ahat.colind, Ahat.rowptr), shape=(A.n, A.n))
    assert np.allclose(np.abs(Hd.diagonal()), 1.0, atol=1e-12)
    b = np.random.default_rng(0).standard_normal(A.n)
    y = np.linalg.solve(Hd.toarray(), dl * b)
    x = np.zeros(A.n)
    x[sigma] = dr[sigma] * y
    Ad = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    assert np.linalg.norm(Ad @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_matching_errors():
    d = np.array([[1.0, 0, 0], [2.0, 0, 0], [1.0, 1.0, 1.0]])
    A = W.from_dense(d, keep_zeros_on_diag=False)
    with pytest.raises(B.BiluError) as e:
        B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
    assert e.value.status == B.BILU_ERR_SINGULAR and "singular" in str(e.value)
    bad = A.val.copy()
    bad[0] = np.inf
    with pytest.raises(B.BiluError, match="non-finite"):
        B.bilu_mwm(A.n, A.rowptr, A.colind, bad)
    with pytest.raises(B.BiluError, match="rowperm"):
        B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, rowperm=np.array([0, 0, 1], np.int32))
