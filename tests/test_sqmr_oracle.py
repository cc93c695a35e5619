"""Pins of the oracle's simplified QMR (the Krylov solver paired with BILDL, Sec. 4.2)
against what the mathematics fixes, through library routines that share nothing with it.

- Without preconditioning on a symmetric A the Lanczos vectors are orthogonal, so the
  quasi-minimal residual is the minimal one: the iterates are MINRES's (scipy), on a
  definite and on an indefinite matrix.  A wrong theta, c or tau breaks it.
- With a symmetric positive definite preconditioner (Jacobi, built as a BILDL factor with
  scalar blocks and every off-diagonal candidate dropped) the BCG part is preconditioned CG,
  and the QMR iterate is the residual smoothing of the CG iterates (scipy's cg):
  x_k = x_{k-1} + c_k^2 (x_k^CG - x_{k-1}), c_k^2 = 1 / (1 + theta_k^2),
  theta_k = ||r_k^CG|| / tau_{k-1}, tau_k = tau_{k-1} theta_k c_k.  A wrong alpha, beta, rho,
  sigma or d recurrence breaks it.
- With the exact factor as preconditioner (one dense block, tau = 0) one step solves.
- The stop: the backward error reported is the normwise one of the returned x, below tol,
  and the one before the last step is above it.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1908_10169_gb300 import workloads as W


def _laplace2d(m, shift=0.0):
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(m, m))
    A = (sp.kron(sp.eye(m), T) + sp.kron(T, sp.eye(m)) - shift * sp.eye(m * m)).tocsr()
    A.sort_indices()
    return A


def _csr(S):
    return W.CSR(S.shape[0], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


def _iterates(A, F, b, ks):
    return [O.sqmr(A, F, b, tol=0.0, maxit=k).x for k in ks]


@pytest.mark.parametrize("shift", [0.0, 0.7])
def test_unpreconditioned_sqmr_is_minres(shift):
    S = _laplace2d(12, shift)
    if shift:
        assert np.linalg.eigvalsh(S.toarray()).min() < 0  # indefinite
    A = _csr(S)
    b = np.random.default_rng(1).standard_normal(A.n)
    ks = list(range(1, 16))
    got = _iterates(A, None, b, ks)
    want = []
    spla.minres(S, b, rtol=1e-30, maxiter=ks[-1], callback=lambda xk: want.append(xk.copy()))
    for k, x in zip(ks, got):
        xm = want[k - 1]
        assert np.abs(x - xm).max() <= 1e-9 * np.abs(xm).max(), k
        # and the residual is the minimal one over x0 + K_k
        assert np.linalg.norm(b - S @ x) <= np.linalg.norm(b - S @ xm) * (1 + 1e-9)


def test_preconditioned_sqmr_is_the_qmr_smoothing_of_pcg():
    S = _laplace2d(10)
    S = (S + sp.diags(np.linspace(0.0, 3.0, S.shape[0]))).tocsr()  # uneven diagonal
    S.sort_indices()
    A = _csr(S)
    b = np.random.default_rng(2).standard_normal(A.n)
    # Jacobi: scalar blocks, every candidate dropped, D_K = 1 / a_kk
    F = O.bildl_factor(A, np.arange(A.n + 1, dtype=np.int32), 1e300)
    assert F.nnz_L() == 0
    np.testing.assert_array_equal(F.Dinv, 1.0 / S.diagonal())
    cg = []
    spla.cg(S, b, rtol=1e-30, maxiter=12, M=sp.diags(1.0 / S.diagonal()), callback=lambda xk: cg.append(xk.copy()))
    tau = np.linalg.norm(b)
    xq = np.zeros(A.n)
    got = _iterates(A, F, b, range(1, 13))
    for k in range(12):
        theta = np.linalg.norm(b - S @ cg[k]) / tau
        c2 = 1.0 / (1.0 + theta * theta)
        tau = tau * theta * np.sqrt(c2)
        xq = xq + c2 * (cg[k] - xq)
        assert np.abs(got[k] - xq).max() <= 1e-10 * np.abs(xq).max(), k


def test_exact_preconditioner_solves_in_one_step():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((30, 30))
    Ad = B + B.T
    A = W.from_dense(Ad)
    F = O.bildl_factor(A, np.array([0, 30], np.int32), 0.0)
    b = rng.standard_normal(30)
    res = O.sqmr(A, F, b, tol=1e-12, maxit=5)
    assert res.status == 0 and res.iters == 1
    np.testing.assert_allclose(res.x, np.linalg.solve(Ad, b), rtol=1e-10, atol=1e-12)


def test_backward_error_stop():
    w = W.elasticity3d_shifted(side=6, block=24)
    A = w.A
    S = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    F = O.bildl_factor(A, O.partition_fixed(A.n, 24), 1e-1)
    res = O.sqmr(A, F, w.b, tol=1e-6, maxit=500)
    assert res.status == 0 and res.iters > 1
    anorm = np.abs(S).sum(axis=1).max()
    eta = np.abs(w.b - S @ res.x).max() / (anorm * np.abs(res.x).max() + np.abs(w.b).max())
    assert abs(eta - res.berr) <= 1e-12 and eta <= 1e-6 < res.hist[-2]
    prev = O.sqmr(A, F, w.b, tol=1e-6, maxit=res.iters - 1)
    assert prev.status == 1 and prev.berr > 1e-6


def test_zero_rhs_and_converged_start():
    S = _laplace2d(5)
    A = _csr(S)
    res = O.sqmr(A, None, np.zeros(A.n), tol=1e-6, maxit=10)
    assert res.status == 0 and res.iters == 0 and not res.x.any()
    x = np.linalg.solve(S.toarray(), np.ones(A.n))
    res = O.sqmr(A, None, np.ones(A.n), tol=1e-6, maxit=10, x0=x)
    assert res.status == 0 and res.iters == 0


def test_breakdown_is_reported():
    """[[0, 1], [1, 0]] with b = e_1 and no preconditioner: q = r = e_1 and q^T A q = 0, so the
    first step cannot be taken (sigma = 0): a breakdown after zero steps, x unchanged."""
    A = W.from_dense(np.array([[0.0, 1.0], [1.0, 0.0]]))
    res = O.sqmr(A, None, np.array([1.0, 0.0]), tol=1e-12, maxit=10)
    assert res.status == 3 and res.iters == 0 and not res.x.any()
