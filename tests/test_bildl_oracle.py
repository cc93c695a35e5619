"""Pins of the oracle's BILDL, the symmetric variant (incomplete block L D L^T, Sec. 4.2),
against what the paper and the mathematics fix.

- tau = 0 on a dense symmetric indefinite matrix with zero diagonal entries: nothing is
  dropped, so L P L^T is A (numpy), U-breve's columns are P_K L rows, D_K = P_K^{-1}.
- On a symmetric matrix BILU itself (pinned elsewhere) computes the same factor: its T_U is
  the transpose of T_L, so BILDL must keep the same rows and columns and give the same L,
  U-breve and D to rounding; a dropped term or a wrong index in the symmetric loop breaks it.
- Symmetry: every D_K is symmetric bit for bit, every pivot block too, and the preconditioner
  M^{-1} (assembled column by column with the oracle's apply) is symmetric.
- The symmetric perturbation of Sec. 3.6 on a singular 2 x 2 block, worked by hand.
- A matrix that is not symmetric is refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_10169_gb300 import workloads as W


def _sym_indefinite(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    A = B + B.T
    A[np.arange(0, n, 3), np.arange(0, n, 3)] = 0.0  # zero diagonal entries: pivoting needed
    return A


def test_tau0_dense_is_the_exact_ldlt():
    A = _sym_indefinite(12, 1)
    bs = np.array([0, 4, 8, 12], np.int32)
    F = O.bildl_factor(W.from_dense(A), bs, 0.0)
    Ld, Ud = F.dense_L(), F.dense_Ubreve()
    np.testing.assert_allclose(Ld @ Ud, A, rtol=0, atol=1e-12 * np.abs(A).max())
    for K in range(F.nb):
        P, D = F.P_block(K), F.D_block(K)
        assert np.array_equal(D, D.T) and np.array_equal(P, P.T)
        np.testing.assert_allclose(D @ P, np.eye(4), rtol=0, atol=1e-11)
        rows, lv = F.L_block(K)
        cols, uv = F.U_block(K)
        assert np.array_equal(rows, cols)
        if len(rows):
            np.testing.assert_allclose(uv, lv @ P, rtol=0, atol=1e-12 * np.abs(uv).max())
    # the upper factor is P L^T: U-breve = blockdiag(P) L^T
    Pd = np.zeros_like(A)
    for K in range(F.nb):
        s0, s1 = F.bstart[K], F.bstart[K + 1]
        Pd[s0:s1, s0:s1] = F.P_block(K)
    np.testing.assert_allclose(Ud, Pd @ Ld.T, rtol=0, atol=1e-12 * np.abs(A).max())


def _sym_cases():
    w = W.elasticity3d_shifted(side=6, block=24)
    yield "shifted elasticity 6^3, blocks of 24", w.A, O.partition_fixed(w.A.n, 24), 1e-2
    yield "shifted elasticity 6^3, node blocks", w.A, np.arange(0, w.A.n + 1, 3, dtype=np.int32), 1e-2
    A = _sym_indefinite(40, 2)
    A[np.abs(A) < 1.0] = 0.0  # sparse, symmetric pattern
    A += 6.0 * np.eye(40) * (np.arange(40) % 2)
    yield "random symmetric indefinite 40", W.from_dense(A), np.array([0, 5, 12, 20, 27, 33, 40], np.int32), 3e-2


@pytest.mark.parametrize("case", list(range(3)))
def test_bildl_equals_bilu_on_symmetric_matrices(case):
    name, A, bs, tau = list(_sym_cases())[case]
    F = O.bildl_factor(A, bs, tau)
    G = O.bilu_factor(A, bs, tau)
    assert np.array_equal(F.Lptr, G.Lptr) and np.array_equal(F.Lrow, G.Lrow), name
    assert np.array_equal(F.Uptr, G.Uptr) and np.array_equal(F.Ucol, G.Ucol), name
    assert np.array_equal(F.Lrow, F.Ucol), name
    for a, b in ((F.Lval, G.Lval), (F.Uval, G.Uval), (F.Dinv, G.Dinv), (F.Pblk, G.Pblk)):
        assert np.abs(a - b).max() <= 1e-11 * max(np.abs(b).max(), 1.0), name
    # the BILU factor's U-breve columns are the rows of its T_L: again the same values
    r = np.random.default_rng(3).standard_normal(A.n)
    zf, zg = O.bilu_apply(F, r), O.bilu_apply(G, r)
    assert np.abs(zf - zg).max() <= 1e-10 * np.abs(zg).max(), name
    # half the update and scaling work
    assert F.counters["flop_upd_U"] == 0 and F.counters["flop_upd_L"] == G.counters["flop_upd_L"]


@pytest.mark.parametrize("case", list(range(3)))
def test_bildl_is_symmetric(case):
    name, A, bs, tau = list(_sym_cases())[case]
    F = O.bildl_factor(A, bs, tau)
    for K in range(F.nb):
        D, P = F.D_block(K), F.P_block(K)
        assert np.array_equal(D, D.T) and np.array_equal(P, P.T), (name, K)
    n = A.n
    Minv = np.stack([O.bilu_apply(F, e) for e in np.eye(n)], axis=1)
    assert np.abs(Minv - Minv.T).max() <= 1e-12 * np.abs(Minv).max(), name


def test_symmetric_perturbation_worked_example():
    """Blocks of 2 on [[9, 3], [3, 1]] (singular): the LU breaks down at column 1; BILU
    perturbs the largest entry of that column, 3 (2|1| < 3), BILDL the diagonal entry:
    1 (1 + rho) + tau alpha with alpha = max |a_ij| = 9 (Sec. 3.6, beta_j = 1)."""
    A = np.array([[9.0, 3.0], [3.0, 1.0]])
    F = O.bildl_factor(W.from_dense(A), np.array([0, 2], np.int32), 0.0, pert_tau=1e-2, pert_rho=1e-1)
    want = np.array([[9.0, 3.0], [3.0, 1.0 * 1.1 + 1e-2 * 9.0]])
    assert F.status == 2 and F.counters["nperturb"] == 1
    np.testing.assert_allclose(F.P_block(0), want, rtol=1e-15)
    np.testing.assert_allclose(F.D_block(0), np.linalg.inv(want), rtol=1e-12)
    G = O.bilu_factor(W.from_dense(A), np.array([0, 2], np.int32), 0.0, pert_tau=1e-2, pert_rho=1e-1)
    assert G.P_block(0)[0, 1] != 3.0 and G.P_block(0)[1, 1] == 1.0  # the unsymmetric choice


def test_zero_diagonal_block_is_perturbed_on_its_diagonal():
    """A symmetric matrix whose first 2 x 2 block is zero: its columns are zero, so both
    diagonal entries get tau alpha (Sec. 3.6) and the block stays symmetric."""
    A = np.zeros((4, 4))
    A[2:, 2:] = [[4.0, 1.0], [1.0, 3.0]]
    A[0, 2] = A[2, 0] = 0.5
    F = O.bildl_factor(W.from_dense(A), np.array([0, 2, 4], np.int32), 0.0, pert_tau=1e-2, pert_rho=1e-1)
    # column 0 holds 0.5 below the block, but inside the pivot block both columns are zero
    np.testing.assert_array_equal(F.P_block(0), np.diag([4e-2, 4e-2]))
    assert F.counters["nperturb"] == 2


def test_unsymmetric_matrix_is_refused():
    A = _sym_indefinite(8, 4)
    A[1, 5] += 1e-3
    with pytest.raises(ValueError):
        O.bildl_factor(W.from_dense(A), np.array([0, 4, 8], np.int32), 1e-2)
