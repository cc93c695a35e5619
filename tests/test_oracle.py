"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something independent of it: the literal
scalar Crout ILU of Algorithm 1 (written separately below), dense right-looking block
elimination with the same drop rule, LAPACK through scipy/numpy, closed forms, and
hand-derived values of the ILU(1,tau) growth rule and of the perturbation rule.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1908_10169_gb300 import workloads as W


# ----------------------------------------------------------------- independent references

def crout_ilu_alg1(Ad: np.ndarray, tau: float):
    """Algorithm 1 (Crout ILU) written out literally on dense storage.

    Column k of L: l_ik = a_ik - sum_{j<k} l_ij u_jk (i >= k); drop |l_ik| <= tau |l_kk|;
    divide by l_kk.  Row k of U: u_ki = a_ki - sum_{j<k} l_kj u_ji; drop |u_ki| <= tau |u_kk|.
    Dropped entries are stored as zeros, so they take no part in later updates.
    """
    n = Ad.shape[0]
    L = np.zeros((n, n))
    U = np.zeros((n, n))
    for k in range(n):
        l = Ad[k:, k] - L[k:, :k] @ U[:k, k]
        lkk = l[0]
        drop = np.abs(l) <= tau * abs(lkk)
        drop[0] = False
        l[drop] = 0.0
        L[k:, k] = l / lkk
        u = Ad[k, k:] - L[k, :k] @ U[:k, k:]
        ukk = u[0]
        dropu = np.abs(u) <= tau * abs(ukk)
        dropu[0] = False
        u[dropu] = 0.0
        U[k, k:] = u
    return L, U


def dense_block_elimination(Ad: np.ndarray, bstart, tau: float):
    """Right-looking dense block elimination with the block drop rule (independent of the
    Crout ordering; equivalent because a block column is only dropped after all of its
    updates).  Returns dense L (unit block lower), U-breve (P_K on the diagonal) and D."""
    n = Ad.shape[0]
    Wm = Ad.copy()
    L = np.eye(n)
    Ub = np.zeros((n, n))
    Ds = []
    for K in range(len(bstart) - 1):
        s0, s1 = bstart[K], bstart[K + 1]
        P = Wm[s0:s1, s0:s1].copy()
        D = np.linalg.inv(P)
        Ds.append(D)
        Ub[s0:s1, s0:s1] = P
        if s1 < n:
            ell = Wm[s1:, s0:s1] @ D
            keepr = np.linalg.norm(ell, axis=1) > tau
            uh = D @ Wm[s0:s1, s1:]
            keepc = np.linalg.norm(uh, axis=0) > tau
            L[s1:, s0:s1] = np.where(keepr[:, None], ell, 0.0)
            Ub[s0:s1, s1:] = np.where(keepc[None, :], Wm[s0:s1, s1:], 0.0)
            Wm[s1:, s1:] -= L[s1:, s0:s1] @ Ub[s0:s1, s1:]
    return L, Ub, Ds


def random_partition(n, maxb, rng):
    bs = [0]
    while bs[-1] < n:
        bs.append(min(n, bs[-1] + int(rng.integers(1, maxb + 1))))
    return np.array(bs, dtype=np.int32)


def lapack_perm(piv):
    """LAPACK ipiv (row swaps) -> permutation p with (P A)[i] = A[p[i]]."""
    p = np.arange(len(piv))
    for i, j in enumerate(piv):
        p[i], p[j] = p[j], p[i]
    return p


# ----------------------------------------------------------------- algorithm 1 special case

@pytest.mark.parametrize("seed,tau", [(0, 0.0), (1, 1e-3), (2, 1e-2), (3, 5e-2), (4, 0.2)])
def test_scalar_blocks_equal_algorithm1(seed, tau):
    """BILU with all blocks of size 1 is the scalar Crout ILU (Sec. 4: BILU without
    blocking reduces to scalar ILU; Algorithm 1)."""
    A = W.random_diag_dominant(60, 0.12, seed, dominance=1.1)
    F = O.bilu_factor(A, O.partition_fixed(A.n, 1), tau)
    L, U = crout_ilu_alg1(A.to_dense(), tau)
    Lo, Uo = F.dense_L(), F.dense_Ubreve()
    assert np.array_equal(Lo != 0, L != 0), "drop pattern of L differs from Algorithm 1"
    assert np.array_equal(Uo != 0, U != 0), "drop pattern of U differs from Algorithm 1"
    assert np.allclose(Lo, L, rtol=1e-13, atol=1e-14)
    assert np.allclose(Uo, U, rtol=1e-13, atol=1e-13 * np.abs(U).max())
    # D holds the inverted 1x1 pivots
    assert np.allclose(F.Dinv, 1.0 / np.diag(U), rtol=1e-14)


def test_scalar_blocks_equal_algorithm1_convdiff():
    w = W.cd2d_32()
    F = O.bilu_factor(w.A, O.partition_fixed(w.A.n, 1), 1e-2)
    L, U = crout_ilu_alg1(w.A.to_dense(), 1e-2)
    assert np.array_equal(F.dense_L() != 0, L != 0)
    assert np.array_equal(F.dense_Ubreve() != 0, U != 0)
    assert np.allclose(F.dense_L(), L, rtol=1e-12, atol=1e-14)
    assert np.allclose(F.dense_Ubreve(), U, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------- exactness at tau = 0

@pytest.mark.parametrize("seed,maxb", [(10, 1), (11, 3), (12, 7), (13, 16), (14, 40)])
def test_tau0_gives_exact_block_lu(seed, maxb):
    """No dropping: L D^{-1} U = L U-breve reproduces A (block LU, pivoting only inside the
    diagonal blocks, Sec. 2.2)."""
    rng = np.random.default_rng(seed)
    A = W.random_diag_dominant(120, 0.05, seed)
    bs = random_partition(A.n, maxb, rng)
    F = O.bilu_factor(A, bs, 0.0)
    Ad = A.to_dense()
    M = F.dense_L() @ F.dense_Ubreve()
    assert np.linalg.norm(Ad - M) / np.linalg.norm(Ad) <= 1e-13
    # L is unit lower block triangular: every stored row lies below its block
    for K in range(F.nb):
        rows, _ = F.L_block(K)
        cols, _ = F.U_block(K)
        assert np.all(rows >= bs[K + 1]) and np.all(np.diff(rows) > 0)
        assert np.all(cols >= bs[K + 1]) and np.all(np.diff(cols) > 0)


def test_tau0_convdiff_exact():
    w = W.cd2d_32()
    F = O.bilu_factor(w.A, O.partition_fixed(w.A.n, 8), 0.0)
    Ad = w.A.to_dense()
    assert np.linalg.norm(Ad - F.dense_L() @ F.dense_Ubreve()) / np.linalg.norm(Ad) <= 1e-13
    r = O.gmres(w.A, F, w.b)
    assert r.iters == 1 and r.relres <= 1e-12


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (64, 3), (257, 4)])
def test_single_block_is_dense_partial_pivot_lu(n, seed):
    """One block covering the whole matrix: the diagonal-block getrf is dense LU with
    partial pivoting, ||PA - LU|| / ||A|| <= 1e-13, identical pivots to LAPACK."""
    rng = np.random.default_rng(seed)
    Ad = rng.standard_normal((n, n))
    A = W.from_dense(Ad)
    F = O.bilu_factor(A, np.array([0, n], np.int32), 0.0)
    LU, perm = F.LU_block(0)
    Lf = np.tril(LU, -1) + np.eye(n)
    Uf = np.triu(LU)
    assert np.linalg.norm(Ad[perm] - Lf @ Uf) / np.linalg.norm(Ad) <= 1e-13
    lu, piv = sla.lu_factor(Ad)
    assert np.array_equal(perm, lapack_perm(piv))
    assert np.allclose(LU, lu, rtol=1e-10, atol=1e-12)
    D = F.D_block(0)
    assert np.linalg.norm(D @ Ad - np.eye(n)) <= 1e-12 * np.linalg.cond(Ad)
    assert np.allclose(D, np.linalg.inv(Ad), rtol=1e-9, atol=1e-12 * np.abs(D).max())


def test_block_diagonal_matrix_gives_per_block_inverse():
    rng = np.random.default_rng(5)
    bs = random_partition(90, 12, rng)
    Ad = np.zeros((90, 90))
    for K in range(len(bs) - 1):
        s0, s1 = bs[K], bs[K + 1]
        Ad[s0:s1, s0:s1] = rng.standard_normal((s1 - s0, s1 - s0)) + 3 * np.eye(s1 - s0)
    A = W.from_dense(Ad)
    F = O.bilu_factor(A, bs, 1e-2)
    assert F.Lrow.size == 0 and F.Ucol.size == 0
    for K in range(F.nb):
        s0, s1 = bs[K], bs[K + 1]
        assert np.allclose(F.D_block(K), np.linalg.inv(Ad[s0:s1, s0:s1]), rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------------- dropping: brute force

@pytest.mark.parametrize("seed", range(8))
def test_dropping_matches_dense_block_elimination(seed):
    """n <= 64: identical keep masks and values (to 1e-12) against right-looking dense block
    elimination with the same rule ||l_i D_K|| <= tau, ||D_K u_j|| <= tau (Sec. 2.2)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 65))
    A = W.random_diag_dominant(n, 0.15, 200 + seed, dominance=1.05)
    tau = [1e-3, 1e-2, 3e-2, 1e-1][seed % 4]
    bs = random_partition(n, int(rng.integers(1, 9)), rng)
    F = O.bilu_factor(A, bs, tau)
    L, Ub, Ds = dense_block_elimination(A.to_dense(), bs, tau)
    Lo, Uo = F.dense_L(), F.dense_Ubreve()
    # compare per row / per column keep decisions
    for K in range(len(bs) - 1):
        s0, s1 = bs[K], bs[K + 1]
        assert np.array_equal(np.any(Lo[s1:, s0:s1] != 0, axis=1), np.any(L[s1:, s0:s1] != 0, axis=1))
        assert np.array_equal(np.any(Uo[s0:s1, s1:] != 0, axis=0), np.any(Ub[s0:s1, s1:] != 0, axis=0))
        assert np.allclose(F.D_block(K), Ds[K], rtol=1e-11, atol=1e-12 * np.abs(Ds[K]).max())
    assert np.allclose(Lo, L, rtol=1e-11, atol=1e-12)
    assert np.allclose(Uo, Ub, rtol=1e-11, atol=1e-12 * np.abs(Ub).max())


def test_kept_norms_exceed_tau_and_dropped_are_not_stored():
    A = W.convdiff_upwind((10, 10, 10), seed=3)
    tau = 1e-2
    F = O.bilu_factor(A, O.partition_fixed(A.n, 10), tau)
    for K in range(F.nb):
        rows, lv = F.L_block(K)
        cols, uv = F.U_block(K)
        if rows.size:
            assert np.all(np.linalg.norm(lv, axis=1) > tau)
        if cols.size:
            uh = F.D_block(K) @ uv.T
            assert np.all(np.linalg.norm(uh, axis=0) > tau)
        assert np.allclose(F.D_block(K) @ F.P_block(K), np.eye(F.bsize(K)), atol=1e-10)


# ----------------------------------------------------------------- application

@pytest.mark.parametrize("blk", [1, 5, 16])
def test_apply_inverts_LU(blk):
    """z = M^{-1} r with M = L U-breve: apply(M x) = x."""
    A = W.convdiff_upwind((8, 8, 6), seed=4)
    F = O.bilu_factor(A, O.partition_fixed(A.n, blk), 1e-2)
    M = F.dense_L() @ F.dense_Ubreve()
    x = np.random.default_rng(0).standard_normal(A.n)
    z = O.bilu_apply(F, M @ x)
    assert np.linalg.norm(z - x) <= 1e-12 * np.linalg.norm(x) * np.linalg.cond(M) ** 0.5
    assert np.linalg.norm(z - np.linalg.solve(M, M @ x)) <= 1e-11 * np.linalg.norm(x)


# ----------------------------------------------------------------- GMRES

def test_gmres_exact_preconditioner_one_step():
    A = W.convdiff_upwind((6, 6, 6), seed=2)
    F = O.bilu_factor(A, O.partition_fixed(A.n, 6), 0.0)
    r = O.gmres(A, F, W.rhs_ones(A), tol=1e-8)
    assert r.iters == 1 and r.relres <= 1e-12


def test_gmres_unpreconditioned_matches_scipy_count():
    """Identity preconditioner: the inner-step count agrees with scipy's GMRES(30) (+-1)."""
    w = W.cd2d_32()
    r = O.gmres(w.A, None, w.b, tol=1e-8, restart=30, maxit=5000)
    As = sp.csr_matrix((w.A.val, w.A.colind, w.A.rowptr), shape=(w.A.n, w.A.n))
    count = [0]

    def cb(_):
        count[0] += 1

    xs, info = spla.gmres(As, w.b, rtol=1e-8, atol=0.0, restart=30, maxiter=200, callback=cb,
                          callback_type="pr_norm")
    assert info == 0
    assert abs(count[0] - r.iters) <= 1, (count[0], r.iters)
    assert r.relres <= 1e-8
    assert np.abs(r.x - 1.0).max() < 1e-5


def test_gmres_preconditioned_solution():
    A = W.convdiff_upwind((12, 12, 12), seed=1)
    b = W.rhs_ones(A)
    F = O.bilu_factor(A, O.partition_fixed(A.n, 12), 1e-2)
    r = O.gmres(A, F, b, tol=1e-8)
    r0 = O.gmres(A, None, b, tol=1e-8)
    assert r.status == 0 and r.relres <= 1e-8
    assert r.iters < r0.iters
    xs = spla.spsolve(sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n)).tocsc(), b)
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) <= 1e-8 * np.linalg.cond(A.to_dense())
    # the recorded Givens estimate ends below tol
    assert r.hist[-1] <= 1e-8


def test_gmres_is_scale_invariant():
    """GMRES is invariant under b -> 2^-30 b (stopping test relative to ||b||, Sec. 4 setup):
    the same number of steps and x scaled by the same power of two."""
    A = W.convdiff_upwind((12, 12, 12), seed=1)
    b = W.rhs_ones(A)
    F = O.bilu_factor(A, O.partition_fixed(A.n, 12), 1e-2)
    s = 2.0 ** -30
    for M in (F, None):
        r = O.gmres(A, M, b, tol=1e-8)
        rs = O.gmres(A, M, b * s, tol=1e-8)
        assert rs.iters == r.iters and rs.status == 0
        assert np.max(np.abs(rs.x / s - r.x)) <= 1e-12 * np.max(np.abs(r.x))


def test_gmres_zero_rhs():
    A = W.convdiff_upwind((4, 4, 4), seed=1)
    r = O.gmres(A, None, np.zeros(A.n))
    assert r.iters == 0 and np.all(r.x == 0)


# ----------------------------------------------------------------- perturbation (Sec. 3.6)

def test_zero_column_in_diagonal_block_is_perturbed():
    """Column 1 of the 2x2 diagonal block [[2,0],[1,0]] is zero: its diagonal entry becomes
    sign(0) tau alpha = 1e-2 * alpha (beta_j := 1, sign(0) := +1)."""
    Ad = np.array([[2.0, 0.0, 1.0], [1.0, 0.0, 5.0], [0.5, 1.0, 4.0]])
    A = W.from_dense(Ad)
    alpha = np.abs(Ad).max()
    bs = np.array([0, 2, 3], np.int32)
    F = O.bilu_factor(A, bs, 0.0, perturb=True)
    assert F.status == 2 and F.counters["nperturb"] == 1
    P = F.P_block(0)
    assert P[1, 1] == pytest.approx(1e-2 * alpha, rel=1e-15)
    assert np.allclose(F.D_block(0), np.linalg.inv(np.array([[2.0, 0.0], [1.0, 1e-2 * alpha]])))
    with pytest.raises(RuntimeError):
        O.bilu_factor(A, bs, 0.0, perturb=False)


def test_zero_row_in_diagonal_block_is_perturbed():
    """Row 1 of the 2x2 diagonal block [[2,1],[0,0]] is zero (row 1 of A has its only entry
    outside the block): its diagonal entry becomes sign(0) tau alpha = 1e-2 * alpha, alpha =
    max|a_ij| = 4 (Sec. 3.6, rows like columns)."""
    Ad = np.array([[2.0, 1.0, 0.5], [0.0, 0.0, 3.0], [1.0, 0.5, 4.0]])
    F = O.bilu_factor(W.from_dense(Ad), np.array([0, 2, 3], np.int32), 0.0, perturb=True)
    assert F.status == 2 and F.counters["nperturb"] == 1
    Pexp = np.array([[2.0, 1.0], [0.0, 4e-2]])
    assert np.allclose(F.P_block(0), Pexp, rtol=1e-15, atol=0)
    assert np.allclose(F.D_block(0), np.linalg.inv(Pexp), rtol=1e-12)


def test_singular_block_perturbed_at_diagonal():
    """[[1,1],[1,1]] breaks at pivot 2; column 1's largest entry is a_01 = 1 but the diagonal
    wins (2|d_11| >= |d_01|): d_11 <- d_11 (1 + rho) + tau alpha."""
    Ad = np.array([[1.0, 1.0], [1.0, 1.0]])
    A = W.from_dense(Ad)
    F = O.bilu_factor(A, np.array([0, 2], np.int32), 0.0, perturb=True, pert_tau=1e-2, pert_rho=1e-1)
    assert F.status == 2 and F.counters["nperturb"] == 1
    Pexp = np.array([[1.0, 1.0], [1.0, 1.0 * 1.1 + 1e-2 * 1.0]])
    assert np.allclose(F.P_block(0), Pexp, rtol=1e-15)
    assert np.allclose(F.D_block(0), np.linalg.inv(Pexp), rtol=1e-12)


@pytest.mark.parametrize("d11,expect", [
    # 2|d_11| = 3 >= |d_01| = 2: the diagonal entry is perturbed, 1.5 (1 + 0.1) + 0.01 * 2
    (1.5, [[1.0, 2.0], [0.75, 1.67]]),
    # 2|d_11| = 1 < |d_01| = 2: the largest entry of the column is perturbed, 2 (1 + 0.1) + 0.01 * 2
    (0.5, [[1.0, 2.22], [0.25, 0.5]])])
def test_breakdown_perturbs_diagonal_only_within_factor_two(d11, expect):
    """Singular [[1, 2], [d_10, d_11]] with d_10 = d_11 / 2 breaks at pivot 2 (first pivot row 0,
    l_10 = d_10, u_11 = d_11 - 2 d_10 = 0).  Column 1's largest entry is d_01 = 2; the diagonal
    entry is taken instead when 2|d_11| >= |d_01| (Sec. 3.6); alpha = max|a_ij| = 2."""
    Ad = np.array([[1.0, 2.0], [d11 / 2, d11]])
    F = O.bilu_factor(W.from_dense(Ad), np.array([0, 2], np.int32), 0.0, perturb=True,
                      pert_tau=1e-2, pert_rho=1e-1)
    assert F.status == 2 and F.counters["nperturb"] == 1
    assert np.allclose(F.P_block(0), np.array(expect), rtol=1e-15, atol=0)
    assert np.allclose(F.D_block(0), np.linalg.inv(np.array(expect)), rtol=1e-12)


def test_no_perturbation_on_regular_workloads():
    w = W.cd2d_32()
    F = O.bilu_factor(w.A, O.partition_fixed(w.A.n, 32), 1e-2)
    assert F.status == 0 and F.counters["nperturb"] == 0


# ----------------------------------------------------------------- counters

def test_flop_counters_single_dense_block():
    n = 10
    Ad = np.random.default_rng(1).standard_normal((n, n)) + 5 * np.eye(n)
    F = O.bilu_factor(W.from_dense(Ad), np.array([0, n], np.int32), 0.0)
    c = F.counters
    assert c["flop_getrf"] == pytest.approx(2 / 3 * n ** 3)
    assert c["flop_inv"] == pytest.approx(4 / 3 * n ** 3)
    assert c["flop_upd_L"] == 0 and c["cand_rows"] == 0


def test_flop_counters_two_blocks_dense():
    """Two dense blocks of 3: the L-side update of block 1 is a 3x3x3 product (2*27 flops),
    the U side has no columns beyond the last block."""
    Ad = np.random.default_rng(2).standard_normal((6, 6)) + 6 * np.eye(6)
    F = O.bilu_factor(W.from_dense(Ad), np.array([0, 3, 6], np.int32), 0.0)
    c = F.counters
    assert c["flop_upd_L"] == 2 * 3 * 3 * 3
    assert c["flop_upd_U"] == 0
    assert c["cand_rows"] == 3 and c["cand_cols"] == 3


# ----------------------------------------------------------------- threshold and tie pins

def test_drop_at_exact_threshold_scalar():
    """|l_ik| <= tau |l_kk| drops (Algorithm 1): with tau = 1/2, a_10 / a_00 = 1/2 is dropped
    and so is u_01 / u_00; the second pivot is then a_11 unchanged."""
    A = W.from_dense(np.array([[2.0, 1.0], [1.0, 3.0]]))
    F = O.bilu_factor(A, O.partition_fixed(2, 1), 0.5)
    assert F.Lrow.size == 0 and F.Ucol.size == 0
    assert F.P_block(1)[0, 0] == 3.0
    F2 = O.bilu_factor(A, O.partition_fixed(2, 1), 0.49)
    assert F2.Lrow.size == 1 and F2.P_block(1)[0, 0] == 2.5


@pytest.mark.parametrize("tau,kept", [(0.6, True), (0.625, False), (0.7, False)])
def test_drop_norm_is_euclidean_row_norm(tau, kept):
    """Block row l_i = T_L[i, B_K] D_K = [0.375, 0.5] (exact in binary): 2-norm 0.625,
    inf-norm 0.5, 1-norm 0.875.  tau = 0.6 separates the 2-norm from the inf-norm, tau = 0.7
    from the 1-norm; tau = 0.625 is the exact threshold (dropped)."""
    Ad = np.array([[2.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.75, 1.0, 5.0]])
    F = O.bilu_factor(W.from_dense(Ad), np.array([0, 2, 3], np.int32), tau)
    assert (F.Lrow.size == 1) == kept
    if kept:
        assert np.array_equal(F.L_block(0)[1][0], [0.375, 0.5])
        assert F.P_block(1)[0, 0] == 5.0  # U side of block 0 is empty, no update


def test_pivot_tie_takes_first_row_like_lapack():
    Ad = np.array([[1.0, 2.0], [-1.0, 3.0]])
    F = O.bilu_factor(W.from_dense(Ad), np.array([0, 2], np.int32), 0.0)
    LU, perm = F.LU_block(0)
    assert list(perm) == [0, 1]
    # ties in the first column (before any arithmetic): rows 2 and 4 share the largest |.|
    rng = np.random.default_rng(7)
    for _ in range(10):
        Bd = rng.uniform(-1.0, 1.0, size=(6, 6))
        Bd[2, 0], Bd[4, 0] = 5.0, -5.0
        Fb = O.bilu_factor(W.from_dense(Bd), np.array([0, 6], np.int32), 0.0)
        _, pb = Fb.LU_block(0)
        _, piv = sla.lu_factor(Bd)
        assert pb[0] == 2 and lapack_perm(piv)[0] == 2
