"""Pins of the oracle's progressive aggregation (Sec. 3.5) against what the paper and the
mathematics fix.

- The merge test, evaluated on counts worked out by hand from its two inequalities,
  including both boundaries.
- Two dense blocks that merge into one: the merged block is then the LU of the whole
  matrix, so its pivot block is A and its inverse is A^{-1} (numpy).
- The defining identity: a merge only rewrites finished blocks, so the product of the
  factors, L (block diagonal P) U, is the same with and without aggregation (to rounding);
  a dropped term or a wrong sign in any of the rewritten pieces breaks it.
- The common pattern: a merged block stores the union of its members' rows (columns),
  taken from the factor computed without aggregation.
- The sequence of merges: replaying the test on the unaggregated factor's patterns, block
  after block, gives the same block boundaries.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_10169_gb300 import workloads as W


# ----------------------------------------------------------------- the merge test

@pytest.mark.parametrize("counts,merge", [
    # p q r s r' s' t t' u v: mu = 2(2+2+0+2+0) + 2(2) = 16, nu = 4*4 = 16 <= 19.2
    ((2, 2, 2, 0, 2, 0, 0, 0, 0, 0), True),
    # mu = 4(4+4+8+4+8) + 4(4+8+8) = 192, nu = 8(8+12+12) = 256 > 230.4 and > 208
    ((4, 4, 4, 8, 4, 8, 8, 8, 12, 12), False),
    # mu = (1+1+2+1+2) + (1+2+2) = 12; nu = 2(2+3+3) = 16: not <= 14.4, but <= 12 + 4
    ((1, 1, 1, 2, 1, 2, 2, 2, 3, 3), True),
    # nu = 2(2+4+3) = 18 > 14.4 and > 16
    ((1, 1, 1, 2, 1, 2, 2, 2, 4, 3), False),
    # mu = (1+2+7+2+6) + (1+3+3) = 25; nu = 2(2+7+6) = 30 = 1.2 mu exactly (> mu + 4 = 29)
    ((1, 1, 2, 7, 2, 6, 3, 3, 7, 6), True),
    # nu = 2(2+7+7) = 32 > 30 and > 29
    ((1, 1, 2, 7, 2, 6, 3, 3, 7, 7), False),
])
def test_merge_rule_hand_counts(counts, merge):
    assert O.agg_rule(*counts) == merge


# ----------------------------------------------------------------- two dense blocks

def test_two_dense_blocks_merge_into_the_whole_lu():
    """4 x 4 dense, blocks of 2, tau = 0: mu = nu = 16, so the blocks merge; the merged
    block is the whole matrix, P-hat = A and D-hat = A^{-1}, with nothing left in L or U."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4, 4)) + 4 * np.eye(4)
    F = O.bilu_factor(W.from_dense(A), np.array([0, 2, 4], np.int32), 0.0, agg_max=64)
    assert F.merges == 1
    assert list(F.bstart) == [0, 0, 4]
    assert F.Lrow.size == 0 and F.Ucol.size == 0
    np.testing.assert_allclose(F.P_block(1), A, rtol=0, atol=1e-14 * np.abs(A).max())
    np.testing.assert_allclose(F.D_block(1), np.linalg.inv(A), rtol=0, atol=1e-13)


def test_three_dense_blocks_merge_step_by_step():
    """6 x 6 dense, blocks of 2: the first merge gives a block of 4 that the third block then
    joins (the test is taken against the merged block), again the whole LU."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((6, 6)) + 5 * np.eye(6)
    bs = np.array([0, 2, 4, 6], np.int32)
    F = O.bilu_factor(W.from_dense(A), bs, 0.0, agg_max=64)
    assert F.merges == 2 and list(F.bstart) == [0, 0, 0, 6]
    np.testing.assert_allclose(F.D_block(2), np.linalg.inv(A), rtol=0, atol=1e-13)
    # capped at 4 columns: only the first merge happens, and the operator is still A
    F4 = O.bilu_factor(W.from_dense(A), bs, 0.0, agg_max=4)
    assert F4.merges == 1 and list(F4.bstart) == [0, 0, 4, 6]
    np.testing.assert_allclose(F4.dense_L() @ F4.dense_Ubreve(), A, rtol=0, atol=1e-13)


# ----------------------------------------------------------------- identity and pattern

def _cases():
    w2 = W.cd2d_32()
    yield "cd2d_32 scalar blocks", w2.A, np.arange(w2.A.n + 1, dtype=np.int32)
    w3 = W.cd3d(side=10, seed=1, block=4)
    yield "cd3d 10^3 scalar blocks", w3.A, np.arange(w3.A.n + 1, dtype=np.int32)
    we = W.elasticity3d(side=6, seed=2, block=24)
    yield "elasticity 6^3 node blocks", we.A, np.arange(0, we.A.n + 1, 3, dtype=np.int32)
    yield "elasticity 6^3 ILU(1,tau) blocks", we.A, O.partition_ilu1t(we.A, 1e-2, 64)


@pytest.mark.parametrize("case", list(range(4)))
def test_aggregated_factor_has_the_same_product(case):
    name, A, bs = list(_cases())[case]
    F0 = O.bilu_factor(A, bs, 1e-2)
    F1 = O.bilu_factor(A, bs, 1e-2, agg_max=64)
    assert F1.merges > 0, name
    sz = np.diff(F1.bstart)
    assert sz.min() >= 0 and sz.max() <= 64 and F1.bstart[-1] == A.n
    assert int((sz == 0).sum()) == F1.merges
    M0 = F0.dense_L() @ F0.dense_Ubreve()
    M1 = F1.dense_L() @ F1.dense_Ubreve()
    assert np.abs(M1 - M0).max() <= 1e-12 * np.abs(M0).max(), name
    for K in range(F1.nb):
        b = F1.bsize(K)
        if b == 0:  # a void block stores nothing
            assert F1.Lptr[K + 1] == F1.Lptr[K] and F1.Uptr[K + 1] == F1.Uptr[K]
            continue
        np.testing.assert_allclose(F1.D_block(K) @ F1.P_block(K), np.eye(b), rtol=0, atol=1e-11)
    r = np.random.default_rng(0).standard_normal(A.n)
    z0, z1 = O.bilu_apply(F0, r), O.bilu_apply(F1, r)
    assert np.abs(z1 - z0).max() <= 1e-11 * np.abs(z0).max(), name


@pytest.mark.parametrize("case", list(range(4)))
def test_merged_blocks_store_the_union_of_their_members(case):
    """The rows (columns) of a merged block are those of its members beyond the merged
    block, read off the factor computed without aggregation; and replaying the merge test
    on those patterns, block after block, gives the same boundaries."""
    name, A, bs = list(_cases())[case]
    F0 = O.bilu_factor(A, bs, 1e-2)
    F1 = O.bilu_factor(A, bs, 1e-2, agg_max=64)
    nb = len(bs) - 1
    rows0 = [set(F0.L_block(K)[0].tolist()) for K in range(nb)]
    cols0 = [set(F0.U_block(K)[0].tolist()) for K in range(nb)]
    for K in range(nb):
        a, e = int(F1.bstart[K]), int(F1.bstart[K + 1])
        if a == e:
            continue
        members = [J for J in range(nb) if bs[J] >= a and bs[J + 1] <= e]
        assert bs[members[0]] == a and bs[members[-1] + 1] == e
        want_r = set().union(*(rows0[J] for J in members))
        want_c = set().union(*(cols0[J] for J in members))
        assert set(F1.L_block(K)[0].tolist()) == {i for i in want_r if i >= e}, (name, K)
        assert set(F1.U_block(K)[0].tolist()) == {j for j in want_c if j >= e}, (name, K)
    # replay: a group [a, e) with patterns R (rows >= e), C; block K = [s0, s1) joins it when
    # the test holds on the counts of Sec. 3.5
    bounds = [0]
    a, R, C = int(bs[0]), rows0[0], cols0[0]
    for K in range(1, nb):
        s0, s1 = int(bs[K]), int(bs[K + 1])
        p, q = s0 - a, s1 - s0
        r = sum(1 for i in R if i < s1)
        rp = sum(1 for j in C if j < s1)
        Rb, Cb = {i for i in R if i >= s1}, {j for j in C if j >= s1}
        t, tp = len(rows0[K]), len(cols0[K])
        u, v = len(Rb | rows0[K]), len(Cb | cols0[K])
        if p + q <= 64 and O.agg_rule(p, q, r, len(Rb), rp, len(Cb), t, tp, u, v):
            R, C = Rb | rows0[K], Cb | cols0[K]
        else:
            bounds.append(s0)
            a, R, C = s0, rows0[K], cols0[K]
    bounds.append(A.n)
    got = sorted(set(F1.bstart.tolist()))
    assert got == bounds, name


def test_cap_of_one_block_size_changes_nothing():
    """agg_max below every pair's size: no merge, the factor bit for bit as without."""
    w = W.cd2d_32()
    bs = np.arange(0, w.A.n + 1, 2, dtype=np.int32)
    F0 = O.bilu_factor(w.A, bs, 1e-2)
    F1 = O.bilu_factor(w.A, bs, 1e-2, agg_max=3)
    assert F1.merges == 0
    for k in ("bstart", "Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(F0, k), getattr(F1, k)), k


def test_gmres_iterations_unchanged_by_aggregation():
    """The preconditioner is the same operator, so GMRES(30) takes the same steps."""
    w = W.cd2d_32()
    bs = np.arange(w.A.n + 1, dtype=np.int32)
    F0 = O.bilu_factor(w.A, bs, 1e-2)
    F1 = O.bilu_factor(w.A, bs, 1e-2, agg_max=64)
    g0 = O.gmres(w.A, F0, w.b, tol=1e-8, restart=30, maxit=2000)
    g1 = O.gmres(w.A, F1, w.b, tol=1e-8, restart=30, maxit=2000)
    assert g0.iters == g1.iters
