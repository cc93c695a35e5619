"""Pins of the oracle's ILU(1,tau) block-pattern guess (Sec. 3.4) on hand-derived cases.

Growth rule (Sec. 3.4): a block [k, k+l) with r rows below it and s columns right of it
stores f_l = (r + s + l) l entries against a scalar count that grows by |I~| + |J~| + 1 per
column; column k+l joins while f_{l+1} <= (4/3) s_{l+1} or f_{l+1} <= s_{l+1} + 4 (l+1).
The expected partitions below were worked out by hand from that rule.
"""
import numpy as np

import oracle as O
from paper_1908_10169_gb300 import workloads as W


def test_diagonal_matrix_blocks_of_five():
    """Diagonal: r = s = 0, f = l^2, s_l = l.  l = 5: 25 <= 5 + 4*5 holds (equality);
    l = 6: 36 > 6 + 24 and 36 > 8, so blocks have 5 columns."""
    A = W.from_dense(np.eye(12) * 3.0)
    assert list(O.partition_ilu1t(A, 1e-2, 64)) == [0, 5, 10, 12]


def test_max_block_caps_growth():
    A = W.from_dense(np.eye(12) * 3.0)
    assert list(O.partition_ilu1t(A, 1e-2, 3)) == [0, 3, 6, 9, 12]
    assert list(O.partition_ilu1t(A, 1e-2, 1)) == list(range(13))


def test_tridiagonal_blocks_of_five():
    """diag 4, off -1, tau 0.1: I~_k = J~_k = {k+1} (no fill: column k-1 has no row > k).
    s_1 = 3; adding columns gives (f, s) = (8, 6) [8 <= 4/3*6], (15, 9), (24, 12), (35, 15)
    [35 <= 15 + 20], then (48, 18) is rejected.  The last block [10, 12): (4, 4) accepted."""
    n = 12
    Ad = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    assert list(O.partition_ilu1t(W.from_dense(Ad), 0.1, 64)) == [0, 5, 10, 12]


def test_four_thirds_branch():
    """Column 0 has rows 10..39, column 1 rows 14..43 (entries 1, diagonal 100), tau 1e-3.
    Adding column 1: r = 34, f = 36*2 = 72, s = 31 + 31 = 62: 72 > 62 + 8 but 3*72 <= 4*62,
    so only the 4/3 branch accepts.  Column 2: f = 37*3 = 111 > 63 + 12 and > 84: rejected.
    The rest is diagonal: blocks of five."""
    n = 50
    Ad = 100.0 * np.eye(n)
    Ad[10:40, 0] = 1.0
    Ad[14:44, 1] = 1.0
    bs = O.partition_ilu1t(W.from_dense(Ad), 1e-3, 64)
    assert list(bs) == [0, 2, 7, 12, 17, 22, 27, 32, 37, 42, 47, 50]
    # the rule is symmetric in rows and columns
    assert list(O.partition_ilu1t(W.from_dense(Ad.T.copy()), 1e-3, 64)) == list(bs)


def test_threshold_is_inclusive():
    """Sec. 3.4 keeps an entry with |a_ik| >= tau |a_kk|: the case above with diagonal 64,
    entries 1 and tau = 1/64 (tau |a_kk| = 1 exactly) gives the same blocks; a tau one ulp
    larger drops the entries and leaves the diagonal's blocks of five."""
    n = 50
    Ad = 64.0 * np.eye(n)
    Ad[10:40, 0] = 1.0
    Ad[14:44, 1] = 1.0
    A = W.from_dense(Ad)
    assert list(O.partition_ilu1t(A, 1.0 / 64, 64)) == [0, 2, 7, 12, 17, 22, 27, 32, 37, 42, 47, 50]
    assert list(O.partition_ilu1t(A, np.nextafter(1.0 / 64, 1.0), 64)) == list(range(0, 51, 5))


def test_fill_from_original_entries():
    """a_01 = 1 and column 0 has rows 10..17: column 1 gets the fill rows 10..17 because
    |a_i0 a_01| >= tau |a_00 a_11|.  With them: r = 8, f = 20 <= s + 8 = 19 + 8, accepted;
    without the fill rule s would be 11 and f = 20 > 19: rejected.  tau = 2 drops everything."""
    n = 20
    Ad = np.eye(n)
    Ad[0, 1] = 1.0
    Ad[10:18, 0] = 1.0
    A = W.from_dense(Ad)
    assert list(O.partition_ilu1t(A, 0.5, 64)) == [0, 2, 7, 12, 17, 20]
    assert list(O.partition_ilu1t(W.from_dense(Ad.T.copy()), 0.5, 64)) == [0, 2, 7, 12, 17, 20]
    assert list(O.partition_ilu1t(A, 2.0, 64)) == [0, 5, 10, 15, 20]


def test_dense_matrix_is_one_block():
    """Dense: f_l equals the scalar count for every l, no wasted zeros, one block."""
    Ad = np.random.default_rng(0).uniform(1.0, 2.0, size=(6, 6)) + 6 * np.eye(6)
    assert list(O.partition_ilu1t(W.from_dense(Ad), 0.0, 64)) == [0, 6]


def test_partition_covers_and_respects_cap_on_stencil():
    A = W.convdiff_upwind((12, 12, 12), seed=1)
    bs = O.partition_ilu1t(A, 1e-2, 8)
    assert bs[0] == 0 and bs[-1] == A.n
    assert np.all(np.diff(bs) >= 1) and np.all(np.diff(bs) <= 8)
    fx = O.partition_fixed(A.n, 100)
    assert list(fx[:3]) == [0, 100, 200] and fx[-1] == A.n


# ----------------------------------------------------------------- growth over groups of columns

def test_groups_of_one_are_the_column_rule():
    A = W.convdiff_upwind((8, 8, 8), seed=2)
    for tau, mb in ((1e-2, 64), (1e-3, 16), (0.0, 7)):
        assert list(O.partition_ilu1t_groups(A, tau, mb, np.arange(A.n + 1))) == list(O.partition_ilu1t(A, tau, mb))


def test_diagonal_groups_of_two_and_three():
    """Diagonal, groups of 2 (every column adds 1 to the scalar count, r = s' = 0): the block
    [0, 2) starts with s = 2; adding [2, 4): l = 4, f = 16, s = 4: 48 > 16 but 16 <= 4 + 4*4,
    accepted; adding [4, 6): l = 6, f = 36, s = 6: 36 > 6 + 24, rejected.  Blocks of 4.
    Groups of 3: a second group gives l = 6, f = 36 > 6 + 24: blocks of 3 (the column rule
    makes blocks of 5)."""
    A = W.from_dense(np.eye(12) * 3.0)
    assert list(O.partition_ilu1t_groups(A, 1e-2, 64, np.arange(0, 13, 2))) == [0, 4, 8, 12]
    assert list(O.partition_ilu1t_groups(A, 1e-2, 64, np.arange(0, 13, 3))) == [0, 3, 6, 9, 12]
    # max_block caps whole groups: groups of 2 under max_block 3 never merge
    assert list(O.partition_ilu1t_groups(A, 1e-2, 3, np.arange(0, 13, 2))) == list(range(0, 13, 2))


def test_group_counts_exclude_the_candidate_group():
    """Tridiagonal (diag 4, off -1, tau 0.1), groups of 2.  Column k has I~ = J~ = {k+1}, so a
    group [e, e+2) inside the matrix contributes the scalar count 2 (1 + 1 + 1) = 6 and one row and one
    column at or after its end.  First block [0, 2): R = {1, 2}, C = {1, 2}, s = 6.  Adding
    [2, 4): rows at or after 4: {4} (from column 3), columns {4}: r = s' = 1, l = 4,
    f = (1 + 1 + 4) 4 = 24, s = 12: 72 > 48, 24 <= 12 + 16, accepted.  Adding [4, 6): r = s' = 1,
    l = 6, f = 48, s = 18: 144 > 72, 48 > 18 + 24, rejected.  Blocks of 4; the last group
    [10, 12) adds s = 3 + 1 (column 11 has no neighbour after it) and nothing at or after 12:
    f = 16 <= 10 + 16, so [8, 12) is one block."""
    n = 12
    Ad = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    assert list(O.partition_ilu1t_groups(W.from_dense(Ad), 0.1, 64, np.arange(0, 13, 2))) == [0, 4, 8, 12]


def test_rows_inside_the_candidate_group_do_not_count():
    """Diagonal 4 plus a_43 = -1, tau = 0.1, groups [0, 3) and [3, 5).  Column 3 has
    I~ = {4}, every other set is empty.  Block [0, 3): s = 3.  Adding [3, 5): the row 4 lies
    inside the candidate group, so r = s' = 0, l = 5, f = 25, s = 3 + 2 + 1 = 6: 75 > 24 but
    25 <= 6 + 20, accepted: one block (counting row 4 would give f = 30 > 26)."""
    d = 4 * np.eye(5)
    d[4, 3] = -1.0
    assert list(O.partition_ilu1t_groups(W.from_dense(d), 0.1, 64, [0, 3, 5])) == [0, 5]


def test_blocks_are_unions_of_groups():
    w = W.elasticity3d(side=4, seed=2, block=63)
    groups = np.arange(0, w.A.n + 1, 3)
    bs = O.partition_ilu1t_groups(w.A, 1e-2, 64, groups)
    assert set(bs) <= set(groups) and np.diff(bs).max() <= 63 and bs[-1] == w.A.n


def test_group_arguments_are_checked():
    A = W.from_dense(np.eye(6) * 3.0)
    for groups in ([0, 3, 5], [1, 6], [0, 3, 3, 6], [0, 6]):
        mb = 4 if groups == [0, 6] else 64
        try:
            O.partition_ilu1t_groups(A, 1e-2, mb, groups)
        except ValueError:
            continue
        raise AssertionError(f"groups {groups} accepted")
