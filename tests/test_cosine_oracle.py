"""Pins of the cosine-blocking oracle (Sec. 3.2) against hand-derived cases, closed forms and
structure that the method must recover: not against a retyped copy of it."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cosine_oracle as C
from paper_1908_10169_gb300 import workloads as W


def from_pattern(rows, n):
    """CSR with the given column sets per row (values: 1 off the diagonal, 4 on it)."""
    d = np.zeros((n, n))
    for i, cols in enumerate(rows):
        for j in cols:
            d[i, j] = 4.0 if i == j else 1.0
    return W.from_dense(d, keep_zeros_on_diag=False)


def permuted(A, perm):
    """Q^T A Q through scipy (row and column selection)."""
    M = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))[perm][:, perm].tocsr()
    M.sort_indices()
    return W.CSR(A.n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


def blocks_as_sets(perm, bstart):
    return [frozenset(int(v) for v in perm[bstart[k]:bstart[k + 1]]) for k in range(len(bstart) - 1)]


# patterns of the hand example: rows 0, 3, 5 share {0, 3, 5}; rows 1, 2, 4 overlap in part
HAND = [{0, 3, 5}, {1, 2}, {1, 2, 4}, {0, 3, 5}, {2, 4}, {0, 3, 5}]


@pytest.mark.parametrize("tau,max_block,perm,bstart", [
    # leader 0: partners {3, 5}, |c_0 n c_3|^2 = 9 >= 0.8 * 3 * 3 (both join); leader 1:
    # partners {2, 4}, 2^2 = 4 < 0.8 * 2 * 3 = 4.8 and 1 < 0.8 * 2 * 2; leader 2: partner 4,
    # 4 < 0.8 * 3 * 2; leader 4 alone.  No count exceeds mu + 2 sigma (mu = 8/3).
    (0.8, 64, [0, 3, 5, 1, 2, 4], [0, 3, 4, 5, 6]),
    # tau = 0.6: 4 >= 0.6 * 2 * 3 = 3.6, so 2 joins 1; 1 < 0.6 * 4 keeps 4 out
    (0.6, 64, [0, 3, 5, 1, 2, 4], [0, 3, 5, 6]),
    # max_block = 2: 0 takes 3 only; 5 leads its own block at the end
    (0.8, 2, [0, 3, 1, 2, 4, 5], [0, 2, 3, 4, 5, 6]),
    # tau = 1: only identical patterns pass, at equality (9 >= 1 * 3 * 3)
    (1.0, 64, [0, 3, 5, 1, 2, 4], [0, 3, 4, 5, 6]),
])
def test_hand_example(tau, max_block, perm, bstart):
    A = from_pattern(HAND, 6)
    p, b = C.cosine_blocking(A, tau, max_block)
    assert list(p) == perm and list(b) == bstart


def test_nonsymmetric_pattern_uses_row_counts():
    """Rows 0 and 1 both hold {0, 1, 2}; rows 3, 4 add entries to column 1 (4 entries), so row
    and column counts differ.  Leader 0: |c_0 n c_1|^2 = 9 >= 0.8 * 3 * 3 (row counts) joins
    1; against column 1's count it would be 9 < 0.8 * 3 * 4.  Partners 2, 3, 4 share one
    column: 1 < 0.8 * 3 * 1, 1 < 0.8 * 3 * 2.  Leader 3: 1 < 0.8 * 2 * 2 leaves 4 alone.
    Counts: rows (3, 3, 1, 2, 2), columns (2, 4, 3, 1, 1), mu = 11/5; none exceeds its bound."""
    A = from_pattern([{0, 1, 2}, {0, 1, 2}, {2}, {1, 3}, {1, 4}], 5)
    assert not C.excluded(A).any()
    p, b = C.cosine_blocking(A, 0.8, 64)
    assert list(p) == [0, 1, 2, 3, 4] and list(b) == [0, 2, 3, 4, 5]


def test_tau_zero_closed_form():
    """tau = 0 accepts every partner: on a tridiagonal matrix the leader i takes i+1 and i+2
    (the rows sharing a column with row i), so the blocks are consecutive triples."""
    n = 10
    A = W.from_dense(4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    p, b = C.cosine_blocking(A, 0.0, 64)
    assert list(p) == list(range(n)) and list(b) == [0, 3, 6, 9, 10]
    # tau = 0.8 on the same matrix: neighbouring rows share 2 of 3 columns, 4 < 0.8 * 9
    p, b = C.cosine_blocking(A, 0.8, 64)
    assert list(b) == list(range(n + 1))


@pytest.mark.parametrize("d", [2, 3, 4])
def test_node_blocks_recovered_under_any_ordering(d):
    """A scalar 2D 5-point pattern with d unknowns per node (every unknown of a node has the
    node's pattern): whatever the symmetric ordering, the blocks are exactly the nodes.  Two
    neighbouring nodes share at most 2 of 5 (interior) node columns: (2d)^2 < 0.8 (5d)^2."""
    m = 7
    T = sp.diags([-1.0, 4.0, -1.0], [-1, 0, 1], shape=(m, m))
    S = (sp.kron(sp.eye(m), T) + sp.kron(sp.diags([-1.0, -1.0], [-1, 1], shape=(m, m)), sp.eye(m))).tocsr()
    K = sp.kron(S, np.ones((d, d)) + np.eye(d)).tocsr()
    K.sort_indices()
    A = W.CSR(K.shape[0], K.indptr.astype(np.int64), K.indices.astype(np.int32), K.data.astype(np.float64))
    rng = np.random.default_rng(d)
    for trial in range(3):
        perm = rng.permutation(A.n).astype(np.int32) if trial else np.arange(A.n, dtype=np.int32)
        Ap = permuted(A, perm)
        p, b = C.cosine_blocking(Ap, 0.8, 64)
        got = {frozenset(int(perm[v]) for v in s) for s in blocks_as_sets(p, b)}
        want = {frozenset(range(node * d, node * d + d)) for node in range(m * m)}
        assert got == want
        # each block is led by its smallest index in the permuted order
        assert all(p[b[k]] == min(p[b[k]:b[k + 1]]) for k in range(len(b) - 1))


def test_elasticity_nodes_recovered():
    """Q1 elasticity, 3 unknowns per node: the interior nodes (27 neighbours, 81 entries per
    row) exceed mu + 2 sigma on a 4^3 grid and stay single; every other node is one block of
    3 under a random ordering too."""
    w = W.elasticity3d(side=4, seed=2, block=63)
    A = w.A
    counts = np.diff(A.rowptr)
    rng = np.random.default_rng(9)
    perm = rng.permutation(A.n).astype(np.int32)
    p, b = C.cosine_blocking(permuted(A, perm), 0.8, 64)
    got = {frozenset(int(perm[v]) for v in s) for s in blocks_as_sets(p, b)}
    want = set()
    for node in range(A.n // 3):
        dofs = range(3 * node, 3 * node + 3)
        if counts[3 * node] == 81:
            want |= {frozenset([v]) for v in dofs}
        else:
            want.add(frozenset(dofs))
    assert got == want
    assert sum(len(s) == 1 for s in got) == 8 * 3


def test_dense_row_and_column_take_no_part():
    """Pairs of identical rows (a 1D pattern with 2 unknowns per node) plus one index whose
    row and column are full: that index is a block of its own, its partner too (the only
    row it could join is excluded), every other pair stays together."""
    m, d, x = 12, 2, 9
    S = sp.diags([1.0, 1.0, 1.0], [-1, 0, 1], shape=(m, m))
    K = sp.kron(S, np.ones((d, d))).tolil()
    K[x, :] = 1.0
    K[:, x] = 1.0
    K = K.tocsr()
    K.sort_indices()
    A = W.CSR(K.shape[0], K.indptr.astype(np.int64), K.indices.astype(np.int32), K.data.astype(np.float64))
    ex = C.excluded(A)
    assert list(np.nonzero(ex)[0]) == [x]
    p, b = C.cosine_blocking(A, 0.8, 64)
    sets = blocks_as_sets(p, b)
    assert frozenset([x]) in sets and frozenset([x - 1]) in sets
    for node in range(m):
        if node != x // d:
            assert frozenset([2 * node, 2 * node + 1]) in sets


def test_dense_column_alone_excludes():
    """A full column (not row) at index x: its column count is far above mu + 2 sigma_c, so x
    is a block of its own although its row is ordinary."""
    m, d, x = 12, 2, 9
    S = sp.diags([1.0, 1.0, 1.0], [-1, 0, 1], shape=(m, m))
    K = sp.kron(S, np.ones((d, d))).tolil()
    K[:, x] = 1.0
    K = K.tocsr()
    K.sort_indices()
    A = W.CSR(K.shape[0], K.indptr.astype(np.int64), K.indices.astype(np.int32), K.data.astype(np.float64))
    assert list(np.nonzero(C.excluded(A))[0]) == [x]
    p, b = C.cosine_blocking(A, 0.8, 64)
    assert frozenset([x]) in blocks_as_sets(p, b)


@pytest.mark.parametrize("n,excluded", [(5, False), (6, True)])
def test_exclusion_threshold_is_exact(n, excluded):
    """A diagonal matrix whose last row is full: row counts (1, ..., 1, n).  For n = 5,
    mu = 9/5 and sigma = 2 (c - 1) / 5 = 8/5, so mu + 2 sigma = 5 = c exactly: not above the
    bound, nothing excluded.  For n = 6, mu = 11/6, sigma = sqrt(5) 5 / 6, mu + 2 sigma = 5.56
    < 6: the full row's index is excluded.  (The column counts, 2 or 1, stay below their
    bound.)"""
    d = np.eye(n) * 4.0
    d[n - 1, :] = 1.0
    d[n - 1, n - 1] = 4.0
    A = W.from_dense(d)
    ex = C.excluded(A)
    assert list(np.nonzero(ex)[0]) == ([n - 1] if excluded else [])


# ------------------------------------------------------------ the compressed (unit) form


def _pattern(rows, n):
    import numpy as np
    from paper_1908_10169_gb300 import workloads as W
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    ci = np.array([c for r in rows for c in sorted(r)], dtype=np.int32)
    return W.CSR(n, rp, ci, np.ones(ci.size))


def test_units_of_one_index_give_the_plain_blocking():
    import numpy as np
    from oracle import cosine_oracle as C
    from paper_1908_10169_gb300 import workloads as W
    w = W.cd3d(side=6, seed=2, block=6)
    for mb in (3, 8, 64):
        p1, b1 = C.cosine_blocking(w.A, 0.5, mb)
        p2, b2 = C.cosine_blocking_units(w.A, np.arange(w.A.n + 1), 0.5, mb)
        assert np.array_equal(p1, p2) and np.array_equal(b1, b2)


def test_units_hand_example():
    """Units {0,1}, {2,3}, {4,5}; rows 0: {0,4}, 1: {1}, 2: {2}, 3: {3}, 4: {1,4}, 5: {5}.  The
    compressed rows are u0: {u0, u2}, u1: {u1}, u2: {u0, u2}; no count is above mu + 2 sigma
    (n S - nnz^2 = 27 - 25); u0 and u2 pass (2^2 >= 0.8 * 2 * 2) and hold 4 indices: blocks
    {0, 1, 4, 5}, {2, 3}.  With at most 3 indices per block the two units do not fit together."""
    from oracle import cosine_oracle as C
    A = _pattern([{0, 4}, {1}, {2}, {3}, {1, 4}, {5}], 6)
    perm, bstart = C.cosine_blocking_units(A, [0, 2, 4, 6], 0.8, 64)
    assert perm.tolist() == [0, 1, 4, 5, 2, 3] and bstart.tolist() == [0, 4, 6]
    perm, bstart = C.cosine_blocking_units(A, [0, 2, 4, 6], 0.8, 3)
    assert perm.tolist() == [0, 1, 2, 3, 4, 5] and bstart.tolist() == [0, 2, 4, 6]


def test_units_join_through_their_second_rows():
    """Units {0,1}, {2,3}; rows 0: {0}, 1: {3}, 2: {2}, 3: {1}: only the units' second rows
    couple them, so the compressed rows are u0: {u0, u1}, u1: {u0, u1} and the two units form
    one block."""
    from oracle import cosine_oracle as C
    A = _pattern([{0}, {3}, {2}, {1}], 4)
    perm, bstart = C.cosine_blocking_units(A, [0, 2, 4], 0.8, 64)
    assert perm.tolist() == [0, 1, 2, 3] and bstart.tolist() == [0, 4]
