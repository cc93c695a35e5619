"""Pins of the block nested-dissection oracle and the block elimination tree (Sec. 3.3): the
paper's own illustration, closed forms, and the factorization's actual update structure."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import nd_oracle as N
from paper_1908_10169_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pattern_matrix(rows):
    n = len(rows)
    d = np.zeros((n, n))
    for i, cols in enumerate(rows):
        for j in cols:
            d[i, j] = 4.0 if i == j else -1.0
    return W.from_dense(d, keep_zeros_on_diag=False)


def permuted(A, perm):
    M = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))[perm][:, perm].tocsr()
    M.sort_indices()
    return W.CSR(A.n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


def height(parent):
    h = [1] * len(parent)
    for K in range(len(parent)):
        if parent[K] >= 0:
            h[parent[K]] = max(h[parent[K]], h[K] + 1)
    return max(h) if h else 0


def test_paper_illustration():
    g = json.load(open(os.path.join(GOLDEN, "nd_illustration.json")))
    A = pattern_matrix(g["A_pattern"])
    adj = N.block_graph(A, g["bstart"])
    assert [sorted(adj[K] | {K}) for K in range(len(adj))] == g["B_pattern"]
    perm, nbs, order = N.nd_order(A, g["bstart"])
    assert list(order) == g["block_order"] and list(nbs) == [0, 2, 4, 6]
    Ap = permuted(A, perm)
    got = [list(Ap.colind[Ap.rowptr[i]:Ap.rowptr[i + 1]]) for i in range(Ap.n)]
    assert got == g["PtAP_pattern"]


def test_path_of_seven_is_a_binary_tree():
    """A path 0 - 1 - ... - 6 (one unknown per block): the level structure from node 0 has 7
    levels, the separator is node 3, then 1 and 5: order 0 2 1 4 6 5 3, and the elimination tree
    is a perfect binary tree of height 3."""
    n = 7
    A = W.from_dense(4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    perm, nbs, order = N.nd_order(A, np.arange(n + 1))
    assert list(order) == [0, 2, 1, 4, 6, 5, 3]
    par = N.block_etree(permuted(A, perm), np.arange(n + 1))
    assert list(par) == [2, 2, 6, 5, 5, 6, -1] and height(par) == 3
    # natural order: a chain
    assert height(N.block_etree(A, np.arange(n + 1))) == n


def test_one_sided_coupling_is_symmetrised():
    """A lower bidiagonal pattern (a_{i,i-1} only) couples neighbours in one direction; its
    companion graph is the path, ordered and treed like the path of seven above."""
    n = 7
    A = W.from_dense(4 * np.eye(n) - np.eye(n, k=-1))
    perm, nbs, order = N.nd_order(A, np.arange(n + 1))
    assert list(order) == [0, 2, 1, 4, 6, 5, 3]
    assert list(N.block_etree(A, np.arange(n + 1))) == [1, 2, 3, 4, 5, 6, -1]


def test_root_moves_to_a_pseudo_peripheral_node():
    """The path 5 - 3 - 1 - 0 - 2 - 4 - 6 (node 0 in the middle).  From node 0 the level
    structure has 4 levels; its last level {5, 6} gives node 5 (degree 1, smaller index) with 7
    levels, and node 6 gives no more: root 5.  Separator: level 3 = {0}; first part
    {5, 3, 1} (a path rooted at 1: separator 3), second part {2, 4, 6} (separator 4).
    Order: 1 5 3, 2 6 4, 0."""
    chain = [5, 3, 1, 0, 2, 4, 6]
    rows = [{v} for v in range(7)]
    for a, b in zip(chain, chain[1:]):
        rows[a].add(b)
        rows[b].add(a)
    A = pattern_matrix(rows)
    perm, nbs, order = N.nd_order(A, np.arange(8))
    assert list(order) == [1, 5, 3, 2, 6, 4, 0]


def test_blocks_stay_whole_and_order_is_a_permutation():
    A = W.convdiff_upwind((6, 6, 6), seed=1)
    bs = np.arange(0, A.n + 1, 6)
    perm, nbs, order = N.nd_order(A, bs)
    assert sorted(perm) == list(range(A.n)) and sorted(order) == list(range(len(bs) - 1))
    for k, K in enumerate(order):
        assert list(perm[nbs[k]:nbs[k + 1]]) == list(range(bs[K], bs[K + 1]))


def test_top_separator_disconnects_the_two_parts():
    """On a 2D grid of line blocks (a 9 x 9 grid graph of blocks) the last-ordered nodes of
    the top level form a separator: removing them leaves no edge between the nodes ordered
    before and after the first part's end."""
    A = W.convdiff_upwind((5, 9, 9), seed=1)
    bs = np.arange(0, A.n + 1, 5)
    adj = N.block_graph(A, bs)
    nodes = set(range(len(adj)))
    root, levels = N._pseudo_peripheral(adj, nodes)
    m = len(levels) // 2
    first = {v for lv in levels[:m] for v in lv}
    second = {v for lv in levels[m + 1:] for v in lv}
    assert first and second
    assert not any(w in second for v in first for w in adj[v])
    order = N.dissect(adj, nodes)
    assert set(order[-len(levels[m]):]) == set(levels[m])
    assert set(order[:len(first)]) == first


@pytest.mark.parametrize("case", ["natural", "nd", "random_blocks"])
@pytest.mark.parametrize("tau", [0.0, 1e-2])
def test_every_producer_is_a_descendant(case, tau):
    """The factorization's actual updates (J has a kept L row or U column inside B_K) only
    come from descendants of K in the block elimination tree; with tau = 0 the parent of J is
    exactly the first block J updates."""
    A = W.convdiff_upwind((4, 6, 6), seed=3)
    bs = np.arange(0, A.n + 1, 4)
    nb = len(bs) - 1
    if case == "nd":
        perm, bs2, _ = N.nd_order(A, bs)
    elif case == "random_blocks":
        order = np.random.default_rng(2).permutation(nb)
        perm = np.concatenate([np.arange(bs[K], bs[K + 1]) for K in order]).astype(np.int32)
        bs2 = bs
    else:
        perm, bs2 = np.arange(A.n, dtype=np.int32), bs
    Ap = permuted(A, perm)
    par = N.block_etree(Ap, bs2)
    F = O.bilu_factor(Ap, bs2, tau)
    blk = np.repeat(np.arange(nb), np.diff(bs2))

    def ancestors(J):
        out, p = set(), par[J]
        while p >= 0:
            out.add(int(p))
            p = par[p]
        return out

    for J in range(nb):
        rows, _ = F.L_block(J)
        cols, _ = F.U_block(J)
        targets = set(int(blk[i]) for i in rows) | set(int(blk[j]) for j in cols)
        assert targets <= ancestors(J), (J, targets - ancestors(J))
        if tau == 0.0 and targets:
            assert par[J] == min(targets)
