"""Plain reference of the block nested-dissection reordering (Sec. 3.3) and of the block
elimination tree, small problems only.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the test suite may use it; the
product never imports it.

Sec. 3.3 compresses every diagonal block of A into one node (the companion matrix B: K and L
are adjacent when an entry of A couples B_K and B_L), reorders B by nested dissection and
expands the node permutation into a block permutation P that keeps the blocks intact:
A' = P^T A P.  The paper uses METIS for the dissection; this reference uses George's
level-structure dissection (readings N1-N4):

  N1  the graph of B is symmetrised (K ~ L when A couples the blocks in either direction);
  N2  a connected part of more than `leaf` nodes is split by a breadth-first level structure
      rooted at a pseudo-peripheral node (George-Liu: start at the part's smallest node,
      move to a node of least degree, ties by index, in the last level while the number of
      levels grows); the separator is the middle level (index L // 2 of L levels), the
      first part the levels before it, the second part the levels after it; a part of at
      most `leaf` nodes, or with fewer than 3 levels, keeps its increasing order;
  N3  the order of a part is: its first part, its second part (each dissected in turn, their
      connected components one after another by smallest node), then its separator in
      increasing node order;
  N4  a disconnected set is ordered component by component, by smallest node.

The block elimination tree of the reordered matrix is the elimination tree of its symmetrised
block graph: eliminating blocks in order, each block joins its later neighbours into a clique
(fill), and its parent is its first later neighbour at that time.  Every block J that updates a
block K in the factorization (a kept L row or U column of J inside B_K) is a descendant of K.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def block_graph(A, bstart):
    """Adjacency sets of the symmetrised companion graph (reading N1)."""
    bs = np.asarray(bstart, dtype=np.int64)
    nb = len(bs) - 1
    blk = np.zeros(A.n, dtype=np.int64)
    for K in range(nb):
        blk[bs[K]:bs[K + 1]] = K
    adj = [set() for _ in range(nb)]
    for i in range(A.n):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            K, L = int(blk[i]), int(blk[A.colind[e]])
            if K != L:
                adj[K].add(L)
                adj[L].add(K)
    return adj


def _levels(adj, nodes, root):
    """Breadth-first level structure of the induced subgraph on `nodes` from `root`."""
    seen = {root}
    levels = [[root]]
    while True:
        nxt = sorted({w for v in levels[-1] for w in adj[v] if w in nodes and w not in seen})
        if not nxt:
            return levels
        seen.update(nxt)
        levels.append(nxt)


def _components(adj, nodes):
    left = set(nodes)
    comps = []
    while left:
        start = min(left)
        comp = {start}
        q = deque([start])
        while q:
            v = q.popleft()
            for w in adj[v]:
                if w in left and w not in comp:
                    comp.add(w)
                    q.append(w)
        left -= comp
        comps.append(comp)
    return comps


def _pseudo_peripheral(adj, nodes):
    deg = lambda v: sum(1 for w in adj[v] if w in nodes)
    root = min(nodes)
    levels = _levels(adj, nodes, root)
    while True:
        cand = min(levels[-1], key=lambda v: (deg(v), v))
        lv = _levels(adj, nodes, cand)
        if len(lv) <= len(levels):
            return root, levels
        root, levels = cand, lv


def dissect(adj, nodes, leaf=1):
    """The order of `nodes` (readings N2-N4)."""
    order = []
    for comp in _components(adj, nodes):
        if len(comp) <= leaf:
            order += sorted(comp)
            continue
        root, levels = _pseudo_peripheral(adj, comp)
        if len(levels) < 3:
            order += sorted(comp)
            continue
        m = len(levels) // 2
        first = {v for lv in levels[:m] for v in lv}
        second = {v for lv in levels[m + 1:] for v in lv}
        order += dissect(adj, first, leaf) + dissect(adj, second, leaf) + sorted(levels[m])
    return order


def nd_order(A, bstart, leaf=1):
    """(perm, new_bstart, block_order): the node order of the dissection, expanded to the
    unknowns (perm[k] = original index at position k, blocks kept whole) and the block starts
    of P^T A P."""
    bs = np.asarray(bstart, dtype=np.int64)
    adj = block_graph(A, bs)
    order = dissect(adj, set(range(len(bs) - 1)), leaf)
    perm, nbs = [], [0]
    for K in order:
        perm.extend(range(int(bs[K]), int(bs[K + 1])))
        nbs.append(len(perm))
    return np.array(perm, dtype=np.int32), np.array(nbs, dtype=np.int32), np.array(order, dtype=np.int32)


def block_etree(A, bstart):
    """Parent of every block in the elimination tree of the symmetrised block graph (-1 for
    a root), by simulating the block elimination with fill."""
    adj = block_graph(A, bstart)
    nb = len(adj)
    later = [set(w for w in adj[K] if w > K) for K in range(nb)]
    parent = [-1] * nb
    for K in range(nb):
        if later[K]:
            p = min(later[K])
            parent[K] = p
            # eliminating K joins its later neighbours into a clique: all of them become
            # neighbours of the first one (the others follow when p is eliminated)
            later[p] |= later[K] - {p}
    return np.array(parent, dtype=np.int32)
