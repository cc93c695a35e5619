"""Plain reference of the cosine-based blocking (Sec. 3.2): a symmetric permutation that groups
rows (and the columns of the same index) with nearly the same nonzero pattern.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the test suite may use it; the
product never imports it.

The paper's test: rows i and j belong together when their 0/1 pattern vectors c_i, c_j satisfy
c_i^T c_j ~ ||c_i|| ||c_j||, checked by integer counting as

    nz(a_i n a_j)^2 >= tau * nz(a_i) * nz(a_j),        tau = 0.8 by default,

over the pattern of the upper triangular part of A A^T (pairs j > i that share a column),
among indices not yet placed in a block.  Rows or columns with more than mu + 2 sigma_{r,c}
nonzeros (mu the mean count per row/column, sigma_r, sigma_c the standard deviations of the
row and column counts) take no part.  Q groups the blocks together; A~ = Q^T A Q.

Readings (where the paper leaves details open):
  C1  the pattern of a row is its stored entries (explicit zeros included);
  C2  rows are visited in increasing index; an index not yet in a block leads a new block and
      collects, in increasing index order, every unplaced partner j > i (sharing a column)
      that passes the test against the leader, until the block holds max_block indices;
  C3  an index is excluded when its row count exceeds mu + 2 sigma_r or its column count
      exceeds mu + 2 sigma_c (mu = nnz / n, population standard deviations); an excluded
      index is a block of its own at its place in the sweep and joins no other block.  The
      comparison is decided exactly in integers: count > mu + 2 sigma iff n count > nnz and
      (n count - nnz)^2 > 4 (n S - nnz^2), S the sum of the squared counts;
  C4  the test is evaluated in float64 as float(cnt)**2 >= (tau * nz_i) * nz_j;
  C5  Q lists the blocks in the order of their leaders, each block as leader then members in
      increasing index: perm[k] = original index at position k, A~[k, l] = A[perm[k], perm[l]].
"""
from __future__ import annotations

import numpy as np


def _row_sets(A):
    rp, ci = A.rowptr, A.colind
    return [set(int(c) for c in ci[rp[i]:rp[i + 1]]) for i in range(A.n)]


def _above_two_sigma(counts, nnz):
    """count > mu + 2 sigma for every count, in exact integer arithmetic (reading C3)."""
    n = len(counts)
    S = sum(c * c for c in counts)
    var4 = 4 * (n * S - nnz * nnz)  # 4 n^2 sigma^2
    out = []
    for c in counts:
        d = n * c - nnz            # n (count - mu)
        out.append(d > 0 and d * d > var4)
    return out


def excluded(A) -> np.ndarray:
    """Reading C3: indices whose row or column count exceeds mu + 2 sigma."""
    n = A.n
    nnz = int(A.rowptr[-1]) if n else 0
    rcount = [int(A.rowptr[i + 1] - A.rowptr[i]) for i in range(n)]
    ccount = [0] * n
    for c in A.colind:
        ccount[int(c)] += 1
    r, c = _above_two_sigma(rcount, nnz), _above_two_sigma(ccount, nnz)
    return np.array([a or b for a, b in zip(r, c)], dtype=bool)


def cosine_blocking(A, tau: float = 0.8, max_block: int = 64, weights=None):
    """Returns (perm, bstart): the permutation Q as the original index of every new position
    and the block starts of A~ = Q^T A Q (Sec. 3.2, readings C1-C5).  With weights (the sizes
    of the compressed units, see cosine_blocking_units) a block holds at most max_block of
    weight: a partner that passes the test but does not fit is passed over."""
    n = A.n
    w = [1] * n if weights is None else [int(x) for x in weights]
    rows = _row_sets(A)
    # rows having an entry in column k (the pattern of A A^T is reached through them)
    cols = [[] for _ in range(n)]
    for i in range(n):
        for k in sorted(rows[i]):
            cols[k].append(i)
    skip = excluded(A)
    placed = [False] * n
    perm, bstart = [], [0]
    for i in range(n):
        if placed[i]:
            continue
        placed[i] = True
        block = [i]
        bw = w[i]
        if not skip[i]:
            partners = sorted({j for k in rows[i] for j in cols[k] if j > i})
            for j in partners:
                if bw >= max_block:
                    break
                if placed[j] or skip[j] or bw + w[j] > max_block:
                    continue
                cnt = len(rows[i] & rows[j])
                if float(cnt) ** 2 >= (tau * len(rows[i])) * len(rows[j]):
                    block.append(j)
                    bw += w[j]
                    placed[j] = True
        perm.extend(block)
        bstart.append(len(perm))
    return np.array(perm, dtype=np.int32), np.array(bstart, dtype=np.int32)


def cosine_blocking_units(A, ustart, tau: float = 0.8, max_block: int = 64):
    """Cosine blocking of the compressed matrix (Sec. 4.2: after the symmetrised matching the
    2 x 2 pivots are merged before the cosine test; reading R27).  The consecutive units
    [ustart[p], ustart[p + 1]) of A are the indices of the compressed matrix, whose row p holds
    the units of the columns of A's rows in unit p; cosine_blocking runs on it with the unit
    sizes as weights (a block holds at most max_block indices of A), and the result is
    expanded: the units of a block in its order, the indices of a unit in theirs.  Returns
    (perm, bstart) over the indices of A."""
    ustart = [int(x) for x in ustart]
    nu = len(ustart) - 1
    unit_of = [0] * A.n
    for p in range(nu):
        for i in range(ustart[p], ustart[p + 1]):
            unit_of[i] = p
    rowptr, colind = [0], []
    for p in range(nu):
        cols = sorted({unit_of[int(c)] for i in range(ustart[p], ustart[p + 1])
                       for c in A.colind[A.rowptr[i]:A.rowptr[i + 1]]})
        colind.extend(cols)
        rowptr.append(len(colind))

    class _C:
        pass
    C = _C()
    C.n, C.rowptr, C.colind = nu, np.array(rowptr, dtype=np.int64), np.array(colind, dtype=np.int32)
    uperm, ub = cosine_blocking(C, tau, max_block, weights=[ustart[p + 1] - ustart[p] for p in range(nu)])
    perm, bstart = [], [0]
    for b in range(len(ub) - 1):
        for p in uperm[ub[b]:ub[b + 1]]:
            perm.extend(range(ustart[p], ustart[p + 1]))
        bstart.append(len(perm))
    return np.array(perm, dtype=np.int32), np.array(bstart, dtype=np.int32)
