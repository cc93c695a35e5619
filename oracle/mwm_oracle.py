"""Plain reference of the maximum weight matching with scaling (Sec. 3.1), small n only.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the test suite may use it; the
product never imports it.

Sec. 3.1 replaces A by A^ = D_l A D_r Pi with |a^_ij| <= 1 and |a^_ii| = 1: a maximum product
transversal (a permutation that maximises the product of the absolute values of the entries
it puts on the diagonal) found as a linear assignment problem on negative logarithms, and
diagonal scalings from the exponentials of its dual variables.  Written out:

  costs      c_ij = log(a_j) - log|a_ij| >= 0 for every stored nonzero a_ij, a_j = max_k |a_kj|
             (no edge where a_ij = 0);
  matching   sigma (row i -> column sigma(i)) minimising sum_i c_{i sigma(i)};
  duals      u_i + v_j <= c_ij on every edge, with equality on the matching (LP duality);
  scaling    D_l = diag(e^{u_i}), D_r = diag(e^{v_j} / a_j), so that
             |a^_ij| = e^{u_i + v_j - c_ij} <= 1, with equality on the matching;
  Pi         moves column sigma(i) to position i: A^[i, i] = d_l[i] a_{i sigma(i)} d_r[sigma(i)].

The assignment is solved here by the Hungarian method with potentials on the dense cost
matrix (one shortest augmenting path per row, O(n^3)), in plain Python loops.
"""
from __future__ import annotations

import math

import numpy as np

INF = math.inf


def costs(A):
    """Dense cost matrix (inf where there is no edge) and the column maxima a_j."""
    n = A.n
    C = np.full((n, n), INF)
    amax = np.zeros(n)
    for i in range(n):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            j = int(A.colind[e])
            amax[j] = max(amax[j], abs(float(A.val[e])))
    for i in range(n):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            j, a = int(A.colind[e]), abs(float(A.val[e]))
            if a > 0.0:
                C[i, j] = math.log(amax[j]) - math.log(a)
    return C, amax


def hungarian(C):
    """Minimum-cost perfect matching of the dense cost matrix C (inf = no edge).  Returns
    (sigma, u, v) with u_i + v_j <= C_ij everywhere and equality on (i, sigma(i)); raises
    ValueError when no perfect matching exists."""
    n = C.shape[0]
    u = [0.0] * n            # row potentials
    v = [0.0] * n            # column potentials
    row_of = [-1] * n        # row matched to each column
    for s in range(n):
        # Dijkstra over columns with reduced costs C_ij - u_i - v_j >= 0, from row s
        dist = [INF] * n
        prev = [-1] * n      # the row from which each column was reached
        done = [False] * n
        for j in range(n):
            if C[s, j] < INF:
                dist[j] = C[s, j] - u[s] - v[j]
                prev[j] = s
        while True:
            j = -1
            for k in range(n):
                if not done[k] and dist[k] < INF and (j < 0 or dist[k] < dist[j]):
                    j = k
            if j < 0:
                raise ValueError("structurally singular: no perfect matching")
            done[j] = True
            if row_of[j] < 0:
                free = j
                break
            i = row_of[j]
            for k in range(n):
                if not done[k] and C[i, k] < INF:
                    d = dist[j] + C[i, k] - u[i] - v[k]
                    if d < dist[k]:
                        dist[k] = d
                        prev[k] = i
        D = dist[free]
        # potentials: reached rows gain D - dist(column they were reached through), finished
        # columns lose D - dist; reduced costs stay >= 0 and vanish along the path
        u[s] += D
        for j in range(n):
            if done[j] and j != free:
                u[row_of[j]] += D - dist[j]
                v[j] -= D - dist[j]
        # augment along the path
        j = free
        while True:
            i = prev[j]
            nxt = -1
            for k in range(n):
                if row_of[k] == i:
                    nxt = k
            row_of[j] = i
            if i == s:
                break
            row_of[nxt] = -1
            j = nxt
    sigma = [0] * n
    for j in range(n):
        sigma[row_of[j]] = j
    return np.array(sigma, dtype=np.int32), np.array(u), np.array(v)


def mwm(A):
    """(sigma, d_l, d_r, u, v, cost): the matching, the scalings of Sec. 3.1, the duals and the
    optimal sum of costs."""
    C, amax = costs(A)
    sigma, u, v = hungarian(C)
    dl = np.array([math.exp(x) for x in u])
    dr = np.array([math.exp(v[j]) / (amax[j] if amax[j] > 0 else 1.0) for j in range(A.n)])
    total = float(sum(C[i, sigma[i]] for i in range(A.n)))
    return sigma, dl, dr, u, v, total


# ------------------------------------------------------------------ symmetric matching
#
# Sec. 4.2 (the symmetric variant) replaces the matching by a symmetrised one (Duff and
# Pralet): A^ = P^T D A D P with |a^_ij| <= 1, where the cycles of the matching sigma give
# pivots of size 1 x 1 (|a^_ii| = 1) and 2 x 2 (|a^_{i,i+1}| = 1) that stay together.  Written
# out (readings R25, R26):
#   scaling   D = diag(sqrt(d_l d_r)) from the scalings of the unsymmetric matching above, so
#             that |a^_ij|^2 = |a^_ij of D_l A D_r| |a^_ji of D_l A D_r| <= 1 for symmetric A;
#   cycles    i -> sigma(i) -> ... ; a cycle of one index is a 1 x 1 unit, of two a 2 x 2 unit;
#             a longer cycle c_0 .. c_{k-1} is cut into pairs of neighbours (c_t, c_{t+1}),
#             whose coupling a_{c_t c_{t+1}} is a matched entry: for even k the one of the two
#             cuts (starting at c_0 or at c_1) with the larger sum of log |a_pair|, for odd k
#             the cut leaving c_s alone that maximises log |a_{c_s c_s}| + sum log |a_pair|
#             (the first on ties; a zero diagonal counts as -inf);
#   order     units by their smallest index, the indices of a unit increasing.


def _abs_entry(A, i, j):
    for e in range(A.rowptr[i], A.rowptr[i + 1]):
        if int(A.colind[e]) == j:
            return abs(float(A.val[e]))
    return 0.0


def _log(x):
    return math.log(x) if x > 0.0 else -INF


def sym_units(A, sigma):
    """The 1 x 1 / 2 x 2 units from the cycles of the matching sigma (see above)."""
    n = A.n
    seen = [False] * n
    units = []
    for i in range(n):
        if seen[i]:
            continue
        cyc = [i]
        seen[i] = True
        j = int(sigma[i])
        while j != i:
            cyc.append(j)
            seen[j] = True
            j = int(sigma[j])
        k = len(cyc)
        if k <= 2:
            units.append(sorted(cyc))
            continue
        if k % 2 == 0:
            best_score, first = None, 0
            for start in (0, 1):
                score = 0.0
                for t in range(start, start + k, 2):
                    score += _log(_abs_entry(A, cyc[t % k], cyc[(t + 1) % k]))
                if best_score is None or score > best_score:
                    best_score, first = score, start
            for t in range(first, first + k, 2):
                units.append(sorted([cyc[t % k], cyc[(t + 1) % k]]))
        else:
            best_score, alone = None, 0
            for s in range(k):
                score = _log(_abs_entry(A, cyc[s], cyc[s]))
                for t in range(s + 1, s + k, 2):
                    score += _log(_abs_entry(A, cyc[t % k], cyc[(t + 1) % k]))
                if best_score is None or score > best_score:
                    best_score, alone = score, s
            units.append([cyc[alone]])
            for t in range(alone + 1, alone + k, 2):
                units.append(sorted([cyc[t % k], cyc[(t + 1) % k]]))
    units.sort(key=lambda u: u[0])
    perm = np.array([i for u in units for i in u], dtype=np.int32)
    ustart = np.concatenate([[0], np.cumsum([len(u) for u in units])]).astype(np.int32)
    return perm, ustart


def sym_matching(A):
    """(perm, ds, ustart, sigma): the symmetric permutation (original index at each new
    position), the symmetric scaling, the unit boundaries in the new order, the matching."""
    sigma, dl, dr, _, _, _ = mwm(A)
    ds = np.sqrt(dl * dr)
    perm, ustart = sym_units(A, sigma)
    return perm, ds, ustart, sigma
