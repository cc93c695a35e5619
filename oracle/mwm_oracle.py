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
