"""Pins of the maximum-weight-matching oracle (Sec. 3.1): brute force over all permutations,
scipy's assignment solver, LP duality and closed forms."""
import itertools
import math

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import mwm_oracle as M
from paper_1908_10169_gb300 import workloads as W


def random_matchable(n, density, seed):
    """Random sparse matrix with a hidden perfect matching (entries of random sign)."""
    rng = np.random.default_rng(seed)
    d = (rng.random((n, n)) < density) * rng.uniform(-3, 3, (n, n))
    d[np.arange(n), rng.permutation(n)] = rng.uniform(0.1, 5, n) * rng.choice([-1, 1], n)
    return W.from_dense(d, keep_zeros_on_diag=False), d


def check_invariants(d, sigma, dl, dr, u, v, C):
    n = d.shape[0]
    assert sorted(sigma) == list(range(n))
    Ah = dl[:, None] * d * dr[None, :]
    assert np.all(np.abs(Ah) <= 1 + 1e-12)
    assert np.allclose(np.abs(Ah[np.arange(n), sigma]), 1.0, rtol=0, atol=1e-12)
    fin = np.isfinite(C)
    slack = C - u[:, None] - v[None, :]
    assert np.all(slack[fin] >= -1e-12)                            # dual feasibility
    assert np.allclose(slack[np.arange(n), sigma], 0, atol=1e-12)   # complementary slackness


@pytest.mark.parametrize("seed", range(40))
def test_optimum_equals_brute_force(seed):
    n = 1 + seed % 6
    A, d = random_matchable(n, 0.5, seed)
    sigma, dl, dr, u, v, total = M.mwm(A)
    C, _ = M.costs(A)
    best = min(sum(C[i, p[i]] for i in range(n)) for p in itertools.permutations(range(n)))
    assert math.isfinite(best) and abs(total - best) <= 1e-12 * max(1.0, abs(best))
    check_invariants(d, sigma, dl, dr, u, v, C)


@pytest.mark.parametrize("seed", range(6))
def test_optimum_equals_scipy_assignment(seed):
    A, d = random_matchable(50, 0.08, 100 + seed)
    sigma, dl, dr, u, v, total = M.mwm(A)
    C, _ = M.costs(A)
    big = np.where(np.isfinite(C), C, 1e6)
    r, c = linear_sum_assignment(big)
    assert abs(big[r, c].sum() - total) <= 1e-10
    check_invariants(d, sigma, dl, dr, u, v, C)


def test_costs_are_column_normalised():
    """c_ij = log a_j - log|a_ij| with a_j the largest |a_kj| of column j: every cost is >= 0
    and each column's largest entry costs exactly 0 (so that D_r = e^v / a_j)."""
    A, d = random_matchable(30, 0.2, 7)
    C, amax = M.costs(A)
    fin = np.isfinite(C)
    assert np.all(C[fin] >= 0.0)
    for j in range(A.n):
        col = np.abs(d[:, j])
        assert amax[j] == col.max() and C[int(np.argmax(col)), j] == 0.0


def test_scaled_permutation_matrix_becomes_signed_identity():
    """A = diag(s) P: the only perfect matching is P itself; every column has one entry, its
    cost is 0, and A^ = D_l A D_r Pi has entries +-1 on the diagonal and nothing else."""
    n = 7
    rng = np.random.default_rng(3)
    p = rng.permutation(n)
    d = np.zeros((n, n))
    d[np.arange(n), p] = rng.uniform(0.5, 8.0, n) * rng.choice([-1, 1], n)
    A = W.from_dense(d, keep_zeros_on_diag=False)
    sigma, dl, dr, u, v, total = M.mwm(A)
    assert list(sigma) == list(p) and total == 0.0
    Ah = (dl[:, None] * d * dr[None, :])[:, sigma]
    assert np.allclose(np.abs(np.diag(Ah)), 1.0, atol=1e-15)
    assert np.count_nonzero(Ah) == n


def test_dominant_diagonal_is_kept():
    """A column-wise strictly dominant diagonal (|a_jj| the largest entry of column j) costs 0
    on the identity, and every other entry costs > 0: the identity is the unique optimum."""
    A = W.convdiff_upwind((5, 5, 5), seed=1)
    sigma, dl, dr, u, v, total = M.mwm(A)
    assert list(sigma) == list(range(A.n)) and total == 0.0


def test_structurally_singular_is_reported():
    """Rows 0 and 1 have their only entries in column 0 (Hall's condition fails)."""
    d = np.array([[1.0, 0, 0], [2.0, 0, 0], [1.0, 1.0, 1.0]])
    with pytest.raises(ValueError, match="singular"):
        M.mwm(W.from_dense(d, keep_zeros_on_diag=False))
