"""Pins of the oracle's symmetrised matching (Sec. 4.2, Duff and Pralet): the symmetric scaling
and the 1 x 1 / 2 x 2 pivot units cut from the cycles of the maximum weight matching.

- Hand-worked cycles: a 3-cycle (the one nonzero diagonal is left alone), a 5-cycle whose
  maximum matching beats every matching with 2-cycles, and a 4-ring where every perfect
  matching ties (the units are then neighbour pairs of the ring, whichever matching is found).
- Closed form: a diagonally dominant matrix is matched to its diagonal, every unit is 1 x 1 and
  ds_i = |a_ii|^{-1/2}.
- Saddle point: every multiplier (zero diagonal, one coupling) forms a 2 x 2 unit with the
  displacement it fixes, with |a^| = 1 on the coupling; |a^_ij| <= 1 everywhere.
- What the matching is for: BILDL of the saddle-point system with its multipliers first
  perturbs every multiplier pivot; after the matching (units kept inside the blocks) nothing is
  perturbed and SQMR needs fewer steps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import oracle.mwm_oracle as M
from paper_1908_10169_gb300 import workloads as W


def _scaled(A, ds):
    S = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n)).tocoo()
    return sp.csr_matrix((S.data * (ds[S.row] * ds[S.col]), (S.row, S.col)), shape=(A.n, A.n))


def _units(perm, ustart):
    return [sorted(perm[ustart[u]:ustart[u + 1]].tolist()) for u in range(len(ustart) - 1)]


def test_three_cycle_leaves_the_nonzero_diagonal_alone():
    # matchings: the two orientations of the 3-cycle, product 1 * 4 * 4 = 16; any matching with
    # a 2-cycle needs a diagonal entry at 0 or 1 (zero): the cycle is cut next to a_22
    A = W.from_dense(np.array([[0.0, 1.0, 4.0], [1.0, 0.0, 4.0], [4.0, 4.0, 1.0]]))
    perm, ds, ustart, sigma = M.sym_matching(A)
    assert sorted(sigma.tolist()) == [0, 1, 2] and all(sigma[i] != i for i in range(3))
    assert _units(perm, ustart) == [[0, 1], [2]] and perm.tolist() == [0, 1, 2]


def test_five_cycle_cut_around_its_diagonal_entry():
    # ring 0-1-2-3-4-0 with a_23 = a_34 = 3, the others 1, and a_33 = 2 the only diagonal entry:
    # the 5-cycle gives 1 * 1 * 3 * 3 * 1 = 9, the best matching with 2-cycles (1,2)(0,4) and
    # the diagonal at 3 gives 1 * 1 * 2 = 2; the cut leaves 3 alone: units {0,4}, {1,2}, {3}
    D = np.zeros((5, 5))
    for (i, j, v) in ((0, 1, 1.0), (1, 2, 1.0), (2, 3, 3.0), (3, 4, 3.0), (4, 0, 1.0)):
        D[i, j] = D[j, i] = v
    D[3, 3] = 2.0
    perm, ds, ustart, sigma = M.sym_matching(W.from_dense(D))
    k, i = 0, 0
    while True:  # sigma is one 5-cycle
        i, k = int(sigma[i]), k + 1
        if i == 0:
            break
    assert k == 5
    assert _units(perm, ustart) == [[0, 4], [1, 2], [3]] and perm.tolist() == [0, 4, 1, 2, 3]


def test_four_ring_ties_give_neighbour_pairs():
    D = np.zeros((4, 4))
    for (i, j) in ((0, 1), (1, 2), (2, 3), (3, 0)):
        D[i, j] = D[j, i] = 1.0
    perm, ds, ustart, _ = M.sym_matching(W.from_dense(D))
    units = _units(perm, ustart)
    assert sorted(sum(units, [])) == [0, 1, 2, 3] and all(len(u) == 2 and D[u[0], u[1]] != 0 for u in units)


def test_diagonally_dominant_matrix_keeps_its_diagonal():
    rng = np.random.default_rng(1)
    Bm = rng.uniform(-1, 1, (12, 12)) * (rng.random((12, 12)) < 0.3)
    Dm = Bm + Bm.T
    np.fill_diagonal(Dm, np.abs(Dm).sum(axis=1) + rng.uniform(1, 3, 12))
    A = W.from_dense(Dm)
    perm, ds, ustart, sigma = M.sym_matching(A)
    assert sigma.tolist() == list(range(12)) and np.diff(ustart).max() == 1 and perm.tolist() == list(range(12))
    np.testing.assert_allclose(ds, 1.0 / np.sqrt(np.diag(Dm)), rtol=1e-14)


def test_saddle_point_pairs_every_multiplier_with_its_displacement():
    w = W.kkt_elasticity(side=4, block=24)
    A = w.A
    m = 3 * 4 * 4  # multipliers first
    perm, ds, ustart, sigma = M.sym_matching(A)
    units = _units(perm, ustart)
    S = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    pair = {}
    for u in units:
        if len(u) == 2:
            pair[u[0]] = u[1]
    for k in range(m):
        d = int(S[k].indices[0])  # the one displacement multiplier k fixes
        assert pair.get(k) == d
    Ah = _scaled(A, ds)
    assert np.abs(Ah.data).max() <= 1 + 1e-12
    for k in range(m):
        assert abs(abs(Ah[k, pair[k]]) - 1.0) <= 1e-12


def _unit_blocks(ustart, bmax):
    out = [0]
    for k in range(1, len(ustart)):
        if ustart[k] - out[-1] > bmax:
            out.append(int(ustart[k - 1]))
    if out[-1] != ustart[-1]:
        out.append(int(ustart[-1]))
    return np.array(out, np.int32)


@pytest.mark.parametrize("side,tau", [(6, 1e-2), (6, 1e-3)])
def test_matching_removes_the_perturbations_of_bildl(side, tau):
    w = W.kkt_elasticity(side=side, block=24)
    A, n = w.A, w.A.n
    F = O.bildl_factor(A, O.partition_fixed(n, 24), tau)
    r = O.sqmr(A, F, w.b, 1e-6, 2000)
    assert F.counters["nperturb"] == 3 * side * side  # every multiplier pivot
    perm, ds, ustart, _ = M.sym_matching(A)
    Ah = _scaled(A, ds)[perm][:, perm].tocsr()
    Ah.sort_indices()
    Awh = W.CSR(n, Ah.indptr.astype(np.int64), Ah.indices.astype(np.int32), Ah.data)
    G = O.bildl_factor(Awh, _unit_blocks(ustart, 24), tau)
    r2 = O.sqmr(Awh, G, (ds * w.b)[perm], 1e-6, 2000)
    assert G.counters["nperturb"] == 0 and r.status == 0 and r2.status == 0 and r2.iters < r.iters
    # the solution maps back: x[perm] = ds[perm] y
    x = np.empty(n)
    x[perm] = ds[perm] * r2.x
    assert np.abs(x - 1.0).max() < 1e-3
