"""The library's symmetrised matching (bilu_sym_mwm, host only) against the oracle, and the
exactly symmetric scaling of bilu_scale_permute_csr.

Bar: the same permutation and units as the oracle wherever the maximum matching is unique
(random values); the scaling may differ with the duals (they are not unique), so it is checked
by what it must satisfy: |a^_ij| <= 1, |a^| = 1 on a 2-cycle's coupling and on a 1-cycle's
diagonal.  A^ = P^T D A D P formed by bilu_scale_permute_csr is symmetric bit for bit."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.mwm_oracle as M
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import workloads as W


def _random_symmetric(n, seed, zero_diag):
    rng = np.random.default_rng(seed)
    Bm = rng.uniform(-4, 4, (n, n)) * (rng.random((n, n)) < 0.25)
    D = Bm + Bm.T
    D[np.arange(n), np.arange(n)] = rng.uniform(-1, 1, n) * (rng.random(n) >= zero_diag)
    D += np.eye(n, k=1) + np.eye(n, k=-1)  # a perfect matching exists
    return W.from_dense(D)


CASES = {f"random {n} zero diagonal {z}": (n, s, z) for (n, s, z) in
         ((9, 1, 1.0), (16, 2, 0.7), (25, 3, 0.4), (40, 4, 1.0), (33, 5, 0.5))}


def _case(name):
    if name.startswith("kkt"):
        return W.kkt_elasticity(side=4, block=24).A
    n, s, z = CASES[name]
    return _random_symmetric(n, s, z)


NAMES = sorted(CASES) + ["kkt elasticity 4^3"]


@pytest.mark.parametrize("name", NAMES)
def test_library_matches_oracle(name):
    A = _case(name)
    perm, ds, ustart = B.bilu_sym_mwm(A.n, A.rowptr, A.colind, A.val)
    po, do, uo, sigma = M.sym_matching(A)
    assert np.array_equal(perm, po) and np.array_equal(ustart, uo), name
    Ah = W.CSR(A.n, *B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, perm, perm, ds, ds))
    S = sp.csr_matrix((Ah.val, Ah.colind, Ah.rowptr), shape=(A.n, A.n))
    assert (S != S.T).nnz == 0  # symmetric bit for bit
    assert np.abs(S.data).max() <= 1 + 1e-12
    for u in range(len(ustart) - 1):
        a, b = ustart[u], ustart[u + 1]
        i = perm[a]
        if b - a == 1 and sigma[i] == i:
            assert abs(abs(S[a, a]) - 1) <= 1e-12
        if b - a == 2 and sigma[perm[a]] == perm[a + 1] and sigma[perm[a + 1]] == perm[a]:
            assert abs(abs(S[a, a + 1]) - 1) <= 1e-12


def test_refuses_unsymmetric_and_singular():
    A = _random_symmetric(10, 7, 0.5)
    D = sp.csr_matrix((A.val.copy(), A.colind, A.rowptr), shape=(10, 10)).toarray()
    D[0, 1] += 1.0
    U = W.from_dense(D)
    with pytest.raises(B.BiluError) as ei:
        B.bilu_sym_mwm(U.n, U.rowptr, U.colind, U.val)
    assert ei.value.status == B.BILU_ERR_ARG
    Z = np.zeros((4, 4))
    Z[0, 1] = Z[1, 0] = Z[1, 2] = Z[2, 1] = 1.0  # row 3 empty: no perfect matching
    Zc = W.from_dense(Z)
    with pytest.raises(B.BiluError) as ei:
        B.bilu_sym_mwm(Zc.n, Zc.rowptr, Zc.colind, Zc.val)
    assert ei.value.status == B.BILU_ERR_SINGULAR


def test_empty_matrix():
    perm, ds, ustart = B.bilu_sym_mwm(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert perm.size == 0 and ustart.tolist() == [0]
