"""The library's host-side cosine blocking (Sec. 3.2) and symmetric permutation against the
oracle, bit for bit, on the CPU (both calls are host code: no context, no device)."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1908_10169_gb300 as B
from oracle import cosine_oracle as C
from paper_1908_10169_gb300 import workloads as W
from tests.test_cosine_oracle import HAND, from_pattern, permuted


def _random_pattern(n, density, seed):
    rng = np.random.default_rng(seed)
    d = (rng.random((n, n)) < density) * rng.uniform(0.5, 1.5, (n, n))
    d[np.arange(n), np.arange(n)] = 4.0
    heavy = rng.integers(0, n, 2)  # a few long rows / columns
    d[heavy[0], :] = 1.0
    d[:, heavy[1]] = 1.0
    return W.from_dense(d, keep_zeros_on_diag=False)


def _cases():
    rng = np.random.default_rng(0)
    el = W.elasticity3d(side=4, seed=2, block=63).A
    yield "hand", from_pattern(HAND, 6)
    yield "nonsymmetric", from_pattern([{0, 1, 2}, {0, 1, 2}, {2}, {1, 3}, {1, 4}], 5)
    yield "elasticity_permuted", permuted(el, rng.permutation(el.n).astype(np.int32))
    yield "laplace27x4", W.laplace27_4dof(side=4, seed=3, block=64).A
    yield "cd3d", W.cd3d(side=6, seed=1, block=6).A
    for s in range(4):
        yield f"random{s}", _random_pattern(60 + 17 * s, 0.05 + 0.03 * s, s)
    yield "n1", W.from_dense(np.array([[2.0]]))


CASES = dict(_cases())


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tau,max_block", [(0.8, 64), (0.0, 64), (0.5, 5), (1.0, 64), (0.8, 1), (0.3, 2)])
def test_library_cosine_blocking_matches_oracle(name, tau, max_block):
    A = CASES[name]
    p, b = B.bilu_cosine_blocking(A.n, A.rowptr, A.colind, tau, max_block)
    po, bo = C.cosine_blocking(A, tau, max_block)
    assert np.array_equal(p, po) and np.array_equal(b, bo)
    assert np.array_equal(np.sort(p), np.arange(A.n))
    assert np.all(np.diff(b) >= 1) and np.all(np.diff(b) <= max_block)


def test_larger_matrices_match_oracle():
    """Scrambled Q1 elasticity on a 7^3 grid (1,029 unknowns, rows of up to 81 entries) and the
    4-unknown 27-point operator on 5^3 nodes."""
    el = W.elasticity3d(side=7, seed=2, block=63).A
    l27 = W.laplace27_4dof(side=5, seed=3, block=64).A
    for A in (permuted(el, np.random.default_rng(8).permutation(el.n).astype(np.int32)), l27):
        p, b = B.bilu_cosine_blocking(A.n, A.rowptr, A.colind, 0.8, 64)
        po, bo = C.cosine_blocking(A, 0.8, 64)
        assert np.array_equal(p, po) and np.array_equal(b, bo)


def test_empty_matrix():
    p, b = B.bilu_cosine_blocking(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert p.size == 0 and list(b) == [0]


@pytest.mark.parametrize("name", sorted(CASES))
def test_permute_csr_matches_scipy(name):
    A = CASES[name]
    perm = np.random.default_rng(len(name)).permutation(A.n).astype(np.int32)
    rp, ci, va = B.bilu_permute_csr(A.n, A.rowptr, A.colind, A.val, perm)
    R = permuted(A, perm)
    assert np.array_equal(rp, R.rowptr) and np.array_equal(ci, R.colind) and np.array_equal(va, R.val)


def test_host_calls_report_errors():
    A = from_pattern(HAND, 6)
    with pytest.raises(B.BiluError, match="permutation"):
        B.bilu_permute_csr(A.n, A.rowptr, A.colind, A.val, np.array([0, 1, 2, 3, 4, 4], np.int32))
    with pytest.raises(B.BiluError, match="tau"):
        B.bilu_cosine_blocking(A.n, A.rowptr, A.colind, -0.1)
    with pytest.raises(B.BiluError, match="max_block"):
        B.bilu_cosine_blocking(A.n, A.rowptr, A.colind, 0.8, 65)
    bad = A.colind.copy()
    bad[0], bad[1] = bad[1], bad[0]
    with pytest.raises(B.BiluError, match="increasing"):
        B.bilu_cosine_blocking(A.n, A.rowptr, bad)


def test_unit_blocking_matches_oracle():
    """bilu_cosine_blocking_units against the oracle on random patterns and random units:
    the same permutation and blocks, every block made of whole units and at most max_block."""
    import numpy as np
    from oracle import cosine_oracle as C
    import paper_1908_10169_gb300 as B
    from paper_1908_10169_gb300 import workloads as W
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(1, 60))
        dens = [0.05, 0.15, 0.4][trial % 3]
        D = (rng.random((n, n)) < dens).astype(float)
        D[np.arange(n), np.arange(n)] = 1.0
        A = W.from_dense(D)
        cuts = sorted(set(rng.choice(np.arange(1, n), size=min(n - 1, int(rng.integers(0, n))), replace=False).tolist())) if n > 1 else []
        us = np.array([0] + cuts + [n], np.int32)
        us = us[np.concatenate([[True], np.diff(us) > 0])]
        mb = int(max(np.diff(us).max(), rng.integers(1, 20)))
        tau = float(rng.choice([0.3, 0.5, 0.8]))
        p1, b1 = B.bilu_cosine_blocking_units(n, A.rowptr, A.colind, us, tau, mb)
        p2, b2 = C.cosine_blocking_units(A, us, tau, mb)
        assert np.array_equal(p1, p2) and np.array_equal(b1, b2), trial
        assert set(b1.tolist()) >= {0, n} and np.diff(b1).max() <= mb
        starts = set(us.tolist())
        for k in range(len(b1) - 1):  # a block is a run of whole units of the original order
            assert p1[b1[k]] in starts


def test_unit_blocking_refuses_bad_units():
    import numpy as np
    import pytest
    import paper_1908_10169_gb300 as B
    from paper_1908_10169_gb300 import workloads as W
    A = W.from_dense(np.eye(6))
    for us, mb in (([0, 3, 5], 64), ([0, 3, 3, 6], 64), ([0, 4, 6], 3)):
        with pytest.raises(B.BiluError):
            B.bilu_cosine_blocking_units(6, A.rowptr, A.colind, us, 0.8, mb)
