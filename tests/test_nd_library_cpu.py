"""The library's host-side block nested dissection and block elimination tree (Sec. 3.3)
against the oracle, bit for bit, on the CPU (host code: no context, no device)."""
import numpy as np
import pytest

import paper_1908_10169_gb300 as B
from oracle import nd_oracle as N
from paper_1908_10169_gb300 import workloads as W
from tests.test_nd_oracle import pattern_matrix, permuted


def _cases():
    yield "cd3d_lines", W.convdiff_upwind((8, 8, 8), seed=2), 8
    yield "cd3d_planes", W.convdiff_upwind((6, 6, 6), seed=1), 36
    yield "cd2d", W.cd2d_32().A, 32
    yield "elasticity", W.elasticity3d(side=4, seed=2, block=63).A, 12
    yield "random", W.random_diag_dominant(300, 0.01, seed=4), 7
    yield "path", W.from_dense(4 * np.eye(15) - np.eye(15, k=1) - np.eye(15, k=-1)), 1
    yield "one_sided", W.from_dense(4 * np.eye(9) - np.eye(9, k=-1)), 1
    chain = [5, 3, 1, 0, 2, 4, 6]
    rows = [{v} for v in range(7)]
    for a, b in zip(chain, chain[1:]):
        rows[a].add(b)
        rows[b].add(a)
    yield "relabelled_path", pattern_matrix(rows), 1
    yield "disconnected", W.from_dense(np.kron(np.eye(3), 4 * np.eye(6) - np.eye(6, k=1) - np.eye(6, k=-1))), 2


CASES = {name: (A, b) for name, A, b in _cases()}


def _bs(A, b):
    return np.append(np.arange(0, A.n, b), A.n).astype(np.int32)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("leaf", [1, 3])
def test_nd_order_matches_oracle(name, leaf):
    A, b = CASES[name]
    bs = _bs(A, b)
    got = B.bilu_nd_order(A.n, A.rowptr, A.colind, bs, leaf)
    want = N.nd_order(A, bs, leaf)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("name", sorted(CASES))
def test_block_etree_matches_oracle(name):
    A, b = CASES[name]
    bs = _bs(A, b)
    for Ap, bsp in ((A, bs), (None, None)):
        if Ap is None:
            perm, bsp, _ = N.nd_order(A, bs)
            Ap = permuted(A, perm)
        parent, height = B.bilu_block_etree(Ap.n, Ap.rowptr, Ap.colind, bsp)
        want = N.block_etree(Ap, bsp)
        assert np.array_equal(parent, want)
        h = np.ones(len(want), int)
        for K in range(len(want)):
            if want[K] >= 0:
                h[want[K]] = max(h[want[K]], h[K] + 1)
        assert height == h.max()


def test_larger_grids_match_oracle():
    """Line blocks of 16^3 and 12 x 20 x 24 convection-diffusion grids (256 and 240 blocks)."""
    for A, b in ((W.convdiff_upwind((16, 16, 16), seed=1), 16), (W.convdiff_upwind((12, 20, 24), seed=2), 12)):
        bs = _bs(A, b)
        got = B.bilu_nd_order(A.n, A.rowptr, A.colind, bs)
        want = N.nd_order(A, bs)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
        Ap = permuted(A, got[0])
        parent, height = B.bilu_block_etree(Ap.n, Ap.rowptr, Ap.colind, got[1])
        assert np.array_equal(parent, N.block_etree(Ap, got[1]))


def test_nd_and_etree_errors():
    A = pattern_matrix([{0, 1}, {0, 1, 2}, {1, 2}])
    with pytest.raises(B.BiluError, match="partition"):
        B.bilu_nd_order(A.n, A.rowptr, A.colind, [0, 2, 2, 3])
    with pytest.raises(B.BiluError, match="leaf"):
        B.bilu_nd_order(A.n, A.rowptr, A.colind, [0, 1, 2, 3], 0)
    with pytest.raises(B.BiluError, match="partition"):
        B.bilu_block_etree(A.n, A.rowptr, A.colind, [0, 4])
    p, bs, order = B.bilu_nd_order(0, np.zeros(1, np.int64), np.zeros(0, np.int32), [0])
    assert p.size == 0 and list(bs) == [0] and order.size == 0
