"""The library's host-side ILU(1,tau) partition (Sec. 3.4), column by column and over groups
of columns, against the oracle bit for bit on the CPU (bilu_partition_ilu1t is host code)."""
import numpy as np
import pytest

import oracle as O
import paper_1908_10169_gb300 as B
from oracle import cosine_oracle as C
from paper_1908_10169_gb300 import workloads as W
from tests.test_cosine_oracle import permuted


def _cases():
    yield "cd2d", W.cd2d_32().A
    yield "cd3d", W.convdiff_upwind((10, 10, 10), seed=3)
    yield "elasticity", W.elasticity3d(side=4, seed=2, block=63).A
    yield "laplace27x4", W.laplace27_4dof(side=4, seed=3, block=64).A
    for s in range(3):
        yield f"random{s}", W.random_diag_dominant(150 + 50 * s, 0.03 + 0.02 * s, seed=s)
    yield "tridiagonal", W.from_dense(4 * np.eye(12) - np.eye(12, k=1) - np.eye(12, k=-1))
    yield "diagonal", W.from_dense(3 * np.eye(12))


CASES = dict(_cases())


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tau,max_block", [(1e-2, 64), (1e-3, 16), (0.0, 7), (0.5, 64)])
def test_column_rule_matches_oracle(name, tau, max_block):
    A = CASES[name]
    got = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, tau, max_block)
    assert np.array_equal(got, O.partition_ilu1t(A, tau, max_block))


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("grouping", ["cosine", "pairs", "uneven"])
def test_group_rule_matches_oracle(name, grouping):
    A = CASES[name]
    if grouping == "cosine":  # the cosine blocks of a scrambled copy, as the library finds them
        A = permuted(A, np.random.default_rng(1).permutation(A.n).astype(np.int32))
        perm, groups = C.cosine_blocking(A, 0.8, 64)
        A = permuted(A, perm)
    elif grouping == "pairs":
        groups = np.append(np.arange(0, A.n, 2), A.n)
    else:
        rng = np.random.default_rng(A.n)
        cuts = np.sort(rng.choice(np.arange(1, A.n), size=A.n // 4, replace=False))
        groups = np.concatenate([[0], cuts, [A.n]])
        groups = groups[np.concatenate([[True], np.diff(groups) > 0])]
        # split any group above the cap
        out = [0]
        for e in groups[1:]:
            while e - out[-1] > 16:
                out.append(out[-1] + 16)
            out.append(int(e))
        groups = np.array(out)
    for tau, mb in ((1e-2, 64), (0.0, 32)):
        got = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, tau, mb, groups)
        assert np.array_equal(got, O.partition_ilu1t_groups(A, tau, mb, groups))
        assert set(got) <= set(groups)


def test_partition_errors():
    A = CASES["diagonal"]
    with pytest.raises(B.BiluError, match="groups"):
        B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, 1e-2, 64, [0, 5, 11])
    with pytest.raises(B.BiluError, match="group size"):
        B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, 1e-2, 4, [0, 6, 12])
    assert list(B.bilu_partition_ilu1t(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))) == [0]
