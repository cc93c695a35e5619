"""Pins of the single-block-step checker (oracle/block_check.py, numpy + LAPACK) against the
full C oracle (an independent implementation): recomputing every block of the C oracle's own
factor from its earlier blocks reproduces it, and a planted change is detected."""
import numpy as np
import pytest

import oracle as O
from oracle import block_check as BC
from paper_1908_10169_gb300 import workloads as W


def _export(F):
    return {"bstart": F.bstart, "Lptr": F.Lptr, "Lrow": F.Lrow, "Lval": F.Lval, "Uptr": F.Uptr,
            "Ucol": F.Ucol, "Uval": F.Uval, "Dinv": F.Dinv, "Pblk": F.Pblk}


@pytest.mark.parametrize("case", ["cd2d", "cd3d", "random"])
def test_block_step_reproduces_the_c_oracle(case):
    if case == "cd2d":
        w = W.cd2d_32()
        A, bs, tau = w.A, np.arange(0, w.A.n + 1, 32), w.droptol
    elif case == "cd3d":
        w = W.cd3d(side=8, seed=3, block=16)
        A, bs, tau = w.A, np.arange(0, w.A.n + 1, 16), w.droptol
    else:
        A = W.random_diag_dominant(150, 0.05, seed=4)
        bs, tau = np.array([0, 7, 20, 41, 64, 90, 97, 120, 150]), 3e-2
    F = O.bilu_factor(A, bs, tau)
    E = _export(F)
    blocks = BC._blocks(E)
    worst = 0.0
    for K in range(len(bs) - 1):
        flips, err = BC.compare_block(A, E, K, tau, rtol=1e-12, blocks=blocks)
        assert flips == 0
        worst = max(worst, err)
    assert worst < 1e-12


def test_block_check_detects_a_changed_value():
    w = W.cd3d(side=8, seed=3, block=16)
    bs = np.arange(0, w.A.n + 1, 16)
    F = O.bilu_factor(w.A, bs, w.droptol)
    E = _export(F)
    K = 5
    b = 16
    # perturb one stored value of block K's L part
    lo = int(F.Lptr[K]) * b
    E["Lval"] = E["Lval"].copy()
    E["Lval"][lo + 3] += 1e-8 * np.abs(E["Lval"][lo:lo + b]).max()  # relative change 1e-8 of the row
    with pytest.raises(AssertionError):
        BC.compare_block(w.A, E, K, w.droptol)


def test_block_check_rejects_a_flip_far_from_tau():
    """A kept row of L removed from the factor (its norm far above tau) is a drop decision
    that differs for a reason other than rounding: the checker raises."""
    w = W.cd3d(side=8, seed=3, block=16)
    bs = np.arange(0, w.A.n + 1, 16)
    F = O.bilu_factor(w.A, bs, w.droptol)
    E = _export(F)
    K, b = 5, 16
    p = int(F.Lptr[K])
    lo = p * b
    assert np.linalg.norm(F.Lval[lo:lo + b]) > 10 * w.droptol
    E["Lrow"] = np.delete(F.Lrow, p)
    E["Lval"] = np.delete(F.Lval, np.arange(lo, lo + b))
    E["Lptr"] = F.Lptr.copy()
    E["Lptr"][K + 1:] -= 1
    with pytest.raises(AssertionError, match="drop decision"):
        BC.compare_block(w.A, E, K, w.droptol)
