"""Hand-derived worked examples (``tests/golden/*.json``) against the oracle.

Each fixture states the passage it follows and its derivation in exact fractions; the values
were worked out by hand, not produced by any code. The GPU tests check the library against the
same fixtures.
"""
import glob
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1908_10169_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def frac(x):
    """A fixture value (a fraction string, nested lists of them) as float64."""
    if isinstance(x, list):
        return np.array([frac(v) for v in x], dtype=np.float64)
    return float(Fraction(x))


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def factor_fixtures():
    return sorted(os.path.basename(p) for p in glob.glob(os.path.join(GOLDEN, "*.json"))
                  if "blocks" in load(os.path.basename(p)))


def check_factor(g, F, rtol=1e-15):
    """Compare a factor F (oracle Factor, or any object with the same block accessors) with
    the fixture g block by block."""
    for K, blk in enumerate(g["blocks"]):
        rows, lv = F.L_block(K)
        cols, uv = F.U_block(K)
        assert list(rows) == blk["Lrow"], (K, list(rows))
        assert list(cols) == blk["Ucol"], (K, list(cols))
        for got, want in ((F.P_block(K), blk["P"]), (F.D_block(K), blk["D"]), (lv, blk["L"]), (uv, blk["U"])):
            w = frac(want).reshape(np.shape(got))
            assert np.allclose(got, w, rtol=rtol, atol=rtol * max(1.0, np.abs(w).max(initial=0.0))), (K, got, w)


def test_fixtures_are_present():
    assert set(os.listdir(GOLDEN)) >= {"block_crout_4x4.json", "scalar_crout_3x3_fill.json", "perturbation_2x2.json"}
    for name in os.listdir(GOLDEN):
        if not name.endswith(".json"):  # computed/: oracle runs written by a script, not by hand
            continue
        g = load(name)
        assert g["citation"] and g["derivation"]


@pytest.mark.parametrize("name", factor_fixtures())
def test_oracle_matches_worked_example(name):
    g = load(name)
    A = W.from_dense(frac(g["A"]))
    F = O.bilu_factor(A, np.array(g["bstart"], np.int32), frac(g["tau"]))
    assert F.status == 0
    check_factor(g, F)


@pytest.mark.parametrize("case", [c["case"] for c in load("perturbation_2x2.json")["cases"]])
def test_oracle_matches_perturbation_example(case):
    c = next(c for c in load("perturbation_2x2.json")["cases"] if c["case"] == case)
    F = O.bilu_factor(W.from_dense(frac(c["A"])), np.array(c["bstart"], np.int32), 0.0, perturb=True,
                      pert_tau=1e-2, pert_rho=1e-1)
    assert F.status == 2 and F.counters["nperturb"] == 1
    assert np.allclose(F.P_block(0), frac(c["P0"]), rtol=1e-15, atol=0)
