"""Pins of the learned skip's oracle (features, labels, classifier gradient) to values fixed
by hand, by an independent implementation, or by the mathematics -- not by retyping it."""
import numpy as np
import pytest

import oracle as O
from oracle import skip_oracle as S
from paper_1908_10169_gb300 import workloads as W


def _lg(x):
    return np.log10(max(x, 1e-30))


def test_features_hand_example():
    """A = [[4,-1,-1],[-1,4,0],[-1,0,4]], blocks of 1, tau = 1e-2 (scalar Algorithm 1).
    Block 0: l = (-1/4, -1/4), U-breve row (-1, -1), D_0 = 1/4.  Block 1 sees the fill
    entry (2,1) through producer 0: T_L(2,1) = 0 - (-1/4)(-1) = -1/4, P_1 = 15/4, so
    l_21 = -1/15 is kept; likewise the U-side fill (1,2)."""
    d = np.array([[4.0, -1, -1], [-1, 4, 0], [-1, 0, 4]])
    A = W.from_dense(d)
    F = O.bilu_factor(A, np.array([0, 1, 2, 3]), 1e-2)
    x, y, tags = S.skip_features(A, F, 1e-2)
    got = {int(t): (xx, yy) for t, xx, yy in zip(tags, x, y)}
    tag = lambda K, side, i: (K << 33) | (side << 32) | i
    f7, f8 = np.log10(1e-2), 1 / 64
    # block 0 candidates: A entries only, no producers, d = 1 / max|a| = 1/4
    for side, i in ((0, 1), (0, 2), (1, 1), (1, 2)):
        xx, yy = got[tag(0, side, i)]
        want = [_lg(1.0), 1, -30, -30, 0, _lg(0.25), _lg(0.25), f7, f8, 0, np.log2(1 + (i - 1) / 64), side]
        np.testing.assert_allclose(xx, want, atol=1e-12)
        assert yy == 0.0
    # block 1: the fill candidates, one producer each (||X|| ||Y||_F = 1/4 * 1 on both sides)
    for side in (0, 1):
        xx, yy = got[tag(1, side, 2)]
        want = [-30, 0, _lg(0.25), _lg(0.25), 1, _lg(0.25), _lg(0.25 * 0.25), f7, f8, 1 / 64, 0, side]
        np.testing.assert_allclose(xx, want, atol=1e-12)
        assert yy == 0.0
    assert len(tags) == 6


@pytest.mark.parametrize("case", ["cd2d", "cd3d"])
def test_feature_candidates_match_oracle_counters(case):
    """The candidate sets of skip_features (Python, from the exported factor) have the sizes
    the C oracle counts during its own factorization, and the labels match its kept sets."""
    if case == "cd2d":
        w = W.cd2d_32()
        bs = np.arange(0, w.A.n + 1, 32)
    else:
        w = W.cd3d(side=8, seed=2, block=8)
        bs = np.arange(0, w.A.n + 1, 8)
    F = O.bilu_factor(w.A, bs, w.droptol)
    x, y, tags = S.skip_features(w.A, F, w.droptol)
    side = (tags >> 32) & 1
    assert (side == 0).sum() == F.counters["cand_rows"]
    assert (side == 1).sum() == F.counters["cand_cols"]
    assert ((side == 0) & (y == 0)).sum() == len(F.Lrow)
    assert ((side == 1) & (y == 0)).sum() == len(F.Ucol)
    assert np.all(np.diff(tags) > 0)
    assert np.isfinite(x).all()


def _rand_model(seed):
    rng = np.random.default_rng(seed)
    p = {"mean": rng.normal(size=S.NF), "std": rng.uniform(0.5, 2, size=S.NF),
         "W1": rng.normal(size=(S.NH, S.NF)) / 3, "b1": rng.normal(size=S.NH) / 3,
         "W2": rng.normal(size=(S.NH, S.NH)) / 8, "b2": rng.normal(size=S.NH) / 3,
         "w3": rng.normal(size=S.NH) / 8, "b3": 0.1}
    return p


def test_mlp_gradient_matches_finite_differences():
    """Analytic gradient of the mean cross-entropy against central differences (FP64)."""
    rng = np.random.default_rng(1)
    p = _rand_model(2)
    X = rng.normal(size=(40, S.NF))
    y = (rng.random(40) < 0.5).astype(float)
    g = S.mlp_grad(p, X, y)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3"):
        arr = p[name]
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
            old = arr[idx]
            arr[idx] = old + h
            lp = S.mlp_loss(p, X, y)
            arr[idx] = old - h
            lm = S.mlp_loss(p, X, y)
            arr[idx] = old
            assert abs((lp - lm) / (2 * h) - g[name][idx]) < 1e-7, (name, idx)
    b3 = p["b3"]
    p["b3"] = b3 + h
    lp = S.mlp_loss(p, X, y)
    p["b3"] = b3 - h
    lm = S.mlp_loss(p, X, y)
    p["b3"] = b3
    assert abs((lp - lm) / (2 * h) - g["b3"]) < 1e-7


def test_mlp_constant_logit_closed_form():
    """With every weight zero the logit is b3 for every sample: the loss is
    log(1 + e^b3) - mean(y) b3, dL/db3 = sigmoid(b3) - mean(y), all other gradients 0."""
    p = {k: np.zeros_like(v) if isinstance(v, np.ndarray) else 0.0 for k, v in _rand_model(3).items()}
    p["std"] = np.ones(S.NF)
    p["b3"] = 0.7
    rng = np.random.default_rng(4)
    X = rng.normal(size=(25, S.NF))
    y = (rng.random(25) < 0.3).astype(float)
    assert abs(S.mlp_loss(p, X, y) - (np.log1p(np.exp(0.7)) - y.mean() * 0.7)) < 1e-14
    g = S.mlp_grad(p, X, y)
    assert abs(g["b3"] - (1 / (1 + np.exp(-0.7)) - y.mean())) < 1e-14
    for k in ("W1", "b1", "W2", "b2", "w3"):
        assert np.all(g[k] == 0)


def test_mlp_pack_roundtrip_and_fp16():
    p = _rand_model(5)
    m = S.mlp_pack(p).astype(np.float32)
    assert m.size == S.NPARAMS == 5081
    q = S.mlp_unpack(m, fp16=True)
    # weights are FP16 values, the normalisation stays FP32
    assert np.array_equal(q["W2"], q["W2"].astype(np.float16).astype(np.float64))
    assert np.array_equal(q["mean"], p["mean"].astype(np.float32).astype(np.float64))
