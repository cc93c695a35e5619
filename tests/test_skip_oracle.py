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


def _dense_features(A, F, tau):
    """The same features computed another way: from dense n x n copies of A (with its stored
    pattern as a boolean mask), of L and of U-breve (kept rows / columns only, diagonal
    blocks left out), with producers and candidates found by tests on dense slices."""
    n = A.n
    bs = np.asarray(F.bstart, dtype=np.int64)
    nb = len(bs) - 1
    Ad = A.to_dense()
    pat = np.zeros((n, n), bool)
    pat[np.repeat(np.arange(n), np.diff(A.rowptr)), A.colind] = True
    Ld, Ud = np.zeros((n, n)), np.zeros((n, n))
    keptL, keptU = np.zeros((nb, n), bool), np.zeros((nb, n), bool)
    for J in range(nb):
        rows, lv = F.L_block(J)
        cols, uv = F.U_block(J)
        Ld[rows, bs[J]:bs[J + 1]] = lv
        Ud[bs[J]:bs[J + 1], cols] = uv.T
        keptL[J, rows] = True
        keptU[J, cols] = True
    alpha = np.abs(A.val).max()
    xs, ys, tags = [], [], []
    for K in range(nb):
        s0, s1 = bs[K], bs[K + 1]
        d = np.linalg.norm(F.D_block(K - 1)) if K > 0 else 1.0 / alpha
        for side in (0, 1):
            if side == 0:   # rows i >= s1 of the block column
                Aside, Pside, Xd, keptX, keptY = Ad[:, s0:s1], pat[:, s0:s1], Ld, keptL, keptU
                Yblk = lambda J: Ud[bs[J]:bs[J + 1], s0:s1]
                Xrow = lambda J, i: Ld[i, bs[J]:bs[J + 1]]
            else:           # columns j >= s1 of the block row
                Aside, Pside, Xd, keptX, keptY = Ad[s0:s1, :].T, pat[s0:s1, :].T, Ud, keptU, keptL
                Yblk = lambda J: Ld[s0:s1, bs[J]:bs[J + 1]]
                Xrow = lambda J, i: Ud[bs[J]:bs[J + 1], i]
            prods = [J for J in range(K) if keptY[J, s0:s1].any()]
            for i in range(s1, n):
                mine = [J for J in prods if keptX[J, i]]
                stored = bool(Pside[i].any())
                if not stored and not mine:
                    continue
                a = np.linalg.norm(Aside[i])
                v = [np.linalg.norm(Xrow(J, i)) * np.linalg.norm(Yblk(J)) for J in mine]
                widths = [bs[J + 1] - bs[J] for J in mine]
                S_, M_ = float(np.sum(v)), float(np.max(v)) if v else 0.0
                xs.append([_lg(a), float(stored), _lg(S_), _lg(M_), np.log2(1 + len(mine)), _lg(d),
                           _lg((a + S_) * d), _lg(tau), (s1 - s0) / 64, np.mean(widths) / 64 if mine else 0.0,
                           np.log2(1 + (i - s1) / 64), side])
                ys.append(0.0 if (keptL if side == 0 else keptU)[K, i] else 1.0)
                tags.append((K << 33) | (side << 32) | i)
    return np.array(xs), np.array(ys), np.array(tags, dtype=np.int64)


@pytest.mark.parametrize("case", ["cd3d", "random"])
def test_features_match_dense_computation(case):
    """Several producers per candidate (3D stencil, lines of 8) and several entries of A per
    candidate in B_K (random matrix, uneven blocks): the features agree with the dense
    computation to rounding, labels and tags exactly."""
    if case == "cd3d":
        w = W.cd3d(side=6, seed=2, block=6)
        A, bs, tau = w.A, np.arange(0, w.A.n + 1, 6), w.droptol
    else:
        A = W.random_diag_dominant(90, 0.08, seed=5)
        bs, tau = np.array([0, 5, 17, 30, 34, 52, 60, 77, 90]), 3e-2
    F = O.bilu_factor(A, bs, tau)
    x, y, t = S.skip_features(A, F, tau)
    xd, yd, td = _dense_features(A, F, tau)
    assert np.array_equal(t, td) and np.array_equal(y, yd)
    assert np.max(np.abs(x - xd)) < 1e-12
    # the cases exercise what they are meant to: several producers, several entries, both labels
    assert x[:, 4].max() >= np.log2(4) and 0 < y.mean() < 1
    if case == "random":  # a candidate row with two or more stored entries in its block column
        pat = A.to_dense() != 0
        assert any((pat[bs[K + 1]:, bs[K]:bs[K + 1]].sum(axis=1) >= 2).any() for K in range(len(bs) - 1))


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


def test_mlp_forward_closed_form():
    """A hand-set network that computes |x_0 - mean_0| / std_0 - 1/2: h1 = (relu(z), relu(-z))
    for the normalised z, h2_0 = h1_0 + h1_1 + 1/2 = |z| + 1/2, h2_1 = relu(-h1_0) = 0, and
    z_out = h2_0 + h2_1 - 1."""
    rng = np.random.default_rng(6)
    p = {"mean": rng.normal(size=S.NF), "std": rng.uniform(0.5, 3.0, size=S.NF),
         "W1": np.zeros((S.NH, S.NF)), "b1": np.zeros(S.NH), "W2": np.zeros((S.NH, S.NH)),
         "b2": np.zeros(S.NH), "w3": np.zeros(S.NH), "b3": -1.0}
    p["W1"][0, 0], p["W1"][1, 0] = 1.0, -1.0
    p["W2"][0, 0], p["W2"][0, 1], p["W2"][1, 0] = 1.0, 1.0, -1.0
    p["b2"][0] = 0.5
    p["w3"][0], p["w3"][1] = 1.0, 1.0
    X = rng.normal(size=(50, S.NF)) * 3
    z, _ = S.mlp_forward(p, X)
    np.testing.assert_allclose(z, np.abs(X[:, 0] - p["mean"][0]) / p["std"][0] - 0.5, rtol=0, atol=1e-13)
