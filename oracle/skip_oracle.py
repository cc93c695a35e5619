"""Plain FP64 reference of the learned skip: candidate features, labels and the classifier.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the test suite may use it; the
product never imports it.

The paper drops a row of L (column of U) after computing it when its norm is <= tau (Sec. 3,
the block form of Algorithm 1).  The learned skip predicts that outcome from features that
are available before the row's Schur updates; this module states those features and the
classifier plainly:

* ``skip_features`` computes, from an exported oracle factor, for every block K and every
  candidate row i >= s_K of the L side (column j >= s_K of the U side), the 12 features and
  the label (1 = dropped) -- by their definitions, with Python loops over the kept sets.
* ``mlp_*`` is the 3-layer classifier (F -> 64 -> 64 -> 1, ReLU) in float64 numpy, with its
  binary cross-entropy and the analytic gradient.

Candidate sets (structural, reading Q8 of the oracle): L side of block K = rows i >= s_K with a
stored entry of A in columns B_K, or a kept row of L_J for a producer J (an earlier block with
a kept column of U-breve_J in B_K); U side likewise with rows of A in B_K and kept columns of
U-breve_J for producers J with a kept row of L_J in B_K.

Features (lg x = log10(max(x, 1e-30))), for a candidate with producers J (those whose kept
rows (columns) contain it), X_J its row of L_J (column of U-breve_J), Y_J = L_J's kept rows in
B_K (U side) or U-breve_J's kept columns in B_K (L side):
  0 lg a, a = ||A(i, B_K)||_2            1 1 if A(i, B_K) has a stored entry
  2 lg s, s = sum_J ||X_J|| ||Y_J||_F     3 lg max_J ||X_J|| ||Y_J||_F
  4 log2(1 + #producers)                 5 lg d, d = ||D_{K-1}||_F (1 / max|a_ij| for K = 0)
  6 lg ((a + s) d)                       7 lg tau
  8 b_K / 64                             9 mean b_J / 64 (0 without producers)
  10 log2(1 + (i - s_K) / 64)            11 side (0 L, 1 U)
"""
from __future__ import annotations

import numpy as np

NF = 12
NH = 64
NPARAMS = 2 * NF + NH * NF + NH + NH * NH + NH + NH + 1


def _lg(x: float) -> float:
    return float(np.log10(max(x, 1e-30)))


def skip_features(A, F, tau: float):
    """Features, labels and tags of every candidate of the factorization F of A (an oracle
    Factor from ``oracle.bilu_factor``).  Returns (x [m, 12] float64, y [m] float64, tags [m]
    int64) with tag = K * 2^33 + side * 2^32 + global index, in increasing tag order."""
    bs = np.asarray(F.bstart, dtype=np.int64)
    nb = len(bs) - 1
    n = A.n
    alpha = float(np.max(np.abs(A.val))) if A.val.size else 0.0
    rp, ci, va = A.rowptr, A.colind, A.val
    # column access of A
    order = np.lexsort((np.repeat(np.arange(n), np.diff(rp)), ci))
    ccol = ci[order]
    crow = np.repeat(np.arange(n), np.diff(rp))[order]
    cval = va[order]
    cptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(ccol, minlength=n), out=cptr[1:])

    # kept rows of L_J (normalised, b_J values each) and kept columns of U-breve_J
    Lrows, Lnorm, Ucols, Unorm, Dfro = [], [], [], [], []
    Lvp = Uvp = 0
    for J in range(nb):
        bJ = int(bs[J + 1] - bs[J])
        lr = F.Lrow[F.Lptr[J]:F.Lptr[J + 1]]
        uc = F.Ucol[F.Uptr[J]:F.Uptr[J + 1]]
        lv = F.Lval[Lvp:Lvp + len(lr) * bJ].reshape(len(lr), bJ)
        uv = F.Uval[Uvp:Uvp + len(uc) * bJ].reshape(len(uc), bJ)
        Lvp += len(lr) * bJ
        Uvp += len(uc) * bJ
        Lrows.append({int(i): k for k, i in enumerate(lr)})
        Ucols.append({int(j): k for k, j in enumerate(uc)})
        Lnorm.append(np.sqrt(np.sum(lv * lv, axis=1)))
        Unorm.append(np.sqrt(np.sum(uv * uv, axis=1)))
    dp = 0
    for K in range(nb):
        b = int(bs[K + 1] - bs[K])
        D = F.Dinv[dp:dp + b * b]
        dp += b * b
        Dfro.append(float(np.sqrt(np.sum(D * D))))

    xs, ys, tags = [], [], []
    for K in range(nb):
        s0, s1 = int(bs[K]), int(bs[K + 1])
        b = s1 - s0
        d = Dfro[K - 1] if K > 0 else (1.0 / alpha if alpha > 0 else 1.0)
        for side in (0, 1):
            # producers: earlier blocks whose kept U columns (side 0) / L rows (side 1) hit B_K
            prods = []
            for J in range(K):
                Yset = Ucols[J] if side == 0 else Lrows[J]
                Ynorms = Unorm[J] if side == 0 else Lnorm[J]
                ys_in = [k for idx, k in Yset.items() if s0 <= idx < s1]
                if ys_in:
                    yf = float(np.sqrt(sum(Ynorms[k] ** 2 for k in ys_in)))
                    prods.append((J, yf))
            # A part of every candidate
            apart = {}
            if side == 0:
                for c in range(s0, s1):
                    for e in range(cptr[c], cptr[c + 1]):
                        i = int(crow[e])
                        if i >= s1:
                            apart.setdefault(i, 0.0)
                            apart[i] += float(cval[e]) ** 2
            else:
                for r in range(s0, s1):
                    for e in range(rp[r], rp[r + 1]):
                        j = int(ci[e])
                        if j >= s1:
                            apart.setdefault(j, 0.0)
                            apart[j] += float(va[e]) ** 2
            cand = set(apart)
            for J, _ in prods:
                Xset = Lrows[J] if side == 0 else Ucols[J]
                cand.update(i for i in Xset if i >= s1)
            kept = Lrows[K] if side == 0 else Ucols[K]
            for i in sorted(cand):
                a = float(np.sqrt(apart[i])) if i in apart else 0.0
                S, M, C, SB = 0.0, 0.0, 0, 0
                for J, yf in prods:
                    Xset = Lrows[J] if side == 0 else Ucols[J]
                    if i in Xset:
                        xn = float((Lnorm[J] if side == 0 else Unorm[J])[Xset[i]])
                        v = xn * yf
                        S += v
                        M = max(M, v)
                        C += 1
                        SB += int(bs[J + 1] - bs[J])
                f = [_lg(a), 1.0 if i in apart else 0.0, _lg(S), _lg(M), float(np.log2(1.0 + C)), _lg(d),
                     _lg((a + S) * d), _lg(tau), b / 64.0, (SB / C / 64.0) if C else 0.0,
                     float(np.log2(1.0 + max(0, i - s1) / 64.0)), float(side)]
                xs.append(f)
                ys.append(0.0 if i in kept else 1.0)
                tags.append((K << 33) | (side << 32) | i)
    return np.array(xs, dtype=np.float64).reshape(-1, NF), np.array(ys), np.array(tags, dtype=np.int64)


# ---- classifier ----------------------------------------------------------------------------

def mlp_unpack(model: np.ndarray, fp16: bool = True) -> dict:
    """Split a model array (mean, std, W1, b1, W2, b2, w3, b3) into float64 arrays; the weights
    are rounded to FP16 first when fp16 (as wherever the model is used)."""
    m = np.asarray(model, dtype=np.float32)
    assert m.size == NPARAMS
    o = 0

    def take(k, shape=None, half=True):
        nonlocal o
        v = m[o:o + k]
        o += k
        if half and fp16:
            v = v.astype(np.float16)
        v = v.astype(np.float64)
        return v.reshape(shape) if shape else v

    p = {"mean": take(NF, half=False), "std": take(NF, half=False)}
    p["W1"] = take(NH * NF, (NH, NF))
    p["b1"] = take(NH)
    p["W2"] = take(NH * NH, (NH, NH))
    p["b2"] = take(NH)
    p["w3"] = take(NH)
    p["b3"] = take(1)[0]
    return p


def mlp_pack(p: dict) -> np.ndarray:
    return np.concatenate([p["mean"], p["std"], p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["w3"],
                           [p["b3"]]]).astype(np.float64)


def mlp_forward(p: dict, X: np.ndarray):
    """Logits and the activations: xs = (x - mean) / std, h1 = relu(W1 xs + b1),
    h2 = relu(W2 h1 + b2), z = w3 . h2 + b3."""
    xs = (np.asarray(X, np.float64) - p["mean"]) / p["std"]
    a1 = xs @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"] + p["b3"]
    return z, (xs, a1, h1, a2, h2)


def mlp_loss(p: dict, X: np.ndarray, y: np.ndarray) -> float:
    """Mean binary cross-entropy of the logits: mean(log(1 + e^z) - y z)."""
    z, _ = mlp_forward(p, X)
    return float(np.mean(np.logaddexp(0.0, z) - y * z))


def mlp_grad(p: dict, X: np.ndarray, y: np.ndarray) -> dict:
    """Gradient of mlp_loss by the chain rule (dL/dz = (sigmoid(z) - y) / n)."""
    z, (xs, a1, h1, a2, h2) = mlp_forward(p, X)
    n = len(y)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n
    g = {"mean": np.zeros(NF), "std": np.zeros(NF)}
    g["w3"] = h2.T @ dz
    g["b3"] = float(np.sum(dz))
    da2 = np.outer(dz, p["w3"]) * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ p["W2"]) * (a1 > 0)
    g["W1"] = da1.T @ xs
    g["b1"] = da1.sum(axis=0)
    return g
