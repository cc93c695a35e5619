"""Training pipeline of the learned skip (BILU_SKIP_LEARNED).

Every numerical step runs in the library's kernels: the factorization records (features,
label) samples of its candidates (bilu_record_samples), the classifier is trained by the
library's own forward / backward / Adam kernels (bilu_mlp_train), and its logits come from the
library's inference kernel (bilu_mlp_forward).  This module only drives those calls and picks
the logit threshold from the logits (a quantile on the host).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import (BILU_MLP_FEATURES, BILU_PREC_FP64, bilu_analyze, bilu_create, bilu_destroy, bilu_factor,
               bilu_get_samples, bilu_mlp_forward, bilu_mlp_train, bilu_params_default, bilu_record_samples,
               bilu_stats)


@dataclasses.dataclass
class SkipModel:
    model: np.ndarray       # BILU_MLP_PARAMS float32
    logit_hi: float         # skip when logit >= logit_hi
    train_loss: float
    samples: int
    drop_fraction: float    # share of dropped candidates in the training samples
    false_drop_rate: float  # kept training samples with logit >= logit_hi, over all kept ones
    skip_rate: float        # training samples with logit >= logit_hi, over all samples


def record(problems, device: int = 0, rate: float = 0.05, cap_per_problem: int = 200000, seed: int = 7,
           precision: int = BILU_PREC_FP64):
    """Factor each Workload exactly with sample recording; returns (x [m, F] float32, y [m])."""
    import torch
    dev = torch.device("cuda", device)
    xs, ys = [], []
    for k, w in enumerate(problems):
        ctx = bilu_create(device)
        try:
            bilu_analyze(ctx, w.A.n, torch.from_numpy(w.A.rowptr).to(dev), torch.from_numpy(w.A.colind).to(dev),
                         torch.from_numpy(w.A.val).to(dev),
                         bilu_params_default(fixed_block=w.fixed_block, max_block=64, precision=precision))
            bilu_record_samples(ctx, cap_per_problem, rate, seed + k)
            bilu_factor(ctx, w.droptol)
            m = bilu_get_samples(ctx)
            m = min(m, cap_per_problem)
            x = np.zeros((m, BILU_MLP_FEATURES), np.float32)
            y = np.zeros(m, np.float32)
            bilu_get_samples(ctx, x, y, None, m)
            xs.append(x)
            ys.append(y)
        finally:
            bilu_destroy(ctx)
    return np.concatenate(xs), np.concatenate(ys)


def logit_threshold(logits: np.ndarray, y: np.ndarray, max_false_drop: float) -> float:
    """Smallest threshold t such that at most max_false_drop of the kept samples (y = 0) have
    a logit >= t (t is just above that kept sample's logit)."""
    kept = np.sort(logits[y == 0])[::-1]
    allow = int(np.floor(max_false_drop * kept.size))
    if kept.size == 0:
        return float(np.min(logits)) if logits.size else 0.0
    return float(np.nextafter(np.float32(kept[allow]), np.float32(np.inf))) if allow < kept.size else float(kept[-1])


def train(x: np.ndarray, y: np.ndarray, device: int = 0, epochs: int = 4, batch: int = 4096, lr: float = 2e-3,
          seed: int = 0, max_false_drop: float = 2e-3) -> SkipModel:
    """Train the classifier on the samples and choose the logit threshold."""
    ctx = bilu_create(device)
    try:
        model, loss = bilu_mlp_train(ctx, x, y, epochs=epochs, batch=batch, lr=lr, seed=seed)
        logits = np.zeros(y.shape[0], np.float32)
        bilu_mlp_forward(ctx, model, x, logits)
    finally:
        bilu_destroy(ctx)
    t = logit_threshold(logits, y, max_false_drop)
    kept = y == 0
    fd = float(np.mean(logits[kept] >= t)) if kept.any() else 0.0
    return SkipModel(model, t, loss, int(y.size), float(np.mean(y)), fd, float(np.mean(logits >= t)))
