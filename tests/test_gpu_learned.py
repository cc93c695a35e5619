"""GPU tests of the learned skip: classifier kernels against the FP64 oracle, recorded
features and labels against the oracle's definition, the skip inside the factorization."""
import numpy as np
import pytest

import oracle as O
from oracle import skip_oracle as S
import paper_1908_10169_gb300 as B
from paper_1908_10169_gb300 import learned_skip as LS
from paper_1908_10169_gb300 import workloads as W
from tests.gpu_helpers import gpu_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.bilu_create(0)
    yield c
    B.bilu_destroy(c)


def _samples(seed, n):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, S.NF)).astype(np.float32) * np.linspace(0.5, 3, S.NF).astype(np.float32)
    x += np.linspace(-2, 2, S.NF).astype(np.float32)
    y = ((x[:, 0] + 0.5 * x[:, 3] - x[:, 7] + rng.normal(size=n) * 0.3) > 0).astype(np.float32)
    return x, y


def _init_model(ctx, x, y, seed=3):
    """Initial weights and the data's normalisation: zero epochs of training."""
    model, _ = B.bilu_mlp_train(ctx, x, y, epochs=0, seed=seed)
    return model


def test_mlp_forward_and_gradient_match_oracle(ctx):
    """Logits and the loss gradient of the CUDA kernels (FP16 weights, FP32 accumulation)
    against the FP64 oracle at the same FP16-rounded weights."""
    x, y = _samples(1, 3000)
    model, _ = B.bilu_mlp_train(ctx, x, y, epochs=1, batch=512, seed=5)  # a trained, non-trivial point
    p = S.mlp_unpack(model)
    z_ref, _ = S.mlp_forward(p, x.astype(np.float64))
    z = np.zeros(len(y), np.float32)
    B.bilu_mlp_forward(ctx, model, x, z)
    assert np.max(np.abs(z - z_ref) / (1 + np.abs(z_ref))) < 2e-5
    g = B.bilu_mlp_grad(ctx, model, x, y)
    gr = S.mlp_pack(S.mlp_grad(p, x.astype(np.float64), y.astype(np.float64)))
    for name, lo, hi in (("W1", 24, 792), ("b1", 792, 856), ("W2", 856, 4952), ("b2", 4952, 5016),
                         ("w3", 5016, 5080), ("b3", 5080, 5081)):
        scale = max(np.max(np.abs(gr[lo:hi])), 1e-12)
        assert np.max(np.abs(g[lo:hi] - gr[lo:hi])) / scale < 1e-3, name
    assert np.all(g[:24] == 0)


def test_mlp_training_is_deterministic_and_learns(ctx):
    x, y = _samples(2, 20000)
    m1, l1 = B.bilu_mlp_train(ctx, x, y, epochs=3, batch=1024, lr=3e-3, seed=11)
    m2, l2 = B.bilu_mlp_train(ctx, x, y, epochs=3, batch=1024, lr=3e-3, seed=11)
    assert np.array_equal(m1, m2) and l1 == l2
    m0, l0 = B.bilu_mlp_train(ctx, x, y, epochs=0, seed=11)
    assert l1 < 0.5 * l0
    z = np.zeros(len(y), np.float32)
    B.bilu_mlp_forward(ctx, m1, x, z)
    assert np.mean((z > 0) == (y > 0.5)) > 0.9


def _recorded(ctx, w, bs_block):
    p = B.bilu_params_default(fixed_block=bs_block, max_block=64)
    B.bilu_analyze(ctx, w.A.n, w.A.rowptr, w.A.colind, w.A.val, p)
    B.bilu_record_samples(ctx, 10 ** 6, 1.0, 0)
    try:
        B.bilu_factor(ctx, w.droptol)
        m = B.bilu_get_samples(ctx)
        x = np.zeros((m, S.NF), np.float32)
        y = np.zeros(m, np.float32)
        t = np.zeros(m, np.int64)
        B.bilu_get_samples(ctx, x, y, t, m)
    finally:
        B.bilu_record_samples(ctx, 0)
    o = np.argsort(t)
    return x[o], y[o], t[o]


@pytest.mark.parametrize("case", ["cd2d_32", "cd3d_10", "cd3d_12_b24"])
def test_recorded_features_match_oracle(ctx, case):
    """Every candidate's features (recording at rate 1) equal the oracle's definition, its
    label (dropped or kept) exactly."""
    if case == "cd2d_32":
        w, blk = W.cd2d_32(), 32
    elif case == "cd3d_10":
        w, blk = W.cd3d(side=10, seed=4, block=10), 10
    else:
        w, blk = W.cd3d(side=12, seed=5, block=24), 24
    x, y, t = _recorded(ctx, w, blk)
    bs = np.arange(0, w.A.n + 1, blk)
    if bs[-1] != w.A.n:
        bs = np.append(bs, w.A.n)
    F = O.bilu_factor(w.A, bs, w.droptol)
    xr, yr, tr = S.skip_features(w.A, F, w.droptol)
    assert np.array_equal(t, tr)
    assert np.array_equal(y, yr)
    assert np.max(np.abs(x - xr)) < 2e-5


def test_recording_keeps_only_the_final_run(ctx):
    """A factorization re-run with grown storage records its candidates once."""
    w = W.cd3d(side=10, seed=4, block=10)
    x1, y1, t1 = _recorded(ctx, w, 10)
    c = B.bilu_create(0)
    try:
        B.bilu_debug_set(c, B.BILU_DEBUG_SMALL_POOLS, 1)
        x2, y2, t2 = _recorded(c, w, 10)
        assert B.bilu_stats(c).pool_retries > 0
    finally:
        B.bilu_debug_set(c, B.BILU_DEBUG_SMALL_POOLS, 0)
        B.bilu_destroy(c)
    assert np.array_equal(t1, t2) and np.array_equal(y1, y2) and np.array_equal(x1, x2)


def test_learned_skip_without_false_drops_gives_the_exact_factor(ctx):
    """With the threshold above every kept candidate's logit the skipped candidates are
    exactly those with logit >= threshold, all of them dropped ones: the factor is the exact
    factor bit for bit, with fewer update flops."""
    w = W.cd3d(side=12, seed=5, block=12)
    x, y, t = _recorded(ctx, w, 12)
    model, _ = B.bilu_mlp_train(ctx, x, y, epochs=20, batch=256, lr=3e-3, seed=1)
    z = np.zeros(len(y), np.float32)
    B.bilu_mlp_forward(ctx, model, x, z)
    hi = float(np.nextafter(np.float32(z[y == 0].max()), np.float32(np.inf)))
    expect_skip = int(np.sum(z >= hi))
    assert expect_skip > 0
    p = B.bilu_params_default(fixed_block=12, max_block=64)
    ref = gpu_factor(ctx, w.A, w.droptol, p)
    c = B.bilu_create(0)
    try:
        B.bilu_set_skip_model(c, model, hi)
        g = gpu_factor(c, w.A, w.droptol, B.bilu_params_default(fixed_block=12, max_block=64, skip=B.BILU_SKIP_LEARNED))
        s = B.bilu_stats(c)
    finally:
        B.bilu_destroy(c)
    assert s.skipped_rows + s.skipped_cols == expect_skip
    for k in ("Lptr", "Lrow", "Lval", "Uptr", "Ucol", "Uval", "Dinv", "Pblk"):
        assert np.array_equal(getattr(g, k), getattr(ref, k)), k
    assert s.flop_upd_l + s.flop_upd_u < ref.stats.flop_upd_l + ref.stats.flop_upd_u


def test_learned_skip_needs_a_model(ctx):
    w = W.cd2d_32()
    c = B.bilu_create(0)
    try:
        B.bilu_analyze(c, w.A.n, w.A.rowptr, w.A.colind, w.A.val,
                       B.bilu_params_default(fixed_block=32, max_block=64, skip=B.BILU_SKIP_LEARNED))
        with pytest.raises(B.BiluError):
            B.bilu_factor(c, w.droptol)
    finally:
        B.bilu_destroy(c)


def test_learned_skip_gain_on_held_out_problem(ctx):
    """Trained on small 3D problems (seeds 1000..), applied to a held-out one, against the
    exact norm-bound skip (BILU_SKIP_BOUND, the method without the classifier that skips only
    what it can prove dropped) and against no skip: the classifier skips candidates before
    their updates, so its update flops are below both; GMRES(30) stays within 10 % of the
    iterations of the exact factor.  (Without a skip, the scaling phase already drops, unscaled,
    every candidate whose norm bound is below tau: the total flops of the three differ mainly in
    the updates.)"""
    import torch
    train = list(W.cd3d_skip_train(count=12, seed0=1000, side_lo=14, side_hi=20, block=64))
    x, y = LS.record(train, rate=0.5, cap_per_problem=200000)
    sm = LS.train(x, y, epochs=6, batch=2048, lr=3e-3, seed=2, max_false_drop=2e-3)
    assert sm.skip_rate > 0.05
    w = W.cd3d(side=24, seed=77, block=64)
    bt = torch.from_numpy(w.b).cuda()
    res = {}
    for mode in (B.BILU_SKIP_NONE, B.BILU_SKIP_BOUND, B.BILU_SKIP_LEARNED):
        c = B.bilu_create(0)
        try:
            if mode == B.BILU_SKIP_LEARNED:
                B.bilu_set_skip_model(c, sm.model, sm.logit_hi)
            gpu_factor(c, w.A, w.droptol, B.bilu_params_default(fixed_block=64, max_block=64, skip=mode), export=False)
            s = B.bilu_stats(c)
            x0 = torch.zeros_like(bt)
            info = B.gmres_solve(c, bt, x0, 1e-8, 30, 10000)
            res[mode] = (s, info)
        finally:
            B.bilu_destroy(c)
    s0, i0 = res[B.BILU_SKIP_NONE]
    sb, ib = res[B.BILU_SKIP_BOUND]
    s1, i1 = res[B.BILU_SKIP_LEARNED]
    upd = {k: v[0].flop_upd_l + v[0].flop_upd_u for k, v in res.items()}
    print(f"update flops: none {upd[B.BILU_SKIP_NONE]}, bound {upd[B.BILU_SKIP_BOUND]}, learned "
          f"{upd[B.BILU_SKIP_LEARNED]}; total flops {s0.flops_factor:.4g} / {sb.flops_factor:.4g} / "
          f"{s1.flops_factor:.4g}; skipped bound {sb.skipped_rows + sb.skipped_cols}, learned "
          f"{s1.skipped_rows + s1.skipped_cols}; GMRES {i0.iters} / {ib.iters} / {i1.iters}")
    assert s1.skipped_rows + s1.skipped_cols > sb.skipped_rows + sb.skipped_cols > 0
    assert upd[B.BILU_SKIP_LEARNED] < upd[B.BILU_SKIP_BOUND] < upd[B.BILU_SKIP_NONE]
    assert ib.iters == i0.iters  # the exact skip gives the same factor
    assert i1.relres_true <= 1e-8
    assert i1.iters <= 1.1 * i0.iters + 1, (i1.iters, i0.iters)
