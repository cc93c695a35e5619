"""The learned skip's threshold choice (host logic): the smallest FP32 threshold that lets at
most the allowed share of kept samples (label 0) through as false drops."""
import numpy as np

from paper_1908_10169_gb300 import learned_skip as LS


def f32(x):
    return np.float32(x)


def test_hand_cases():
    z = np.array([0.5, 0.1, -0.3, -1.0, 2.0, 1.0], np.float32)
    y = np.array([0, 0, 0, 0, 1, 1], np.float32)
    # 25 % of 4 kept samples: one may pass; the threshold sits just above the second largest
    t = LS.logit_threshold(z, y, 0.25)
    assert f32(t) == np.nextafter(f32(0.1), f32(np.inf))
    assert np.sum(z[y == 0] >= f32(t)) == 1 and np.all(z[y == 1] >= f32(t))
    # no false drop allowed: just above the largest kept logit
    assert f32(LS.logit_threshold(z, y, 0.0)) == np.nextafter(f32(0.5), f32(np.inf))
    # ties at the cut are all kept out: kept (0.5, 0.5, 0.1), one may pass, none does
    z2 = np.array([0.5, 0.5, 0.1, 3.0], np.float32)
    y2 = np.array([0, 0, 0, 1], np.float32)
    t2 = LS.logit_threshold(z2, y2, 0.34)
    assert f32(t2) == np.nextafter(f32(0.5), f32(np.inf)) and np.sum(z2[y2 == 0] >= f32(t2)) == 0
    # no kept sample: everything may be skipped
    assert LS.logit_threshold(np.array([1.0, 2.0], np.float32), np.ones(2, np.float32), 0.0) == 1.0


def test_bound_holds_and_is_tight():
    rng = np.random.default_rng(0)
    for trial in range(50):
        n = int(rng.integers(5, 400))
        z = rng.normal(size=n).astype(np.float32)
        y = (rng.random(n) < 0.5).astype(np.float32)
        fd = float(rng.choice([0.0, 0.002, 0.05, 0.3]))
        t = f32(LS.logit_threshold(z, y, fd))
        kept = z[y == 0]
        if kept.size == 0:
            continue
        allow = int(np.floor(fd * kept.size))
        assert np.sum(kept >= t) <= allow
        # one FP32 step lower lets one kept sample too many through
        lower = np.nextafter(t, f32(-np.inf))
        assert np.sum(kept >= lower) > allow
