"""Randomised parity of the library's host analysis (Sec. 3.1-3.4) with the oracles: small
random patterns (empty and full rows, single unknowns, disconnected parts, structurally
singular matrices) drawn by hypothesis, compared bit for bit (cosine, ILU(1,tau), dissection,
elimination tree) or by the unique optimum (matching)."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle as O  # noqa: E402
import paper_1908_10169_gb300 as B  # noqa: E402
from oracle import cosine_oracle as C  # noqa: E402
from oracle import mwm_oracle as M  # noqa: E402
from oracle import nd_oracle as N  # noqa: E402
from paper_1908_10169_gb300 import workloads as W  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@st.composite
def matrices(draw, max_n=24, diagonal=True):
    n = draw(st.integers(0, max_n))
    density = draw(st.sampled_from([0.0, 0.05, 0.2, 0.5, 1.0]))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    d = (rng.random((n, n)) < density) * rng.uniform(-2.0, 2.0, (n, n))
    if diagonal and n:
        d[np.arange(n), np.arange(n)] = rng.uniform(2.0, 6.0, n) * (1 + (rng.random(n) < 0.2) * 10)
    return W.from_dense(d, keep_zeros_on_diag=False), rng


def partition(rng, n, max_block):
    bs = [0]
    while bs[-1] < n:
        bs.append(min(n, bs[-1] + int(rng.integers(1, max_block + 1))))
    return np.array(bs, dtype=np.int32)


@SETTINGS
@given(matrices(), st.sampled_from([0.0, 0.5, 0.8, 1.0]), st.sampled_from([1, 2, 3, 64]))
def test_cosine(m, tau, mb):
    A, _ = m
    p, b = B.bilu_cosine_blocking(A.n, A.rowptr, A.colind, tau, mb)
    po, bo = C.cosine_blocking(A, tau, mb)
    assert np.array_equal(p, po) and np.array_equal(b, bo)


@SETTINGS
@given(matrices(), st.sampled_from([0.0, 1e-2, 0.3]), st.sampled_from([1, 3, 8, 64]), st.booleans())
def test_ilu1t(m, tau, mb, grouped):
    A, rng = m
    groups = partition(rng, A.n, mb) if grouped else None
    got = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, tau, mb, groups)
    want = (O.partition_ilu1t_groups(A, tau, mb, groups) if grouped else O.partition_ilu1t(A, tau, mb))
    assert np.array_equal(got, want)


@SETTINGS
@given(matrices(), st.sampled_from([1, 2, 4]), st.sampled_from([1, 2]))
def test_dissection_and_tree(m, mb, leaf):
    A, rng = m
    bs = partition(rng, A.n, mb)
    got = B.bilu_nd_order(A.n, A.rowptr, A.colind, bs, leaf)
    want = N.nd_order(A, bs, leaf)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    parent, height = B.bilu_block_etree(A.n, A.rowptr, A.colind, bs)
    assert np.array_equal(parent, N.block_etree(A, bs))


@SETTINGS
@given(matrices(max_n=14, diagonal=False))
def test_matching(m):
    A, _ = m
    try:
        _, _, _, _, _, total = M.mwm(A)
    except ValueError:
        with pytest.raises(B.BiluError) as e:
            B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
        assert e.value.status == B.BILU_ERR_SINGULAR
        return
    sigma, dl, dr = B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
    Cm, _ = M.costs(A)
    assert sorted(sigma) == list(range(A.n))
    assert abs(sum(Cm[i, sigma[i]] for i in range(A.n)) - total) <= 1e-11 * max(1.0, abs(total))
    d = A.to_dense()
    Ah = dl[:, None] * d * dr[None, :]
    assert np.all(np.abs(Ah) <= 1 + 1e-12)
    if A.n:
        assert np.allclose(np.abs(Ah[np.arange(A.n), sigma]), 1.0, rtol=0, atol=1e-12)
