"""Pins of the synthetic matrix generators to closed forms: stencil sizes, symmetry, positive
definiteness, rigid-body modes of the elasticity element, row sums of the diffusion element."""
import numpy as np

from paper_1908_10169_gb300 import workloads as W


def test_q1_elasticity_element():
    Ke = W.q1_elasticity_element(0.3)
    assert np.abs(Ke - Ke.T).max() < 1e-14
    ev = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(ev) < 1e-12) == 6 and ev[6] > 1e-3  # 3 translations + 3 rotations
    x = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], float)
    rot = np.zeros(24)
    rot[0::3], rot[1::3] = -x[:, 1], x[:, 0]  # rotation about z
    assert np.abs(Ke @ rot).max() < 1e-12


def test_q1_laplace_element():
    L = W.q1_laplace_element()
    assert np.abs(L.sum(axis=1)).max() < 1e-15
    assert abs(L[0, 0] - 1.0 / 3.0) < 1e-15  # the Q1 stiffness diagonal on the unit cube


def test_elasticity_matrix_sizes_and_spd():
    for s in (3, 5):
        w = W.elasticity3d(side=s, seed=2, block=9)
        assert w.A.n == 3 * s ** 3
        assert w.A.nnz == 9 * (3 * s - 2) ** 3  # 27-point couplings of 3 x 3 blocks
        d = w.A.to_dense()
        assert np.abs(d - d.T).max() <= 1e-12 * np.abs(d).max()
        assert np.linalg.eigvalsh(d)[0] > 0


def test_laplace27_4dof_sizes():
    for s in (3, 5):
        w = W.laplace27_4dof(side=s, seed=3, block=8)
        assert w.A.n == 4 * s ** 3
        assert w.A.nnz == 16 * (3 * s - 2) ** 3
        d = w.A.to_dense()
        # K (x) C with K symmetric positive definite and C diagonally dominant: every 4 x 4
        # diagonal block is a positive multiple of C
        blk = d[:4, :4]
        C = blk / blk[0, 0]
        assert np.all(np.abs(np.diag(C)) > np.abs(C).sum(axis=1) - np.abs(np.diag(C)))


def test_full_size_counts_match_the_configurations():
    # the closed forms at the configured sizes (48^3 elasticity, 64^3 4-dof 27-point)
    assert 9 * (3 * 48 - 2) ** 3 == 25_769_592
    assert 16 * (3 * 64 - 2) ** 3 == 109_744_000


def test_shifted_elasticity_is_symmetric_and_indefinite():
    """(K + K^T) / 2 - 0.3 diag(K): exactly symmetric, a few negative eigenvalues (those of the
    Jacobi-scaled K below 0.3), b = A * ones."""
    import numpy as np
    import scipy.sparse as sp
    from paper_1908_10169_gb300 import workloads as W
    w = W.elasticity3d_shifted(side=6, block=24)
    A = w.A
    S = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    assert A.n == 3 * 6 ** 3 and (S != S.T).nnz == 0
    K = W.elasticity3d(side=6, block=24).A
    Ks = sp.csr_matrix((K.val, K.colind, K.rowptr), shape=(K.n, K.n))
    d = Ks.diagonal()
    ev = np.linalg.eigvalsh(S.toarray())
    evj = np.linalg.eigvalsh((sp.diags(d ** -0.5) @ ((Ks + Ks.T) * 0.5) @ sp.diags(d ** -0.5)).toarray())
    assert (ev < 0).sum() == (evj < 0.3).sum() > 0  # Sylvester's law of inertia
    np.testing.assert_allclose(w.b, S @ np.ones(A.n), rtol=1e-14)


def test_saddle_point_system_structure():
    import numpy as np
    import scipy.sparse as sp
    from paper_1908_10169_gb300 import workloads as W
    side = 4
    w = W.kkt_elasticity(side=side, block=24)
    A = w.A
    m = 3 * side * side
    S = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    assert A.n == 3 * side ** 3 + m and (S != S.T).nnz == 0
    assert not S.diagonal()[:m].any() and (S.diagonal()[m:] > 0).all()
    rows = [S[k].indices for k in range(m)]
    assert all(len(r) == 1 for r in rows) and len({int(r[0]) for r in rows}) == m  # distinct displacements
    ev = np.linalg.eigvalsh(S.toarray())
    assert (ev < 0).sum() == m  # inertia of a saddle point with a full-rank constraint block
