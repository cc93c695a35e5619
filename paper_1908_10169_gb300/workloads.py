"""Seeded synthetic test matrices (convection-diffusion and elasticity stencils).

This module only builds inputs: sparse matrices in CSR form, right-hand sides and
the parameters a run uses.  It holds none of the factorization's arithmetic, so both
the FP64 CPU oracle (through the tests) and the CUDA path consume the very same
arrays.  The paper's own test matrices (SuiteSparse, n >= 50000, Sec. 4) are not
available; these stencils stand in for them.

Conventions shared by every generator:
  * unknowns are grid nodes in natural lexicographic order, x fastest;
  * Dirichlet boundary nodes are eliminated (the matrix covers interior nodes only);
  * random numbers come from numpy's PCG64 with the stated seed;
  * rows are scaled by h^2 so entries are O(1) (the drop test and the relative
    GMRES residual are scale-invariant, so this changes no result);
  * CSR: rowptr int64 (n+1), colind int32 sorted within each row, val float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int64, n+1
    colind: np.ndarray  # int32, nnz
    val: np.ndarray     # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A x (input preparation only, e.g. the right-hand side b = A*1)."""
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        return np.bincount(rows, weights=self.val * x[self.colind], minlength=self.n)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.colind] = self.val
        return d


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    # no duplicates are produced by the generators; guard anyway
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate entries in generated matrix")
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n, rowptr, cols.astype(np.int32), vals.astype(np.float64))


def from_dense(d: np.ndarray, keep_zeros_on_diag: bool = True) -> CSR:
    """CSR of a dense matrix (test helper): keeps nonzeros (and the diagonal)."""
    n = d.shape[0]
    mask = d != 0
    if keep_zeros_on_diag:
        mask |= np.eye(n, dtype=bool)
    rows, cols = np.nonzero(mask)
    return _from_coo(n, rows.astype(np.int64), cols.astype(np.int64), d[rows, cols])


def convdiff2d_central(nx: int, ny: int, vmax: float = 10.0, seed: int = 0) -> CSR:
    """-Laplace(u) + v.grad(u) on the unit square, 5-point, central differences.

    Velocity (v_x, v_y) is drawn per node from U[-vmax, vmax] (seed).  h = 1/(nx+1)
    (nx == ny assumed for h; the square grid is what the workloads use).
    Row p (times h^2): diag 4, east/west -1 +/- v_x h/2, north/south -1 +/- v_y h/2.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nx * ny
    h = 1.0 / (nx + 1)
    v = rng.uniform(-vmax, vmax, size=(2, n))
    p = np.arange(n)
    x, y = p % nx, p // nx
    rows = [p]
    cols = [p]
    vals = [np.full(n, 4.0)]
    for (dx, dy, comp, sgn) in ((1, 0, 0, +1), (-1, 0, 0, -1), (0, 1, 1, +1), (0, -1, 1, -1)):
        m = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        q = p + dx + dy * nx
        rows.append(p[m])
        cols.append(q[m])
        vals.append(-1.0 + sgn * v[comp, m] * h / 2.0)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def _harmonic(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return 2.0 * a * b / (a + b)


def convdiff_upwind(dims: tuple, kappa_decades: tuple = (-3.0, 3.0), vel: tuple | None = None,
                    seed: int = 1) -> CSR:
    """-div(kappa grad u) + v.grad(u), 2D 5-point or 3D 7-point, first-order upwind.

    kappa per node is log-uniform in [10^kappa_decades[0], 10^kappa_decades[1]] (seed);
    the face coefficient between two interior nodes is the harmonic mean of theirs, a face
    to an (eliminated) Dirichlet node uses the interior node's own kappa.  h = 1/(dims[0]+1).
    Row p (times h^2): diag = sum_faces kappa_f + h * sum_d |v_d|;
    off-diagonal to q = -kappa_f, minus h*|v_d| more when q is the upwind neighbour.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dim = len(dims)
    n = int(np.prod(dims))
    h = 1.0 / (dims[0] + 1)
    if vel is None:
        vel = tuple([100.0 / math.sqrt(dim)] * dim)
    kappa = 10.0 ** rng.uniform(kappa_decades[0], kappa_decades[1], size=n)
    p = np.arange(n)
    coords = []
    rem = p.copy()
    strides = []
    s = 1
    for d in range(dim):
        coords.append(rem % dims[d])
        rem = rem // dims[d]
        strides.append(s)
        s *= dims[d]
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for d in range(dim):
        vd = vel[d]
        for sgn in (-1, +1):
            inside = (coords[d] + sgn >= 0) & (coords[d] + sgn < dims[d])
            q = p + sgn * strides[d]
            kf = kappa.copy()
            kf[inside] = _harmonic(kappa[inside], kappa[q[inside]])
            diag += kf
            upwind = (sgn < 0) if vd >= 0 else (sgn > 0)
            off = -kf[inside] - (h * abs(vd) if upwind else 0.0)
            rows.append(p[inside])
            cols.append(q[inside])
            vals.append(off)
        diag += h * abs(vd)
    rows.append(p)
    cols.append(p)
    vals.append(diag)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def rhs_ones(A: CSR) -> np.ndarray:
    """b = A * (1,...,1): the exact solution is the all-ones vector."""
    return A.matvec(np.ones(A.n))


def random_diag_dominant(n: int, density: float, seed: int, dominance: float = 1.5) -> CSR:
    """Random sparse nonsymmetric matrix with a dominant diagonal (test input)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = rng.random((n, n)) < density
    d = np.where(mask, rng.uniform(-1.0, 1.0, size=(n, n)), 0.0)
    np.fill_diagonal(d, 0.0)
    rs = np.abs(d).sum(axis=1)
    np.fill_diagonal(d, (rs + 1.0) * dominance * np.where(rng.random(n) < 0.5, -1.0, 1.0))
    return from_dense(d)


# --- named workloads --------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    A: CSR
    b: np.ndarray
    droptol: float
    max_block: int
    blocking: str        # "fixed" or "ilu1t"
    fixed_block: int
    gmres_tol: float = 1e-8
    restart: int = 30


def cd2d_32(seed: int = 0) -> Workload:
    """2D convection-diffusion, 32x32 interior grid (n = 1024), central differences,
    v per node uniform in [-10, 10], drop tolerance 1e-2, blocks of one grid line (32)."""
    A = convdiff2d_central(32, 32, 10.0, seed)
    return Workload("cd2d_5pt_32x32", A, rhs_ones(A), 1e-2, 32, "fixed", 32)


def cd3d(side: int = 64, seed: int = 1, block: int = 64) -> Workload:
    """3D convection-diffusion, side^3 interior grid, 7-point upwind, kappa log-uniform in
    [1e-3, 1e3] per node, |v| = 100 along (1,1,1); drop tolerance 1e-2; blocks of `block`."""
    A = convdiff_upwind((side, side, side), seed=seed)
    return Workload(f"cd3d_7pt_{side}^3", A, rhs_ones(A), 1e-2, 64, "fixed", block)


def rows_scrambled(w: Workload, seed: int = 5) -> Workload:
    """The same system with its equations (rows of A and entries of b) in a seeded random order:
    a nonsymmetric matrix with zeros on its diagonal, the kind that needs the matching of
    Sec. 3.1 before an incomplete factorization.  The solution x is unchanged."""
    rng = np.random.Generator(np.random.PCG64(seed))
    order = rng.permutation(w.A.n)
    counts = np.diff(w.A.rowptr)[order]
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    take = np.concatenate([np.arange(w.A.rowptr[i], w.A.rowptr[i + 1]) for i in order]) if w.A.n else np.zeros(0, int)
    A = CSR(w.A.n, rowptr, w.A.colind[take].astype(np.int32), w.A.val[take].astype(np.float64))
    return dataclasses.replace(w, name=w.name + "_rows_scrambled", A=A, b=w.b[order].copy())


def cd_batch(count: int = 64, seed0: int = 100, n_lo: float = 1e4, n_hi: float = 2e5, block: int = 64):
    """Batch of uneven convection-diffusion matrices.  Matrix k has seed seed0 + k: even seeds
    give 2D 5-point, odd seeds 3D 7-point upwind problems; the target size is log-uniform in
    [n_lo, n_hi] (drawn from the seed), the grid side round(n^(1/2)) or round(n^(1/3)); kappa
    log-uniform in [1e-3, 1e3] per node, |v| = 10 (Peclet 10 against kappa = 1).  Returns a list
    of Workloads (fixed blocks of `block`, drop tolerance 1e-2)."""
    out = []
    for k in range(count):
        seed = seed0 + k
        rng = np.random.Generator(np.random.PCG64(seed))
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        dim = 2 if seed % 2 == 0 else 3
        side = max(2, int(round(n_target ** (1.0 / dim))))
        vel = tuple([10.0 / math.sqrt(dim)] * dim)
        A = convdiff_upwind(tuple([side] * dim), vel=vel, seed=seed)
        out.append(Workload(f"cd{dim}d_{side}_s{seed}", A, rhs_ones(A), 1e-2, 64, "fixed", min(block, side)))
    return out


def cd3d_skip_train(count: int = 200, seed0: int = 1000, side_lo: int = 32, side_hi: int = 48, block: int = 64):
    """Training problems of the learned skip: 3D 7-point upwind convection-diffusion, matrix k
    with seed seed0 + k, side uniform in {side_lo..side_hi} and Peclet number log-uniform in
    [1, 1000] (|v| = Pe along (1,1,1), kappa log-uniform in [1e-3, 1e3] per node), drop
    tolerance 1e-2, fixed blocks of `block`.  Yields Workloads (generated lazily)."""
    for k in range(count):
        seed = seed0 + k
        rng = np.random.Generator(np.random.PCG64(seed))
        side = int(rng.integers(side_lo, side_hi + 1))
        pe = 10.0 ** rng.uniform(0.0, 3.0)
        A = convdiff_upwind((side, side, side), vel=tuple([pe / math.sqrt(3.0)] * 3), seed=seed)
        yield Workload(f"cd3d_train_{side}_pe{pe:.0f}_s{seed}", A, rhs_ones(A), 1e-2, 64, "fixed", min(block, side * side))


# --- trilinear (Q1) hexahedral finite elements --------------------------------------------

_GAUSS = (-1.0 / math.sqrt(3.0), 1.0 / math.sqrt(3.0))
_CORNERS = [(i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]  # local node a = i + 2j + 4k


def _q1_grads():
    """Gradients (x, y, z) of the 8 trilinear shape functions on the unit cube at the 2x2x2
    Gauss points: array [8 points][8 nodes][3]."""
    out = []
    for gz in _GAUSS:
        for gy in _GAUSS:
            for gx in _GAUSS:
                p = [(1 + gx) / 2, (1 + gy) / 2, (1 + gz) / 2]
                gr = []
                for (i, j, k) in _CORNERS:
                    f = [p[0] if i else 1 - p[0], p[1] if j else 1 - p[1], p[2] if k else 1 - p[2]]
                    s = [1 if i else -1, 1 if j else -1, 1 if k else -1]
                    gr.append([s[0] * f[1] * f[2], f[0] * s[1] * f[2], f[0] * f[1] * s[2]])
                out.append(gr)
    return np.array(out)  # Gauss weights are 1/8 each on the unit cube


def q1_laplace_element() -> np.ndarray:
    """8 x 8 element matrix of -div(grad u) for Q1 on the unit cube (2x2x2 Gauss)."""
    G = _q1_grads()
    return sum(g @ g.T for g in G) / 8.0


def q1_elasticity_element(nu: float = 0.3) -> np.ndarray:
    """24 x 24 element stiffness of isotropic linear elasticity (E = 1) for Q1 on the unit
    cube, 2x2x2 Gauss; dof order (node a, component d) -> 3a + d."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = np.eye(3) * mu
    Ke = np.zeros((24, 24))
    for g in _q1_grads():
        Bm = np.zeros((6, 24))
        for a in range(8):
            gx, gy, gz = g[a]
            c = 3 * a
            Bm[0, c], Bm[1, c + 1], Bm[2, c + 2] = gx, gy, gz
            Bm[3, c], Bm[3, c + 1] = gy, gx          # gamma_xy
            Bm[4, c + 1], Bm[4, c + 2] = gz, gy      # gamma_yz
            Bm[5, c], Bm[5, c + 2] = gz, gx          # gamma_xz
        Ke += Bm.T @ D @ Bm / 8.0
    return Ke


def _assemble_q1(side: int, dof: int, Ke: np.ndarray, coef: np.ndarray) -> CSR:
    """Assemble a Q1 operator on the (side+1)^3 elements of a grid with side^3 interior nodes
    (Dirichlet nodes eliminated), dof unknowns per node interleaved, element matrix Ke scaled
    by coef[element]."""
    import scipy.sparse as sp
    ne = side + 1
    e = np.arange(ne ** 3)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    nodes = []
    for (i, j, k) in _CORNERS:  # interior node index or -1
        x, y, z = ex + i - 1, ey + j - 1, ez + k - 1  # interior coordinates 0..side-1
        inside = (x >= 0) & (x < side) & (y >= 0) & (y < side) & (z >= 0) & (z < side)
        nodes.append(np.where(inside, x + side * (y + side * z), -1))
    nodes = np.stack(nodes, axis=1)  # ne^3 x 8
    ld = Ke.shape[0]
    la = np.arange(ld)
    gdof = np.where(nodes[:, la // dof] >= 0, nodes[:, la // dof] * dof + la % dof, -1)  # ne^3 x ld
    n = side ** 3 * dof
    rows, cols, vals = [], [], []
    for a in range(ld):
        ra = gdof[:, a]
        m = ra >= 0
        for b_ in range(ld):
            if Ke[a, b_] == 0.0:
                continue
            cb = gdof[:, b_]
            mm = m & (cb >= 0)
            rows.append(ra[mm])
            cols.append(cb[mm])
            vals.append(coef[mm] * Ke[a, b_])
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return CSR(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


def elasticity3d(side: int = 48, seed: int = 2, block: int = 63) -> Workload:
    """Q1 hexahedral linear elasticity, side^3 interior nodes (Dirichlet boundary), 3 dof per
    node interleaved: n = 3 side^3 (331,776 for side 48); Poisson ratio 0.3; Young's modulus
    E = 10^(4u), u ~ U[0, 1] per macro-cell of 8^3 elements (jumps 1 .. 1e4, seed); 2x2x2
    Gauss quadrature; drop tolerance 1e-2, fixed blocks of `block` (a multiple of 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = side + 1
    nm = (ne + 7) // 8
    u = rng.uniform(0.0, 1.0, size=nm ** 3)
    e = np.arange(ne ** 3)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    E = 10.0 ** (4.0 * u[(ex // 8) + nm * ((ey // 8) + nm * (ez // 8))])
    A = _assemble_q1(side, 3, q1_elasticity_element(0.3), E)
    return Workload(f"elasticity_q1_{side}^3x3", A, rhs_ones(A), 1e-2, 63, "fixed", block)


def elasticity3d_shifted(side: int = 48, seed: int = 2, block: int = 63, shift: float = 0.3) -> Workload:
    """Symmetric indefinite operator: the Q1 elasticity matrix K of elasticity3d (same seed),
    made exactly symmetric as (K + K^T) / 2, minus shift times its diagonal, so that the
    eigenvalues of diag(K)^{-1/2} K diag(K)^{-1/2} below the shift turn negative.  It stands in
    for the symmetric indefinite af_shell matrices of the paper's BILDL experiments (sheet
    metal forming; not available here).  Right-hand side A * ones; drop tolerance 1e-2."""
    import scipy.sparse as sp
    K = elasticity3d(side, seed, block).A
    Ks = sp.csr_matrix((K.val, K.colind, K.rowptr), shape=(K.n, K.n))
    S = (Ks + Ks.T).tocsr() * 0.5
    S = (S - shift * sp.diags(S.diagonal())).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    A = CSR(S.shape[0], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))
    return Workload(f"elasticity_q1_shifted_{side}^3x3", A, rhs_ones(A), 1e-2, 63, "fixed", block, gmres_tol=1e-6)


def kkt_elasticity(side: int = 16, seed: int = 2, block: int = 63, multipliers_first: bool = True) -> Workload:
    """Symmetric saddle-point system [[K, B^T], [B, 0]]: K is the exactly symmetric Q1 elasticity
    matrix (K + K^T) / 2 of elasticity3d (same seed); B holds one row per displacement of every
    node of the middle plane z = side // 2 (3 side^2 Lagrange multipliers that fix them), the
    row of the identity scaled by the mean diagonal of K.  The multiplier unknowns have a zero
    diagonal, the case the symmetric matching of Sec. 4.2 is for; with multipliers_first they
    come first, so that a block of them has a zero pivot block and no earlier block to fill it.
    n = 3 side^3 + 3 side^2; b = A * ones; drop tolerance 1e-3."""
    import scipy.sparse as sp
    K = elasticity3d(side, seed, block).A
    Ks = sp.csr_matrix((K.val, K.colind, K.rowptr), shape=(K.n, K.n))
    Ks = ((Ks + Ks.T) * 0.5).tocsr()
    z = side // 2
    nodes = np.array([x + side * (y + side * z) for y in range(side) for x in range(side)], dtype=np.int64)
    dofs = (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)
    m = dofs.size
    beta = float(Ks.diagonal().mean())
    Bm = sp.csr_matrix((np.full(m, beta), (np.arange(m), dofs)), shape=(m, K.n))
    if multipliers_first:
        M = sp.bmat([[None, Bm], [Bm.T, Ks]], format="csr")
    else:
        M = sp.bmat([[Ks, Bm.T], [Bm, None]], format="csr")
    M.sum_duplicates()
    M.sort_indices()
    A = CSR(M.shape[0], M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))
    return Workload(f"kkt_elasticity_{side}^3", A, rhs_ones(A), 1e-3, 63, "fixed", block, gmres_tol=1e-6)


def laplace27_4dof(side: int = 64, seed: int = 3, block: int = 64) -> Workload:
    """Q1 27-point scalar diffusion operator (kappa log-uniform in [1e-3, 1e3] per element,
    seed) on side^3 interior nodes, coupled across 4 unknowns per node by the Kronecker product
    with C = I + 0.3 R (R uniform in [-1, 1], rows scaled so that C is diagonally dominant):
    n = 4 side^3 (1,048,576 for side 64), interleaved; drop tolerance 1e-2, blocks of `block`."""
    import scipy.sparse as sp
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = side + 1
    kappa = 10.0 ** rng.uniform(-3.0, 3.0, size=ne ** 3)
    K = _assemble_q1(side, 1, q1_laplace_element(), kappa)
    R = rng.uniform(-1.0, 1.0, size=(4, 4))
    np.fill_diagonal(R, 0.0)
    R *= 0.9 / np.maximum(np.abs(R).sum(axis=1, keepdims=True), 1e-12)
    C = np.eye(4) + 0.3 * R
    Ks = sp.csr_matrix((K.val, K.colind, K.rowptr), shape=(K.n, K.n))
    M = sp.kron(Ks, sp.csr_matrix(C), format="csr")
    M.sort_indices()
    A = CSR(M.shape[0], M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))
    return Workload(f"laplace27_4dof_{side}^3", A, rhs_ones(A), 1e-2, 64, "fixed", block)
