"""Seeded synthetic linear systems shaped like the workloads of the two-level
ASSS + mrs scheme (Manguoglu & Mehrmann, arXiv 2009.06954).

This module only *generates inputs*: sparse matrices, right-hand sides and
sparsity patterns for the skew-symmetrizer S.  It holds none of the method's
arithmetic, so both the FP64 CPU oracle (``oracle/``) and the CUDA path (via
``bench.py`` and the tests) may draw their inputs from here.

Workload families (the paper's test matrices are not available, so these stand
in for them; the introduction motivates dissipative Hamiltonian systems, §1):

* ``convection_diffusion_2d``  - 5-point central-difference -Lap(u) + beta.grad(u)
  on an m x m interior grid, Dirichlet boundary (h = 1/(m+1)).
* ``dissipative_hamiltonian_3d`` - one implicit-Euler step of E z' = (J - R) z + f
  (§1): A = E + h (R - J) with E = diag U[1,2], R = r_scale * 7-point Laplacian and
  J an exactly skew face-velocity convection operator.
* ``random_powerlaw`` - general nonsymmetric sparse matrix with power-law row
  lengths, a banded column fraction and a partly dominant diagonal.

All matrices are ``scipy.sparse.csr_matrix`` in float64 with sorted, duplicate-free
column indices.  Every generator takes an explicit integer seed and uses numpy's
PCG64 stream, so a (generator, arguments, seed) triple fixes the input bit for bit.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "convection_diffusion_2d",
    "dissipative_hamiltonian_3d",
    "random_powerlaw",
    "batched_dissipative_hamiltonian",
    "pattern_of",
    "pattern_symmetrized",
    "pattern_diagonal",
    "pattern_tridiagonal",
    "CONFIGS",
]


def _csr(rows, cols, vals, n):
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


# ----------------------------------------------------------------------------
# 2D convection-diffusion
# ----------------------------------------------------------------------------
def convection_diffusion_2d(m: int = 64, beta=(10.0, 10.0), seed: int = 0):
    """-Lap(u) + beta.grad(u) on the unit square, m x m interior nodes.

    Central differences, multiplied through by h^2 (h = 1/(m+1)); node (ix, iy)
    has index iy*m + ix.  Returns (A, b, x_true) with x_true ~ U(-1, 1) and
    b = A x_true.
    """
    n = m * m
    h = 1.0 / (m + 1)
    bx, by = float(beta[0]), float(beta[1])
    ix, iy = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ix = ix.ravel()
    iy = iy.ravel()
    idx = iy * m + ix
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 4.0)]
    for dx, dy, coef in (
        (1, 0, -1.0 + bx * h / 2.0),
        (-1, 0, -1.0 - bx * h / 2.0),
        (0, 1, -1.0 + by * h / 2.0),
        (0, -1, -1.0 - by * h / 2.0),
    ):
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < m) & (jy >= 0) & (jy < m)
        rows.append(idx[ok])
        cols.append((jy * m + jx)[ok])
        vals.append(np.full(int(ok.sum()), coef))
    A = _csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    rng = np.random.default_rng(seed)
    x_true = rng.uniform(-1.0, 1.0, n)
    b = A @ x_true
    return A, b, x_true


# ----------------------------------------------------------------------------
# 3D dissipative Hamiltonian implicit-Euler step
# ----------------------------------------------------------------------------
def _velocity_faces(side, rng, n_modes, vmax):
    """Face-normal velocity v_a on every interior face along axis a.

    v_a(x) = sum_m c_{a,m} sin(2 pi k_{a,m}.x + phi_{a,m}), x in (0,1)^3, with
    integer wavevectors k in {1..4}^3, c ~ N(0,1)/|k| and phi ~ U(0, 2 pi); the
    three components are rescaled together so that max |v_a| over faces = vmax.
    Returns a list of three arrays shaped (s-1, s, s) along the face axis.
    """
    s = side
    ks = rng.integers(1, 5, size=(3, n_modes, 3)).astype(np.float64)
    amp = rng.standard_normal((3, n_modes)) / np.linalg.norm(ks, axis=2)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(3, n_modes))
    g = (np.arange(s, dtype=np.float64) + 1.0) / (s + 1.0)
    gf = (np.arange(s - 1, dtype=np.float64) + 1.5) / (s + 1.0)
    faces = []
    for a in range(3):
        axes = [g, g, g]
        axes[a] = gf
        # arrays indexed [i0, i1, i2] (x, y, z)
        X0, X1, X2 = np.meshgrid(axes[0], axes[1], axes[2], indexing="ij")
        v = np.zeros(X0.shape)
        for mm in range(n_modes):
            k = ks[a, mm]
            v += amp[a, mm] * np.sin(2.0 * np.pi * (k[0] * X0 + k[1] * X1 + k[2] * X2) + phase[a, mm])
        faces.append(v)
    vm = max(np.abs(v).max() for v in faces)
    scale = vmax / vm if vm > 0 else 0.0
    return [v * scale for v in faces]


def dissipative_hamiltonian_3d(side: int = 100, h: float = 1e-2, r_scale: float = 1e-2,
                               vmax: float = 50.0, n_modes: int = 8, seed: int = 1,
                               with_rhs: bool = True):
    """A = E + h (R - J) on a side^3 grid (unit grid spacing), node index
    i0 + s*(i1 + s*i2).

    E = diag U[1,2]; R = r_scale * (7-point Laplacian: 6 on the diagonal, -1 to
    each grid neighbour, Dirichlet); J[p, p+e_a] = v_a/2, J[p+e_a, p] = -v_a/2 with
    the face velocity v_a between the two nodes, so J = -J^T exactly.
    Returns (A, b, parts) where b = E z + h f with z, f ~ N(0,1) (if with_rhs) and
    parts holds E, R, J for tests.
    """
    s = int(side)
    n = s ** 3
    rng = np.random.default_rng(seed)
    E = rng.uniform(1.0, 2.0, n)
    faces = _velocity_faces(s, rng, n_modes, vmax)
    lin = np.arange(n).reshape(s, s, s, order="F")  # lin[i0,i1,i2] = i0 + s*i1 + s*s*i2
    r_rows, r_cols, r_vals = [np.arange(n)], [np.arange(n)], [np.full(n, 6.0 * r_scale)]
    j_rows, j_cols, j_vals = [], [], []
    for a in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, s - 1)
        hi[a] = slice(1, s)
        p = lin[tuple(lo)].ravel()
        q = lin[tuple(hi)].ravel()
        v = faces[a].ravel()
        r_rows += [p, q]
        r_cols += [q, p]
        r_vals += [np.full(p.size, -r_scale), np.full(p.size, -r_scale)]
        j_rows += [p, q]
        j_cols += [q, p]
        j_vals += [0.5 * v, -0.5 * v]
    R = _csr(np.concatenate(r_rows), np.concatenate(r_cols), np.concatenate(r_vals), n)
    J = _csr(np.concatenate(j_rows), np.concatenate(j_cols), np.concatenate(j_vals), n)
    A = (sp.diags(E) + h * (R - J)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    b = None
    if with_rhs:
        z = rng.standard_normal(n)
        f = rng.standard_normal(n)
        b = E * z + h * f
    return A, b, {"E": E, "R": R, "J": J}


def batched_dissipative_hamiltonian(count: int = 256, side_lo: int = 10, side_hi: int = 40,
                                    nrhs: int = 32, seed: int = 3, **kw):
    """Many dissipative-Hamiltonian matrices of uneven size, each with nrhs
    right-hand sides ~ N(0,1).  Matrix m uses seed*100003 + m; its side is drawn
    uniformly from {side_lo..side_hi}.  Returns a list of (A, B) with B n x nrhs."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    out = []
    for m, s in enumerate(sides):
        A, _, _ = dissipative_hamiltonian_3d(side=int(s), seed=seed * 100003 + m,
                                             with_rhs=False, **kw)
        r = np.random.default_rng(seed * 100003 + m + 7)
        B = r.standard_normal((A.shape[0], nrhs))
        out.append((A, B))
    return out


# ----------------------------------------------------------------------------
# general random sparse, power-law rows
# ----------------------------------------------------------------------------
def _powerlaw_exponent(lmin, lmax, lmean):
    L = np.arange(lmin, lmax + 1, dtype=np.float64)
    lo, hi = 0.0, 6.0
    for _ in range(200):
        a = 0.5 * (lo + hi)
        w = L ** (-a)
        mean = (w * L).sum() / w.sum()
        if mean > lmean:
            lo = a
        else:
            hi = a
    return 0.5 * (lo + hi)


def random_powerlaw(n: int = 2_000_000, lmin: int = 4, lmean: float = 16.0, lmax: int = 512,
                    band: int = 1000, band_frac: float = 0.6, dom_frac: float = 0.3,
                    seed: int = 2):
    """General nonsymmetric sparse matrix.

    Row lengths (diagonal included) follow a discrete power law on
    {lmin..lmax} whose exponent makes the mean lmean; each off-diagonal column is
    within |i-j| <= band with probability band_frac and uniform on [0, n)
    otherwise (duplicates merged, so a row can come out slightly shorter).
    Off-diagonal values ~ N(0,1).  A seeded dom_frac of the rows get the diagonal
    1.1 * (row abs-sum of off-diagonals); the others get N(0,1).
    Returns (A, b) with b ~ N(0,1).
    """
    rng = np.random.default_rng(seed)
    a = _powerlaw_exponent(lmin, lmax, lmean)
    L = np.arange(lmin, lmax + 1)
    w = L.astype(np.float64) ** (-a)
    cdf = np.cumsum(w) / w.sum()
    lens = L[np.minimum(np.searchsorted(cdf, rng.random(n)), L.size - 1)]
    noff = lens - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), noff)
    m = rows.size
    banded = rng.random(m) < band_frac
    off = rng.integers(1, band + 1, size=m) * np.where(rng.random(m) < 0.5, -1, 1)
    cols = np.where(banded, rows + off, rng.integers(0, n, size=m))
    cols = np.clip(cols, 0, n - 1)
    keep = cols != rows
    rows, cols = rows[keep], cols[keep]
    vals = rng.standard_normal(rows.size)
    Aoff = _csr(rows, cols, vals, n)
    rowabs = np.asarray(abs(Aoff).sum(axis=1)).ravel()
    dom = rng.random(n) < dom_frac
    diag = np.where(dom, 1.1 * rowabs, rng.standard_normal(n))
    A = (Aoff + sp.diags(diag)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    b = rng.standard_normal(n)
    return A, b


# ----------------------------------------------------------------------------
# sparsity patterns for S
# ----------------------------------------------------------------------------
def _pattern(M):
    P = sp.csr_matrix((np.ones(M.nnz), M.indices.copy(), M.indptr.copy()), shape=M.shape)
    P.sort_indices()
    return P


def pattern_of(A):
    """Pattern of A (unit values)."""
    return _pattern(sp.csr_matrix(A))


def indefinite_zero_diagonal(n: int, seed: int = 0):
    """Sparse indefinite matrix whose diagonal is zero: random N(0,1) entries (about 4
    per row) plus one large entry of random sign per row at a random permuted
    position (|a| in [3, 4)), so that a row permutation exists that puts large
    entries on the diagonal - the situation the matching of §2 (Eq. mc64) is for."""
    rng = np.random.default_rng(seed)
    K = sp.random(n, n, density=4.0 / n, random_state=rng, data_rvs=rng.standard_normal).tolil()
    perm = rng.permutation(n)
    for i in range(n):
        K[i, perm[i]] = (3.0 + rng.random()) * rng.choice([-1.0, 1.0])
    for i in np.flatnonzero(perm == np.arange(n)):   # keep the diagonal zero
        K[i, i] = 0.0
        K[i, (i + 1) % n] = 5.0
    K = K.tocsr()
    K.setdiag(0.0)
    K.eliminate_zeros()
    K.sort_indices()
    return K


def saddle_pairs(n: int, seed: int = 0, singles: int = 0):
    """Nonsymmetric sparse matrix whose symmetric part has zero diagonal entries coupled in
    pairs: rows pi(2t), pi(2t+1) (pi a seeded permutation) have a zero diagonal and a
    symmetric coupling of modulus in [1, 2) between them, the last `singles` rows a
    diagonal in [2, 3); about 3 random symmetric couplings N(0, 0.1^2) per row connect
    everything, and a skew part N(0, 0.3^2) on a random pattern is added.  No 1x1 pivot
    order factors the symmetric part of the pairs (zero diagonal); 2x2 pivots do."""
    rng = np.random.default_rng(seed)
    pi = rng.permutation(n)
    npair = (n - singles) // 2
    rows, cols, vals = [], [], []
    for t in range(npair):
        i, j = int(pi[2 * t]), int(pi[2 * t + 1])
        v = (1.0 + rng.random()) * rng.choice([-1.0, 1.0])
        rows += [i, j]
        cols += [j, i]
        vals += [v, v]
    for t in range(2 * npair, n):
        i = int(pi[t])
        rows.append(i)
        cols.append(i)
        vals.append(2.0 + rng.random())
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    R = sp.random(n, n, density=1.5 / n, random_state=rng, data_rvs=lambda k: 0.1 * rng.standard_normal(k))
    R = sp.csr_matrix(R)
    R.setdiag(0.0)
    K = sp.random(n, n, density=2.0 / n, random_state=rng, data_rvs=lambda k: 0.3 * rng.standard_normal(k))
    K = sp.csr_matrix(K)
    K.setdiag(0.0)
    A = (M + R + R.T + K - K.T).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    A.sort_indices()
    return A


def pattern_symmetrized(A):
    """Pattern of A + A^T (unit values)."""
    P = (abs(sp.csr_matrix(A)) + abs(sp.csr_matrix(A)).T).tocsr()
    P.sum_duplicates()
    return _pattern(P)


def pattern_diagonal(n):
    """Diagonal pattern (the paper's S_d)."""
    return _pattern(sp.identity(n, format="csr"))


def pattern_tridiagonal(n):
    """Tridiagonal pattern (the paper's S_t)."""
    return _pattern(sp.diags([np.ones(n - 1), np.ones(n), np.ones(n - 1)], [-1, 0, 1]).tocsr())


# ----------------------------------------------------------------------------
# named workload configurations
# ----------------------------------------------------------------------------
CONFIGS = {
    "cd2d_64": dict(kind="cd2d", m=64, seed=0, s_pattern="A", precision="fp64",
                    outer="tfqmr", inner_tol=1e-10, outer_tol=1e-8),
    "dh3d_100": dict(kind="dh3d", side=100, seed=1, s_pattern="A", precision="mixed",
                     outer="fgmres", inner_tol=1e-6, outer_tol=1e-8),
    "powerlaw_2m": dict(kind="powerlaw", n=2_000_000, seed=2, s_pattern="A+At",
                        precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-8),
    "dh3d_batch256": dict(kind="dh3d_batch", count=256, nrhs=32, seed=3, s_pattern="A",
                          precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-8),
    "dh3d_64_adjoint": dict(kind="dh3d", side=64, seed=4, s_pattern="A", precision="mixed",
                            outer="fgmres", inner_tol=1e-6, outer_tol=1e-8),
}
