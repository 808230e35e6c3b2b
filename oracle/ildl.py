"""Incomplete LDL^T without fill (the ~ildl(0) variant of §4.1) and the factored inner
operator of Eq. (preconditioner): J~ = L~^-1 J^ L~^-T with L~ = L_1 |D|^(1/2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

§3 factors M^ = (A^ + A^T)/2 as L D L^T (Bunch-Kaufman-Parlett, Eq. absfac) and, for
large systems, replaces it by an incomplete factorization; §4.1's ~ildl(0) keeps no
more entries than M^ has.  Readings taken here (the paper names sym-ildl and stops):
  * pattern: exactly the structural pattern of A^ + A^T (no fill at all);
  * pivots: 1x1 only (no 2x2 Bunch-Kaufman blocks), a tiny |d_i| is an error;
  * order: the factorization runs in a multicolour order - vertices sorted by
    (colour, index) - where the colours come from Jones-Plassmann rounds with
    first-fit colours and splitmix64 priorities (a published, deterministic rule), so
    that every colour is a set of rows that can be eliminated, and later solved for,
    at the same time.
Library primitives used as single steps: scipy.sparse products and triangular
solves.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_MASK64 = (1 << 64) - 1
# the colouring priorities draw on a splitmix64 stream of their own
COLOUR_SEED_XOR = 0xA5A5A5A5A5A5A5A5


def splitmix64_u64(seed: int, n: int) -> np.ndarray:
    """Raw 64-bit outputs of Vigna's splitmix64: state_i = seed + (i+1)*0x9E3779B97F4A7C15
    (mod 2^64), z = state_i; z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
    z *= 0x94D049BB133111EB; z ^= z>>31."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def colouring_priorities(seed: int, n: int) -> np.ndarray:
    return splitmix64_u64((seed ^ COLOUR_SEED_XOR) & _MASK64, n)


def structural_pattern(Abar, S):
    """Structural pattern of Abar S + (Abar S)^T (no cancellation can remove an entry),
    diagonal included: CSR with unit values and sorted indices."""
    A1 = sp.csr_matrix((np.ones(Abar.nnz), Abar.indices, Abar.indptr), shape=Abar.shape)
    S1 = sp.csr_matrix((np.ones(S.nnz), S.indices, S.indptr), shape=S.shape)
    C1 = (A1 @ S1).tocsr()
    P = (C1 + C1.T).tocsr()
    P = (P + sp.identity(P.shape[0], format="csr")).tocsr()
    P.data[:] = 1.0
    P.sort_indices()
    return P


def jp_colouring(G, prio):
    """Jones-Plassmann colouring of the undirected graph with pattern G (diagonal
    ignored).  Round after round, each uncoloured vertex whose (priority, index) is
    larger than that of every uncoloured neighbour takes the smallest colour that no
    coloured neighbour holds.  Returns (colour (int64, n), rounds)."""
    G = sp.csr_matrix(G)
    n = G.shape[0]
    rows = np.repeat(np.arange(n), np.diff(G.indptr))
    cols = G.indices.astype(np.int64)
    off = rows != cols
    rows, cols = rows[off], cols[off]
    prio = np.asarray(prio, dtype=np.uint64)
    # (priority, index) of the neighbour above that of the row
    above = (prio[cols] > prio[rows]) | ((prio[cols] == prio[rows]) & (cols > rows))
    colour = np.full(n, -1, dtype=np.int64)
    rounds = 0
    while np.any(colour < 0):
        unc = colour < 0
        beaten = np.zeros(n, dtype=bool)
        e = unc[rows] & unc[cols] & above
        beaten[rows[e]] = True
        winners = np.flatnonzero(unc & ~beaten)
        for i in winners:
            nb = G.indices[G.indptr[i]:G.indptr[i + 1]]
            used = set(int(c) for c in colour[nb] if c >= 0)
            c = 0
            while c in used:
                c += 1
            colour[i] = c
        rounds += 1
    return colour, rounds


def colour_order(colour):
    """The factorization order: vertices sorted by (colour, index)."""
    n = colour.size
    return np.lexsort((np.arange(n), colour))


def values_on_pattern(M, P):
    """M's values at every position of the pattern P (explicit zeros where M has none)."""
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    n = P.shape[0]
    pr = np.repeat(np.arange(n, dtype=np.int64), np.diff(P.indptr))
    pk = pr * n + P.indices
    mr = np.repeat(np.arange(n, dtype=np.int64), np.diff(M.indptr))
    mk = mr * n + M.indices
    pos = np.searchsorted(mk, pk)
    pos = np.minimum(pos, max(mk.size - 1, 0))
    hit = (mk.size > 0) & (mk[pos] == pk) if mk.size else np.zeros(pk.size, dtype=bool)
    vals = np.where(hit, M.data[pos] if M.nnz else 0.0, 0.0)
    return sp.csr_matrix((vals, P.indices.copy(), P.indptr.copy()), shape=P.shape)


def ildl0(MP, order, zero_tol: float = 1e-14):
    """No-fill incomplete L D L^T of the symmetric matrix MP (values on its own
    structural pattern) eliminated in the given order, 1x1 pivots.  In the permuted
    matrix Mc = MP[order][:, order], row by row (i ascending), for each lower entry
    j < i in ascending order
        l_ij = (m_ij - sum_{k < j, (i,k) and (j,k) in the pattern} l_ik d_k l_jk) / d_j
    and then d_i = m_ii - sum_{k < i} l_ik^2 d_k.
    Returns (L, d): L strictly lower in the order, in the ORIGINAL indexing (n x n CSR,
    the entry for (order[i'], order[j'])), d the pivots in the original indexing."""
    n = MP.shape[0]
    Mc = sp.csr_matrix(MP)[order][:, order].tocsr()
    Mc.sort_indices()
    dmax = np.abs(Mc.diagonal()).max() if n else 0.0
    d = np.zeros(n)
    Lrows = [None] * n
    for i in range(n):
        a, b = Mc.indptr[i], Mc.indptr[i + 1]
        cols = Mc.indices[a:b]
        vals = Mc.data[a:b]
        li = {}
        mii = 0.0
        for j, mij in zip(cols, vals):
            j = int(j)
            if j > i:
                break
            if j == i:
                mii = mij
                break
            s = mij
            for k, ljk in Lrows[j].items():
                lik = li.get(k)
                if lik is not None:
                    s -= lik * d[k] * ljk
            li[j] = s / d[j]
        di = mii
        for k, lik in li.items():
            di -= lik * lik * d[k]
        if di == 0.0 or abs(di) < zero_tol * dmax:
            raise ZeroDivisionError(f"zero pivot in the incomplete LDL^T at position {i}")
        d[i] = di
        Lrows[i] = li
    r, c, v = [], [], []
    for i in range(n):
        for j, lij in Lrows[i].items():
            r.append(order[i])
            c.append(order[j])
            v.append(lij)
    L = sp.csr_matrix((np.array(v), (np.array(r, dtype=np.int64), np.array(c, dtype=np.int64))), shape=(n, n))
    L.sort_indices()
    dout = np.zeros(n)
    dout[order] = d
    return L, dout


class FactoredSkew:
    """The factored operators of §3 in the original indexing:
        F v = |D|^(-1/2) (I + L)^-1 v      (the application of L~^-1)
        G v = (I + L)^-T |D|^(-1/2) v      (the application of L~^-T)
    and J~ = F J^ G (Eq. preconditioner), applied without forming it.  (I + L) is
    lower triangular in the factorization order: the triangular solves run on the
    permuted matrices."""

    def __init__(self, L, d, order, Jh):
        n = d.size
        self.n = n
        self.order = np.asarray(order)
        self.wd = 1.0 / np.sqrt(np.abs(d))
        Lc = sp.csr_matrix(L)[self.order][:, self.order].tocsr()
        self.L1c = (Lc + sp.identity(n, format="csr")).tocsr()
        self.L1cT = self.L1c.T.tocsr()
        self.Jh = sp.csr_matrix(Jh)
        self.shape = (n, n)
        self.dtype = np.float64

    def _lower_solve(self, v):
        o = self.order
        out = np.empty_like(v)
        out[o] = spla.spsolve_triangular(self.L1c, v[o], lower=True, unit_diagonal=True)
        return out

    def _upper_solve(self, v):
        o = self.order
        out = np.empty_like(v)
        out[o] = spla.spsolve_triangular(self.L1cT, v[o], lower=False, unit_diagonal=True)
        return out

    def F(self, v):
        v = np.asarray(v, dtype=np.float64)
        if v.ndim == 2:
            return np.column_stack([self.F(v[:, c]) for c in range(v.shape[1])]) if v.shape[1] else v.copy()
        return self.wd * self._lower_solve(v)

    def G(self, v):
        v = np.asarray(v, dtype=np.float64)
        if v.ndim == 2:
            return np.column_stack([self.G(v[:, c]) for c in range(v.shape[1])]) if v.shape[1] else v.copy()
        return self._upper_solve(self.wd * v)

    def __matmul__(self, v):
        """J~ v = F (J^ (G v))."""
        return self.F(self.Jh @ self.G(v))

    def dense(self):
        return self @ np.eye(self.n)
