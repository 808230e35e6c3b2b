"""Incomplete LDL^T without fill (the ~ildl(0) variant of §4.1) and the factored inner
operator of Eq. (preconditioner): J~ = L~^-1 J^ L~^-T with L~ = L_1 |D|^(1/2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

§3 factors M^ = (A^ + A^T)/2 as L D L^T (Bunch-Kaufman-Parlett, Eq. absfac) and, for
large systems, replaces it by an incomplete factorization; §4.1's ~ildl(0) keeps no
more entries than M^ has.  Readings taken here (the paper names sym-ildl and stops):
  * pattern: exactly the structural pattern of A^ + A^T (no fill at all);
  * pivots: 1x1 (ildl0), or 1x1 and 2x2 blocks (ildl0_blocks, reading R20): a row whose
    diagonal fails the first Bunch-Kaufman test |m_ii| >= alpha max_j |m_ij| pairs with
    the column of that maximum when that row fails it too and points back (a static,
    parallel choice made before the ordering); the pattern is then closed so that every
    block between two pivots is full, and the pairs are coloured as single vertices;
    a tiny |d_i| or 2x2 determinant is an error;
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

    def __init__(self, L, d, order, Jh, W=None):
        """W (optional): the block-diagonal |D|^(-1/2) of a factor with 2x2 pivots, used
        in place of the diagonal weights |d|^(-1/2)."""
        n = L.shape[0]
        self.n = n
        self.order = np.asarray(order)
        self.W = None if W is None else sp.csr_matrix(W)
        self.wd = None if W is not None else 1.0 / np.sqrt(np.abs(d))
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

    def _weight(self, v):
        return self.W @ v if self.W is not None else self.wd * v

    def F(self, v):
        v = np.asarray(v, dtype=np.float64)
        if v.ndim == 2:
            return np.column_stack([self.F(v[:, c]) for c in range(v.shape[1])]) if v.shape[1] else v.copy()
        return self._weight(self._lower_solve(v))

    def G(self, v):
        v = np.asarray(v, dtype=np.float64)
        if v.ndim == 2:
            return np.column_stack([self.G(v[:, c]) for c in range(v.shape[1])]) if v.shape[1] else v.copy()
        return self._upper_solve(self._weight(v))

    def __matmul__(self, v):
        """J~ v = F (J^ (G v))."""
        return self.F(self.Jh @ self.G(v))

    def dense(self):
        return self @ np.eye(self.n)


# ----------------------------------------------------------------------------
# 2x2 pivot blocks (reading R20): a static Bunch-Kaufman choice, the block pattern,
# the colouring of the quotient graph and the block factor
# ----------------------------------------------------------------------------
BK_ALPHA = (1.0 + np.sqrt(17.0)) / 8.0   # Bunch-Kaufman's growth-optimal threshold


def bk_pairs(MP, alpha: float = BK_ALPHA):
    """Static 2x2 pivot choice on the symmetric matrix MP (values on its pattern).
    For every i: gamma_i = max_{j != i} |m_ij| over the stored entries, r_i its column
    (the smallest j on ties); i asks for a 2x2 pivot when |m_ii| < alpha gamma_i (the
    first Bunch-Kaufman test).  i and r_i form a pair when each asks and each is the
    other's r.  Returns partner (int64, -1 for a 1x1 pivot)."""
    M = sp.csr_matrix(MP)
    n = M.shape[0]
    partner = np.full(n, -1, dtype=np.int64)
    r = np.full(n, -1, dtype=np.int64)
    need = np.zeros(n, dtype=bool)
    diag = M.diagonal()
    for i in range(n):
        cols = M.indices[M.indptr[i]:M.indptr[i + 1]]
        vals = np.abs(M.data[M.indptr[i]:M.indptr[i + 1]])
        off = cols != i
        if not np.any(off):
            continue
        c, v = cols[off], vals[off]
        g = v.max()
        r[i] = int(c[v == g].min())
        need[i] = abs(diag[i]) < alpha * g
    for i in range(n):
        j = r[i]
        if need[i] and j >= 0 and need[j] and r[j] == i:
            partner[i] = j
    return partner


def block_pattern(P, partner):
    """The pattern the block factor keeps: P plus what makes every block between two
    pivots full, i.e. the pattern of (I + E) P (I + E) with E linking the members of
    each pair.  Unit values, sorted indices."""
    n = P.shape[0]
    p = np.asarray(partner)
    rows = np.flatnonzero(p >= 0)
    E = sp.csr_matrix((np.ones(rows.size), (rows, p[rows])), shape=(n, n))
    B = (sp.identity(n, format="csr") + E).tocsr()
    P1 = sp.csr_matrix((np.ones(P.nnz), P.indices, P.indptr), shape=P.shape)
    Q = (B @ P1 @ B).tocsr()
    Q.data[:] = 1.0
    Q.sort_indices()
    return Q


def jp_colouring_blocks(P, prio, partner):
    """Jones-Plassmann colouring of the quotient graph in which each pair is one vertex
    (its leader: the smaller index, whose priority it takes); both members get the
    leader's colour.  Returns (colour (int64, n), rounds)."""
    n = P.shape[0]
    p = np.asarray(partner)
    lead = np.where(p >= 0, np.minimum(np.arange(n), p), np.arange(n))
    leaders = np.flatnonzero(lead == np.arange(n))
    slot = np.full(n, -1, dtype=np.int64)
    slot[leaders] = np.arange(leaders.size)
    R = sp.csr_matrix((np.ones(n), (np.arange(n), slot[lead])), shape=(n, leaders.size))
    P1 = sp.csr_matrix((np.ones(P.nnz), P.indices, P.indptr), shape=P.shape)
    Gq = (R.T @ P1 @ R).tocsr()
    Gq.sort_indices()
    cq, rounds = jp_colouring(Gq, np.asarray(prio)[leaders])
    return cq[slot[lead]], rounds


def ildl0_blocks(MP, colour, partner, zero_tol: float = 1e-14):
    """No-fill incomplete block L D L^T of the symmetric matrix MP (values on its block
    pattern, see block_pattern) with 1x1 and 2x2 pivots, in the order of the pivot
    blocks by (colour, leader index).  For each block I in that order and each lower
    block K adjacent to it, in order:
        L_IK = (M_IK - sum_{K' < K adjacent to I and K} L_IK' D_K' L_KK'^T) D_K^-1,
    then D_I = M_II - sum_{K < I} L_IK D_K L_IK^T.  A zero (or tiny) 1x1 pivot, or a 2x2
    pivot with a zero (or tiny) determinant, is an error.
    Returns (L, D): L strictly block-lower (n x n CSR, original indexing), D the block
    diagonal (n x n CSR: the pivots, and m_{i,partner(i)} updated for pairs)."""
    M = sp.csr_matrix(MP)
    n = M.shape[0]
    p = np.asarray(partner)
    lead = np.where(p >= 0, np.minimum(np.arange(n), p), np.arange(n))
    leaders = np.flatnonzero(lead == np.arange(n))
    order = leaders[np.lexsort((leaders, np.asarray(colour)[leaders]))]
    rank = np.full(n, -1, dtype=np.int64)
    rank[order] = np.arange(order.size)
    members = {int(i): ([int(i)] if p[i] < 0 else sorted([int(i), int(p[i])])) for i in leaders}
    Md = M.toarray() if n <= 2000 else None

    def mblock(I, K):
        if Md is not None:
            return Md[np.ix_(members[I], members[K])]
        return M[members[I]][:, members[K]].toarray()

    dmax = np.abs(M.diagonal()).max() if n else 0.0
    Lb = {}      # block I -> {K: L_IK}
    Db = {}
    for I in order:
        I = int(I)
        rows = members[I]
        nb = set()
        for r_ in rows:
            for c in M.indices[M.indptr[r_]:M.indptr[r_ + 1]]:
                K = int(lead[c])
                if rank[K] < rank[I]:
                    nb.add(K)
        LI = {}
        for K in sorted(nb, key=lambda k: rank[k]):
            S = mblock(I, K).copy()
            for K2, LK2 in Lb[K].items():
                if K2 in LI:
                    S -= LI[K2] @ Db[K2] @ LK2.T
            LI[K] = S @ np.linalg.inv(Db[K])
        DI = mblock(I, I).copy()
        for K, LIK in LI.items():
            DI -= LIK @ Db[K] @ LIK.T
        if DI.shape[0] == 1:
            if DI[0, 0] == 0.0 or abs(DI[0, 0]) < zero_tol * dmax:
                raise ZeroDivisionError(f"zero pivot in the incomplete block LDL^T at {rows}")
        else:
            det = DI[0, 0] * DI[1, 1] - DI[0, 1] * DI[1, 0]
            if det == 0.0 or abs(det) < zero_tol * dmax * dmax:
                raise ZeroDivisionError(f"singular 2x2 pivot in the incomplete block LDL^T at {rows}")
            DI = 0.5 * (DI + DI.T)
        Db[I] = DI
        Lb[I] = LI
    r_, c_, v_ = [], [], []
    for I, LI in Lb.items():
        for K, LIK in LI.items():
            for a, ra in enumerate(members[I]):
                for b, cb in enumerate(members[K]):
                    r_.append(ra)
                    c_.append(cb)
                    v_.append(LIK[a, b])
    L = sp.csr_matrix((np.array(v_, dtype=np.float64), (np.array(r_, dtype=np.int64), np.array(c_, dtype=np.int64))),
                      shape=(n, n))
    L.sort_indices()
    dr, dc, dv = [], [], []
    for I, DI in Db.items():
        for a, ra in enumerate(members[I]):
            for b, cb in enumerate(members[I]):
                dr.append(ra)
                dc.append(cb)
                dv.append(DI[a, b])
    D = sp.csr_matrix((np.array(dv), (np.array(dr, dtype=np.int64), np.array(dc, dtype=np.int64))), shape=(n, n))
    D.sort_indices()
    return L, D


def block_pivot_split(D, partner):
    """For the block diagonal D of 1x1 and 2x2 pivots: W = |D|^(-1/2) (block by block:
    V |Lambda|^(-1/2) V^T of each symmetric 2x2 block) and M~_r = sign(D) - I as
    U_r Sigma_r U_r^T (Fig. 1: a 1x1 negative pivot gives e_i with -2; a 2x2 block with
    eigenpairs (lambda, v) gives v with -2 for each negative lambda).
    Returns (W (n x n CSR), U_r (n x r dense), sigma_r (r,))."""
    n = D.shape[0]
    p = np.asarray(partner)
    Dd = sp.csr_matrix(D)
    wr, wc, wv = [], [], []
    cols, sig = [], []
    for i in range(n):
        j = int(p[i])
        if j >= 0 and j < i:
            continue
        if j < 0:
            d = Dd[i, i]
            wr.append(i)
            wc.append(i)
            wv.append(1.0 / np.sqrt(abs(d)))
            if d < 0:
                u = np.zeros(n)
                u[i] = 1.0
                cols.append(u)
                sig.append(-2.0)
            continue
        idx = [i, j]
        B = np.array([[Dd[i, i], Dd[i, j]], [Dd[j, i], Dd[j, j]]])
        lam, V = np.linalg.eigh(0.5 * (B + B.T))
        Wb = V @ np.diag(1.0 / np.sqrt(np.abs(lam))) @ V.T
        for a in range(2):
            for b in range(2):
                wr.append(idx[a])
                wc.append(idx[b])
                wv.append(Wb[a, b])
        for t in range(2):
            if lam[t] < 0:
                u = np.zeros(n)
                u[idx] = V[:, t]
                cols.append(u)
                sig.append(-2.0)
    W = sp.csr_matrix((np.array(wv), (np.array(wr, dtype=np.int64), np.array(wc, dtype=np.int64))), shape=(n, n))
    U = np.array(cols).T if cols else np.zeros((n, 0))
    return W, U, np.array(sig)


def block_order(colour, partner):
    """Vertex order of the block factor: pivot blocks by (colour, leader index), the two
    members of a pair next to each other (smaller index first)."""
    n = len(colour)
    p = np.asarray(partner)
    lead = np.where(p >= 0, np.minimum(np.arange(n), p), np.arange(n))
    leaders = np.flatnonzero(lead == np.arange(n))
    ordl = leaders[np.lexsort((leaders, np.asarray(colour)[leaders]))]
    out = []
    for i in ordl:
        out.append(int(i))
        if p[i] >= 0:
            out.append(int(p[i]))
    return np.array(out, dtype=np.int64)
