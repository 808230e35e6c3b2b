"""Pins for the oracle's no-fill incomplete L D L^T (§3 after Eq. absfac, §4.1 ~ildl(0))
and its multicolour order, against mathematics that does not come from the oracle:
the defining property of a no-fill factorization, exact factorizations where no fill
can occur (tridiagonal, dense: Cholesky), a sequential greedy colouring written out
here, and the exactness of the preconditioner for a complete factorization (§3: with
the full L D L^T, P equals the preconditioned matrix).  None of them calls the CUDA
path.
"""
import inspect
import textwrap

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import convection_diffusion_2d, dissipative_hamiltonian_3d


def _sym_random(n, dens, rng, shift):
    R = sp.random(n, n, density=dens, random_state=rng, format="csr")
    M = (R + R.T).tocsr()
    M = (M + sp.diags(shift + rng.random(n))).tocsr()
    M.sort_indices()
    return M


def _greedy_by_priority(G, prio):
    """Sequential first-fit colouring, vertices taken by decreasing (priority, index)."""
    n = G.shape[0]
    order = sorted(range(n), key=lambda i: (int(prio[i]), i), reverse=True)
    colour = [-1] * n
    for i in order:
        used = {colour[j] for j in G.indices[G.indptr[i]:G.indptr[i + 1]] if j != i and colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return np.array(colour)


def _on_pattern(M, P):
    return O.values_on_pattern(M, P).data


def test_splitmix64_u64_published_first_output():
    assert int(O.splitmix64_u64(0, 1)[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_jp_colouring_is_greedy_in_priority_order(seed):
    """Jones-Plassmann rounds colour every vertex after all its higher-priority
    neighbours, so the result is the sequential greedy colouring in priority order."""
    rng = np.random.default_rng(seed)
    G = _sym_random(80, 0.06, rng, 1.0)
    prio = O.colouring_priorities(seed, 80)
    col, rounds = O.jp_colouring(G, prio)
    np.testing.assert_array_equal(col, _greedy_by_priority(G, prio))
    rows = np.repeat(np.arange(80), np.diff(G.indptr))
    off = rows != G.indices
    assert np.all(col[rows[off]] != col[G.indices[off]])            # a proper colouring
    deg = np.diff(G.indptr) - 1
    assert col.max() <= deg.max()


def test_jp_colouring_on_a_grid_pattern():
    A, _, _ = convection_diffusion_2d(m=12)
    G = (abs(A) + abs(A.T)).tocsr()
    prio = O.colouring_priorities(7, A.shape[0])
    col, _ = O.jp_colouring(G, prio)
    np.testing.assert_array_equal(col, _greedy_by_priority(G, prio))


@pytest.mark.parametrize("shift", [4.0, 0.3])
def test_ildl0_reproduces_the_matrix_on_its_pattern(shift):
    """The defining property of a no-fill incomplete factorization: (I + L) D (I + L)^T
    equals M at every position of M's pattern (diagonal included), and L has entries
    only there.  shift 0.3 gives an indefinite matrix with negative pivots."""
    rng = np.random.default_rng(5)
    n = 70
    M = _sym_random(n, 0.08, rng, shift)
    if shift < 1:
        M = (M - sp.diags(np.where(np.arange(n) % 7 == 0, 2.5, 0.0))).tocsr()
        M.sort_indices()
    order = rng.permutation(n)
    L, d = O.ildl0(M, order)
    L1 = (L + sp.identity(n)).tocsr()
    R = (L1 @ sp.diags(d) @ L1.T).tocsr()
    np.testing.assert_allclose(_on_pattern(R, M), M.data, rtol=0, atol=1e-12 * abs(M).max())
    Lp = sp.csr_matrix((np.ones(L.nnz), L.indices, L.indptr), shape=L.shape)
    Mp = sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape)
    assert (Lp - Lp.multiply(Mp)).nnz == 0                          # no fill
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(L.indptr))
    assert np.all(pos[L.indices] < pos[rows])                       # lower in the order
    if shift < 1:
        assert np.any(d < 0)


def test_ildl0_is_exact_without_fill():
    """Where elimination creates no fill the incomplete factorization is the complete
    one: a tridiagonal matrix in natural order (indefinite values), and a dense SPD
    matrix in any order, where (I + L) D^(1/2) is the Cholesky factor."""
    rng = np.random.default_rng(6)
    n = 30
    off = rng.standard_normal(n - 1)
    T = sp.diags([off, 3 * rng.standard_normal(n) + 0.5, off], [-1, 0, 1]).tocsr()
    L, d = O.ildl0(T, np.arange(n))
    L1 = (L + sp.identity(n)).toarray()
    np.testing.assert_allclose(L1 @ np.diag(d) @ L1.T, T.toarray(), atol=1e-12 * abs(T).max())
    B = rng.standard_normal((12, 12))
    Md = B @ B.T + 12 * np.eye(12)
    order = rng.permutation(12)
    L, d = O.ildl0(sp.csr_matrix(Md), order)
    Lc = (L + sp.identity(12)).toarray()[np.ix_(order, order)]
    np.testing.assert_allclose(Lc @ np.diag(np.sqrt(d[order])), np.linalg.cholesky(Md[np.ix_(order, order)]),
                               atol=1e-12)


def test_ildl0_zero_pivot_is_an_error():
    M = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, 1.0]]))
    with pytest.raises(ZeroDivisionError):
        O.ildl0(M, np.arange(2))


@pytest.mark.parametrize("seed", [0, 2])
def test_preconditioner_is_exact_for_a_complete_factor(seed):
    """§3: with the complete L D L^T of M^ the preconditioner of Eq. (preconditioner)
    equals the preconditioned matrix, P = M~_r + I + J~ = L~^-1 A^ L~^-T, since
    L~^-1 M^ L~^-T = sign(D).  A dense A with a diagonal S makes A^ dense, so the
    no-fill factorization is complete; these seeds give negative pivots (r > 0)."""
    rng = np.random.default_rng(seed)
    n = 14
    A = sp.csr_matrix(rng.standard_normal((n, n)) + 2.0 * np.eye(n))
    o = O.AsssOracle(A, S_pattern=sp.identity(n, format="csr"), k=0, factor="ildl0")
    assert o.r > 0 and abs(o.L).max() > 1.0
    Acal = np.column_stack([o.apply_op(e) for e in np.eye(n)])
    np.testing.assert_allclose(o.prec_dense(), Acal, rtol=0, atol=1e-10 * np.abs(Acal).max())
    J = o.fac.dense()
    np.testing.assert_allclose(J, -J.T, rtol=0, atol=1e-13 * np.abs(J).max())
    Acal_t = np.column_stack([o.apply_op(e, transpose=True) for e in np.eye(n)])
    np.testing.assert_allclose(Acal_t, Acal.T, rtol=0, atol=1e-12 * np.abs(Acal).max())


@pytest.mark.parametrize("kind", ["dh", "cd"])
def test_factored_solve_matches_dense_lu(kind):
    """The whole scheme with the incomplete factor: x agrees with a dense solve; the
    colours come from the structural pattern of A^ + A^T."""
    if kind == "dh":
        A, b, _ = dissipative_hamiltonian_3d(side=6, seed=11)
    else:
        A, b, _ = convection_diffusion_2d(m=10, seed=5)
    o = O.AsssOracle(A, k=6, inner_tol=1e-10, factor="ildl0")
    P = O.structural_pattern(o.Abar, o.S)
    rows = np.repeat(np.arange(o.n), np.diff(P.indptr))
    off = rows != P.indices
    assert np.all(o.colour[rows[off]] != o.colour[P.indices[off]])
    x, st = o.solve(b, tol=1e-10, outer="fgmres")
    xd = np.linalg.solve(A.toarray(), b)
    assert st["status"] == "ok"
    assert np.linalg.norm(x - xd) <= np.linalg.cond(A.toarray()) * 1e-10 * np.linalg.norm(xd)
    lam, _, st2 = o.solve_adjoint(b, tol=1e-10, outer="fgmres")
    np.testing.assert_allclose(A.T @ lam, b, atol=1e-9 * np.linalg.norm(b))


# ----------------------------------------------------------------------------
# planted mistakes: each must make a pin above fail
# ----------------------------------------------------------------------------
def _mutant(func_name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(O.ildl, func_name)))
    assert old in src, (func_name, old)
    ns = dict(vars(O.ildl))
    exec(compile(src.replace(old, new, 1), "<mutant>", "exec"), ns)
    return ns[func_name]


@pytest.mark.parametrize("old,new", [
    ("s -= lik * d[k] * ljk", "s -= lik * ljk"),
    ("di -= lik * lik * d[k]", "di -= lik * d[k]"),
    ("li[j] = s / d[j]", "li[j] = s"),
])
def test_planted_ildl_mistakes_are_caught(old, new):
    bad = _mutant("ildl0", old, new)
    rng = np.random.default_rng(5)
    n = 70
    M = _sym_random(n, 0.08, rng, 4.0)
    L, d = bad(M, rng.permutation(n))
    L1 = (L + sp.identity(n)).tocsr()
    R = (L1 @ sp.diags(d) @ L1.T).tocsr()
    assert np.abs(_on_pattern(R, M) - M.data).max() > 1e-6


def test_planted_colouring_mistake_is_caught():
    bad = _mutant("jp_colouring", "above = (prio[cols] > prio[rows])", "above = (prio[cols] < prio[rows])")
    rng = np.random.default_rng(1)
    G = _sym_random(80, 0.06, rng, 1.0)
    prio = O.colouring_priorities(1, 80)
    col, _ = bad(G, prio)
    assert not np.array_equal(col, _greedy_by_priority(G, prio))


# ----------------------------------------------------------------------------
# 2x2 pivot blocks (reading R20)
# ----------------------------------------------------------------------------
from workloads import saddle_pairs  # noqa: E402


def _pairs_of(partner):
    return sorted((int(i), int(j)) for i, j in enumerate(partner) if j > i)


def test_bk_pairs_follow_the_first_bunch_kaufman_test():
    """Each zero-diagonal row of saddle_pairs is coupled most strongly to its partner,
    which is zero-diagonal too: exactly those pairs are formed; a diagonally dominant
    matrix gets none."""
    A = saddle_pairs(30, seed=4, singles=6)
    M = 0.5 * (A + A.T)
    partner = O.ildl.bk_pairs(M)
    expect = []
    M1 = sp.csr_matrix(M)
    for i in range(30):
        if M1[i, i] == 0.0:
            row = M1.getrow(i).toarray().ravel()
            row[i] = 0.0
            j = int(np.argmax(np.abs(row)))
            if i < j:
                expect.append((i, j))
    assert len(expect) == 12 and _pairs_of(partner) == expect
    assert np.all(partner[partner >= 0] >= 0) and np.all(partner[partner[partner >= 0]] == np.flatnonzero(partner >= 0))
    rng = np.random.default_rng(2)
    assert np.all(O.ildl.bk_pairs(_sym_random(40, 0.1, rng, 4.0)) == -1)


def test_block_factor_without_pairs_is_the_1x1_factor():
    """With no pairs the block pattern, the quotient colouring and the block factor are
    the 1x1 ones."""
    rng = np.random.default_rng(5)
    n = 70
    M = _sym_random(n, 0.08, rng, 0.3)
    none = np.full(n, -1)
    Pb = O.ildl.block_pattern(M, none)
    assert (abs(Pb - sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape))).nnz == 0
    prio = O.colouring_priorities(9, n)
    col, _ = O.ildl.jp_colouring_blocks(M, prio, none)
    col1, _ = O.jp_colouring(M, prio)
    np.testing.assert_array_equal(col, col1)
    L, D = O.ildl.ildl0_blocks(M, col, none)
    L1, d1 = O.ildl0(M, O.colour_order(col1))
    # equal up to rounding (the block form multiplies by D_K^-1 where the 1x1 form divides)
    np.testing.assert_allclose(L.toarray(), L1.toarray(), rtol=1e-10, atol=1e-12 * abs(L1).max())
    np.testing.assert_allclose(D.toarray(), np.diag(d1), rtol=1e-10, atol=1e-12 * np.abs(d1).max())


@pytest.mark.parametrize("seed", [1, 6])
def test_block_factor_reproduces_the_matrix_on_its_block_pattern(seed):
    """The defining property of a no-fill factorization, for pivot blocks: (I + L) D
    (I + L)^T equals M at every position of the block pattern; L has entries only
    there, between blocks of smaller colour; the colouring is proper on the quotient
    graph (no two adjacent blocks share a colour; both members of a pair share one)."""
    A = saddle_pairs(60, seed=seed, singles=8)
    M = (0.5 * (A + A.T)).tocsr()
    partner = O.ildl.bk_pairs(M)
    Pb = O.ildl.block_pattern(M, partner)
    MP = O.values_on_pattern(M, Pb)
    col, _ = O.ildl.jp_colouring_blocks(Pb, O.colouring_priorities(seed, 60), partner)
    p = partner
    rows = np.repeat(np.arange(60), np.diff(Pb.indptr))
    cols = Pb.indices
    same_block = (cols == rows) | (p[rows] == cols)
    assert np.all(col[rows[~same_block]] != col[cols[~same_block]])
    assert np.all(col[p >= 0] == col[p[p >= 0]])
    L, D = O.ildl.ildl0_blocks(MP, col, partner)
    L1 = (L + sp.identity(60)).tocsr()
    R = (L1 @ D @ L1.T).tocsr()
    np.testing.assert_allclose(_on_pattern(R, Pb), MP.data, rtol=0, atol=1e-12 * abs(M).max())
    Lc = L.tocoo()
    assert np.all(col[Lc.row] > col[Lc.col])
    assert (abs(L) - abs(L).multiply(Pb)).nnz == 0 or abs(abs(L) - abs(L).multiply(Pb)).max() == 0


def test_block_factor_is_exact_on_a_dense_indefinite_matrix():
    """No fill is possible in a dense pattern, so the block factor is an exact
    factorization - also of a matrix with a zero diagonal that no 1x1 pivot order can
    factor (the 1x1 factor meets a zero pivot)."""
    rng = np.random.default_rng(3)
    n = 10
    B = rng.standard_normal((n, n))
    M = 0.1 * (B + B.T)
    for t in range(0, n, 2):
        M[t, t] = M[t + 1, t + 1] = 0.0
        M[t, t + 1] = M[t + 1, t] = 2.0 + t
    Ms = sp.csr_matrix(M)
    partner = O.ildl.bk_pairs(Ms)
    assert _pairs_of(partner) == [(t, t + 1) for t in range(0, n, 2)]
    Pb = O.ildl.block_pattern(Ms, partner)
    col, _ = O.ildl.jp_colouring_blocks(Pb, O.colouring_priorities(0, n), partner)
    L, D = O.ildl.ildl0_blocks(O.values_on_pattern(Ms, Pb), col, partner)
    L1 = L.toarray() + np.eye(n)
    np.testing.assert_allclose(L1 @ D.toarray() @ L1.T, M, rtol=0, atol=1e-12 * np.abs(M).max())
    with pytest.raises(ZeroDivisionError):
        O.ildl0(sp.csr_matrix(M + 0.0 * np.ones((n, n))), O.colour_order(col))


def test_block_pivot_split_is_fig1():
    """|D|^(-1/2) D |D|^(-1/2) = sign(D) block by block, and sign(D) - I = U_r Sigma_r
    U_r^T with Sigma_r = -2 I: a 2x2 block with eigenvalues of both signs contributes its
    negative eigenvector (sign(D_I) - I has the eigenvalues {-2, 0} of Fig. 1), a
    negative definite one two columns, a positive definite one none, a negative 1x1
    pivot e_i."""
    D = sp.csr_matrix(np.array([[0.5, 2.0, 0, 0, 0, 0, 0],
                                [2.0, -1.0, 0, 0, 0, 0, 0],
                                [0, 0, -3.0, 1.0, 0, 0, 0],
                                [0, 0, 1.0, -2.0, 0, 0, 0],
                                [0, 0, 0, 0, 4.0, 1.0, 0],
                                [0, 0, 0, 0, 1.0, 3.0, 0],
                                [0, 0, 0, 0, 0, 0, -0.25]]))
    partner = np.array([1, 0, 3, 2, 5, 4, -1])
    W, U, sig = O.ildl.block_pivot_split(D, partner)
    Dd, Wd = D.toarray(), W.toarray()
    lam, V = np.linalg.eigh(Dd)
    sgn = V @ np.diag(np.sign(lam)) @ V.T
    np.testing.assert_allclose(Wd @ Dd @ Wd, sgn, atol=1e-13)
    np.testing.assert_allclose(U @ np.diag(sig) @ U.T, sgn - np.eye(7), atol=1e-13)
    assert U.shape[1] == 4 and np.all(sig == -2.0)
    ev = np.linalg.eigvalsh((sgn - np.eye(7))[:2, :2])
    np.testing.assert_allclose(np.sort(ev), [-2.0, 0.0], atol=1e-13)


def test_block_preconditioner_is_exact_for_a_complete_factor():
    """§3 with 2x2 pivots: with a complete block factor (dense A, S = I) P = M~_r + I + J~
    equals the preconditioned matrix L~^-1 A^ L~^-T."""
    rng = np.random.default_rng(4)
    n = 12
    Ad = 0.2 * rng.standard_normal((n, n))
    for t in range(0, n, 2):
        Ad[t, t] = Ad[t + 1, t + 1] = 0.0
        Ad[t, t + 1] += 1.5
        Ad[t + 1, t] += 1.5
    A = sp.csr_matrix(Ad)
    I = sp.identity(n, format="csr")
    o = O.AsssOracle(A, S=I, dr=np.ones(n), dc=np.ones(n), k=0, factor="ildl0_bk")
    assert int((o.partner >= 0).sum()) == n and o.r > 0
    Acal = np.column_stack([o.apply_op(e) for e in np.eye(n)])
    np.testing.assert_allclose(o.prec_dense(), Acal, rtol=0, atol=1e-10 * np.abs(Acal).max())
    J = o.fac.dense()
    np.testing.assert_allclose(J, -J.T, rtol=0, atol=1e-12 * np.abs(J).max())


def test_block_factored_solve_matches_dense_lu():
    """The whole scheme on a matrix only 2x2 pivots factor: x and the adjoint agree with
    dense solves, both outer methods."""
    A = saddle_pairs(50, seed=8, singles=6)
    n = 50
    b = np.random.default_rng(8).standard_normal(n)
    I = sp.identity(n, format="csr")
    o = O.AsssOracle(A, S=I, dr=np.ones(n), dc=np.ones(n), k=4, inner_tol=1e-12, factor="ildl0_bk")
    xd = np.linalg.solve(A.toarray(), b)
    for outer in ("fgmres", "tfqmr"):
        x, st = o.solve(b, tol=1e-10, outer=outer)
        assert st["status"] == "ok"
        assert np.linalg.norm(x - xd) <= np.linalg.cond(A.toarray()) * 1e-10 * np.linalg.norm(xd)
    lam, _, _ = o.solve_adjoint(b, tol=1e-10, outer="fgmres")
    np.testing.assert_allclose(A.T @ lam, b, atol=1e-9 * np.linalg.norm(b))


@pytest.mark.parametrize("old,new", [
    ("LI[K] = S @ np.linalg.inv(Db[K])", "LI[K] = S"),
    ("S -= LI[K2] @ Db[K2] @ LK2.T", "S -= LI[K2] @ LK2.T"),
    ("DI -= LIK @ Db[K] @ LIK.T", "DI -= LIK @ LIK.T"),
])
def test_planted_block_factor_mistakes_are_caught(old, new):
    bad = _mutant("ildl0_blocks", old, new)
    A = saddle_pairs(60, seed=1, singles=8)
    M = (0.5 * (A + A.T)).tocsr()
    partner = O.ildl.bk_pairs(M)
    Pb = O.ildl.block_pattern(M, partner)
    MP = O.values_on_pattern(M, Pb)
    col, _ = O.ildl.jp_colouring_blocks(Pb, O.colouring_priorities(1, 60), partner)
    try:
        L, D = bad(MP, col, partner)
    except ZeroDivisionError:
        return
    L1 = (L + sp.identity(60)).tocsr()
    R = (L1 @ D @ L1.T).tocsr()
    assert np.abs(_on_pattern(R, Pb) - MP.data).max() > 1e-6
