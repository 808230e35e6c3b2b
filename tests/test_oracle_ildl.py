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
