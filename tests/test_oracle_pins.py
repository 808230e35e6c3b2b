"""Pins for the FP64 CPU oracle against the paper and against mathematics that does
not come from the oracle itself (arXiv 2009.06954).

Each test names the passage it pins.  None of them calls the CUDA path.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from workloads import (convection_diffusion_2d, dissipative_hamiltonian_3d,
                       pattern_diagonal, pattern_of, pattern_tridiagonal)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
def _read_lls_golden():
    cases = []
    with open(os.path.join(GOLDEN, "lls_small.txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        tok = lines[i].split()
        assert tok[0] == "case"
        name, gamma = tok[1], float(tok[2])
        i += 1
        mats = {}
        while lines[i] != "end":
            tok = lines[i].split()
            if tok[0] == "v":
                mats["v"] = np.array([float(t) for t in tok[1:]])
                i += 1
                continue
            r, c = int(tok[1]), int(tok[2])
            mats[tok[0]] = np.array([[float(t) for t in lines[i + 1 + k].split()] for k in range(r)])
            assert mats[tok[0]].shape == (r, c)
            i += 1 + r
        i += 1
        cases.append((name, gamma, mats))
    return cases


def _random_sparse(n, density, rng, diag=True):
    M = sp.random(n, n, density=density, random_state=rng, data_rvs=rng.standard_normal).tocsr()
    if diag:
        M = M + sp.diags(rng.uniform(0.5, 2.0, n) * rng.choice([-1, 1], n))
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return M


def _dense_lls_minimiser(Abar, Spat, gamma):
    """Brute force, independent of the B assembly: the residual map
    s -> [((Abar S) + (Abar S)^T)_ij for ALL i<j ; sqrt(gamma)(diag(Abar S) - 1)]
    is affine in s; build its Jacobian column by column from dense products and
    solve the least-squares problem with a dense SVD-based solver (§2 Eq. regularized)."""
    Ad = Abar.toarray()
    Sp = sp.csr_matrix(Spat)
    Sp.sort_indices()
    n = Ad.shape[0]
    rows = np.repeat(np.arange(n), np.diff(Sp.indptr))
    cols = Sp.indices
    iu = np.triu_indices(n, 1)

    def resid(s):
        S = np.zeros((n, n))
        S[rows, cols] = s
        C = Ad @ S
        return np.concatenate([(C + C.T)[iu], np.sqrt(gamma) * (np.diag(C) - 1.0)])

    r0 = resid(np.zeros(rows.size))
    Jm = np.column_stack([resid(np.eye(rows.size)[u]) - r0 for u in range(rows.size)])
    s = np.linalg.lstsq(Jm, -r0, rcond=None)[0]
    return s, rows, cols


# ----------------------------------------------------------------------------
# counter-based generator
# ----------------------------------------------------------------------------
def test_splitmix64_published_first_output():
    # splitmix64 seeded with 0 returns 0xE220A8397B1DCDAF first (published value).
    u = O.splitmix64_uniform(0, 3)
    expect = ((0xE220A8397B1DCDAF >> 11) * 2.0 ** -53) * 2.0 - 1.0
    assert u[0] == expect
    v = O.splitmix64_uniform(12345, 200000)
    assert np.all(np.abs(v) < 1.0) and abs(v.mean()) < 0.01 and abs(v.var() - 1 / 3) < 0.01


# ----------------------------------------------------------------------------
# §2 Eq. (mc64): scaling
# ----------------------------------------------------------------------------
def test_equilibrate_bounds():
    rng = np.random.default_rng(1)
    A = _random_sparse(60, 0.08, rng) * 37.0
    Abar, dr, dc, perm = O.equilibrate(A)
    M = abs(Abar).toarray()
    assert M.max() <= 1.0 + 1e-15
    np.testing.assert_allclose(M.max(axis=0), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(Abar.toarray(), np.diag(dr) @ A.toarray() @ np.diag(dc), rtol=1e-15, atol=0)
    p = rng.permutation(60)
    Abar2, _, _, _ = O.equilibrate(A, row_perm=p, dr=dr, dc=dc)
    np.testing.assert_array_equal(Abar2.toarray(), Abar.toarray()[p])


# ----------------------------------------------------------------------------
# §2 and App. A: the least-squares problem
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("case", _read_lls_golden(), ids=lambda c: c[0])
def test_lls_matrix_matches_hand_derivation(case):
    name, gamma, m = case
    B, v, _ = O.lls_system(sp.csr_matrix(m["A"]), sp.csr_matrix(m["S"]), gamma)
    np.testing.assert_array_equal(B.toarray(), m["B"])
    np.testing.assert_array_equal(v, m["v"])


def test_lls_diagonal_counts():
    """§2 after Eq. (lls_problem): with diagonal S each symmetry row has the two
    entries abar_ij, abar_ji, so nnz(B) = nnz(Abar) and the row count is
    n + nnz(triu(pat(Abar) + pat(Abar)^T, 1)) (the S_d columns of Table 2 obey this)."""
    rng = np.random.default_rng(2)
    for n in (5, 40, 200):
        A = _random_sparse(n, 0.05, rng)
        B, v, _ = O.lls_system(A, pattern_diagonal(n), 1.0)
        P = abs(A) + abs(A).T
        assert B.nnz == A.nnz
        assert B.shape == (n + sp.triu(P, 1).nnz, n)
        assert np.all(np.diff(B.indptr)[: B.shape[0] - n] <= 2)


def test_lls_exact_skew_symmetrizer_recovered():
    """If Abar = (I + K) D^-1 with K skew and D diagonal, S = D makes Abar S = I + K,
    a zero of f (Eqs. eq1, eq2); with the diagonal pattern it is the unique minimiser."""
    rng = np.random.default_rng(3)
    n = 50
    K = sp.random(n, n, density=0.06, random_state=rng, data_rvs=rng.standard_normal)
    K = sp.csr_matrix(K - K.T)
    D = rng.uniform(0.5, 2.0, n)
    Abar = ((sp.identity(n) + K) @ sp.diags(1.0 / D)).tocsr()
    Abar.sort_indices()
    for method in ("normal", "lsqr", "dense"):
        S = O.skew_symmetrizer(Abar, pattern_diagonal(n), 1.0, method)
        np.testing.assert_allclose(S.diagonal(), D, rtol=1e-10)
    # Abar already I + K: S = I
    IK = (sp.identity(n) + K).tocsr()
    S = O.skew_symmetrizer(IK, pattern_diagonal(n), 1.0)
    np.testing.assert_allclose(S.diagonal(), 1.0, rtol=1e-12)
    # a wider pattern still reaches a zero residual
    S = O.skew_symmetrizer(Abar, pattern_of(Abar), 1.0)
    C = (Abar @ S).toarray()
    off = C + C.T - 2 * np.diag(np.diag(C))
    assert np.abs(off).max() < 1e-10 and np.abs(np.diag(C) - 1).max() < 1e-10


@pytest.mark.parametrize("gamma", [1.0, 10.0, 0.1])
@pytest.mark.parametrize("pattern", ["diag", "tri", "A", "random"])
def test_lls_minimiser_matches_dense_brute_force(gamma, pattern):
    rng = np.random.default_rng(4)
    n = 9
    A = _random_sparse(n, 0.25, rng)
    Abar, _, _, _ = O.equilibrate(A)
    if pattern == "diag":
        Sp = pattern_diagonal(n)
    elif pattern == "tri":
        Sp = pattern_tridiagonal(n)
    elif pattern == "A":
        Sp = pattern_of(Abar)
    else:
        Sp = (sp.random(n, n, density=0.3, random_state=rng) + sp.identity(n)).tocsr()
        Sp.data[:] = 1.0
        Sp.sort_indices()
    s_ref, rows, cols = _dense_lls_minimiser(Abar, Sp, gamma)
    for method in ("normal", "dense"):
        S = O.skew_symmetrizer(Abar, Sp, gamma, method)
        np.testing.assert_allclose(np.asarray(S[rows, cols]).ravel(), s_ref, rtol=1e-8, atol=1e-10)


# ----------------------------------------------------------------------------
# §3: diagonal factor, M~_r and its low-rank decomposition (Fig. 1)
# ----------------------------------------------------------------------------
def test_lowrank_decomposition_fig1():
    d = np.array([1.2, -0.7, 0.9, -3.0, -0.1, 2.0])
    Mr = np.diag(np.sign(d)) - np.eye(d.size)     # L_|D|^-1 D L_|D|^-T - I
    ind = np.flatnonzero(np.diag(Mr))
    U, sig = O.lowrank_decomposition(Mr[np.ix_(ind, ind)])
    Ur = np.zeros((d.size, U.shape[1]))
    Ur[ind] = U
    np.testing.assert_array_equal(Ur @ np.diag(sig) @ Ur.T, Mr)
    np.testing.assert_array_equal(sig, -2.0)
    # a 2x2 block with eigenvalues {-2, 0} (§3, the 2x2 case of Fig. 1)
    c, s = np.cos(0.3), np.sin(0.3)
    blk = -2.0 * np.outer([c, s], [c, s])
    U2, sig2 = O.lowrank_decomposition(blk)
    assert U2.shape == (2, 1)
    np.testing.assert_allclose(sig2, [-2.0], atol=1e-14)
    np.testing.assert_allclose(U2 @ np.diag(sig2) @ U2.T, blk, atol=1e-14)


def _small_setup(kind="dh", **kw):
    if kind == "dh":
        A, b, _ = dissipative_hamiltonian_3d(side=6, seed=11)
    elif kind == "cd":
        A, b, _ = convection_diffusion_2d(m=10, seed=5)
    else:
        rng = np.random.default_rng(12)
        A = _random_sparse(120, 0.04, rng)
        b = rng.standard_normal(120)
    return A, b, O.AsssOracle(A, **kw)


@pytest.mark.parametrize("kind", ["dh", "cd", "rand"])
def test_inner_skew_operator(kind):
    """J~ = W (Abar S - (Abar S)^T)/2 W is exactly skew (§3) and W Abar S W has the
    diagonal sign(d) (W = |d|^-1/2, reading R5)."""
    A, b, o = _small_setup(kind, k=4)
    Jt = o.Jt
    assert abs(Jt + Jt.T).max() == 0.0
    C = (o.Abar @ o.S).toarray()
    W = np.diag(o.w)
    np.testing.assert_allclose(Jt.toarray(), W @ (C - C.T) / 2 @ W, rtol=0, atol=1e-14 * np.abs(C).max())
    np.testing.assert_allclose(np.diag(W @ C @ W), np.sign(o.d), rtol=0, atol=1e-14)
    Mr = np.diag(np.sign(o.d)) - np.eye(o.n)
    assert np.count_nonzero(np.diag(Mr)) == np.sum(o.d < 0)


# ----------------------------------------------------------------------------
# §3.2 Fig. 2: skew-Lanczos
# ----------------------------------------------------------------------------
def test_skew_lanczos_relations():
    A, b, o = _small_setup("dh", k=12)
    Q, a = o.Q, o.alpha
    J = o.Jt
    assert Q.shape[1] == 12 and a.size == 11
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-12)
    np.testing.assert_allclose(Q.T @ (J @ Q), O.lanczos_tridiagonal(a), atol=1e-12)
    # Fig. 2 sign convention: q_2 = -J q_1 / alpha_1, S_k(1,2) = +alpha_1
    np.testing.assert_allclose(Q[:, 1], -(J @ Q[:, 0]) / a[0], atol=1e-14)
    assert np.all(a > 0)


def test_skew_lanczos_full_run_spectrum():
    """k = n (n even, tiny): S_k is orthogonally similar to J, so the spectra agree."""
    rng = np.random.default_rng(7)
    n = 10
    K = rng.standard_normal((n, n))
    J = sp.csr_matrix(K - K.T)
    Q, a = O.skew_lanczos(J, rng.standard_normal(n), n, reorth=True)
    assert Q.shape == (n, n)
    e1 = np.sort(np.linalg.eigvals(O.lanczos_tridiagonal(a)).imag)
    e2 = np.sort(np.linalg.eigvals(J.toarray()).imag)
    np.testing.assert_allclose(e1, e2, atol=1e-10)
    # without re-orthogonalisation a few steps stay orthogonal too
    Q2, a2 = O.skew_lanczos(J, rng.standard_normal(n), 4, reorth=False)
    np.testing.assert_allclose(Q2.T @ Q2, np.eye(4), atol=1e-10)


def test_skew_lanczos_breakdown():
    """An invariant subspace of dimension 2 ends the process (alpha_2 = 0, Fig. 2)."""
    n = 6
    J = np.zeros((n, n))
    J[0, 1], J[1, 0] = 2.0, -2.0
    J[2, 3], J[3, 2] = 1.0, -1.0
    q1 = np.zeros(n)
    q1[0] = 1.0
    Q, a = O.skew_lanczos(sp.csr_matrix(J), q1, 5)
    assert Q.shape[1] == 2 and a.size == 1 and a[0] == 2.0


# ----------------------------------------------------------------------------
# §3.1 and App. B: mrs
# ----------------------------------------------------------------------------
def _skew_dense(n, rng, scale=1.0):
    K = rng.standard_normal((n, n)) * scale
    return K - K.T


@pytest.mark.parametrize("alpha", [1.0, 0.3, 4.0])
def test_mrs_matches_dense_solve(alpha):
    rng = np.random.default_rng(8)
    n = 40
    J = _skew_dense(n, rng, 0.3)
    b = rng.standard_normal(n)
    x, its, ratio, hist = O.mrs(alpha, lambda V: J @ V, b, 4 * n, 1e-14)
    xd = np.linalg.solve(alpha * np.eye(n) + J, b)
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-12 * np.abs(xd).max())
    assert its <= 2 * n      # round-off delays the exact-arithmetic bound of n steps


def test_mrs_finite_termination_and_closed_form_2x2():
    """For J = [[0, w], [-w, 0]]: (I + J)^-1 = (I - J)/(1 + w^2); a 2-dimensional
    Krylov space is exhausted after 2 steps."""
    w = 3.7
    J = np.array([[0.0, w], [-w, 0.0]])
    b = np.array([0.4, -1.3])
    x, its, ratio, _ = O.mrs(1.0, lambda V: J @ V, b, 10, 1e-15)
    np.testing.assert_allclose(x, (np.eye(2) - J) @ b / (1 + w * w), rtol=1e-14)
    assert its == 2


def test_mrs_zero_skew_one_step():
    b = np.array([1.0, -2.0, 0.5])
    x, its, ratio, _ = O.mrs(2.5, lambda V: 0.0 * V, b, 10, 1e-12)
    assert its == 1 and ratio == 0.0
    np.testing.assert_allclose(x, b / 2.5, rtol=1e-15)


def test_mrs_residual_recursion_is_true_residual_and_monotone():
    """The recursive |g_k| equals ||b - (alpha I + J) x_k|| (Givens QR of the
    Lanczos relation) and never increases (minimal residual property, §3.1)."""
    rng = np.random.default_rng(9)
    n = 60
    J = _skew_dense(n, rng, 0.2)
    b = rng.standard_normal(n)
    nb = np.linalg.norm(b)
    prev = np.inf
    for k in range(1, 25):
        x, its, ratio, hist = O.mrs(1.0, lambda V: J @ V, b, k, 0.0)
        true = np.linalg.norm(b - x - J @ x) / nb
        assert abs(ratio - true) <= 1e-10 * max(true, 1e-300) + 1e-15
        assert ratio <= prev * (1 + 1e-14)
        prev = ratio
    h = np.array(hist)
    assert np.all(np.diff(h) <= 1e-15)


def test_mrs_multi_rhs_freeze_equals_independent_columns():
    """Reading R9: per-column freezing gives each column exactly its own single-RHS
    solve; the printed variant (no freezing) iterates all columns to the worst one."""
    rng = np.random.default_rng(10)
    n = 50
    J = _skew_dense(n, rng, 0.25)
    B = rng.standard_normal((n, 4))
    B[:, 2] = 0.0   # a zero column gives x = 0
    # apply J column by column so both runs do the same arithmetic per column
    colwise = lambda V: np.column_stack([J @ V[:, c] for c in range(V.shape[1])])
    X, its, ratio, _ = O.mrs(1.0, colwise, B, 200, 1e-9, freeze=True)
    for j in (0, 1, 3):
        xj, itj, rj, _ = O.mrs(1.0, lambda v: J @ v, B[:, j], 200, 1e-9)
        # (vector and matrix 2-norms still sum in different orders)
        np.testing.assert_allclose(X[:, j], xj, rtol=0, atol=1e-9 * np.abs(xj).max())
        assert abs(int(its[j]) - int(itj)) <= 1
    np.testing.assert_array_equal(X[:, 2], 0.0)
    X2, its2, ratio2, _ = O.mrs(1.0, lambda V: J @ V, B, 200, 1e-9, freeze=False)
    assert np.all(its2[[0, 1, 3]] == its.max()) and ratio2.max() < 1e-9
    Xd = np.linalg.solve(np.eye(n) + J, B)
    np.testing.assert_allclose(X2, Xd, atol=1e-7)


# ----------------------------------------------------------------------------
# §3.2 Eqs. (preconditioner), (smw): the combined low-rank preconditioner
# ----------------------------------------------------------------------------
def test_preconditioner_identity_and_smw_inverse():
    """P = [Q_k, U_r] blkdiag(S_k, Sig_r) [Q_k, U_r]^T + S_bar equals M~_r + I + J~
    for any Q_k (the deflation terms cancel), and the SMW application inverts P."""
    A, b, o = _small_setup("dh", k=8, inner_tol=1e-14, inner_maxit=2000)
    o.set_lowrank(np.array([3, 17, 40, 41, 100]))       # force r = 5
    P = o.prec_dense()
    Sbar = np.eye(o.n) + o.Jt.toarray() - o.Q @ o.Sk @ o.Q.T
    np.testing.assert_allclose(o.Ub @ o.Sig @ o.Ub.T + Sbar, P, atol=1e-14)
    rng = np.random.default_rng(13)
    u = rng.standard_normal(o.n)
    z = o.apply_prec_inv(u)
    np.testing.assert_allclose(P @ z, u, atol=1e-10)
    zt = o.apply_prec_inv(u, transpose=True)
    np.testing.assert_allclose(P.T @ zt, u, atol=1e-10)


# ----------------------------------------------------------------------------
# outer Krylov methods and the whole solve (§4.1)
# ----------------------------------------------------------------------------
def test_tfqmr_matches_independent_implementation():
    """Identity preconditioner: the oracle's TFQMR iterates equal scipy's
    independent TFQMR (Freund 1993) step for step."""
    A, b, _ = convection_diffusion_2d(m=8)
    xs = []
    spla.tfqmr(A, b, rtol=1e-30, maxiter=12, callback=lambda xk: xs.append(xk.copy()))
    for steps in range(1, 6):
        d, nsteps, _ = O.tfqmr_cycle(lambda v: A @ v, lambda u: u, b, 0.0, steps)
        np.testing.assert_allclose(d, xs[2 * steps - 1], rtol=0, atol=1e-12)


def test_fgmres_finite_termination():
    rng = np.random.default_rng(14)
    n = 25
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal(n)
    d, steps, _ = O.fgmres_cycle(lambda v: A @ v, lambda u: u, b, 0.0, n)
    np.testing.assert_allclose(d, np.linalg.solve(A, b), atol=1e-10)
    Ainv = np.linalg.inv(A)
    d, steps, _ = O.fgmres_cycle(lambda v: A @ v, lambda u: Ainv @ u, b, 1e-12, n)
    assert steps == 1
    np.testing.assert_allclose(d, np.linalg.solve(A, b), atol=1e-12)


@pytest.mark.parametrize("kind", ["dh", "cd", "rand"])
@pytest.mark.parametrize("outer", ["tfqmr", "fgmres"])
def test_solve_matches_dense_lu(kind, outer):
    A, b, o = _small_setup(kind, k=6, inner_tol=1e-10)
    # the random indefinite case has eigenvalues of P^-1 A_cal near 0, where
    # restarted GMRES(30) stagnates; an unrestarted cycle converges
    x, st = o.solve(b, tol=1e-10, outer=outer, restart=30 if kind != "rand" else o.n)
    xd = np.linalg.solve(A.toarray(), b)
    cond = np.linalg.cond(A.toarray())
    assert st["status"] == "ok"
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= cond * 1e-10 * np.linalg.norm(xd)


def test_solve_zero_rhs():
    A, b, o = _small_setup("dh", k=3)
    x, st = o.solve(np.zeros(o.n))
    assert st["status"] == "ok" and np.all(x == 0)


# ----------------------------------------------------------------------------
# adjoint: A^T lambda = dL/dx, dL/dA_ij = -lambda_i x_j
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["dh", "rand"])
def test_adjoint_matches_dense_and_finite_differences(kind):
    A, b, o = _small_setup(kind, k=6, inner_tol=1e-12)
    x, st = o.solve(b, tol=1e-12)
    rng = np.random.default_rng(15)
    xs = rng.standard_normal(o.n)
    g = 2.0 * (x - xs)                                   # L = ||x - x*||^2
    lam, dA, st2 = o.solve_adjoint(g, x=x, tol=1e-12)
    Ad = A.toarray()
    lam_d = np.linalg.solve(Ad.T, g)
    np.testing.assert_allclose(lam, lam_d, atol=1e-9 * np.abs(lam_d).max())
    x_d = np.linalg.solve(Ad, b)
    rows = np.repeat(np.arange(o.n), np.diff(A.indptr))
    dA_d = -np.linalg.solve(Ad.T, 2.0 * (x_d - xs))[rows] * x_d[A.indices]
    np.testing.assert_allclose(dA, dA_d, atol=1e-8 * np.abs(dA_d).max())
    # central differences of L in a few entries of A (dense solves, step 1e-6); the
    # truncation error of the difference quotient bounds the agreement
    for e in rng.choice(A.nnz, 6, replace=False):
        i, j = rows[e], A.indices[e]
        h = 1e-6
        Lp = np.sum((np.linalg.solve(Ad + h * np.eye(o.n)[i][:, None] * np.eye(o.n)[j][None, :], b) - xs) ** 2)
        Lm = np.sum((np.linalg.solve(Ad - h * np.eye(o.n)[i][:, None] * np.eye(o.n)[j][None, :], b) - xs) ** 2)
        fd = (Lp - Lm) / (2 * h)
        assert abs(dA[e] - fd) <= 1e-4 * max(1.0, abs(fd))


# ----------------------------------------------------------------------------
# planted mistakes: each of these must make a pin above fail
# ----------------------------------------------------------------------------
def _mutant(func_name, old, new):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(O.asss, func_name)))
    assert old in src, (func_name, old)
    ns = dict(vars(O.asss))
    exec(compile(src.replace(old, new, 1), "<mutant>", "exec"), ns)
    return ns[func_name]


@pytest.mark.parametrize("old,new", [
    ("delta = -s_prev * beta", "delta = s_prev * beta"),
    ("theta_t = c_prev * theta", "theta_t = c * theta"),
    ("g = np.where(upd, -g * s, g)", "g = np.where(upd, g * s, g)"),
    ("qh = apply_skew(q) + q_prev * beta", "qh = apply_skew(q) - q_prev * beta"),
])
def test_planted_mrs_mistakes_are_caught(old, new):
    bad = _mutant("mrs", old, new)
    rng = np.random.default_rng(8)
    n = 40
    J = _skew_dense(n, rng, 0.3)
    b = rng.standard_normal(n)
    x, its, ratio, _ = bad(1.0, lambda V: J @ V, b, 4 * n, 1e-14)
    xd = np.linalg.solve(np.eye(n) + J, b)
    true = np.linalg.norm(b - x - J @ x) / np.linalg.norm(b)
    assert np.abs(x - xd).max() > 1e-6 or abs(true - ratio) > 1e-6


@pytest.mark.parametrize("old,new", [
    ("val = np.where(off, p_a, np.sqrt(gamma) * p_a)", "val = np.where(off, p_a, gamma * p_a)"),
    ("p_j = s_cols[p_unk]", "p_j = a_cols.repeat(1)[np.minimum(p_unk, a_cols.size - 1)]"),
])
def test_planted_lls_mistakes_are_caught(old, new):
    bad = _mutant("lls_system", old, new)
    caught = False
    for name, gamma, m in _read_lls_golden():
        try:
            B, v, _ = bad(sp.csr_matrix(m["A"]), sp.csr_matrix(m["S"]), gamma)
            if B.shape != m["B"].shape or not np.array_equal(B.toarray(), m["B"]):
                caught = True
        except Exception:
            caught = True
    assert caught


def test_planted_lanczos_sign_mistake_is_caught():
    bad = _mutant("skew_lanczos", "Q[:, i] = -z / a", "Q[:, i] = z / a")
    A, b, o = _small_setup("dh", k=6)
    Q, a = bad(o.Jt, O.splitmix64_uniform(1, o.n), 6)
    err = np.abs(Q.T @ (o.Jt @ Q) - O.lanczos_tridiagonal(a)).max()
    assert err > 1e-3
