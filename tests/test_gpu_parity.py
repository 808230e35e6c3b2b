"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every test here needs a GB300 (marked gpu).  Sizes span several 32-row slices with
a ragged tail; the oracle computes the expected values on the same seeded inputs.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import (convection_diffusion_2d, dissipative_hamiltonian_3d, pattern_diagonal,
                       pattern_of, pattern_tridiagonal)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_06954_gb300 as p
    return p


@pytest.fixture(params=["auto", "evict_first"])
def loads(request, monkeypatch):
    """Both load paths of the kernels: "auto" takes evict-first loads only when a
    pass's data exceed L2 (the full-size bench), "evict_first" forces them here at
    small sizes (ASSS_FORCE_EVICT_FIRST, read when the library makes a context)."""
    if request.param == "evict_first":
        monkeypatch.setenv("ASSS_FORCE_EVICT_FIRST", "1")
    else:
        monkeypatch.delenv("ASSS_FORCE_EVICT_FIRST", raising=False)
    return request.param


def random_skew(n, per_row, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    K = sp.random(n, n, density=per_row / (2.0 * n), random_state=rng, data_rvs=rng.standard_normal)
    J = (K - K.T).tocsr() * scale
    J.sum_duplicates()
    J.sort_indices()
    J.eliminate_zeros()
    return J


# ----------------------------------------------------------------------------
# mrs (the hot kernel), same operator on both sides
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [37, 1000, 50001])
@pytest.mark.parametrize("k", [0, 20])
@pytest.mark.parametrize("shift,sign", [(1.0, 1.0), (1.0, -1.0), (0.5, 1.0)])
def test_mrs_fp64_matches_oracle(pkg, n, k, shift, sign):
    J = random_skew(n, 12, seed=n + k)
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n)
    Q = alpha = None
    if k:
        Q, alpha = O.skew_lanczos(J, rng.standard_normal(n), k)
    kk = 0 if Q is None else Q.shape[1]
    Sk = O.lanczos_tridiagonal(alpha) if kk else None

    def apply(V):
        out = J @ V
        if kk:
            out = out - Q @ (Sk @ (Q.T @ V))
        return sign * out

    xo, its_o, ratio_o, _ = O.mrs(shift, apply, b, 3000, 1e-12)
    xg, its_g, ratio_g = pkg.mrs(J, b, Q, alpha, shift=shift, sign=sign, tol=1e-12, maxit=3000)
    assert abs(its_g - its_o) <= 2, (its_g, its_o)
    assert ratio_g < 1e-12
    np.testing.assert_allclose(xg, xo, rtol=0, atol=1e-9 * np.abs(xo).max())
    true = np.linalg.norm(b - shift * xg - apply(xg)) / np.linalg.norm(b)
    assert true <= 1e-11


@pytest.mark.parametrize("n", [1000, 50001])
def test_mrs_fp32(pkg, n, loads):
    J = random_skew(n, 12, seed=3 * n)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(n)
    Q, alpha = O.skew_lanczos(J, rng.standard_normal(n), 20)
    Sk = O.lanczos_tridiagonal(alpha)
    apply = lambda V: J @ V - Q @ (Sk @ (Q.T @ V))
    xo, its_o, _, _ = O.mrs(1.0, apply, b, 3000, 1e-12)
    xg, its_g, ratio_g = pkg.mrs(J, b, Q, alpha, tol=1e-5, maxit=3000, precision="mixed")
    true = np.linalg.norm(b - xg - apply(xg)) / np.linalg.norm(b)
    assert ratio_g < 1e-5 and true <= 5e-5
    np.testing.assert_allclose(xg, xo, rtol=0, atol=1e-4 * np.abs(xo).max())


def test_mrs_edge_cases(pkg):
    n = 70
    J = random_skew(n, 6, seed=1)
    x, its, ratio = pkg.mrs(J, np.zeros(n), tol=1e-10)
    assert its == 0 and np.all(x == 0)
    Z = sp.csr_matrix((np.zeros(n), np.arange(n), np.arange(n + 1)), shape=(n, n))
    b = np.random.default_rng(2).standard_normal(n)
    x, its, ratio = pkg.mrs(Z, b, shift=2.0, tol=1e-12)
    assert its == 1 and np.allclose(x, b / 2.0, rtol=1e-15)
    # 2x2 closed form: (I + J)^-1 = (I - J)/(1 + w^2)
    w = 3.7
    J2 = sp.csr_matrix(np.array([[0.0, w], [-w, 0.0]]))
    b2 = np.array([0.4, -1.3])
    x, its, ratio = pkg.mrs(J2, b2, tol=1e-15, maxit=10)
    np.testing.assert_allclose(x, (np.eye(2) - J2.toarray()) @ b2 / (1 + w * w), rtol=1e-14)
    assert its == 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mrs_stops_at_maxit_with_the_oracle_iterate(pkg, precision):
    """An iteration limit below convergence: its = maxit, the ratio above tol, and x is
    the oracle's iterate after the same number of steps (App. B, reading R9)."""
    n = 2000
    J = random_skew(n, 10, seed=31)
    b = np.random.default_rng(32).standard_normal(n)
    xo, its_o, ratio_o, _ = O.mrs(1.0, lambda V: J @ V, b, 3, 1e-14)
    x, its, ratio = pkg.mrs(J, b, tol=1e-14, maxit=3, precision=precision)
    assert its == 3 and its_o == 3
    rtol = 1e-12 if precision == "fp64" else 2e-5
    assert abs(ratio - ratio_o) <= rtol * ratio_o
    np.testing.assert_allclose(x, xo, rtol=0, atol=rtol * np.abs(xo).max())


# ----------------------------------------------------------------------------
# skew-Lanczos (Fig. 2)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("reorth", [True, False])
def test_skew_lanczos_matches_oracle(pkg, reorth):
    n = 3001
    J = random_skew(n, 10, seed=11)
    q1 = np.random.default_rng(3).standard_normal(n)
    k = 20 if reorth else 8
    Qo, ao = O.skew_lanczos(J, q1, k, reorth=reorth)
    Qg, ag = pkg.skew_lanczos(J, q1, k, reorth=reorth)
    assert Qg.shape == Qo.shape
    np.testing.assert_allclose(ag, ao, rtol=1e-10)
    assert np.abs(Qg - Qo).max() <= 1e-9


def test_skew_lanczos_breakdown_matches_oracle(pkg):
    """q1 inside an invariant subspace of dimension 4 (two 2x2 rotation blocks of a
    block-diagonal skew J): the process stops with k_eff = 4 (Fig. 2 breakdown)."""
    nb = 40
    rng = np.random.default_rng(21)
    w = 0.5 + rng.random(nb)
    rows, cols, vals = [], [], []
    for b, wb in enumerate(w):
        i = 2 * b
        rows += [i, i + 1]
        cols += [i + 1, i]
        vals += [wb, -wb]
    J = sp.csr_matrix((vals, (rows, cols)), shape=(2 * nb, 2 * nb))
    q1 = np.zeros(2 * nb)
    q1[[4, 5, 10, 11]] = rng.standard_normal(4)
    Qo, ao = O.skew_lanczos(J, q1, 10)
    Qg, ag = pkg.skew_lanczos(J, q1, 10)
    assert Qo.shape[1] == 4 and Qg.shape[1] == 4
    np.testing.assert_allclose(ag, ao, rtol=1e-12)
    assert np.abs(Qg - Qo).max() <= 1e-12


# ----------------------------------------------------------------------------
# the least-squares fit of S (§2, App. A)
# ----------------------------------------------------------------------------
def _objective(Abar, S, gamma):
    C = (Abar @ S).tocsr()
    U = sp.triu(C + C.T, 1)
    d = C.diagonal()
    return float((U.data ** 2).sum() + gamma * ((d - 1.0) ** 2).sum())


@pytest.mark.parametrize("case", ["cd", "dh", "dh_tri", "dh_diag"])
def test_skew_symmetrizer_matches_oracle(pkg, case):
    if case == "cd":
        A, _, _ = convection_diffusion_2d(m=40)
    else:
        A, _, _ = dissipative_hamiltonian_3d(side=9, seed=4)
    Abar, _, _, _ = O.equilibrate(A)
    n = A.shape[0]
    Sp = {"cd": pattern_of(Abar), "dh": pattern_of(Abar), "dh_tri": pattern_tridiagonal(n),
          "dh_diag": pattern_diagonal(n)}[case]
    So = O.skew_symmetrizer(Abar, Sp, 1.0)
    sg, st = pkg.skew_symmetrizer(Abar, Sp, gamma=1.0)
    Sg = sp.csr_matrix((sg, Sp.indices, Sp.indptr), shape=Sp.shape)
    fo, fg = _objective(Abar, So, 1.0), _objective(Abar, Sg, 1.0)
    assert fg <= fo * (1 + 1e-9) + 1e-14
    assert np.linalg.norm(sg - So[np.repeat(np.arange(n), np.diff(Sp.indptr)), Sp.indices].A1) \
        <= 1e-6 * np.linalg.norm(So.data)
    assert st["lls_relgrad"] <= 1e-12


def test_skew_symmetrizer_exact_case(pkg):
    """Abar = (I + K) D^-1: S = D exactly on the diagonal pattern (Eqs. eq1, eq2)."""
    rng = np.random.default_rng(3)
    n = 500
    K = sp.random(n, n, density=0.01, random_state=rng, data_rvs=rng.standard_normal)
    K = sp.csr_matrix(K - K.T)
    D = rng.uniform(0.5, 2.0, n)
    Abar = ((sp.identity(n) + K) @ sp.diags(1.0 / D)).tocsr()
    Abar.sort_indices()
    sg, _ = pkg.skew_symmetrizer(Abar, pattern_diagonal(n))
    np.testing.assert_allclose(sg, D, rtol=1e-9)


# ----------------------------------------------------------------------------
# whole set-up and solve
# ----------------------------------------------------------------------------
def test_setup_matches_oracle_cd64(pkg):
    A, b, _ = convection_diffusion_2d(m=64)
    o = O.AsssOracle(A, inner_tol=1e-10)
    s = pkg.Solver(A, inner_tol=1e-10)
    ex = s.export(A.nnz)
    np.testing.assert_allclose(ex["dr"], o.dr, rtol=1e-15)
    np.testing.assert_allclose(ex["dc"], o.dc, rtol=1e-15)
    np.testing.assert_allclose(ex["d"], o.d, rtol=1e-7)
    np.testing.assert_allclose(ex["w"], o.w, rtol=1e-7)
    assert ex["Q"].shape == o.Q.shape
    np.testing.assert_allclose(ex["alpha"], o.alpha, rtol=1e-6)
    assert s.setup_stats["r"] == o.r


@pytest.mark.parametrize("outer", ["tfqmr", "fgmres"])
def test_solve_cd64_fp64_matches_oracle(pkg, outer):
    A, b, xt = convection_diffusion_2d(m=64)
    o = O.AsssOracle(A, inner_tol=1e-10)
    xo, sto = o.solve(b, tol=1e-8, outer=outer)
    s = pkg.Solver(A, inner_tol=1e-10, outer=outer)
    xg, stg = s.solve(b)
    assert stg["status"] == 0
    res = np.linalg.norm(b - A @ xg) / np.linalg.norm(b)
    assert res <= 1e-8
    assert abs(stg["outer_its"] - sto["outer_its"]) <= 2, (stg["outer_its"], sto["outer_its"])
    assert abs(stg["inner_its_avg"] - sto["inner_its_avg"]) <= 0.02 * sto["inner_its_avg"] + 2
    assert np.linalg.norm(xg - xo) <= 1e-5 * np.linalg.norm(xo)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_dh_matches_dense(pkg, precision):
    A, b, _ = dissipative_hamiltonian_3d(side=16, seed=9)
    s = pkg.Solver(A, precision=precision, outer="fgmres",
                   inner_tol=1e-6 if precision == "mixed" else 1e-10)
    x, st = s.solve(b)
    assert st["status"] == 0
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    xd = sp.linalg.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_solve_multiple_rhs_and_zero(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=8, seed=2)
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6)
    B = np.column_stack([b, np.zeros_like(b), 2 * b])
    X, st = s.solve(B)
    assert np.all(X[:, 1] == 0)
    np.testing.assert_allclose(X[:, 2], 2 * X[:, 0], rtol=1e-6)


def test_adjoint_matches_dense(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=8, seed=4)
    n = A.shape[0]
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-11)
    x, _ = s.solve(b)
    rng = np.random.default_rng(1)
    xs = rng.standard_normal(n)
    g = 2.0 * (x - xs)
    lam, dA, st = s.solve_adjoint(g, x=x)
    Ad = A.toarray()
    lam_d = np.linalg.solve(Ad.T, g)
    assert np.linalg.norm(lam - lam_d) <= 1e-9 * np.linalg.norm(lam_d)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    np.testing.assert_allclose(dA, -lam[rows] * x[A.indices], rtol=1e-14)
    # the same gradient into caller-owned pinned host buffers, and into device buffers
    import torch
    lam_p = torch.empty(n, dtype=torch.float64).pin_memory()
    dA_p = torch.empty(A.nnz, dtype=torch.float64).pin_memory()
    r = s.solve_adjoint(torch.tensor(g).pin_memory(), torch.tensor(x).pin_memory(), lam=lam_p, dA=dA_p)
    assert r[0] is lam_p and r[1] is dA_p
    # (same path; tolerance rather than bit equality, as a SELL inner operator sums in a
    # dynamic slice order)
    close = lambda u, v: np.linalg.norm(u - v) <= 1e-9 * np.linalg.norm(v)
    assert close(lam_p.numpy(), lam) and close(dA_p.numpy(), dA)
    lam_d2 = torch.empty(n, dtype=torch.float64, device="cuda")
    dA_d2 = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    s.solve_adjoint(torch.tensor(g, device="cuda"), torch.tensor(x, device="cuda"), lam=lam_d2, dA=dA_d2)
    assert close(lam_d2.cpu().numpy(), lam) and close(dA_d2.cpu().numpy(), dA)
    with pytest.raises(ValueError):
        s.solve_adjoint(g, x, dA=np.empty(A.nnz - 1))


def test_torch_autograd(pkg):
    import torch
    A, b, _ = dissipative_hamiltonian_3d(side=8, seed=6)
    n = A.shape[0]
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-11)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    av = torch.tensor(A.data, device="cuda", requires_grad=True)
    xs = torch.randn(n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    x = pkg.asss_solve(s, bt, av)
    loss = ((x - xs) ** 2).sum()
    loss.backward()
    Ad = A.toarray()
    xd = np.linalg.solve(Ad, b)
    lam_d = np.linalg.solve(Ad.T, 2 * (xd - xs.cpu().numpy()))
    np.testing.assert_allclose(bt.grad.cpu().numpy(), lam_d, rtol=0, atol=1e-8 * np.abs(lam_d).max())
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    np.testing.assert_allclose(av.grad.cpu().numpy(), -lam_d[rows] * xd[A.indices], rtol=0,
                               atol=1e-8 * np.abs(lam_d).max() * np.abs(xd).max())


# ----------------------------------------------------------------------------
# skew half-diagonal storage of J~ (same results as SELL-C and the oracle)
# ----------------------------------------------------------------------------
def banded_skew(n, offsets, seed, fill=0.9, scale=0.1):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for m in offsets:
        i = np.arange(n - m)
        i = i[rng.random(i.size) < fill]
        v = rng.standard_normal(i.size) * scale
        rows += [i, i + m]
        cols += [i + m, i]
        vals += [v, -v]
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    J.sort_indices()
    return J


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mrs_diag_storage_matches_sell_and_oracle(pkg, precision, loads):
    n = 40001
    J = banded_skew(n, (1, 3, 64, 1000, 20000), seed=5)
    rng = np.random.default_rng(6)
    b = rng.standard_normal(n)
    Q, alpha = O.skew_lanczos(J, rng.standard_normal(n), 20)
    Sk = O.lanczos_tridiagonal(alpha)
    apply = lambda V: J @ V - Q @ (Sk @ (Q.T @ V))
    xo, its_o, _, _ = O.mrs(1.0, apply, b, 3000, 1e-12)
    tol = 1e-12 if precision == "fp64" else 1e-5
    xd, its_d, rd = pkg.mrs(J, b, Q, alpha, tol=tol, maxit=3000, precision=precision, fmt="diag")
    xs, its_s, rs = pkg.mrs(J, b, Q, alpha, tol=tol, maxit=3000, precision=precision, fmt="sell")
    true = np.linalg.norm(b - xd - apply(xd)) / np.linalg.norm(b)
    if precision == "fp64":
        assert abs(its_d - its_o) <= 2 and abs(its_s - its_o) <= 2
        np.testing.assert_allclose(xd, xo, rtol=0, atol=1e-9 * np.abs(xo).max())
        np.testing.assert_allclose(xs, xo, rtol=0, atol=1e-9 * np.abs(xo).max())
        assert true <= 1e-11
    else:
        assert rd < 1e-5 and true <= 5e-5
        np.testing.assert_allclose(xd, xo, rtol=0, atol=1e-4 * np.abs(xo).max())
        np.testing.assert_allclose(xs, xo, rtol=0, atol=1e-4 * np.abs(xo).max())


def test_mrs_diag_storage_rejects_non_skew(pkg):
    n = 500
    J = banded_skew(n, (1, 5), seed=1).tolil()
    J[3, 4] += 1e-3   # no longer exactly skew
    J = J.tocsr()
    with pytest.raises(pkg.AsssError):
        pkg.mrs(J, np.ones(n), fmt="diag")
    x, its, ratio = pkg.mrs(J, np.ones(n), fmt="auto", tol=1e-8)   # falls back to SELL-C
    assert ratio < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solver_storage_formats_agree(pkg, precision):
    A, b, _ = dissipative_hamiltonian_3d(side=16, seed=9)
    tol = 1e-6 if precision == "mixed" else 1e-10
    res = {}
    for fmt in ("sell", "diag"):
        s = pkg.Solver(A, precision=precision, outer="fgmres", inner_tol=tol, inner_format=fmt)
        x, st = s.solve(b)
        assert st["status"] == 0 and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
        res[fmt] = (x, st)
        s.close()
    assert abs(res["sell"][1]["outer_its"] - res["diag"][1]["outer_its"]) <= 1
    assert np.linalg.norm(res["sell"][0] - res["diag"][0]) <= 1e-7 * np.linalg.norm(res["sell"][0])


# ----------------------------------------------------------------------------
# failure detection: a device wait that runs out is reported, the context survives
# ----------------------------------------------------------------------------
def test_device_wait_timeout_is_reported_and_context_survives(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=12, seed=3)
    # a budget of ~1 ns: the first block to reach a grid barrier gives up at once
    with pytest.raises(pkg.AsssError) as e:
        pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, wait_timeout_ms=1e-6)
    assert e.value.status == 8
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6)
    x, st = s.solve(b)
    assert st["status"] == 0 and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)


# ----------------------------------------------------------------------------
# the benchmark's configuration at full size (n = 10^6): properties that hold at
# any size, checked on the CPU from the oracle's definitions
# ----------------------------------------------------------------------------
@pytest.mark.slow
def test_full_size_dh100_properties(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=100, seed=1)
    n = A.shape[0]
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-8, k=20)
    x, st = s.solve(b)
    assert st["status"] == 0
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    ex = s.export(A.nnz)
    Abar, dr, dc, _ = O.equilibrate(A)
    np.testing.assert_allclose(ex["dr"], dr, rtol=1e-15)
    np.testing.assert_allclose(ex["dc"], dc, rtol=1e-15)
    S = sp.csr_matrix((ex["s_val"], Abar.indices, Abar.indptr), shape=A.shape)
    # d_i = (Abar S)_ii on sampled rows and W = |d|^-1/2 (§3, 1x1 pivots)
    rng = np.random.default_rng(0)
    rows = rng.choice(n, 2000, replace=False)
    ST = S.T.tocsr()
    d_ref = np.array([Abar[i].multiply(ST[i]).sum() for i in rows])
    np.testing.assert_allclose(ex["d"][rows], d_ref, rtol=1e-12)
    np.testing.assert_allclose(ex["w"], 1.0 / np.sqrt(np.abs(ex["d"])), rtol=1e-14)
    # the LLS minimiser: normal-equation gradient vanishes relative to B^T v (§2, App. A)
    B, v, _ = O.lls_system(Abar, S, 1.0)
    g = B.T @ (v - B @ ex["s_val"])
    assert np.linalg.norm(g) <= 1e-8 * np.linalg.norm(B.T @ v), s.setup_stats["lls_relgrad"]
    # skew-Lanczos relations on the J~ built from the definition (§3.2)
    Jt = O.inner_skew_operator(Abar, S, ex["w"])
    Q = ex["Q"]
    np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-10)
    np.testing.assert_allclose(Q.T @ (Jt @ Q), O.lanczos_tridiagonal(ex["alpha"]), atol=1e-8)
    # P^-1 u and P^-T u element by element at full size, through the kernels the
    # benchmark runs (FP32 mrs with evict-first Q loads, FP32 SMW correction with
    # evict-first Y): r = 0 here, so P = I + J~ exactly (Eq. preconditioner with
    # M~_r = 0, the Q_k S_k Q_k^T terms cancel), and the oracle's App. B mrs on the
    # undeflated I +- J~ to 1e-12 gives P^-1 u itself
    assert s.setup_stats["r"] == 0 and np.all(ex["d"] > 0)
    u = np.random.default_rng(17).standard_normal(n)
    for tr, sgn in ((False, 1.0), (True, -1.0)):
        zg, its = s.apply_preconditioner(u, transpose=tr)
        zo, its_o, ratio_o, _ = O.mrs(1.0, lambda V: sgn * (Jt @ V), u, 5000, 1e-12)
        assert ratio_o < 1e-12 and its > 0
        np.testing.assert_allclose(zg, zo, rtol=0, atol=1e-4 * np.abs(zo).max())


def test_solver_bf16_deflation_basis(pkg):
    """Mixed precision with Q_k rounded to BF16 everywhere: P is unchanged, so the
    solve reaches the same residual and solution."""
    A, b, _ = dissipative_hamiltonian_3d(side=16, seed=9)
    res = {}
    for qb in (False, True):
        s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, q_bf16=qb)
        x, st = s.solve(b)
        assert st["status"] == 0 and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
        res[qb] = (x, st)
        s.close()
    assert abs(res[True][1]["outer_its"] - res[False][1]["outer_its"]) <= 1
    assert np.linalg.norm(res[True][0] - res[False][0]) <= 1e-7 * np.linalg.norm(res[False][0])


# ----------------------------------------------------------------------------
# differentiation at the 64^3 size: adjoint vs finite differences on 64 seeded entries
# ----------------------------------------------------------------------------
@pytest.mark.slow
def test_adjoint_finite_differences_dh64(pkg):
    """L = ||x - x*||^2 on the 64^3 dissipative-Hamiltonian step (n = 262 144),
    FP32 inner / FP64 outer; central differences with step h = 1e-6 on 32 entries
    of b and 32 nonzeros of A (seeded), evaluated without cancellation:

      [L(+) - L(-)] / 2h = (x+ - x-) . (x+ + x- - 2x*) / 2h      (exact identity)

    b: L is quadratic in b, x+ - x- = A^-1 (2h e_i) and x+ + x- = 2x.
    A (entry e = (i, j), E = e_i e_j^T): (A +- hE) x+- = b gives
       A (x+ - x-) = -h E (x+ + x-), i.e. x+ - x- = -h (x+_j + x-_j) A^-1 e_i,
    so the difference of two nearly equal solves is never formed; x+ and x- come from
    their own set-ups and solves, A^-1 e_i from one more forward solve."""
    A, b, _ = dissipative_hamiltonian_3d(side=64, seed=4)
    n = A.shape[0]
    rng = np.random.default_rng(44)
    xs = rng.standard_normal(n)
    opts = dict(precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-13)
    s = pkg.Solver(A, **opts)
    x, st = s.solve(b)
    assert st["status"] == 0
    g = 2.0 * (x - xs)
    lam, dA, st2 = s.solve_adjoint(g, x=x)
    assert st2["status"] == 0
    h = 1e-6
    scale_b = np.abs(lam).max()
    errs = []
    for i in rng.choice(n, 32, replace=False):
        e = np.zeros(n)
        e[i] = 2.0 * h
        dx, _ = s.solve(e)
        fd = np.dot(dx, 2.0 * x - 2.0 * xs) / (2.0 * h)
        errs.append(abs(fd - lam[i]) / max(abs(fd), 1e-3 * scale_b))
    assert max(errs) <= 1e-6, max(errs)

    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    scale_a = np.abs(dA).max()
    errs = []
    for e_idx in rng.choice(A.nnz, 32, replace=False):
        i, j = rows[e_idx], A.indices[e_idx]
        xpm = []
        for sgn in (1.0, -1.0):
            Ap = A.copy()
            Ap.data[e_idx] += sgn * h
            sp_ = pkg.Solver(Ap, **opts)
            xp_, stp = sp_.solve(b)
            assert stp["status"] == 0
            xpm.append(xp_)
            sp_.close()
        xp, xm = xpm
        ei = np.zeros(n)
        ei[i] = 1.0
        ai, _ = s.solve(ei)
        dxpm = -h * (xp[j] + xm[j]) * ai
        fd = np.dot(dxpm, xp + xm - 2.0 * xs) / (2.0 * h)
        errs.append(abs(fd - dA[e_idx]) / max(abs(fd), 1e-3 * scale_a))
    assert max(errs) <= 1e-6, max(errs)
    s.close()


# ----------------------------------------------------------------------------
# the outer operator and the preconditioner, checked against the oracle's own
# building blocks evaluated on the set-up the GPU exported (so the comparison
# isolates the products: diagonal storage for stencils, CSR otherwise)
# ----------------------------------------------------------------------------
def _general_sparse(n, seed):
    rng = np.random.default_rng(seed)
    K = sp.random(n, n, density=6.0 / n, random_state=rng, data_rvs=rng.standard_normal)
    A = (K + sp.diags(4.0 + rng.random(n))).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


@pytest.mark.parametrize("case", ["stencil", "general"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_operator_and_preconditioner_match_oracle_blocks(pkg, case, precision, loads):
    if case == "stencil":
        A, _, _ = dissipative_hamiltonian_3d(side=13, seed=5)
    else:
        A = _general_sparse(3001, seed=7)
    tol_in = 1e-10 if precision == "fp64" else 1e-6
    s = pkg.Solver(A, precision=precision, inner_tol=tol_in)
    ex = s.export(A.nnz)
    Abar, dr, dc, _ = O.equilibrate(A)
    np.testing.assert_allclose(ex["dr"], dr, rtol=1e-15)
    np.testing.assert_allclose(ex["dc"], dc, rtol=1e-15)
    S = sp.csr_matrix((ex["s_val"], Abar.indices.copy(), Abar.indptr.copy()), shape=A.shape)
    Pat = pattern_of(A)
    assert np.array_equal(Pat.indptr, Abar.indptr) and np.array_equal(Pat.indices, Abar.indices)
    w = ex["w"]
    W = sp.diags(w)
    Acal = (W @ Abar @ S @ W).tocsr()
    rng = np.random.default_rng(11)
    v = rng.standard_normal(A.shape[0])
    for tr in (False, True):
        ref = (Acal.T if tr else Acal) @ v
        got = s.apply_operator(v, transpose=tr)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # P = M~_r + I + J~ = diag(sign d) + J~ (reading R5), J~ from the oracle
    Jt = O.inner_skew_operator(Abar, S, w)
    P = (sp.diags(np.sign(ex["d"])) + Jt).tocsr()
    u = rng.standard_normal(A.shape[0])
    bound = 1e-8 if precision == "fp64" else 1e-4
    for tr in (False, True):
        z, its = s.apply_preconditioner(u, transpose=tr)
        r = ((P.T if tr else P) @ z) - u
        assert its > 0
        assert np.linalg.norm(r) <= bound * np.linalg.norm(u), (tr, np.linalg.norm(r) / np.linalg.norm(u))
    s.close()


# ----------------------------------------------------------------------------
# general matrices with power-law rows: some rows of Abar S have more candidate
# columns than the shared-memory sort holds and take the bitmap path
# ----------------------------------------------------------------------------
def test_powerlaw_rows_pattern_and_fit(pkg):
    from workloads import pattern_symmetrized, random_powerlaw
    A, b = random_powerlaw(n=3000, seed=2, band=300)
    A = sp.csr_matrix(A)
    Sp = pattern_symmetrized(A)
    Abar, _, _, _ = O.equilibrate(A)
    # candidates of the heaviest row exceed the shared-memory sort (8192 per row)
    Ap = pattern_of(Abar)
    cand = Ap @ np.diff(Sp.indptr) + Sp.T.tocsr() @ np.diff(Ap.T.tocsr().indptr)
    assert cand.max() > 8192
    s = pkg.Solver(A, s_pattern=Sp, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_maxit=40)
    C = pattern_of(Abar) @ Sp
    P = (pattern_of(C) + pattern_of(C).T + sp.identity(A.shape[0])).tocsr()
    P.sum_duplicates()
    assert s.setup_stats["nnz_pattern"] == P.nnz
    ex = s.export(Sp.nnz)
    B, v, _ = O.lls_system(Abar, Sp, 1.0)
    sv = ex["s_val"]
    g = B.T @ (v - B @ sv)
    assert np.linalg.norm(g) <= 1e-8 * np.linalg.norm(B.T @ v), s.setup_stats["lls_relgrad"]
    x, st = s.solve(b)
    assert st["status"] in (0, 5, 6)  # converged, not converged or stagnated: no failure
    assert np.all(np.isfinite(x))
    s.close()


# ----------------------------------------------------------------------------
# resuming a set-up from saved S values (options.s_values)
# ----------------------------------------------------------------------------
def test_setup_resumes_from_saved_s_values(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=20, seed=6)
    s1 = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6)
    assert s1.setup_stats["lls_its"] > 8
    saved = s1.export(A.nnz)["s_val"].copy()
    x1, st1 = s1.solve(b)
    s1.close()
    s2 = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, s_values=saved)
    assert s2.setup_stats["lls_its"] == 0
    assert s2.setup_stats["lls_relgrad"] <= 1e-13
    np.testing.assert_array_equal(s2.export(A.nnz)["s_val"], saved)
    x2, st2 = s2.solve(b)
    assert st2["status"] == 0 and st2["outer_its"] == st1["outer_its"]
    assert np.linalg.norm(x2 - x1) <= 1e-12 * np.linalg.norm(x1)
    # a perturbed start converges back to the fit
    s3 = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, s_values=saved * (1 + 1e-3))
    assert 0 < s3.setup_stats["lls_its"]
    assert np.linalg.norm(s3.export(A.nnz)["s_val"] - saved) <= 1e-9 * np.linalg.norm(saved)
    s3.close()
    s2.close()


# ----------------------------------------------------------------------------
# an indefinite matrix: diag(Abar S) has negative entries, so M~_r has rank r > 0 and
# the SMW correction carries U_r next to the Lanczos vectors (§3, Fig. 1; Eq. smw)
# ----------------------------------------------------------------------------
def _indefinite(n, seed, sym, skew):
    rng = np.random.default_rng(seed)
    K = sp.random(n, n, density=5.0 / n, random_state=rng, data_rvs=rng.standard_normal)
    D = sp.diags(rng.choice([-1.0, 1.0], size=n) * (1.0 + rng.random(n)))
    A = (D + 0.5 * (K + K.T) * sym + 0.5 * (K - K.T) * skew).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_negative_pivots_low_rank_part(pkg, precision):
    A = _indefinite(600, 4, 0.6, 1.0)
    Sd = pattern_diagonal(A.shape[0])
    o = O.AsssOracle(A, S_pattern=Sd, gamma=0.1, inner_tol=1e-10)
    assert o.r > 0
    tol_in = 1e-10 if precision == "fp64" else 1e-6
    s = pkg.Solver(A, s_pattern=Sd, gamma=0.1, precision=precision, inner_tol=tol_in)
    assert s.setup_stats["r"] == o.r
    ex = s.export(Sd.nnz)
    np.testing.assert_array_equal(np.sort(ex["neg"]), np.sort(np.flatnonzero(o.d < 0)))
    np.testing.assert_allclose(ex["d"], o.d, rtol=1e-8, atol=1e-12 * np.abs(o.d).max())
    # P z = u with P = diag(sign d) + J~ built by the oracle from the exported S
    Abar, _, _, _ = O.equilibrate(A)
    S = sp.csr_matrix((ex["s_val"], Sd.indices.copy(), Sd.indptr.copy()), shape=A.shape)
    Jt = O.inner_skew_operator(Abar, S, ex["w"])
    P = (sp.diags(np.sign(ex["d"])) + Jt).tocsr()
    u = np.random.default_rng(12).standard_normal(A.shape[0])
    bound = 1e-8 if precision == "fp64" else 1e-4
    for tr in (False, True):
        z, _ = s.apply_preconditioner(u, transpose=tr)
        r = ((P.T if tr else P) @ z) - u
        assert np.linalg.norm(r) <= bound * np.linalg.norm(u), (tr, np.linalg.norm(r) / np.linalg.norm(u))
    s.close()


# ----------------------------------------------------------------------------
# App. B's simultaneous iterations: several right-hand sides in one launch (the
# columns share the passes over J~ and Q_k), per-column freezing (reading R9)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["sell", "diag"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_mrs_multi_matches_oracle_freeze(pkg, storage, precision, sign, loads):
    n = 20001
    J = random_skew(n, 12, seed=41) if storage == "sell" else banded_skew(n, (1, 3, 64, 1000), seed=42)
    rng = np.random.default_rng(43)
    Q, alpha = O.skew_lanczos(J, rng.standard_normal(n), 20)
    Sk = O.lanczos_tridiagonal(alpha)
    apply = lambda V: sign * (J @ V - Q @ (Sk @ (Q.T @ V)))
    B = rng.standard_normal((n, 11))       # two launches: 8 + 3 columns
    B[:, 3] = 0.0                          # a zero column gives x = 0 and its = 0
    B[:, 5] *= 1e3                         # scale does not change the per-column stop
    B[:, 9] = 0.0
    B[7, 9] = 1.0                          # a unit vector, as in the SMW set-up
    tol = 1e-12 if precision == "fp64" else 1e-5
    Xo, its_o, ratio_o, _ = O.mrs(1.0, apply, B, 3000, 1e-12 if precision == "fp64" else 1e-7, freeze=True)
    Xg, its_g, ratio_g = pkg.mrs_multi(J, B, Q, alpha, sign=sign, tol=tol, maxit=3000, precision=precision,
                                       fmt=storage)
    assert its_g[3] == 0 and np.all(Xg[:, 3] == 0)
    for c in range(B.shape[1]):
        if c == 3:
            continue
        xo = Xo[:, c]
        if precision == "fp64":
            assert abs(int(its_g[c]) - int(its_o[c])) <= 2, (c, its_g[c], its_o[c])
            assert ratio_g[c] < 1e-12
            np.testing.assert_allclose(Xg[:, c], xo, rtol=0, atol=1e-9 * np.abs(xo).max())
        else:
            assert ratio_g[c] < 1e-5
            np.testing.assert_allclose(Xg[:, c], xo, rtol=0, atol=1e-4 * np.abs(xo).max())
    # the same as separate single-column solves
    for c in (0, 5, 10):
        x1, its1, _ = pkg.mrs(J, B[:, c], Q, alpha, sign=sign, tol=tol, maxit=3000, precision=precision, fmt=storage)
        assert abs(int(its_g[c]) - its1) <= 2
        atol = (1e-9 if precision == "fp64" else 1e-4) * np.abs(x1).max()
        np.testing.assert_allclose(Xg[:, c], x1, rtol=0, atol=atol)


def test_mrs_multi_stops_at_maxit_with_the_oracle_iterates(pkg):
    """Every column at its iteration limit: its = maxit, X equals the oracle's iterates."""
    n = 3001
    J = random_skew(n, 10, seed=44)
    B = np.random.default_rng(45).standard_normal((n, 5))
    Xo, its_o, ratio_o, _ = O.mrs(1.0, lambda V: J @ V, B, 4, 1e-14, freeze=True)
    Xg, its_g, ratio_g = pkg.mrs_multi(J, B, tol=1e-14, maxit=4)
    assert np.all(its_g == 4) and np.all(its_o == 4)
    np.testing.assert_allclose(ratio_g, ratio_o, rtol=1e-12)
    np.testing.assert_allclose(Xg, Xo, rtol=0, atol=1e-12 * np.abs(Xo).max())


# ----------------------------------------------------------------------------
# the general power-law recipe (heavy-tailed rows: SELL-C-sigma storage of J~)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_powerlaw_inner_operator_mrs_steps_match_oracle(pkg, precision):
    """J~ of the power-law recipe built by the oracle from the GPU's exported S and w
    (§3, Eq. preconditioner): five App. B steps with k = 20 deflation vectors agree
    element by element with the oracle's; the heavy-tailed rows make the SELL-C
    storage sort rows within windows (SELL-C-sigma)."""
    from workloads import pattern_symmetrized, random_powerlaw
    A, b = random_powerlaw(n=20000, seed=2, band=1000)
    A = sp.csr_matrix(A)
    Sp = pattern_symmetrized(A)
    s = pkg.Solver(A, s_pattern=Sp, precision="mixed", outer="fgmres", inner_tol=1e-6, lls_maxit=400)
    ex = s.export(Sp.nnz)
    s.close()
    Abar, _, _, _ = O.equilibrate(A)
    S = sp.csr_matrix((ex["s_val"], Sp.indices.copy(), Sp.indptr.copy()), shape=A.shape)
    Jt = O.inner_skew_operator(Abar, S, ex["w"])
    lens = np.diff(Jt.indptr)
    assert lens.max() > 8 * lens.mean()          # heavy tail: unsorted slices would pad heavily
    rng = np.random.default_rng(51)
    Q, alpha = O.skew_lanczos(Jt, rng.standard_normal(Jt.shape[0]), 20)
    Sk = O.lanczos_tridiagonal(alpha)
    u = rng.standard_normal(Jt.shape[0])
    apply = lambda V: Jt @ V - Q @ (Sk @ (Q.T @ V))
    xo, its_o, ratio_o, _ = O.mrs(1.0, apply, u, 5, 1e-14)
    xg, its_g, ratio_g = pkg.mrs(Jt, u, Q, alpha, tol=1e-14, maxit=5, precision=precision, fmt="sell")
    assert its_g == 5 and its_o == 5
    rtol = 1e-11 if precision == "fp64" else 2e-5
    assert abs(ratio_g - ratio_o) <= rtol * ratio_o
    np.testing.assert_allclose(xg, xo, rtol=0, atol=rtol * np.abs(xo).max())
    # the multi-column kernel on the same storage
    B = np.column_stack([u, rng.standard_normal(u.size)])
    Xo, _, _, _ = O.mrs(1.0, apply, B, 5, 1e-14, freeze=True)
    Xg, its_m, _ = pkg.mrs_multi(Jt, B, Q, alpha, tol=1e-14, maxit=5, precision=precision, fmt="sell")
    assert np.all(its_m == 5)
    np.testing.assert_allclose(Xg, Xo, rtol=0, atol=rtol * np.abs(Xo).max())


def test_powerlaw_sell_layouts_agree(pkg):
    """The SELL-C layout of J~ (sorting window sigma, work-unit width) changes only the
    summation order of J~ v: FP64 solves of the power-law recipe with the extreme
    layouts (narrow units that split long slices into many parts finished by the last
    warp, wide units that keep them whole) reach the same x, each meeting the outer
    tolerance on the original system."""
    from workloads import random_powerlaw
    A, b = random_powerlaw(n=20000, seed=2, band=1000, dom_frac=1.0)   # every row dominant: converges
    A = sp.csr_matrix(A)
    xs = []
    for sigma, split in ((1024, 64), (16384, 4096), (4096, 0)):
        s = pkg.Solver(A, precision="fp64", outer="fgmres", inner_tol=1e-10, lls_maxit=400,
                       sell_sigma=sigma, sell_split=split)
        st0 = s.setup_stats
        assert st0["sell_sigma"] == sigma            # heavy tail: the rows are sorted
        assert st0["sell_split"] == (split or 1024)
        x, st = s.solve(b)
        s.close()
        assert st["status"] == 0
        assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
        xs.append(x)
    for x in xs[1:]:
        np.testing.assert_allclose(x, xs[0], rtol=0, atol=1e-7 * np.abs(xs[0]).max())
    with pytest.raises(pkg.AsssError):
        pkg.Solver(A, precision="fp64", sell_sigma=3000)
    with pytest.raises(pkg.AsssError):
        pkg.Solver(A, precision="fp64", sell_split=8)


def test_powerlaw_sell_tuner_picks_a_candidate(pkg):
    """Mixed precision at 10^5 rows or more tunes the SELL-C layout at set-up by timing
    mrs steps; the chosen pair is one of the candidates and the solve converges."""
    from workloads import random_powerlaw
    A, b = random_powerlaw(n=120000, seed=4, band=4000, dom_frac=1.0)
    A = sp.csr_matrix(A)
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, lls_maxit=400)
    st0 = s.setup_stats
    assert (st0["sell_sigma"], st0["sell_split"]) in {(4096, 1024), (1024, 1024), (16384, 1024),
                                                      (4096, 256), (4096, 4096)}
    x, st = s.solve(b)
    s.close()
    assert st["status"] == 0
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)


# ----------------------------------------------------------------------------
# several right-hand sides in one call: lockstep FGMRES blocks whose preconditioner
# applications are one multi-column mrs launch (App. B) per Arnoldi step
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_block_solve_matches_single_solves_and_direct(pkg, precision):
    A, b, _ = dissipative_hamiltonian_3d(side=16, seed=9)
    n = A.shape[0]
    rng = np.random.default_rng(61)
    B = rng.standard_normal((n, 11))          # one block of 8 and one of 3
    B[:, 4] = 0.0
    B[:, 7] = 3.0 * B[:, 1]
    s = pkg.Solver(A, precision=precision, outer="fgmres", inner_tol=1e-6 if precision == "mixed" else 1e-10,
                   rhs_block=True)
    X, st = s.solve(B)
    assert st["status"] == 0 and st["inner_solves"] > 0
    assert np.all(X[:, 4] == 0)
    Xd = sp.linalg.splu(A.tocsc()).solve(B)
    for c in range(B.shape[1]):
        if c == 4:
            continue
        assert np.linalg.norm(B[:, c] - A @ X[:, c]) <= 1e-8 * np.linalg.norm(B[:, c])
        np.testing.assert_allclose(X[:, c], Xd[:, c], rtol=0, atol=1e-7 * np.abs(Xd[:, c]).max())
    np.testing.assert_allclose(X[:, 7], 3.0 * X[:, 1], rtol=0, atol=1e-7 * np.abs(X[:, 7]).max())
    for c in (0, 9):                           # the same as a call with that column alone
        x1, st1 = s.solve(B[:, c])
        assert abs(st1["outer_its"] - st["outer_its"]) <= 3
        np.testing.assert_allclose(X[:, c], x1, rtol=0, atol=1e-7 * np.abs(x1).max())
    s.close()


def test_block_solve_fp64_matches_oracle_cd64(pkg):
    A, b, _ = convection_diffusion_2d(m=64)
    rng = np.random.default_rng(62)
    B = np.column_stack([b, rng.standard_normal(A.shape[0])])
    o = O.AsssOracle(A, inner_tol=1e-10)
    s = pkg.Solver(A, inner_tol=1e-10, outer="fgmres", rhs_block=True)
    X, st = s.solve(B)
    assert st["status"] == 0
    for c in range(2):
        xo, sto = o.solve(B[:, c], tol=1e-8, outer="fgmres")
        assert np.linalg.norm(B[:, c] - A @ X[:, c]) <= 1e-8 * np.linalg.norm(B[:, c])
        assert np.linalg.norm(X[:, c] - xo) <= 1e-5 * np.linalg.norm(xo)
    s.close()
