"""The GPU incomplete L D L^T (factor='ildl0': §3 after Eq. absfac, §4.1's ~ildl(0))
against the oracle: the multicolour order (bit for bit), the factor L and the pivots
D, the factored operators F A^ G and L~^-1 J^ L~^-T inside the mrs kernel (P^-1 u
element by element), whole solves and the adjoint, and the options that do not
combine with it."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import convection_diffusion_2d, dissipative_hamiltonian_3d, random_powerlaw

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


def _case(kind):
    if kind == "cd64":
        A, b, _ = convection_diffusion_2d(m=64)
    elif kind == "dh12":
        A, b, _ = dissipative_hamiltonian_3d(side=12, seed=1)
    else:
        A, b = random_powerlaw(n=3000, lmean=6.0, lmax=64, seed=5, band=300, dom_frac=1.0)
        A = sp.csr_matrix(A)
    return A, b


@pytest.mark.parametrize("kind", ["cd64", "dh12", "powerlaw3000"])
def test_factor_matches_oracle(pkg, kind):
    """Colours equal the oracle's Jones-Plassmann colouring of the same pattern and
    seed; L (same pattern) and D agree to rounding; (I + L) D (I + L)^T equals M^ on
    its pattern (the defining property), checked on the GPU's own factor."""
    A, b = _case(kind)
    o = O.AsssOracle(A, inner_tol=1e-10, factor="ildl0")
    s = pkg.Solver(A, inner_tol=1e-10, factor="ildl0")
    colour, L = s.export_factor()
    ex = s.export(o.S.nnz)
    assert s.setup_stats["factor_colours"] == o.colour.max() + 1
    np.testing.assert_array_equal(colour, o.colour)
    assert L.nnz == o.L.nnz
    np.testing.assert_array_equal(L.indptr, o.L.indptr)
    np.testing.assert_array_equal(L.indices, o.L.indices)
    # the two sides fit S separately (LLS to 1e-13 in the normal-equation gradient)
    np.testing.assert_allclose(L.data, o.L.data, rtol=0, atol=1e-7 * max(1.0, np.abs(o.L.data).max()))
    np.testing.assert_allclose(ex["d"], o.d, rtol=1e-7)
    assert np.all(ex["w"] == 1.0)
    S = sp.csr_matrix((ex["s_val"], o.S.indices, o.S.indptr), shape=A.shape)
    C = (o.Abar @ S).tocsr()
    P = O.structural_pattern(o.Abar, S)
    MP = O.values_on_pattern(0.5 * (C + C.T), P)
    L1 = (L + sp.identity(A.shape[0])).tocsr()
    R = O.values_on_pattern((L1 @ sp.diags(ex["d"]) @ L1.T).tocsr(), P)
    np.testing.assert_allclose(R.data, MP.data, rtol=0, atol=1e-10 * np.abs(MP.data).max())
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("force_stream", [False, True])
def test_factored_operator_and_preconditioner_match_oracle(pkg, precision, force_stream, monkeypatch):
    """A_cal v = F A^ G v (both transposes) and P^-1 u through the factored mrs kernel
    (one grid barrier per colour of each triangular solve), element by element."""
    if force_stream:
        monkeypatch.setenv("ASSS_FORCE_EVICT_FIRST", "1")
    A, b = _case("dh12")
    tol = 1e-12 if precision == "fp64" else 1e-7
    o = O.AsssOracle(A, inner_tol=1e-13, inner_maxit=2000, factor="ildl0")
    s = pkg.Solver(A, precision=precision, inner_tol=tol, inner_maxit=2000, outer="fgmres", factor="ildl0")
    rng = np.random.default_rng(71)
    v = rng.standard_normal(A.shape[0])
    for tr in (False, True):
        yo = o.apply_op(v, transpose=tr)
        yg = s.apply_operator(v, transpose=tr)
        np.testing.assert_allclose(yg, yo, rtol=0, atol=1e-8 * np.abs(yo).max())
        zo = o.apply_prec_inv(v, transpose=tr)
        zg, its = s.apply_preconditioner(v, transpose=tr)
        assert its > 0
        atol = (1e-7 if precision == "fp64" else 1e-4) * np.abs(zo).max()
        np.testing.assert_allclose(zg, zo, rtol=0, atol=atol)
    s.close()


@pytest.mark.parametrize("outer", ["tfqmr", "fgmres"])
def test_factored_solve_cd64_fp64_matches_oracle(pkg, outer):
    A, b = _case("cd64")
    o = O.AsssOracle(A, inner_tol=1e-10, factor="ildl0")
    xo, sto = o.solve(b, tol=1e-8, outer=outer)
    s = pkg.Solver(A, inner_tol=1e-10, outer=outer, factor="ildl0")
    xg, stg = s.solve(b)
    assert stg["status"] == 0
    assert np.linalg.norm(b - A @ xg) <= 1e-8 * np.linalg.norm(b)
    assert abs(stg["outer_its"] - sto["outer_its"]) <= 2, (stg["outer_its"], sto["outer_its"])
    assert np.linalg.norm(xg - xo) <= 1e-5 * np.linalg.norm(xo)
    lam, dA, sta = s.solve_adjoint(b, xg)
    assert sta["status"] == 0
    assert np.linalg.norm(b - A.T @ lam) <= 1e-8 * np.linalg.norm(b)
    s.close()


def test_factored_mixed_solve_dh16_and_fewer_outer_steps(pkg):
    """Mixed precision with the incomplete factor meets the tolerance; on this family
    it needs no more outer steps than the diagonal factor (the oracle's counts agree)."""
    A, b, _ = dissipative_hamiltonian_3d(side=16, seed=3)
    sf = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, factor="ildl0")
    xf, stf = sf.solve(b)
    sd = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6)
    xd, std = sd.solve(b)
    assert stf["status"] == 0 and std["status"] == 0
    assert np.linalg.norm(b - A @ xf) <= 1e-8 * np.linalg.norm(b)
    assert stf["outer_its"] <= std["outer_its"]
    np.testing.assert_allclose(xf, xd, rtol=0, atol=1e-6 * np.abs(xd).max())
    sf.close()
    sd.close()


def test_factor_options_that_do_not_combine(pkg):
    A, b = _case("cd64")
    with pytest.raises(pkg.AsssError):
        pkg.Solver(A, precision="mixed", factor="ildl0", q_bf16=True)
    with pytest.raises(pkg.AsssError):
        pkg.Solver(A, factor=7)
    s = pkg.Solver(A, inner_tol=1e-8)
    with pytest.raises(pkg.AsssError):
        s.export_factor()
    s.close()
    with pytest.raises(pkg.AsssError):
        pkg.BatchSolver([A], factor="ildl0")


# ----------------------------------------------------------------------------
# 2x2 pivot blocks (factor='ildl0_bk', reading R20)
# ----------------------------------------------------------------------------
from workloads import saddle_pairs  # noqa: E402


def _given_s(n):
    """S = I taken as given (no least-squares fit) and no scaling: M^ is the symmetric
    part of A itself, so its zero-diagonal pairs reach the factor."""
    I = sp.identity(n, format="csr")
    return dict(s_pattern=I, s_values=np.ones(n), lls_maxit=0, dr=np.ones(n), dc=np.ones(n),
                row_perm=np.arange(n, dtype=np.int32)), I


@pytest.mark.parametrize("n,seed", [(300, 1), (2000, 4)])
def test_block_factor_matches_oracle(pkg, n, seed):
    """The pairs (bit for bit), the colours of the quotient graph (bit for bit), the block
    factor L, the pivot blocks D and M~_r = -2 U_r U_r^T agree with the oracle; the GPU's
    own (I + L) D (I + L)^T equals M^ on the block closure of its pattern; the 1x1 factor
    meets a zero pivot on the same matrix."""
    A = saddle_pairs(n, seed=seed, singles=n // 10)
    opts, I = _given_s(n)
    o = O.AsssOracle(A, S=I, dr=np.ones(n), dc=np.ones(n), k=4, factor="ildl0_bk")
    s = pkg.Solver(A, k=4, factor="ildl0_bk", **opts)
    pv = s.export_pivots()
    assert pv is not None and pv["npairs"] == int((o.partner >= 0).sum()) // 2
    assert s.setup_stats["factor_pairs"] == pv["npairs"]
    np.testing.assert_array_equal(pv["partner"], o.partner)
    colour, L = s.export_factor()
    np.testing.assert_array_equal(colour, o.colour)
    Lo = o.L.tocsr()
    Lo.sort_indices()
    np.testing.assert_array_equal(L.indptr, Lo.indptr)
    np.testing.assert_array_equal(L.indices, Lo.indices)
    np.testing.assert_allclose(L.data, Lo.data, rtol=0, atol=1e-10 * max(1.0, np.abs(Lo.data).max()))
    ex = s.export(A.nnz)
    Do = o.D.toarray()
    np.testing.assert_allclose(ex["d"], np.diag(Do), rtol=0, atol=1e-10 * np.abs(Do).max())
    p = o.partner
    np.testing.assert_allclose(pv["d_off"][p >= 0], Do[np.flatnonzero(p >= 0), p[p >= 0]], rtol=0,
                               atol=1e-10 * np.abs(Do).max())
    assert s.setup_stats["r"] == o.r
    np.testing.assert_allclose(pv["Ur"] @ pv["Ur"].T, o.Ur_cols @ o.Ur_cols.T, rtol=0, atol=1e-10)
    D = sp.diags(ex["d"]).tolil()
    for i in np.flatnonzero(pv["partner"] >= 0):
        D[i, pv["partner"][i]] = pv["d_off"][i]
    L1 = (L + sp.identity(n)).tocsr()
    Pb = O.ildl.block_pattern(O.structural_pattern(A, I), pv["partner"])
    M = (0.5 * (A + A.T)).tocsr()
    R = O.values_on_pattern((L1 @ D.tocsr() @ L1.T).tocsr(), Pb)
    np.testing.assert_allclose(R.data, O.values_on_pattern(M, Pb).data, rtol=0, atol=1e-10 * abs(M).max())
    s.close()
    with pytest.raises(pkg.AsssError):
        pkg.Solver(A, k=4, factor="ildl0", **opts)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_factored_operator_and_preconditioner_match_oracle(pkg, precision):
    """F A^ G (both transposes) with |D|^-1/2 block by block, and P^-1 u through the
    factored mrs kernel with the pairs' weights and the two-entry U_r columns of the
    SMW correction, element by element against the oracle."""
    n = 400
    A = saddle_pairs(n, seed=2, singles=40)
    opts, I = _given_s(n)
    tol = 1e-12 if precision == "fp64" else 1e-7
    o = O.AsssOracle(A, S=I, dr=np.ones(n), dc=np.ones(n), k=6, inner_tol=1e-13, inner_maxit=3000,
                     factor="ildl0_bk")
    s = pkg.Solver(A, k=6, precision=precision, inner_tol=tol, inner_maxit=3000, outer="fgmres",
                   factor="ildl0_bk", **opts)
    assert o.r > 0
    rng = np.random.default_rng(5)
    v = rng.standard_normal(n)
    for tr in (False, True):
        yo = o.apply_op(v, transpose=tr)
        yg = s.apply_operator(v, transpose=tr)
        np.testing.assert_allclose(yg, yo, rtol=0, atol=1e-9 * np.abs(yo).max())
        zo = o.apply_prec_inv(v, transpose=tr)
        zg, its = s.apply_preconditioner(v, transpose=tr)
        atol = (1e-7 if precision == "fp64" else 1e-4) * np.abs(zo).max()
        np.testing.assert_allclose(zg, zo, rtol=0, atol=atol)
    s.close()


@pytest.mark.parametrize("precision,outer", [("fp64", "fgmres"), ("fp64", "tfqmr"), ("mixed", "fgmres")])
def test_block_factored_solve_matches_dense(pkg, precision, outer):
    """Whole solves (and the adjoint) on a matrix that only 2x2 pivots factor: the true
    residual meets the tolerance, x agrees with a dense solve and the outer counts with
    the oracle's (FP64)."""
    n = 600
    A = saddle_pairs(n, seed=7, singles=60)
    b = np.random.default_rng(7).standard_normal(n)
    opts, I = _given_s(n)
    s = pkg.Solver(A, k=6, precision=precision, outer=outer, inner_tol=1e-10 if precision == "fp64" else 1e-6,
                   outer_tol=1e-10, factor="ildl0_bk", **opts)
    x, st = s.solve(b)
    assert st["status"] == 0 and np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    if precision == "fp64":
        o = O.AsssOracle(A, S=I, dr=np.ones(n), dc=np.ones(n), k=6, inner_tol=1e-10, factor="ildl0_bk")
        _, sto = o.solve(b, tol=1e-10, outer=outer)
        assert abs(st["outer_its"] - sto["outer_its"]) <= 2, (st["outer_its"], sto["outer_its"])
    lam, dA, sta = s.solve_adjoint(b, x)
    assert sta["status"] == 0 and np.linalg.norm(b - A.T @ lam) <= 1e-9 * np.linalg.norm(b)
    s.close()


def test_block_factor_without_pairs_is_the_1x1_factor(pkg):
    """On a matrix whose diagonal passes the Bunch-Kaufman test everywhere no pair is
    formed and the factor, colours and solve are those of factor='ildl0'."""
    A, b = _case("dh12")
    s1 = pkg.Solver(A, inner_tol=1e-10, factor="ildl0")
    s2 = pkg.Solver(A, inner_tol=1e-10, factor="ildl0_bk")
    assert s2.export_pivots() is None and s2.setup_stats["factor_pairs"] == 0
    c1, L1 = s1.export_factor()
    c2, L2 = s2.export_factor()
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(L1.indices, L2.indices)
    np.testing.assert_array_equal(L1.data, L2.data)
    x1, _ = s1.solve(b)
    x2, _ = s2.solve(b)
    np.testing.assert_array_equal(x1, x2)
    s1.close()
    s2.close()
