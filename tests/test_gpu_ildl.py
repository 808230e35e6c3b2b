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
