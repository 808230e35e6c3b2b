"""The GPU matching and scaling (§2, Eq. mc64; the role of MC64) against the oracle.

The auction's matching is within n * eps of the optimum the oracle's Hungarian
method finds, the scaled matrix has |diag| = 1 and entries <= 1 (to the auction's
epsilon), a matrix with a zero diagonal that the default scaling cannot set up
(zero pivots) solves once matched, and a structurally singular matrix is rejected."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from workloads import indefinite_zero_diagonal

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


@pytest.mark.parametrize("n,seed", [(37, 3), (2000, 0), (20001, 1)])
def test_matching_scaling_matches_oracle_optimum(pkg, n, seed):
    A = indefinite_zero_diagonal(n, seed)
    perm, dr, dc, rounds = pkg.matching_scaling(A)
    assert sorted(perm.tolist()) == list(range(n)) and rounds > 0
    C, _ = O.matching_costs(A)
    got = sum(C[perm[j], j] for j in range(n))
    _, _, _, opt = O.max_product_matching(A)
    eps = 1e-12 * max(1.0, C.data.max())          # the auction's final epsilon
    assert got <= opt + n * eps + 1e-12, (got, opt)
    Abar, _, _, _ = O.equilibrate(A, row_perm=perm, dr=dr, dc=dc)
    np.testing.assert_allclose(np.abs(Abar.diagonal()), 1.0, rtol=1e-12)
    assert np.abs(Abar.data).max() <= np.exp(eps) + 1e-14


def test_solver_with_matching_solves_zero_diagonal_matrix(pkg):
    A = indefinite_zero_diagonal(3000, 2)
    b = np.random.default_rng(2).standard_normal(3000)
    with pytest.raises(pkg.AsssError) as e:
        pkg.Solver(A, inner_tol=1e-10)                 # default scaling: zero pivots
    assert e.value.status == 3
    for precision in ("fp64", "mixed"):
        s = pkg.Solver(A, scaling="matching", precision=precision, outer="fgmres",
                       inner_tol=1e-10 if precision == "fp64" else 1e-6)
        perm = s.export_permutation()
        ex = s.export(A.nnz)
        Abar, _, _, _ = O.equilibrate(A, row_perm=perm, dr=ex["dr"], dc=ex["dc"])
        np.testing.assert_allclose(np.abs(Abar.diagonal()), 1.0, rtol=1e-12)
        x, st = s.solve(b)
        assert st["status"] == 0 and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
        xd = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
        s.close()


def test_matching_rejects_structurally_singular(pkg):
    A = sp.csr_matrix(np.array([[1.0, 2.0, 3.0], [4.0, 0.0, 0.0], [5.0, 0.0, 0.0]]))
    with pytest.raises(pkg.AsssError) as e:
        pkg.matching_scaling(A)
    assert e.value.status == 2


def test_matching_scalings_stay_in_a_moderate_range(pkg):
    """Rows with a single entry must not drive their column's price (and the scalings)
    up by a large bid in every epsilon phase: lopsided scalings of e^100 and more defeat
    the outer iteration in floating point."""
    A = indefinite_zero_diagonal(600, 0)
    C, colmax = O.matching_costs(A)
    assert (np.diff(C.indptr) == 1).sum() > 0             # the case has single-entry rows
    perm, dr, dc, _ = pkg.matching_scaling(A)
    span = np.log(dr).max() - np.log(dr).min()
    assert span <= 4 * max(1.0, C.data.max()), span
