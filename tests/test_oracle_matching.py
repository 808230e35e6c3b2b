"""Pins of the oracle's maximum-product matching and scaling (§2, Eq. mc64).

The matching is pinned to an independent solver of the same assignment problem
(scipy's min_weight_full_bipartite_matching) and to brute force over all
permutations on tiny inputs; the scaling to the properties Eq. mc64 asks for
(modulus one on the diagonal, at most one elsewhere) and to LP duality."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import min_weight_full_bipartite_matching

import oracle as O


def _indefinite_zero_diag(n, seed):
    from workloads import indefinite_zero_diagonal
    return indefinite_zero_diagonal(n, seed)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matching_cost_equals_independent_solver(seed):
    A = _indefinite_zero_diag(300, seed)
    C, _ = O.matching_costs(A)
    rc, u, v, total = O.max_product_matching(A)
    # scipy treats stored zeros as missing edges: shift every cost by one (every
    # perfect matching gains exactly n, so the argmin is unchanged)
    W = C.copy()
    W.data = W.data + 1.0
    r, c = min_weight_full_bipartite_matching(W)
    ref = float(sum(C[i, j] for i, j in zip(r, c)))
    assert abs(total - ref) <= 1e-9 * max(1.0, ref)
    assert sorted(rc) == list(range(300))


def test_matching_brute_force_tiny():
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = 6
        A = sp.random(n, n, density=0.6, random_state=rng, data_rvs=rng.standard_normal).tocsr()
        A = A + sp.csr_matrix((np.full(n, 1e-3), (np.arange(n), rng.permutation(n))), shape=(n, n))
        A = sp.csr_matrix(A)
        A.sort_indices()
        D = np.abs(A.toarray())
        best = -np.inf
        for p in itertools.permutations(range(n)):
            vals = D[list(p), range(n)]
            if np.all(vals > 0):
                best = max(best, np.sum(np.log(vals)))
        rc, _, _, _ = O.max_product_matching(A)
        got = np.sum(np.log(D[rc, np.arange(n)]))
        assert abs(got - best) <= 1e-12 * max(1.0, abs(best))


def test_scaling_properties_and_duality():
    A = _indefinite_zero_diag(500, 5)
    perm, dr, dc = O.matching_scaling(A)
    Abar, _, _, _ = O.equilibrate(A, row_perm=perm, dr=dr, dc=dc)
    d = np.abs(Abar.diagonal())
    np.testing.assert_allclose(d, 1.0, rtol=1e-12)
    assert np.abs(Abar.data).max() <= 1.0 + 1e-12
    # dual feasibility c_ij >= u_i + v_j with equality on the matching
    C, _ = O.matching_costs(A)
    rc, u, v, total = O.max_product_matching(A)
    rows = np.repeat(np.arange(500), np.diff(C.indptr))
    slack = C.data - u[rows] - v[C.indices]
    assert slack.min() >= -1e-10
    assert abs(total - (u.sum() + v.sum())) <= 1e-9 * max(1.0, abs(total))   # strong duality


def test_structurally_singular_is_rejected():
    """Rows 1 and 2 both have column 0 only (Hall's condition fails)."""
    A = sp.csr_matrix(np.array([[1.0, 2.0, 3.0], [4.0, 0.0, 0.0], [5.0, 0.0, 0.0]]))
    with pytest.raises(ValueError):
        O.max_product_matching(A)


def test_matching_makes_the_setup_possible():
    """Eq. mc64's purpose: on a matrix with a zero diagonal the default scaling leaves
    zero pivots in diag(Abar S), the matched scaling gives a set-up that solves."""
    A = _indefinite_zero_diag(400, 0)
    b = np.random.default_rng(0).standard_normal(400)
    with pytest.raises(ZeroDivisionError):
        O.AsssOracle(A, inner_tol=1e-10)
    perm, dr, dc = O.matching_scaling(A)
    o = O.AsssOracle(A, inner_tol=1e-10, row_perm=perm, dr=dr, dc=dc)
    x, st = o.solve(b, tol=1e-8, outer="fgmres")
    assert st["status"] == "ok" and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)


def test_planted_dual_update_mistake_is_caught():
    """A dual update with the wrong sign breaks feasibility or optimality."""
    import inspect
    src = inspect.getsource(O.matching)
    bad = src.replace("v[j] -= D - dist_c[j]", "v[j] += D - dist_c[j]")
    assert bad != src
    ns = {}
    exec(compile(bad, "planted", "exec"), ns)
    A = _indefinite_zero_diag(120, 3)
    C, _ = ns["matching_costs"](A)
    try:
        rc, u, v, total = ns["max_product_matching"](A)
    except Exception:
        return
    W = C.copy()
    W.data = W.data + 1.0
    r, c = min_weight_full_bipartite_matching(W)
    ref = float(sum(C[i, j] for i, j in zip(r, c)))
    rows = np.repeat(np.arange(120), np.diff(C.indptr))
    slack = C.data - u[rows] - v[C.indices]
    assert abs(total - ref) > 1e-9 or slack.min() < -1e-10
