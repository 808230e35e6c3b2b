"""Failure detection through the C ABI, with the failures made on the host (bad
inputs, a forced iteration limit, a NaN right-hand side): every call returns a
status code, nothing aborts, and the handle stays usable afterwards. (The device
wait that runs out is covered in test_gpu_parity.py.)"""
import numpy as np
import pytest
import scipy.sparse as sp

from workloads import dissipative_hamiltonian_3d, pattern_diagonal

pytestmark = pytest.mark.gpu

ERR_PATTERN, ERR_ZERO_DIAG, ERR_BREAKDOWN, NOT_CONVERGED = 2, 3, 4, 5


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_06954_gb300 as p
    return p


def _small():
    A, b, _ = dissipative_hamiltonian_3d(side=6, seed=3)
    return sp.csr_matrix(A), b


class _RawCSR(tuple):
    """(indptr, indices, data, n) handed to the library as is (no sorting on the way)."""

    @property
    def shape(self):
        return (self[3], self[3])

    @property
    def nnz(self):
        return len(self[1])


def test_unsorted_columns_are_rejected(pkg):
    A, _ = _small()
    indices = A.indices.copy()
    r = 10
    a, e = A.indptr[r], A.indptr[r + 1]
    indices[a], indices[e - 1] = indices[e - 1], indices[a]
    with pytest.raises(pkg.AsssError) as ei:
        pkg.Solver(_RawCSR((A.indptr.copy(), indices, A.data.copy(), A.shape[0])))
    assert ei.value.status == ERR_PATTERN


def test_column_out_of_range_is_rejected(pkg):
    A, _ = _small()
    indices = A.indices.copy()
    r = 20
    indices[A.indptr[r + 1] - 1] = A.shape[0] + 5
    with pytest.raises(pkg.AsssError) as ei:
        pkg.Solver(_RawCSR((A.indptr.copy(), indices, A.data.copy(), A.shape[0])))
    assert ei.value.status == ERR_PATTERN


def test_empty_row_is_rejected(pkg):
    A, _ = _small()
    A = A.tolil()
    A.rows[7] = []
    A.data[7] = []
    with pytest.raises(pkg.AsssError) as ei:
        pkg.Solver(A.tocsr())
    assert ei.value.status == ERR_PATTERN


def test_zero_pivot_is_reported(pkg):
    # with a diagonal S, (Abar S)_ii = abar_ii s_ii vanishes where A has no diagonal entry
    A, _ = _small()
    A = A.tolil()
    A[11, 11] = 0.0
    A = A.tocsr()
    A.eliminate_zeros()
    with pytest.raises(pkg.AsssError) as ei:
        pkg.Solver(A, s_pattern=pattern_diagonal(A.shape[0]))
    assert ei.value.status == ERR_ZERO_DIAG


def test_iteration_limit_and_nan_rhs_leave_the_handle_usable(pkg):
    A, b = _small()
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_maxit=1)
    x, st = s.solve(b)
    assert st["status"] == NOT_CONVERGED
    assert np.all(np.isfinite(x)) and st["outer_its"] == 1
    assert np.linalg.norm(b - A @ x) < np.linalg.norm(b)
    s.close()
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6)
    bn = b.copy()
    bn[3] = np.nan
    _, st = s.solve(bn)  # a soft status: the call returns, the status says why
    assert st["status"] == ERR_BREAKDOWN
    x, st = s.solve(b)  # the same handle solves a valid system afterwards
    assert st["status"] == 0 and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    s.close()
