"""The allocation-free mrs entry point (asss_mrs_noalloc).

asss_mrs_noalloc serves callers that may not allocate device memory during a
call (a memory-capped service with a fixed device budget, or code running under
an allocator whose pool must not grow while a request is in flight).  It takes
device arrays only and keeps its scratch in a static device array of the
library.  Its result must equal the FP64 oracle's mrs (App. B) on the same
operator, element by element, and the ordinary entry point asss_mrs - here on
two calls in a row, which also checks that the reused scratch starts clean and
that neither call changes the device's free memory.  Bad arguments (a malformed
CSR, a misaligned q, non-zero padding columns of q, a sign other than +-1, n
beyond the scratch) are rejected on the host side before any launch.

This file is collected last on purpose; it passes alone and after the rest.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O

pytestmark = pytest.mark.gpu


def _skew(n, seed):
    rng = np.random.default_rng(seed)
    K = sp.random(n, n, density=12.0 / (2.0 * n), random_state=rng, data_rvs=rng.standard_normal)
    J = (K - K.T).tocsr() * 0.1
    J.sum_duplicates()
    J.sort_indices()
    J.eliminate_zeros()
    return J


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_06954_gb300 as pkg
    return torch, pkg, pkg.lib(), torch.device("cuda", 0)


class _Case:
    """Device copies of J, a padded row-major Q and alpha for one operator."""

    def __init__(self, torch, dev, n, k, kp, seed):
        self.n, self.k, self.kp = n, k, kp
        self.J = _skew(n, seed)
        rng = np.random.default_rng(seed + 5)
        self.Q, self.alpha = O.skew_lanczos(self.J, rng.standard_normal(n), k)
        self.Sk = O.lanczos_tridiagonal(self.alpha)
        qpad = np.zeros((n, kp))
        qpad[:, :k] = self.Q
        self.rp = torch.tensor(self.J.indptr.astype(np.int64), device=dev)
        self.ci = torch.tensor(self.J.indices.astype(np.int32), device=dev)
        self.vv = torch.tensor(self.J.data, device=dev)
        self.q = torch.tensor(qpad, device=dev)          # n x kp row-major
        self.al = torch.tensor(self.alpha, device=dev)

    def apply(self, V, sign):
        return sign * (self.J @ V - self.Q @ (self.Sk @ (self.Q.T @ V)))


def _call(L, c, b_dev, x_dev, sign=1.0, tol=1e-12, maxit=3000, q_ptr=None, rp_ptr=None, ci_ptr=None, n=None):
    its, ratio = C.c_int(0), C.c_double(0.0)
    st = L.asss_mrs_noalloc(c.n if n is None else n, c.J.nnz, rp_ptr or c.rp.data_ptr(), ci_ptr or c.ci.data_ptr(),
                            c.vv.data_ptr(), c.k, c.kp, q_ptr or c.q.data_ptr(), c.al.data_ptr(), 1.0, sign,
                            b_dev.data_ptr(), x_dev.data_ptr(), tol, maxit, C.byref(its), C.byref(ratio), None)
    return st, its.value, ratio.value


@pytest.mark.parametrize("kp,sign", [(20, 1.0), (24, 1.0), (20, -1.0)])
def test_mrs_noalloc_matches_oracle_and_asss_mrs_on_two_calls(env, kp, sign):
    """Two calls in a row, each against the oracle's mrs (element by element) and
    against asss_mrs; kp > k exercises zero padding columns, sign = -1 the
    transposed system D - J that the adjoint solve relies on."""
    torch, pkg, L, dev = env
    c = _Case(torch, dev, 30001, 20, kp, seed=4)
    rng = np.random.default_rng(9)
    x = torch.empty(c.n, dtype=torch.float64, device=dev)
    # one call first so that the library's module (with its static array) is resident
    # before free memory is compared
    bw = torch.tensor(rng.standard_normal(c.n), device=dev)
    assert _call(L, c, bw, x, sign=sign)[0] == 0, L.asss_last_error()
    for call in range(2):
        b = rng.standard_normal(c.n)
        bd = torch.tensor(b, device=dev)
        x.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        st, its, ratio = _call(L, c, bd, x, sign=sign)
        assert st == 0, L.asss_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(dev)[0] == free_before, call
        xg = x.cpu().numpy()
        xo, its_o, ratio_o, _ = O.mrs(1.0, lambda V: c.apply(V, sign), b, 3000, 1e-12)
        assert abs(its - its_o) <= 2, (its, its_o)
        assert ratio < 1e-12
        np.testing.assert_allclose(xg, xo, rtol=0, atol=1e-9 * np.abs(xo).max())
        x_ref, its_ref, _ = pkg.mrs(c.J, b, c.Q, c.alpha, sign=sign, tol=1e-12, maxit=3000)
        assert abs(its - its_ref) <= 2
        np.testing.assert_allclose(xg, x_ref, rtol=0, atol=1e-9 * np.abs(x_ref).max())


def test_mrs_noalloc_rejects_bad_arguments_before_any_launch(env):
    torch, pkg, L, dev = env
    c = _Case(torch, dev, 4001, 8, 12, seed=7)
    b = torch.ones(c.n, dtype=torch.float64, device=dev)
    x = torch.zeros(c.n, dtype=torch.float64, device=dev)
    # n beyond the static scratch
    st = L.asss_mrs_noalloc(65537, 0, None, None, None, 0, 0, None, None, 1.0, 1.0, None, None, 1e-8, 10,
                            None, None, None)
    assert st == 1 and b"65536" in L.asss_last_error()
    # a sign other than +-1
    assert _call(L, c, b, x, sign=0.5)[0] == 1
    # q offset by one double: not 16-byte aligned for the kernel's row loads
    qbig = torch.zeros(c.n * c.kp + 1, dtype=torch.float64, device=dev)
    assert _call(L, c, b, x, q_ptr=qbig.data_ptr() + 8)[0] == 1
    assert b"aligned" in L.asss_last_error()
    # non-zero padding column of q
    qbad = c.q.clone()
    qbad[17, c.k + 1] = float("nan")
    assert _call(L, c, b, x, q_ptr=qbad.data_ptr())[0] == 1
    # host memory where device memory is required
    qh = np.zeros(c.n * c.kp)
    assert _call(L, c, b, x, q_ptr=qh.ctypes.data)[0] == 1
    # a row pointer out of range and a column index out of range: ASSS_ERR_PATTERN
    rp_bad = c.rp.clone()
    rp_bad[c.n // 2] = c.J.nnz + 5
    assert _call(L, c, b, x, rp_ptr=rp_bad.data_ptr())[0] == 2
    ci_bad = c.ci.clone()
    ci_bad[c.J.nnz // 3] = c.n
    assert _call(L, c, b, x, ci_ptr=ci_bad.data_ptr())[0] == 2
    # the same arrays unchanged still solve
    st, its, ratio = _call(L, c, b, x, tol=1e-10)
    assert st == 0 and ratio < 1e-10
