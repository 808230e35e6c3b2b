"""The allocation-free mrs entry point (asss_mrs_noalloc) against asss_mrs.

asss_mrs_noalloc serves callers that may not allocate device memory during a
call (a memory-capped service with a fixed device budget, or code running under
an allocator whose pool must not grow while a request is in flight).  It takes
device arrays only and keeps its scratch in a static device array of the
library, so it must give the same answer as the ordinary entry point - here on
two calls in a row, which also checks that the reused scratch starts clean.

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


def test_mrs_noalloc_matches_asss_mrs_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_06954_gb300 as pkg
    L = pkg.lib()
    n, k = 30001, 20
    J = _skew(n, 4)
    rng = np.random.default_rng(9)
    Q, alpha = O.skew_lanczos(J, rng.standard_normal(n), k)
    dev = torch.device("cuda", 0)
    rp = torch.tensor(J.indptr.astype(np.int64), device=dev)
    ci = torch.tensor(J.indices.astype(np.int32), device=dev)
    vv = torch.tensor(J.data, device=dev)
    q_rm = torch.tensor(np.ascontiguousarray(Q), device=dev)          # n x k row-major, kp = k = 20
    al = torch.tensor(alpha, device=dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    for call in range(2):
        b = rng.standard_normal(n)
        x_ref, its_ref, ratio_ref = pkg.mrs(J, b, Q, alpha, tol=1e-12, maxit=3000)
        bd = torch.tensor(b, device=dev)
        x.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        its, ratio = C.c_int(0), C.c_double(0.0)
        st = L.asss_mrs_noalloc(n, J.nnz, rp.data_ptr(), ci.data_ptr(), vv.data_ptr(), k, k, q_rm.data_ptr(),
                                al.data_ptr(), 1.0, 1.0, bd.data_ptr(), x.data_ptr(), 1e-12, 3000, C.byref(its),
                                C.byref(ratio), None)
        assert st == 0, L.asss_last_error()
        if call == 1:   # the static scratch is already resident: nothing new on the device
            assert torch.cuda.mem_get_info(dev)[0] == free_before
        xg = x.cpu().numpy()
        assert abs(its.value - its_ref) <= 2, (its.value, its_ref)
        assert ratio.value < 1e-12
        assert np.linalg.norm(xg - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_mrs_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_06954_gb300 as pkg
    L = pkg.lib()
    st = L.asss_mrs_noalloc(65537, 0, None, None, None, 0, 0, None, None, 1.0, 1.0, None, None, 1e-8, 10,
                            None, None, None)
    assert st == 1 and b"65536" in L.asss_last_error()
