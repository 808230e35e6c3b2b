"""Batched solves (many dissipative-Hamiltonian systems of uneven size, several
right-hand sides each) through the C ABI: every (system, column) must meet the
outer tolerance on the true FP64 residual and agree with the exact solution
and with the one-system path; graph replays are deterministic."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from workloads import batched_dissipative_hamiltonian, dissipative_hamiltonian_3d

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


@pytest.fixture(scope="module")
def batch():
    # sides 5..14: n from 125 (a ragged single slice) to 2744
    return batched_dissipative_hamiltonian(count=9, side_lo=5, side_hi=14, nrhs=3, seed=11)


def _check_columns(mats, X, B, tol=1e-8):
    for (A, _), x, b in zip(mats, X, B):
        for c in range(b.shape[1]):
            bn = np.linalg.norm(b[:, c])
            assert np.linalg.norm(b[:, c] - A @ x[:, c]) <= tol * bn * (1 + 1e-9)


def test_batched_matches_exact_solutions(pkg, batch):
    As = [A for A, _ in batch]
    Bs = [B for _, B in batch]
    bs = pkg.BatchSolver(As, inner_tol=1e-6, restart=24)
    assert bs.cta_threads == 0
    nrhs = Bs[0].shape[1]
    x, st = bs.solve(bs.pack(Bs), nrhs=nrhs)
    assert (bs.cta_threads, bs.cta_registers) in {(256, 64), (512, 64), (256, 80), (384, 80), (256, 128),
                                                  (512, 128)}
    assert st["status"] == 0
    assert st["inner_solves"] == len(As) * nrhs
    assert st["relres"] <= 1e-8
    X = bs.unpack(x, nrhs)
    _check_columns(batch, X, Bs)
    for A, Xm, Bm in zip(As, X, Bs):
        lu = spla.splu(A.tocsc())
        xs = lu.solve(Bm)
        assert np.linalg.norm(Xm - xs) <= 1e-6 * np.linalg.norm(xs)
    bs.close()


def test_batched_agrees_with_single_system_path(pkg, batch):
    As = [A for A, _ in batch[:4]]
    Bs = [B[:, :2] for _, B in batch[:4]]
    bs = pkg.BatchSolver(As, inner_tol=1e-6, restart=24)
    x, st = bs.solve(bs.pack(Bs), nrhs=2)
    assert st["status"] == 0
    X = bs.unpack(x, 2)
    for A, Xm, Bm in zip(As, X, Bs):
        s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, restart=24)
        xs, st1 = s.solve(Bm)
        assert st1["status"] == 0
        assert np.linalg.norm(Xm - xs) <= 1e-6 * np.linalg.norm(xs)
        s.close()
    bs.close()


def test_batched_device_buffers_and_replay_are_deterministic(pkg, batch):
    import torch
    As = [A for A, _ in batch]
    Bs = [B for _, B in batch]
    bs = pkg.BatchSolver(As, inner_tol=1e-6, restart=24)
    nrhs = Bs[0].shape[1]
    bh = bs.pack(Bs)
    x_host, _ = bs.solve(bh, nrhs=nrhs)
    bd = torch.from_numpy(bh).cuda()
    xd = torch.empty_like(bd)
    x1, st1 = bs.solve(bd, nrhs=nrhs, x=xd)
    r1 = x1.cpu().numpy().copy()
    x2, st2 = bs.solve(bd, nrhs=nrhs, x=xd)   # replay of the captured graph
    r2 = x2.cpu().numpy()
    assert st1["status"] == 0 and st2["status"] == 0
    assert np.array_equal(r1, r2)
    assert np.array_equal(r1, x_host)
    bs.close()


def test_batched_zero_column_and_single_matrix(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=7, seed=21)
    bs = pkg.BatchSolver([A], inner_tol=1e-6)
    B = np.stack([b, np.zeros_like(b), -2.0 * b], axis=1)
    x, st = bs.solve(bs.pack([B]), nrhs=3)
    assert st["status"] == 0
    X = bs.unpack(x, 3)[0]
    assert np.all(X[:, 1] == 0.0)
    assert np.linalg.norm(b - A @ X[:, 0]) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(-2 * b - A @ X[:, 2]) <= 1e-8 * 2 * np.linalg.norm(b)
    bs.close()


def test_batched_rejects_wrong_lengths(pkg):
    A, b, _ = dissipative_hamiltonian_3d(side=6, seed=2)
    bs = pkg.BatchSolver([A, A], inner_tol=1e-6)
    with pytest.raises(ValueError):
        bs.solve(np.zeros(A.shape[0]), nrhs=1)
    bs.close()


@pytest.mark.slow
def test_batched_full_size_workload(pkg):
    """The 256-system x 32-column workload of the batched benchmark, in the launch
    configuration the benchmark times: every item meets the tolerance on the host, and
    sampled items (the smallest systems, one column each) agree with the FP64 oracle."""
    import oracle as O
    batch = batched_dissipative_hamiltonian(count=256, side_lo=10, side_hi=40, nrhs=32, seed=3)
    As = [A for A, _ in batch]
    Bs = [B for _, B in batch]
    bs = pkg.BatchSolver(As, inner_tol=1e-6, outer_tol=1e-8, k=20, restart=24)
    x, st = bs.solve(bs.pack(Bs), nrhs=32)
    assert st["status"] == 0 and st["inner_solves"] == 256 * 32
    X = bs.unpack(x, 32)
    worst = max(float(np.max(np.linalg.norm(B - A @ Xm, axis=0) / np.linalg.norm(B, axis=0)))
                for (A, B), Xm in zip(batch, X))
    assert worst <= 1e-8
    order = np.argsort([A.shape[0] for A in As])[:3]
    for m in order:
        o = O.AsssOracle(As[m], inner_tol=1e-6)
        xo, sto = o.solve(Bs[m][:, 5], tol=1e-8, outer="fgmres")
        assert np.linalg.norm(X[m][:, 5] - xo) <= 1e-6 * np.linalg.norm(xo)
    bs.close()


def test_batched_bf16_basis_and_a_tiny_system(pkg, batch):
    # the BF16 deflation basis (the kernel reads Q in BF16): same tolerance, nearly the
    # same solutions as the FP32 basis
    As = [A for A, _ in batch[:5]]
    Bs = [B[:, :2] for _, B in batch[:5]]
    x32, st32 = pkg.BatchSolver(As, inner_tol=1e-6).solve(np.concatenate(
        [b.ravel(order="F") for b in Bs]), nrhs=2)
    b16 = pkg.BatchSolver(As, inner_tol=1e-6, q_bf16=True)
    x16, st16 = b16.solve(b16.pack(Bs), nrhs=2)
    assert st16["status"] == 0 and st16["relres"] <= 1e-8
    _check_columns(list(zip(As, Bs)), b16.unpack(x16, 2), Bs)
    assert np.linalg.norm(x16 - x32) <= 1e-6 * np.linalg.norm(x32)
    b16.close()
    # a 27-row system (smaller than one 32-row slice, fewer Lanczos vectors than asked)
    A, b, _ = dissipative_hamiltonian_3d(side=3, seed=8)
    bs = pkg.BatchSolver([A], inner_tol=1e-6)
    x, st = bs.solve(b, nrhs=1)
    assert st["status"] == 0
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    bs.close()


def test_batched_general_patterns_use_sell(pkg):
    """Matrices whose J~ does not fit skew diagonals (general sparse patterns, power-law
    rows) join the batch in SELL-C-sigma storage, next to stencil matrices in skew
    diagonals; every item meets the tolerance and the exact solution."""
    import scipy.sparse as sp
    rng = np.random.default_rng(71)
    mats = []
    for n in (700, 1300, 2111):
        K = sp.random(n, n, density=6.0 / n, random_state=rng, data_rvs=rng.standard_normal)
        A = (K + sp.diags(4.0 + rng.random(n))).tocsr()
        A.sum_duplicates()
        A.sort_indices()
        mats.append(A)
    # a few long rows (heavy tail, so the SELL slices are sorted by length)
    n = 1500
    K = sp.random(n, n, density=5.0 / n, random_state=rng, data_rvs=rng.standard_normal).tolil()
    for i in rng.choice(n, 12, replace=False):
        cols = rng.choice(n, 300, replace=False)
        K[i, cols] = 0.01 * rng.standard_normal(300)
    A = (K.tocsr() + sp.diags(4.0 + rng.random(n))).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    mats.append(A)
    mats.append(dissipative_hamiltonian_3d(side=9, seed=3)[0])
    nrhs = 2
    Bs = [rng.standard_normal((A.shape[0], nrhs)) for A in mats]
    bs = pkg.BatchSolver(mats, inner_tol=1e-6, restart=24, outer_maxit=400)
    x, st = bs.solve(bs.pack(Bs), nrhs=nrhs)
    X = bs.unpack(x, nrhs)
    for A, Xm, Bm in zip(mats, X, Bs):
        xs = spla.splu(A.tocsc()).solve(Bm)
        for c in range(nrhs):
            r = np.linalg.norm(Bm[:, c] - A @ Xm[:, c]) / np.linalg.norm(Bm[:, c])
            assert r <= 1e-8, r
        assert np.linalg.norm(Xm - xs) <= 1e-6 * np.linalg.norm(xs)
    assert st["status"] == 0
    bs.close()


@pytest.mark.parametrize("shape,regs", [("256x4", 64), ("512x2", 64), ("256x3", 80), ("384x2", 80), ("256x2", 128),
                                        ("512x1", 128)])
def test_batched_every_cta_shape_meets_the_tolerance(pkg, batch, shape, regs, monkeypatch):
    """Each CTA shape the tuner may pick (threads per CTA x resident CTAs per SM, which
    sets the registers a thread may use; at 128 registers a row's loads are unrolled)
    solves every item to the outer tolerance and agrees with the exact solution."""
    monkeypatch.setenv("ASSS_BATCH_CTA", shape)
    As = [A for A, _ in batch]
    Bs = [B for _, B in batch]
    bs = pkg.BatchSolver(As, inner_tol=1e-6, restart=24)
    nrhs = Bs[0].shape[1]
    x, st = bs.solve(bs.pack(Bs), nrhs=nrhs)
    assert bs.cta_threads == int(shape.split("x")[0])
    assert bs.cta_registers == regs
    assert st["status"] == 0 and st["relres"] <= 1e-8
    X = bs.unpack(x, nrhs)
    _check_columns(batch, X, Bs)
    for (A, _), xm, b in zip(batch, X, Bs):
        xe = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(xm - xe) <= 1e-6 * np.linalg.norm(xe)
    bs.close()


def test_batched_setup_reports_a_bad_matrix_and_recovers(pkg, batch):
    """The matrices are set up concurrently (host threads with streams of their own): a
    malformed matrix among them (an empty row, rejected on the host) makes the whole
    set-up return its status with the error text, and a valid batch sets up and solves
    afterwards."""
    As = [A for A, _ in batch]
    bad = As[3].tolil()
    bad[5, :] = 0.0
    bad = bad.tocsr()
    bad.eliminate_zeros()
    with pytest.raises(pkg.AsssError) as ei:
        pkg.BatchSolver(As[:3] + [bad] + As[4:], inner_tol=1e-3, restart=24)
    assert "asss_setup_batched" in str(ei.value)
    bs = pkg.BatchSolver(As, inner_tol=1e-3, restart=24)
    Bs = [B for _, B in batch]
    x, st = bs.solve(bs.pack(Bs), nrhs=Bs[0].shape[1])
    assert st["status"] == 0
    _check_columns(batch, bs.unpack(x, Bs[0].shape[1]), Bs)
    bs.close()
