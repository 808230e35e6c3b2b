"""Pattern, weight and deflation study on synthetic inputs (GPU).

For one matrix of the dissipative-Hamiltonian family (or the 2D convection-diffusion
matrix) this sets the method up with different choices the paper discusses and prints
one markdown row per choice:

* the pattern of S: diagonal (S_d), tridiagonal (S_t) or the pattern of A (§2, Table 3),
* the weight gamma of the diagonal equations (§2, Eq. regularized),
* the number k of skew-Lanczos vectors used for deflation (§3.2),
* the factor L~ of M^: 1x1 pivots without fill ("diag"), the no-fill incomplete
  L D L^T ("ildl0", §3 after Eq. absfac, §4.1's ~ildl(0)), or the same with 2x2 pivot
  blocks ("ildl0_bk", Fig. 1; --matrix saddle).

Columns: the least-squares fit (iterations of the GPU solver), how skew-symmetric the
off-diagonal part of Abar S is (||(C - C^T)/2||_F / ||C - diag C||_F, C = Abar S), how far
its diagonal is from the identity (||diag C - 1||_F / sqrt(n)), the number r of negative
diagonal entries, and the solve: outer iterations, average inner (mrs) iterations per
preconditioner application, device solve time and the final relative residual.

    python -m paper_2009_06954_gb300.study [--side 48] [--matrix dh|cd|saddle]
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import norm as spnorm

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2009_06954_gb300 import Solver  # noqa: E402
from workloads import (convection_diffusion_2d, dissipative_hamiltonian_3d, pattern_diagonal,  # noqa: E402
                       pattern_of, pattern_tridiagonal)


def _scaled(A):
    """Abar = D_r A D_c with the row-max then column-max scalings (the set-up's default)."""
    A = sp.csr_matrix(A)
    dr = 1.0 / np.asarray(abs(A).max(axis=1).todense()).ravel()
    dc = 1.0 / np.asarray(abs(sp.diags(dr) @ A).max(axis=0).todense()).ravel()
    return (sp.diags(dr) @ A @ sp.diags(dc)).tocsr()


def skew_measures(Abar, S):
    C = (Abar @ S).tocsr()
    d = C.diagonal()
    off = C - sp.diags(d)
    skew = 0.5 * (off - off.T)
    n_off = spnorm(off)
    frac = spnorm(skew) / n_off if n_off > 0 else 1.0
    return frac, float(np.linalg.norm(d - 1.0) / np.sqrt(len(d)))


def measure_case(A, b, S_pat, gamma, k, precision, outer, inner_tol, factor="diag", **extra):
    """Set up and solve once with one choice; returns the study's measures as a dict
    (extra: further Solver options, e.g. given S values)."""
    s = Solver(A, s_pattern=S_pat, gamma=gamma, k=k, precision=precision, outer=outer,
               inner_tol=inner_tol, factor=factor, **extra)
    st0 = s.setup_stats
    ex = s.export(S_pat.nnz)
    S = sp.csr_matrix((ex["s_val"], S_pat.indices.copy(), S_pat.indptr.copy()), shape=A.shape)
    frac, ddev = skew_measures(_scaled(A), S)
    x, st = s.solve(b)
    s.close()
    relres = float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    return {"lls_its": st0["lls_its"], "skew_fraction": frac, "diag_dev": ddev, "r": st0["r"],
            "pairs": st0["factor_pairs"], "outer_its": st["outer_its"], "inner_its_avg": st["inner_its_avg"],
            "solve_ms": st["t_solve_ms"], "relres": relres, "status": st["status"]}


def run_case(A, b, pattern_name, S_pat, gamma, k, precision, outer, inner_tol, factor="diag"):
    m = measure_case(A, b, S_pat, gamma, k, precision, outer, inner_tol, factor)
    return (f"| {factor} | {pattern_name} | {gamma:g} | {k} | {m['lls_its']} | {m['skew_fraction']:.4f} | "
            f"{m['diag_dev']:.2e} | {m['r']} | {m['outer_its']} | {m['inner_its_avg']:.1f} | "
            f"{m['solve_ms']:.1f} | {m['relres']:.1e} |")


def saddle_rows(n=1200, seed=1):
    """2x2 pivots (Fig. 1, reading R20): on saddle_pairs, whose symmetric part has
    zero-diagonal pairs, with S = I taken as given (M^ = the symmetric part of A: no 1x1
    pivot order factors it) and with S fitted on pat(A) (§2: the fit pulls diag(Abar S)
    towards 1)."""
    from paper_2009_06954_gb300 import AsssError
    from workloads import saddle_pairs
    A = saddle_pairs(n, seed=seed, singles=n // 10)
    b = np.random.default_rng(seed).standard_normal(n)
    I = sp.identity(n, format="csr")
    given = dict(s_values=np.ones(n), lls_maxit=0, dr=np.ones(n), dc=np.ones(n),
                 row_perm=np.arange(n, dtype=np.int32), r_max=n)
    rows = []
    for S_name, S_pat, extra in (("I (given)", I, given), ("pat(A) (fitted)", pattern_of(A), {"r_max": n})):
        for factor in ("diag", "ildl0", "ildl0_bk"):
            try:
                m = measure_case(A, b, S_pat, 1.0, 20, "fp64", "fgmres", 1e-10, factor, **extra)
                rows.append(f"| {factor} | {S_name} | {m['pairs']} | {m['r']} | {m['outer_its']} | "
                            f"{m['inner_its_avg']:.1f} | {m['solve_ms']:.1f} | {m['relres']:.1e} |")
            except AsssError as e:
                rows.append(f"| {factor} | {S_name} | - | - | set-up fails: {str(e).split(':')[1].strip()} | | | |")
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--matrix", default="dh", choices=["dh", "cd", "saddle"])
    ap.add_argument("--side", type=int, default=48)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args(argv)
    if args.matrix == "saddle":
        print("saddle_pairs n = 1200 (120 rows with a diagonal, 540 zero-diagonal pairs), r_max = n, FP64, "
              "FGMRES, inner tol 1e-10\n")
        print("| L~ | S | 2x2 pivots | r | outer its | inner its | solve ms | relres |")
        print("|---|---|---|---|---|---|---|---|")
        for row in saddle_rows():
            print(row, flush=True)
        return
    if args.matrix == "dh":
        A, b, _ = dissipative_hamiltonian_3d(side=args.side, seed=1)
        title = f"dissipative Hamiltonian {args.side}^3 (n = {A.shape[0]})"
    else:
        A, b, _ = convection_diffusion_2d(m=64)
        title = f"convection-diffusion 64^2 (n = {A.shape[0]})"
    n = A.shape[0]
    inner_tol = 1e-6 if args.precision == "mixed" else 1e-10
    outer = "fgmres" if args.precision == "mixed" else "tfqmr"
    pats = {"S_d": pattern_diagonal(n), "S_t": pattern_tridiagonal(n), "pat(A)": pattern_of(A)}
    print(f"{title}, {args.precision}, outer {outer}, inner tol {inner_tol:g}\n")
    print("| L~ | S pattern | gamma | k | LLS its | skew fraction | diag dev | r | outer its | inner its | "
          "solve ms | relres |")
    print("|---|---|---|---|---|---|---|---|---|---|---|---|")
    for name, P in pats.items():
        for gamma in (0.1, 1.0, 10.0):
            print(run_case(A, b, name, P, gamma, 20, args.precision, outer, inner_tol), flush=True)
    for k in (0, 10, 50):
        print(run_case(A, b, "pat(A)", pats["pat(A)"], 1.0, k, args.precision, outer, inner_tol), flush=True)
    for name in ("S_t", "pat(A)"):
        print(run_case(A, b, name, pats[name], 1.0, 20, args.precision, outer, inner_tol, "ildl0"), flush=True)


if __name__ == "__main__":
    main()
