"""FP64 restatement of the ASSS + mrs two-level scheme (arXiv 2009.06954).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Library primitives used as
single steps: scipy.sparse products, a sparse direct solve / LSQR for the
least-squares problem, numpy dense LU for the small SMW matrix.

Readings of the paper taken where it is silent or ambiguous (listed in full in the
design notes of the repository):
  R1 scaling: identity permutation, D_r = 1/row-max|a|, then D_c = 1/col-max|D_r a|.
  R3 the LLS minimiser itself is the result (solver-independent).
  R5 incomplete LDL^T restricted to 1x1 pivots without fill: L~ = |diag(A^)|^(1/2);
     factor="ildl0": the no-fill incomplete L D L^T in a multicolour order (ildl.py).
  R7 Lanczos start vector from a counter-based splitmix64 stream; optional full
     re-orthogonalisation (two classical Gram-Schmidt passes).
  R8 SMW written in the inverse-free form  S^-1 - X Sig (I + U^T X Sig)^-1 U^T S^-1.
  R9 multi-RHS mrs either as printed (all columns until the worst converges) or with
     per-column freezing (identical to independent single-RHS solves).
  R11 outer method: TFQMR (Freund) or flexible GMRES(m), right preconditioned, run in
     cycles of a refinement loop on the true FP64 residual of the original system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------
# counter-based random stream (Lanczos start vector)
# ----------------------------------------------------------------------------
def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """U(-1,1) numbers from Vigna's splitmix64 (published definition):
    state_i = seed + (i+1) * 0x9E3779B97F4A7C15 (mod 2^64), output = mix(state_i),
    mix(z) = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB;
    z ^= z>>31.  u = (out >> 11) * 2^-53, returned as 2u - 1."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


# ----------------------------------------------------------------------------
# §2 Eq. (mc64): permutation and scaling
# ----------------------------------------------------------------------------
def equilibrate(A, row_perm=None, dr=None, dc=None):
    """Abar = P D_r A D_c  (§2, Eq. mc64).

    MC64 is not available; when dr/dc are not given they come from one row-max
    sweep followed by one column-max sweep (reading R1), which leaves every
    entry of modulus <= 1.  (P M)_{i,:} = M_{row_perm[i],:}.
    Returns (Abar csr, dr, dc, row_perm)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    n = A.shape[0]
    perm = np.arange(n) if row_perm is None else np.asarray(row_perm, dtype=np.int64)
    if dr is None:
        rmax = np.asarray(abs(A).max(axis=1).todense()).ravel()
        if np.any(rmax == 0):
            raise ValueError("A has an empty (all-zero) row")
        dr = 1.0 / rmax
    if dc is None:
        cmax = np.asarray(abs(sp.diags(dr) @ A).max(axis=0).todense()).ravel()
        if np.any(cmax == 0):
            raise ValueError("A has an empty (all-zero) column")
        dc = 1.0 / cmax
    Abar = (sp.diags(dr) @ A @ sp.diags(dc)).tocsr()[perm, :]
    Abar.sort_indices()
    return Abar.tocsr(), np.asarray(dr, float), np.asarray(dc, float), perm


# ----------------------------------------------------------------------------
# §2 Eqs. (eq1),(eq2),(regularized) and Appendix A: the least-squares problem
# ----------------------------------------------------------------------------
def lls_system(Abar, S_pattern, gamma: float = 1.0):
    """Assemble the weighted LLS of §2 for S on a given pattern (Appendix A).

    Unknowns: the nonzeros of S, numbered in S's CSR (row-major) order.
    Rows 0..neq-1: one per nonzero (i, j), i < j, of the strictly upper part of
    pat(Abar S) + pat(Abar S)^T, stating (Abar S)_ij + (Abar S)_ji = 0 (Eq. eq1):
    coefficient abar_il on unknown S_lj for every l with abar_il != 0, S_lj in
    the pattern, and abar_jl on S_li likewise.
    Rows neq..neq+n-1: sqrt(gamma) * (Abar S)_ii = sqrt(gamma) (Eq. eq2 weighted as in
    Eq. regularized).
    Returns (B csr, v, (s_rows, s_cols)) with v = [0; sqrt(gamma) 1]."""
    Abar = sp.csr_matrix(Abar)
    Sp = sp.csr_matrix(S_pattern)
    Sp.sort_indices()
    n = Abar.shape[0]
    s_rows = np.repeat(np.arange(n), np.diff(Sp.indptr))
    s_cols = Sp.indices.astype(np.int64)
    nu = s_cols.size
    # pattern of Abar S and the constraint pairs (strict upper of pat + pat^T)
    ones_A = sp.csr_matrix((np.ones(Abar.nnz), Abar.indices, Abar.indptr), shape=Abar.shape)
    ones_S = sp.csr_matrix((np.ones(nu), Sp.indices, Sp.indptr), shape=Sp.shape)
    AA = (ones_A @ ones_S).tocsr()
    U = sp.triu(AA + AA.T, 1).tocoo()
    pair_key = np.sort(U.row.astype(np.int64) * n + U.col.astype(np.int64))
    neq = pair_key.size
    # every path i -l-> j: abar_il != 0 and (l, j) in pat(S) contributes abar_il on
    # unknown (l, j) to the constraint of the pair {i, j}
    a_rows = np.repeat(np.arange(n), np.diff(Abar.indptr)).astype(np.int64)
    a_cols = Abar.indices.astype(np.int64)
    a_vals = Abar.data
    cnt = np.diff(Sp.indptr)[a_cols]
    p_i = np.repeat(a_rows, cnt)
    p_a = np.repeat(a_vals, cnt)
    starts = np.repeat(Sp.indptr[a_cols], cnt)
    within = np.arange(p_i.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    p_unk = starts + within                      # unknown index of S_lj
    p_j = s_cols[p_unk]
    lo = np.minimum(p_i, p_j)
    hi = np.maximum(p_i, p_j)
    row = np.empty(p_i.size, dtype=np.int64)
    off = lo != hi
    row[off] = np.searchsorted(pair_key, lo[off] * n + hi[off])
    row[~off] = neq + p_i[~off]
    val = np.where(off, p_a, np.sqrt(gamma) * p_a)
    B = sp.csr_matrix((val, (row, p_unk)), shape=(neq + n, nu))
    B.sum_duplicates()
    v = np.concatenate([np.zeros(neq), np.full(n, np.sqrt(gamma))])
    return B, v, (s_rows, s_cols)


def skew_symmetrizer(Abar, S_pattern, gamma: float = 1.0, method: str = "auto"):
    """S = argmin f(s, gamma) on the given pattern (§2, Eq. regularized; App. A).

    The paper solves the LLS with a sparse QR (Matlab backslash); the minimiser is
    what matters (reading R3).  Small problems: sparse LU of the normal equations;
    large ones: LSQR to near machine precision."""
    B, v, (s_rows, s_cols) = lls_system(Abar, S_pattern, gamma)
    nu = B.shape[1]
    if method == "auto":
        method = "normal" if nu <= 30_000 else "lsqr"
    if method == "normal":
        N = (B.T @ B).tocsc()
        s = spla.spsolve(N, B.T @ v)
    elif method == "lsqr":
        s = spla.lsqr(B, v, atol=1e-15, btol=1e-15, iter_lim=50_000)[0]
    elif method == "dense":
        s = np.linalg.lstsq(B.toarray(), v, rcond=None)[0]
    else:
        raise ValueError(method)
    n = Abar.shape[0]
    S = sp.csr_matrix((s, (s_rows, s_cols)), shape=(n, n))
    S.sort_indices()
    return S


# ----------------------------------------------------------------------------
# §3 Eq. (absfac), Fig. 1, Eq. (preconditioner): scaling and the rank-r part
# ----------------------------------------------------------------------------
def shift_and_lowrank(Abar, S, zero_tol: float = 1e-14):
    """d = diag(Abar S) = diag(M^); under reading R5 the incomplete factor is
    L~ = |D~|^(1/2) with D~ = diag(d), so W = L~^-1 = |d|^(-1/2) and
    M~_r = sign(d) - I (entries -2 where d < 0, §3 after Eq. absfac).
    Returns (d, w, neg) with neg the sorted indices where d < 0."""
    C = (sp.csr_matrix(Abar) @ sp.csr_matrix(S)).tocsr()
    d = C.diagonal().copy()
    dmax = np.abs(d).max() if d.size else 0.0
    if d.size and (dmax == 0 or np.any(np.abs(d) < zero_tol * dmax)):
        raise ZeroDivisionError("zero pivot in the diagonal factor (|d_i| tiny)")
    w = 1.0 / np.sqrt(np.abs(d))
    neg = np.flatnonzero(d < 0)
    return d, w, neg


def lowrank_decomposition(Mr_dense_sub):
    """Fig. 1: M_r = U_r Sigma_r U_r^T from the submatrix of M_r on its nonzero
    indices (1x1 blocks, or 2x2 blocks whose nonzero eigenpair is taken).
    Returns (U_sub, sigma) with U_sub (len(Ind) x r) and sigma (r,)."""
    M = np.asarray(Mr_dense_sub, dtype=np.float64)
    m = M.shape[0]
    cols, sig = [], []
    i = 0
    while i < m:
        if i + 1 < m and M[i, i + 1] != 0.0:
            lam, vec = np.linalg.eigh(M[i:i + 2, i:i + 2])
            kk = int(np.argmax(np.abs(lam)))
            u = np.zeros(m)
            u[i:i + 2] = vec[:, kk]
            cols.append(u)
            sig.append(lam[kk])
            i += 2
        else:
            u = np.zeros(m)
            u[i] = 1.0
            cols.append(u)
            sig.append(M[i, i])
            i += 1
    U = np.array(cols).T if cols else np.zeros((m, 0))
    return U, np.array(sig)


def inner_skew_operator(Abar, S, w):
    """J~ = L~^-1 J^ L~^-T = W (Abar S - (Abar S)^T)/2 W  (§3, Eq. preconditioner).

    Assembled from the strictly upper part and mirrored with opposite sign, so that
    J~ = -J~^T holds bit for bit."""
    C = (sp.csr_matrix(Abar) @ sp.csr_matrix(S)).tocsr()
    Jh = 0.5 * (C - C.T)
    Wd = sp.diags(w)
    Jt = (Wd @ Jh @ Wd).tocsr()
    U = sp.triu(Jt, 1).tocsr()
    Jt = (U - U.T).tocsr()
    Jt.sort_indices()
    return Jt


# ----------------------------------------------------------------------------
# §3.2 Fig. 2: skew-Lanczos; the deflated skew matrix
# ----------------------------------------------------------------------------
def skew_lanczos(J, q1, k: int, reorth: bool = True, breakdown_tol: float = 1e-12):
    """k steps of the skew-Lanczos process of Fig. 2 on J (J = -J^T).

    q_1 = q1/||q1||; z = J q_1, alpha_1 = ||z||, q_2 = -z/alpha_1; then for
    i = 2..k-1: z = J q_i - alpha_{i-1} q_{i-1}, alpha_i = ||z||, q_{i+1} = -z/alpha_i.
    With reorth, z is orthogonalised against all previous q by two classical
    Gram-Schmidt passes before its norm is taken (reading R7).  The process stops
    early when alpha_i <= breakdown_tol * alpha_1 (or alpha_1 == 0).
    Returns (Q n x k_eff, alpha (k_eff-1,))."""
    if sp.issparse(J) or isinstance(J, np.ndarray):
        J = sp.csr_matrix(J)
    n = J.shape[0]
    k = int(min(k, n))
    if k <= 0:
        return np.zeros((n, 0)), np.zeros(0)
    Q = np.zeros((n, k))
    alpha = np.zeros(max(k - 1, 0))
    Q[:, 0] = q1 / np.linalg.norm(q1)
    kk = 1
    for i in range(1, k):              # produces column i (q_{i+1} in 1-based terms)
        z = J @ Q[:, i - 1]
        if i >= 2:
            z = z - alpha[i - 2] * Q[:, i - 2]
        if reorth:
            for _ in range(2):
                z = z - Q[:, :i] @ (Q[:, :i].T @ z)
        a = np.linalg.norm(z)
        if a == 0.0 or (i >= 2 and a <= breakdown_tol * alpha[0]):
            break
        alpha[i - 1] = a
        Q[:, i] = -z / a
        kk = i + 1
    return Q[:, :kk], alpha[:kk - 1]


def lanczos_tridiagonal(alpha):
    """S_k of §3.2: skew tridiagonal, superdiagonal +alpha, subdiagonal -alpha."""
    k = alpha.size + 1
    T = np.zeros((k, k))
    for i, a in enumerate(alpha):
        T[i, i + 1] = a
        T[i + 1, i] = -a
    return T


# ----------------------------------------------------------------------------
# Appendix B: simultaneous mrs iterations for (alpha I + S) X = B
# ----------------------------------------------------------------------------
def mrs(alpha: float, apply_skew, B, maxit: int, tol: float, freeze: bool = True):
    """Minimal residual method for shifted skew-symmetric systems (§3.1, App. B).

    Each column runs the skew-Lanczos short recurrence
        q^ = S q_j + beta_{j-1} q_{j-1},  beta_j = ||q^||,  q_{j+1} = q^/beta_j,
    and a Givens QR of the (j+1) x j matrix with alpha on the diagonal, whose
    skew structure leaves only two nonzero superdiagonals in R (the middle one is
    exactly zero); the update directions obey
        p_j = (q_j - delta_{j-1} p_{j-2}) / theta_j,  x += g_j c_j p_j,  g_{j+1} = -g_j s_j.
    |g_{j+1}| is the residual norm.  A column whose |g|/||b|| < tol stops updating
    when freeze=True (reading R9); with freeze=False every column iterates until
    the worst ratio < tol, as printed.  A zero column gives x = 0.
    Returns (X, its[ncol], ratio[ncol], history list of ratio arrays)."""
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    if one:
        B = B[:, None]
    n, m = B.shape
    X = np.zeros((n, m))
    r0 = np.linalg.norm(B, axis=0)
    live = r0 > 0
    safe_r0 = np.where(live, r0, 1.0)
    g = r0.copy()
    q = B / safe_r0
    beta = np.zeros(m)
    theta_t = np.full(m, float(alpha))      # pre-rotation diagonal of the next column
    c_prev = np.ones(m)
    s_prev = np.zeros(m)
    delta_prev = np.zeros(m)
    q_prev = np.zeros((n, m))
    p_prev = np.zeros((n, m))
    p_prev2 = np.zeros((n, m))
    ratio = np.where(live, 1.0, 0.0)
    its = np.zeros(m, dtype=np.int64)
    active = live & (ratio >= tol)
    hist = [ratio.copy()]
    for it in range(1, maxit + 1):
        if not active.any():
            break
        qh = apply_skew(q) + q_prev * beta
        q_prev = q
        beta = np.linalg.norm(qh, axis=0)
        nz = beta != 0
        q = np.where(nz, qh / np.where(nz, beta, 1.0), q)
        theta = np.sqrt(theta_t * theta_t + beta * beta)
        c = theta_t / theta
        s = beta / theta
        delta = -s_prev * beta
        theta_t = c_prev * theta
        p = (q_prev - p_prev2 * delta_prev) / theta
        upd = active if freeze else live
        X[:, upd] += (p * (g * c))[:, upd]
        g = np.where(upd, -g * s, g)
        ratio = np.where(live, np.abs(g) / safe_r0, 0.0)
        its[upd] = it
        hist.append(ratio.copy())
        if freeze:
            active = active & (ratio >= tol)
        else:
            if ratio.max() < tol:
                active[:] = False
        p_prev2 = p_prev
        p_prev = p
        s_prev = s
        c_prev = c
        delta_prev = delta
    if one:
        return X[:, 0], its[0], ratio[0], hist
    return X, its, ratio, hist


# ----------------------------------------------------------------------------
# §4.1: outer Krylov cycles (right preconditioned)
# ----------------------------------------------------------------------------
def tfqmr_cycle(apply_op, apply_prec, r, eta: float, max_steps: int):
    """One TFQMR run (Freund 1993) on op(M^-1 u) = r from zero, right
    preconditioned, with the direction vectors kept in the solution space.

    Stops when the quasi-residual bound tau_m sqrt(m+1) <= eta ||r|| (m = half steps
    done), on breakdown (rho or sigma = 0), or after max_steps full steps.
    Returns (delta, full_steps, precond_applications)."""
    n = r.size
    delta = np.zeros(n)
    rnorm = np.linalg.norm(r)
    if rnorm == 0.0:
        return delta, 0, 0
    target = eta * rnorm
    w = r.copy()
    u = r.copy()
    ut = apply_prec(u)
    v = apply_op(ut)
    Bu_even = v                      # A_cal M^-1 u_m for the current even m
    Bu_odd = None
    d = np.zeros(n)
    tau = rnorm
    theta = 0.0
    eta_q = 0.0
    rstar = r.copy()
    rho = rstar @ r
    m = 0
    napp = 1
    for step in range(1, max_steps + 1):
        sigma = rstar @ v
        if sigma == 0.0 or rho == 0.0:
            return delta, step - 1, napp
        a = rho / sigma
        for half in range(2):
            if half == 0:
                Bu = Bu_even
            else:
                u = u - a * v
                ut = apply_prec(u)
                napp += 1
                Bu = apply_op(ut)
                Bu_odd = Bu
            w = w - a * Bu
            d = ut + (theta * theta * eta_q / a) * d
            theta = np.linalg.norm(w) / tau
            c = 1.0 / np.sqrt(1.0 + theta * theta)
            tau = tau * theta * c
            eta_q = c * c * a
            delta = delta + eta_q * d
            m += 1
            if tau * np.sqrt(m + 1.0) <= target:
                return delta, step, napp
        rho_new = rstar @ w
        beta = rho_new / rho
        rho = rho_new
        u = w + beta * u
        ut = apply_prec(u)
        napp += 1
        Bu_even = apply_op(ut)
        v = Bu_even + beta * (Bu_odd + beta * v)
    return delta, max_steps, napp


def fgmres_cycle(apply_op, apply_prec, r, eta: float, m: int):
    """One cycle of flexible GMRES(m) (Saad 1993) from zero with classical
    Gram-Schmidt applied twice and Givens rotations on the Hessenberg matrix.
    Stops when the residual estimate |g_{j+1}| <= eta ||r||, on a happy breakdown,
    or after m Arnoldi steps.  Returns (delta, steps, precond_applications)."""
    n = r.size
    beta0 = np.linalg.norm(r)
    if beta0 == 0.0:
        return np.zeros(n), 0, 0
    V = np.zeros((n, m + 1))
    Z = np.zeros((n, m))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta0
    V[:, 0] = r / beta0
    steps = 0
    for j in range(m):
        Z[:, j] = apply_prec(V[:, j])
        w = apply_op(Z[:, j])
        h = V[:, :j + 1].T @ w
        w = w - V[:, :j + 1] @ h
        h2 = V[:, :j + 1].T @ w
        w = w - V[:, :j + 1] @ h2
        h = h + h2
        hn = np.linalg.norm(w)
        col = np.zeros(m + 1)
        col[:j + 1] = h
        col[j + 1] = hn
        for i in range(j):
            t = cs[i] * col[i] + sn[i] * col[i + 1]
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
            col[i] = t
        rr = np.hypot(col[j], col[j + 1])
        cs[j] = col[j] / rr
        sn[j] = col[j + 1] / rr
        col[j] = rr
        col[j + 1] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        H[:, j] = col
        steps = j + 1
        if hn == 0.0 or abs(g[j + 1]) <= eta * beta0:
            break
        V[:, j + 1] = w / hn
    y = sla.solve_triangular(H[:steps, :steps], g[:steps])
    return Z[:, :steps] @ y, steps, steps


# ----------------------------------------------------------------------------
# the whole scheme
# ----------------------------------------------------------------------------
class AsssOracle:
    """Set-up (§2, §3, §4.1 pre-processing) and solve (§4.1) of the two-level scheme.

    Set-up, independent of b: scaling (Eq. mc64), S from the LLS (§2), the
    diagonal factor and M~_r (reading R5, Fig. 1), J~, skew-Lanczos (Fig. 2), the
    combined rank-(r+k) SMW data of Eq. (preconditioner)/(smw): X = S_bar^-1 U_bar
    by multi-RHS mrs and K = I + U_bar^T X Sig_bar.
    Solve: outer Krylov on  A_cal y = W P D_r b,  A_cal = W Abar S W, with
    preconditioner P^-1 applied via mrs + SMW; x = D_c S W y (§3, Eq. modified).

    factor="ildl0" replaces the diagonal factor by the no-fill incomplete L D L^T of M^
    (§3 after Eq. absfac, §4.1 ~ildl(0); ildl.py): L~^-1 and L~^-T are applied by
    triangular solves (F and G of FactoredSkew), A_cal = F Abar S G, J~ = F J^ G, the
    right-hand side F P D_r b and x = D_c S G y; M~_r = sign(D) - I.  factor="ildl0_bk"
    also takes 2x2 pivot blocks where the first Bunch-Kaufman test asks for them (reading
    R20): |D|^(-1/2) and M~_r = sign(D) - I = U_r Sigma_r U_r^T block by block (Fig. 1).
    S (optional) is used as given instead of the least-squares fit of §2."""

    def __init__(self, A, S_pattern=None, gamma=1.0, k=20, reorth=True, seed=0x5eed,
                 inner_tol=1e-10, inner_maxit=1000, setup_tol=None, r_max=256,
                 row_perm=None, dr=None, dc=None, q1=None, lls_method="auto",
                 zero_tol=1e-14, factor="diag", S=None):
        A = sp.csr_matrix(A, dtype=np.float64)
        A.sort_indices()
        self.A = A
        n = A.shape[0]
        self.n = n
        self.Abar, self.dr, self.dc, self.perm = equilibrate(A, row_perm, dr, dc)
        if S_pattern is None:           # "having the sparsity of Abar" (§2)
            Ab = self.Abar
            S_pattern = sp.csr_matrix((np.ones(Ab.nnz), Ab.indices, Ab.indptr), shape=Ab.shape)
        # S given (values already fitted, or chosen by a test) or fitted here (§2)
        self.S = sp.csr_matrix(S, dtype=np.float64) if S is not None else \
            skew_symmetrizer(self.Abar, S_pattern, gamma, lls_method)
        self.factor = factor
        self.fac = None
        if factor == "ildl0":
            from . import ildl
            C = (sp.csr_matrix(self.Abar) @ sp.csr_matrix(self.S)).tocsr()
            P = ildl.structural_pattern(self.Abar, self.S)
            MP = ildl.values_on_pattern(0.5 * (C + C.T), P)
            self.colour, self.jp_rounds = ildl.jp_colouring(P, ildl.colouring_priorities(seed, n))
            self.order = ildl.colour_order(self.colour)
            self.L, self.d = ildl.ildl0(MP, self.order, zero_tol)
            neg = np.flatnonzero(self.d < 0)
            self.w = np.ones(n)                 # L~ enters through F and G instead
            self.fac = ildl.FactoredSkew(self.L, self.d, self.order,
                                         inner_skew_operator(self.Abar, self.S, self.w))
        elif factor == "ildl0_bk":
            # 2x2 pivot blocks where the first Bunch-Kaufman test asks for them (R20)
            from . import ildl
            C = (sp.csr_matrix(self.Abar) @ sp.csr_matrix(self.S)).tocsr()
            Mh = 0.5 * (C + C.T)
            P = ildl.structural_pattern(self.Abar, self.S)
            self.partner = ildl.bk_pairs(ildl.values_on_pattern(Mh, P))
            Pb = ildl.block_pattern(P, self.partner)
            MP = ildl.values_on_pattern(Mh, Pb)
            self.colour, self.jp_rounds = ildl.jp_colouring_blocks(Pb, ildl.colouring_priorities(seed, n),
                                                                   self.partner)
            self.order = ildl.block_order(self.colour, self.partner)
            self.L, self.D = ildl.ildl0_blocks(MP, self.colour, self.partner, zero_tol)
            self.d = self.D.diagonal()
            W, self.Ur, self.sig_r = ildl.block_pivot_split(self.D, self.partner)
            self.w = np.ones(n)
            self.fac = ildl.FactoredSkew(self.L, None, self.order,
                                         inner_skew_operator(self.Abar, self.S, self.w), W=W)
            neg = np.arange(self.Ur.shape[1])       # r columns (counted; U_r set below)
        elif factor == "diag":
            self.d, self.w, neg = shift_and_lowrank(self.Abar, self.S, zero_tol)
        else:
            raise ValueError(f"unknown factor {factor!r}")
        self.prec2 = neg.size > r_max          # Eq. (preconditioner2) fallback
        self.neg = np.zeros(0, dtype=np.int64) if self.prec2 else neg
        self.r = self.neg.size
        self.Jt = self.fac if self.fac is not None else inner_skew_operator(self.Abar, self.S, self.w)
        if q1 is None:
            q1 = splitmix64_uniform(seed, n)
        self.Q, self.alpha = skew_lanczos(self.Jt, q1, k, reorth)
        self.k = self.Q.shape[1]
        self.Sk = lanczos_tridiagonal(self.alpha) if self.k > 0 else np.zeros((0, 0))
        self.inner_tol = inner_tol
        self.inner_maxit = inner_maxit
        self.setup_tol = inner_tol if setup_tol is None else setup_tol
        if factor == "ildl0_bk":
            if self.prec2:
                self.set_lowrank_columns(np.zeros((n, 0)), np.zeros(0))
            else:
                self.set_lowrank_columns(self.Ur, self.sig_r)
        else:
            self.set_lowrank(self.neg)
        self.inner_its = []
        # outer operator pieces: A_cal = (W Abar)(S W)
        self.Aw = (sp.diags(self.w) @ self.Abar).tocsr()
        self.Sw = (self.S @ sp.diags(self.w)).tocsr()

    def set_lowrank(self, neg):
        """U_bar = [Q_k, U_r], Sig_bar = blkdiag(S_k, -2 I_r)  (Eq. preconditioner);
        U_r = [e_i : i in neg] (Fig. 1 with 1x1 blocks).  Drops cached SMW data."""
        n = self.n
        neg = np.asarray(neg, dtype=np.int64)
        Ur = np.zeros((n, neg.size))
        Ur[neg, np.arange(neg.size)] = 1.0
        self.set_lowrank_columns(Ur, -2.0 * np.ones(neg.size))
        self.neg = neg

    def set_lowrank_columns(self, Ur, sig):
        """U_bar = [Q_k, U_r], Sig_bar = blkdiag(S_k, diag(sig)) for any U_r (Fig. 1: the
        eigenvectors of 2x2 pivot blocks, unit vectors of 1x1 ones).  Drops cached SMW
        data."""
        n = self.n
        Ur = np.asarray(Ur, dtype=np.float64).reshape(n, -1)
        self.Ur_cols, self.sig_cols = Ur, np.asarray(sig, dtype=np.float64)
        self.r = Ur.shape[1]
        self.neg = np.arange(self.r)
        m = self.k + self.r
        Ub = np.zeros((n, m))
        Ub[:, :self.k] = self.Q
        Ub[:, self.k:] = Ur
        Sig = np.zeros((m, m))
        Sig[:self.k, :self.k] = self.Sk
        Sig[self.k:, self.k:] = np.diag(self.sig_cols)
        self.Ub, self.Sig = Ub, Sig
        self._X = {}
        self._K = {}

    def prec_dense(self):
        """P = M~_r + I + J~ as a dense matrix (tiny problems, tests only)."""
        P = (self.fac.dense() if self.fac is not None else self.Jt.toarray()) + np.eye(self.n)
        P += self.Ur_cols @ np.diag(self.sig_cols) @ self.Ur_cols.T
        return P

    # -- deflated inner operator  J_bar = J~ - Q S_k Q^T  (§3.2) ------------------
    def apply_Jbar(self, V, sign=1.0):
        out = self.Jt @ V
        if self.k:
            out = out - self.Q @ (self.Sk @ (self.Q.T @ V))
        return sign * out

    def _smw(self, transpose):
        if transpose not in self._X:
            sign = -1.0 if transpose else 1.0
            m = self.Ub.shape[1]
            if m:
                X, _, _, _ = mrs(1.0, lambda V: self.apply_Jbar(V, sign), self.Ub,
                                 self.inner_maxit, self.setup_tol, freeze=True)
            else:
                X = np.zeros((self.n, 0))
            SigT = self.Sig.T if transpose else self.Sig
            K = np.eye(m) + self.Ub.T @ X @ SigT
            self._X[transpose] = X
            self._K[transpose] = (sla.lu_factor(K) if m else None, SigT)
        return self._X[transpose], self._K[transpose]

    def apply_prec_inv(self, u, transpose=False):
        """P^-1 u = z - X Sig (I + U^T X Sig)^-1 U^T z,  z = S_bar^-1 u  (Eq. smw, R8).
        transpose=True applies P^-T with S_bar^T = I - J_bar and Sig^T."""
        X, (lu, SigT) = self._smw(transpose)
        sign = -1.0 if transpose else 1.0
        z, its, _, _ = mrs(1.0, lambda V: self.apply_Jbar(V, sign), u,
                           self.inner_maxit, self.inner_tol, freeze=True)
        self.inner_its.append(int(its))
        if X.shape[1] == 0:
            return z
        wv = self.Ub.T @ z
        return z - X @ (SigT @ sla.lu_solve(lu, wv))

    def apply_op(self, v, transpose=False):
        """A_cal v = W Abar S W v, or A_cal^T v = W S^T Abar^T W v (with the incomplete
        factor: F Abar S G v, or F S^T Abar^T G v)."""
        f = self.fac
        if f is not None:
            if transpose:
                return f.F(self.Sw.T @ (self.Aw.T @ f.G(v)))
            return f.F(self.Aw @ (self.Sw @ f.G(v)))
        if transpose:
            return self.Sw.T @ (self.Aw.T @ v)
        return self.Aw @ (self.Sw @ v)

    # -- §4.1 outer solve ---------------------------------------------------------
    def _refine(self, rhs, apply_orig, to_scaled, from_scaled, transpose, tol, maxit,
                outer, restart, stagnation_cycles=5):
        n = self.n
        x = np.zeros(n)
        bnorm = np.linalg.norm(rhs)
        st = {"outer_its": 0, "cycles": 0, "status": "ok", "relres": 0.0,
              "precond_apps": 0}
        self.inner_its = []
        if bnorm == 0.0:
            return x, st
        r = rhs.copy()
        best = np.inf
        stall = 0
        while True:
            rn = np.linalg.norm(r)
            st["relres"] = rn / bnorm
            if rn / bnorm <= tol:
                break
            if st["outer_its"] >= maxit:
                st["status"] = "not_converged"
                break
            if rn < 0.999 * best:
                best = rn
                stall = 0
            else:
                stall += 1
                if stall >= stagnation_cycles:
                    st["status"] = "stagnation"
                    break
            rh = to_scaled(r)
            eta = min(0.5, 0.5 * tol * bnorm / rn)
            op = lambda v: self.apply_op(v, transpose)
            pc = lambda u: self.apply_prec_inv(u, transpose)
            budget = maxit - st["outer_its"]
            if outer == "tfqmr":
                dy, steps, napp = tfqmr_cycle(op, pc, rh, eta, budget)
            else:
                dy, steps, napp = fgmres_cycle(op, pc, rh, eta, min(restart, budget))
            st["outer_its"] += steps
            st["precond_apps"] += napp
            st["cycles"] += 1
            x = x + from_scaled(dy)
            r = rhs - apply_orig(x)
        inn = self.inner_its
        st["inner_its_total"] = int(np.sum(inn)) if inn else 0
        st["inner_its_avg"] = float(np.mean(inn)) if inn else 0.0
        return x, st

    def solve(self, b, tol=1e-8, maxit=2000, outer="tfqmr", restart=60):
        """x with ||b - A x|| <= tol ||b|| (§4.1)."""
        b = np.asarray(b, dtype=np.float64)
        A = self.A

        f = self.fac

        def to_scaled(r):          # W P D_r r  (F P D_r r)
            t = self.w * (self.dr * r)[self.perm]
            return f.F(t) if f is not None else t

        def from_scaled(dy):       # D_c S W dy  (D_c S G dy)
            return self.dc * (self.S @ (f.G(dy) if f is not None else self.w * dy))

        return self._refine(b, lambda x: A @ x, to_scaled, from_scaled, False, tol,
                            maxit, outer, restart)

    def solve_adjoint(self, g, x=None, tol=1e-8, maxit=2000, outer="tfqmr", restart=60):
        """lambda with A^T lambda = g, via A_cal^T mu = W S^T D_c g, lambda = D_r P^T W mu,
        preconditioned by P^T = M~_r + I - J~ (mrs on the transposed inner system).
        With x given, also dL/dA_ij = -lambda_i x_j on the pattern of A."""
        g = np.asarray(g, dtype=np.float64)
        A = self.A
        AT = A.T.tocsr()
        n = self.n

        f = self.fac

        def to_scaled(r):          # W S^T D_c r  (F S^T D_c r)
            t = self.w * (self.S.T @ (self.dc * r))
            return f.F(t) if f is not None else t

        def from_scaled(dmu):      # D_r P^T W dmu  (D_r P^T G dmu)
            t = np.zeros(n)
            t[self.perm] = f.G(dmu) if f is not None else self.w * dmu
            return self.dr * t

        lam, st = self._refine(g, lambda v: AT @ v, to_scaled, from_scaled, True, tol,
                               maxit, outer, restart)
        dA = None
        if x is not None:
            rows = np.repeat(np.arange(n), np.diff(A.indptr))
            dA = -lam[rows] * x[A.indices]
        return lam, dA, st
