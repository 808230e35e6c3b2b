/*
 * asss.h - C ABI of a GB300 (sm_103a) implementation of the two-level iterative
 * scheme for general sparse A x = b based on approximate shifted skew-symmetrizers
 * (Manguoglu & Mehrmann, arXiv 2009.06954).
 *
 * The scheme (paper §2-§4.1):
 *   Abar = P D_r A D_c                                   (§2, Eq. mc64)
 *   S    = argmin ||B_u s||^2 + gamma ||B_l s - 1||^2     (§2, Eqs. eq1, eq2, regularized; App. A)
 *   d = diag(Abar S), W = |d|^-1/2, M~_r = sign(d) - I  (§3, Eq. absfac, Fig. 1; 1x1 pivots)
 *   J~ = W (Abar S - (Abar S)^T)/2 W                      (§3, Eq. preconditioner)
 *   Q_k, S_k from k steps of skew-Lanczos on J~          (§3.2, Fig. 2)
 *   P = [Q_k U_r] blkdiag(S_k, -2I) [Q_k U_r]^T + (I + J~ - Q_k S_k Q_k^T)   (§3.2, Eq. preconditioner)
 *   outer Krylov on  W Abar S W y = W P D_r b,  x = D_c S W y                (§3 Eq. modified, §4.1)
 *   P^-1 by SMW (Eq. smw) around inner mrs solves of the deflated shifted skew
 *   system (§3.1, App. B).
 *
 * Conventions shared by every entry point:
 *  - Pointers may be host or device memory; the library inspects each pointer
 *    (cudaPointerGetAttributes) and copies host data in and out itself.
 *  - Dense vectors are float64.  Multi-vector arguments are column-major with a
 *    leading dimension (ld >= n).
 *  - CSR matrices are 0-based, square, column indices sorted and unique within a
 *    row, every index in range; violations return ASSS_ERR_PATTERN.  nnz must be
 *    below 2^31.
 *  - The caller owns every buffer it passes; the library never keeps a caller
 *    pointer after a call returns.  asss_setup copies A into memory owned by the
 *    handle; asss_destroy frees it.
 *  - All device work is enqueued on options.stream (a cudaStream_t, NULL = the
 *    legacy default stream); each call synchronises that stream before it returns.
 *  - Errors are reported by return code, never by abort/exit.  asss_last_error()
 *    returns a human-readable message for the last failing call of this thread.
 *  - Device-side waits (grid barriers of the persistent kernels) give up after
 *    options.wait_timeout_ms and the call returns ASSS_ERR_TIMEOUT.
 */
#ifndef ASSS_H
#define ASSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ASSS_OK = 0,
    ASSS_ERR_ARG = 1,            /* invalid argument or option                        */
    ASSS_ERR_PATTERN = 2,        /* malformed CSR (unsorted, duplicate, out of range) */
    ASSS_ERR_ZERO_DIAG = 3,      /* |d_i| < zero_tol * max|d|: zero pivot (§4.1 Table 4 legend) */
    ASSS_ERR_BREAKDOWN = 4,      /* Krylov breakdown that prevented any progress      */
    ASSS_ERR_NOT_CONVERGED = 5,  /* iteration limit reached; outputs hold the best iterate */
    ASSS_ERR_STAGNATION = 6,     /* outer residual stopped decreasing                  */
    ASSS_ERR_RANK = 7,           /* rank of M~_r above r_max (Eq. preconditioner2 used) - informational */
    ASSS_ERR_TIMEOUT = 8,        /* a device-side wait exceeded wait_timeout_ms        */
    ASSS_ERR_OOM = 9,            /* device allocation failed                           */
    ASSS_ERR_CUDA = 10,          /* any other CUDA error                               */
    ASSS_ERR_UNSUPPORTED = 11    /* input beyond what this build handles (text says which) */
} asss_status;

enum { ASSS_PREC_FP64 = 0, ASSS_PREC_MIXED = 1 };      /* inner solve in FP64 or FP32 */
enum { ASSS_OUTER_TFQMR = 0, ASSS_OUTER_FGMRES = 1 };  /* §4.1: tfqmr; flexible GMRES for inexact inner solves */

/* Square sparse matrix in CSR. val may be NULL where only a pattern is needed. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr;   /* n+1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
    const int32_t* col_idx;   /* nnz entries */
    const double*  val;       /* nnz entries or NULL */
} asss_csr;

typedef struct {
    double gamma;             /* weight of the diagonal constraints, Eq. regularized (paper: 1) */
    int    k_lanczos;         /* number of skew-Lanczos vectors k (§4.3: 20)                     */
    int    reorth;            /* 1: two classical Gram-Schmidt passes per Lanczos step; 0: Fig. 2 as printed */
    const asss_csr* s_pattern;/* sparsity of S (values ignored); NULL: the pattern of A (§2)     */
    const int32_t* row_perm;  /* optional row permutation P of Eq. mc64: row i of Abar is row row_perm[i] of D_r A D_c */
    const double*  dr;        /* optional row scaling D_r (n); NULL: 1/row-max|a|               */
    const double*  dc;        /* optional column scaling D_c (n); NULL: 1/col-max|D_r a|        */
    double inner_tol;         /* mrs stopping tolerance on |g|/||rhs|| (App. B)                  */
    double setup_tol;         /* tolerance of the multi-RHS mrs solve S_bar X = U_bar (§4.1); <= 0: inner_tol */
    double outer_tol;         /* ||b - A x|| <= outer_tol ||b||                                  */
    int    inner_maxit;       /* mrs iteration limit                                            */
    int    outer_maxit;       /* total outer Krylov steps (§4.1: 2000)                          */
    int    restart;           /* flexible GMRES restart length                                  */
    int    precision;         /* ASSS_PREC_FP64 or ASSS_PREC_MIXED (inner FP32, outer FP64)      */
    int    outer;             /* ASSS_OUTER_TFQMR or ASSS_OUTER_FGMRES                           */
    int    r_max;             /* largest rank r of M~_r kept; above it Eq. (preconditioner2)   */
    uint64_t seed;            /* splitmix64 seed of the Lanczos start vector                    */
    double lls_tol;           /* normal-equation gradient tolerance of the LLS solve            */
    int    lls_maxit;
    double zero_tol;          /* |d_i| < zero_tol*max|d| is a zero pivot                        */
    double wait_timeout_ms;   /* budget of each device-side wait                                */
    void*  stream;            /* cudaStream_t                                                   */
    int    inner_format;      /* storage of J~ for mrs: ASSS_FORMAT_AUTO (skew diagonals when J~ has
                                 at most 64 positive offsets filling >= 50% of them, else SELL-C),
                                 ASSS_FORMAT_SELL, ASSS_FORMAT_DIAG (fails with UNSUPPORTED if J~
                                 does not qualify)                                              */
    int    q_bf16;            /* mixed precision only: round the Lanczos basis Q_k to BF16 values
                                 and use those rounded values everywhere (set-up SMW data and the
                                 FP32 inner solve, which then reads Q_k in BF16); P is unchanged,
                                 the deflation slightly less sharp                              */
    const double* s_values;   /* optional (host or device): values of S on s_pattern, in its CSR order,
                                 e.g. from asss_export of an earlier set-up of the same matrix and
                                 options. The least-squares fit of §2 starts from them and stops at
                                 once when they already meet lls_tol, so a saved S resumes a set-up
                                 without refitting; NULL: start from S = 0                       */
    int    scaling;           /* how Eq. mc64's P, D_r, D_c are found when row_perm, dr and dc are
                                 all NULL: ASSS_SCALING_MAXES (identity P, row then column maxima)
                                 or ASSS_SCALING_MATCHING (maximum-product matching and its dual
                                 scalings, the role of MC64 in §2: |diag| = 1, other entries
                                 <= 1 up to a relative 1e-12 * max(1, max cost))                */
    int    rhs_block;         /* 1: asss_solve with several right-hand sides (FGMRES, k <= 32, FP32 Q)
                                 runs them in lockstep blocks of up to 8 whose preconditioner
                                 applications are one multi-column mrs launch per Arnoldi step
                                 (App. B's simultaneous iterations); 0: one column after another */
    int    sell_sigma;        /* J~ in SELL-C (general patterns): rows are sorted by length within
                                 windows of sell_sigma rows when natural-order slices would pad the
                                 storage by more than a fifth; a power of two in [1024, 16384], or
                                 0: picked at set-up by timing mrs steps (mixed precision, n >=
                                 10^5), else 4096. Other values: ASSS_ERR_ARG                   */
    int    sell_split;        /* entries per lane in one SELL-C work unit: wider slices are cut
                                 into parts taken by different warps; >= 64, or 0 (picked with
                                 sell_sigma, else 1024). Both only change summation order      */
    int    factor;            /* the factor L~ of M^ = (A^ + A^T)/2 (§3 after Eq. absfac):
                                 ASSS_FACTOR_DIAG: 1x1 pivots without fill, L~ = |diag(A^)|^1/2;
                                 ASSS_FACTOR_ILDL0: the no-fill incomplete L D L^T (§4.1's
                                 ~ildl(0); 1x1 pivots, factored in a multicolour order from
                                 Jones-Plassmann rounds seeded by `seed`), J~ = L~^-1 J^ L~^-T
                                 applied by triangular solves (one parallel step per colour).
                                 ASSS_FACTOR_ILDL0_BK: the same with 2x2 pivot blocks where the
                                 first Bunch-Kaufman test |m_ii| >= alpha max_j |m_ij| (alpha =
                                 (1 + 17^1/2)/8) fails for a row and for the column of that
                                 maximum, which points back (a static pairing made before the
                                 ordering; the pattern is closed so that every block between two
                                 pivots is full, pairs are coloured as one vertex); |D|^-1/2 and
                                 M~_r = sign(D) - I are taken block by block (Fig. 1: a 2x2 block
                                 with one negative eigenvalue adds its eigenvector to U_r).
                                 Not with q_bf16 (ASSS_ERR_UNSUPPORTED) nor in asss_setup_batched;
                                 rhs_block is ignored                                           */
} asss_options;

enum { ASSS_SCALING_MAXES = 0, ASSS_SCALING_MATCHING = 1 };

enum { ASSS_FORMAT_AUTO = 0, ASSS_FORMAT_SELL = 1, ASSS_FORMAT_DIAG = 2 };

enum { ASSS_FACTOR_DIAG = 0, ASSS_FACTOR_ILDL0 = 1, ASSS_FACTOR_ILDL0_BK = 2 };

typedef struct {
    int    status;            /* asss_status of the call                                        */
    int    outer_its;         /* outer Krylov steps (TFQMR: full steps; FGMRES: Arnoldi steps)   */
    int    cycles;            /* refinement cycles (true-residual restarts)                     */
    long long inner_its_total;/* mrs iterations over all inner solves                           */
    int    inner_solves;      /* number of inner solves (preconditioner applications)           */
    double inner_its_avg;
    double relres;            /* final ||b - A x|| / ||b|| in FP64 (original system)            */
    int    r;                 /* rank of M~_r (negative d_i kept; with 2x2 pivots, the negative
                                 eigenvalues of the pivot blocks)                               */
    int    k_eff;             /* Lanczos vectors kept after breakdown checks                    */
    int    prec2;             /* 1 if Eq. (preconditioner2) was used because r > r_max          */
    int    lls_its;           /* iterations of the LLS solve                                    */
    double lls_relgrad;       /* final ||B^T (v - B s)|| / ||B^T v||                            */
    long long nnz_pattern;    /* entries of pat(Abar S) + pat(Abar S)^T (LLS rows + mirror)      */
    double t_setup_ms;
    double t_solve_ms;
    double t_inner_ms;        /* device time of the mrs kernel launches (CUDA events on the stream) */
    long long inner_bytes;    /* algorithmic bytes those launches move (matrix entries, Q_k rows, vectors) */
    int    inner_launches;    /* mrs kernel launches counted in t_inner_ms / inner_bytes */
    int    sell_sigma;        /* set-up, J~ in SELL-C: sorting window in rows (0: natural order) */
    int    sell_split;        /* set-up, J~ in SELL-C: entries per lane of one work unit; both picked
                                 by timing mrs steps for systems of 10^5 rows and more (FP32 path) */
    int    factor_colours;    /* set-up, ASSS_FACTOR_ILDL0: colours of the factorization order  */
    double t_op_ms;           /* solve: CUDA-event time of the outer operator applications      */
    int    op_calls;
    long long op_bytes;       /* their algorithmic bytes (stored values, x and y per product)   */
    long long op_flops;       /* and FP64 flops (one FMA per stored value)                      */
    double t_orth_ms;         /* solve: CUDA-event time of the fused Arnoldi steps (FGMRES)     */
    int    orth_calls;
    long long orth_bytes;     /* their algorithmic bytes (basis read twice, w r/w, v_{j+1} out) */
    long long orth_flops;     /* and FP64 flops (4(j+1) FMAs a row)                             */
    int    factor_pairs;      /* set-up, ASSS_FACTOR_ILDL0_BK: 2x2 pivot blocks formed          */
} asss_stats;

typedef struct asss_handle asss_handle;

/* Fill *opt with the defaults: gamma 1, k 20, reorth 1, S on the pattern of A,
 * identity permutation with computed scalings, inner_tol 1e-10, outer_tol 1e-8,
 * inner_maxit 1000, outer_maxit 2000, restart 60, FP64, TFQMR, r_max 256,
 * lls_tol 1e-13, lls_maxit 20000, zero_tol 1e-14, wait_timeout_ms 2000. */
void asss_default_options(asss_options* opt);

/* Set-up phase (§4.1, everything that does not depend on b): scaling, S, d/W/r,
 * J~, skew-Lanczos, the SMW data for P^-1.  A is copied; *out receives a new
 * handle (NULL on error).  st may be NULL. */
asss_status asss_setup(const asss_csr* A, const asss_options* opt, asss_handle** out,
                       asss_stats* st);

/* Solve A x_j = b_j for nrhs right-hand sides (column-major, leading dimensions
 * ldb, ldx >= n) with the handle's options (§4.1).  On NOT_CONVERGED/STAGNATION x
 * holds the last iterate.  st (may be NULL) receives the statistics of the last
 * column. */
asss_status asss_solve(asss_handle* h, int nrhs, const double* b, int64_t ldb,
                       double* x, int64_t ldx, asss_stats* st);

/* Adjoint solve A^T lambda_j = g_j (the transposed system two-sidedly
 * preconditioned with P^T = M~_r + I - J~, inner mrs on the transposed deflated
 * system).  If x and dA are non-NULL, also dA[e] = -lambda_i x_j for every
 * nonzero e = (i, j) of A (the gradient of a loss L with dL/dx = g with respect to
 * A's values, on A's pattern); dA then has nnz(A) entries per right-hand side,
 * column-major with leading dimension nnz(A). */
asss_status asss_solve_adjoint(asss_handle* h, int nrhs, const double* g, int64_t ldg,
                               double* lambda, int64_t ldl, const double* x, int64_t ldx,
                               double* dA, asss_stats* st);

/* Apply the outer operator A_cal v = W Abar S W v (transpose=0) or its transpose
 * (transpose=1) to one vector of length n (§3 Eq. modified). */
asss_status asss_apply_operator(asss_handle* h, int transpose, const double* v, double* out);

/* Apply the preconditioner inverse P^-1 u (Eq. smw) or P^-T u, including one
 * inner mrs solve; st->inner_its_total receives its iteration count. */
asss_status asss_apply_preconditioner(asss_handle* h, int transpose, const double* u,
                                      double* out, asss_stats* st);

/* Copy set-up results out (any pointer may be NULL to skip it):
 *  dr, dc, w, d: n values each; s_val: nnz(S) values of S on its pattern (CSR
 *  order of the pattern); q: n x k_eff column-major Lanczos vectors; alpha: k_eff-1
 *  values; neg: r indices.  k_eff and r are in asss_stats of the setup call. */
asss_status asss_export(asss_handle* h, double* dr, double* dc, double* w, double* d,
                        double* s_val, double* q, double* alpha, int32_t* neg);

/* The row permutation of Eq. mc64 used by the handle: row i of Abar is row
 * row_perm[i] of D_r A D_c (n entries; the identity unless given or matched). */
asss_status asss_export_permutation(asss_handle* h, int32_t* row_perm);

/* The incomplete factor of a handle set up with ASSS_FACTOR_ILDL0 (host or device
 * pointers, each may be NULL): colour (n) of every row in the factorization order,
 * and L, strictly lower in that order, in the original indexing as CSR: l_row_ptr
 * (n+1), l_col / l_val (l_cap >= the entry count, which *l_nnz receives; the columns
 * of a row ascend).  (I + L) D (I + L)^T equals M^ on M^'s pattern; D is the `d` of
 * asss_export (which exports w = 1 for such a handle).  ASSS_ERR_ARG without a
 * factor or with l_cap too small. */
asss_status asss_export_factor(asss_handle* h, int32_t* colour, int64_t* l_row_ptr, int32_t* l_col, double* l_val,
                               int64_t l_cap, int64_t* l_nnz);

/* The 2x2 pivots of a handle set up with ASSS_FACTOR_ILDL0_BK (§3 Eq. absfac with
 * Bunch-Kaufman blocks, Fig. 1; host or device pointers, each may be NULL):
 * partner (n; -1 for a 1x1 pivot), d_off (n; D_{i,partner(i)}, 0 for a 1x1 pivot;
 * the diagonal of D is asss_export's d), and the r columns of U_r (r from the
 * set-up statistics) - column a holds ur_c1[a] at row ur_i1[a] and ur_c2[a] at row
 * ur_i2[a] (ur_i2[a] = -1: a unit column), M~_r = -2 U_r U_r^T.  L of
 * asss_export_factor is then block-lower: (I + L) D (I + L)^T equals M^ on the block
 * closure of M^'s pattern.  *npairs receives the number of 2x2 blocks (0: the factor
 * has 1x1 pivots only, and the other outputs are left untouched).  ASSS_ERR_ARG
 * without an incomplete factor. */
asss_status asss_export_pivots(asss_handle* h, int32_t* partner, double* d_off, int32_t* ur_i1, int32_t* ur_i2,
                               double* ur_c1, double* ur_c2, int* npairs);

void asss_destroy(asss_handle* h);

/* ------------------------------------------------------------------------
 * Batched solves: many matrices of uneven size, each with its own set-up, and
 * many right-hand sides, solved by one persistent launch (§4.1 solve phase per
 * system: refinement on the FP64 residual, flexible GMRES outer, P^-1 by
 * Eq. smw around FP32 mrs, App. B).  Each CTA takes (matrix, right-hand side)
 * items from a global counter, largest matrices first, and runs the whole solve
 * of one item in block scope.  The launch is captured once into a CUDA graph
 * and replayed while b, x and nrhs stay the same.
 * ------------------------------------------------------------------------ */
typedef struct asss_batch asss_batch;

/* Set up nmat systems A[0..nmat) with one option set.  Forces the mixed-precision
 * path, flexible GMRES and skew-diagonal storage of J~ (UNSUPPORTED if a J~ does
 * not fit it, if the matrices end with different Lanczos widths, or if k > 32,
 * k + r > 320 or J~ has more than 64 diagonals).  The restart length is
 * min(opt->restart, 24).  Device scratch: (6 + 2 restart) FP64 and about 6 FP32
 * vectors of the largest system per resident CTA.  st (may be NULL): t_setup_ms
 * and k_eff of matrix 0. */
asss_status asss_setup_batched(int nmat, const asss_csr* const* A, const asss_options* opt,
                               asss_batch** out, asss_stats* st);

/* Solve every system for nrhs right-hand sides.  b and x (host or device) hold
 * the systems one after the other: system m occupies entries
 * [off_m * nrhs, (off_m + n_m) * nrhs) with off_m = n_0 + ... + n_{m-1}, column-major
 * n_m x nrhs inside.  x is overwritten.  st (may be NULL): outer_its = the largest
 * over items, inner_its_total and cycles summed, relres = the largest, inner_solves
 * = number of items, t_inner_ms = device time of the batched launch, inner_bytes =
 * the algorithmic bytes of the inner mrs steps (each column's vectors, plus J~ and
 * Q of its matrix divided among the nrhs columns that share them).  Returns the
 * first non-OK item status (x then holds every item's last iterate).  The first
 * call for a given nrhs tunes the CTA shape: it solves the batch once with each of
 * six shapes - 256 and 512 threads per CTA at 64 registers a thread, 256 and 384
 * threads at 80, 256 and 512 threads at 128 (as many CTAs per SM as fit, at most one
 * CTA per item) - and keeps the fastest for later calls; that call takes about seven
 * times as long. */
asss_status asss_solve_batched(asss_batch* b, int nrhs, const double* rhs, double* x,
                               asss_stats* st);

/* CTA size chosen by the tuner (0 before the first solve). */
int asss_batch_cta_threads(const asss_batch* b);

/* Registers a thread of the CTA shape chosen by the tuner (64, 80 or 128; 0 before
 * the first solve). */
int asss_batch_cta_registers(const asss_batch* b);

void asss_destroy_batched(asss_batch* b);

const char* asss_status_str(asss_status s);
const char* asss_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all handles); a monotone counter for accounting. */
unsigned long long asss_kernel_launches(void);

/* ------------------------------------------------------------------------
 * Single steps of the path, each callable on its own.
 * ------------------------------------------------------------------------ */

/* The least-squares fit of §2 (Eq. regularized, App. A) for S on s_pattern given
 * an already scaled matrix Abar.  s_val receives nnz(s_pattern) values in the
 * pattern's CSR order.  Uses gamma, lls_tol, lls_maxit and stream from opt. */
asss_status asss_skew_symmetrizer(const asss_csr* Abar, const asss_csr* s_pattern,
                                  const asss_options* opt, double* s_val, asss_stats* st);

/* Maximum-product matching and scaling of a square A (§2, Eq. mc64, the role MC64
 * plays in the paper): costs c_ij = log(max_k |a_kj|) - log|a_ij| on A's nonzeros, a
 * perfect matching of minimum total cost (maximum product of matched |a_ij|) by an
 * auction algorithm with epsilon-scaling down to eps = 1e-12 * max(1, max c), within
 * n * eps of the optimum, and scalings from its dual variables.  row_perm (n), dr (n),
 * dc (n), host or device, receive P, D_r, D_c with row i of P D_r A D_c equal to row
 * row_perm[i] of D_r A D_c, |diagonal| = 1 and every other entry <= exp(eps) in modulus.  Explicit
 * zeros of A are not matched.  ASSS_ERR_PATTERN when A has no perfect matching
 * (structurally singular) or an empty column.  *rounds (may be NULL): auction rounds. */
asss_status asss_matching_scaling(const asss_csr* A, int32_t* row_perm, double* dr, double* dc, int* rounds,
                                  void* stream);

/* k steps of skew-Lanczos (§3.2, Fig. 2) on the skew matrix J (values used as
 * given) from start vector q1 (n values, need not be normalised).  q receives
 * n x k_eff column-major vectors, alpha k_eff-1 values, *k_eff the number kept.
 * reorth as in asss_options. */
asss_status asss_skew_lanczos(const asss_csr* J, const double* q1, int k, int reorth,
                              double* q, double* alpha, int* k_eff, void* stream);

/* mrs (§3.1, App. B) on (shift I + sign*(J - Q S_k Q^T)) x = b for one right-hand
 * side, where J is skew (not checked), Q is n x k column-major (k may be 0) and
 * S_k the skew tridiagonal matrix with superdiagonal alpha (k-1 values).
 * precision selects FP64 or FP32 storage and arithmetic (the FP32 solve sums in FP32
 * within a warp and in float pairs, about 44 bits, across warps and blocks); format
 * selects the storage of J as in asss_options.inner_format (the skew-diagonal
 * storage also requires J to be exactly skew, J_ij == -J_ji bit for bit).
 * Stops when |g|/||b|| < tol or after maxit steps; *its and *ratio receive the
 * step count and the final recursive residual ratio. */
asss_status asss_mrs(const asss_csr* J, int k, const double* q, const double* alpha,
                     double shift, double sign, const double* b, double* x, double tol,
                     int maxit, int precision, int format, int* its, double* ratio, void* stream);

/* mrs for nrhs right-hand sides at once: App. B's simultaneous iterations on
 * (shift I + sign*(J - Q S_k Q^T)) X = B, B and X n x nrhs column-major with leading
 * dimensions ldb, ldx >= n (host or device).  Every column runs its own recurrence
 * and freezes once its |g|/||b_j|| < tol (the result equals nrhs separate asss_mrs
 * calls); the columns share each pass over J and Q (up to 8 columns per launch, the
 * SpMM form of the product).  k at most 32.  its and ratio (may be NULL) receive
 * nrhs values each.  Other arguments as for asss_mrs. */
asss_status asss_mrs_multi(const asss_csr* J, int k, const double* q, const double* alpha, double shift,
                           double sign, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                           int maxit, int precision, int format, int* its, double* ratio, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free variant of asss_mrs.
 *
 * For callers that must not allocate device memory during a call: code that runs
 * inside a memory-capped service with a fixed device budget, or under an
 * allocator whose pool must not grow while a request is served.  The paper has
 * no counterpart; it is an interface convenience of this library.
 *
 * Same method and stopping rule as asss_mrs with precision FP64, on J given as
 * plain CSR that is read in place (every array - row_ptr, col_idx, val, q, alpha,
 * b, x - must already be memory of the current device (or managed memory);
 * nothing is copied).  Each array must be aligned to its element size, and q to
 * 16 bytes: other pointers are rejected with ASSS_ERR_ARG before any launch.  q is
 * the deflation basis in ROW-major layout with leading dimension kp (kp one of 0, 4,
 * 8, 12, 16, 20, 24, 32, 48, 64, kp >= k); its columns k..kp-1 must be zero
 * (checked: ASSS_ERR_ARG otherwise).  sign must be +1 or -1.  Scratch comes from one
 * static device array of the library (about 3.2 MB per device, held by every GPU
 * that loads the library until the process exits), so n must be at most 65536;
 * larger n returns ASSS_ERR_ARG.  The call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *
 * The first call on a device looks up the device address of that array (once per
 * device, with the device current); make that first call before any stream
 * capture.  The address is cached for the life of the process: after a
 * cudaDeviceReset (or any teardown of the device's primary context) this entry
 * point must not be called again in that process.  All calls share the array and
 * it keeps the last call's contents:
 * calls that overlap on the GPU (different streams, threads or processes sharing
 * a context) race and must not be issued.  The call synchronises the stream
 * before returning.  The CSR is checked (row pointers, then column indices) and
 * ASSS_ERR_PATTERN is returned if it is malformed.
 */
asss_status asss_mrs_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                             const double* val, int k, int kp, const double* q_rowmajor,
                             const double* alpha, double shift, double sign, const double* b,
                             double* x, double tol, int maxit, int* its, double* ratio,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ASSS_H */
