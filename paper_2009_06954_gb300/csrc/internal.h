// Internal host-side interfaces shared by the library's translation units.
#pragma once

#include <vector>

#include "common.cuh"

namespace asss {

// sparse.cu
asss_status upload_csr(const asss_csr* A, DCsr& out, bool need_values, cudaStream_t s);
asss_status copy_csr(const DCsr& a, DCsr& out, cudaStream_t s);
asss_status transpose_csr(const DCsr& a, DCsr& t, DBuf<int>* srcpos, cudaStream_t s);
asss_status spmv(const DCsr& A, const double* x, double* y, const double* lscale, cudaStream_t s);
// attach a diagonal copy (DDia) when A's entries lie on at most max_diag diagonals
// that are at least min_fill full; *ok tells whether it was attached
asss_status attach_dia(DCsr& A, int max_diag, double min_fill, int* ok, cudaStream_t s);
asss_status build_pattern(const DCsr& Abar, const DCsr& AbarT, const DCsr& S, const DCsr& ST, DCsr& P,
                          DBuf<int>& mirror, DBuf<int>& diagpos, cudaStream_t s);
template <class T>
asss_status build_sell(const DCsr& A, bool skip_diag, DSell<T>& out, cudaStream_t s, int sigma = 0, int split = 0);
// Skew half-diagonal storage of J when J is exactly skew, has at most max_diag
// positive offsets and fills at least min_fill of the stored diagonals; *ok = 0
// (and nothing allocated) otherwise.
template <class T>
asss_status build_skew_dia(const DCsr& J, int max_diag, double min_fill, DSkewDia<T>& out, int* ok,
                           cudaStream_t s);

// dense.cu : small dense / tall-skinny / vector kernels (all FP64 unless noted)
asss_status splitmix64_fill(uint64_t seed, int n, double* out, cudaStream_t s);
// G (p x q, row-major) = A^T B with A n x p (col-major, lda) and B n x q (col-major, ldb)
asss_status gram(const double* A, int lda, int p, const double* B, int ldb, int q, int n, double* G,
                 cudaStream_t s);
// out = z - Y w, Y n x m row-major; w on device (m)
asss_status sub_rowmajor_gemv(const double* Y, int m, const double* w, const double* z, int n, double* out,
                              cudaStream_t s, const int* skip = nullptr);
// out (n) = A (n x p col-major) c  (+ beta*out)
asss_status colmajor_gemv(const double* A, int lda, int p, const double* c, int n, double beta, double* out,
                          cudaStream_t s);
// in-place inverse of an m x m row-major matrix (Gauss-Jordan, partial pivoting)
asss_status small_inverse(double* K, int m, int* singular, cudaStream_t s);
// col-major n x p -> row-major n x kp (zero padded), in double or float
asss_status to_rowmajor(const double* A, int lda, int p, int n, int kp, double* out, cudaStream_t s);
asss_status to_rowmajor_f(const double* A, int lda, int p, int n, int kp, float* out, cudaStream_t s);

// vector helpers (device scalars where noted)
asss_status vscale(double* y, const double* x, double a, int n, cudaStream_t s);                 // y = a x
asss_status vaxpy(double* y, const double* x, double a, int n, cudaStream_t s);                  // y += a x
asss_status vaxpy_dev(double* y, const double* x, const double* a, double sign, int n, cudaStream_t s);  // y += sign*(*a) x
asss_status vmul(double* y, const double* a, const double* b, int n, cudaStream_t s);            // y = a .* b
asss_status vcopy(double* y, const double* x, int n, cudaStream_t s);
asss_status vfill(double* y, double v, int n, cudaStream_t s);

struct IldlFactor;

// mrs.cu
struct MrsOperator {
    // J~ (exactly skew) in SELL-C, FP64 and/or FP32 copies
    const DSell<double>* J64 = nullptr;
    const DSell<float>* J32 = nullptr;
    // skew half-diagonal copies (used instead of SELL when present)
    const DSkewDia<double>* D64 = nullptr;
    const DSkewDia<float>* D32 = nullptr;
    int k = 0, kp = 0;           // Lanczos vectors and padded row stride
    const double* Q64 = nullptr; // n x kp row-major
    const float* Q32 = nullptr;
    const void* Q16 = nullptr;   // BF16 n x kp16 row-major (FP32 solve only); used instead of Q32 when set
    int kp16 = 0;
    const double* alpha = nullptr;  // device, k-1 values (S_k superdiagonal)
    // factored J~ = L~^-1 J^ L~^-T (incomplete L D L^T); used instead of the storages above
    const IldlFactor* F = nullptr;
};

struct MrsTotals {
    long long its = 0;     // mrs steps summed over the launches
    int launches = 0;
    double ms = 0.0;       // kernel time from CUDA events around each launch
    long long bytes = 0;   // algorithmic bytes of those launches
};

struct MrsWork;  // opaque persistent workspace (owned by a handle)
asss_status mrs_work_create(MrsWork** w, int n, int sms);
void mrs_work_destroy(MrsWork* w);

struct MrsResult {
    int its = 0;
    double ratio = 0.0;
    int status = 0;
    double ms = 0.0;          // kernel time from CUDA events around the launch
    long long bytes = 0;      // algorithmic bytes of the launch
};

unsigned long long launches();

// One single-RHS mrs solve (App. B) of (shift I + sign*(J~ - Q S_k Q^T)) x = rhs.
// fp32: use the FP32 operator and vectors; rhs is FP64 in both cases, x is FP64
// (x64) or FP32 (x32) - exactly one of them non-null.
// qtz (optional, k values): Q^T x of the final iterate, reduced inside the kernel.
// With sync_result false the step count and timing stay on the device until
// mrs_collect; with true they are read back into *res before returning.
asss_status mrs_solve(const Ctx& c, MrsWork* w, const MrsOperator& op, bool fp32, double shift, double sign,
                      const double* rhs, double* x64, float* x32, double tol, int maxit, double* qtz,
                      MrsResult* res, bool sync_result);
// Synchronise the stream, fold every logged launch into the totals and report a
// timed-out device wait.
asss_status mrs_collect(const Ctx& c, MrsWork* w, std::vector<MrsResult>* out);
MrsTotals mrs_take_totals(MrsWork* w);
// launches enqueued while flag is set (non-null) read *flag on the device first and
// do nothing if it is non-zero (speculative work enqueued ahead of a host decision)
void mrs_set_skip(MrsWork* w, const int* flag);
const int* mrs_get_skip(const MrsWork* w);

// mrs_multi.cu: App. B's simultaneous iterations for ncol right-hand sides (B, X
// column-major with leading dimensions ldb, ldx; X in FP64 or FP32 as fp32 says), in
// launches of up to 8 columns that share every pass over J~ and Q_k; per-column
// freezing.  its / ratio: host arrays of ncol entries (may be null).  Supports padded
// Lanczos widths up to MRS_MULTI_KPMAX.
constexpr int MRS_MULTI_KPMAX = 32;
asss_status mrs_multi_solve(const Ctx& c, const MrsOperator& op, bool fp32, double shift, double sign, int ncol,
                            const double* B, long long ldb, double* X64, float* X32, long long ldx, double tol,
                            int maxit, int* its, double* ratio);
// the same with one pointer per column (B[t], X64[t] or X32[t]: n values each)
asss_status mrs_multi_solve_cols(const Ctx& c, const MrsOperator& op, bool fp32, double shift, double sign,
                                 int ncol, const double* const* B, double* const* X64, float* const* X32, double tol,
                                 int maxit, int* its, double* ratio, MrsTotals* tot = nullptr);

// ildl.cu: no-fill incomplete L D L^T of M^ in a multicolour order (§3 after Eq.
// absfac, §4.1 ~ildl(0)); original indexing, "lower" = of a smaller colour.
constexpr int ILDL_MAXCOL = 256;
struct IldlFactor {
    int n = 0, ncol = 0, rounds = 0;
    int64_t nl = 0, nu = 0, nj = 0;
    std::vector<int> hls;            // ncol + 1 level offsets (host)
    DBuf<int> ls;                    // the same on the device
    DBuf<int> colour, lvl;           // colour of each vertex; vertices by (colour, index)
    DBuf<int> lrp, lci, urp, uci;    // L: entries of smaller colour; U: of larger colour
    DBuf<double> lv, uv, wd;         // l_ij; the mirrored l_ji; |D|^-1/2
    DBuf<float> lv32, uv32, wd32, jv32;
    DBuf<double> ft, fw;             // scratch of one application
    DBuf<float> ft32, fw32;
    const int* jrp = nullptr;        // J^ (exactly skew) on the pattern, not owned
    const int* jci = nullptr;
    const double* jv = nullptr;
    // 2x2 pivots (factor ASSS_FACTOR_ILDL0_BK; all empty when no pair was formed):
    // partner of each vertex (-1: 1x1 pivot), the off-diagonal D_{i,partner(i)}, the
    // off-diagonal of |D|^-1/2, and U_r of M~_r = sign(D) - I column by column: entries
    // ur_c1 at ur_i1 and ur_c2 at ur_i2 (ur_i2 = -1 for a unit vector), Sigma_r = -2 I
    int npairs = 0;
    DBuf<int> part;
    DBuf<double> doff, wo;
    DBuf<float> wo32;
    int nur = 0;
    DBuf<int> ur_i1, ur_i2;
    DBuf<double> ur_c1, ur_c2;
};
// P: symmetric pattern of A^ (diagonal included), mirror[e] = position of the transposed
// entry, Cval = A^ on P; d: diag(A^) on entry, the pivots D on return; *nzero: pivots
// below zero_tol * max|diag|
// pivots2: also 2x2 pivot blocks where the first Bunch-Kaufman test asks for them (the
// factor then works on the block closure of P; U_r comes back in F.ur_*)
asss_status ildl_build(const Ctx& c, const DCsr& P, const int* mirror, const double* Cval, double* d,
                       uint64_t seed, double zero_tol, bool fp32, IldlFactor& F, int* nzero,
                       bool pivots2 = false);
asss_status ildl_set_skew(const Ctx& c, IldlFactor& F, const DCsr& Jh, bool fp32);
asss_status ildl_F(const Ctx& c, IldlFactor& F, const double* v, double* out);  // |D|^-1/2 (I + L)^-1 v
asss_status ildl_G(const Ctx& c, IldlFactor& F, const double* v, double* out);  // (I + L)^-T |D|^-1/2 v

// matching.cu: maximum-product matching (auction, epsilon-scaling) and the dual
// scalings of Eq. mc64; perm, dr, dc: device arrays of n entries (row i of Abar is
// row perm[i] of D_r A D_c)
asss_status matching_scaling(const Ctx& c, const DCsr& A, int* perm, double* dr, double* dc, int* rounds,
                             double* eps);

// lls.cu
struct LlsResult {
    int its = 0;
    double relgrad = 0.0;
};
// S values on the pattern of Spat given Abar, AbarT (with values); also returns
// P (symmetric pattern), mirror, diagpos, and C = Abar S on P.
asss_status lls_fit(const Ctx& c, const DCsr& Abar, const DCsr& AbarT, const DCsr& Spat, double gamma,
                    double tol, int maxit, DBuf<double>& s_val, DCsr& P, DBuf<int>& mirror,
                    DBuf<int>& diagpos, DBuf<double>& Cval, LlsResult* res, const double* s0 = nullptr);
// C = Abar S on P for given S values
asss_status lls_product_on_pattern(const Ctx& c, const DCsr& Abar, const DCsr& ST, const int* st_src,
                                   const double* s_val, const DCsr& P, const int* prow, double* Cval);

// batch.cu: one matrix of a batched solve, as device pointers into its handle
struct BatchMat {
    int n;
    int k;           // Lanczos vectors
    int m;           // k + r (SMW rank)
    int r;
    int ndiag;       // skew diagonals of J~
    int halo;        // largest diagonal offset
    long long ustride;
    const int* off;  // ndiag offsets
    const float* U;  // J~ diagonals (FP32), diagonal d at U + d*ustride, entries [-halo, n)
    // J~ in SELL-C-sigma (FP32) when it does not fit the diagonals (ndiag = 0 then)
    int nslots;           // 32 * slices
    const int* sptr;      // slice offsets
    const int* scol;
    const float* sval;
    const int* rowmap;    // slot -> row (n for padding), or null for the identity
    const float* Q32;               // n x kp row-major (or null)
    const void* Q16;                // BF16 n x kp row-major (or null)
    const double* alpha;            // k-1
    const float* Y32;               // SMW data, n x m row-major
    const int* neg;                 // r indices
    const int *arp, *aci;           // A (original) for the residual
    const double* av;
    const int *awrp, *awci;         // W Abar
    const double* awv;
    const int *swrp, *swci;         // S W
    const double* swv;
    const int *srp, *sci;           // S
    const double* sv;
    const double *dr, *dc, *w;
    const int* perm;                // row permutation or null
};

struct BatchItemStat {
    int outer_its;
    int inner_its;
    int status;
    int cycles;
    double relres;
};

struct BatchLaunch {
    const BatchMat* mats;
    const int2* items;          // (matrix, column), largest matrices first
    int nitems;
    int nrhs;
    const long long* row_off;   // first row of each matrix in the concatenated vectors
    const double* b;            // concatenated right-hand sides, matrix m at row_off[m]*nrhs, n_m x nrhs
    double* x;
    double* work;               // per-CTA workspace
    long long work_stride;      // doubles per CTA
    int n_max, halo_max;
    int kp, qbf16;              // common padded Lanczos width and Q storage of the batch
    int restart;
    double outer_tol;
    int outer_maxit;
    double inner_tol;
    int inner_maxit;
    unsigned* next_item;
    BatchItemStat* stats;
    unsigned long long* prof;   // optional (may be null): nanoseconds per phase summed over CTAs
};
constexpr int BATCH_NPROF = 6;  // mrs, SMW correction, operator, Gram-Schmidt, x update + residual, rest

// launches the persistent batched solver on stream s with nthreads per CTA and nblk CTAs,
// built for minb resident CTAs per SM (which sets the registers a thread may use)
asss_status batch_launch(const BatchLaunch& L, int nthreads, int minb, int nblk, cudaStream_t s);
// resident CTAs per SM of the batched solver for a CTA shape
asss_status batch_occupancy(int kp, int qbf16, int nthreads, int minb, int* occ);
constexpr int BATCH_RMAX = 24;

// fused Arnoldi step of FGMRES (arnoldi.cu): CGS2 + norm + Givens + next basis vector
constexpr int AO_MAXV = 64;
struct ArnoldiWork {
    int n = 0, nblk = 0;
    unsigned phase = 0;  // grid barriers completed on bar[0]
    DBuf<double> part;
    DBuf<unsigned> bar;
    DBuf<int> err;
};
// *stop receives 1 when the cycle ends at this step (||w|| = 0 or |g[j+1]| <= thr)
asss_status arnoldi_orth(const Ctx& c, ArnoldiWork& aw, const double* V, double* w, int n, int j, int m, double* H,
                         double* cs, double* sn, double* g, double* hv, double* hv2, double* hn2, double* inv_hn,
                         double thr, int* stop);    // restart length bound of the batched FGMRES
long long batch_work_doubles(int n_max, int halo_max, int restart);

}  // namespace asss
