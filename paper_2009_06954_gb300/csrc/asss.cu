// C ABI of the library: set-up, solve, adjoint and single-step entry points.
// Host code here only orders kernel launches and reads back the scalars that
// decide control flow (convergence, breakdown); all arithmetic runs on the GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

using namespace asss;

namespace asss {

// ---------------------------------------------------------------------------
// small kernels used by the drivers below
// ---------------------------------------------------------------------------
__global__ void k_rowmax_abs(const int* rp, const double* v, int n, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) m = fmax(m, fabs(v[e]));
    out[i] = m;
}
// column max of |dr_i a_ij| via atomicMax on the bit pattern (valid for x >= 0)
__global__ void k_colmax_abs(const int* rp, const int* ci, const double* v, const double* dr, int n,
                             unsigned long long* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        double a = fabs(dr[i] * v[e]);
        atomicMax(&out[ci[e]], (unsigned long long)__double_as_longlong(a));
    }
}
__global__ void k_recip_check(const double* in, int n, double* out, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = in[i];
    if (!(v > 0.0) || !isfinite(v)) {
        atomicOr(bad, 1);
        out[i] = 1.0;
    } else {
        out[i] = 1.0 / v;
    }
}
// Abar row i = dr[perm[i]] * A row perm[i] * dc  (row lengths gathered first)
__global__ void k_perm_rowlen(const int* rp, const int* perm, int n, int* len) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = perm ? perm[i] : i;
    len[i] = rp[r + 1] - rp[r];
}
__global__ void k_perm_scale_rows(const int* rp, const int* ci, const double* v, const int* perm, const double* dr,
                                  const double* dc, int n, const int* orp, int* oci, double* ov) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = perm ? perm[i] : i;
    int o = orp[i];
    double f = dr[r];
    for (int e = rp[r]; e < rp[r + 1]; ++e, ++o) {
        oci[o] = ci[e];
        ov[o] = f * v[e] * dc[ci[e]];
    }
}
__global__ void k_check_perm(const int* perm, int n, int* seen, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = perm[i];
    if (r < 0 || r >= n || atomicAdd(&seen[r], 1) != 0) atomicOr(bad, 1);
}
// d = C on the diagonal of P; W = |d|^-1/2; zero-pivot flag
__global__ void k_diag_w(const double* C, const int* diagpos, int n, double* d, double* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = C[diagpos[i]];
    d[i] = v;
    w[i] = (v != 0.0) ? 1.0 / sqrt(fabs(v)) : 0.0;
}
__global__ void k_absmax(const double* a, int n, unsigned long long* out) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmax(m, fabs(a[i]));
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
__global__ void k_zero_pivots(const double* d, int n, double thr, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && fabs(d[i]) < thr) atomicAdd(cnt, 1);
}
__global__ void k_neg_flag(const double* d, int n, int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = d[i] < 0.0 ? 1 : 0;
}
__global__ void k_neg_compact(const int* flag, const int* pos, int n, int* neg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) neg[pos[i]] = i;
}
// J~ on P: for upper k, v = (C_ij - C_ji)/2 w_i w_j at k and -v at the mirror; 0 on the diagonal
__global__ void k_assemble_jt(int n, const int* prp, const int* pci, const int* mirror, const double* C,
                              const double* w, double* jt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = prp[i]; k < prp[i + 1]; ++k) {
        int j = pci[k];
        if (j == i) {
            jt[k] = 0.0;
        } else if (j > i && mirror[k] >= 0) {
            double v = 0.5 * (C[k] - C[mirror[k]]) * w[i] * w[j];
            jt[k] = v;
            jt[mirror[k]] = -v;
        }
    }
}
__global__ void k_scale_rows(const int* rp, double* v, const double* s, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) v[e] *= s[i];
}
__global__ void k_scale_cols(const int* rp, const int* ci, double* v, const double* s, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) v[e] *= s[ci[e]];
}
__global__ void k_f2d(const float* a, double* b, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}
// round to the nearest BF16 value, kept in FP64 (the rounded basis is used everywhere)
__global__ void k_round_bf16(double* a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (double)__bfloat162float(__double2bfloat16(a[i]));
}
// col-major FP64 n x p -> row-major BF16 n x kp (zero padded)
__global__ void k_to_rowmajor_bf16(const double* A, int lda, int p, int n, int kp, __nv_bfloat16* out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * kp) return;
    int i = (int)(t / kp), a = (int)(t % kp);
    out[t] = __double2bfloat16(a < p ? A[(size_t)a * lda + i] : 0.0);
}
// U_r^T z: column a of U_r is e_{neg[a]}, or (with 2x2 pivots, neg2 != null) c1[a] at
// neg[a] plus c2[a] at neg2[a] (neg2[a] = -1 for a unit column)
struct UrCols {
    const int* neg = nullptr;
    const int* neg2 = nullptr;
    const double* c1 = nullptr;
    const double* c2 = nullptr;
};
template <class T>
__device__ __forceinline__ double ur_dot(const UrCols& U, int a, const T* z) {
    if (!U.neg2) return (double)z[U.neg[a]];
    double v = U.c1[a] * (double)z[U.neg[a]];
    const int j = U.neg2[a];
    if (j >= 0) v += U.c2[a] * (double)z[j];
    return v;
}
__global__ void k_gather_neg_f(const float* z, UrCols U, int r, double* out) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < r) out[a] = ur_dot(U, a, z);
}
__global__ void k_d2f(const double* a, int64_t n, float* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
// out = z - Y w for the mixed-precision path: z and Y in FP32, w and out in FP64
// (w is converted to FP32 once per block: per-row conversions would run on the
// FP64 pipe, which is narrow on this part; rows of Y are read as float4 when m
// is a multiple of 4)
__global__ void k_smw_apply_f32(const float* __restrict__ z, const float* __restrict__ Y, int m,
                                const double* __restrict__ w, int n, double* __restrict__ out, int evict_first,
                                const int* skip) {
    extern __shared__ float sw_f[];
    if (skip && *skip) return;   // the speculative application the outer method did not need
    for (int t = threadIdx.x; t < m; t += blockDim.x) sw_f[t] = (float)w[t];
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = 0.f;
    if (m > 0) {
        const float* row = Y + (size_t)i * m;
        if ((m & 3) == 0) {
            const float4* r4 = reinterpret_cast<const float4*>(row);
            for (int c = 0; c < (m >> 2); ++c) {
                const float4 v = evict_first ? __ldcs(r4 + c) : __ldg(r4 + c);  // Y: read once per application
                a += v.x * sw_f[4 * c] + v.y * sw_f[4 * c + 1] + v.z * sw_f[4 * c + 2] + v.w * sw_f[4 * c + 3];
            }
        } else {
            for (int c = 0; c < m; ++c) a += row[c] * sw_f[c];
        }
    }
    out[i] = (double)(z[i] - a);
}
__global__ void k_gather_neg(const double* z, UrCols U, int r, double* out) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < r) out[a] = ur_dot(U, a, z);
}
// y = column a of U_r
__global__ void k_ur_column(double* y, int n, UrCols U, int a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    if (!U.neg2) {
        v = (i == U.neg[a]) ? 1.0 : 0.0;
    } else {
        if (i == U.neg[a]) v += U.c1[a];
        if (i == U.neg2[a]) v += U.c2[a];
    }
    y[i] = v;
}
// rows k..m-1 of G = U_bar^T X: U_r^T X (rows neg[a] of X, or their combinations)
__global__ void k_gram_neg_rows(const double* X, int n, int m, UrCols U, int k, int r, double* G) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r * m) return;
    int a = t / m, c = t % m;
    G[(size_t)(k + a) * m + c] = ur_dot(U, a, X + (size_t)c * n);
}
// Sig_bar (m x m row-major) = blkdiag(S_k, -2 I_r), transposed if tr
__global__ void k_sigma(const double* alpha, int k, int m, int tr, double* Sig) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * m) return;
    int a = t / m, b = t % m;
    double v = 0.0;
    if (a < k && b < k) {
        if (b == a + 1) v = alpha[a];
        if (a == b + 1) v = -alpha[b];
    } else if (a >= k && a == b) {
        v = -2.0;
    }
    if (tr) {
        // transpose: swap the roles
        double u = 0.0;
        int aa = b, bb = a;
        if (aa < k && bb < k) {
            if (bb == aa + 1) u = alpha[aa];
            if (aa == bb + 1) u = -alpha[bb];
        } else if (aa >= k && aa == bb) {
            u = -2.0;
        }
        v = u;
    }
    Sig[t] = v;
}
// C = (I if add_identity) + A B for m x m row-major matrices (one thread per entry)
__global__ void k_small_mm(const double* A, const double* B, int m, int add_identity, double* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * m) return;
    int a = t / m, c = t % m;
    double acc = (add_identity && a == c) ? 1.0 : 0.0;
    for (int b = 0; b < m; ++b) acc += A[a * m + b] * B[b * m + c];
    C[t] = acc;
}
// Y (n x m row-major) = X (n x m col-major) Z (m x m row-major)
__global__ void k_x_times_small(const double* X, const double* Z, int n, int m, double* Y) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * m) return;
    int i = (int)(t / m), c = (int)(t % m);
    double acc = 0.0;
    for (int b = 0; b < m; ++b) acc += X[(size_t)b * n + i] * Z[b * m + c];
    Y[t] = acc;
}
// w -= V h (V n x p col-major)
__global__ void k_sub_colmajor(const double* V, int ldv, int p, const double* h, int n, double* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int a = 0; a < p; ++a) acc += V[(size_t)a * ldv + i] * h[a];
    w[i] -= acc;
}
__global__ void k_add(double* h, const double* h2, int p) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < p) h[a] += h2[a];
}
// refinement helpers
__global__ void k_to_scaled_fwd(const double* r, const double* dr, const double* w, const int* perm, int n,
                                double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = perm ? perm[i] : i;
    out[i] = w[i] * dr[p] * r[p];
}
__global__ void k_from_scaled_adj(const double* dmu, const double* dr, const double* w, const int* perm, int n,
                                  double* lam) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = perm ? perm[i] : i;
    lam[p] += dr[p] * w[i] * dmu[i];
}
__global__ void k_axpy_mul(double* x, const double* a, const double* b, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += a[i] * b[i];
}
__global__ void k_sub(const double* b, const double* t, double* r, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - t[i];
}
__global__ void k_grad_A(const int* rp, const int* ci, const double* lam, const double* x, int n, double* dA) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double l = lam[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) dA[e] = -l * x[ci[e]];
}

// ---------------------------------------------------------------------------
// TFQMR / FGMRES device scalar kernels
// ---------------------------------------------------------------------------
// scalar slots of TFQMR
enum { TF_TAU = 0, TF_THETA, TF_ETA, TF_RHO, TF_ALPHA, TF_SIGMA, TF_WN2, TF_RHON, TF_BETA, TF_BREAK, TF_NSC };

__global__ void k_tf_init(double* T, const double* rr) {
    T[TF_TAU] = sqrt(*rr);
    T[TF_THETA] = 0.0;
    T[TF_ETA] = 0.0;
    T[TF_RHO] = *rr;
    T[TF_BREAK] = 0.0;
}
__global__ void k_tf_alpha(double* T) {
    double sg = T[TF_SIGMA];
    if (sg == 0.0 || T[TF_RHO] == 0.0) {
        T[TF_BREAK] = 1.0;
        T[TF_ALPHA] = 0.0;
    } else {
        T[TF_ALPHA] = T[TF_RHO] / sg;
    }
}
// w -= alpha Bu ; d = ut + (theta^2 eta / alpha) d
__global__ void k_tf_wd(double* w, const double* Bu, double* d, const double* ut, const double* T, int n) {
    double a = T[TF_ALPHA];
    double coef = (a != 0.0) ? T[TF_THETA] * T[TF_THETA] * T[TF_ETA] / a : 0.0;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    w[i] -= a * Bu[i];
    d[i] = ut[i] + coef * d[i];
}
__global__ void k_tf_theta(double* T) {
    double th = sqrt(T[TF_WN2]) / T[TF_TAU];
    double c = 1.0 / sqrt(1.0 + th * th);
    T[TF_THETA] = th;
    T[TF_TAU] = T[TF_TAU] * th * c;
    T[TF_ETA] = c * c * T[TF_ALPHA];
}
__global__ void k_tf_beta(double* T) {
    double rn = T[TF_RHON];
    if (T[TF_RHO] == 0.0) {
        T[TF_BREAK] = 1.0;
        T[TF_BETA] = 0.0;
    } else {
        T[TF_BETA] = rn / T[TF_RHO];
    }
    T[TF_RHO] = rn;
}
__global__ void k_tf_uminus(double* u, const double* v, const double* T, int n) {
    double a = T[TF_ALPHA];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] -= a * v[i];
}
__global__ void k_tf_axpy_eta(double* x, const double* d, const double* T, int n) {
    double e = T[TF_ETA];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += e * d[i];
}
__global__ void k_tf_unew(double* u, const double* w, const double* T, int n) {
    double b = T[TF_BETA];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = w[i] + b * u[i];
}
__global__ void k_tf_vnew(double* v, const double* Bue, const double* Buo, const double* T, int n) {
    double b = T[TF_BETA];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = Bue[i] + b * (Buo[i] + b * v[i]);
}

// FGMRES: H (m+1) x m column-major, cs, sn, g (m+1)
__global__ void k_fg_init(double* g, int m, const double* rr, double* inv) {
    double b = sqrt(*rr);
    for (int a = 0; a <= m; ++a) g[a] = 0.0;
    g[0] = b;
    *inv = (b > 0.0) ? 1.0 / b : 0.0;
}
__global__ void k_fg_column(double* H, double* cs, double* sn, double* g, const double* h, const double* h2,
                            const double* hn2, int j, int m, double* inv_hn) {
    double* col = H + (size_t)j * (m + 1);
    for (int a = 0; a <= j; ++a) col[a] = h[a] + h2[a];
    double hn = sqrt(*hn2);
    col[j + 1] = hn;
    for (int a = 0; a < j; ++a) {
        double t = cs[a] * col[a] + sn[a] * col[a + 1];
        col[a + 1] = -sn[a] * col[a] + cs[a] * col[a + 1];
        col[a] = t;
    }
    double rr = hypot(col[j], col[j + 1]);
    double c = (rr != 0.0) ? col[j] / rr : 1.0;
    double s = (rr != 0.0) ? col[j + 1] / rr : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = rr;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    *inv_hn = (hn > 0.0) ? 1.0 / hn : 0.0;
}
__global__ void k_fg_backsolve(const double* H, const double* g, int steps, int m, double* y) {
    for (int a = steps - 1; a >= 0; --a) {
        double acc = g[a];
        for (int b = a + 1; b < steps; ++b) acc -= H[(size_t)b * (m + 1) + a] * y[b];
        y[a] = acc / H[(size_t)a * (m + 1) + a];
    }
}
__global__ void k_scale_dev(double* y, const double* x, const double* s, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (*s) * x[i];
}

}  // namespace asss

// ===========================================================================
// the handle
// ===========================================================================
struct KrylovWork {
    int n = 0, m = 0;
    DBuf<double> w, u, ut, v, Bue, Buo, d, rstar;
    DBuf<double> V, Z, H, cs, sn, g, hv, hv2, y;
    DBuf<double> T;
    ArnoldiWork ao;   // fused Arnoldi step (FGMRES)
    DBuf<int> stop;   // set by the fused step when the cycle ends
    double* hpin = nullptr;        // pinned read-back slots
    cudaEvent_t ev_rb = nullptr;   // marks the read-back in the stream
    cudaEvent_t ev_bn = nullptr;   // marks the read-back of ||b||^2 (slot 6)
    int outer = -1;
    ~KrylovWork() {
        if (hpin) cudaFreeHost(hpin);
        if (ev_rb) cudaEventDestroy(ev_rb);
        if (ev_bn) cudaEventDestroy(ev_bn);
    }
    // allocates on first use or when the size changes; kept by the handle across solves
    asss_status init(int n_, int m_, int outer_) {
        if (n == n_ && m == m_ && outer == outer_) return ASSS_OK;
        outer = -1;  // marked ready only when every buffer exists
        ASSS_TRY(T.alloc(32));
        if (!hpin) ASSS_CUDA(cudaMallocHost((void**)&hpin, 8 * sizeof(double)));
        if (!ev_rb) ASSS_CUDA(cudaEventCreateWithFlags(&ev_rb, cudaEventDisableTiming));
        if (!ev_bn) ASSS_CUDA(cudaEventCreateWithFlags(&ev_bn, cudaEventDisableTiming));
        if (!stop.p) ASSS_TRY(stop.alloc(1));
        if (outer_ == ASSS_OUTER_TFQMR) {
            ASSS_TRY(w.alloc(n_));
            ASSS_TRY(u.alloc(n_));
            ASSS_TRY(ut.alloc(n_));
            ASSS_TRY(v.alloc(n_));
            ASSS_TRY(Bue.alloc(n_));
            ASSS_TRY(Buo.alloc(n_));
            ASSS_TRY(d.alloc(n_));
            ASSS_TRY(rstar.alloc(n_));
        } else {
            ASSS_TRY(V.alloc((int64_t)n_ * (m_ + 1)));
            ASSS_TRY(Z.alloc((int64_t)n_ * m_));
            ASSS_TRY(H.alloc((int64_t)(m_ + 1) * m_));
            ASSS_TRY(cs.alloc(m_ + 1));
            ASSS_TRY(sn.alloc(m_ + 1));
            ASSS_TRY(g.alloc(m_ + 2));
            ASSS_TRY(hv.alloc(m_ + 1));
            ASSS_TRY(hv2.alloc(m_ + 1));
            ASSS_TRY(y.alloc(m_ + 1));
            ASSS_TRY(w.alloc(n_));
        }
        n = n_;
        m = m_;
        outer = outer_;
        return ASSS_OK;
    }
};

// Optional phase timing of a solve (environment variable ASSS_TRACE=1): CUDA
// events at phase boundaries on the solve's stream, summed and printed to stderr
// after the solve.  Off by default; no events are recorded then.
struct Tracer {
    enum { PREC = 0, OP, ORTH, REFINE, SCALAR, NPH };
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> tag;
    void mark(cudaStream_t s, int t) {
        if (!on) return;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, s);
        ev.push_back(e);
        tag.push_back(t);
    }
    void report(cudaStream_t s, int outer_its, long long inner) {
        if (!on || ev.size() < 2) return;
        cudaStreamSynchronize(s);
        double ph[NPH] = {0, 0, 0, 0, 0};
        for (size_t i = 0; i + 1 < ev.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            ph[tag[i]] += ms;
        }
        float tot = 0.f;
        cudaEventElapsedTime(&tot, ev.front(), ev.back());
        fprintf(stderr,
                "asss trace: total %.3f ms | preconditioner %.3f | operator %.3f | orthogonalisation %.3f | "
                "refinement %.3f | scalars+readback %.3f | outer its %d, inner its %lld\n",
                tot, ph[PREC], ph[OP], ph[ORTH], ph[REFINE], ph[SCALAR], outer_its, inner);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        tag.clear();
    }
};

// CUDA events around the outer operator and the fused Arnoldi step of a solve, with
// the work each launch does; summed into the solve's statistics after its last
// synchronisation (the pairs are reused from one solve to the next)
struct PhaseClock {
    enum { OP = 0, ORTH = 1 };
    std::vector<cudaEvent_t> ev;
    std::vector<int> cat;
    std::vector<double> bytes, flops;
    int used = 0;
    void start(cudaStream_t s) {
        while ((int)ev.size() < 2 * (used + 1)) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            ev.push_back(e);
        }
        cudaEventRecord(ev[2 * used], s);
    }
    void stop(cudaStream_t s, int c, double b, double f) {
        if ((int)ev.size() < 2 * (used + 1)) return;
        cudaEventRecord(ev[2 * used + 1], s);
        if ((int)cat.size() <= used) {
            cat.resize(used + 1);
            bytes.resize(used + 1);
            flops.resize(used + 1);
        }
        cat[used] = c;
        bytes[used] = b;
        flops[used] = f;
        ++used;
    }
    // the stream has been synchronised
    void collect(asss_stats* st) {
        for (int i = 0; i < used; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) continue;
            if (cat[i] == OP) {
                st->t_op_ms += ms;
                st->op_calls += 1;
                st->op_bytes += (long long)bytes[i];
                st->op_flops += (long long)flops[i];
            } else {
                st->t_orth_ms += ms;
                st->orth_calls += 1;
                st->orth_bytes += (long long)bytes[i];
                st->orth_flops += (long long)flops[i];
            }
        }
        used = 0;
    }
    ~PhaseClock() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

struct SmwData {
    bool ready = false;
    int m = 0;
    DBuf<double> Y;    // n x m row-major: X Sig (I + U^T X Sig)^-1
    DBuf<float> Y32;   // FP32 copy for the mixed-precision preconditioner
};

struct asss_handle {
    asss_options opt;
    Ctx ctx;
    int n = 0;
    DCsr A;            // original matrix (residuals)
    DCsr AT;           // A^T (adjoint residuals), lazily
    DCsr Abar, AbarT;
    DCsr S;            // S with values (pattern = s_pattern)
    DCsr ST;           // S^T with values, lazily (adjoint)
    DCsr Aw, Sw;       // W Abar, S W (outer operator)
    DCsr AwT, SwT;     // lazily (adjoint)
    DCsr Jt;           // J~ on P (FP64)
    DSell<double> J64;
    DSell<float> J32;
    DSkewDia<double> D64;
    DSkewDia<float> D32;
    bool use_dia = false;
    // incomplete L D L^T (options.factor = ASSS_FACTOR_ILDL0): J~ in factored form, W = 1
    // in the operators above and L~ applied by triangular solves instead
    bool factored = false;
    IldlFactor fac;
    DBuf<double> fa, fb;
    DBuf<double> dr, dc, w, d;
    DBuf<int> perm;
    bool has_perm = false;
    DBuf<double> xf_stage, dA_stage;   // adjoint gradient with host x / dA (allocated on first use)
    DBuf<int> neg;
    // 2x2 pivots: the second index and both coefficients of each U_r column (owned by
    // fac; null when every column is a unit vector)
    const int* neg2 = nullptr;
    const double* negc1 = nullptr;
    const double* negc2 = nullptr;
    int r = 0;
    int prec2 = 0;
    int k = 0, kp = 0;
    DBuf<double> Qcm;   // n x k column-major
    DBuf<double> Q64;   // n x kp row-major
    DBuf<float> Q32;
    DBuf<__nv_bfloat16> Q16;  // n x kp16 row-major (q_bf16)
    int kp16 = 0;
    DBuf<double> alpha_d;
    std::vector<double> alpha_h;
    SmwData smw[2];
    MrsWork* mw = nullptr;
    // work vectors
    DBuf<double> t1, t2, t3, zt, wv, scal;
    DBuf<float> z32;
    // per-solve work buffers, allocated once
    KrylovWork kw;
    Tracer tr;
    PhaseClock pc;
    DBuf<double> rr, rh, dy, rscal, bb, xx;
    // statistics of the current solve
    int inner_solves = 0;
    asss_stats setup_stats;
    // block solve (several right-hand sides in lockstep): per-column Krylov work and
    // buffers, allocated on first use
    static constexpr int BLK = 8;
    std::unique_ptr<KrylovWork> kwb[BLK];
    DBuf<double> blk_r, blk_rh, blk_dy, blk_z64, blk_G, blk_T, blk_b, blk_x;
    DBuf<float> blk_z32;
    ~asss_handle() {
        if (mw) mrs_work_destroy(mw);
    }
};

static UrCols ur_cols(const asss_handle* h) {
    UrCols U;
    U.neg = h->neg.p;
    U.neg2 = h->neg2;
    U.c1 = h->negc1;
    U.c2 = h->negc2;
    return U;
}

static void fill_defaults(asss_options* o) {
    memset(o, 0, sizeof(*o));
    o->gamma = 1.0;
    o->k_lanczos = 20;
    o->reorth = 1;
    o->inner_tol = 1e-10;
    o->setup_tol = 0.0;
    o->outer_tol = 1e-8;
    o->inner_maxit = 1000;
    o->outer_maxit = 2000;
    o->restart = 60;
    o->precision = ASSS_PREC_FP64;
    o->outer = ASSS_OUTER_TFQMR;
    o->r_max = 256;
    o->seed = 0x5eedull;
    o->lls_tol = 1e-13;
    o->lls_maxit = 20000;
    o->zero_tol = 1e-14;
    o->wait_timeout_ms = 2000.0;
    o->stream = nullptr;
    o->inner_format = ASSS_FORMAT_AUTO;
    o->q_bf16 = 0;
    o->s_values = nullptr;
    o->scaling = ASSS_SCALING_MAXES;
    o->rhs_block = 0;
    o->sell_sigma = 0;
    o->sell_split = 0;
    o->factor = ASSS_FACTOR_DIAG;
}

static int pick_kp(int k) {
    const int opts[] = {0, 4, 8, 12, 16, 20, 24, 32, 48, 64};
    for (int v : opts)
        if (v >= k) return v;
    return -1;
}

// ---------------------------------------------------------------------------
// skew-Lanczos (Fig. 2) with optional two-pass classical Gram-Schmidt
// ---------------------------------------------------------------------------
// J~ v in factored form: F (J^ (G v)), ta and tb n-vectors of scratch
static asss_status apply_jt_factored(const Ctx& c, IldlFactor& F, const DCsr& Jh, const double* v, double* out,
                                     double* ta, double* tb) {
    ASSS_TRY(ildl_G(c, F, v, ta));
    ASSS_TRY(spmv(Jh, ta, tb, nullptr, c.stream));
    return ildl_F(c, F, tb, out);
}

static asss_status lanczos(const Ctx& c, const DCsr& J, const double* q1, int n, int k, int reorth,
                           DBuf<double>& Qcm, std::vector<double>& alpha, int* k_eff, IldlFactor* F = nullptr,
                           double* ta = nullptr, double* tb = nullptr) {
    cudaStream_t s = c.stream;
    if (k > n) k = n;
    alpha.assign(k > 1 ? k - 1 : 0, 0.0);
    *k_eff = 0;
    if (k <= 0) return ASSS_OK;
    ASSS_TRY(Qcm.alloc((int64_t)n * k));
    DBuf<double> z, h, h2, sc;
    ASSS_TRY(z.alloc(n));
    ASSS_TRY(h.alloc(k));
    ASSS_TRY(h2.alloc(k));
    ASSS_TRY(sc.alloc(1));
    ASSS_TRY(dot(q1, q1, n, sc.p, s));
    double nn = 0.0;
    ASSS_CUDA(cudaMemcpyAsync(&nn, sc.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (!(nn > 0.0)) {
        set_error("Lanczos start vector is zero");
        return ASSS_ERR_ARG;
    }
    ASSS_TRY(vscale(Qcm.p, q1, 1.0 / sqrt(nn), n, s));
    int kk = 1;
    for (int i = 1; i < k; ++i) {
        if (F) ASSS_TRY(apply_jt_factored(c, *F, J, Qcm.p + (size_t)(i - 1) * n, z.p, ta, tb));
        else ASSS_TRY(spmv(J, Qcm.p + (size_t)(i - 1) * n, z.p, nullptr, s));
        if (i >= 2) ASSS_TRY(vaxpy(z.p, Qcm.p + (size_t)(i - 2) * n, -alpha[i - 2], n, s));
        if (reorth) {
            for (int pass = 0; pass < 2; ++pass) {
                ASSS_TRY(gram(Qcm.p, n, i, z.p, n, 1, n, h.p, s));
                k_sub_colmajor<<<cdiv(n, 256), 256, 0, s>>>(Qcm.p, n, i, h.p, n, z.p);
                ASSS_CHECK_LAUNCH();
            }
        }
        ASSS_TRY(dot(z.p, z.p, n, sc.p, s));
        ASSS_CUDA(cudaMemcpyAsync(&nn, sc.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        double a = sqrt(nn);
        if (a == 0.0 || (i >= 2 && a <= 1e-12 * alpha[0])) break;
        alpha[i - 1] = a;
        ASSS_TRY(vscale(Qcm.p + (size_t)i * n, z.p, -1.0 / a, n, s));
        kk = i + 1;
    }
    alpha.resize(kk - 1);
    *k_eff = kk;
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// preconditioner pieces
// ---------------------------------------------------------------------------
static asss_status ensure_smw(asss_handle* h, int tr) {
    SmwData& S = h->smw[tr];
    if (S.ready) return ASSS_OK;
    const Ctx& c = h->ctx;
    cudaStream_t s = c.stream;
    int n = h->n, k = h->k, r = h->r, m = k + r;
    S.m = m;
    if (m == 0) {
        S.ready = true;
        return ASSS_OK;
    }
    DBuf<double> X, rhs, G, Sig, K, Z;
    ASSS_TRY(X.alloc((int64_t)n * m));
    ASSS_TRY(rhs.alloc(n));
    MrsOperator op;
    op.J64 = h->use_dia ? nullptr : &h->J64;
    op.D64 = h->use_dia ? &h->D64 : nullptr;
    op.F = h->factored ? &h->fac : nullptr;
    op.k = h->k;
    op.kp = h->kp;
    op.Q64 = h->Q64.p;
    op.alpha = h->alpha_d.p;
    double tol = h->opt.setup_tol > 0 ? h->opt.setup_tol : h->opt.inner_tol;
    double sign = tr ? -1.0 : 1.0;
    const UrCols U = ur_cols(h);
    if (h->kp <= MRS_MULTI_KPMAX && !h->factored) {
        // S_bar X = U_bar as App. B's simultaneous iterations: the k + r columns share
        // every pass over J~ and Q_k (groups of up to 8 per launch)
        DBuf<double> Ub;
        ASSS_TRY(Ub.alloc((int64_t)n * m));
        if (k) ASSS_CUDA(cudaMemcpyAsync(Ub.p, h->Qcm.p, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, s));
        for (int t = 0; t < r; ++t) {
            k_ur_column<<<cdiv(n, 256), 256, 0, s>>>(Ub.p + (size_t)(k + t) * n, n, U, t);
            ASSS_CHECK_LAUNCH();
        }
        ASSS_TRY(mrs_multi_solve(c, op, false, 1.0, sign, m, Ub.p, n, X.p, nullptr, n, tol, h->opt.inner_maxit,
                                 nullptr, nullptr));
    } else {
        for (int col = 0; col < m; ++col) {
            const double* b;
            if (col < k) {
                b = h->Qcm.p + (size_t)col * n;
            } else {
                k_ur_column<<<cdiv(n, 256), 256, 0, s>>>(rhs.p, n, U, col - k);
                ASSS_CHECK_LAUNCH();
                b = rhs.p;
            }
            ASSS_TRY(mrs_solve(c, h->mw, op, false, 1.0, sign, b, X.p + (size_t)col * n, nullptr, tol,
                               h->opt.inner_maxit, nullptr, nullptr, false));
        }
    }
    ASSS_TRY(G.alloc((int64_t)m * m));
    ASSS_TRY(Sig.alloc((int64_t)m * m));
    ASSS_TRY(K.alloc((int64_t)m * m));
    ASSS_TRY(Z.alloc((int64_t)m * m));
    if (k) ASSS_TRY(gram(h->Qcm.p, n, k, X.p, n, m, n, G.p, s));
    if (r) {
        k_gram_neg_rows<<<cdiv(r * m, 256), 256, 0, s>>>(X.p, n, m, U, k, r, G.p);
        ASSS_CHECK_LAUNCH();
    }
    k_sigma<<<cdiv(m * m, 256), 256, 0, s>>>(h->alpha_d.p, k, m, tr, Sig.p);
    ASSS_CHECK_LAUNCH();
    k_small_mm<<<cdiv(m * m, 256), 256, 0, s>>>(G.p, Sig.p, m, 1, K.p);  // K = I + (U^T X) Sig
    ASSS_CHECK_LAUNCH();
    int singular = 0;
    ASSS_TRY(small_inverse(K.p, m, &singular, s));
    if (singular) {
        set_error("the SMW matrix I + U^T S_bar^-1 U Sig is singular");
        return ASSS_ERR_BREAKDOWN;
    }
    k_small_mm<<<cdiv(m * m, 256), 256, 0, s>>>(Sig.p, K.p, m, 0, Z.p);  // Z = Sig K^-1
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(mrs_collect(c, h->mw, nullptr));
    mrs_take_totals(h->mw);
    ASSS_TRY(S.Y.alloc((int64_t)n * m));
    k_x_times_small<<<cdiv((int64_t)n * m, 256), 256, 0, s>>>(X.p, Z.p, n, m, S.Y.p);
    ASSS_CHECK_LAUNCH();
    if (h->opt.precision == ASSS_PREC_MIXED) {
        ASSS_TRY(S.Y32.alloc((int64_t)n * m));
        k_d2f<<<cdiv((int64_t)n * m, 256), 256, 0, s>>>(S.Y.p, (int64_t)n * m, S.Y32.p);
        ASSS_CHECK_LAUNCH();
    }
    ASSS_CUDA(cudaStreamSynchronize(s));
    S.ready = true;
    return ASSS_OK;
}

// out = P^-1 u (tr = 0) or P^-T u (tr = 1): z = S_bar^-1 u by mrs, then SMW (Eq. smw)
//   P^-1 u = z - Y (U_bar^T z),  U_bar^T z = [Q_k^T z ; z(neg)]
// Q_k^T z comes out of the mrs kernel's final pass.  Step counts and timings stay
// on the device until the solve collects them.
static asss_status apply_prec(asss_handle* h, int tr, const double* u, double* out) {
    NvtxRange nv_("asss:preconditioner");
    const Ctx& c = h->ctx;
    cudaStream_t s = c.stream;
    int n = h->n;
    ASSS_TRY(ensure_smw(h, tr));
    MrsOperator op;
    op.J64 = h->use_dia ? nullptr : &h->J64;
    op.J32 = (!h->use_dia && h->J32.n) ? &h->J32 : nullptr;
    op.D64 = h->use_dia ? &h->D64 : nullptr;
    op.D32 = (h->use_dia && h->D32.n) ? &h->D32 : nullptr;
    op.F = h->factored ? &h->fac : nullptr;
    op.k = h->k;
    op.kp = h->kp;
    op.Q64 = h->Q64.p;
    op.Q32 = h->Q32.p;
    op.Q16 = h->Q16.p;
    op.kp16 = h->kp16;
    op.alpha = h->alpha_d.p;
    bool fp32 = h->opt.precision == ASSS_PREC_MIXED;
    double sign = tr ? -1.0 : 1.0;
    SmwData& S = h->smw[tr];
    double* qtz = (S.m > 0 && h->k > 0) ? h->wv.p : nullptr;
    if (fp32) {
        ASSS_TRY(mrs_solve(c, h->mw, op, true, 1.0, sign, u, nullptr, h->z32.p, h->opt.inner_tol,
                           h->opt.inner_maxit, qtz, nullptr, false));
        if (h->r && S.m > 0) {
            k_gather_neg_f<<<cdiv(h->r, 128), 128, 0, s>>>(h->z32.p, ur_cols(h), h->r, h->wv.p + h->k);
            ASSS_CHECK_LAUNCH();
        }
        k_smw_apply_f32<<<cdiv(n, 256), 256, sizeof(float) * (S.m > 0 ? S.m : 1), s>>>(
            h->z32.p, S.m > 0 ? S.Y32.p : nullptr, S.m, h->wv.p, n, out,
            stream_evict_first(c, (long long)n * (4LL * h->kp + 28) + 4LL * h->D32.nnz) ? 1 : 0,
            mrs_get_skip(h->mw));
        ASSS_CHECK_LAUNCH();
    } else {
        double* z = (S.m > 0) ? h->zt.p : out;
        ASSS_TRY(mrs_solve(c, h->mw, op, false, 1.0, sign, u, z, nullptr, h->opt.inner_tol, h->opt.inner_maxit,
                           qtz, nullptr, false));
        if (S.m > 0) {
            if (h->r) {
                k_gather_neg<<<cdiv(h->r, 128), 128, 0, s>>>(z, ur_cols(h), h->r, h->wv.p + h->k);
                ASSS_CHECK_LAUNCH();
            }
            ASSS_TRY(sub_rowmajor_gemv(S.Y.p, S.m, h->wv.p, z, n, out, s, mrs_get_skip(h->mw)));
        }
    }
    h->inner_solves += 1;
    return ASSS_OK;
}

static asss_status ensure_adjoint_ops(asss_handle* h) {
    cudaStream_t s = h->ctx.stream;
    if (!h->AwT.nnz && h->Aw.nnz) ASSS_TRY(transpose_csr(h->Aw, h->AwT, nullptr, s));
    if (!h->SwT.nnz && h->Sw.nnz) ASSS_TRY(transpose_csr(h->Sw, h->SwT, nullptr, s));
    if (!h->ST.nnz && h->S.nnz) ASSS_TRY(transpose_csr(h->S, h->ST, nullptr, s));
    if (!h->AT.nnz && h->A.nnz) ASSS_TRY(transpose_csr(h->A, h->AT, nullptr, s));
    int ok = 0;
    for (DCsr* M : {&h->AwT, &h->SwT, &h->ST, &h->AT})
        if (M->nnz) ASSS_TRY(attach_dia(*M, 16, 0.5, &ok, s));
    return ASSS_OK;
}

// algorithmic bytes of one product: the stored values (a diagonal copy has no column
// indices) and x, y once each; its FP64 flops: one FMA per stored value
static long long spmv_bytes(const DCsr& A) {
    const long long n = A.n;
    if (A.dia.ndiag > 0) return (long long)A.dia.ndiag * n * 8 + 16 * n;
    return (long long)A.nnz * 12 + 4 * (n + 1) + 16 * n;
}
static long long spmv_flops(const DCsr& A) {
    return 2LL * (A.dia.ndiag > 0 ? (long long)A.dia.ndiag * A.n : (long long)A.nnz);
}

static asss_status apply_op_impl(asss_handle* h, int tr, const double* v, double* out);

// out = A_cal v or A_cal^T v, timed into the solve's statistics
static asss_status apply_op(asss_handle* h, int tr, const double* v, double* out) {
    cudaStream_t s = h->ctx.stream;
    h->pc.start(s);
    ASSS_TRY(apply_op_impl(h, tr, v, out));
    const DCsr& a = tr ? h->AwT : h->Aw;
    const DCsr& b = tr ? h->SwT : h->Sw;
    double bytes = (double)(spmv_bytes(a) + spmv_bytes(b));
    double flops = (double)(spmv_flops(a) + spmv_flops(b));
    if (h->factored) {
        bytes += (double)(h->fac.nl + h->fac.nu) * 12 + 6.0 * 8 * h->n;
        flops += 2.0 * (double)(h->fac.nl + h->fac.nu) + 2.0 * h->n;
    }
    h->pc.stop(s, PhaseClock::OP, bytes, flops);
    return ASSS_OK;
}

static asss_status apply_op_impl(asss_handle* h, int tr, const double* v, double* out) {
    cudaStream_t s = h->ctx.stream;
    if (h->factored) {
        // F A^ G v or F A^T G v (Eq. preconditioner with the incomplete factor)
        ASSS_TRY(ildl_G(h->ctx, h->fac, v, h->fa.p));
        if (!tr) {
            ASSS_TRY(spmv(h->Sw, h->fa.p, h->t3.p, nullptr, s));
            ASSS_TRY(spmv(h->Aw, h->t3.p, h->fb.p, nullptr, s));
        } else {
            ASSS_TRY(ensure_adjoint_ops(h));
            ASSS_TRY(spmv(h->AwT, h->fa.p, h->t3.p, nullptr, s));
            ASSS_TRY(spmv(h->SwT, h->t3.p, h->fb.p, nullptr, s));
        }
        return ildl_F(h->ctx, h->fac, h->fb.p, out);
    }
    if (!tr) {
        ASSS_TRY(spmv(h->Sw, v, h->t3.p, nullptr, s));
        ASSS_TRY(spmv(h->Aw, h->t3.p, out, nullptr, s));
    } else {
        ASSS_TRY(ensure_adjoint_ops(h));
        ASSS_TRY(spmv(h->AwT, v, h->t3.p, nullptr, s));
        ASSS_TRY(spmv(h->SwT, h->t3.p, out, nullptr, s));
    }
    return ASSS_OK;
}

static double read_scalar(const double* d, cudaStream_t s, asss_status* st) {
    double v = 0.0;
    cudaError_t e = cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("scalar read-back failed: %s", cudaGetErrorString(e));
        *st = ASSS_ERR_CUDA;
    }
    return v;
}

// ---------------------------------------------------------------------------
// one TFQMR run (Freund 1993), right preconditioned, from zero: op(M^-1 u) = r
// ---------------------------------------------------------------------------


static asss_status tfqmr_cycle(asss_handle* h, KrylovWork& kw, int tr, const double* r, double eta, int max_steps,
                               double* delta, int* steps_out, int* napp_out) {
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    int nb = cdiv(n, 256);
    asss_status st = ASSS_OK;
    double* T = kw.T.p;
    ASSS_CUDA(cudaMemsetAsync(delta, 0, sizeof(double) * n, s));
    ASSS_TRY(dot(r, r, n, T + TF_WN2, s));
    double rr = read_scalar(T + TF_WN2, s, &st);
    ASSS_TRY(st);
    *steps_out = 0;
    *napp_out = 0;
    if (rr == 0.0) return ASSS_OK;
    double target = eta * sqrt(rr);
    ASSS_TRY(vcopy(kw.w.p, r, n, s));
    ASSS_TRY(vcopy(kw.u.p, r, n, s));
    ASSS_TRY(vcopy(kw.rstar.p, r, n, s));
    ASSS_CUDA(cudaMemsetAsync(kw.d.p, 0, sizeof(double) * n, s));
    k_tf_init<<<1, 1, 0, s>>>(T, T + TF_WN2);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(apply_prec(h, tr, kw.u.p, kw.ut.p));
    *napp_out += 1;
    ASSS_TRY(apply_op(h, tr, kw.ut.p, kw.v.p));
    ASSS_TRY(vcopy(kw.Bue.p, kw.v.p, n, s));
    int mcount = 0;
    for (int step = 1; step <= max_steps; ++step) {
        ASSS_TRY(dot(kw.rstar.p, kw.v.p, n, T + TF_SIGMA, s));
        k_tf_alpha<<<1, 1, 0, s>>>(T);
        ASSS_CHECK_LAUNCH();
        for (int half = 0; half < 2; ++half) {
            const double* Bu;
            if (half == 0) {
                Bu = kw.Bue.p;
            } else {
                k_tf_uminus<<<nb, 256, 0, s>>>(kw.u.p, kw.v.p, T, n);
                ASSS_CHECK_LAUNCH();
                ASSS_TRY(apply_prec(h, tr, kw.u.p, kw.ut.p));
                *napp_out += 1;
                ASSS_TRY(apply_op(h, tr, kw.ut.p, kw.Buo.p));
                Bu = kw.Buo.p;
            }
            k_tf_wd<<<nb, 256, 0, s>>>(kw.w.p, Bu, kw.d.p, kw.ut.p, T, n);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(dot(kw.w.p, kw.w.p, n, T + TF_WN2, s));
            k_tf_theta<<<1, 1, 0, s>>>(T);
            ASSS_CHECK_LAUNCH();
            k_tf_axpy_eta<<<nb, 256, 0, s>>>(delta, kw.d.p, T, n);
            ASSS_CHECK_LAUNCH();
            ++mcount;
            double hostT[TF_NSC];
            ASSS_CUDA(cudaMemcpyAsync(hostT, T, sizeof(hostT), cudaMemcpyDeviceToHost, s));
            ASSS_CUDA(cudaStreamSynchronize(s));
            if (hostT[TF_BREAK] != 0.0) {
                *steps_out = step - 1;
                return ASSS_OK;
            }
            if (hostT[TF_TAU] * sqrt(mcount + 1.0) <= target) {
                *steps_out = step;
                return ASSS_OK;
            }
        }
        ASSS_TRY(dot(kw.rstar.p, kw.w.p, n, T + TF_RHON, s));
        k_tf_beta<<<1, 1, 0, s>>>(T);
        ASSS_CHECK_LAUNCH();
        k_tf_unew<<<nb, 256, 0, s>>>(kw.u.p, kw.w.p, T, n);
        ASSS_CHECK_LAUNCH();
        ASSS_TRY(apply_prec(h, tr, kw.u.p, kw.ut.p));
        *napp_out += 1;
        ASSS_TRY(apply_op(h, tr, kw.ut.p, kw.Bue.p));
        k_tf_vnew<<<nb, 256, 0, s>>>(kw.v.p, kw.Bue.p, kw.Buo.p, T, n);
        ASSS_CHECK_LAUNCH();
        *steps_out = step;
    }
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// one cycle of flexible GMRES(m) (Saad 1993) with two classical Gram-Schmidt passes
// ---------------------------------------------------------------------------
static asss_status fgmres_cycle(asss_handle* h, KrylovWork& kw, int tr, const double* r, double eta, int m,
                                double* delta, int* steps_out, int* napp_out) {
    NvtxRange nv_("asss:fgmres-cycle");
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    int M = kw.m;
    if (m > M) m = M;
    double* T = kw.T.p;  // 0: rr, 1: inv, 2: hn2, 3: inv_hn
    double* hp = kw.hpin;
    *steps_out = 0;
    *napp_out = 0;
    // v_0 = r / ||r||, and P^-1 v_0 enqueued before ||r|| reaches the host
    ASSS_TRY(dot(r, r, n, T, s));
    k_fg_init<<<1, 1, 0, s>>>(kw.g.p, M, T, T + 1);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaMemcpyAsync(hp, T, sizeof(double), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaEventRecord(kw.ev_rb, s));
    ASSS_CUDA(cudaMemsetAsync(delta, 0, sizeof(double) * n, s));
    k_scale_dev<<<cdiv(n, 256), 256, 0, s>>>(kw.V.p, r, T + 1, n);
    ASSS_CHECK_LAUNCH();
    h->tr.mark(s, Tracer::PREC);
    ASSS_TRY(apply_prec(h, tr, kw.V.p, kw.Z.p));
    bool have_z = true;  // Z[:, j] is already enqueued
    ASSS_CUDA(cudaEventSynchronize(kw.ev_rb));
    const double rr = hp[0];
    if (rr == 0.0 || !(rr == rr) || rr == INFINITY) return ASSS_OK;  // nothing to do, or a NaN the caller reports
    *napp_out = 1;
    const double beta0 = sqrt(rr);
    const double thr = eta * beta0;
    int steps = 0;
    for (int j = 0; j < m; ++j) {
        double* vj = kw.V.p + (size_t)j * n;
        double* zj = kw.Z.p + (size_t)j * n;
        if (!have_z) {
            h->tr.mark(s, Tracer::PREC);
            ASSS_TRY(apply_prec(h, tr, vj, zj));
            *napp_out += 1;
        }
        have_z = false;
        h->tr.mark(s, Tracer::OP);
        ASSS_TRY(apply_op(h, tr, zj, kw.w.p));
        h->tr.mark(s, Tracer::ORTH);
        const bool fused = j + 1 < AO_MAXV;
        if (fused) {
            // CGS2, ||w||, the Givens update, v_{j+1} and the stop test in one launch;
            // work: V read twice, w three times, w and v_{j+1} written; 4(j+1) FP64 FMAs a row
            h->pc.start(s);
            ASSS_TRY(arnoldi_orth(h->ctx, kw.ao, kw.V.p, kw.w.p, n, j, M, kw.H.p, kw.cs.p, kw.sn.p, kw.g.p,
                                  kw.hv.p, kw.hv2.p, T + 2, T + 3, thr, kw.stop.p));
            h->pc.stop(s, PhaseClock::ORTH, 8.0 * n * (2.0 * (j + 1) + 5.0), 8.0 * n * (j + 1));
            h->tr.mark(s, Tracer::SCALAR);
        } else {
            ASSS_TRY(gram(kw.V.p, n, j + 1, kw.w.p, n, 1, n, kw.hv.p, s));
            k_sub_colmajor<<<cdiv(n, 256), 256, 0, s>>>(kw.V.p, n, j + 1, kw.hv.p, n, kw.w.p);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(gram(kw.V.p, n, j + 1, kw.w.p, n, 1, n, kw.hv2.p, s));
            k_sub_colmajor<<<cdiv(n, 256), 256, 0, s>>>(kw.V.p, n, j + 1, kw.hv2.p, n, kw.w.p);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(dot(kw.w.p, kw.w.p, n, T + 2, s));
            h->tr.mark(s, Tracer::SCALAR);
            k_fg_column<<<1, 1, 0, s>>>(kw.H.p, kw.cs.p, kw.sn.p, kw.g.p, kw.hv.p, kw.hv2.p, T + 2, j, M, T + 3);
            ASSS_CHECK_LAUNCH();
        }
        steps = j + 1;
        // read-back slots: 0 g[j+1], 1 ||w||^2, 2 (int) device wait status, 3 (int) stop flag
        int* hi = reinterpret_cast<int*>(hp + 2);
        hi[0] = 0;
        hi[2] = 0;
        ASSS_CUDA(cudaMemcpyAsync(hp, kw.g.p + j + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaMemcpyAsync(hp + 1, T + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (fused) {
            ASSS_CUDA(cudaMemcpyAsync(hi, kw.ao.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            ASSS_CUDA(cudaMemcpyAsync(hi + 2, kw.stop.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        ASSS_CUDA(cudaEventRecord(kw.ev_rb, s));
        // while the host waits for the stop test, P^-1 v_{j+1} runs; if the cycle
        // ends here the mrs launch finds the device stop flag set and does nothing
        if (fused && j + 1 < m) {
            h->tr.mark(s, Tracer::PREC);
            mrs_set_skip(h->mw, kw.stop.p);
            asss_status ps = apply_prec(h, tr, kw.V.p + (size_t)(j + 1) * n, kw.Z.p + (size_t)(j + 1) * n);
            mrs_set_skip(h->mw, nullptr);
            ASSS_TRY(ps);
            have_z = true;
        }
        ASSS_CUDA(cudaEventSynchronize(kw.ev_rb));
        if (hi[0]) {
            kw.ao.n = 0;  // the barrier counter is re-initialised on the next launch
            set_error("a device wait in the Arnoldi step ran out (status %d)", hi[0]);
            return (asss_status)hi[0];
        }
        const bool stop = fused ? (hi[2] != 0) : (hp[1] == 0.0 || fabs(hp[0]) <= thr);
        if (stop) break;
        if (have_z) *napp_out += 1;
        if (!fused) {
            k_scale_dev<<<cdiv(n, 256), 256, 0, s>>>(kw.V.p + (size_t)(j + 1) * n, kw.w.p, T + 3, n);
            ASSS_CHECK_LAUNCH();
        }
    }
    k_fg_backsolve<<<1, 1, 0, s>>>(kw.H.p, kw.g.p, steps, M, kw.y.p);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(colmajor_gemv(kw.Z.p, n, steps, kw.y.p, n, 0.0, delta, s));
    *steps_out = steps;
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// refinement loop on the true FP64 residual of the original system (§4.1 stop)
// ---------------------------------------------------------------------------
static asss_status refine(asss_handle* h, int tr, const double* rhs, double* x, asss_stats* st) {
    NvtxRange nv_(tr ? "asss:adjoint-solve" : "asss:solve");
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    int nb = cdiv(n, 256);
    const asss_options& o = h->opt;
    asss_status es = ASSS_OK;
    KrylovWork& kw = h->kw;
    ASSS_TRY(kw.init(n, o.restart > 0 ? o.restart : 60, o.outer));
    if (kw.n != n || kw.outer != o.outer || !kw.w.p) {
        set_error("internal: Krylov workspace not allocated");
        return ASSS_ERR_CUDA;
    }
    if (!h->rr.p) {
        ASSS_TRY(h->rr.alloc(n));
        ASSS_TRY(h->rh.alloc(n));
        ASSS_TRY(h->dy.alloc(n));
        ASSS_TRY(h->rscal.alloc(2));
    }
    DBuf<double>& r = h->rr;
    DBuf<double>& rh = h->rh;
    DBuf<double>& dy = h->dy;
    DBuf<double>& scal = h->rscal;
    h->inner_solves = 0;
    ASSS_TRY(mrs_collect(h->ctx, h->mw, nullptr));
    mrs_take_totals(h->mw);
    h->pc.used = 0;   // pairs recorded outside a solve (single operator applications) are dropped
    st->t_op_ms = st->t_orth_ms = 0.0;
    st->op_calls = st->orth_calls = 0;
    st->op_bytes = st->op_flops = st->orth_bytes = st->orth_flops = 0;
    ASSS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    ASSS_TRY(vcopy(r.p, rhs, n, s));
    ASSS_TRY(dot(rhs, rhs, n, scal.p, s));
    // FGMRES: the first cycle needs ||b|| only through ||r|| / ||b|| = 1, so its read-back
    // is left in flight and the cycle is enqueued at once (b = 0 and a NaN in b come back
    // through the cycle's own ||r^|| and are decided after it); TFQMR waits for it here
    const bool defer_bn = o.outer == ASSS_OUTER_FGMRES && o.outer_tol < 1.0 && o.outer_maxit > 0;
    double bn = -1.0;
    if (defer_bn) {
        ASSS_CUDA(cudaMemcpyAsync(kw.hpin + 6, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaEventRecord(kw.ev_bn, s));
    } else {
        bn = sqrt(read_scalar(scal.p, s, &es));
        ASSS_TRY(es);
    }
    st->outer_its = 0;
    st->cycles = 0;
    st->relres = 0.0;
    st->status = ASSS_OK;
    if (tr) ASSS_TRY(ensure_adjoint_ops(h));
    if (bn == 0.0) return ASSS_OK;
    double best = INFINITY;
    int stall = 0;
    int* perm = h->has_perm ? h->perm.p : nullptr;
    h->tr.on = getenv("ASSS_TRACE") != nullptr;
    bool first = true;  // r = b (x = 0) on the first pass: ||r|| = ||b|| is known
    while (true) {
        h->tr.mark(s, Tracer::REFINE);
        double rn = bn;
        if (!first) {
            ASSS_TRY(dot(r.p, r.p, n, scal.p, s));
            rn = sqrt(read_scalar(scal.p, s, &es));
            ASSS_TRY(es);
        }
        first = false;
        if (bn < 0.0) {  // ||b|| still in flight: r = b, so ||r|| / ||b|| = 1 (not below tol < 1)
            rn = 1.0;
            bn = 1.0;
        }
        st->relres = rn / bn;
        if (rn / bn <= o.outer_tol) break;
        if (!(rn == rn)) {
            st->status = ASSS_ERR_BREAKDOWN;
            set_error("residual became NaN");
            break;
        }
        if (st->outer_its >= o.outer_maxit) {
            st->status = ASSS_ERR_NOT_CONVERGED;
            break;
        }
        if (rn < 0.999 * best) {
            best = rn;
            stall = 0;
        } else if (++stall >= 5) {
            st->status = ASSS_ERR_STAGNATION;
            break;
        }
        if (!tr) {
            // W P D_r r  (F P D_r r with the incomplete factor, W = 1 there)
            k_to_scaled_fwd<<<nb, 256, 0, s>>>(r.p, h->dr.p, h->w.p, perm, n, h->factored ? h->fa.p : rh.p);
            ASSS_CHECK_LAUNCH();
            if (h->factored) ASSS_TRY(ildl_F(h->ctx, h->fac, h->fa.p, rh.p));
        } else {
            ASSS_TRY(vmul(h->t1.p, h->dc.p, r.p, n, s));  // W S^T D_c r  (F S^T D_c r)
            ASSS_TRY(spmv(h->ST, h->t1.p, h->t2.p, nullptr, s));
            if (h->factored) ASSS_TRY(ildl_F(h->ctx, h->fac, h->t2.p, rh.p));
            else ASSS_TRY(vmul(rh.p, h->w.p, h->t2.p, n, s));
        }
        double eta = fmin(0.5, 0.5 * o.outer_tol * bn / rn);
        int budget = o.outer_maxit - st->outer_its;
        int steps = 0, napp = 0;
        if (o.outer == ASSS_OUTER_TFQMR) {
            ASSS_TRY(tfqmr_cycle(h, kw, tr, rh.p, eta, budget, dy.p, &steps, &napp));
        } else {
            int m = o.restart < budget ? o.restart : budget;
            ASSS_TRY(fgmres_cycle(h, kw, tr, rh.p, eta, m, dy.p, &steps, &napp));
        }
        if (defer_bn && st->cycles == 0) {
            // the true ||b|| (its read-back finished long ago); the first cycle ran with
            // the ratio 1, which is what r = b gives for any non-zero finite b
            ASSS_CUDA(cudaEventSynchronize(kw.ev_bn));
            bn = sqrt(kw.hpin[6]);
            if (bn == 0.0) {  // the cycle saw r^ = 0 and added nothing: x = 0
                st->relres = 0.0;
                break;
            }
            if (!(bn == bn) || bn == INFINITY) {
                st->status = ASSS_ERR_BREAKDOWN;
                set_error("right-hand side has a NaN or infinite entry");
                break;
            }
            best = bn;  // the first pass's ||r|| in its true scale
        }
        st->outer_its += steps;
        st->cycles += 1;
        h->tr.mark(s, Tracer::REFINE);
        if (!tr) {
            // x += D_c S W dy  (D_c S G dy)
            if (h->factored) ASSS_TRY(ildl_G(h->ctx, h->fac, dy.p, h->t1.p));
            else ASSS_TRY(vmul(h->t1.p, h->w.p, dy.p, n, s));
            ASSS_TRY(spmv(h->S, h->t1.p, h->t2.p, nullptr, s));
            k_axpy_mul<<<nb, 256, 0, s>>>(x, h->dc.p, h->t2.p, n);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(spmv(h->A, x, h->t1.p, nullptr, s));
        } else {
            // lambda += D_r P^T W dmu  (D_r P^T G dmu)
            if (h->factored) ASSS_TRY(ildl_G(h->ctx, h->fac, dy.p, h->fa.p));
            k_from_scaled_adj<<<nb, 256, 0, s>>>(h->factored ? h->fa.p : dy.p, h->dr.p, h->w.p, perm, n, x);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(spmv(h->AT, x, h->t1.p, nullptr, s));
        }
        k_sub<<<nb, 256, 0, s>>>(rhs, h->t1.p, r.p, n);
        ASSS_CHECK_LAUNCH();
    }
    h->tr.mark(s, Tracer::REFINE);
    ASSS_TRY(mrs_collect(h->ctx, h->mw, nullptr));
    MrsTotals t = mrs_take_totals(h->mw);
    h->tr.report(s, st->outer_its, t.its);
    h->pc.collect(st);   // mrs_collect synchronised the stream
    st->inner_its_total = t.its;
    st->inner_solves = t.launches;
    st->inner_its_avg = t.launches ? (double)t.its / t.launches : 0.0;
    st->t_inner_ms = t.ms;
    st->inner_bytes = t.bytes;
    st->inner_launches = t.launches;
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// several right-hand sides in lockstep: every column runs its own refinement loop
// and flexible GMRES (same arithmetic as refine / fgmres_cycle), but the
// preconditioner applications of one Arnoldi step are a single multi-column mrs
// launch (App. B's simultaneous iterations), so the columns share each pass over J~
// and Q_k
// ---------------------------------------------------------------------------
__global__ void k_gather_col(const double* G, int ldg, int col, int k, double* out) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < k) out[a] = G[(size_t)a * ldg + col];
}

// out_c = P^-1 u_c (tr = 0) or P^-T u_c for the columns listed (Eq. smw around one
// multi-column mrs launch per 8 columns)
static asss_status apply_prec_block(asss_handle* h, int tr, int nc, const double* const* u, double* const* out,
                                    long long* its_sum, int* launches, MrsTotals* tot) {
    NvtxRange nv_("asss:preconditioner-block");
    const Ctx& c = h->ctx;
    cudaStream_t s = c.stream;
    const int n = h->n;
    ASSS_TRY(ensure_smw(h, tr));
    MrsOperator op;
    op.J64 = h->use_dia ? nullptr : &h->J64;
    op.J32 = (!h->use_dia && h->J32.n) ? &h->J32 : nullptr;
    op.D64 = h->use_dia ? &h->D64 : nullptr;
    op.D32 = (h->use_dia && h->D32.n) ? &h->D32 : nullptr;
    op.F = h->factored ? &h->fac : nullptr;
    op.k = h->k;
    op.kp = h->kp;
    op.Q64 = h->Q64.p;
    op.Q32 = h->Q32.p;
    op.alpha = h->alpha_d.p;
    const bool fp32 = h->opt.precision == ASSS_PREC_MIXED;
    const double sign = tr ? -1.0 : 1.0;
    SmwData& S = h->smw[tr];
    const int B = asss_handle::BLK;
    int its[B];
    double ratio[B];
    double* z64[B];
    float* z32[B];
    for (int t = 0; t < nc; ++t) {
        z64[t] = (S.m > 0 || fp32) ? h->blk_z64.p + (size_t)t * n : out[t];
        z32[t] = h->blk_z32.p ? h->blk_z32.p + (size_t)t * n : nullptr;
    }
    if (fp32) {
        ASSS_TRY(mrs_multi_solve_cols(c, op, true, 1.0, sign, nc, u, nullptr, z32, h->opt.inner_tol,
                                      h->opt.inner_maxit, its, ratio, tot));
        for (int t = 0; t < nc; ++t) {
            k_f2d<<<cdiv(n, 256), 256, 0, s>>>(z32[t], z64[t], n);
            ASSS_CHECK_LAUNCH();
        }
    } else {
        ASSS_TRY(mrs_multi_solve_cols(c, op, false, 1.0, sign, nc, u, z64, nullptr, h->opt.inner_tol,
                                      h->opt.inner_maxit, its, ratio, tot));
    }
    for (int t = 0; t < nc; ++t) *its_sum += its[t];
    *launches += nc;
    if (S.m > 0) {
        // U_bar^T z = [Q_k^T z ; z(neg)] for every column at once (one pass over Q_k)
        if (h->k) ASSS_TRY(gram(h->Qcm.p, n, h->k, h->blk_z64.p, n, nc, n, h->blk_G.p, s));
        for (int t = 0; t < nc; ++t) {
            double* wv = h->blk_T.p + (size_t)t * (S.m + 1);
            if (h->k) {
                k_gather_col<<<cdiv(h->k, 64), 64, 0, s>>>(h->blk_G.p, nc, t, h->k, wv);
                ASSS_CHECK_LAUNCH();
            }
            if (h->r) {
                k_gather_neg<<<cdiv(h->r, 128), 128, 0, s>>>(z64[t], ur_cols(h), h->r, wv + h->k);
                ASSS_CHECK_LAUNCH();
            }
            if (fp32) {
                k_smw_apply_f32<<<cdiv(n, 256), 256, sizeof(float) * S.m, s>>>(
                    z32[t], S.Y32.p, S.m, wv, n, out[t],
                    stream_evict_first(c, (long long)n * (4LL * h->kp + 28) + 4LL * h->D32.nnz) ? 1 : 0, nullptr);
                ASSS_CHECK_LAUNCH();
            } else {
                ASSS_TRY(sub_rowmajor_gemv(S.Y.p, S.m, wv, z64[t], n, out[t], s));
            }
        }
    } else if (fp32) {
        for (int t = 0; t < nc; ++t) ASSS_TRY(vcopy(out[t], z64[t], n, s));
    }
    return ASSS_OK;
}

static asss_status refine_block(asss_handle* h, int nb, const double* const* rhs, double* const* x,
                                asss_stats* st) {
    NvtxRange nv_("asss:solve-block");
    cudaStream_t s = h->ctx.stream;
    const int n = h->n;
    const int nbk = cdiv(n, 256);
    const asss_options& o = h->opt;
    const int B = asss_handle::BLK;
    const int M = o.restart > 0 ? o.restart : 60;
    for (int t = 0; t < nb; ++t) {
        if (!h->kwb[t]) h->kwb[t].reset(new KrylovWork());
        ASSS_TRY(h->kwb[t]->init(n, M, ASSS_OUTER_FGMRES));
    }
    if (!h->blk_r.p) {
        ASSS_TRY(h->blk_r.alloc((int64_t)B * n));
        ASSS_TRY(h->blk_rh.alloc((int64_t)B * n));
        ASSS_TRY(h->blk_dy.alloc((int64_t)B * n));
        ASSS_TRY(h->blk_z64.alloc((int64_t)B * n));
        if (o.precision == ASSS_PREC_MIXED) ASSS_TRY(h->blk_z32.alloc((int64_t)B * n));
        ASSS_TRY(h->blk_G.alloc((int64_t)B * (h->k + 1)));
        ASSS_TRY(h->blk_T.alloc((int64_t)B * (h->k + h->r + 2)));
    }
    if (!h->t1.p) {
        set_error("internal: work vectors missing");
        return ASSS_ERR_CUDA;
    }
    ASSS_TRY(mrs_collect(h->ctx, h->mw, nullptr));
    mrs_take_totals(h->mw);
    double* r[B];
    double* rh[B];
    double* dy[B];
    double bn[B], best[B];
    int stall[B], active[B];
    long long its_sum = 0;
    int launches = 0;
    MrsTotals mt;
    int* perm = h->has_perm ? h->perm.p : nullptr;
    for (int t = 0; t < nb; ++t) {
        r[t] = h->blk_r.p + (size_t)t * n;
        rh[t] = h->blk_rh.p + (size_t)t * n;
        dy[t] = h->blk_dy.p + (size_t)t * n;
        st[t] = h->setup_stats;
        st[t].outer_its = 0;
        st[t].cycles = 0;
        st[t].relres = 0.0;
        st[t].status = ASSS_OK;
        ASSS_CUDA(cudaMemsetAsync(x[t], 0, sizeof(double) * n, s));
        ASSS_TRY(vcopy(r[t], rhs[t], n, s));
        ASSS_TRY(dot(rhs[t], rhs[t], n, h->kwb[t]->T.p + 8, s));
        best[t] = INFINITY;
        stall[t] = 0;
    }
    std::vector<double> hv(nb);
    for (int t = 0; t < nb; ++t) {
        asss_status es = ASSS_OK;
        bn[t] = sqrt(read_scalar(h->kwb[t]->T.p + 8, s, &es));
        ASSS_TRY(es);
        active[t] = bn[t] > 0.0;
    }
    bool first = true;
    while (true) {
        // the true residual of every active column; stop tests as in refine
        for (int t = 0; t < nb; ++t)
            if (active[t] && !first) ASSS_TRY(dot(r[t], r[t], n, h->kwb[t]->T.p + 8, s));
        int na = 0;
        for (int t = 0; t < nb; ++t) {
            if (!active[t]) continue;
            double rn = bn[t];
            if (!first) {
                asss_status es = ASSS_OK;
                rn = sqrt(read_scalar(h->kwb[t]->T.p + 8, s, &es));
                ASSS_TRY(es);
            }
            st[t].relres = rn / bn[t];
            hv[t] = rn;
            if (rn / bn[t] <= o.outer_tol) {
                active[t] = 0;
            } else if (!(rn == rn)) {
                st[t].status = ASSS_ERR_BREAKDOWN;
                active[t] = 0;
            } else if (st[t].outer_its >= o.outer_maxit) {
                st[t].status = ASSS_ERR_NOT_CONVERGED;
                active[t] = 0;
            } else if (rn < 0.999 * best[t]) {
                best[t] = rn;
                stall[t] = 0;
            } else if (++stall[t] >= 5) {
                st[t].status = ASSS_ERR_STAGNATION;
                active[t] = 0;
            }
            na += active[t];
        }
        first = false;
        if (!na) break;
        // one FGMRES cycle per active column, the Arnoldi steps in lockstep
        int cols[B], nc = 0;
        double thr[B];
        int steps[B], live[B];
        for (int t = 0; t < nb; ++t) {
            if (!active[t]) continue;
            cols[nc++] = t;
            KrylovWork& kw = *h->kwb[t];
            k_to_scaled_fwd<<<nbk, 256, 0, s>>>(r[t], h->dr.p, h->w.p, perm, n, rh[t]);  // W P D_r r
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(dot(rh[t], rh[t], n, kw.T.p, s));
            k_fg_init<<<1, 1, 0, s>>>(kw.g.p, kw.m, kw.T.p, kw.T.p + 1);
            ASSS_CHECK_LAUNCH();
            ASSS_CUDA(cudaMemsetAsync(dy[t], 0, sizeof(double) * n, s));
            k_scale_dev<<<nbk, 256, 0, s>>>(kw.V.p, rh[t], kw.T.p + 1, n);
            ASSS_CHECK_LAUNCH();
        }
        std::vector<double> beta0(nb, 0.0);
        for (int q = 0; q < nc; ++q) {
            const int t = cols[q];
            asss_status es = ASSS_OK;
            beta0[t] = sqrt(read_scalar(h->kwb[t]->T.p, s, &es));
            ASSS_TRY(es);
            const double eta = fmin(0.5, 0.5 * o.outer_tol * bn[t] / hv[t]);
            const int budget = o.outer_maxit - st[t].outer_its;
            thr[t] = eta * beta0[t];
            steps[t] = 0;
            live[t] = beta0[t] > 0.0 && budget > 0;
        }
        const int mcyc = M;
        for (int j = 0; j < mcyc; ++j) {
            int lc[B], nl = 0;
            for (int q = 0; q < nc; ++q)
                if (live[cols[q]] && j < o.outer_maxit - st[cols[q]].outer_its) lc[nl++] = cols[q];
                else live[cols[q]] = 0;
            if (!nl) break;
            // z_j = P^-1 v_j for every live column in one multi-column launch
            const double* uin[B];
            double* zout[B];
            for (int q = 0; q < nl; ++q) {
                KrylovWork& kw = *h->kwb[lc[q]];
                uin[q] = kw.V.p + (size_t)j * n;
                zout[q] = kw.Z.p + (size_t)j * n;
            }
            ASSS_TRY(apply_prec_block(h, 0, nl, uin, zout, &its_sum, &launches, &mt));
            for (int q = 0; q < nl; ++q) {
                const int t = lc[q];
                KrylovWork& kw = *h->kwb[t];
                ASSS_TRY(apply_op(h, 0, kw.Z.p + (size_t)j * n, kw.w.p));
                ASSS_TRY(arnoldi_orth(h->ctx, kw.ao, kw.V.p, kw.w.p, n, j, kw.m, kw.H.p, kw.cs.p, kw.sn.p, kw.g.p,
                                      kw.hv.p, kw.hv2.p, kw.T.p + 2, kw.T.p + 3, thr[t], kw.stop.p));
                int* hi = reinterpret_cast<int*>(kw.hpin + 2);
                hi[0] = 0;
                hi[2] = 0;
                ASSS_CUDA(cudaMemcpyAsync(hi, kw.ao.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
                ASSS_CUDA(cudaMemcpyAsync(hi + 2, kw.stop.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            }
            ASSS_CUDA(cudaStreamSynchronize(s));
            for (int q = 0; q < nl; ++q) {
                const int t = lc[q];
                KrylovWork& kw = *h->kwb[t];
                const int* hi = reinterpret_cast<const int*>(kw.hpin + 2);
                if (hi[0]) {
                    kw.ao.n = 0;
                    set_error("a device wait in the Arnoldi step ran out (status %d)", hi[0]);
                    return (asss_status)hi[0];
                }
                steps[t] = j + 1;
                if (hi[2]) live[t] = 0;
            }
        }
        for (int q = 0; q < nc; ++q) {
            const int t = cols[q];
            KrylovWork& kw = *h->kwb[t];
            if (steps[t] > 0) {
                k_fg_backsolve<<<1, 1, 0, s>>>(kw.H.p, kw.g.p, steps[t], kw.m, kw.y.p);
                ASSS_CHECK_LAUNCH();
                ASSS_TRY(colmajor_gemv(kw.Z.p, n, steps[t], kw.y.p, n, 0.0, dy[t], s));
            }
            st[t].outer_its += steps[t];
            st[t].cycles += 1;
            ASSS_TRY(vmul(h->t1.p, h->w.p, dy[t], n, s));  // x += D_c S W dy
            ASSS_TRY(spmv(h->S, h->t1.p, h->t2.p, nullptr, s));
            k_axpy_mul<<<nbk, 256, 0, s>>>(x[t], h->dc.p, h->t2.p, n);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(spmv(h->A, x[t], h->t1.p, nullptr, s));
            k_sub<<<nbk, 256, 0, s>>>(rhs[t], h->t1.p, r[t], n);
            ASSS_CHECK_LAUNCH();
        }
    }
    for (int t = 0; t < nb; ++t) {
        st[t].inner_its_total = its_sum;
        st[t].inner_solves = launches;
        st[t].inner_its_avg = launches ? (double)its_sum / launches : 0.0;
        st[t].t_inner_ms = mt.ms;
        st[t].inner_bytes = mt.bytes;
        st[t].inner_launches = mt.launches;
    }
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// SELL-C-sigma autotuner: J~ in general patterns is stored with a sorting window sigma
// and cut into work units of `split` entries per lane; the best pair depends on the row
// length distribution and on locality (a larger window pads less but scatters a slice's
// rows further apart).  Each candidate is built in FP32 and timed on four mrs steps
// (k = 0, the operator dominates); the fastest is kept.
// ---------------------------------------------------------------------------
static asss_status tune_sell(asss_handle* h, int* sigma_out, int* split_out) {
    NvtxRange nv_("asss:sell-tuner");
    const Ctx& c = h->ctx;
    const int n = h->n;
    const int cand[][2] = {{4096, 1024}, {1024, 1024}, {16384, 1024}, {4096, 256}, {4096, 4096}};
    MrsWork* w = nullptr;
    ASSS_TRY(mrs_work_create(&w, n, c.sms));
    struct WGuard {
        MrsWork* w;
        ~WGuard() { mrs_work_destroy(w); }
    } wg{w};
    DBuf<float> x32;
    DBuf<double> alpha;
    ASSS_TRY(x32.alloc(n));
    ASSS_TRY(alpha.alloc(1));
    double best = INFINITY;
    *sigma_out = 0;
    *split_out = 0;
    for (const auto& cd : cand) {
        DSell<float> J;
        ASSS_TRY(build_sell<float>(h->Jt, true, J, c.stream, cd[0], cd[1]));
        MrsOperator op;
        op.J32 = &J;
        op.k = 0;
        op.kp = 0;
        op.alpha = alpha.p;
        double ms = 0.0;
        for (int rep = 0; rep < 2; ++rep) {   // the second run is timed
            MrsResult r;
            ASSS_TRY(mrs_solve(c, w, op, true, 1.0, 1.0, h->d.p, nullptr, x32.p, 0.0, 4, nullptr, &r, true));
            ms = r.ms;
        }
        mrs_take_totals(w);
        if (ms < best) {
            best = ms;
            *sigma_out = J.sigma > 0 ? cd[0] : 0;
            *split_out = cd[1];
        }
        if (J.sigma == 0) break;   // rows of even length: no window is built, nothing to tune
    }
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------
static asss_status do_setup(asss_handle* h, const asss_csr* Ain, asss_stats* st) {
    NvtxRange nv_("asss:setup");
    const asss_options& o = h->opt;
    Ctx& c = h->ctx;
    cudaStream_t s = c.stream;
    if (o.k_lanczos < 0 || o.gamma <= 0 || o.inner_maxit < 1 || o.outer_maxit < 0 ||
        (o.precision != ASSS_PREC_FP64 && o.precision != ASSS_PREC_MIXED) ||
        (o.outer != ASSS_OUTER_TFQMR && o.outer != ASSS_OUTER_FGMRES) || (o.outer == ASSS_OUTER_FGMRES && o.restart < 1) ||
        o.inner_format < ASSS_FORMAT_AUTO || o.inner_format > ASSS_FORMAT_DIAG ||
        (o.scaling != ASSS_SCALING_MAXES && o.scaling != ASSS_SCALING_MATCHING) ||
        (o.factor != ASSS_FACTOR_DIAG && o.factor != ASSS_FACTOR_ILDL0 && o.factor != ASSS_FACTOR_ILDL0_BK)) {
        set_error("invalid option");
        return ASSS_ERR_ARG;
    }
    if (o.factor != ASSS_FACTOR_DIAG && o.q_bf16) {
        set_error("the incomplete factor reads Q_k in FP32 or FP64 only (q_bf16 unsupported)");
        return ASSS_ERR_UNSUPPORTED;
    }
    ASSS_TRY(upload_csr(Ain, h->A, true, s));
    int n = h->A.n;
    h->n = n;
    // Eq. mc64 by the maximum-product matching (the role of MC64) when nothing is given
    const bool match = o.scaling == ASSS_SCALING_MATCHING && !o.row_perm && !o.dr && !o.dc;
    // scalings (Eq. mc64, reading: row max then column max unless given)
    ASSS_TRY(h->dr.alloc(n));
    ASSS_TRY(h->dc.alloc(n));
    DBuf<int> flag;
    ASSS_TRY(flag.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    DBuf<double> tmp;
    ASSS_TRY(tmp.alloc(n));
    if (match) {
        ASSS_TRY(h->perm.alloc(n));
        ASSS_TRY(matching_scaling(c, h->A, h->perm.p, h->dr.p, h->dc.p, nullptr, nullptr));
        h->has_perm = true;
    } else if (o.dr) {
        DBuf<double> t;
        ASSS_TRY(to_device(t, o.dr, n, s));
        ASSS_TRY(vcopy(h->dr.p, t.p, n, s));
    } else {
        k_rowmax_abs<<<cdiv(n, 256), 256, 0, s>>>(h->A.rp.p, h->A.v.p, n, tmp.p);
        ASSS_CHECK_LAUNCH();
        k_recip_check<<<cdiv(n, 256), 256, 0, s>>>(tmp.p, n, h->dr.p, flag.p);
        ASSS_CHECK_LAUNCH();
    }
    if (match) {
        // dc came with the matching
    } else if (o.dc) {
        DBuf<double> t;
        ASSS_TRY(to_device(t, o.dc, n, s));
        ASSS_TRY(vcopy(h->dc.p, t.p, n, s));
    } else {
        DBuf<unsigned long long> cm;
        ASSS_TRY(cm.alloc(n));
        ASSS_CUDA(cudaMemsetAsync(cm.p, 0, sizeof(unsigned long long) * n, s));
        k_colmax_abs<<<cdiv(n, 256), 256, 0, s>>>(h->A.rp.p, h->A.ci.p, h->A.v.p, h->dr.p, n, cm.p);
        ASSS_CHECK_LAUNCH();
        k_recip_check<<<cdiv(n, 256), 256, 0, s>>>((const double*)cm.p, n, h->dc.p, flag.p);
        ASSS_CHECK_LAUNCH();
    }
    int hflag = 0;
    ASSS_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hflag) {
        set_error("A has an empty row or column (scaling undefined)");
        return ASSS_ERR_PATTERN;
    }
    if (o.row_perm) {
        ASSS_TRY(to_device(h->perm, o.row_perm, n, s));
        DBuf<int> seen;
        ASSS_TRY(seen.alloc(n));
        ASSS_CUDA(cudaMemsetAsync(seen.p, 0, sizeof(int) * n, s));
        ASSS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
        k_check_perm<<<cdiv(n, 256), 256, 0, s>>>(h->perm.p, n, seen.p, flag.p);
        ASSS_CHECK_LAUNCH();
        ASSS_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        if (hflag) {
            set_error("row_perm is not a permutation of 0..n-1");
            return ASSS_ERR_ARG;
        }
        h->has_perm = true;
    }
    {
        DBuf<int> len;
        ASSS_TRY(len.alloc(n));
        k_perm_rowlen<<<cdiv(n, 256), 256, 0, s>>>(h->A.rp.p, h->has_perm ? h->perm.p : nullptr, n, len.p);
        ASSS_CHECK_LAUNCH();
        h->Abar.n = n;
        h->Abar.nnz = h->A.nnz;
        ASSS_TRY(h->Abar.rp.alloc(n + 1));
        ASSS_TRY(exclusive_scan(len.p, h->Abar.rp.p, n, nullptr, s));
        ASSS_TRY(h->Abar.ci.alloc(h->A.nnz));
        ASSS_TRY(h->Abar.v.alloc(h->A.nnz));
        k_perm_scale_rows<<<cdiv(n, 256), 256, 0, s>>>(h->A.rp.p, h->A.ci.p, h->A.v.p,
                                                        h->has_perm ? h->perm.p : nullptr, h->dr.p, h->dc.p, n,
                                                        h->Abar.rp.p, h->Abar.ci.p, h->Abar.v.p);
        ASSS_CHECK_LAUNCH();
    }
    ASSS_TRY(transpose_csr(h->Abar, h->AbarT, nullptr, s));
    // S pattern: given, or the pattern of Abar
    DCsr Spat;
    if (o.s_pattern) {
        ASSS_TRY(upload_csr(o.s_pattern, Spat, false, s));
        if (Spat.n != n) {
            set_error("s_pattern has the wrong dimension");
            return ASSS_ERR_ARG;
        }
        Spat.v.free();
    } else {
        Spat.n = n;
        Spat.nnz = h->Abar.nnz;
        ASSS_TRY(Spat.rp.alloc(n + 1));
        ASSS_TRY(Spat.ci.alloc(h->Abar.nnz));
        ASSS_CUDA(cudaMemcpyAsync(Spat.rp.p, h->Abar.rp.p, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, s));
        ASSS_CUDA(cudaMemcpyAsync(Spat.ci.p, h->Abar.ci.p, sizeof(int) * h->Abar.nnz, cudaMemcpyDeviceToDevice, s));
    }
    // the LLS (§2, App. A)
    DCsr P;
    DBuf<int> mirror, diagpos;
    DBuf<double> Cval, s_val;
    LlsResult lr;
    DBuf<double> s_start;  // saved S values to resume from (options.s_values)
    if (o.s_values) ASSS_TRY(to_device(s_start, o.s_values, Spat.nnz, s));
    ASSS_TRY(lls_fit(c, h->Abar, h->AbarT, Spat, o.gamma, o.lls_tol, o.lls_maxit, s_val, P, mirror, diagpos, Cval,
                     &lr, o.s_values ? s_start.p : nullptr));
    st->lls_its = lr.its;
    st->lls_relgrad = lr.relgrad;
    st->nnz_pattern = P.nnz;
    h->S.n = n;
    h->S.nnz = Spat.nnz;
    h->S.rp.p = Spat.rp.p;
    h->S.rp.n = Spat.rp.n;
    Spat.rp.p = nullptr;
    h->S.ci.p = Spat.ci.p;
    h->S.ci.n = Spat.ci.n;
    Spat.ci.p = nullptr;
    h->S.v.p = s_val.p;
    h->S.v.n = s_val.n;
    s_val.p = nullptr;
    // d, W, zero pivots, negative set (§3, reading: 1x1 pivots)
    ASSS_TRY(h->d.alloc(n));
    ASSS_TRY(h->w.alloc(n));
    k_diag_w<<<cdiv(n, 256), 256, 0, s>>>(Cval.p, diagpos.p, n, h->d.p, h->w.p);
    ASSS_CHECK_LAUNCH();
    h->factored = o.factor == ASSS_FACTOR_ILDL0 || o.factor == ASSS_FACTOR_ILDL0_BK;
    if (h->factored) {
        // the no-fill incomplete L D L^T of M^ (§3 after Eq. absfac, §4.1 ~ildl(0)):
        // d becomes the pivots D, W = 1 (L~ = (I + L)|D|^1/2 is applied by triangular solves)
        ASSS_TRY(vfill(h->w.p, 1.0, n, s));
        int nzero = 0;
        ASSS_TRY(ildl_build(c, P, mirror.p, Cval.p, h->d.p, o.seed, o.zero_tol, o.precision == ASSS_PREC_MIXED,
                            h->fac, &nzero, o.factor == ASSS_FACTOR_ILDL0_BK));
        if (nzero) {
            set_error("%d zero pivot(s) in the incomplete L D L^T", nzero);
            return ASSS_ERR_ZERO_DIAG;
        }
        st->factor_pairs = h->fac.npairs;
        st->factor_colours = h->fac.ncol;
    } else {
        DBuf<unsigned long long> mx;
        ASSS_TRY(mx.alloc(1));
        ASSS_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
        k_absmax<<<256, 256, 0, s>>>(h->d.p, n, mx.p);
        ASSS_CHECK_LAUNCH();
        unsigned long long bits = 0;
        ASSS_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        double dmax;
        memcpy(&dmax, &bits, sizeof(double));
        ASSS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
        k_zero_pivots<<<cdiv(n, 256), 256, 0, s>>>(h->d.p, n, o.zero_tol * dmax, flag.p);
        ASSS_CHECK_LAUNCH();
        ASSS_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        if (dmax == 0.0 || hflag) {
            set_error("%d zero pivot(s) in diag(Abar S)", hflag);
            return ASSS_ERR_ZERO_DIAG;
        }
    }
    if (h->factored && h->fac.npairs > 0) {
        // M~_r = sign(D) - I block by block (Fig. 1): the factor's U_r columns
        if (h->fac.nur > o.r_max) {
            h->prec2 = 1;
            h->r = 0;
        } else {
            h->r = h->fac.nur;
            if (h->r) {
                ASSS_TRY(h->neg.alloc(h->r));
                ASSS_CUDA(cudaMemcpyAsync(h->neg.p, h->fac.ur_i1.p, sizeof(int) * (size_t)h->r,
                                          cudaMemcpyDeviceToDevice, s));
                h->neg2 = h->fac.ur_i2.p;
                h->negc1 = h->fac.ur_c1.p;
                h->negc2 = h->fac.ur_c2.p;
            }
        }
    } else {
        DBuf<int> nf, npos;
        ASSS_TRY(nf.alloc(n));
        ASSS_TRY(npos.alloc(n + 1));
        k_neg_flag<<<cdiv(n, 256), 256, 0, s>>>(h->d.p, n, nf.p);
        ASSS_CHECK_LAUNCH();
        int64_t r = 0;
        ASSS_TRY(exclusive_scan(nf.p, npos.p, n, &r, s));
        if (r > o.r_max) {
            h->prec2 = 1;  // Eq. (preconditioner2): drop M~_r
            h->r = 0;
        } else {
            h->r = (int)r;
            if (r) {
                ASSS_TRY(h->neg.alloc(r));
                k_neg_compact<<<cdiv(n, 256), 256, 0, s>>>(nf.p, npos.p, n, h->neg.p);
                ASSS_CHECK_LAUNCH();
            }
        }
    }
    // J~ on P (exactly skew), SELL copies
    h->Jt.n = n;
    h->Jt.nnz = P.nnz;
    h->Jt.rp.p = P.rp.p;
    h->Jt.rp.n = P.rp.n;
    P.rp.p = nullptr;
    h->Jt.ci.p = P.ci.p;
    h->Jt.ci.n = P.ci.n;
    P.ci.p = nullptr;
    ASSS_TRY(h->Jt.v.alloc(h->Jt.nnz));
    k_assemble_jt<<<cdiv(n, 256), 256, 0, s>>>(n, h->Jt.rp.p, h->Jt.ci.p, mirror.p, Cval.p, h->w.p, h->Jt.v.p);
    ASSS_CHECK_LAUNCH();
    if (h->factored) {
        // Jt holds J^ itself (W = 1); the inner kernel applies L~^-1 J^ L~^-T
        ASSS_TRY(ildl_set_skew(c, h->fac, h->Jt, o.precision == ASSS_PREC_MIXED));
        ASSS_TRY(h->fa.alloc(n));
        ASSS_TRY(h->fb.alloc(n));
    } else if (o.inner_format != ASSS_FORMAT_SELL) {
        int ok = 0;
        ASSS_TRY(build_skew_dia<double>(h->Jt, 64, 0.5, h->D64, &ok, s));
        if (ok && o.precision == ASSS_PREC_MIXED) ASSS_TRY(build_skew_dia<float>(h->Jt, 64, 0.5, h->D32, &ok, s));
        h->use_dia = ok != 0;
        if (!ok && o.inner_format == ASSS_FORMAT_DIAG) {
            set_error("J~ does not qualify for skew diagonal storage");
            return ASSS_ERR_UNSUPPORTED;
        }
    }
    if (!h->use_dia && !h->factored) {
        int sigma = o.sell_sigma, split = o.sell_split;
        if (sigma == 0 && split == 0 && o.precision == ASSS_PREC_MIXED && n >= 100000)
            ASSS_TRY(tune_sell(h, &sigma, &split));
        ASSS_TRY(build_sell<double>(h->Jt, true, h->J64, s, sigma, split));
        if (o.precision == ASSS_PREC_MIXED) ASSS_TRY(build_sell<float>(h->Jt, true, h->J32, s, sigma, split));
        st->sell_sigma = h->J64.sigma;
        st->sell_split = h->J64.split;
    }
    // outer operator pieces: W Abar and S W
    ASSS_TRY(copy_csr(h->Abar, h->Aw, s));
    k_scale_rows<<<cdiv(n, 256), 256, 0, s>>>(h->Aw.rp.p, h->Aw.v.p, h->w.p, n);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(copy_csr(h->S, h->Sw, s));
    k_scale_cols<<<cdiv(n, 256), 256, 0, s>>>(h->Sw.rp.p, h->Sw.ci.p, h->Sw.v.p, h->w.p, n);
    ASSS_CHECK_LAUNCH();
    // stencil-like matrices also get a diagonal copy for the solve-phase products
    {
        int ok = 0;
        for (DCsr* M : {&h->Aw, &h->Sw, &h->A, &h->S}) ASSS_TRY(attach_dia(*M, 16, 0.5, &ok, s));
    }
    // skew-Lanczos (§3.2, Fig. 2)
    {
        DBuf<double> q1;
        ASSS_TRY(q1.alloc(n));
        ASSS_TRY(splitmix64_fill(o.seed, n, q1.p, s));
        ASSS_TRY(lanczos(c, h->Jt, q1.p, n, o.k_lanczos, o.reorth, h->Qcm, h->alpha_h, &h->k,
                         h->factored ? &h->fac : nullptr, h->fa.p, h->fb.p));
    }
    h->kp = pick_kp(h->k);
    if (h->kp < 0) {
        set_error("k_lanczos above 64 is not supported by this build");
        return ASSS_ERR_UNSUPPORTED;
    }
    if (h->k > 1) ASSS_TRY(to_device(h->alpha_d, h->alpha_h.data(), (int64_t)h->alpha_h.size(), s));
    else ASSS_TRY(h->alpha_d.alloc(1));
    bool qb = o.q_bf16 && o.precision == ASSS_PREC_MIXED && h->k > 0;
    if (qb) {
        // Q' = bf16(Q): every later use (SMW set-up in FP64, U^T z, the inner kernel) sees Q'
        k_round_bf16<<<cdiv((int64_t)n * h->k, 256), 256, 0, s>>>(h->Qcm.p, (int64_t)n * h->k);
        ASSS_CHECK_LAUNCH();
        h->kp16 = (h->k + 7) / 8 * 8;
        if (h->kp16 == 40 || h->kp16 == 56) h->kp16 += 8;
        ASSS_TRY(h->Q16.alloc((int64_t)n * h->kp16));
        k_to_rowmajor_bf16<<<cdiv((int64_t)n * h->kp16, 256), 256, 0, s>>>(h->Qcm.p, n, h->k, n, h->kp16, h->Q16.p);
        ASSS_CHECK_LAUNCH();
    }
    if (h->kp) {
        ASSS_TRY(h->Q64.alloc((int64_t)n * h->kp));
        ASSS_TRY(to_rowmajor(h->Qcm.p, n, h->k, n, h->kp, h->Q64.p, s));
        if (o.precision == ASSS_PREC_MIXED && !qb) {
            ASSS_TRY(h->Q32.alloc((int64_t)n * h->kp));
            ASSS_TRY(to_rowmajor_f(h->Qcm.p, n, h->k, n, h->kp, h->Q32.p, s));
        }
    }
    // work buffers and the mrs workspace
    ASSS_TRY(h->t1.alloc(n));
    ASSS_TRY(h->t2.alloc(n));
    ASSS_TRY(h->t3.alloc(n));
    ASSS_TRY(h->zt.alloc(n));
    ASSS_TRY(h->wv.alloc(h->k + h->r + 1));
    if (o.precision == ASSS_PREC_MIXED) ASSS_TRY(h->z32.alloc(n));
    ASSS_TRY(mrs_work_create(&h->mw, n, c.sms));
    // SMW data for P^-1 (Eq. smw; S_bar X = U_bar by mrs)
    ASSS_TRY(ensure_smw(h, 0));
    ASSS_CUDA(cudaStreamSynchronize(s));
    st->r = h->r;
    st->k_eff = h->k;
    st->prec2 = h->prec2;
    return ASSS_OK;
}

// ===========================================================================
// exported functions
// ===========================================================================
extern "C" {

void asss_default_options(asss_options* opt) {
    if (opt) fill_defaults(opt);
}

const char* asss_status_str(asss_status s) {
    switch (s) {
        case ASSS_OK: return "ok";
        case ASSS_ERR_ARG: return "invalid argument";
        case ASSS_ERR_PATTERN: return "malformed sparsity pattern";
        case ASSS_ERR_ZERO_DIAG: return "zero pivot in the diagonal factor";
        case ASSS_ERR_BREAKDOWN: return "breakdown";
        case ASSS_ERR_NOT_CONVERGED: return "not converged";
        case ASSS_ERR_STAGNATION: return "stagnation";
        case ASSS_ERR_RANK: return "rank above r_max";
        case ASSS_ERR_TIMEOUT: return "device wait timed out";
        case ASSS_ERR_OOM: return "out of device memory";
        case ASSS_ERR_CUDA: return "CUDA error";
        case ASSS_ERR_UNSUPPORTED: return "unsupported input";
    }
    return "unknown status";
}

const char* asss_last_error(void) { return get_error(); }

unsigned long long asss_kernel_launches(void) { return launches(); }

asss_status asss_setup(const asss_csr* A, const asss_options* opt, asss_handle** out, asss_stats* st) {
    if (!out) {
        set_error("out is NULL");
        return ASSS_ERR_ARG;
    }
    *out = nullptr;
    set_error("");
    auto t0 = std::chrono::steady_clock::now();
    asss_handle* h = new asss_handle();
    if (opt) h->opt = *opt;
    else fill_defaults(&h->opt);
    asss_stats lst;
    memset(&lst, 0, sizeof(lst));
    asss_status s = make_ctx(h->ctx, h->opt.stream, h->opt.wait_timeout_ms);
    if (s == ASSS_OK) s = do_setup(h, A, &lst);
    if (s != ASSS_OK) {
        cudaStreamSynchronize(h->ctx.stream);
        delete h;
        lst.status = s;
        if (st) *st = lst;
        return s;
    }
    lst.t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    lst.status = ASSS_OK;
    h->setup_stats = lst;
    if (st) *st = lst;
    *out = h;
    return ASSS_OK;
}

void asss_destroy(asss_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->ctx.stream);
    delete h;
}

static asss_status solve_common(asss_handle* h, int tr, int nrhs, const double* b, int64_t ldb, double* x,
                                int64_t ldx, const double* xfwd, int64_t ldxf, double* dA, asss_stats* st) {
    if (!h || nrhs < 0 || (nrhs > 0 && (!b || !x)) || ldb < h->n || ldx < h->n) {
        set_error("invalid solve arguments");
        return ASSS_ERR_ARG;
    }
    set_error("");
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    auto t0 = std::chrono::steady_clock::now();
    bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    DBuf<double>& xf = h->xf_stage;    // staging of host x / dA for the gradient, kept by the handle
    DBuf<double>& dAd = h->dA_stage;
    if (!h->bb.p) {
        ASSS_TRY(h->bb.alloc(n));
        ASSS_TRY(h->xx.alloc(n));
    }
    DBuf<double>& bb = h->bb;
    DBuf<double>& xx = h->xx;
    asss_stats lst = h->setup_stats;
    asss_status worst = ASSS_OK;
    // several right-hand sides of a forward FGMRES solve: lockstep blocks of up to 8
    // columns whose preconditioner applications share each pass over J~ and Q_k
    const bool block = h->opt.rhs_block && !tr && nrhs >= 2 && h->opt.outer == ASSS_OUTER_FGMRES &&
                       h->kp <= MRS_MULTI_KPMAX && !h->Q16.p && !h->factored;
    if (block) {
        const int B = asss_handle::BLK;
        if (!h->blk_b.p) {
            ASSS_TRY(h->blk_b.alloc((int64_t)B * n));
            ASSS_TRY(h->blk_x.alloc((int64_t)B * n));
        }
        long long its_all = 0, bytes_all = 0;
        int outer_max = 0, cycles = 0, solves = 0, mlaunch = 0;
        double ms_all = 0.0;
        double relres_max = 0.0;
        for (int j0 = 0; j0 < nrhs; j0 += B) {
            const int nb = nrhs - j0 < B ? nrhs - j0 : B;
            const double* bp[B];
            double* xp[B];
            for (int t = 0; t < nb; ++t) {
                if (bdev) {
                    bp[t] = b + (size_t)(j0 + t) * ldb;
                } else {
                    ASSS_CUDA(cudaMemcpyAsync(h->blk_b.p + (size_t)t * n, b + (size_t)(j0 + t) * ldb,
                                              sizeof(double) * n, cudaMemcpyHostToDevice, s));
                    bp[t] = h->blk_b.p + (size_t)t * n;
                }
                xp[t] = xdev ? x + (size_t)(j0 + t) * ldx : h->blk_x.p + (size_t)t * n;
            }
            asss_stats bst[B];
            ASSS_TRY(refine_block(h, nb, bp, xp, bst));
            for (int t = 0; t < nb; ++t) {
                if (!xdev)
                    ASSS_CUDA(cudaMemcpyAsync(x + (size_t)(j0 + t) * ldx, xp[t], sizeof(double) * n,
                                              cudaMemcpyDeviceToHost, s));
                if (bst[t].status != ASSS_OK && worst == ASSS_OK) worst = (asss_status)bst[t].status;
                outer_max = std::max(outer_max, bst[t].outer_its);
                cycles += bst[t].cycles;
                relres_max = std::max(relres_max, bst[t].relres);
            }
            its_all += bst[0].inner_its_total;
            solves += bst[0].inner_solves;
            ms_all += bst[0].t_inner_ms;
            bytes_all += bst[0].inner_bytes;
            mlaunch += bst[0].inner_launches;
            ASSS_CUDA(cudaStreamSynchronize(s));
        }
        lst.outer_its = outer_max;
        lst.cycles = cycles;
        lst.relres = relres_max;
        lst.inner_its_total = its_all;
        lst.inner_solves = solves;
        lst.inner_its_avg = solves ? (double)its_all / solves : 0.0;
        lst.t_inner_ms = ms_all;          // the multi-column mrs launches
        lst.inner_bytes = bytes_all;
        lst.inner_launches = mlaunch;
        nrhs = 0;   // every column is done
    }
    for (int j = 0; j < nrhs; ++j) {
        ASSS_CUDA(cudaMemcpyAsync(bb.p, b + (size_t)j * ldb, sizeof(double) * n,
                                  bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        double* xt = xdev ? x + (size_t)j * ldx : xx.p;
        ASSS_TRY(refine(h, tr, bb.p, xt, &lst));
        if (!xdev) {
            ASSS_CUDA(cudaMemcpyAsync(x + (size_t)j * ldx, xt, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        }
        if (tr && xfwd && dA) {
            bool fdev = is_device_ptr(xfwd), adev = is_device_ptr(dA);
            const double* xf_p = xfwd + (size_t)j * ldxf;
            if (!fdev) {
                if (xf.n < n) ASSS_TRY(xf.alloc(n));
                ASSS_CUDA(cudaMemcpyAsync(xf.p, xf_p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
                xf_p = xf.p;
            }
            double* dA_p = dA + (size_t)j * h->A.nnz;
            if (!adev) {
                if (dAd.n < h->A.nnz) ASSS_TRY(dAd.alloc(h->A.nnz));
                dA_p = dAd.p;
            }
            k_grad_A<<<cdiv(n, 256), 256, 0, s>>>(h->A.rp.p, h->A.ci.p, xt, xf_p, n, dA_p);
            ASSS_CHECK_LAUNCH();
            if (!adev) {
                ASSS_CUDA(cudaMemcpyAsync(dA + (size_t)j * h->A.nnz, dA_p, sizeof(double) * h->A.nnz,
                                          cudaMemcpyDeviceToHost, s));
            }
        }
        ASSS_CUDA(cudaStreamSynchronize(s));
        if (lst.status != ASSS_OK && worst == ASSS_OK) worst = (asss_status)lst.status;
    }
    lst.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    lst.status = worst;
    if (st) *st = lst;
    if (worst != ASSS_OK) set_error("solve ended with status %d (%s)", (int)worst, asss_status_str(worst));
    return worst;
}

asss_status asss_solve(asss_handle* h, int nrhs, const double* b, int64_t ldb, double* x, int64_t ldx,
                       asss_stats* st) {
    return solve_common(h, 0, nrhs, b, ldb, x, ldx, nullptr, 0, nullptr, st);
}

asss_status asss_solve_adjoint(asss_handle* h, int nrhs, const double* g, int64_t ldg, double* lambda, int64_t ldl,
                               const double* x, int64_t ldx, double* dA, asss_stats* st) {
    if (h && x && ldx < h->n) {
        set_error("ldx < n");
        return ASSS_ERR_ARG;
    }
    return solve_common(h, 1, nrhs, g, ldg, lambda, ldl, x, ldx, dA, st);
}

asss_status asss_apply_operator(asss_handle* h, int transpose, const double* v, double* out) {
    if (!h || !v || !out) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    DBuf<double> vi, vo;
    ASSS_TRY(to_device(vi, v, n, s));
    ASSS_TRY(vo.alloc(n));
    ASSS_TRY(apply_op(h, transpose ? 1 : 0, vi.p, vo.p));
    ASSS_CUDA(cudaMemcpyAsync(out, vo.p, sizeof(double) * n, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status asss_apply_preconditioner(asss_handle* h, int transpose, const double* u, double* out, asss_stats* st) {
    if (!h || !u || !out) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    DBuf<double> vi, vo;
    ASSS_TRY(to_device(vi, u, n, s));
    ASSS_TRY(vo.alloc(n));
    ASSS_TRY(mrs_collect(h->ctx, h->mw, nullptr));
    mrs_take_totals(h->mw);
    ASSS_TRY(apply_prec(h, transpose ? 1 : 0, vi.p, vo.p));
    ASSS_CUDA(cudaMemcpyAsync(out, vo.p, sizeof(double) * n, cudaMemcpyDefault, s));
    ASSS_TRY(mrs_collect(h->ctx, h->mw, nullptr));
    MrsTotals t = mrs_take_totals(h->mw);
    if (st) {
        *st = h->setup_stats;
        st->inner_its_total = t.its;
        st->inner_solves = t.launches;
        st->inner_its_avg = (double)t.its;
        st->t_inner_ms = t.ms;
        st->inner_bytes = t.bytes;
        st->inner_launches = t.launches;
    }
    return ASSS_OK;
}

asss_status asss_export(asss_handle* h, double* dr, double* dc, double* w, double* d, double* s_val, double* q,
                        double* alpha, int32_t* neg) {
    if (!h) {
        set_error("handle is NULL");
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = h->ctx.stream;
    int n = h->n;
    if (dr) ASSS_CUDA(cudaMemcpyAsync(dr, h->dr.p, sizeof(double) * n, cudaMemcpyDefault, s));
    if (dc) ASSS_CUDA(cudaMemcpyAsync(dc, h->dc.p, sizeof(double) * n, cudaMemcpyDefault, s));
    if (w) ASSS_CUDA(cudaMemcpyAsync(w, h->w.p, sizeof(double) * n, cudaMemcpyDefault, s));
    if (d) ASSS_CUDA(cudaMemcpyAsync(d, h->d.p, sizeof(double) * n, cudaMemcpyDefault, s));
    if (s_val) ASSS_CUDA(cudaMemcpyAsync(s_val, h->S.v.p, sizeof(double) * h->S.nnz, cudaMemcpyDefault, s));
    if (q && h->k) ASSS_CUDA(cudaMemcpyAsync(q, h->Qcm.p, sizeof(double) * (size_t)n * h->k, cudaMemcpyDefault, s));
    if (alpha && h->k > 1)
        ASSS_CUDA(cudaMemcpyAsync(alpha, h->alpha_d.p, sizeof(double) * (h->k - 1), cudaMemcpyDefault, s));
    if (neg && h->r) ASSS_CUDA(cudaMemcpyAsync(neg, h->neg.p, sizeof(int) * h->r, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status asss_export_factor(asss_handle* h, int32_t* colour, int64_t* l_row_ptr, int32_t* l_col, double* l_val,
                               int64_t l_cap, int64_t* l_nnz) {
    if (!h) {
        set_error("handle is NULL");
        return ASSS_ERR_ARG;
    }
    if (!h->factored) {
        set_error("the handle has no incomplete factor (options.factor)");
        return ASSS_ERR_ARG;
    }
    IldlFactor& F = h->fac;
    const int n = h->n;
    if (l_nnz) *l_nnz = F.nl;
    if ((l_col || l_val) && l_cap < F.nl) {
        set_error("l_cap %lld below the %lld entries of L", (long long)l_cap, (long long)F.nl);
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = h->ctx.stream;
    if (colour) ASSS_CUDA(cudaMemcpyAsync(colour, F.colour.p, sizeof(int) * n, cudaMemcpyDefault, s));
    if (l_row_ptr) {
        std::vector<int> rp(n + 1);
        ASSS_CUDA(cudaMemcpyAsync(rp.data(), F.lrp.p, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i <= n; ++i) l_row_ptr[i] = rp[i];
    }
    if (l_col && F.nl) ASSS_CUDA(cudaMemcpyAsync(l_col, F.lci.p, sizeof(int) * F.nl, cudaMemcpyDefault, s));
    if (l_val && F.nl) ASSS_CUDA(cudaMemcpyAsync(l_val, F.lv.p, sizeof(double) * F.nl, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status asss_export_pivots(asss_handle* h, int32_t* partner, double* d_off, int32_t* ur_i1, int32_t* ur_i2,
                               double* ur_c1, double* ur_c2, int* npairs) {
    if (!h) {
        set_error("handle is NULL");
        return ASSS_ERR_ARG;
    }
    if (!h->factored) {
        set_error("the handle has no incomplete factor (options.factor)");
        return ASSS_ERR_ARG;
    }
    IldlFactor& F = h->fac;
    if (npairs) *npairs = F.npairs;
    if (F.npairs == 0) return ASSS_OK;
    const int n = h->n, r = h->r;
    cudaStream_t s = h->ctx.stream;
    if (partner) ASSS_CUDA(cudaMemcpyAsync(partner, F.part.p, sizeof(int) * n, cudaMemcpyDefault, s));
    if (d_off) ASSS_CUDA(cudaMemcpyAsync(d_off, F.doff.p, sizeof(double) * n, cudaMemcpyDefault, s));
    if (r > 0) {
        if (ur_i1) ASSS_CUDA(cudaMemcpyAsync(ur_i1, F.ur_i1.p, sizeof(int) * r, cudaMemcpyDefault, s));
        if (ur_i2) ASSS_CUDA(cudaMemcpyAsync(ur_i2, F.ur_i2.p, sizeof(int) * r, cudaMemcpyDefault, s));
        if (ur_c1) ASSS_CUDA(cudaMemcpyAsync(ur_c1, F.ur_c1.p, sizeof(double) * r, cudaMemcpyDefault, s));
        if (ur_c2) ASSS_CUDA(cudaMemcpyAsync(ur_c2, F.ur_c2.p, sizeof(double) * r, cudaMemcpyDefault, s));
    }
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status asss_skew_symmetrizer(const asss_csr* Abar_in, const asss_csr* s_pattern, const asss_options* opt,
                                  double* s_val, asss_stats* st) {
    asss_options o;
    if (opt) o = *opt;
    else fill_defaults(&o);
    Ctx c;
    ASSS_TRY(make_ctx(c, o.stream, o.wait_timeout_ms));
    if (!s_pattern || !s_val || o.gamma <= 0) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    DCsr Abar, AbarT, Spat, P;
    ASSS_TRY(upload_csr(Abar_in, Abar, true, c.stream));
    ASSS_TRY(upload_csr(s_pattern, Spat, false, c.stream));
    Spat.v.free();
    if (Spat.n != Abar.n) {
        set_error("pattern dimension mismatch");
        return ASSS_ERR_ARG;
    }
    ASSS_TRY(transpose_csr(Abar, AbarT, nullptr, c.stream));
    DBuf<int> mirror, diagpos;
    DBuf<double> Cval, sv;
    LlsResult lr;
    ASSS_TRY(lls_fit(c, Abar, AbarT, Spat, o.gamma, o.lls_tol, o.lls_maxit, sv, P, mirror, diagpos, Cval, &lr));
    ASSS_CUDA(cudaMemcpyAsync(s_val, sv.p, sizeof(double) * Spat.nnz, cudaMemcpyDefault, c.stream));
    ASSS_CUDA(cudaStreamSynchronize(c.stream));
    if (st) {
        memset(st, 0, sizeof(*st));
        st->lls_its = lr.its;
        st->lls_relgrad = lr.relgrad;
        st->nnz_pattern = P.nnz;
    }
    return ASSS_OK;
}

asss_status asss_skew_lanczos(const asss_csr* J, const double* q1, int k, int reorth, double* q, double* alpha,
                              int* k_eff, void* stream) {
    Ctx c;
    ASSS_TRY(make_ctx(c, stream, 2000.0));
    if (!q1 || !q || !k_eff || k < 0) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    DCsr Jd;
    ASSS_TRY(upload_csr(J, Jd, true, c.stream));
    DBuf<double> q1d, Qcm;
    ASSS_TRY(to_device(q1d, q1, Jd.n, c.stream));
    std::vector<double> al;
    int ke = 0;
    ASSS_TRY(lanczos(c, Jd, q1d.p, Jd.n, k, reorth, Qcm, al, &ke));
    *k_eff = ke;
    if (ke) ASSS_CUDA(cudaMemcpyAsync(q, Qcm.p, sizeof(double) * (size_t)Jd.n * ke, cudaMemcpyDefault, c.stream));
    if (alpha && ke > 1) {
        DBuf<double> ad;
        ASSS_TRY(to_device(ad, al.data(), ke - 1, c.stream));
        ASSS_CUDA(cudaMemcpyAsync(alpha, ad.p, sizeof(double) * (ke - 1), cudaMemcpyDefault, c.stream));
        ASSS_CUDA(cudaStreamSynchronize(c.stream));
    }
    ASSS_CUDA(cudaStreamSynchronize(c.stream));
    return ASSS_OK;
}

asss_status asss_export_permutation(asss_handle* h, int32_t* row_perm) {
    if (!h || !row_perm) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = h->ctx.stream;
    if (h->has_perm) {
        ASSS_CUDA(cudaMemcpyAsync(row_perm, h->perm.p, sizeof(int) * h->n, cudaMemcpyDefault, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
    } else {
        std::vector<int32_t> id(h->n);
        for (int i = 0; i < h->n; ++i) id[i] = i;
        ASSS_CUDA(cudaMemcpy(row_perm, id.data(), sizeof(int32_t) * h->n, cudaMemcpyDefault));
    }
    return ASSS_OK;
}

asss_status asss_matching_scaling(const asss_csr* A, int32_t* row_perm, double* dr, double* dc, int* rounds,
                                  void* stream) {
    Ctx c;
    ASSS_TRY(make_ctx(c, stream, 2000.0));
    if (!A || !row_perm || !dr || !dc) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = c.stream;
    DCsr Ad;
    ASSS_TRY(upload_csr(A, Ad, true, s));
    const int n = Ad.n;
    DBuf<int> perm;
    DBuf<double> r, cc;
    ASSS_TRY(perm.alloc(n));
    ASSS_TRY(r.alloc(n));
    ASSS_TRY(cc.alloc(n));
    ASSS_TRY(matching_scaling(c, Ad, perm.p, r.p, cc.p, rounds, nullptr));
    ASSS_CUDA(cudaMemcpyAsync(row_perm, perm.p, sizeof(int) * n, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaMemcpyAsync(dr, r.p, sizeof(double) * n, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaMemcpyAsync(dc, cc.p, sizeof(double) * n, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status asss_mrs_multi(const asss_csr* J, int k, const double* q, const double* alpha, double shift,
                           double sign, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                           int maxit, int precision, int format, int* its, double* ratio, void* stream) {
    Ctx c;
    ASSS_TRY(make_ctx(c, stream, 2000.0));
    if (!J || !B || !X || nrhs < 0 || k < 0 || (k > 0 && !q) || (k > 1 && !alpha) || maxit < 1 || !(shift > 0.0) ||
        ldb < J->n || ldx < J->n) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    if (nrhs == 0) return ASSS_OK;
    cudaStream_t s = c.stream;
    DCsr Jd;
    ASSS_TRY(upload_csr(J, Jd, true, s));
    const int n = Jd.n;
    const int kp = pick_kp(k);
    if (kp < 0 || kp > MRS_MULTI_KPMAX) {
        set_error("k above %d is not supported by the multi-column mrs", MRS_MULTI_KPMAX);
        return ASSS_ERR_UNSUPPORTED;
    }
    DSell<double> J64;
    DSell<float> J32;
    DSkewDia<double> D64;
    DSkewDia<float> D32;
    DBuf<double> Qcm, Q64, ad, bd, xd;
    DBuf<float> Q32, x32;
    const bool fp32 = precision == ASSS_PREC_MIXED;
    int dia = 0;
    if (format != ASSS_FORMAT_SELL) {
        if (fp32) ASSS_TRY(build_skew_dia<float>(Jd, 64, 0.5, D32, &dia, s));
        else ASSS_TRY(build_skew_dia<double>(Jd, 64, 0.5, D64, &dia, s));
        if (!dia && format == ASSS_FORMAT_DIAG) {
            set_error("J does not qualify for skew diagonal storage");
            return ASSS_ERR_UNSUPPORTED;
        }
    }
    if (!dia) {
        if (fp32) ASSS_TRY(build_sell<float>(Jd, false, J32, s));
        else ASSS_TRY(build_sell<double>(Jd, false, J64, s));
    }
    if (k) {
        ASSS_TRY(to_device(Qcm, q, (int64_t)n * k, s));
        if (fp32) {
            ASSS_TRY(Q32.alloc((int64_t)n * kp));
            ASSS_TRY(to_rowmajor_f(Qcm.p, n, k, n, kp, Q32.p, s));
        } else {
            ASSS_TRY(Q64.alloc((int64_t)n * kp));
            ASSS_TRY(to_rowmajor(Qcm.p, n, k, n, kp, Q64.p, s));
        }
    }
    if (k > 1) ASSS_TRY(to_device(ad, alpha, k - 1, s));
    else ASSS_TRY(ad.alloc(1));
    ASSS_TRY(bd.alloc((int64_t)n * nrhs));
    ASSS_CUDA(cudaMemcpy2DAsync(bd.p, sizeof(double) * n, B, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                                cudaMemcpyDefault, s));
    ASSS_TRY(xd.alloc((int64_t)n * nrhs));
    MrsOperator op;
    op.J64 = (fp32 || dia) ? nullptr : &J64;
    op.J32 = (fp32 && !dia) ? &J32 : nullptr;
    op.D64 = (!fp32 && dia) ? &D64 : nullptr;
    op.D32 = (fp32 && dia) ? &D32 : nullptr;
    op.k = k;
    op.kp = kp;
    op.Q64 = Q64.p;
    op.Q32 = Q32.p;
    op.alpha = ad.p;
    if (fp32) {
        ASSS_TRY(x32.alloc((int64_t)n * nrhs));
        ASSS_TRY(mrs_multi_solve(c, op, true, shift, sign, nrhs, bd.p, n, nullptr, x32.p, n, tol, maxit, its, ratio));
        k_f2d<<<cdiv((int64_t)n * nrhs, 256), 256, 0, s>>>(x32.p, xd.p, n * nrhs);
        ASSS_CHECK_LAUNCH();
    } else {
        ASSS_TRY(mrs_multi_solve(c, op, false, shift, sign, nrhs, bd.p, n, xd.p, nullptr, n, tol, maxit, its, ratio));
    }
    ASSS_CUDA(cudaMemcpy2DAsync(X, sizeof(double) * ldx, xd.p, sizeof(double) * n, sizeof(double) * n, nrhs,
                                cudaMemcpyDefault, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status asss_mrs(const asss_csr* J, int k, const double* q, const double* alpha, double shift, double sign,
                     const double* b, double* x, double tol, int maxit, int precision, int format, int* its,
                     double* ratio, void* stream) {
    Ctx c;
    ASSS_TRY(make_ctx(c, stream, 2000.0));
    if (!b || !x || k < 0 || (k > 0 && !q) || (k > 1 && !alpha) || maxit < 1 || !(shift > 0.0)) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    cudaStream_t s = c.stream;
    DCsr Jd;
    ASSS_TRY(upload_csr(J, Jd, true, s));
    int n = Jd.n;
    int kp = pick_kp(k);
    if (kp < 0) {
        set_error("k above 64 is not supported");
        return ASSS_ERR_UNSUPPORTED;
    }
    DSell<double> J64;
    DSell<float> J32;
    DSkewDia<double> D64;
    DSkewDia<float> D32;
    DBuf<double> Qcm, Q64, ad, bd, xd;
    DBuf<float> Q32, x32;
    bool fp32 = precision == ASSS_PREC_MIXED;
    int dia = 0;
    if (format != ASSS_FORMAT_SELL) {
        if (fp32) ASSS_TRY(build_skew_dia<float>(Jd, 64, 0.5, D32, &dia, s));
        else ASSS_TRY(build_skew_dia<double>(Jd, 64, 0.5, D64, &dia, s));
        if (!dia && format == ASSS_FORMAT_DIAG) {
            set_error("J does not qualify for skew diagonal storage");
            return ASSS_ERR_UNSUPPORTED;
        }
    }
    if (!dia) {
        if (fp32) ASSS_TRY(build_sell<float>(Jd, false, J32, s));
        else ASSS_TRY(build_sell<double>(Jd, false, J64, s));
    }
    if (k) {
        ASSS_TRY(to_device(Qcm, q, (int64_t)n * k, s));
        if (fp32) {
            ASSS_TRY(Q32.alloc((int64_t)n * kp));
            ASSS_TRY(to_rowmajor_f(Qcm.p, n, k, n, kp, Q32.p, s));
        } else {
            ASSS_TRY(Q64.alloc((int64_t)n * kp));
            ASSS_TRY(to_rowmajor(Qcm.p, n, k, n, kp, Q64.p, s));
        }
    }
    if (k > 1) ASSS_TRY(to_device(ad, alpha, k - 1, s));
    else ASSS_TRY(ad.alloc(1));
    ASSS_TRY(to_device(bd, b, n, s));
    ASSS_TRY(xd.alloc(n));
    MrsWork* w = nullptr;
    ASSS_TRY(mrs_work_create(&w, n, c.sms));
    MrsOperator op;
    op.J64 = (fp32 || dia) ? nullptr : &J64;
    op.J32 = (fp32 && !dia) ? &J32 : nullptr;
    op.D64 = (!fp32 && dia) ? &D64 : nullptr;
    op.D32 = (fp32 && dia) ? &D32 : nullptr;
    op.k = k;
    op.kp = kp;
    op.Q64 = Q64.p;
    op.Q32 = Q32.p;
    op.alpha = ad.p;
    MrsResult res;
    asss_status stt;
    if (fp32) {
        ASSS_TRY(x32.alloc(n));
        stt = mrs_solve(c, w, op, true, shift, sign, bd.p, nullptr, x32.p, tol, maxit, nullptr, &res, true);
        if (stt == ASSS_OK) {
            k_f2d<<<cdiv(n, 256), 256, 0, s>>>(x32.p, xd.p, n);
            stt = cudaGetLastError() == cudaSuccess ? ASSS_OK : ASSS_ERR_CUDA;
        }
    } else {
        stt = mrs_solve(c, w, op, false, shift, sign, bd.p, xd.p, nullptr, tol, maxit, nullptr, &res, true);
    }
    mrs_work_destroy(w);
    ASSS_TRY(stt);
    ASSS_CUDA(cudaMemcpyAsync(x, xd.p, sizeof(double) * n, cudaMemcpyDefault, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (its) *its = res.its;
    if (ratio) *ratio = res.ratio;
    return ASSS_OK;
}

}  // extern "C"

// ===========================================================================
// batched solves: many matrices (own set-up each) x many right-hand sides,
// one persistent launch captured in a CUDA graph
// ===========================================================================
struct asss_batch {
    asss_options opt;
    Ctx ctx;
    cudaStream_t own = nullptr;      // the batch's stream (graphs cannot capture the legacy stream)
    cudaEvent_t ev_in = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    std::vector<asss_handle*> hs;
    std::vector<int> n_of;
    std::vector<long long> off_h;
    long long total_rows = 0;
    int n_max = 0, halo_max = 0, kp = 0, qbf16 = 0, restart = 20;
    DBuf<BatchMat> mats;
    DBuf<long long> row_off;
    DBuf<double> work;
    long long work_stride = 0;
    int nblk = 0, nthreads = 0, minb = 0, tuned_nrhs = -1;
    DBuf<unsigned> counter;
    DBuf<BatchItemStat> stats;
    DBuf<unsigned long long> prof;  // ASSS_BATCH_PROFILE: phase times
    DBuf<int2> items;
    std::vector<int2> items_h;
    // mrs byte model per matrix: per step, the bytes of one column (vectors) and the bytes
    // its columns share (J~ and Q: an SpMM reads them once per step for all columns);
    // per call, the set-up and final passes of one column and the Q row they share
    std::vector<double> step_col_bytes, step_shared_bytes, call_col_bytes, call_shared_bytes;
    int items_nrhs = -1;
    DBuf<double> bdev, xdev;
    cudaGraphExec_t gexec = nullptr;
    const void* g_b = nullptr;
    const void* g_x = nullptr;
    int g_nrhs = -1, g_nt = -1, g_minb = -1;
    std::vector<cudaStream_t> setup_streams;   // streams of the concurrent set-ups (the handles keep them)
    ~asss_batch() {
        if (gexec) cudaGraphExecDestroy(gexec);
        for (asss_handle* h : hs) delete h;
        for (cudaStream_t w : setup_streams)
            if (w) cudaStreamDestroy(w);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_t0) cudaEventDestroy(ev_t0);
        if (ev_t1) cudaEventDestroy(ev_t1);
        if (own) cudaStreamDestroy(own);
    }
};

static asss_status batch_view(asss_handle* h, BatchMat* v) {
    const bool dia = h->use_dia && h->D32.n;
    if (h->opt.precision != ASSS_PREC_MIXED || (!dia && !h->J32.n)) {
        set_error("batched solves need the mixed-precision path (FP32 storage of J~)");
        return ASSS_ERR_UNSUPPORTED;
    }
    SmwData& S = h->smw[0];
    if (!S.ready || (S.m > 0 && !S.Y32.p) || S.m > 320 || h->k > 32 || (dia && h->D32.ndiag > 64)) {
        set_error("batched solves support k <= 32, k + r <= 320 and at most 64 diagonals");
        return ASSS_ERR_UNSUPPORTED;
    }
    memset(v, 0, sizeof(*v));
    v->n = h->n;
    v->k = h->k;
    v->m = S.m;
    v->r = h->r;
    if (dia) {
        v->ndiag = h->D32.ndiag;
        v->halo = h->D32.halo;
        v->ustride = h->D32.ustride;
        v->off = h->D32.off.p;
        v->U = h->D32.U.p + h->D32.halo;
    } else {   // general pattern: SELL-C-sigma
        v->ndiag = 0;
        v->halo = 0;
        v->nslots = h->J32.nslices * 32;
        v->sptr = h->J32.sptr.p;
        v->scol = h->J32.col.p;
        v->sval = h->J32.val.p;
        v->rowmap = h->J32.rowmap.p;
    }
    v->Q32 = h->Q32.p;
    v->Q16 = h->Q16.p;
    v->alpha = h->alpha_d.p;
    v->Y32 = S.Y32.p;
    v->neg = h->neg.p;
    v->arp = h->A.rp.p;
    v->aci = h->A.ci.p;
    v->av = h->A.v.p;
    v->awrp = h->Aw.rp.p;
    v->awci = h->Aw.ci.p;
    v->awv = h->Aw.v.p;
    v->swrp = h->Sw.rp.p;
    v->swci = h->Sw.ci.p;
    v->swv = h->Sw.v.p;
    v->srp = h->S.rp.p;
    v->sci = h->S.ci.p;
    v->sv = h->S.v.p;
    v->dr = h->dr.p;
    v->dc = h->dc.p;
    v->w = h->w.p;
    v->perm = h->has_perm ? h->perm.p : nullptr;
    return ASSS_OK;
}

// work items (matrix, column), largest matrices first so the tail of the launch is short
static asss_status batch_items(asss_batch* B, int nrhs) {
    if (B->items_nrhs == nrhs) return ASSS_OK;
    int nm = (int)B->hs.size();
    std::vector<int> order(nm);
    for (int i = 0; i < nm; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->n_of[a] > B->n_of[b]; });
    std::vector<int2> it;
    it.reserve((size_t)nm * nrhs);
    for (int m : order)
        for (int c = 0; c < nrhs; ++c) it.push_back(make_int2(m, c));
    ASSS_TRY(to_device(B->items, it.data(), (int64_t)it.size(), B->own));
    B->items_h = it;
    ASSS_TRY(B->stats.alloc((int64_t)it.size()));
    B->items_nrhs = nrhs;
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    return ASSS_OK;
}

static asss_status batch_run(asss_batch* B, int nrhs, const double* bd, double* xd, int nthreads, int minb,
                             bool use_graph, float* ms) {
    ASSS_TRY(batch_items(B, nrhs));
    BatchLaunch L;
    L.mats = B->mats.p;
    L.items = B->items.p;
    L.nitems = (int)B->items.n;
    L.nrhs = nrhs;
    L.row_off = B->row_off.p;
    L.b = bd;
    L.x = xd;
    L.work = B->work.p;
    L.work_stride = B->work_stride;
    L.n_max = B->n_max;
    L.halo_max = B->halo_max;
    L.kp = B->kp;
    L.qbf16 = B->qbf16;
    L.restart = B->restart;
    L.outer_tol = B->opt.outer_tol;
    L.outer_maxit = B->opt.outer_maxit;
    L.inner_tol = B->opt.inner_tol;
    L.inner_maxit = B->opt.inner_maxit;
    L.next_item = B->counter.p;
    L.stats = B->stats.p;
    L.prof = nullptr;
    // ASSS_BATCH_PROFILE=1: per-phase device time of the CTAs (the plain launch, not the
    // graph), printed to stderr; for analysis only
    const bool prof = getenv("ASSS_BATCH_PROFILE") != nullptr;
    if (prof) {
        if (!B->prof.p) ASSS_TRY(B->prof.alloc(BATCH_NPROF));
        ASSS_CUDA(cudaMemsetAsync(B->prof.p, 0, sizeof(unsigned long long) * BATCH_NPROF, B->own));
        L.prof = B->prof.p;
        use_graph = false;
    }
    int nblk = B->nblk < L.nitems ? B->nblk : L.nitems;
    if (nblk < 1) nblk = 1;
    cudaStream_t s = B->own;
    if (use_graph) {
        if (!B->gexec || B->g_b != bd || B->g_x != xd || B->g_nrhs != nrhs || B->g_nt != nthreads ||
            B->g_minb != minb) {
            if (B->gexec) {
                cudaGraphExecDestroy(B->gexec);
                B->gexec = nullptr;
            }
            cudaGraph_t g;
            ASSS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            asss_status st = ASSS_OK;
            if (cudaMemsetAsync(B->counter.p, 0, sizeof(unsigned), s) != cudaSuccess) st = ASSS_ERR_CUDA;
            if (st == ASSS_OK) st = batch_launch(L, nthreads, minb, nblk, s);
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st != ASSS_OK) return st;
            if (e != cudaSuccess) {
                set_error("graph capture failed: %s", cudaGetErrorString(e));
                return ASSS_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&B->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                set_error("graph instantiate failed: %s", cudaGetErrorString(e));
                return ASSS_ERR_CUDA;
            }
            B->g_b = bd;
            B->g_x = xd;
            B->g_nrhs = nrhs;
            B->g_nt = nthreads;
            B->g_minb = minb;
        }
        ASSS_CUDA(cudaEventRecord(B->ev_t0, s));
        ASSS_CUDA(cudaGraphLaunch(B->gexec, s));
        count_launch();
        ASSS_CUDA(cudaEventRecord(B->ev_t1, s));
    } else {
        ASSS_CUDA(cudaEventRecord(B->ev_t0, s));
        ASSS_CUDA(cudaMemsetAsync(B->counter.p, 0, sizeof(unsigned), s));
        ASSS_TRY(batch_launch(L, nthreads, minb, nblk, s));
        ASSS_CUDA(cudaEventRecord(B->ev_t1, s));
    }
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (ms) ASSS_CUDA(cudaEventElapsedTime(ms, B->ev_t0, B->ev_t1));
    if (prof) {
        unsigned long long t[BATCH_NPROF];
        ASSS_CUDA(cudaMemcpy(t, B->prof.p, sizeof(t), cudaMemcpyDeviceToHost));
        const double per = 1e-6 / (nblk > 0 ? nblk : 1);
        fprintf(stderr,
                "asss batch profile (%d threads x %d per SM, %d CTAs, launch %.2f ms; ms per CTA): mrs %.2f | smw %.2f | "
                "operator %.2f | gram-schmidt %.2f | update+residual %.2f | rest %.2f\n",
                nthreads, minb, nblk, ms ? *ms : 0.f, t[0] * per, t[1] * per, t[2] * per,
                t[3] * per, t[4] * per, t[5] * per);
    }
    return ASSS_OK;
}

// CTA shape for a number of right-hand sides: each candidate (threads per CTA and the
// resident CTAs per SM it is built for, which set the registers a thread may use: 64 at
// 1024 threads per SM, 80 at 768, 128 at 512; as many CTAs as fit on the GPU, at most one
// per item) solves the caller's batch once, timed with CUDA events; the fastest is kept
// for later calls
static asss_status batch_tune(asss_batch* B, int nrhs, const double* bd, double* xd) {
    constexpr int NC = 6;
    const int cand[NC][2] = {{256, 4}, {512, 2}, {256, 3}, {384, 2}, {256, 2}, {512, 1}};
    const long long nitems = (long long)B->hs.size() * nrhs;
    int best_nt = 0, best_minb = 0, best_nb = 0;
    float best_ms = 0.f;
    // ASSS_BATCH_CTA = "<threads>x<CTAs per SM>" restricts the tuner to that one shape
    // (tests run every shape this way)
    int force_nt = 0, force_minb = 0;
    if (const char* f = getenv("ASSS_BATCH_CTA")) {
        force_nt = atoi(f);
        const char* xpos = strchr(f, 'x');
        force_minb = xpos ? atoi(xpos + 1) : 0;
    }
    for (int c = 0; c < NC; ++c) {
        if (force_nt && (cand[c][0] != force_nt || cand[c][1] != force_minb)) continue;
        int occ = 0;
        ASSS_TRY(batch_occupancy(B->kp, B->qbf16, cand[c][0], cand[c][1], &occ));
        if (occ < 1) continue;
        long long nb = (long long)B->ctx.sms * occ;
        if (nb > nitems) nb = nitems;
        if (B->work.n < B->work_stride * nb) ASSS_TRY(B->work.alloc(B->work_stride * nb));
        B->nblk = (int)nb;
        float ms = 0.f;
        ASSS_TRY(batch_run(B, nrhs, bd, xd, cand[c][0], cand[c][1], false, &ms));
        if (!best_nt || ms < best_ms) {
            best_nt = cand[c][0];
            best_minb = cand[c][1];
            best_nb = (int)nb;
            best_ms = ms;
        }
    }
    if (!best_nt) {
        set_error("batched solver: no CTA shape fits on this device");
        return ASSS_ERR_UNSUPPORTED;
    }
    B->nthreads = best_nt;
    B->minb = best_minb;
    B->nblk = best_nb;
    B->tuned_nrhs = nrhs;
    return ASSS_OK;
}

extern "C" {

asss_status asss_setup_batched(int nmat, const asss_csr* const* A, const asss_options* opt, asss_batch** out,
                               asss_stats* st) {
    if (!out || nmat < 1 || !A) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    *out = nullptr;
    if (opt && opt->factor != ASSS_FACTOR_DIAG) {
        set_error("the batched form runs with the diagonal factor only");
        return ASSS_ERR_UNSUPPORTED;
    }
    auto t0 = std::chrono::steady_clock::now();
    asss_batch* B = new asss_batch();
    if (opt) B->opt = *opt;
    else fill_defaults(&B->opt);
    B->opt.precision = ASSS_PREC_MIXED;
    B->opt.outer = ASSS_OUTER_FGMRES;
    // J~ of each matrix: skew diagonals when its pattern fits them, SELL-C-sigma otherwise
    // (ASSS_FORMAT_AUTO), or as the options force
    B->restart = B->opt.restart > 0 ? (B->opt.restart < BATCH_RMAX ? B->opt.restart : BATCH_RMAX) : 20;
    asss_status s = make_ctx(B->ctx, B->opt.stream, B->opt.wait_timeout_ms);
    if (s == ASSS_OK && cudaStreamCreateWithFlags(&B->own, cudaStreamNonBlocking) != cudaSuccess) s = ASSS_ERR_CUDA;
    if (s == ASSS_OK && (cudaEventCreate(&B->ev_in) != cudaSuccess || cudaEventCreate(&B->ev_t0) != cudaSuccess ||
                         cudaEventCreate(&B->ev_t1) != cudaSuccess))
        s = ASSS_ERR_CUDA;
    std::vector<BatchMat> views(nmat);
    long long rows = 0;
    // The set-ups of small systems are bound by launch latency and host round trips, so
    // they run concurrently: a few host threads, each with a stream of its own, take the
    // matrices one at a time (every handle keeps the stream it was set up on).
    if (s == ASSS_OK) {
        const int nw = nmat < 8 ? nmat : 8;
        B->hs.assign(nmat, nullptr);
        B->setup_streams.assign(nw, nullptr);
        for (int w = 0; w < nw && s == ASSS_OK; ++w)
            if (cudaStreamCreateWithFlags(&B->setup_streams[w], cudaStreamNonBlocking) != cudaSuccess) {
                set_error("cudaStreamCreate failed");
                s = ASSS_ERR_CUDA;
            }
        std::atomic<int> next{0};
        std::atomic<int> failed{0};
        std::mutex mu;
        asss_status first = ASSS_OK;
        std::string first_text;
        auto worker = [&](int w) {
            if (cudaSetDevice(B->ctx.device) != cudaSuccess) {
                std::lock_guard<std::mutex> lk(mu);
                if (first == ASSS_OK) {
                    first = ASSS_ERR_CUDA;
                    first_text = "cudaSetDevice failed in a set-up thread";
                }
                failed = 1;
                return;
            }
            asss_options ow = B->opt;
            ow.stream = B->setup_streams[w];
            for (;;) {
                const int m = next.fetch_add(1);
                if (m >= nmat || failed.load()) break;
                asss_handle* h = nullptr;
                asss_stats hst;
                asss_status r = asss_setup(A[m], &ow, &h, &hst);
                if (r == ASSS_OK) {
                    B->hs[m] = h;
                    r = batch_view(h, &views[m]);
                }
                if (r != ASSS_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    if (first == ASSS_OK) {
                        first = r;
                        first_text = get_error();
                    }
                    failed = 1;
                    break;
                }
            }
            cudaStreamSynchronize(B->setup_streams[w]);
            release_thread_scratch();
        };
        if (s == ASSS_OK) {
            std::vector<std::thread> th;
            for (int w = 0; w < nw; ++w) th.emplace_back(worker, w);
            for (std::thread& t : th) t.join();
            if (first != ASSS_OK) {
                set_error("%s", first_text.c_str());
                s = first;
            }
        }
    }
    for (int m = 0; m < nmat && s == ASSS_OK; ++m) {
        asss_handle* h = B->hs[m];
        int kpm = h->Q16.p ? h->kp16 : h->kp;
        if (m == 0) {
            B->kp = kpm;
            B->qbf16 = h->Q16.p ? 1 : 0;
        } else if (kpm != B->kp || (h->Q16.p ? 1 : 0) != B->qbf16) {
            set_error("matrices of a batch must keep the same number of Lanczos vectors");
            s = ASSS_ERR_UNSUPPORTED;
            break;
        }
        // algorithmic bytes of the inner solve: per step the stored entries of J~ and the
        // Q rows - shared by all columns of the matrix, as the SpMM form of the step reads
        // them once per step - and per column y (own, old, new), p and z read and
        // written; per call the set-up pass (b in FP64, y, z, p written; Q shared) and the
        // final pass (no Q there: Q^T z follows from the reduced Q^T y of the steps)
        {
            double nn = h->n, qrow = h->Q16.p ? 2.0 * h->kp16 : 4.0 * h->kp;
            const double mat = h->use_dia ? 4.0 * (double)h->D32.nnz : 8.0 * (double)h->J32.nnz;
            B->step_col_bytes.push_back(nn * 28.0);
            B->step_shared_bytes.push_back(mat + nn * qrow);
            B->call_col_bytes.push_back(nn * (8.0 + 16.0) + nn * 16.0);
            B->call_shared_bytes.push_back(nn * qrow);
        }
        B->n_of.push_back(h->n);
        B->off_h.push_back(rows);
        rows += h->n;
        if (h->n > B->n_max) B->n_max = h->n;
        if (h->use_dia && h->D32.halo > B->halo_max) B->halo_max = h->D32.halo;
    }
    if (s == ASSS_OK) {
        B->total_rows = rows;
        s = to_device(B->mats, views.data(), nmat, B->own);
        if (s == ASSS_OK) s = to_device(B->row_off, B->off_h.data(), nmat, B->own);
        if (s == ASSS_OK) s = B->counter.alloc(1);
    }
    if (s == ASSS_OK) B->work_stride = batch_work_doubles(B->n_max, B->halo_max, B->restart);
    if (s != ASSS_OK) {
        if (B->own) cudaStreamSynchronize(B->own);
        delete B;
        if (st) {
            memset(st, 0, sizeof(*st));
            st->status = s;
        }
        return s;
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->k_eff = B->hs[0]->k;
        st->t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    *out = B;
    return ASSS_OK;
}

asss_status asss_solve_batched(asss_batch* B, int nrhs, const double* b, double* x, asss_stats* st) {
    NvtxRange nv_("asss:batched-solve");
    if (!B || nrhs < 1 || !b || !x) {
        set_error("invalid arguments");
        return ASSS_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    long long total = B->total_rows * nrhs;
    bool bdv = is_device_ptr(b), xdv = is_device_ptr(x);
    // order after the caller's stream
    ASSS_CUDA(cudaEventRecord(B->ev_in, (cudaStream_t)B->opt.stream));
    ASSS_CUDA(cudaStreamWaitEvent(B->own, B->ev_in, 0));
    const double* bd = b;
    double* xd = x;
    if (!bdv) {
        if (B->bdev.n < total) ASSS_TRY(B->bdev.alloc(total));
        ASSS_CUDA(cudaMemcpyAsync(B->bdev.p, b, sizeof(double) * total, cudaMemcpyHostToDevice, B->own));
        bd = B->bdev.p;
    }
    if (!xdv) {
        if (B->xdev.n < total) ASSS_TRY(B->xdev.alloc(total));
        xd = B->xdev.p;
    }
    if (B->tuned_nrhs != nrhs) ASSS_TRY(batch_tune(B, nrhs, bd, xd));
    float ms = 0.f;
    ASSS_TRY(batch_run(B, nrhs, bd, xd, B->nthreads, B->minb, true, &ms));
    if (!xdv) ASSS_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * total, cudaMemcpyDeviceToHost, B->own));
    std::vector<BatchItemStat> hs(B->items.n);
    ASSS_CUDA(cudaMemcpyAsync(hs.data(), B->stats.p, sizeof(BatchItemStat) * hs.size(), cudaMemcpyDeviceToHost,
                              B->own));
    ASSS_CUDA(cudaStreamSynchronize(B->own));
    asss_stats a;
    memset(&a, 0, sizeof(a));
    int worst = ASSS_OK;
    double bytes = 0.0;
    for (size_t q = 0; q < hs.size(); ++q) {
        const BatchItemStat& t = hs[q];
        const int m = B->items_h[q].x;
        bytes += t.inner_its * (B->step_col_bytes[m] + B->step_shared_bytes[m] / nrhs) +
                 t.outer_its * (B->call_col_bytes[m] + B->call_shared_bytes[m] / nrhs);
        if (t.outer_its > a.outer_its) a.outer_its = t.outer_its;
        a.inner_its_total += t.inner_its;
        a.cycles += t.cycles;
        if (t.relres > a.relres) a.relres = t.relres;
        if (t.status != ASSS_OK && worst == ASSS_OK) worst = t.status;
    }
    a.inner_solves = (int)hs.size();
    a.inner_its_avg = hs.empty() ? 0.0 : (double)a.inner_its_total / hs.size();
    a.status = worst;
    a.t_inner_ms = ms;   // device time of the batched launch
    a.inner_launches = 1;
    a.inner_bytes = (long long)bytes;
    a.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    a.k_eff = B->hs[0]->k;
    if (st) *st = a;
    if (worst != ASSS_OK) set_error("batched solve: an item ended with status %d", worst);
    return (asss_status)worst;
}

int asss_batch_cta_threads(const asss_batch* B) { return B ? B->nthreads : 0; }

int asss_batch_cta_registers(const asss_batch* B) {
    if (!B || !B->nthreads || !B->minb) return 0;
    const int r = 65536 / (B->nthreads * B->minb);
    return (r > 255 ? 255 : r) & ~7;
}

void asss_destroy_batched(asss_batch* B) {
    if (!B) return;
    if (B->own) cudaStreamSynchronize(B->own);
    delete B;
}

}  // extern "C"
