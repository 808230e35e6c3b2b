// Multi-right-hand-side mrs (paper App. B: the simultaneous iterations for
//     (shift I + sign * (J~ - Q_k S_k Q_k^T)) X = B,  B with several columns)
// as one persistent cooperative launch per group of up to MM_R columns.
//
// The columns share one pass over the operator per step: a warp covers 32/MM_R rows
// x MM_R columns, thread (row i, column c).  The MM_R lanes of a row read the same
// J~ entries and the same Q_k row (one L1 broadcast, fetched from memory once), and
// their own column of the three Lanczos vectors, which are stored interleaved (row
// i of column c at i*MM_R + c) so that the lanes of a row read consecutive words.
// Per row and step the shared data are read once for all columns instead of once
// per column (the SpMM form of the product).
//
// Every column runs its own recurrence (its own scalars beta, theta, c, s, g) on the
// same grid-wide reduction: the warp sums are segmented by column (shuffles over
// the lanes of equal column), the block partials hold MM_R x (k+1) values, and one
// bounded grid barrier per step serves all columns (§3.1's one synchronisation per
// step).  A column whose |g|/||b_c|| falls below tol freezes (reading R9); its last
// update of x runs in the next pass, and the launch ends once every column is
// frozen.  This equals independent single-column solves.
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mrs_dev.cuh"

namespace asss {

constexpr int MM_R = 8;                 // columns per launch
constexpr int MM_RPW = 32 / MM_R;       // rows per warp and pass iteration

template <class T>
struct MultiParams {
    int n, ncol;
    // SELL-C operator (rowpos: row -> slot for SELL-C-sigma, null for the identity)
    const int* sptr;
    const int* col;
    const T* val;
    const int* rowpos;
    // skew half-diagonal operator (U points at U_0[0], diagonal d starts ustride later)
    int ndiag;
    const int* off;
    const T* U;
    long long ustride;
    int halo;                 // zero rows in front of and behind each Y slot
    long long yslot;          // elements per Y slot: (n + 2 halo) * MM_R
    const T* Q;               // n x KP row-major
    const double* alpha;      // k-1 values
    int k;
    double shift, sign;
    const double* rhs[MM_R];  // column c of the right-hand side (n values, FP64)
    T* x[MM_R];               // column c of the solution (n values)
    T* Y;                     // 3 slots, row 0 of slot 0 (halo rows before it)
    T* P;                     // 2 slots of n x MM_R
    double* part;             // [2][MM_R * (KP+1)][nblk]
    GridBarrier gb;
    const int* blk_slice;
    double tol;
    int maxit;
    long long budget;
    int* out_its;             // ncol
    double* out_ratio;        // ncol
    int qcs;                  // evict-first Q row loads
};

template <class T, int KP, int FMT>
__global__ void __launch_bounds__(MRS_THREADS, 1) k_mrs_multi(MultiParams<T> p) {
    constexpr int NV = KP + 1;
    constexpr int KQ = KP > 0 ? KP : 1;
    __shared__ T s_wsum[MRS_WARPS][MM_R][NV];
    __shared__ T s_red[MM_R][NV];
    __shared__ T s_u[MM_R][KQ];
    __shared__ int s_off[FMT == 1 ? MRS_MAXDIAG : 1];
    __shared__ MrsScalars<T> sc[MM_R];
    __shared__ T s_alpha[MRS_KPMAX];
    // per column: 0 sign*nu, 1 sign, 2 beta_{j-1} nu_{j-1}, 3 nu_p, 4 delta_pp, 5 1/theta_p, 6 xcoef_p
    __shared__ T s_cf[MM_R][8];
    __shared__ int s_live[MM_R], s_pend[MM_R];
    __shared__ int s_anylive;

    const int nblk = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % MM_R, rsub = lane / MM_R;
    const bool colok = c < p.ncol;
    const int n = p.n;
    const int r0 = p.blk_slice[blockIdx.x] * 32;
    const int r1 = min(p.blk_slice[blockIdx.x + 1] * 32, n);
    volatile int* err = p.gb.err;
    if constexpr (FMT == 1) {
        for (int d = threadIdx.x; d < p.ndiag; d += MRS_THREADS) s_off[d] = p.off[d];
    }
    for (int m = threadIdx.x; m + 1 < p.k && m < MRS_KPMAX; m += MRS_THREADS) s_alpha[m] = (T)p.alpha[m];

    // segmented warp sums (lanes of equal column), then across warps in a fixed order
    // (float pairs for the FP32 solve) into this block's partials
    auto block_partials = [&](T(&tacc)[NV], double* buf) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            T d = tacc[v];
#pragma unroll
            for (int o = 16; o >= MM_R; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane < MM_R) s_wsum[warp][lane][v] = d;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < MM_R * NV; idx += MRS_THREADS) {
            const int cc = idx / NV, v = idx % NV;
            if constexpr (sizeof(T) == 4) {
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int w = 0; w < MRS_WARPS; ++w) a = df_add(a, make_float2(s_wsum[w][cc][v], 0.f));
                reinterpret_cast<float2*>(buf)[(size_t)idx * nblk + blockIdx.x] = a;
            } else {
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < MRS_WARPS; ++w) t += s_wsum[w][cc][v];
                buf[(size_t)idx * nblk + blockIdx.x] = t;
            }
        }
    };
    // every block adds the block partials in the same order (bitwise equal results)
    auto reduce_all = [&](const double* buf) {
        for (int idx = warp; idx < MM_R * NV; idx += MRS_WARPS) {
            const int cc = idx / NV, v = idx % NV;
            if (cc >= p.ncol || !s_live[cc]) continue;   // warp-uniform
            if constexpr (sizeof(T) == 4) {
                const float2* b2 = reinterpret_cast<const float2*>(buf) + (size_t)idx * nblk;
                float2 acc = make_float2(0.f, 0.f);
                for (int b = lane; b < nblk; b += 32) acc = df_add(acc, __ldcg(&b2[b]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float2 other;
                    other.x = __shfl_xor_sync(0xffffffffu, acc.x, o);
                    other.y = __shfl_xor_sync(0xffffffffu, acc.y, o);
                    acc = df_add(acc, other);
                }
                if (lane == 0) s_red[cc][v] = acc.x + acc.y;
            } else {
                double t = 0.0;
                for (int b = lane; b < nblk; b += 32) t += __ldcg(&buf[(size_t)idx * nblk + b]);
                t = warp_sum(t);
                if (lane == 0) s_red[cc][v] = t;
            }
        }
        __syncthreads();
    };
    // u_c = S_k h_c with h_c = nu_c * Q^T y_c, for the live columns (warp 0)
    auto make_u_warp0 = [&]() {
        if constexpr (KP > 0) {
            for (int idx = lane; idx < MM_R * KP; idx += 32) {
                const int cc = idx / KP, m = idx % KP;
                T u = (T)0;
                if (cc < p.ncol && s_live[cc] && m < p.k) {
                    const T nu = sc[cc].nu;
                    if (m + 1 < p.k) u += s_alpha[m] * s_red[cc][2 + m] * nu;
                    if (m > 0) u -= s_alpha[m - 1] * s_red[cc][m] * nu;
                }
                s_u[cc][m] = u;
            }
        }
    };
    auto set_coefs = [&](int cc) {   // lane cc of warp 0
        s_cf[cc][0] = (T)p.sign * sc[cc].nu;
        s_cf[cc][1] = (T)p.sign;
        s_cf[cc][2] = sc[cc].coef_old;
        s_cf[cc][3] = sc[cc].nu_p;
        s_cf[cc][4] = sc[cc].delta_pp;
        s_cf[cc][5] = sc[cc].rtheta_p;
        s_cf[cc][6] = sc[cc].xcoef_p;
    };
    unsigned phase = 0;

    // ---- phase 0: y_1 = b (interleaved), x = 0, p = 0, ||b_c||^2 and Q^T b_c ----
    T tacc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) tacc[v] = (T)0;
    for (int base = r0 + warp * MM_RPW; base < r1; base += MRS_WARPS * MM_RPW) {
        const int i = base + rsub;
        if (i < r1) {
            const size_t e = (size_t)i * MM_R + c;
            T b = colok ? (T)p.rhs[c][i] : (T)0;
            p.Y[e] = b;
            p.P[e] = (T)0;
            p.P[(size_t)n * MM_R + e] = (T)0;
            if (colok) p.x[c][i] = (T)0;
            tacc[0] += b * b;
            T q[KQ];
            load_qrow<T, KP>(p.Q, i, q, p.qcs != 0);
#pragma unroll
            for (int m = 0; m < KP; ++m) tacc[1 + m] += q[m] * b;
        }
    }
    if (threadIdx.x < MM_R) s_live[threadIdx.x] = 1;   // reduce_all reads every column once
    block_partials(tacc, p.part);
    grid_sync_phase(p.gb, nblk, phase++, p.budget);
    if (*err) return;
    reduce_all(p.part);
    if (warp == 0) {
        if (lane < MM_R) {
            const int cc = lane;
            const T zero = (T)0, one = (T)1;
            MrsScalars<T>& s = sc[cc];
            const T r0v = cc < p.ncol ? sqrt(s_red[cc][0]) : zero;
            s.r0 = r0v;
            s.rr0 = r0v > zero ? one / r0v : zero;
            s.nu = s.rr0;
            s.coef_old = zero;
            s.theta_t = (T)p.shift;
            s.c_prev = one;
            s.s_prev = zero;
            s.delta_prev = zero;
            s.G = r0v;
            s.nu_p = zero;
            s.delta_pp = zero;
            s.rtheta_p = one;
            s.xcoef_p = zero;
            s.ratio = zero;
            s.its = 0;
            s_live[cc] = (cc < p.ncol && r0v > zero) ? 1 : 0;   // a zero column gives x = 0
            s_pend[cc] = 0;
            set_coefs(cc);
        }
        __syncwarp();
        if (lane == 0) {
            int any = 0;
            for (int cc = 0; cc < MM_R; ++cc) any |= s_live[cc];
            s_anylive = any;
        }
        __syncwarp();
        make_u_warp0();
    }
    __syncthreads();

    for (int j = 1;; ++j) {
        const bool finalpass = !s_anylive;   // only the deferred updates are left
        const size_t ys = (size_t)p.yslot;
        const T* __restrict__ Ycur = p.Y + (size_t)((j - 1) % 3) * ys;
        const T* __restrict__ Yold = p.Y + (size_t)((j + 1) % 3) * ys;
        T* __restrict__ Ynew = p.Y + (size_t)(j % 3) * ys;
        T* __restrict__ Pj1 = p.P + (size_t)((j - 1) & 1) * n * MM_R;
        const bool lv = colok && s_live[c];
        const bool pd = colok && s_pend[c];
        const T tnu = s_cf[c][0], tsg = s_cf[c][1], tco = s_cf[c][2];
        const T tnp = s_cf[c][3], tdpp = s_cf[c][4], tthp = s_cf[c][5], txp = s_cf[c][6];
#pragma unroll
        for (int v = 0; v < NV; ++v) tacc[v] = (T)0;
        for (int base = r0 + warp * MM_RPW; base < r1; base += MRS_WARPS * MM_RPW) {
            const int i = base + rsub;
            if (i >= r1) continue;
            const size_t e = (size_t)i * MM_R + c;
            const T yold = ((lv || pd) && j >= 2) ? Yold[e] : (T)0;
            const T pold = pd ? Pj1[e] : (T)0;
            if (lv) {
                T acc = (T)0;
                if constexpr (FMT == 0) {
                    const int slot = p.rowpos ? __ldg(&p.rowpos[i]) : i;
                    const int sl = slot >> 5, t = slot & 31;
                    const int sb = __ldg(&p.sptr[sl]);
                    const int width = (__ldg(&p.sptr[sl + 1]) - sb) >> 5;
                    const int* cp = p.col + sb + t;
                    const T* vp = p.val + sb + t;
#pragma unroll 4
                    for (int kk = 0; kk < width; ++kk)
                        acc += __ldg(vp + kk * 32) * Ycur[(size_t)__ldg(cp + kk * 32) * MM_R + c];
                } else {
                    // (J~ y)_i = sum_d U_d[i] y[i + m_d] - U_d[i - m_d] y[i - m_d]; the zero halos
                    // of U (front) and of the Y slots (both ends) keep the loop branch-free
                    const T* Ud = p.U + i;
                    const T* yi = Ycur + e;
#pragma unroll 12
                    for (int d = 0; d < p.ndiag; ++d, Ud += p.ustride) {
                        const int m = s_off[d];
                        acc += __ldg(Ud) * yi[(ptrdiff_t)m * MM_R] - __ldg(Ud - m) * yi[-(ptrdiff_t)m * MM_R];
                    }
                }
                T q[KQ];
                load_qrow<T, KP>(p.Q, i, q, p.qcs != 0);
                T dq = (T)0;
#pragma unroll
                for (int m = 0; m < KP; ++m) dq += q[m] * s_u[c][m];
                const T ynew = tnu * acc - tsg * dq + tco * yold;
                Ynew[e] = ynew;
                tacc[0] += ynew * ynew;
#pragma unroll
                for (int m = 0; m < KP; ++m) tacc[1 + m] += q[m] * ynew;
            }
            if (pd) {   // the p/x update of the previous step of this column
                const T pv = (tnp * yold - tdpp * pold) * tthp;
                Pj1[e] = pv;
                p.x[c][i] += txp * pv;
            }
        }
        if (finalpass) break;
        double* buf = p.part + (size_t)(j & 1) * MM_R * NV * nblk;
        block_partials(tacc, buf);
        grid_sync_phase(p.gb, nblk, phase++, p.budget);
        if (*err) break;
        reduce_all(buf);
        if (warp == 0) {
            if (lane < MM_R) {
                const int cc = lane;
                MrsScalars<T>& s = sc[cc];
                if (s_live[cc]) {
                    const T beta = sqrt(s_red[cc][0]);
                    const T theta = sqrt(s.theta_t * s.theta_t + beta * beta);
                    const T rth = (T)1 / theta;
                    const T cs = s.theta_t * rth, sn = beta * rth;
                    const T delta = -s.s_prev * beta;
                    const T theta_t_next = s.c_prev * theta;
                    const T xcoef = s.G * cs;
                    const T Gn = -s.G * sn;
                    s.ratio = fabs(Gn) * s.rr0;
                    s.its = j;
                    // the update of step j (p_j, x += g_j c_j p_j) runs in the next pass
                    s.nu_p = s.nu;
                    s.delta_pp = s.delta_prev;
                    s.rtheta_p = rth;
                    s.xcoef_p = xcoef;
                    s_pend[cc] = 1;
                    if (s.ratio < (T)p.tol || j >= p.maxit) {
                        s_live[cc] = 0;
                    } else {
                        s.coef_old = beta * s.nu;
                        s.nu = (beta != (T)0) ? (T)1 / beta : (T)0;
                        s.s_prev = sn;
                        s.c_prev = cs;
                        s.delta_prev = delta;
                        s.theta_t = theta_t_next;
                        s.G = Gn;
                    }
                    set_coefs(cc);
                } else {
                    s_pend[cc] = 0;   // its last update ran in this pass
                }
            }
            __syncwarp();
            if (lane == 0) {
                int any = 0;
                for (int cc = 0; cc < MM_R; ++cc) any |= s_live[cc];
                s_anylive = any;
            }
            __syncwarp();
            make_u_warp0();
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x < p.ncol) {
        p.out_its[threadIdx.x] = sc[threadIdx.x].its;
        p.out_ratio[threadIdx.x] = (double)sc[threadIdx.x].ratio;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <class T, int KP, int FMT>
static asss_status launch_multi(const Ctx& c, MultiParams<T>& prm, int nslices, DBuf<int>& blk, DBuf<double>& part,
                                DBuf<unsigned>& bar) {
    int occ = 0;
    ASSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mrs_multi<T, KP, FMT>, MRS_THREADS, 0));
    if (occ < 1) {
        set_error("multi-column mrs kernel cannot be resident");
        return ASSS_ERR_CUDA;
    }
    if (occ > 4) occ = 4;
    int nblk = c.sms * occ;
    int need = cdiv(nslices, MRS_WARPS);
    if (need < 1) need = 1;
    if (nblk > need) nblk = need;
    if (blk.n < nblk + 1) ASSS_TRY(blk.alloc(nblk + 1));
    const long long np = 2LL * MM_R * (KP + 1) * nblk;
    if (part.n < np) ASSS_TRY(part.alloc(np));
    k_partition<<<cdiv(nblk + 1, 128), 128, 0, c.stream>>>(FMT == 0 ? prm.sptr : nullptr, nslices, nblk, blk.p);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaMemsetAsync(bar.p, 0, 2 * sizeof(unsigned), c.stream));
    prm.blk_slice = blk.p;
    prm.part = part.p;
    void* args[] = {&prm};
    ASSS_CUDA(cudaLaunchCooperativeKernel((const void*)k_mrs_multi<T, KP, FMT>, dim3(nblk), dim3(MRS_THREADS), args,
                                          0, c.stream));
    count_launch();
    return ASSS_OK;
}

template <class T, int FMT>
static asss_status dispatch_multi(const Ctx& c, int kp, MultiParams<T>& prm, int nslices, DBuf<int>& blk,
                                  DBuf<double>& part, DBuf<unsigned>& bar) {
    switch (kp) {
#define ASSS_MM_CASE(KPV) \
    case KPV:             \
        return launch_multi<T, KPV, FMT>(c, prm, nslices, blk, part, bar);
        ASSS_MM_CASE(0)
        ASSS_MM_CASE(4)
        ASSS_MM_CASE(8)
        ASSS_MM_CASE(12)
        ASSS_MM_CASE(16)
        ASSS_MM_CASE(20)
        ASSS_MM_CASE(24)
        ASSS_MM_CASE(32)
#undef ASSS_MM_CASE
        default:
            set_error("multi-column mrs: padded Lanczos width %d above %d", kp, MRS_MULTI_KPMAX);
            return ASSS_ERR_UNSUPPORTED;
    }
}

template <class T>
static asss_status multi_typed(const Ctx& c, const DSell<T>* sell, const DSkewDia<T>* dia, const T* Q, int kp,
                               const double* alpha, int k, double shift, double sign, int ncol,
                               const double* const* Bc, T* const* Xc, double tol, int maxit, int* its, double* ratio,
                               MrsTotals* tot) {
    if (dia && dia->ndiag > MRS_MAXDIAG) dia = nullptr;
    if (!dia && !sell) {
        set_error("mrs: no operator storage");
        return ASSS_ERR_ARG;
    }
    const int n = dia ? dia->n : sell->n;
    const int H = dia ? dia->halo : 0;
    cudaStream_t s = c.stream;
    DBuf<T> Y, P;
    DBuf<double> part;
    DBuf<int> blk, oits;
    DBuf<double> oratio;
    DBuf<unsigned> bar;
    DBuf<int> errw;
    const long long yslot = ((long long)n + 2LL * H) * MM_R;
    ASSS_TRY(Y.alloc(3 * yslot));
    ASSS_TRY(P.alloc(2LL * n * MM_R));
    ASSS_TRY(oits.alloc(MM_R));
    ASSS_TRY(oratio.alloc(MM_R));
    ASSS_TRY(bar.alloc(2));
    ASSS_TRY(errw.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(Y.p, 0, sizeof(T) * (size_t)Y.n, s));   // the halos stay zero
    ASSS_CUDA(cudaMemsetAsync(errw.p, 0, sizeof(int), s));
    const long long qrow = (long long)sizeof(T) * kp;
    const long long nnz = dia ? dia->nnz : sell->nnz;
    MultiParams<T> prm;
    memset(&prm, 0, sizeof(prm));
    prm.n = n;
    if (dia) {
        prm.ndiag = dia->ndiag;
        prm.off = dia->off.p;
        prm.U = dia->U.p + dia->halo;
        prm.ustride = dia->ustride;
    } else {
        prm.sptr = sell->sptr.p;
        prm.col = sell->col.p;
        prm.val = sell->val.p;
        prm.rowpos = sell->rowpos.p;
    }
    prm.halo = H;
    prm.yslot = yslot;
    prm.Q = Q;
    prm.alpha = alpha;
    prm.k = k;
    prm.shift = shift;
    prm.sign = sign;
    prm.Y = Y.p + (size_t)H * MM_R;
    prm.P = P.p;
    prm.gb.count = bar.p;
    prm.gb.gen = bar.p + 1;
    prm.gb.err = errw.p;
    prm.tol = tol;
    prm.maxit = maxit;
    prm.budget = c.wait_cycles;
    prm.out_its = oits.p;
    prm.out_ratio = oratio.p;
    prm.qcs = stream_evict_first(c, nnz * (long long)sizeof(T) + (long long)n * (qrow + 7LL * sizeof(T) * MM_R)) ? 1
                                                                                                                  : 0;
    const int nslices = cdiv(n, 32);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (tot) {
        ASSS_CUDA(cudaEventCreate(&e0));
        ASSS_CUDA(cudaEventCreate(&e1));
    }
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } evg{e0, e1};
    // algorithmic bytes: the matrix entries (with their column index in SELL) and the Q
    // row are read once per step for all columns; each live column reads and writes its
    // own vectors (gathered y, y_old, y_new, p r/w, x r/w); set-up and final passes
    const long long Tb = (long long)sizeof(T);
    const long long per_entry = dia ? Tb : Tb + 4;
    for (int c0 = 0; c0 < ncol; c0 += MM_R) {
        const int nc = ncol - c0 < MM_R ? ncol - c0 : MM_R;
        prm.ncol = nc;
        for (int t = 0; t < MM_R; ++t) {
            prm.rhs[t] = t < nc ? Bc[c0 + t] : nullptr;
            prm.x[t] = t < nc ? Xc[c0 + t] : nullptr;
        }
        if (tot) ASSS_CUDA(cudaEventRecord(e0, s));
        if (dia) ASSS_TRY((dispatch_multi<T, 1>(c, kp, prm, nslices, blk, part, bar)));
        else ASSS_TRY((dispatch_multi<T, 0>(c, kp, prm, nslices, blk, part, bar)));
        if (tot) ASSS_CUDA(cudaEventRecord(e1, s));
        int hi[MM_R];
        double hr[MM_R];
        int herr = 0;
        ASSS_CUDA(cudaMemcpyAsync(hi, oits.p, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaMemcpyAsync(hr, oratio.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaMemcpyAsync(&herr, errw.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        if (herr) {
            set_error("mrs: a grid barrier wait exceeded its budget");
            return (asss_status)herr;
        }
        for (int t = 0; t < nc; ++t) {
            if (its) its[c0 + t] = hi[t];
            if (ratio) ratio[c0 + t] = hr[t];
        }
        if (tot) {
            float ms = 0.f;
            ASSS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            long long sum_its = 0, max_its = 0;
            for (int t = 0; t < nc; ++t) {
                sum_its += hi[t];
                max_its = hi[t] > max_its ? hi[t] : max_its;
            }
            tot->ms += ms;
            tot->launches += 1;
            tot->its += sum_its;
            tot->bytes += (long long)n * (qrow + nc * (8 + 4 * Tb)) +                 // set-up pass
                          max_its * (nnz * per_entry + (long long)n * qrow) +         // shared per step
                          sum_its * (long long)n * 7 * Tb +                           // per column and step
                          (long long)n * nc * 4 * Tb;                                 // final updates
        }
    }
    return ASSS_OK;
}

asss_status mrs_multi_solve_cols(const Ctx& c, const MrsOperator& op, bool fp32, double shift, double sign,
                                 int ncol, const double* const* B, double* const* X64, float* const* X32, double tol,
                                 int maxit, int* its, double* ratio, MrsTotals* tot) {
    NvtxRange nv_("asss:mrs-multi");
    if (ncol <= 0) return ASSS_OK;
    if (fp32) {
        if ((!op.J32 && !op.D32) || !X32 || (!op.Q32 && op.kp > 0)) {
            set_error("FP32 multi-column mrs needs the FP32 operator, FP32 Q and an FP32 output");
            return ASSS_ERR_ARG;
        }
        return multi_typed<float>(c, op.J32, op.D32, op.Q32, op.kp, op.alpha, op.k, shift, sign, ncol, B, X32, tol,
                                  maxit, its, ratio, tot);
    }
    if ((!op.J64 && !op.D64) || !X64) {
        set_error("FP64 multi-column mrs needs the FP64 operator and an FP64 output");
        return ASSS_ERR_ARG;
    }
    return multi_typed<double>(c, op.J64, op.D64, op.Q64, op.kp, op.alpha, op.k, shift, sign, ncol, B, X64, tol,
                               maxit, its, ratio, tot);
}

asss_status mrs_multi_solve(const Ctx& c, const MrsOperator& op, bool fp32, double shift, double sign, int ncol,
                            const double* B, long long ldb, double* X64, float* X32, long long ldx, double tol,
                            int maxit, int* its, double* ratio) {
    std::vector<const double*> bc(ncol);
    std::vector<double*> x64(ncol, nullptr);
    std::vector<float*> x32(ncol, nullptr);
    for (int t = 0; t < ncol; ++t) {
        bc[t] = B + (size_t)t * ldb;
        if (X64) x64[t] = X64 + (size_t)t * ldx;
        if (X32) x32[t] = X32 + (size_t)t * ldx;
    }
    return mrs_multi_solve_cols(c, op, fp32, shift, sign, ncol, bc.data(), X64 ? x64.data() : nullptr,
                                X32 ? x32.data() : nullptr, tol, maxit, its, ratio, nullptr);
}

}  // namespace asss
