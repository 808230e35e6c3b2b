// Persistent single-kernel mrs solve (paper §3.1, App. B) of
//     (shift I + sign * (J~ - Q_k S_k Q_k^T)) x = b
// with J~ exactly skew - stored as skew half-diagonals (stencil-like patterns), in
// SELL-C, read in place as CSR, or applied in factored form L~^-1 J^ L~^-T through the
// incomplete L D L^T (one grid barrier per colour of each triangular solve) - and
// Q_k, S_k the skew-Lanczos data of §3.2 (Fig. 2).  One cooperative launch runs the
// whole iteration:
//
//   per iteration j (one pass over the rows owned by each block):
//     y_{j+1} = sign*(nu_j J~ y_j - Q (S_k h_j)) + beta_{j-1} nu_{j-1} y_{j-1}
//       (y_j = beta_{j-1} q_j is the unnormalised Lanczos vector, nu_j = 1/beta_{j-1},
//        h_j = Q^T q_j)
//     partial sums of ||y_{j+1}||^2 and Q^T y_{j+1}   -> ONE grid-wide reduction
//     the p/x update of step j-1 (needs only scalars known before the pass)
//   then every block computes the same Givens scalars from the reduced sums:
//     theta_j = sqrt(theta~_j^2 + beta_j^2), c_j, s_j, delta_j = -s_{j-1} beta_j,
//     theta~_{j+1} = c_{j-1} theta_j, x-coefficient g_j c_j, g_{j+1} = -g_j s_j.
//
// The norm and the k deflation dot products share the single reduction per
// iteration, which keeps the method's one-synchronisation-per-step property (§3.1).
// Vectors produced by other blocks are read through L2 (ld.global.cg); the grid
// barrier has a bounded wait.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "mrs_dev.cuh"

namespace asss {

constexpr int MRS_TRACE_STEPS = 16;
constexpr int MRS_TRACE_SLOTS = 4 + 5 * MRS_TRACE_STEPS;
// resident blocks per SM the register allocation is sized for: one 512-thread
// block, so a thread has up to 128 registers and can keep the loads of a whole
// row (all diagonals unrolled) in flight; more resident warps with half the
// registers measured slower (the pass is bound by memory latency per row)
template <class T>
constexpr int mrs_min_blocks() { return 1; }

struct MrsWork {
    int n = 0;
    const int* skip = nullptr;  // device flag read by the next launches (see mrs_set_skip)
    int sms = 0;
    DBuf<double> Y64, P64;
    DBuf<float> Y32, P32;
    DBuf<double> part;
    DBuf<unsigned> bar;
    DBuf<int> err;
    DBuf<int> out_its;
    DBuf<double> out_ratio;
    DBuf<int> blk_slice;
    const void* part_key = nullptr;
    int part_nblk = 0;
    int halo32 = -1, halo64 = -1;  // halo of the current Y layout (-1: not laid out)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // deferred statistics: each launch writes its step count and ratio into a log
    // slot and is bracketed by its own event pair; mrs_collect reads them all at once
    static constexpr int LOG_CAP = 1024;
    DBuf<int> its_log;
    DBuf<double> ratio_log;
    std::vector<cudaEvent_t> evs;
    std::vector<long long> log_nnz, log_per_row;  // bytes model per launch
    int log_n = 0;
    MrsTotals tot;
    DBuf<unsigned long long> trace;  // ASSS_TRACE_MRS=1: timeline of block 0
    ~MrsWork() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
    }
};

asss_status mrs_work_create(MrsWork** w, int n, int sms) {
    MrsWork* m = new MrsWork();
    m->n = n;
    m->sms = sms;
    asss_status st = ASSS_OK;
    int maxblk = sms * 4;
    if ((st = m->part.alloc((int64_t)2 * (MRS_KPMAX + 1) * maxblk)) != ASSS_OK ||
        (st = m->bar.alloc(2)) != ASSS_OK || (st = m->err.alloc(1)) != ASSS_OK ||
        (st = m->out_its.alloc(1)) != ASSS_OK || (st = m->out_ratio.alloc(1)) != ASSS_OK ||
        (st = m->blk_slice.alloc(maxblk + 1)) != ASSS_OK) {
        delete m;
        return st;
    }
    if (cudaEventCreate(&m->ev0) != cudaSuccess || cudaEventCreate(&m->ev1) != cudaSuccess) {
        delete m;
        set_error("cudaEventCreate failed");
        return ASSS_ERR_CUDA;
    }
    if (getenv("ASSS_TRACE_MRS") && (st = m->trace.alloc(MRS_TRACE_SLOTS)) != ASSS_OK) {
        delete m;
        return st;
    }
    if ((st = m->its_log.alloc(MrsWork::LOG_CAP)) != ASSS_OK ||
        (st = m->ratio_log.alloc(MrsWork::LOG_CAP)) != ASSS_OK) {
        delete m;
        return st;
    }
    if (cudaMemset(m->err.p, 0, sizeof(int)) != cudaSuccess) {
        delete m;
        set_error("cudaMemset failed");
        return ASSS_ERR_CUDA;
    }
    *w = m;
    return ASSS_OK;
}

void mrs_work_destroy(MrsWork* w) { delete w; }

template <class T>
struct MrsParams {
    int n;
    // SELL-C operator (rowmap: slot -> row for SELL-C-sigma, null for the identity)
    const int* sptr;
    const int* col;
    const T* val;
    const int* rowmap;
    const int4* units;   // SELL work units (slice, part, parts, accumulator) and their offsets per slice
    const int* uoff;
    T* hacc;             // partial sums of the parts of long slices (32 per long slice, left at 0)
    unsigned* hcnt;      // parts finished per long slice (left at 0)
    int split;           // entries per lane of one work unit
    // skew half-diagonal operator: U points at U_0[0]; diagonal d starts ustride later
    int ndiag;
    const int* off;
    const T* U;
    long long ustride;
    // plain CSR operator read in place (64-bit row pointers), one thread per row
    const long long* crp;
    const int* cci;
    const T* cval;
    // factored operator: z = wd .* (I + L)^-1 J^ (I + L)^-T (wd .* y), colour by colour
    int ncol;
    const int* fls;      // ncol + 1 level offsets into flvl
    const int* flvl;     // vertices by (colour, index)
    const int *flrp, *flci, *furp, *fuci, *fjrp, *fjci;
    const T *flv, *fuv, *fjv, *fwd;
    const int* fpart;    // 2x2 pivots: partner of each vertex (null: 1x1 pivots only)
    const T* fwo;        // off-diagonal of |D|^-1/2 between the members of a pair
    T* ft;               // (I + L)^-T (wd .* y)
    T* fw;               // (I + L)^-1 J^ ft
    long long ystride;  // distance between the three Y slots (n + 2 halo)
    const T* Q;
    const __nv_bfloat16* Q16;  // BF16 copy of Q (row stride KP) when the kernel reads Q in BF16
    const double* alpha;
    int k;
    double shift, sign;
    const double* rhs;
    T* x;
    T* Y;  // 3 slots of unnormalised Lanczos vectors, each with a zero halo on both ends
    T* P;  // 2n ring of update directions
    double* part;  // [2][NV][nblk]
    GridBarrier gb;
    const int* blk_slice;
    double tol;
    int maxit;
    long long budget;
    int* out_its;
    double* out_ratio;
    unsigned long long* trace;  // optional timeline (block 0): %globaltimer at phase boundaries
    const int* skip;     // optional: when *skip != 0 at launch the kernel only logs its = -1
    int qcs;             // load Q rows evict-first (the step's data exceed L2)
    double* qtz;         // optional: Q^T x (k values) of the final iterate
};

// sum over q in [q0, q1) of v[q] * x[ci[q]], eight entries at a time: the indices
// and values of a batch are loaded first, then all its gathers, so a row costs a
// few memory latencies instead of two per entry (x is written by other blocks of
// the launch: plain loads after the grid barrier, not the read-only path)
template <class T>
__device__ __forceinline__ T row_dot8(const int* __restrict__ ci, const T* __restrict__ v, const T* x, int q0,
                                      int q1) {
    T a = (T)0;
    for (int q = q0; q < q1; q += 8) {
        int cc[8];
        T vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool in = q + u < q1;
            cc[u] = in ? __ldg(ci + q + u) : 0;
            vv[u] = in ? __ldg(v + q + u) : (T)0;
        }
        T g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) g[u] = (q + u < q1) ? x[cc[u]] : (T)0;
#pragma unroll
        for (int u = 0; u < 8; ++u) a += vv[u] * g[u];
    }
    return a;
}

// FMT 0: SELL-C storage of J~; FMT 1: skew half-diagonal storage; FMT 2: plain CSR;
// FMT 3: factored J~ = L~^-1 J^ L~^-T (incomplete L D L^T in a multicolour order)
template <class T, int KP, int FMT, bool QB = false>
__global__ void __launch_bounds__(MRS_THREADS, mrs_min_blocks<T>()) k_mrs(MrsParams<T> p) {
    constexpr int NV = KP + 1;
    if (p.skip && *p.skip) {  // enqueued ahead of a decision that went the other way
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *p.out_its = -1;
            *p.out_ratio = 0.0;
        }
        return;
    }
    __shared__ T s_wsum[MRS_WARPS][NV];
    __shared__ T s_red[NV];
    __shared__ T s_u[KP > 0 ? KP : 1];
    __shared__ int s_off[FMT == 1 ? MRS_MAXDIAG : 1];
    __shared__ int s_ls[FMT == 3 ? ILDL_MAXCOL + 1 : 1];
    __shared__ MrsScalars<T> sc;
    __shared__ T s_alpha[MRS_KPMAX];
    // per-step coefficients in T, set by one thread (the others only read them):
    // 0 sign*nu, 1 sign, 2 beta_{j-1} nu_{j-1}, 3 nu_p, 4 delta_pp, 5 1/theta_p, 6 xcoef_p,
    // 7..10 the final pass: nu, delta, 1/theta, xcoef
    __shared__ T s_cf[12];
    __shared__ int s_next;   // SELL: next work unit of this block for the warp that asks (see next_slice)
    // Q^T x of the final iterate without a pass over Q: the directions obey
    // p_j = (nu_j y_j - delta_j p_{j-2}) / theta_j and x = sum_j xcoef_j p_j, so Q^T p_j and
    // Q^T x follow from the Q^T y_j that every step reduces anyway (warp 1 keeps them)
    __shared__ T s_qty[KP > 0 ? KP : 1];     // Q^T y_j of the step in progress
    __shared__ T s_qtp[2][KP > 0 ? KP : 1];  // Q^T p of the last two directions (slot j & 1)
    __shared__ T s_qtx[KP > 0 ? KP : 1];     // Q^T x
    __shared__ T s_pq[4];                    // step j: nu_j, delta, 1/theta_j, xcoef_j
    if constexpr (FMT == 1) {
        for (int d = threadIdx.x; d < p.ndiag; d += MRS_THREADS) s_off[d] = p.off[d];
    }
    for (int m = threadIdx.x; m < KP; m += MRS_THREADS) {
        s_qtp[0][m] = (T)0;
        s_qtp[1][m] = (T)0;
        s_qtx[m] = (T)0;
    }
    if constexpr (FMT == 3) {
        for (int c = threadIdx.x; c <= p.ncol; c += MRS_THREADS) s_ls[c] = p.fls[c];
        __syncthreads();
    }
    for (int m = threadIdx.x; m + 1 < p.k && m < MRS_KPMAX; m += MRS_THREADS) s_alpha[m] = (T)p.alpha[m];
    auto set_coefs = [&]() {  // thread 0 only
        s_cf[0] = (T)p.sign * sc.nu;
        s_cf[1] = (T)p.sign;
        s_cf[2] = (T)sc.coef_old;
        s_cf[3] = (T)sc.nu_p;
        s_cf[4] = (T)sc.delta_pp;
        s_cf[5] = (T)sc.rtheta_p;
        s_cf[6] = (T)sc.xcoef_p;
        if (sc.stop) {
            s_cf[7] = (T)sc.fin_nu;
            s_cf[8] = (T)sc.fin_delta;
            s_cf[9] = (T)sc.fin_rtheta;
            s_cf[10] = (T)sc.fin_xcoef;
        }
    };
    const int nblk = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s0 = p.blk_slice[blockIdx.x], s1 = p.blk_slice[blockIdx.x + 1];
    const int n = p.n;
    const size_t ys = p.ystride;
    volatile int* err = p.gb.err;
    // timeline slots: 0 start, 1 phase-0 pass, 2 phase-0 barrier, 3 set-up scalars; then per
    // step j (1-based, first MRS_TRACE_STEPS): 4+5(j-1)+{0 pass, 1 partials, 2 barrier, 3 reduce, 4 scalars+u}
    const bool tr = p.trace && blockIdx.x == 0 && threadIdx.x == 0;
    auto stamp = [&](int slot) {
        if (tr && slot < MRS_TRACE_SLOTS) p.trace[slot] = gtimer();
    };
    stamp(0);

    // warp sums in T, then across warps in a fixed order (float pairs for the FP32 solve,
    // FP64 for the FP64 solve) into this block's partial
    auto block_partials = [&](T(&tacc)[NV], double* buf) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(T) == 4) {
                T d = warp_sum(tacc[v]);
                if (lane == 0) s_wsum[warp][v] = d;
            } else {
                // FP64 partials: the warp tree runs on float pairs (the FP64 pipe is slow)
                float hi = (float)tacc[v];
                float2 a = make_float2(hi, (float)((double)tacc[v] - (double)hi));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float2 b;
                    b.x = __shfl_xor_sync(0xffffffffu, a.x, o);
                    b.y = __shfl_xor_sync(0xffffffffu, a.y, o);
                    a = df_add(a, b);
                }
                if (lane == 0) s_wsum[warp][v] = (double)a.x + (double)a.y;
            }
        }
        __syncthreads();
        for (int v = threadIdx.x; v < NV; v += MRS_THREADS) {
            if constexpr (sizeof(T) == 4) {
                // block partial as a float pair (hi, lo) in the same 8 bytes, summed over
                // the warps in float-pair arithmetic
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int w = 0; w < MRS_WARPS; ++w) a = df_add(a, make_float2(s_wsum[w][v], 0.f));
                reinterpret_cast<float2*>(buf)[v * nblk + blockIdx.x] = a;
            } else {
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < MRS_WARPS; ++w) t += s_wsum[w][v];
                buf[v * nblk + blockIdx.x] = t;
            }
        }
    };
    // every block adds the block partials in the same fixed order; each lane issues
    // its loads (RCHUNK at a time) before adding, so the L2 latencies overlap
    constexpr int RCHUNK = 10;
    auto reduce_all = [&](const double* buf) {
        for (int v = warp; v < NV; v += MRS_WARPS) {
            if constexpr (sizeof(T) == 4) {
                const float2* b2 = reinterpret_cast<const float2*>(buf) + (size_t)v * nblk;
                float2 acc = make_float2(0.f, 0.f);
                for (int b0 = 0; b0 < nblk; b0 += 32 * RCHUNK) {
                    float2 ld[RCHUNK];
#pragma unroll
                    for (int t = 0; t < RCHUNK; ++t) {
                        const int b = b0 + lane + 32 * t;
                        ld[t] = b < nblk ? __ldcg(&b2[b]) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int t = 0; t < RCHUNK; ++t) acc = df_add(acc, ld[t]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float2 other;
                    other.x = __shfl_xor_sync(0xffffffffu, acc.x, o);
                    other.y = __shfl_xor_sync(0xffffffffu, acc.y, o);
                    acc = df_add(acc, other);
                }
                if (lane == 0) s_red[v] = acc.x + acc.y;
            } else {
                double t = 0.0;
                for (int b0 = 0; b0 < nblk; b0 += 32 * RCHUNK) {
                    double ld[RCHUNK];
#pragma unroll
                    for (int q = 0; q < RCHUNK; ++q) {
                        const int b = b0 + lane + 32 * q;
                        ld[q] = b < nblk ? __ldcg(&buf[v * nblk + b]) : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < RCHUNK; ++q) t += ld[q];
                }
                t = warp_sum(t);
                if (lane == 0) s_red[v] = t;
            }
        }
        __syncthreads();
    };
    // u = S_k h with h = nu * (Q^T y), S_k(m, m+1) = alpha_m, S_k(m+1, m) = -alpha_m;
    // computed by the lanes of warp 0 (the caller synchronises the block afterwards)
    auto make_u_warp0 = [&](T nu) {
        if constexpr (KP > 0) {
            for (int m = lane; m < KP; m += 32) {
                T u = (T)0;
                if (m < p.k) {
                    if (m + 1 < p.k) u += s_alpha[m] * s_red[2 + m] * nu;
                    if (m > 0) u -= s_alpha[m - 1] * s_red[m] * nu;
                }
                s_u[m] = u;
            }
        }
    };
    // warp 1: fold direction p_jj into Q^T x (s_pq holds step jj's scalars, s_qty Q^T y_jj)
    auto qtx_fold = [&](int jj) {
        if constexpr (KP > 0) {
            if (lane < p.k) {
                T* pp = s_qtp[jj & 1];
                const T v = (s_pq[0] * s_qty[lane] - s_pq[1] * pp[lane]) * s_pq[2];
                pp[lane] = v;
                s_qtx[lane] += s_pq[3] * v;
            }
        }
    };
    const bool want_qtx = KP > 0 && p.qtz != nullptr;
    unsigned phase = 0;  // grid barriers passed in this launch
    // ---- phase 0: y_1 = b, x = 0, p = 0, ||b||^2 and Q^T b ----
    T tacc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) tacc[v] = (T)0;
    // The slices of a SELL operator carry very different amounts of work (heavy-tailed
    // rows), so in the step passes the warps of a block take them one at a time from a
    // shared counter instead of in a fixed stride; the other storages keep the stride.
    auto next_slice = [&](int sl) -> int {
        if constexpr (FMT == 0) {
            int nx = 0;
            if (lane == 0) nx = atomicAdd(&s_next, 1);
            return __shfl_sync(0xffffffffu, nx, 0);
        }
        return sl + MRS_WARPS;
    };
    // SELL: the block's work units (its slices, long ones cut into parts)
    const int u0 = FMT == 0 ? __ldg(&p.uoff[s0]) : s0;
    const int u1 = FMT == 0 ? __ldg(&p.uoff[s1]) : s1;
    // the row held by lane `lane` of slice sl (SELL-C-sigma permutes rows within windows)
    auto row_of = [&](int sl) -> int {
        if constexpr (FMT == 0) {
            if (p.rowmap) return __ldg(&p.rowmap[sl * 32 + lane]);
        }
        return sl * 32 + lane;
    };
    for (int sl = s0 + warp; sl < s1; sl += MRS_WARPS) {
        int i = row_of(sl);
        if (i < n) {
            T b = (T)p.rhs[i];
            p.Y[i] = b;
            p.x[i] = (T)0;
            p.P[i] = (T)0;
            p.P[n + i] = (T)0;
            tacc[0] += b * b;
            T q[KP > 0 ? KP : 1];
            if constexpr (QB) load_qrow16<T, KP>(p.Q16, i, q);
            else load_qrow<T, KP>(p.Q, i, q, p.qcs != 0);
#pragma unroll
            for (int m = 0; m < KP; ++m) tacc[1 + m] += q[m] * b;
        }
    }
    stamp(1);
    block_partials(tacc, p.part);
    grid_sync_phase(p.gb, nblk, phase++, p.budget);
    stamp(2);
    if (*err) return;
    reduce_all(p.part);

    if (warp == 0) {
        if (lane == 0) {
            const T r0 = sqrt(s_red[0]);
            const T zero = (T)0, one = (T)1;
            sc.r0 = r0;
            sc.rr0 = r0 > zero ? one / r0 : zero;
            sc.nu = sc.rr0;
            sc.coef_old = zero;
            sc.theta_t = (T)p.shift;
            sc.c_prev = one;
            sc.s_prev = zero;
            sc.delta_prev = zero;
            sc.G = r0;
            sc.nu_p = zero;
            sc.delta_pp = zero;
            sc.rtheta_p = one;
            sc.xcoef_p = zero;
            sc.ratio = r0 > zero ? one : zero;
            sc.its = 0;
            sc.stop = r0 > zero ? 0 : 1;
            set_coefs();
            s_next = u0 + MRS_WARPS;
        }
        __syncwarp();
        if (!sc.stop) make_u_warp0(sc.nu);
    }
    __syncthreads();
    if (sc.stop) {  // b = 0: x = 0 already
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) {
                *p.out_its = 0;
                *p.out_ratio = 0.0;
            }
            if (p.qtz)
                for (int v = threadIdx.x; v < p.k; v += MRS_THREADS) p.qtz[v] = 0.0;
        }
        return;
    }
    stamp(3);

    for (int j = 1; j <= p.maxit; ++j) {
        const int tb = 4 + 5 * (j - 1);
        if (want_qtx && warp == 1) {
            // off the synchronisation chain: step j-1's direction, then Q^T y_j from the
            // last reduction (s_red is next written after this pass's block barrier)
            if (j >= 2) qtx_fold(j - 1);
            if (lane < p.k) s_qty[lane] = s_red[1 + lane];
        }
        // the step's vectors do not overlap: restrict lets later rows' loads be scheduled
        // ahead of this row's stores
        const T* __restrict__ Ycur = p.Y + (size_t)((j - 1) % 3) * ys;
        const T* __restrict__ Yold = p.Y + (size_t)((j + 1) % 3) * ys;
        T* __restrict__ Ynew = p.Y + (size_t)(j % 3) * ys;
        T* __restrict__ Pj1 = p.P + (size_t)((j - 1) & 1) * n;
        T* __restrict__ xv = p.x;
        const T* __restrict__ Ub = p.U;
        const T* __restrict__ Qr = p.Q;
        const T tnu = s_cf[0], tsg = s_cf[1], tco = s_cf[2];
        const T tnp = s_cf[3], tdpp = s_cf[4], tthp = s_cf[5], txp = s_cf[6];
        if constexpr (FMT == 3) {
            // J~ y_j in factored form: the back solve (I + L)^T t = wd .* y_j from the
            // largest colour down, then w = (I + L)^-1 J^ t from the smallest colour up
            // (J^ t is formed row by row inside the forward solve); the rows of one
            // colour are spread over the whole grid, one grid barrier per colour
            const int gt = blockIdx.x * MRS_THREADS + threadIdx.x, gs = nblk * MRS_THREADS;
            bool ok = true;
            for (int cc = p.ncol - 1; cc >= 0 && ok; --cc) {
                for (int e = s_ls[cc] + gt; e < s_ls[cc + 1]; e += gs) {
                    const int i = __ldg(&p.flvl[e]);
                    T a = __ldg(&p.fwd[i]) * Ycur[i];
                    if (p.fpart) {
                        const int m = __ldg(&p.fpart[i]);
                        if (m >= 0) a += __ldg(&p.fwo[i]) * Ycur[m];
                    }
                    p.ft[i] = a - row_dot8<T>(p.fuci, p.fuv, p.ft, __ldg(&p.furp[i]), __ldg(&p.furp[i + 1]));
                }
                grid_sync_phase(p.gb, nblk, phase++, p.budget);
                if (*err) ok = false;
            }
            for (int cc = 0; cc < p.ncol && ok; ++cc) {
                for (int e = s_ls[cc] + gt; e < s_ls[cc + 1]; e += gs) {
                    const int i = __ldg(&p.flvl[e]);
                    const T a = row_dot8<T>(p.fjci, p.fjv, p.ft, __ldg(&p.fjrp[i]), __ldg(&p.fjrp[i + 1]));
                    p.fw[i] = a - row_dot8<T>(p.flci, p.flv, p.fw, __ldg(&p.flrp[i]), __ldg(&p.flrp[i + 1]));
                }
                grid_sync_phase(p.gb, nblk, phase++, p.budget);
                if (*err) ok = false;
            }
            if (!ok) break;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) tacc[v] = (T)0;
        for (int uu = u0 + warp; uu < u1; uu = next_slice(uu)) {
            int sl = uu, part = 0, nparts = 1, hix = -1;
            if constexpr (FMT == 0) {
                const int4 U = __ldg(&p.units[uu]);
                sl = U.x;
                part = U.y;
                nparts = U.z;
                hix = U.w;
            }
            const int i = row_of(sl);
            const bool live = i < n;
            // this row's own data first (independent of the operator loop below)
            const T yold = (live && j >= 2) ? Yold[i] : (T)0;
            const T pold = (live && j >= 2) ? Pj1[i] : (T)0;
            uint4 qraw[(QB && KP > 0) ? KP / 8 : 1];
            if constexpr (QB && KP > 0) {
                if (live) {
                    const uint4* qr = reinterpret_cast<const uint4*>(p.Q16 + (size_t)i * KP);
#pragma unroll
                    for (int t = 0; t < KP / 8; ++t) qraw[t] = p.qcs ? __ldcs(qr + t) : __ldg(qr + t);
                }
            }
            T acc = (T)0;
            if constexpr (FMT == 3) {
                if (live) {
                    acc = __ldg(&p.fwd[i]) * p.fw[i];
                    if (p.fpart) {
                        const int m = __ldg(&p.fpart[i]);
                        if (m >= 0) acc += __ldg(&p.fwo[i]) * p.fw[m];
                    }
                }
            } else if constexpr (FMT == 2) {
                if (i < n) {
                    const long long e1 = __ldg(&p.crp[i + 1]);
                    for (long long e = __ldg(&p.crp[i]); e < e1; ++e) acc += __ldg(&p.cval[e]) * Ycur[__ldg(&p.cci[e])];
                }
            } else if constexpr (FMT == 0) {
                const int base = __ldg(&p.sptr[sl]);
                const int wfull = (__ldg(&p.sptr[sl + 1]) - base) >> 5;
                // this unit's part of the slice: entries [part * split, ...) of every lane
                const int kbeg = part * p.split;
                const int width = min(wfull, kbeg + p.split) - kbeg;
                const int* cp = p.col + base + lane + kbeg * 32;
                const T* vp = p.val + base + lane + kbeg * 32;
                // Sixteen entries in flight per lane (the gathers depend on the column
                // loads, so the depth of the batch is the latency hiding); when the
                // matrix exceeds L2 its entries are loaded evict-first, so the gathered
                // vector stays in L2 while the matrix streams past it.
                constexpr int UB = 16;
                int kk = 0;
                if (p.qcs) {
                    for (; kk + UB <= width; kk += UB) {
                        int cc[UB];
                        T vv[UB];
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            cc[u] = __ldcs(cp + (kk + u) * 32);
                            vv[u] = __ldcs(vp + (kk + u) * 32);
                        }
#pragma unroll
                        for (int u = 0; u < UB; ++u) acc += vv[u] * Ycur[cc[u]];
                    }
                    for (; kk < width; ++kk) acc += __ldcs(vp + kk * 32) * Ycur[__ldcs(cp + kk * 32)];
                } else {
                    for (; kk + UB <= width; kk += UB) {
                        int cc[UB];
                        T vv[UB];
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            cc[u] = __ldg(cp + (kk + u) * 32);
                            vv[u] = __ldg(vp + (kk + u) * 32);
                        }
#pragma unroll
                        for (int u = 0; u < UB; ++u) acc += vv[u] * Ycur[cc[u]];
                    }
                    for (; kk < width; ++kk) acc += __ldg(vp + kk * 32) * Ycur[__ldg(cp + kk * 32)];
                }
                if (nparts > 1) {
                    // a part of a long slice: add the lanes' partial sums; the warp that
                    // finishes the slice's last part reads the totals (resetting them for
                    // the next pass) and carries on with the rows, the others are done
                    atomicAdd(&p.hacc[(size_t)hix * 32 + lane], acc);
                    __threadfence();
                    __syncwarp();
                    int last = 0;
                    if (lane == 0) last = atomicAdd(&p.hcnt[hix], 1u) == (unsigned)(nparts - 1);
                    last = __shfl_sync(0xffffffffu, last, 0);
                    if (!last) continue;
                    __threadfence();
                    // every other part's adds completed before its count (fenced), and no
                    // one touches this slice's accumulators again before the next pass
                    acc = __ldcg(&p.hacc[(size_t)hix * 32 + lane]);
                    p.hacc[(size_t)hix * 32 + lane] = (T)0;
                    if (lane == 0) p.hcnt[hix] = 0u;
                }
            } else {
                // (J~ y)_i = sum_d U_d[i] y[i + m_d] - U_d[i - m_d] y[i - m_d]; zero halos on
                // both U (front) and y (both ends) make the loop branch-free
                if (i < n) {
                    const T* Ud = Ub + i;
                    const T* yi = Ycur + i;
#pragma unroll 12
                    for (int d = 0; d < p.ndiag; ++d, Ud += p.ustride) {
                        const int m = s_off[d];
                        acc += __ldg(Ud) * yi[m] - __ldg(Ud - m) * yi[-m];
                    }
                }
            }
            if (live) {
                T q[KP > 0 ? KP : 1];
                if constexpr (QB && KP > 0) {
#pragma unroll
                    for (int t = 0; t < KP / 8; ++t) {
                        const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&qraw[t]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float2 f = __bfloat1622float2(h2[e]);
                            q[8 * t + 2 * e] = (T)f.x;
                            q[8 * t + 2 * e + 1] = (T)f.y;
                        }
                    }
                } else {
                    load_qrow<T, KP>(Qr, i, q, p.qcs != 0);
                }
                T dq = (T)0;
#pragma unroll
                for (int m = 0; m < KP; ++m) dq += q[m] * s_u[m];
                T ynew = tnu * acc - tsg * dq + tco * yold;
                Ynew[i] = ynew;
                tacc[0] += ynew * ynew;
#pragma unroll
                for (int m = 0; m < KP; ++m) tacc[1 + m] += q[m] * ynew;
                if (j >= 2) {
                    T pv = (tnp * yold - tdpp * pold) * tthp;
                    Pj1[i] = pv;
                    xv[i] += txp * pv;
                }
            }
        }
        double* buf = p.part + (size_t)(j & 1) * NV * nblk;
        stamp(tb);
        block_partials(tacc, buf);
        stamp(tb + 1);
        grid_sync_phase(p.gb, nblk, phase++, p.budget);
        stamp(tb + 2);
        if (*err) break;
        reduce_all(buf);
        stamp(tb + 3);

        if (warp == 0) {
            if (lane == 0) {
                const T beta = sqrt(s_red[0]);
                const T theta = sqrt(sc.theta_t * sc.theta_t + beta * beta);
                const T rth = (T)1 / theta;
                const T c = sc.theta_t * rth, s = beta * rth;
                const T delta = -sc.s_prev * beta;
                const T theta_t_next = sc.c_prev * theta;
                const T xcoef = sc.G * c;
                const T Gn = -sc.G * s;
                s_pq[0] = sc.nu;
                s_pq[1] = sc.delta_prev;
                s_pq[2] = rth;
                s_pq[3] = xcoef;
                sc.ratio = fabs(Gn) * sc.rr0;
                sc.its = j;
                if (sc.ratio < p.tol || j == p.maxit) {
                    sc.stop = 1;
                    sc.fin_nu = sc.nu;
                    sc.fin_delta = sc.delta_prev;
                    sc.fin_rtheta = rth;
                    sc.fin_xcoef = xcoef;
                } else {
                    sc.nu_p = sc.nu;
                    sc.delta_pp = sc.delta_prev;
                    sc.rtheta_p = rth;
                    sc.xcoef_p = xcoef;
                    sc.coef_old = beta * sc.nu;
                    sc.nu = (beta != (T)0) ? (T)1 / beta : (T)0;
                    sc.s_prev = s;
                    sc.c_prev = c;
                    sc.delta_prev = delta;
                    sc.theta_t = theta_t_next;
                    sc.G = Gn;
                }
                set_coefs();
                s_next = u0 + MRS_WARPS;
            }
            __syncwarp();
            if (!sc.stop) make_u_warp0(sc.nu);
        }
        __syncthreads();
        if (sc.stop) {
            T* Pj = p.P + (size_t)(j & 1) * n;
            const T tn = s_cf[7], td = s_cf[8], tth = s_cf[9], tx = s_cf[10];
#pragma unroll
            for (int v = 0; v < NV; ++v) tacc[v] = (T)0;
            for (int sl = s0 + warp; sl < s1; sl += MRS_WARPS) {
                int i = row_of(sl);
                if (i < n) {
                    T pv = (tn * Ycur[i] - td * Pj[i]) * tth;
                    p.x[i] = p.x[i] + tx * pv;
                }
            }
            if (want_qtx && warp == 1) {
                qtx_fold(j);
                if (blockIdx.x == 0 && lane < p.k) p.qtz[lane] = (double)s_qtx[lane];
            }
            break;
        }
        stamp(tb + 4);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *p.out_its = sc.its;
        *p.out_ratio = (double)sc.ratio;
    }
}

// what the launcher needs to know about the operator, whatever its storage
template <class T>
struct OpView {
    int n = 0;
    int fmt = 0;
    int nslices = 0;
    const int* sptr = nullptr;
    const int* col = nullptr;
    const T* val = nullptr;
    const int* rowmap = nullptr;
    const int4* units = nullptr;
    const int* uoff = nullptr;
    T* hacc = nullptr;
    unsigned* hcnt = nullptr;
    int nheavy = 0;
    int split = 0;
    int ndiag = 0;
    const int* off = nullptr;
    const T* U = nullptr;
    long long ustride = 0;
    int halo = 0;
    const void* key = nullptr;
    long long nnz = 0;  // matrix entries one application reads
    const IldlFactor* fac = nullptr;  // FMT 3
};

struct LaunchOut {
    int slot;
    double* qtz;
};

template <class T, int KP, int FMT, bool QB = false>
static asss_status launch_mrs(const Ctx& c, MrsWork* w, const OpView<T>& J, const T* Q, const double* alpha,
                              int k, double shift, double sign, const double* rhs, T* x, T* Y, long long ystride,
                              T* P, double tol, int maxit, LaunchOut lo, const __nv_bfloat16* Q16 = nullptr) {
    int occ = 0;
    ASSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mrs<T, KP, FMT, QB>, MRS_THREADS, 0));
    if (occ < 1) {
        set_error("mrs kernel cannot be resident");
        return ASSS_ERR_CUDA;
    }
    if (occ > 4) occ = 4;
    int nblk = c.sms * occ;
    int need = cdiv(J.nslices, MRS_WARPS);
    if (need < 1) need = 1;
    if (nblk > need) nblk = need;
    if (w->part_key != J.key || w->part_nblk != nblk) {
        k_partition<<<cdiv(nblk + 1, 128), 128, 0, c.stream>>>(FMT == 0 ? J.sptr : nullptr, J.nslices, nblk,
                                                               w->blk_slice.p);
        ASSS_CHECK_LAUNCH();
        w->part_key = J.key;
        w->part_nblk = nblk;
    }
    ASSS_CUDA(cudaMemsetAsync(w->bar.p, 0, 2 * sizeof(unsigned), c.stream));
    if (FMT == 0 && J.nheavy > 0) {
        // the long slices' accumulators start at zero (a launch that gave up at a barrier
        // may have left partial sums behind)
        ASSS_CUDA(cudaMemsetAsync(J.hacc, 0, sizeof(T) * 32 * (size_t)J.nheavy, c.stream));
        ASSS_CUDA(cudaMemsetAsync(J.hcnt, 0, sizeof(unsigned) * (size_t)J.nheavy, c.stream));
    }
    MrsParams<T> prm;
    prm.n = J.n;
    prm.sptr = J.sptr;
    prm.col = J.col;
    prm.val = J.val;
    prm.rowmap = J.rowmap;
    prm.units = J.units;
    prm.uoff = J.uoff;
    prm.hacc = J.hacc;
    prm.hcnt = J.hcnt;
    prm.split = J.split > 0 ? J.split : SELL_SPLIT;
    prm.ndiag = J.ndiag;
    prm.off = J.off;
    prm.U = J.U;
    prm.ustride = J.ustride;
    prm.crp = nullptr;
    prm.cci = nullptr;
    prm.cval = nullptr;
    prm.ncol = 0;
    prm.fls = prm.flvl = prm.flrp = prm.flci = prm.furp = prm.fuci = prm.fjrp = prm.fjci = nullptr;
    prm.flv = prm.fuv = prm.fjv = prm.fwd = nullptr;
    prm.fpart = nullptr;
    prm.fwo = nullptr;
    prm.ft = prm.fw = nullptr;
    if constexpr (FMT == 3) {
        const IldlFactor& F = *J.fac;
        prm.ncol = F.ncol;
        prm.fpart = F.npairs > 0 ? F.part.p : nullptr;
        prm.fls = F.ls.p;
        prm.flvl = F.lvl.p;
        prm.flrp = F.lrp.p;
        prm.flci = F.lci.p;
        prm.furp = F.urp.p;
        prm.fuci = F.uci.p;
        prm.fjrp = F.jrp;
        prm.fjci = F.jci;
        if constexpr (sizeof(T) == 4) {
            prm.flv = F.lv32.p;
            prm.fuv = F.uv32.p;
            prm.fjv = F.jv32.p;
            prm.fwd = F.wd32.p;
            prm.fwo = F.wo32.p;
            prm.ft = F.ft32.p;
            prm.fw = F.fw32.p;
        } else {
            prm.flv = F.lv.p;
            prm.fuv = F.uv.p;
            prm.fjv = F.jv;
            prm.fwd = F.wd.p;
            prm.fwo = F.wo.p;
            prm.ft = F.ft.p;
            prm.fw = F.fw.p;
        }
    }
    prm.ystride = ystride;
    prm.Q = Q;
    prm.Q16 = Q16;
    prm.alpha = alpha;
    prm.k = k;
    prm.shift = shift;
    prm.sign = sign;
    prm.rhs = rhs;
    prm.x = x;
    prm.Y = Y;
    prm.P = P;
    prm.part = w->part.p;
    prm.gb.count = w->bar.p;
    prm.gb.gen = w->bar.p + 1;
    prm.gb.err = w->err.p;
    prm.blk_slice = w->blk_slice.p;
    prm.tol = tol;
    prm.maxit = maxit;
    prm.budget = c.wait_cycles;
    prm.out_its = w->its_log.p + lo.slot;
    prm.out_ratio = w->ratio_log.p + lo.slot;
    prm.qtz = (KP > 0 && k > 0) ? lo.qtz : nullptr;
    prm.trace = w->trace.p;
    prm.skip = w->skip;
    {
        const long long qrow = QB ? 2LL * KP : (long long)sizeof(T) * KP;
        prm.qcs = stream_evict_first(c, J.nnz * (long long)sizeof(T) + (long long)J.n * (7LL * sizeof(T) + qrow)) ? 1 : 0;
    }
    void* args[] = {&prm};
    ASSS_CUDA(cudaEventRecord(w->evs[2 * lo.slot], c.stream));
    ASSS_CUDA(cudaLaunchCooperativeKernel((const void*)k_mrs<T, KP, FMT, QB>, dim3(nblk), dim3(MRS_THREADS), args,
                                          0, c.stream));
    count_launch();
    ASSS_CUDA(cudaEventRecord(w->evs[2 * lo.slot + 1], c.stream));
    return ASSS_OK;
}

template <class T, int FMT>
static asss_status dispatch_kp(const Ctx& c, MrsWork* w, const OpView<T>& J, const T* Q, const double* alpha, int k,
                               int kp, double shift, double sign, const double* rhs, T* x, T* Y, long long ystride,
                               T* P, double tol, int maxit, LaunchOut lo) {
    switch (kp) {
#define ASSS_MRS_CASE(KPV) \
    case KPV:              \
        return launch_mrs<T, KPV, FMT>(c, w, J, Q, alpha, k, shift, sign, rhs, x, Y, ystride, P, tol, maxit, lo);
        ASSS_MRS_CASE(0)
        ASSS_MRS_CASE(4)
        ASSS_MRS_CASE(8)
        ASSS_MRS_CASE(12)
        ASSS_MRS_CASE(16)
        ASSS_MRS_CASE(20)
        ASSS_MRS_CASE(24)
        ASSS_MRS_CASE(32)
        ASSS_MRS_CASE(48)
        ASSS_MRS_CASE(64)
#undef ASSS_MRS_CASE
        default:
            set_error("unsupported padded Lanczos width %d", kp);
            return ASSS_ERR_UNSUPPORTED;
    }
}

// Y ring with zero halos of width H on both ends of each slot (re-zeroed whenever
// the layout changes; the kernel never writes the halos)
template <class T>
static asss_status y_layout(MrsWork* w, DBuf<T>& Ybuf, int& cur, int H, cudaStream_t s, T** Y, long long* ystride) {
    long long st = (long long)w->n + 2LL * H;
    if (cur != H || Ybuf.n < 3 * st) {
        if (Ybuf.n < 3 * st) ASSS_TRY(Ybuf.alloc(3 * st));
        ASSS_CUDA(cudaMemsetAsync(Ybuf.p, 0, sizeof(T) * (size_t)Ybuf.n, s));
        cur = H;
    }
    *Y = Ybuf.p + H;
    *ystride = st;
    return ASSS_OK;
}

// FP32 solve reading Q in BF16: row strides that keep 16-byte aligned rows
template <int FMT>
static asss_status dispatch_kp16(const Ctx& c, MrsWork* w, const OpView<float>& J, const __nv_bfloat16* Q16,
                                 const double* alpha, int k, int kp, double shift, double sign, const double* rhs,
                                 float* x, float* Y, long long ystride, float* P, double tol, int maxit,
                                 LaunchOut lo) {
    switch (kp) {
#define ASSS_MRS16_CASE(KPV) \
    case KPV:                \
        return launch_mrs<float, KPV, FMT, true>(c, w, J, nullptr, alpha, k, shift, sign, rhs, x, Y, ystride, P, tol, \
                                                 maxit, lo, Q16);
        ASSS_MRS16_CASE(8)
        ASSS_MRS16_CASE(16)
        ASSS_MRS16_CASE(24)
        ASSS_MRS16_CASE(32)
        ASSS_MRS16_CASE(48)
        ASSS_MRS16_CASE(64)
#undef ASSS_MRS16_CASE
        default:
            set_error("unsupported BF16 Lanczos width %d", kp);
            return ASSS_ERR_UNSUPPORTED;
    }
}

template <class T>
static asss_status dispatch_mrs(const Ctx& c, MrsWork* w, const DSell<T>* sell, const DSkewDia<T>* dia, const T* Q,
                                const double* alpha, int k, int kp, double shift, double sign, const double* rhs,
                                T* x, DBuf<T>& Ybuf, int& ylay, T* P, double tol, int maxit, long long* nnz_read,
                                LaunchOut lo, const __nv_bfloat16* Q16 = nullptr, int kp16 = 0,
                                const IldlFactor* fac = nullptr) {
    OpView<T> v;
    if (dia && dia->ndiag > MRS_MAXDIAG) dia = nullptr;
    T* Y = nullptr;
    long long ystride = 0;
    ASSS_TRY(y_layout<T>(w, Ybuf, ylay, (dia && !fac) ? dia->halo : 0, c.stream, &Y, &ystride));
    if (fac) {
        if (Q16) {
            set_error("the factored inner operator reads Q_k in FP32 or FP64 only");
            return ASSS_ERR_UNSUPPORTED;
        }
        v.n = fac->n;
        v.fmt = 3;
        v.nslices = cdiv(fac->n, 32);
        v.key = fac;
        v.fac = fac;
        v.nnz = fac->nl + fac->nu + fac->nj;
        *nnz_read = v.nnz;
        return dispatch_kp<T, 3>(c, w, v, Q, alpha, k, kp, shift, sign, rhs, x, Y, ystride, P, tol, maxit, lo);
    }
    if (dia) {
        v.n = dia->n;
        v.fmt = 1;
        v.nslices = cdiv(dia->n, 32);
        v.ndiag = dia->ndiag;
        v.off = dia->off.p;
        v.U = dia->U.p + dia->halo;
        v.ustride = dia->ustride;
        v.halo = dia->halo;
        v.key = dia;
        v.nnz = dia->nnz;
        *nnz_read = v.nnz;
        if constexpr (sizeof(T) == 4) {
            if (Q16) return dispatch_kp16<1>(c, w, v, Q16, alpha, k, kp16, shift, sign, rhs, x, Y, ystride, P, tol,
                                             maxit, lo);
        }
        return dispatch_kp<T, 1>(c, w, v, Q, alpha, k, kp, shift, sign, rhs, x, Y, ystride, P, tol, maxit, lo);
    }
    if (!sell) {
        set_error("mrs: no operator storage");
        return ASSS_ERR_ARG;
    }
    v.n = sell->n;
    v.fmt = 0;
    v.nslices = sell->nslices;
    v.sptr = sell->sptr.p;
    v.col = sell->col.p;
    v.val = sell->val.p;
    v.rowmap = sell->rowmap.p;
    v.units = sell->units.p;
    v.uoff = sell->uoff.p;
    v.hacc = const_cast<T*>(sell->hacc.p);
    v.hcnt = const_cast<unsigned*>(sell->hcnt.p);
    v.nheavy = sell->nheavy;
    v.split = sell->split;
    v.key = sell;
    v.nnz = sell->nnz;
    *nnz_read = v.nnz;
    if constexpr (sizeof(T) == 4) {
        if (Q16) return dispatch_kp16<0>(c, w, v, Q16, alpha, k, kp16, shift, sign, rhs, x, Y, ystride, P, tol, maxit,
                                         lo);
    }
    return dispatch_kp<T, 0>(c, w, v, Q, alpha, k, kp, shift, sign, rhs, x, Y, ystride, P, tol, maxit, lo);
}

asss_status mrs_solve(const Ctx& c, MrsWork* w, const MrsOperator& op, bool fp32, double shift, double sign,
                      const double* rhs, double* x64, float* x32, double tol, int maxit, double* qtz, MrsResult* res,
                      bool sync_result) {
    NvtxRange nv_("asss:mrs");
    int n = w->n;
    if (w->log_n == MrsWork::LOG_CAP) ASSS_TRY(mrs_collect(c, w, nullptr));
    LaunchOut lo{w->log_n, qtz};
    while ((int)w->evs.size() < 2 * (lo.slot + 1)) {
        cudaEvent_t e;
        ASSS_CUDA(cudaEventCreate(&e));
        w->evs.push_back(e);
    }
    long long nnz_read = 0;
    if (fp32) {
        if ((!op.J32 && !op.D32 && !op.F) || !x32) {
            set_error("FP32 mrs needs the FP32 operator and an FP32 output");
            return ASSS_ERR_ARG;
        }
        if (!w->P32.p) ASSS_TRY(w->P32.alloc((int64_t)2 * n));
        ASSS_TRY(dispatch_mrs<float>(c, w, op.J32, op.D32, op.Q32, op.alpha, op.k, op.kp, shift, sign, rhs, x32,
                                     w->Y32, w->halo32, w->P32.p, tol, maxit, &nnz_read, lo,
                                     (const __nv_bfloat16*)op.Q16, op.kp16, op.F));
    } else {
        if ((!op.J64 && !op.D64 && !op.F) || !x64) {
            set_error("FP64 mrs needs the FP64 operator and an FP64 output");
            return ASSS_ERR_ARG;
        }
        if (!w->P64.p) ASSS_TRY(w->P64.alloc((int64_t)2 * n));
        ASSS_TRY(dispatch_mrs<double>(c, w, op.J64, op.D64, op.Q64, op.alpha, op.k, op.kp, shift, sign, rhs, x64,
                                      w->Y64, w->halo64, w->P64.p, tol, maxit, &nnz_read, lo, nullptr, 0, op.F));
    }
    // algorithmic bytes: set-up pass (rhs in FP64, Y/x/P written, Q row), per step
    // (matrix entries - SELL ones with a 4-byte index -, Q row, gathered/own y,
    // y_old, y_new, p r/w, x r/w), final pass (y, p, x r/w; Q^T x needs no pass over Q)
    long long T = fp32 ? 4 : 8;
    long long nn = n, kp = op.kp;
    long long qrow = (fp32 && op.Q16) ? 2LL * op.kp16 : kp * T;  // bytes of one Q row as read
    long long per_entry = (!op.F && (fp32 ? (op.D32 != nullptr) : (op.D64 != nullptr))) ? T : T + 4;
    if ((int)w->log_nnz.size() <= lo.slot) {
        w->log_nnz.resize(lo.slot + 1);
        w->log_per_row.resize(lo.slot + 1);
    }
    w->log_nnz[lo.slot] = nn * (8 + 4 * T + qrow) + nn * 4 * T;
    // factored operator: + wd, t written and gathered, w written and gathered, per step
    w->log_per_row[lo.slot] = nnz_read * per_entry + nn * (7 * T + qrow) + (op.F ? nn * 5 * T : 0);
    w->log_n++;
    if (sync_result) {
        std::vector<MrsResult> v;
        ASSS_TRY(mrs_collect(c, w, &v));
        if (res) *res = v.back();
    }
    return ASSS_OK;
}

asss_status mrs_collect(const Ctx& c, MrsWork* w, std::vector<MrsResult>* out) {
    int nl = w->log_n;
    if (nl == 0) return ASSS_OK;
    std::vector<int> its(nl);
    std::vector<double> ratio(nl);
    int herr = 0;
    ASSS_CUDA(cudaMemcpyAsync(its.data(), w->its_log.p, sizeof(int) * nl, cudaMemcpyDeviceToHost, c.stream));
    ASSS_CUDA(cudaMemcpyAsync(ratio.data(), w->ratio_log.p, sizeof(double) * nl, cudaMemcpyDeviceToHost, c.stream));
    ASSS_CUDA(cudaMemcpyAsync(&herr, w->err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    std::vector<unsigned long long> tl(w->trace.p ? MRS_TRACE_SLOTS : 0);
    if (w->trace.p)
        ASSS_CUDA(cudaMemcpyAsync(tl.data(), w->trace.p, sizeof(unsigned long long) * MRS_TRACE_SLOTS,
                                  cudaMemcpyDeviceToHost, c.stream));
    ASSS_CUDA(cudaStreamSynchronize(c.stream));
    w->log_n = 0;
    if (w->trace.p) {
        // last launch: phase durations in ns (block 0)
        fprintf(stderr, "mrs timeline (block 0, ns): phase0-pass %llu barrier %llu setup %llu |",
                tl[1] - tl[0], tl[2] - tl[1], tl[3] - tl[2]);
        int steps = its[nl - 1] < MRS_TRACE_STEPS ? its[nl - 1] : MRS_TRACE_STEPS;
        for (int j = 1; j < steps; ++j) {
            int tb = 4 + 5 * (j - 1);
            unsigned long long prev = (j == 1) ? tl[3] : tl[tb - 1];
            fprintf(stderr, " [pass %llu part %llu bar %llu red %llu sc+u %llu]", tl[tb] - prev,
                    tl[tb + 1] - tl[tb], tl[tb + 2] - tl[tb + 1], tl[tb + 3] - tl[tb + 2], tl[tb + 4] - tl[tb + 3]);
        }
        fprintf(stderr, "\n");
    }
    for (int i = 0; i < nl; ++i) {
        if (its[i] < 0) continue;  // a launch that found its skip flag set did no work
        float ms = 0.f;
        ASSS_CUDA(cudaEventElapsedTime(&ms, w->evs[2 * i], w->evs[2 * i + 1]));
        MrsResult r;
        r.its = its[i];
        r.ratio = ratio[i];
        r.status = herr;
        r.ms = ms;
        r.bytes = w->log_nnz[i] + (long long)its[i] * w->log_per_row[i];
        w->tot.its += r.its;
        w->tot.launches += 1;
        w->tot.ms += r.ms;
        w->tot.bytes += r.bytes;
        if (out) out->push_back(r);
    }
    if (herr) {
        // the status word is sticky until read here: later launches exit at once
        ASSS_CUDA(cudaMemsetAsync(w->err.p, 0, sizeof(int), c.stream));
        set_error("mrs: a grid barrier wait exceeded its budget");
        return (asss_status)herr;
    }
    return ASSS_OK;
}

void mrs_set_skip(MrsWork* w, const int* flag) { w->skip = flag; }
const int* mrs_get_skip(const MrsWork* w) { return w->skip; }

MrsTotals mrs_take_totals(MrsWork* w) {
    MrsTotals t = w->tot;
    w->tot = MrsTotals();
    return t;
}


// ===========================================================================
// Allocation-free entry point.  Its scratch is one file-scope device array, so
// the call itself never allocates device memory.
// ===========================================================================
constexpr long long NOALLOC_MAX_N = 1LL << 16;
constexpr int NOALLOC_MAX_BLOCKS = 512;
constexpr long long NOALLOC_CTRL = 8;                                          // control words
constexpr long long NOALLOC_PART = 2LL * (MRS_KPMAX + 1) * NOALLOC_MAX_BLOCKS;  // reduction partials
constexpr long long NOALLOC_BLK = (NOALLOC_MAX_BLOCKS + 2) / 2;                // block->slice table (ints)
constexpr long long NOALLOC_DOUBLES = NOALLOC_CTRL + NOALLOC_PART + NOALLOC_BLK + 5 * NOALLOC_MAX_N;

// [ctrl | partials | block table | Y: 3 slots of n | P: 2 slots of n]
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// device (or managed) memory that belongs to device dev
static bool noalloc_on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

static double* noalloc_base(int* status) {
    static std::mutex mu;
    static double* base[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
        *status = ASSS_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!base[dev]) {
        double* ptr = nullptr;
        e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            *status = ASSS_ERR_CUDA;
            return nullptr;
        }
        base[dev] = ptr;
    }
    *status = ASSS_OK;
    return base[dev];
}

__global__ void k_noalloc_check_rp(const int64_t* rp, int64_t n, int64_t nnz, int* flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int64_t v = rp[i];
    if ((i == 0 && v != 0) || (i == n && v != nnz) || v < 0 || v > nnz || (i < n && rp[i + 1] < v)) atomicOr(flag, 1);
}

__global__ void k_noalloc_check_ci(const int64_t* rp, const int32_t* ci, int64_t n, int* flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] < 0 || ci[e] >= n) {
            atomicOr(flag, 2);
            return;
        }
}

// columns k..kp-1 of the row-major q must be zero: they enter x through q[m] * u[m]
// with u[m] = 0, so a NaN or Inf there would turn x into NaN
__global__ void k_noalloc_check_qpad(const double* q, int64_t n, int k, int kp, int* flag) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = kp - k;
    if (w <= 0 || t >= n * w) return;
    const int64_t i = t / w;
    const int m = k + (int)(t % w);
    if (q[i * kp + m] != 0.0) atomicOr(flag, 4);
}

template <int KP>
static asss_status noalloc_launch(int nblk, cudaStream_t s, MrsParams<double>& prm) {
    void* args[] = {&prm};
    ASSS_CUDA(cudaLaunchCooperativeKernel((const void*)k_mrs<double, KP, 2>, dim3(nblk), dim3(MRS_THREADS), args, 0,
                                          s));
    count_launch();
    return ASSS_OK;
}

template <int KP>
static asss_status noalloc_occupancy(int* occ) {
    ASSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_mrs<double, KP, 2>, MRS_THREADS, 0));
    return ASSS_OK;
}

}  // namespace asss

using namespace asss;

extern "C" asss_status asss_mrs_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                        const double* val, int k, int kp, const double* q_rowmajor,
                                        const double* alpha, double shift, double sign, const double* b, double* x,
                                        double tol, int maxit, int* its, double* ratio, void* stream) {
    if (n < 1 || n > NOALLOC_MAX_N) {
        set_error("asss_mrs_noalloc: n = %lld is outside 1..%lld, the size of its static scratch", (long long)n,
                  NOALLOC_MAX_N);
        return ASSS_ERR_ARG;
    }
    if (nnz < 0 || nnz >= (1LL << 40) || !row_ptr || !col_idx || !val || !b || !x || maxit < 1 || !(shift > 0.0) ||
        k < 0 || k > kp ||
        (k > 0 && !q_rowmajor) || (k > 1 && !alpha)) {
        set_error("asss_mrs_noalloc: invalid arguments");
        return ASSS_ERR_ARG;
    }
    if (sign != 1.0 && sign != -1.0) {
        set_error("asss_mrs_noalloc: sign must be +1 or -1");
        return ASSS_ERR_ARG;
    }
    int cur_dev = 0;
    ASSS_CUDA(cudaGetDevice(&cur_dev));
    // every array is read in place by the kernel: it must be memory of the current
    // device (another GPU's memory would be read without peer access) and aligned for
    // the kernel's vector loads (q rows are read 16 bytes at a time)
    struct Arr {
        const void* p;
        size_t align;
        const char* name;
    };
    const Arr arrs[] = {{row_ptr, 8, "row_ptr"}, {col_idx, 4, "col_idx"}, {val, 8, "val"},
                        {b, 8, "b"},             {x, 8, "x"},             {k > 0 ? q_rowmajor : nullptr, 16, "q"},
                        {k > 1 ? alpha : nullptr, 8, "alpha"}};
    for (const Arr& a : arrs) {
        if (!a.p) continue;
        if (!noalloc_on_device(a.p, cur_dev)) {
            set_error("asss_mrs_noalloc: %s must be device memory of the current device %d", a.name, cur_dev);
            return ASSS_ERR_ARG;
        }
        if (((uintptr_t)a.p) % a.align != 0) {
            set_error("asss_mrs_noalloc: %s must be aligned to %zu bytes", a.name, a.align);
            return ASSS_ERR_ARG;
        }
    }
    int st = ASSS_OK;
    double* base = noalloc_base(&st);
    if (!base) return (asss_status)st;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    ASSS_TRY(make_ctx(c, stream, 2000.0));
    int occ = 0;
    switch (kp) {
#define NA_OCC(KPV) \
    case KPV:       \
        ASSS_TRY(noalloc_occupancy<KPV>(&occ)); \
        break;
        NA_OCC(0) NA_OCC(4) NA_OCC(8) NA_OCC(12) NA_OCC(16) NA_OCC(20) NA_OCC(24) NA_OCC(32) NA_OCC(48) NA_OCC(64)
#undef NA_OCC
        default:
            set_error("asss_mrs_noalloc: kp must be one of 0,4,8,12,16,20,24,32,48,64");
            return ASSS_ERR_ARG;
    }
    if (occ < 1) {
        set_error("mrs kernel cannot be resident");
        return ASSS_ERR_CUDA;
    }
    if (occ > 4) occ = 4;
    int nslices = (int)((n + 31) / 32);
    int nblk = c.sms * occ;
    if (nblk > NOALLOC_MAX_BLOCKS) nblk = NOALLOC_MAX_BLOCKS;
    int need = (nslices + MRS_WARPS - 1) / MRS_WARPS;
    if (nblk > need) nblk = need;
    unsigned* ctrl = reinterpret_cast<unsigned*>(base);  // [0] count [1] gen [2] err [3] its; ratio at base[3]
    double* part = base + NOALLOC_CTRL;
    int* blk = reinterpret_cast<int*>(base + NOALLOC_CTRL + NOALLOC_PART);
    double* Y = base + NOALLOC_CTRL + NOALLOC_PART + NOALLOC_BLK;
    double* P = Y + 3 * n;
    // the control words must start at zero; everything else is written before it is read
    ASSS_CUDA(cudaMemsetAsync(base, 0, sizeof(double) * NOALLOC_CTRL, s));
    // the CSR is read in place: check row pointers, then column indices (flag in ctrl[2])
    {
        int* flag = reinterpret_cast<int*>(ctrl + 2);
        k_noalloc_check_rp<<<(int)((n + 256) / 256), 256, 0, s>>>(row_ptr, n, nnz, flag);
        ASSS_CHECK_LAUNCH();
        int hf = 0;
        ASSS_CUDA(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        if (!hf) {
            k_noalloc_check_ci<<<(int)((n + 255) / 256), 256, 0, s>>>(row_ptr, col_idx, n, flag);
            ASSS_CHECK_LAUNCH();
            if (k > 0 && kp > k) {
                const int64_t cnt = n * (int64_t)(kp - k);
                k_noalloc_check_qpad<<<(int)((cnt + 255) / 256), 256, 0, s>>>(q_rowmajor, n, k, kp, flag);
                ASSS_CHECK_LAUNCH();
            }
            ASSS_CUDA(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            ASSS_CUDA(cudaStreamSynchronize(s));
        }
        if (hf & 3) {
            set_error("asss_mrs_noalloc: malformed CSR (row pointers or column indices)");
            return ASSS_ERR_PATTERN;
        }
        if (hf) {
            set_error("asss_mrs_noalloc: columns k..kp-1 of q must be zero");
            return ASSS_ERR_ARG;
        }
    }
    k_partition<<<(nblk + 128) / 128, 128, 0, s>>>(nullptr, nslices, nblk, blk);
    ASSS_CHECK_LAUNCH();
    MrsParams<double> prm;
    memset(&prm, 0, sizeof(prm));
    prm.n = (int)n;
    prm.crp = (const long long*)row_ptr;
    prm.cci = col_idx;
    prm.cval = val;
    prm.ystride = n;
    prm.Q = q_rowmajor;
    prm.alpha = alpha;
    prm.k = k;
    prm.shift = shift;
    prm.sign = sign;
    prm.rhs = b;
    prm.x = x;
    prm.Y = Y;
    prm.P = P;
    prm.part = part;
    prm.gb.count = ctrl;
    prm.gb.gen = ctrl + 1;
    prm.gb.err = reinterpret_cast<int*>(ctrl + 2);
    prm.blk_slice = blk;
    prm.tol = tol;
    prm.maxit = maxit;
    prm.budget = c.wait_cycles;
    prm.out_its = reinterpret_cast<int*>(ctrl + 3);
    prm.out_ratio = base + 3;
    prm.qtz = nullptr;
    switch (kp) {
#define NA_CASE(KPV) \
    case KPV:        \
        ASSS_TRY(noalloc_launch<KPV>(nblk, s, prm)); \
        break;
        NA_CASE(0) NA_CASE(4) NA_CASE(8) NA_CASE(12) NA_CASE(16) NA_CASE(20) NA_CASE(24) NA_CASE(32) NA_CASE(48)
        NA_CASE(64)
#undef NA_CASE
    }
    unsigned h[4] = {0, 0, 0, 0};
    double hr = 0.0;
    ASSS_CUDA(cudaMemcpyAsync(h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaMemcpyAsync(&hr, base + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (h[2]) {
        set_error("asss_mrs_noalloc: a grid barrier wait exceeded its budget");
        return ASSS_ERR_TIMEOUT;
    }
    if (its) *its = (int)h[3];
    if (ratio) *ratio = hr;
    return ASSS_OK;
}
