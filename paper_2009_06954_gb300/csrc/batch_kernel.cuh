// Batched solves (many matrices of uneven size, many right-hand sides): one
// persistent launch in which every CTA takes (matrix, right-hand side) work items
// from a global counter and runs the whole solve of that item in block scope:
//   the refinement loop on the true FP64 residual and flexible GMRES (outer, FP64,
//   §4.1), P^-1 by SMW (Eq. smw) around the mrs iteration of App. B on the
//   deflated shifted skew system (FP32, skew-diagonal storage of J~, §3.1-3.2).
// The algorithms are those of the single-system path (asss.cu, mrs.cu); what
// changes is the scope: block reductions and __syncthreads instead of grid
// barriers and kernel launches, so small systems do not pay a launch or a grid
// synchronisation per step.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "mrs_dev.cuh"

namespace asss {

constexpr int BMAX_WARPS = 32;
constexpr int BKPMAX = 32;   // largest padded Lanczos width handled by the batched kernel
constexpr int BMMAX = 320;   // largest SMW rank k + r


// scalar state of the FP32 inner recurrence (kept in FP32 like its vectors: the
// FP64 pipe of this part is narrow and sits on the critical path of every step)
struct BScalars {
    float r0, rr0, nu, coef_old, theta_t, c_prev, s_prev, delta_prev, G;
    float nu_p, delta_pp, rtheta_p, xcoef_p;
    float fin_nu, fin_delta, fin_rtheta, fin_xcoef;
    float ratio;
    int its, stop;
};

struct BatchShared {
    BatchMat M;
    float red[BKPMAX + 1];
    float wsum[BMAX_WARPS][BKPMAX + 1];
    double tmp[BMAX_WARPS + 1];
    double wd[BMAX_WARPS][4];
    float u[BKPMAX];
    float cf[12];
    float alpha[BKPMAX];
    int off[64];
    double H[(BATCH_RMAX + 1) * BATCH_RMAX];
    double cs[BATCH_RMAX + 1], sn[BATCH_RMAX + 1], g[BATCH_RMAX + 2], hv[BATCH_RMAX + 1], hv2[BATCH_RMAX + 1],
        yv[BATCH_RMAX + 1];
    float wv[BMMAX];  // U^T z for the SMW correction (FP32, like the inner solve)
    // Q^T z of the final iterate from the reduced Q^T y_j (no pass over Q): Q^T y_j,
    // Q^T p of the last two directions, Q^T z, and step j's nu, delta, 1/theta, xcoef
    float qty[BKPMAX], qtp[2][BKPMAX], qtx[BKPMAX], pq[4];
    BScalars sc;
    unsigned long long prof[BATCH_NPROF + 1];  // phase times of this CTA (thread 0), last stamp
    int item;
    int steps;
    int brk;
};

// sum over the block of one double per thread; every thread gets the result
__device__ __forceinline__ double bsum(double v, BatchShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh.tmp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? sh.tmp[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sh.tmp[BMAX_WARPS] = t;
    }
    __syncthreads();
    return sh.tmp[BMAX_WARPS];
}

__device__ __forceinline__ double bdot(const double* __restrict__ a, const double* __restrict__ b, int n,
                                       BatchShared& sh) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += a[i] * b[i];
    return bsum(acc, sh);
}

// out[a] = V_a^T x for a < cnt (V column-major with leading dimension ld): four dot
// products per sweep and one block reduction per sweep (warps added in order)
__device__ __forceinline__ void bdots(const double* __restrict__ V, long long ld, int cnt,
                                      const double* __restrict__ x, int n, double* out,
                                      double (&wd)[BMAX_WARPS][4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < cnt; c0 += 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double xi = x[i];
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (c0 + t < cnt) acc[t] += V[(size_t)(c0 + t) * ld + i] * xi;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const double v = warp_sum(acc[t]);
            if (lane == 0) wd[warp][t] = v;
        }
        __syncthreads();
        if (threadIdx.x < 4 && c0 + (int)threadIdx.x < cnt) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += wd[w][threadIdx.x];
            out[c0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// y = A x for a CSR matrix, one row per thread (rows strided over the block); the
// diagonal copies of the one-system path measured slower here, where a CTA's rows are
// few and the gathers hit L1
// (WIDE: 128 registers a thread, so a row's indices and values are loaded eight at a
// time ahead of their gathers)
template <bool WIDE>
__device__ __forceinline__ void bspmv(const int* __restrict__ rp, const int* __restrict__ ci,
                                      const double* __restrict__ v, const double* __restrict__ x,
                                      double* __restrict__ y, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        if constexpr (WIDE) {
            const int e1 = rp[i + 1];
            for (int e = rp[i]; e < e1; e += 8) {
                int cc[8];
                double vv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool in = e + u < e1;
                    cc[u] = in ? ci[e + u] : 0;
                    vv[u] = in ? v[e + u] : 0.0;
                }
                double g[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) g[u] = e + u < e1 ? x[cc[u]] : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u) s += vv[u] * g[u];
            }
        } else {
            for (int e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * x[ci[e]];
        }
        y[i] = s;
    }
    __syncthreads();
}

template <int KP, bool QB>
__device__ __forceinline__ void bq_row(const BatchMat& M, int i, float (&q)[KP > 0 ? KP : 1]) {
    if constexpr (KP > 0) {
        if constexpr (QB) {
            const uint4* row = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(M.Q16) +
                                                             (size_t)i * KP);
#pragma unroll
            for (int t = 0; t < KP / 8; ++t) {
                uint4 v = __ldg(row + t);
                const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float2 f = __bfloat1622float2(h2[e]);
                    q[8 * t + 2 * e] = f.x;
                    q[8 * t + 2 * e + 1] = f.y;
                }
            }
        } else {
            const float4* row = reinterpret_cast<const float4*>(M.Q32 + (size_t)i * KP);
#pragma unroll
            for (int t = 0; t < KP / 4; ++t) {
                float4 v = __ldg(row + t);
                q[4 * t] = v.x;
                q[4 * t + 1] = v.y;
                q[4 * t + 2] = v.z;
                q[4 * t + 3] = v.w;
            }
        }
    }
}

// float-pair (TwoSum) addition, about 44 significant bits without the FP64 pipe
__device__ __forceinline__ float2 bdf_add(float2 a, float2 b) {
    float s = a.x + b.x;
    float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    float hi = s + e;
    float lo = e - (hi - s);
    return make_float2(hi, lo);
}

// block reduction of the KP+1 per-thread sums of an mrs step into sh.red: warp sums
// in FP32, then warp 0 adds the warps' sums in a fixed order in float pairs and holds
// sh.red afterwards (the scalar update that reads it runs in warp 0 too, so one block
// barrier is saved)
template <int KP>
__device__ __forceinline__ void bred_w0(float (&tacc)[KP + 1], BatchShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int v = 0; v <= KP; ++v) {
        float d = warp_sum(tacc[v]);
        if (lane == 0) sh.wsum[warp][v] = d;
    }
    __syncthreads();
    if (warp == 0) {
        for (int v = lane; v <= KP; v += 32) {
            float2 t = make_float2(0.f, 0.f);
            for (int w = 0; w < nw; ++w) t = bdf_add(t, make_float2(sh.wsum[w][v], 0.f));
            sh.red[v] = t.x + t.y;
        }
        __syncwarp();
    }
}

// u = nu S_k (Q^T y) by the lanes of warp 0 (after its lane 0 set nu)
template <int KP>
__device__ __forceinline__ void bmake_u_w0(const BatchMat& M, BatchShared& sh) {
    const int lane = threadIdx.x & 31;
    for (int m = lane; m < KP; m += 32) {
        float u = 0.f;
        if (m < M.k) {
            if (m + 1 < M.k) u += sh.alpha[m] * sh.red[2 + m] * sh.sc.nu;
            if (m > 0) u -= sh.alpha[m - 1] * sh.red[m] * sh.sc.nu;
        }
        sh.u[m] = u;
    }
}

__device__ __forceinline__ void bset_coefs(BatchShared& sh) {
    BScalars& c = sh.sc;
    sh.cf[0] = c.nu;
    sh.cf[2] = c.coef_old;
    sh.cf[3] = c.nu_p;
    sh.cf[4] = c.delta_pp;
    sh.cf[5] = c.rtheta_p;
    sh.cf[6] = c.xcoef_p;
    if (c.stop) {
        sh.cf[7] = c.fin_nu;
        sh.cf[8] = c.fin_delta;
        sh.cf[9] = c.fin_rtheta;
        sh.cf[10] = c.fin_xcoef;
    }
}

// mrs (App. B) in block scope on (I + J_bar) z = u, J_bar = J~ - Q S_k Q^T, FP32 vectors;
// z in FP32, Q^T z of the final iterate into sh.wv[0..k); returns the step count.
template <int KP, bool QB, bool WIDE>
__device__ int bmrs(const double* u, float* z, float* Y, long long ys, float* P, double tol, int maxit,
                    BatchShared& sh) {
    const BatchMat& M = sh.M;
    const int n = M.n;
    const int h = M.halo;
    // zero this matrix's halo band of every slot (the workspace is shared by items)
    for (int t = threadIdx.x; t < 6 * h; t += blockDim.x) {
        int slot = t / (2 * h), e = t % (2 * h);
        int idx = e < h ? -h + e : n + (e - h);
        Y[slot * ys + idx] = 0.f;
    }
    for (int m = threadIdx.x; m < KP; m += blockDim.x) {
        sh.qtp[0][m] = 0.f;
        sh.qtp[1][m] = 0.f;
        sh.qtx[m] = 0.f;
    }
    // warp 1: fold direction p_jj into Q^T z (p_jj = (nu y_jj - delta p_{jj-2}) / theta,
    // z = sum xcoef_jj p_jj)
    auto qtx_fold = [&](int jj) {
        const int ln = threadIdx.x & 31;
        if (ln < M.k) {
            float* pp = sh.qtp[jj & 1];
            const float v = (sh.pq[0] * sh.qty[ln] - sh.pq[1] * pp[ln]) * sh.pq[2];
            pp[ln] = v;
            sh.qtx[ln] += sh.pq[3] * v;
        }
    };
    float tacc[KP + 1];
#pragma unroll
    for (int v = 0; v <= KP; ++v) tacc[v] = 0.f;
    {
    const double* __restrict__ ur = u;
    float* __restrict__ Y0 = Y;
    float* __restrict__ zr = z;
    float* __restrict__ P0 = P;
    float* __restrict__ P1 = P + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float b = (float)ur[i];
        Y0[i] = b;
        zr[i] = 0.f;
        P0[i] = 0.f;
        P1[i] = 0.f;
        tacc[0] += b * b;
        float q[KP > 0 ? KP : 1];
        bq_row<KP, QB>(M, i, q);
#pragma unroll
        for (int m = 0; m < KP; ++m) tacc[1 + m] += q[m] * b;
    }
    }
    bred_w0<KP>(tacc, sh);
    const int lane0 = threadIdx.x & 31, warp0 = threadIdx.x >> 5;
    if (warp0 == 0 && lane0 == 0) {
        BScalars& c = sh.sc;
        const float r0 = sqrtf(sh.red[0]);
        c.r0 = r0;
        c.rr0 = r0 > 0.f ? 1.f / r0 : 0.f;
        c.nu = c.rr0;
        c.coef_old = 0.f;
        c.theta_t = 1.f;
        c.c_prev = 1.f;
        c.s_prev = 0.f;
        c.delta_prev = 0.f;
        c.G = r0;
        c.nu_p = 0.f;
        c.delta_pp = 0.f;
        c.rtheta_p = 1.f;
        c.xcoef_p = 0.f;
        c.ratio = 0.f;
        c.its = 0;
        c.stop = r0 > 0.f ? 0 : 1;
        bset_coefs(sh);
    }
    if (warp0 == 0) {
        __syncwarp();
        if (!sh.sc.stop) bmake_u_w0<KP>(M, sh);
    }
    __syncthreads();
    if (sh.sc.stop) {
        for (int v = threadIdx.x; v < M.k; v += blockDim.x) sh.wv[v] = 0.f;
        __syncthreads();
        return 0;
    }
    // loop invariants in registers, and the vectors of a step marked as not aliasing one
    // another, so loads of later rows may be scheduled ahead of this row's stores
    const float* __restrict__ Ubase = M.U;
    const long long ust = M.ustride;
    const int nd = M.ndiag;
    const int* __restrict__ soff = sh.off;
    for (int j = 1; j <= maxit; ++j) {
        if (KP > 0 && warp0 == 1) {
            // off the step's synchronisation chain: step j-1's direction, then Q^T y_j
            if (j >= 2) qtx_fold(j - 1);
            if (lane0 < M.k) sh.qty[lane0] = sh.red[1 + lane0];
        }
        const float* __restrict__ Ycur = Y + (size_t)((j - 1) % 3) * ys;
        const float* __restrict__ Yold = Y + (size_t)((j + 1) % 3) * ys;
        float* __restrict__ Ynew = Y + (size_t)(j % 3) * ys;
        float* __restrict__ Pj1 = P + (size_t)((j - 1) & 1) * n;
        float* __restrict__ zz = z;
        const float tnu = sh.cf[0], tco = sh.cf[2], tnp = sh.cf[3], tdpp = sh.cf[4], tthp = sh.cf[5],
                    txp = sh.cf[6];
#pragma unroll
        for (int v = 0; v <= KP; ++v) tacc[v] = 0.f;
        // skew diagonals: one row per thread in natural order; SELL-C-sigma: one slot
        // per thread (coalesced matrix reads), its row from the slot map
        const bool sell = nd == 0;
        const int nrun = sell ? M.nslots : n;
        for (int s_ = threadIdx.x; s_ < nrun; s_ += blockDim.x) {
            const int i = (sell && M.rowmap) ? M.rowmap[s_] : s_;
            if (i >= n) continue;
            const float yold = j >= 2 ? Yold[i] : 0.f;
            const float pold = j >= 2 ? Pj1[i] : 0.f;
            float acc = 0.f;
            if (sell) {
                const int sl = s_ >> 5, t = s_ & 31;
                const int b0 = __ldg(&M.sptr[sl]);
                const int width = (__ldg(&M.sptr[sl + 1]) - b0) >> 5;
                const int* cp = M.scol + b0 + t;
                const float* vp = M.sval + b0 + t;
#pragma unroll 4
                for (int kk = 0; kk < width; ++kk) acc += __ldg(vp + kk * 32) * Ycur[__ldg(cp + kk * 32)];
            } else {
                const float* Ud = Ubase + i;
                const float* yi = Ycur + i;
                if constexpr (WIDE) {
                    // 128 registers: the loads of all diagonals of the row in flight together
#pragma unroll 12
                    for (int d = 0; d < nd; ++d, Ud += ust) {
                        const int m = soff[d];
                        acc += __ldg(Ud) * yi[m] - __ldg(Ud - m) * yi[-m];
                    }
                } else {
                    for (int d = 0; d < nd; ++d, Ud += ust) {
                        const int m = soff[d];
                        acc += __ldg(Ud) * yi[m] - __ldg(Ud - m) * yi[-m];
                    }
                }
            }
            float q[KP > 0 ? KP : 1];
            bq_row<KP, QB>(M, i, q);
            float dq = 0.f;
#pragma unroll
            for (int m = 0; m < KP; ++m) dq += q[m] * sh.u[m];
            const float ynew = tnu * acc - dq + tco * yold;
            Ynew[i] = ynew;
            tacc[0] += ynew * ynew;
#pragma unroll
            for (int m = 0; m < KP; ++m) tacc[1 + m] += q[m] * ynew;
            if (j >= 2) {
                float pv = (tnp * yold - tdpp * pold) * tthp;
                Pj1[i] = pv;
                zz[i] += txp * pv;
            }
        }
        bred_w0<KP>(tacc, sh);
        if (warp0 == 0 && lane0 == 0) {
            BScalars& c = sh.sc;
            const float beta = sqrtf(sh.red[0]);
            const float theta = sqrtf(c.theta_t * c.theta_t + beta * beta);
            const float rth = 1.f / theta;
            const float cc = c.theta_t * rth, s = beta * rth;
            const float delta = -c.s_prev * beta;
            const float theta_t_next = c.c_prev * theta;
            const float xcoef = c.G * cc;
            const float Gn = -c.G * s;
            sh.pq[0] = c.nu;
            sh.pq[1] = c.delta_prev;
            sh.pq[2] = rth;
            sh.pq[3] = xcoef;
            c.ratio = fabsf(Gn) * c.rr0;
            c.its = j;
            if (c.ratio < tol || j == maxit) {
                c.stop = 1;
                c.fin_nu = c.nu;
                c.fin_delta = c.delta_prev;
                c.fin_rtheta = rth;
                c.fin_xcoef = xcoef;
            } else {
                c.nu_p = c.nu;
                c.delta_pp = c.delta_prev;
                c.rtheta_p = rth;
                c.xcoef_p = xcoef;
                c.coef_old = beta * c.nu;
                c.nu = (beta != 0.f) ? 1.f / beta : 0.f;
                c.s_prev = s;
                c.c_prev = cc;
                c.delta_prev = delta;
                c.theta_t = theta_t_next;
                c.G = Gn;
            }
            bset_coefs(sh);
        }
        if (warp0 == 0) {
            __syncwarp();
            if (!sh.sc.stop) bmake_u_w0<KP>(M, sh);
        }
        __syncthreads();
        if (sh.sc.stop) {
            const float* __restrict__ Pj = P + (size_t)(j & 1) * n;
            const float tn = sh.cf[7], td = sh.cf[8], tth = sh.cf[9], tx = sh.cf[10];
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                float pv = (tn * Ycur[i] - td * Pj[i]) * tth;
                zz[i] = zz[i] + tx * pv;
            }
            if (warp0 == 1) {
                if (KP > 0) qtx_fold(j);
                if (lane0 < M.k) sh.wv[lane0] = KP > 0 ? sh.qtx[lane0] : 0.f;
            }
            __syncthreads();
            return sh.sc.its;
        }
    }
    return sh.sc.its;
}

// MINB resident CTAs of NT threads per SM fix the register budget of a thread:
// 64 registers at 1024 threads per SM (while one CTA waits in a block reduction the
// others keep loads in flight, but the row loop spills), 80 at 768, and 128 at 512
// (WIDE: a row's loads - all diagonals of J~, a CSR row's entries - in flight together,
// no spills)
template <int KP, bool QB, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_batch(BatchLaunch L) {
    constexpr bool WIDE = NT * MINB <= 512;
    __shared__ BatchShared sh;
    const int R = L.restart;
    const long long nm = L.n_max;
    double* base = L.work + (size_t)blockIdx.x * (size_t)L.work_stride;
    double* r = base;
    double* rh = r + nm;
    double* dy = rh + nm;
    double* t1 = dy + nm;
    double* t2 = t1 + nm;
    double* V = t2 + nm;              // R+1 vectors
    double* Z = V + (R + 1) * nm;     // R vectors
    float* fb = reinterpret_cast<float*>(Z + R * nm);
    const long long ys = nm + 2LL * L.halo_max;
    float* Y = fb + L.halo_max;
    float* P = fb + 3 * ys;
    float* z32 = P + 2 * nm;
    // optional phase timing (thread 0 stamps %globaltimer at block-synchronous points)
    const bool prof = L.prof != nullptr;
    auto mark = [&](int slot) {
        if (prof && threadIdx.x == 0) {
            const unsigned long long t = gtimer();
            sh.prof[slot] += t - sh.prof[BATCH_NPROF];
            sh.prof[BATCH_NPROF] = t;
        }
    };
    if (prof && threadIdx.x == 0) {
        for (int q = 0; q < BATCH_NPROF; ++q) sh.prof[q] = 0ull;
        sh.prof[BATCH_NPROF] = gtimer();
    }

    while (true) {
        if (threadIdx.x == 0) sh.item = (int)atomicAdd(L.next_item, 1u);
        __syncthreads();
        const int it = sh.item;
        if (it >= L.nitems) break;
        const int2 mc = L.items[it];
        if (threadIdx.x == 0) sh.M = L.mats[mc.x];
        __syncthreads();
        const BatchMat& M = sh.M;
        const int n = M.n;
        for (int d = threadIdx.x; d < M.ndiag && d < 64; d += blockDim.x) sh.off[d] = M.off[d];
        for (int a = threadIdx.x; a + 1 < M.k && a < BKPMAX; a += blockDim.x) sh.alpha[a] = (float)M.alpha[a];
        const double* bcol = L.b + L.row_off[mc.x] * L.nrhs + (long long)mc.y * n;
        double* xcol = L.x + L.row_off[mc.x] * L.nrhs + (long long)mc.y * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            xcol[i] = 0.0;
            r[i] = bcol[i];
        }
        __syncthreads();
        const double bn = sqrt(bdot(bcol, bcol, n, sh));
        int outer = 0, inner = 0, cycles = 0, status = ASSS_OK, stall = 0;
        double best = INFINITY, relres = 0.0;
        while (bn > 0.0) {
            const double rn = sqrt(bdot(r, r, n, sh));
            relres = rn / bn;
            if (relres <= L.outer_tol) break;
            if (!(rn == rn)) {
                status = ASSS_ERR_BREAKDOWN;
                break;
            }
            if (outer >= L.outer_maxit) {
                status = ASSS_ERR_NOT_CONVERGED;
                break;
            }
            if (rn < 0.999 * best) {
                best = rn;
                stall = 0;
            } else if (++stall >= 5) {
                status = ASSS_ERR_STAGNATION;
                break;
            }
            // r^ = W P D_r r
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int p = M.perm ? M.perm[i] : i;
                rh[i] = M.w[i] * M.dr[p] * r[p];
            }
            __syncthreads();
            const double eta = fmin(0.5, 0.5 * L.outer_tol * bn / rn);
            int mcyc = R < L.outer_maxit - outer ? R : L.outer_maxit - outer;
            // ---- one flexible GMRES cycle on A_cal dy = r^ ----
            const double beta0 = sqrt(bdot(rh, rh, n, sh));
            if (!(beta0 > 0.0)) {
                status = ASSS_ERR_BREAKDOWN;
                break;
            }
            for (int i = threadIdx.x; i < n; i += blockDim.x) V[i] = rh[i] / beta0;
            if (threadIdx.x == 0) {
                for (int a = 0; a <= R + 1; ++a) sh.g[a] = 0.0;
                sh.g[0] = beta0;
                sh.steps = 0;
            }
            __syncthreads();
            for (int j = 0; j < mcyc; ++j) {
                double* vj = V + j * nm;
                double* zj = Z + j * nm;
                // z_j = P^-1 v_j: mrs, then z - Y (U^T z)
                mark(5);
                inner += bmrs<KP, QB, WIDE>(vj, z32, Y, ys, P, L.inner_tol, L.inner_maxit, sh);
                mark(0);
                for (int a = threadIdx.x; a < M.r; a += blockDim.x) sh.wv[M.k + a] = z32[M.neg[a]];
                __syncthreads();
                // FP32 correction (no per-row FP64 operation); rows of Y as float4 when possible
                const float* __restrict__ Y32 = M.Y32;
                const int mm = M.m;
                const float* __restrict__ z32r = z32;
                double* __restrict__ zjr = zj;
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    float acc = 0.f;
                    const float* yr = Y32 + (size_t)i * mm;
                    if ((mm & 3) == 0) {
                        const float4* y4 = reinterpret_cast<const float4*>(yr);
                        for (int c = 0; c < (mm >> 2); ++c) {
                            const float4 v = __ldg(y4 + c);
                            acc += v.x * sh.wv[4 * c] + v.y * sh.wv[4 * c + 1] + v.z * sh.wv[4 * c + 2] +
                                   v.w * sh.wv[4 * c + 3];
                        }
                    } else {
                        for (int c = 0; c < mm; ++c) acc += yr[c] * sh.wv[c];
                    }
                    zjr[i] = (double)(z32r[i] - acc);
                }
                __syncthreads();
                mark(1);
                // w = A_cal z_j = (W Abar) (S W) z_j, into t2
                bspmv<WIDE>(M.swrp, M.swci, M.swv, zj, t1, n);
                bspmv<WIDE>(M.awrp, M.awci, M.awv, t1, t2, n);
                mark(2);
                // two classical Gram-Schmidt passes
                for (int pass = 0; pass < 2; ++pass) {
                    bdots(V, nm, j + 1, t2, n, pass == 0 ? sh.hv : sh.hv2, sh.wd);
                    const double* hh = pass == 0 ? sh.hv : sh.hv2;
                    const double* __restrict__ Vr = V;
                    double* __restrict__ t2r = t2;
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        double acc = 0.0;
                        for (int a = 0; a <= j; ++a) acc += Vr[a * nm + i] * hh[a];
                        t2r[i] -= acc;
                    }
                    __syncthreads();
                }
                const double hn = sqrt(bdot(t2, t2, n, sh));
                if (threadIdx.x == 0) {
                    double* col = sh.H + j * (R + 1);
                    for (int a = 0; a <= j; ++a) col[a] = sh.hv[a] + sh.hv2[a];
                    col[j + 1] = hn;
                    for (int a = 0; a < j; ++a) {
                        double tq = sh.cs[a] * col[a] + sh.sn[a] * col[a + 1];
                        col[a + 1] = -sh.sn[a] * col[a] + sh.cs[a] * col[a + 1];
                        col[a] = tq;
                    }
                    double rr = hypot(col[j], col[j + 1]);
                    double c = rr != 0.0 ? col[j] / rr : 1.0;
                    double s = rr != 0.0 ? col[j + 1] / rr : 0.0;
                    sh.cs[j] = c;
                    sh.sn[j] = s;
                    col[j] = rr;
                    col[j + 1] = 0.0;
                    sh.g[j + 1] = -s * sh.g[j];
                    sh.g[j] = c * sh.g[j];
                    sh.steps = j + 1;
                    sh.brk = (hn == 0.0 || fabs(sh.g[j + 1]) <= eta * beta0) ? 1 : 0;
                }
                __syncthreads();
                if (sh.brk) {
                    mark(3);
                    break;
                }
                for (int i = threadIdx.x; i < n; i += blockDim.x) V[(j + 1) * nm + i] = t2[i] / hn;
                __syncthreads();
                mark(3);
            }
            const int steps = sh.steps;
            if (threadIdx.x == 0) {
                for (int a = steps - 1; a >= 0; --a) {
                    double acc = sh.g[a];
                    for (int bq = a + 1; bq < steps; ++bq) acc -= sh.H[bq * (R + 1) + a] * sh.yv[bq];
                    sh.yv[a] = acc / sh.H[a * (R + 1) + a];
                }
            }
            __syncthreads();
            // x += D_c S W dy,  dy = Z y
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                double acc = 0.0;
                for (int a = 0; a < steps; ++a) acc += Z[a * nm + i] * sh.yv[a];
                dy[i] = acc;
                t1[i] = M.w[i] * acc;
            }
            __syncthreads();
            bspmv<WIDE>(M.srp, M.sci, M.sv, t1, t2, n);
            for (int i = threadIdx.x; i < n; i += blockDim.x) xcol[i] += M.dc[i] * t2[i];
            __syncthreads();
            bspmv<WIDE>(M.arp, M.aci, M.av, xcol, t1, n);
            for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = bcol[i] - t1[i];
            __syncthreads();
            outer += steps;
            ++cycles;
            mark(4);
        }
        if (threadIdx.x == 0) {
            BatchItemStat st;
            st.outer_its = outer;
            st.inner_its = inner;
            st.status = status;
            st.cycles = cycles;
            st.relres = relres;
            L.stats[it] = st;
        }
        __syncthreads();
    }
    if (prof && threadIdx.x == 0) {
        mark(5);
        for (int q = 0; q < BATCH_NPROF; ++q) atomicAdd(&L.prof[q], sh.prof[q]);
    }
}

// the CTA shapes the tuner chooses from: (threads, resident CTAs per SM)
#define ASSS_BATCH_SHAPES(X) X(256, 4) X(512, 2) X(256, 3) X(384, 2) X(256, 2) X(512, 1)

template <int KP, bool QB>
static asss_status launch_nt(const BatchLaunch& L, int nthreads, int minb, int nblk, cudaStream_t s) {
#define ASSS_BATCH_LAUNCH_CASE(T, B)                     \
    if (nthreads == T && minb == B) {                    \
        k_batch<KP, QB, T, B><<<nblk, T, 0, s>>>(L);     \
        ASSS_CHECK_LAUNCH();                             \
        return ASSS_OK;                                  \
    }
    ASSS_BATCH_SHAPES(ASSS_BATCH_LAUNCH_CASE)
#undef ASSS_BATCH_LAUNCH_CASE
    set_error("batched solver: unsupported CTA shape %d x %d", nthreads, minb);
    return ASSS_ERR_ARG;
}

template <int KP, bool QB>
static asss_status occ_nt(int nthreads, int minb, int* occ) {
#define ASSS_BATCH_OCC_CASE(T, B)                                                           \
    if (nthreads == T && minb == B) {                                                       \
        ASSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_batch<KP, QB, T, B>, T, 0)); \
        return ASSS_OK;                                                                     \
    }
    ASSS_BATCH_SHAPES(ASSS_BATCH_OCC_CASE)
#undef ASSS_BATCH_OCC_CASE
    set_error("batched solver: unsupported CTA shape %d x %d", nthreads, minb);
    return ASSS_ERR_ARG;
}

// one translation unit instantiates the kernel for a few (padded width, Q storage)
// pairs, so the builds of the parts run in parallel; L == nullptr asks for the
// resident CTAs per SM (into occ) instead of a launch
asss_status batch_part0(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ);
asss_status batch_part1(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ);
asss_status batch_part2(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ);
asss_status batch_part3(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ);

}  // namespace asss
