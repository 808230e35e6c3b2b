// One Arnoldi step of the outer flexible GMRES (§4.1 outer method, reading of
// the FGMRES cycle): given w = A_cal z_j, two classical Gram-Schmidt passes
// against v_0..v_j, the norm of what is left, the Givens update of the Hessenberg
// column and of the residual vector g, and v_{j+1} = w / ||w||, all in one
// cooperative launch with two grid barriers (the passes over V are the only HBM
// traffic; the dot products of a pass are reduced deterministically, every block
// adding the block partials in the same order).  The norm after the second pass
// comes from the one before it: with w1 = w - V h1 and h2 = V^T w1,
// ||w1 - V h2||^2 = ||w1||^2 - ||h2||^2 up to the (re-orthogonalised) departure of V
// from orthonormality, so the second correction and the new basis vector share one
// sweep.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace asss {

constexpr int AO_THREADS = 512;
constexpr int AO_WARPS = AO_THREADS / 32;
constexpr int AO_CH = 8;  // dot products accumulated per sweep

struct AoParams {
    const double* V;  // n x (m+1), column-major (ld n); v_0..v_j are read, v_{j+1} written
    double* w;
    int n, nv;        // nv = j + 1
    int j, m;
    double* H;        // (m+1) x m column-major Hessenberg, already rotated
    double* cs;
    double* sn;
    double* g;
    double* hv;       // first-pass coefficients (nv)
    double* hv2;      // second-pass coefficients (nv)
    double* hn2;      // ||w||^2 after both passes
    double* inv_hn;   // 1 / ||w|| (0 when w = 0)
    double* part;     // 2 x [AO_MAXV][nblk] block partials (consecutive passes alternate halves)
    double thr;       // the cycle stops when |g[j+1]| <= thr
    int* stop;
    GridBarrier gb;
    unsigned phase0;  // barriers completed on gb.count before this launch
    long long budget;
};

// Givens update of column j (same arithmetic as the one-step kernel it replaces)
__device__ void ao_fg_column(const AoParams& p, const double* h1, const double* h2, double hn2) {
    const int j = p.j, m = p.m;
    double* col = p.H + (size_t)j * (m + 1);
    for (int a = 0; a <= j; ++a) col[a] = h1[a] + h2[a];
    const double hn = sqrt(hn2);
    col[j + 1] = hn;
    for (int a = 0; a < j; ++a) {
        const double t = p.cs[a] * col[a] + p.sn[a] * col[a + 1];
        col[a + 1] = -p.sn[a] * col[a] + p.cs[a] * col[a + 1];
        col[a] = t;
    }
    const double rr = hypot(col[j], col[j + 1]);
    const double c = (rr != 0.0) ? col[j] / rr : 1.0;
    const double s = (rr != 0.0) ? col[j + 1] / rr : 0.0;
    p.cs[j] = c;
    p.sn[j] = s;
    col[j] = rr;
    col[j + 1] = 0.0;
    p.g[j + 1] = -s * p.g[j];
    p.g[j] = c * p.g[j];
    *p.hn2 = hn2;
    *p.inv_hn = (hn > 0.0) ? 1.0 / hn : 0.0;
    *p.stop = (hn2 == 0.0 || fabs(p.g[j + 1]) <= p.thr) ? 1 : 0;
}

// one 512-thread block per SM: the kernel is bound by GB300's FP64 pipe, and every
// block spends FP64 adds on its partial sums, so fewer, fuller blocks leave more of the
// pipe to the rows (and 128 registers a thread, no spills)
__global__ void __launch_bounds__(AO_THREADS, 1) k_arnoldi_orth(AoParams p) {
    __shared__ double s_w[AO_WARPS][AO_CH];
    __shared__ double s_h1[AO_MAXV];
    __shared__ double s_h2[AO_MAXV];
    __shared__ double s_n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nblk = gridDim.x;
    const long long n = p.n;
    const long long r0 = n * blockIdx.x / nblk, r1 = n * (blockIdx.x + 1) / nblk;
    const int nv = p.nv;
    const double* __restrict__ V = p.V;  // v_0..v_j (read) and v_{j+1} (written) do not overlap w
    double* __restrict__ w = p.w;
    volatile int* err = p.gb.err;
    // a block may still be adding the previous pass's partials while a faster one
    // writes the next pass's, so consecutive passes use the two halves of p.part
    double* part = p.part;

    // block partials of the first cnt accumulators (vectors c0..) into part
    auto put_partials = [&](auto& acc, int c0, int cnt) {
        constexpr int NA = sizeof(acc) / sizeof(double);
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            const double v = warp_sum(acc[t]);
            if (lane == 0) s_w[warp][t] = v;
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt && c0 + (int)threadIdx.x < nv) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < AO_WARPS; ++q) s += s_w[q][threadIdx.x];
            part[(size_t)(c0 + threadIdx.x) * nblk + blockIdx.x] = s;
        }
        __syncthreads();
    };
    // block partials of NVC dot products (slots 0..NVC-1) and one squared norm (last
    // accumulator, slot AO_MAXV - 1)
    auto put_partials_n = [&](auto& acc, int nvc) {
        constexpr int NA = sizeof(acc) / sizeof(double);
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            const double v = warp_sum(acc[t]);
            if (lane == 0) s_w[warp][t] = v;
        }
        __syncthreads();
        if ((int)threadIdx.x <= nvc) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < AO_WARPS; ++q) s += s_w[q][threadIdx.x];
            const int slot = (int)threadIdx.x < nvc ? (int)threadIdx.x : AO_MAXV - 1;
            part[(size_t)slot * nblk + blockIdx.x] = s;
        }
        __syncthreads();
    };
    // dots V_a^T w over this block's rows for a in [c0, c0 + CNT): the count is a
    // template argument, so no FP64 instruction is issued for a vector that is not
    // there (the FP64 pipe is what bounds this kernel on GB300)
    auto dots_n = [&](auto cnt, int c0) {
        constexpr int CNT = decltype(cnt)::value;
        double acc[CNT];
#pragma unroll
        for (int t = 0; t < CNT; ++t) acc[t] = 0.0;
        for (long long i = r0 + threadIdx.x; i < r1; i += AO_THREADS) {
            const double wi = w[i];
#pragma unroll
            for (int t = 0; t < CNT; ++t) acc[t] += V[(size_t)(c0 + t) * n + i] * wi;
        }
        put_partials(acc, c0, CNT);
    };
    // all nv dots, AO_CH vectors per sweep
    auto dots = [&]() {
        for (int c0 = 0; c0 < nv; c0 += AO_CH) {
            switch (nv - c0 < AO_CH ? nv - c0 : AO_CH) {
                case 1: dots_n(std::integral_constant<int, 1>{}, c0); break;
                case 2: dots_n(std::integral_constant<int, 2>{}, c0); break;
                case 3: dots_n(std::integral_constant<int, 3>{}, c0); break;
                case 4: dots_n(std::integral_constant<int, 4>{}, c0); break;
                case 5: dots_n(std::integral_constant<int, 5>{}, c0); break;
                case 6: dots_n(std::integral_constant<int, 6>{}, c0); break;
                case 7: dots_n(std::integral_constant<int, 7>{}, c0); break;
                default: dots_n(std::integral_constant<int, AO_CH>{}, c0); break;
            }
        }
    };
    // every block adds the nblk partials of each vector in block order
    auto reduce = [&](int cnt, double* out) {
        for (int a = warp; a < cnt; a += AO_WARPS) {
            double t = 0.0;
            for (int b = lane; b < nblk; b += 32) t += __ldcg(&part[(size_t)a * nblk + b]);
            t = warp_sum(t);
            if (lane == 0) out[a] = t;
        }
        __syncthreads();
    };

    // ---- pass 1: h1 = V^T w ----
    dots();
    grid_sync_phase(p.gb, nblk, p.phase0 + 0, p.budget);
    if (*err) return;
    reduce(nv, s_h1);
    if (blockIdx.x == 0)
        for (int a = threadIdx.x; a < nv; a += AO_THREADS) p.hv[a] = s_h1[a];

    // ---- pass 2: w -= V h1, then h2 = V^T w (one sweep when all of V fits the accumulators;
    // the vector count is a template argument there, so no FP64 operation is spent on padding) ----
    part = p.part + (size_t)AO_MAXV * nblk;
    // the dot products h2 (slots 0..nv-1) and ||w1||^2 (slot AO_MAXV - 1 of the
    // partials, never a vector slot: nv <= AO_MAXV - 1)
    auto fused2 = [&](auto nvc) {
        constexpr int NVC = decltype(nvc)::value;
        double acc[NVC + 1];
#pragma unroll
        for (int t = 0; t <= NVC; ++t) acc[t] = 0.0;
        for (long long i = r0 + threadIdx.x; i < r1; i += AO_THREADS) {
            double vi[NVC];
            double s = 0.0;
#pragma unroll
            for (int t = 0; t < NVC; ++t) {
                vi[t] = V[(size_t)t * n + i];
                s += vi[t] * s_h1[t];
            }
            const double wi = w[i] - s;
            w[i] = wi;
#pragma unroll
            for (int t = 0; t < NVC; ++t) acc[t] += vi[t] * wi;
            acc[NVC] += wi * wi;
        }
        put_partials_n(acc, NVC);
    };
    if (nv <= 6) {
        switch (nv) {
            case 1: fused2(std::integral_constant<int, 1>{}); break;
            case 2: fused2(std::integral_constant<int, 2>{}); break;
            case 3: fused2(std::integral_constant<int, 3>{}); break;
            case 4: fused2(std::integral_constant<int, 4>{}); break;
            case 5: fused2(std::integral_constant<int, 5>{}); break;
            default: fused2(std::integral_constant<int, 6>{}); break;
        }
    } else {
        double accn[1] = {0.0};
        for (long long i = r0 + threadIdx.x; i < r1; i += AO_THREADS) {
            double s = 0.0;
            for (int a = 0; a < nv; ++a) s += V[(size_t)a * n + i] * s_h1[a];
            const double wi = w[i] - s;
            w[i] = wi;
            accn[0] += wi * wi;
        }
        put_partials_n(accn, 0);
        dots();
    }
    grid_sync_phase(p.gb, nblk, p.phase0 + 1, p.budget);
    if (*err) return;
    reduce(nv, s_h2);
    {
        // ||w1||^2 from its slot
        double t = 0.0;
        if (warp == 0) {
            for (int b = lane; b < nblk; b += 32) t += __ldcg(&part[(size_t)(AO_MAXV - 1) * nblk + b]);
            t = warp_sum(t);
            if (lane == 0) s_n = t;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0)
        for (int a = threadIdx.x; a < nv; a += AO_THREADS) p.hv2[a] = s_h2[a];

    // ---- pass 3: hn2 = ||w1||^2 - ||h2||^2; w2 = w1 - V h2 and v_{j+1} = w2 / ||w2|| in one sweep ----
    double h2n = 0.0;
    for (int a = 0; a < nv; ++a) h2n += s_h2[a] * s_h2[a];
    const double hn2 = fmax(s_n - h2n, 0.0);
    if (blockIdx.x == 0 && threadIdx.x == 0) ao_fg_column(p, s_h1, s_h2, hn2);
    const double hn = sqrt(hn2);
    const double inv = (hn > 0.0) ? 1.0 / hn : 0.0;
    double* vn = const_cast<double*>(V) + (size_t)nv * n;
    // the vector count as a template argument where it is small (the loads of a row are
    // then issued together and no FP64 operation is spent on a loop counter)
    auto pass3 = [&](auto nvc) {
        constexpr int NVC = decltype(nvc)::value;
        for (long long i = r0 + threadIdx.x; i < r1; i += AO_THREADS) {
            double vi[NVC];
#pragma unroll
            for (int t = 0; t < NVC; ++t) vi[t] = V[(size_t)t * n + i];
            double s = 0.0;
#pragma unroll
            for (int t = 0; t < NVC; ++t) s += vi[t] * s_h2[t];
            const double wi = w[i] - s;
            w[i] = wi;
            vn[i] = wi * inv;
        }
    };
    switch (nv) {
        case 1: pass3(std::integral_constant<int, 1>{}); break;
        case 2: pass3(std::integral_constant<int, 2>{}); break;
        case 3: pass3(std::integral_constant<int, 3>{}); break;
        case 4: pass3(std::integral_constant<int, 4>{}); break;
        case 5: pass3(std::integral_constant<int, 5>{}); break;
        case 6: pass3(std::integral_constant<int, 6>{}); break;
        default:
            for (long long i = r0 + threadIdx.x; i < r1; i += AO_THREADS) {
                double s = 0.0;
                for (int a = 0; a < nv; ++a) s += V[(size_t)a * n + i] * s_h2[a];
                const double wi = w[i] - s;
                w[i] = wi;
                vn[i] = wi * inv;
            }
            break;
    }
}

asss_status arnoldi_orth(const Ctx& c, ArnoldiWork& aw, const double* V, double* w, int n, int j, int m, double* H,
                         double* cs, double* sn, double* g, double* hv, double* hv2, double* hn2, double* inv_hn,
                         double thr, int* stop) {
    if (j + 1 > AO_MAXV - 1) {   // one partial slot is kept for the norm
        set_error("Arnoldi step %d exceeds the fused kernel's %d vectors", j, AO_MAXV - 1);
        return ASSS_ERR_UNSUPPORTED;
    }
    if (aw.n != n || !aw.part.p) {
        int occ = 0;
        ASSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi_orth, AO_THREADS, 0));
        if (occ < 1) {
            set_error("Arnoldi kernel cannot be resident");
            return ASSS_ERR_CUDA;
        }
        if (occ > 1) occ = 1;
        int nblk = c.sms * occ;
        int need = cdiv(n, 64);
        if (need < 1) need = 1;
        if (nblk > need) nblk = need;
        ASSS_TRY(aw.part.alloc((int64_t)2 * AO_MAXV * nblk));
        if (!aw.bar.p) ASSS_TRY(aw.bar.alloc(2));
        if (!aw.err.p) ASSS_TRY(aw.err.alloc(1));
        ASSS_CUDA(cudaMemsetAsync(aw.bar.p, 0, 2 * sizeof(unsigned), c.stream));
        ASSS_CUDA(cudaMemsetAsync(aw.err.p, 0, sizeof(int), c.stream));
        aw.nblk = nblk;
        aw.n = n;
        aw.phase = 0;
    }
    AoParams p;
    p.V = V;
    p.w = w;
    p.n = n;
    p.nv = j + 1;
    p.j = j;
    p.m = m;
    p.H = H;
    p.cs = cs;
    p.sn = sn;
    p.g = g;
    p.hv = hv;
    p.hv2 = hv2;
    p.hn2 = hn2;
    p.inv_hn = inv_hn;
    p.part = aw.part.p;
    p.thr = thr;
    p.stop = stop;
    p.gb.count = aw.bar.p;
    p.gb.gen = aw.bar.p + 1;
    p.gb.err = aw.err.p;
    p.phase0 = aw.phase;
    p.budget = c.wait_cycles;
    void* args[] = {&p};
    ASSS_CUDA(cudaLaunchCooperativeKernel((const void*)k_arnoldi_orth, dim3(aw.nblk), dim3(AO_THREADS), args, 0,
                                          c.stream));
    count_launch();
    aw.phase += 2;
    return ASSS_OK;
}

}  // namespace asss
