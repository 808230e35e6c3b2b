// No-fill incomplete L D L^T of M^ = (A^ + A^T)/2 (paper §3 after Eq. absfac; the
// ~ildl(0) variant of §4.1: no more entries than M^ has, 1x1 pivots) and the
// triangular solves that apply L~^-1 = |D|^-1/2 (I + L)^-1 and L~^-T = (I + L)^-T |D|^-1/2.
//
// The factorization runs in a multicolour order: the vertices of the symmetric
// pattern P of A^ are coloured by Jones-Plassmann rounds (first-fit colours, splitmix64
// priorities), and the order is (colour, index).  Rows of one colour are never
// neighbours, so each colour is eliminated - and later solved for - in one parallel
// step: the factorization is one launch per colour, a triangular solve one launch (or,
// inside the persistent mrs kernel, one grid barrier) per colour.  Everything stays in
// the original indexing: "lower" means "of a smaller colour".
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asss {

// the colouring priorities draw on a splitmix64 stream of their own
constexpr unsigned long long COLOUR_SEED_XOR = 0xA5A5A5A5A5A5A5A5ull;

__device__ __forceinline__ unsigned long long splitmix_at(unsigned long long seed, int i) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One Jones-Plassmann round t: a vertex not yet coloured whose (priority, index) is
// above that of every neighbour still uncoloured at the start of the round takes the
// smallest colour no coloured neighbour holds.  rnd[i] = round in which i was
// coloured (INT_MAX: not yet); a neighbour coloured in this same round cannot exist
// for a winner (it would be a larger uncoloured neighbour), so rnd[j] >= t reads as
// "uncoloured" whichever value a concurrent write leaves.
__global__ void k_jp_round(int n, const int* __restrict__ rp, const int* __restrict__ ci, unsigned long long seed,
                           int t, int* rnd, int* colour, unsigned* left, int* overflow) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || rnd[i] < t) return;
    const unsigned long long pi = splitmix_at(seed, i);
    unsigned mask[ILDL_MAXCOL / 32];
#pragma unroll
    for (int w = 0; w < ILDL_MAXCOL / 32; ++w) mask[w] = 0u;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        if (j == i) continue;
        const int rj = rnd[j];
        if (rj >= t) {
            const unsigned long long pj = splitmix_at(seed, j);
            if (pj > pi || (pj == pi && j > i)) {
                atomicAdd(left, 1u);
                return;
            }
        } else {
            const int cj = colour[j];
            if (cj >= 0 && cj < ILDL_MAXCOL) mask[cj >> 5] |= 1u << (cj & 31);
        }
    }
    int c = -1;
#pragma unroll
    for (int w = 0; w < ILDL_MAXCOL / 32; ++w) {
        if (c < 0 && mask[w] != 0xffffffffu) c = 32 * w + __ffs(~mask[w]) - 1;
    }
    if (c < 0) {
        atomicExch(overflow, 1);
        c = ILDL_MAXCOL - 1;
    }
    colour[i] = c;
    rnd[i] = t;
}

__global__ void k_colour_hist(int n, const int* colour, int* hist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&hist[colour[i]], 1);
}

__global__ void k_flag_colour(int n, const int* colour, int c, int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = colour[i] == c ? 1 : 0;
}

// vertices of colour c in index order: lvl[ls_c + rank]
__global__ void k_place_colour(int n, const int* colour, int c, const int* pos, int ls_c, int* lvl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && colour[i] == c) lvl[ls_c + pos[i]] = i;
}

// entries of row i with a column of smaller colour (L) and of larger colour (U)
__global__ void k_split_count(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int* colour,
                              int* lcnt, int* ucnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = colour[i];
    int nl = 0, nu = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        if (j == i) continue;
        if (colour[j] < c) ++nl;
        else ++nu;
    }
    lcnt[i] = nl;
    ucnt[i] = nu;
}

// L entries get m_ij = (C_ij + C_ji)/2 (C = A^ on P, mirror[e] = position of (j, i))
// and their position lpos[e]; U entries keep the position of their mirror, whose L
// value they take once the factor is known.  Order within a row: P's (column index).
__global__ void k_split_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int* colour,
                             const int* __restrict__ mirror, const double* __restrict__ Cval, const int* lrp,
                             const int* urp, int* lci, double* lv, int* lpos, int* uci, int* umir) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = colour[i];
    int ql = lrp[i], qu = urp[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        if (j == i) continue;
        if (colour[j] < c) {
            lci[ql] = j;
            lv[ql] = 0.5 * (Cval[e] + Cval[mirror[e]]);
            lpos[e] = ql;
            ++ql;
        } else {
            uci[qu] = j;
            umir[qu] = mirror[e];
            ++qu;
        }
    }
}

__device__ __forceinline__ int find_sorted(const int* a, int lo, int hi, int key) {
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        const int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// Rows of one colour c, one thread each (their L entries point at smaller colours
// only, all final).  Row i's entries are taken colour by colour, so l_ik of every
// k below the current column's colour is final when it is needed:
//   l_ij = (m_ij - sum_{k in L(i) and L(j)} l_ik d_k l_jk) / d_j,  d_i = m_ii - sum l_ik^2 d_k.
__global__ void k_ildl_level(const int* __restrict__ lvl, int cnt, int c, const int* __restrict__ colour,
                             const int* __restrict__ lrp, const int* __restrict__ lci, double* lv, double* d,
                             double thr, int* nzero) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = lvl[t];
    const int a = lrp[i], b = lrp[i + 1];
    for (int cc = 0; cc < c; ++cc) {
        for (int q = a; q < b; ++q) {
            const int j = lci[q];
            if (colour[j] != cc) continue;
            double s = lv[q];
            for (int q2 = lrp[j]; q2 < lrp[j + 1]; ++q2) {
                const int k = lci[q2];
                const int pos = find_sorted(lci, a, b, k);
                if (pos >= 0) s -= lv[pos] * d[k] * lv[q2];
            }
            lv[q] = s / d[j];
        }
    }
    double di = d[i];
    for (int q = a; q < b; ++q) {
        const double l = lv[q];
        di -= l * l * d[lci[q]];
    }
    if (di == 0.0 || fabs(di) < thr) atomicAdd(nzero, 1);
    d[i] = di;
}

__global__ void k_fill_u(int nu, const int* umir, const int* lpos, const double* lv, double* uv) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nu) uv[q] = lv[lpos[umir[q]]];
}

__global__ void k_inv_sqrt_abs(int n, const double* d, double* wd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wd[i] = 1.0 / sqrt(fabs(d[i]));
}

__global__ void k_d2f_n(const double* a, long long n, float* b) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// one colour of a triangular solve: out_i = in_i - sum_q v_q out[col_q] over the
// entries that point at colours solved before (L: smaller, U: larger)
__global__ void k_tri_level(const int* __restrict__ lvl, int cnt, const int* __restrict__ rp,
                            const int* __restrict__ ci, const double* __restrict__ v, const double* in, double* out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = lvl[t];
    const int q1 = rp[i + 1];
    double s = 0.0;
    for (int q = rp[i]; q < q1; q += 8) {  // the batch's loads first, then its gathers
        int cc[8];
        double vv[8], g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool inb = q + u < q1;
            cc[u] = inb ? ci[q + u] : 0;
            vv[u] = inb ? v[q + u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) g[u] = (q + u < q1) ? out[cc[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += vv[u] * g[u];
    }
    out[i] = in[i] - s;
}

__global__ void k_absmax_bits(const double* a, int n, unsigned long long* out) {
    unsigned long long m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long b = (unsigned long long)__double_as_longlong(fabs(a[i]));
        m = b > m ? b : m;
    }
    atomicMax(out, m);
}

__global__ void k_mul3(int n, const double* a, const double* b, double* y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] * b[i];
}

asss_status ildl_build(const Ctx& c, const DCsr& P, const int* mirror, const double* Cval, double* d,
                       uint64_t seed, double zero_tol, bool fp32, IldlFactor& F, int* nzero) {
    NvtxRange nv_("asss:ildl");
    cudaStream_t s = c.stream;
    const int n = P.n;
    F.n = n;
    *nzero = 0;
    // Jones-Plassmann colouring
    DBuf<int> rnd;
    DBuf<unsigned> left;
    DBuf<int> ovf;
    ASSS_TRY(rnd.alloc(n > 0 ? n : 1));
    ASSS_TRY(F.colour.alloc(n > 0 ? n : 1));
    ASSS_TRY(left.alloc(1));
    ASSS_TRY(ovf.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(rnd.p, 0x7f, sizeof(int) * (size_t)(n > 0 ? n : 1), s));  // 0x7f7f7f7f: not yet
    ASSS_CUDA(cudaMemsetAsync(F.colour.p, 0xff, sizeof(int) * (size_t)(n > 0 ? n : 1), s));
    ASSS_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), s));
    const unsigned long long cseed = (unsigned long long)seed ^ COLOUR_SEED_XOR;
    int t = 0;
    for (;; ++t) {
        if (t > n + 1) {
            set_error("colouring did not finish");
            return ASSS_ERR_BREAKDOWN;
        }
        ASSS_CUDA(cudaMemsetAsync(left.p, 0, sizeof(unsigned), s));
        k_jp_round<<<cdiv(n, 256), 256, 0, s>>>(n, P.rp.p, P.ci.p, cseed, t, rnd.p, F.colour.p, left.p, ovf.p);
        ASSS_CHECK_LAUNCH();
        unsigned hl = 0;
        ASSS_CUDA(cudaMemcpyAsync(&hl, left.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        if (hl == 0) break;
    }
    F.rounds = t + 1;
    int hovf = 0;
    ASSS_CUDA(cudaMemcpyAsync(&hovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    // levels: vertices sorted by (colour, index)
    DBuf<int> hist;
    ASSS_TRY(hist.alloc(ILDL_MAXCOL));
    ASSS_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int) * ILDL_MAXCOL, s));
    k_colour_hist<<<cdiv(n, 256), 256, 0, s>>>(n, F.colour.p, hist.p);
    ASSS_CHECK_LAUNCH();
    std::vector<int> hh(ILDL_MAXCOL);
    ASSS_CUDA(cudaMemcpyAsync(hh.data(), hist.p, sizeof(int) * ILDL_MAXCOL, cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hovf) {
        set_error("the pattern needs more than %d colours", ILDL_MAXCOL);
        return ASSS_ERR_UNSUPPORTED;
    }
    F.ncol = 0;
    for (int k = 0; k < ILDL_MAXCOL; ++k)
        if (hh[k]) F.ncol = k + 1;
    F.hls.assign(F.ncol + 1, 0);
    for (int k = 0; k < F.ncol; ++k) F.hls[k + 1] = F.hls[k] + hh[k];
    ASSS_TRY(to_device(F.ls, F.hls.data(), (int64_t)F.ncol + 1, s));
    ASSS_TRY(F.lvl.alloc(n > 0 ? n : 1));
    {
        DBuf<int> flag, pos;
        ASSS_TRY(flag.alloc(n > 0 ? n : 1));
        ASSS_TRY(pos.alloc(n + 1));
        for (int k = 0; k < F.ncol; ++k) {
            k_flag_colour<<<cdiv(n, 256), 256, 0, s>>>(n, F.colour.p, k, flag.p);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(exclusive_scan(flag.p, pos.p, n, nullptr, s));
            k_place_colour<<<cdiv(n, 256), 256, 0, s>>>(n, F.colour.p, k, pos.p, F.hls[k], F.lvl.p);
            ASSS_CHECK_LAUNCH();
        }
    }
    // L (smaller colours) and U (larger colours) halves of P
    DBuf<int> lcnt, ucnt, lpos, umir;
    ASSS_TRY(lcnt.alloc(n > 0 ? n : 1));
    ASSS_TRY(ucnt.alloc(n > 0 ? n : 1));
    k_split_count<<<cdiv(n, 256), 256, 0, s>>>(n, P.rp.p, P.ci.p, F.colour.p, lcnt.p, ucnt.p);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(F.lrp.alloc(n + 1));
    ASSS_TRY(F.urp.alloc(n + 1));
    int64_t nl = 0, nu = 0;
    ASSS_TRY(exclusive_scan(lcnt.p, F.lrp.p, n, &nl, s));
    ASSS_TRY(exclusive_scan(ucnt.p, F.urp.p, n, &nu, s));
    F.nl = nl;
    F.nu = nu;
    ASSS_TRY(F.lci.alloc(nl > 0 ? nl : 1));
    ASSS_TRY(F.lv.alloc(nl > 0 ? nl : 1));
    ASSS_TRY(F.uci.alloc(nu > 0 ? nu : 1));
    ASSS_TRY(F.uv.alloc(nu > 0 ? nu : 1));
    ASSS_TRY(lpos.alloc(P.nnz > 0 ? P.nnz : 1));
    ASSS_TRY(umir.alloc(nu > 0 ? nu : 1));
    k_split_fill<<<cdiv(n, 256), 256, 0, s>>>(n, P.rp.p, P.ci.p, F.colour.p, mirror, Cval, F.lrp.p, F.urp.p, F.lci.p,
                                              F.lv.p, lpos.p, F.uci.p, umir.p);
    ASSS_CHECK_LAUNCH();
    // the factor, colour by colour; d holds diag(M^) = diag(A^) on entry, the pivots after
    double dmax = 0.0;
    {
        DBuf<unsigned long long> mx;
        ASSS_TRY(mx.alloc(1));
        ASSS_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
        k_absmax_bits<<<256, 256, 0, s>>>(d, n, mx.p);
        ASSS_CHECK_LAUNCH();
        unsigned long long bits = 0;
        ASSS_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        memcpy(&dmax, &bits, sizeof(double));
    }
    DBuf<int> nz;
    ASSS_TRY(nz.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(nz.p, 0, sizeof(int), s));
    for (int k = 0; k < F.ncol; ++k) {
        const int cnt = F.hls[k + 1] - F.hls[k];
        if (cnt == 0) continue;
        k_ildl_level<<<cdiv(cnt, 128), 128, 0, s>>>(F.lvl.p + F.hls[k], cnt, k, F.colour.p, F.lrp.p, F.lci.p, F.lv.p,
                                                     d, zero_tol * dmax, nz.p);
        ASSS_CHECK_LAUNCH();
    }
    ASSS_CUDA(cudaMemcpyAsync(nzero, nz.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    k_fill_u<<<cdiv((int)(nu > 0 ? nu : 1), 256), 256, 0, s>>>((int)nu, umir.p, lpos.p, F.lv.p, F.uv.p);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(F.wd.alloc(n > 0 ? n : 1));
    k_inv_sqrt_abs<<<cdiv(n, 256), 256, 0, s>>>(n, d, F.wd.p);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(F.ft.alloc(n > 0 ? n : 1));
    ASSS_TRY(F.fw.alloc(n > 0 ? n : 1));
    if (fp32) {
        ASSS_TRY(F.lv32.alloc(nl > 0 ? nl : 1));
        ASSS_TRY(F.uv32.alloc(nu > 0 ? nu : 1));
        ASSS_TRY(F.wd32.alloc(n > 0 ? n : 1));
        ASSS_TRY(F.ft32.alloc(n > 0 ? n : 1));
        ASSS_TRY(F.fw32.alloc(n > 0 ? n : 1));
        if (nl) k_d2f_n<<<cdiv(nl, 256), 256, 0, s>>>(F.lv.p, nl, F.lv32.p);
        if (nu) k_d2f_n<<<cdiv(nu, 256), 256, 0, s>>>(F.uv.p, nu, F.uv32.p);
        k_d2f_n<<<cdiv(n, 256), 256, 0, s>>>(F.wd.p, n, F.wd32.p);
        ASSS_CHECK_LAUNCH();
    }
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

asss_status ildl_set_skew(const Ctx& c, IldlFactor& F, const DCsr& Jh, bool fp32) {
    F.jrp = Jh.rp.p;
    F.jci = Jh.ci.p;
    F.jv = Jh.v.p;
    F.nj = Jh.nnz;
    if (fp32) {
        ASSS_TRY(F.jv32.alloc(Jh.nnz > 0 ? Jh.nnz : 1));
        if (Jh.nnz) k_d2f_n<<<cdiv(Jh.nnz, 256), 256, 0, c.stream>>>(Jh.v.p, Jh.nnz, F.jv32.p);
        ASSS_CHECK_LAUNCH();
    }
    return ASSS_OK;
}

// out = |D|^-1/2 (I + L)^-1 v   (out != v)
asss_status ildl_F(const Ctx& c, IldlFactor& F, const double* v, double* out) {
    cudaStream_t s = c.stream;
    for (int k = 0; k < F.ncol; ++k) {
        const int cnt = F.hls[k + 1] - F.hls[k];
        if (cnt == 0) continue;
        k_tri_level<<<cdiv(cnt, 256), 256, 0, s>>>(F.lvl.p + F.hls[k], cnt, F.lrp.p, F.lci.p, F.lv.p, v, F.ft.p);
        ASSS_CHECK_LAUNCH();
    }
    k_mul3<<<cdiv(F.n, 256), 256, 0, s>>>(F.n, F.wd.p, F.ft.p, out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// out = (I + L)^-T |D|^-1/2 v   (out != v)
asss_status ildl_G(const Ctx& c, IldlFactor& F, const double* v, double* out) {
    cudaStream_t s = c.stream;
    k_mul3<<<cdiv(F.n, 256), 256, 0, s>>>(F.n, F.wd.p, v, F.ft.p);
    ASSS_CHECK_LAUNCH();
    for (int k = F.ncol - 1; k >= 0; --k) {
        const int cnt = F.hls[k + 1] - F.hls[k];
        if (cnt == 0) continue;
        k_tri_level<<<cdiv(cnt, 256), 256, 0, s>>>(F.lvl.p + F.hls[k], cnt, F.urp.p, F.uci.p, F.uv.p, F.ft.p, out);
        ASSS_CHECK_LAUNCH();
    }
    return ASSS_OK;
}

}  // namespace asss
