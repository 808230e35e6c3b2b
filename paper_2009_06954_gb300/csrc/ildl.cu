// No-fill incomplete L D L^T of M^ = (A^ + A^T)/2 (paper §3 after Eq. absfac; the
// ~ildl(0) variant of §4.1: no more entries than M^ has; 1x1 pivots, or also 2x2 pivot
// blocks chosen by the first Bunch-Kaufman test before the ordering) and the
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
// With 2x2 pivots (part != null) a pair is one vertex of the quotient graph: its leader
// (the smaller index) takes part in the round with its own priority, scans the rows of
// both members, compares with the neighbours' leaders, and colours both members.
__global__ void k_jp_round(int n, const int* __restrict__ rp, const int* __restrict__ ci, unsigned long long seed,
                           int t, int* rnd, int* colour, unsigned* left, int* overflow, const int* part) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int mate = part ? part[i] : -1;
    if ((mate >= 0 && mate < i) || rnd[i] < t) return;
    const unsigned long long pi = splitmix_at(seed, i);
    unsigned mask[ILDL_MAXCOL / 32];
#pragma unroll
    for (int w = 0; w < ILDL_MAXCOL / 32; ++w) mask[w] = 0u;
    for (int sr = 0; sr < (mate >= 0 ? 2 : 1); ++sr) {
        const int row = sr ? mate : i;
        for (int e = rp[row]; e < rp[row + 1]; ++e) {
            const int j0 = ci[e];
            if (j0 == i || j0 == mate) continue;
            int j = j0;
            if (part) {
                const int pj = part[j0];
                if (pj >= 0 && pj < j0) j = pj;
            }
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
    if (mate >= 0) {
        colour[mate] = c;
        rnd[mate] = t;
    }
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
        else if (colour[j] > c) ++nu;   // same colour: the partner of a 2x2 pivot (in D)
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
        } else if (colour[j] > c) {
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

// ---------------------------------------------------------------------------
// 2x2 pivot blocks: a static choice by the first Bunch-Kaufman test, the block closure
// of the pattern, the block factor, |D|^-1/2 and U_r block by block
// ---------------------------------------------------------------------------
// gamma_i = max_{j != i} |m_ij| over row i of P (m = (C + C^T)/2), rbest = its column (the
// smallest on ties: columns are sorted); i asks for a pair when |m_ii| < alpha gamma_i
__global__ void k_bk_pick(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ mirror,
                          const double* __restrict__ Cval, const double* __restrict__ d, double alpha, int* rbest,
                          int* need) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double g = -1.0;
    int r = -1;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        if (j == i) continue;
        const double v = fabs(0.5 * (Cval[e] + Cval[mirror[e]]));
        if (v > g) {
            g = v;
            r = j;
        }
    }
    rbest[i] = r;
    need[i] = (r >= 0 && fabs(d[i]) < alpha * g) ? 1 : 0;
}

// i and rbest[i] pair when both ask and each is the other's choice
__global__ void k_bk_pair(int n, const int* rbest, const int* need, int* part, int* npair) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = rbest[i];
    const int m = (need[i] && r >= 0 && need[r] && rbest[r] == i) ? r : -1;
    part[i] = m;
    if (m >= 0) atomicAdd(npair, 1);
}

__device__ __forceinline__ bool in_sorted(const int* a, int lo, int hi, int key) {
    return find_sorted(a, lo, hi, key) >= 0;
}

// Block closure of the symmetric pattern P: row i of Pb holds, for every column c of the
// rows of i and of its partner, c and partner(c).  Row i = merge of the two sorted rows,
// then the partners not yet there (distinct: the pairing is a matching), then one
// insertion sort of the appended ones.  out == nullptr: only counts (into cnt).
__global__ void k_bpat_row(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ part,
                           const int* orp, int* cnt, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int mi = part[i];
    const int a0 = rp[i], a1 = rp[i + 1];
    const int b0 = mi >= 0 ? rp[mi] : 0, b1 = mi >= 0 ? rp[mi + 1] : 0;
    int* o = out ? out + orp[i] : nullptr;
    int merged = 0, extra = 0;
    int x = a0, y = b0;
    while (x < a1 || y < b1) {
        int v;
        if (y >= b1 || (x < a1 && ci[x] < ci[y])) v = ci[x++];
        else if (x >= a1 || ci[y] < ci[x]) v = ci[y++];
        else {
            v = ci[x];
            ++x;
            ++y;
        }
        if (o) o[merged] = v;
        ++merged;
        const int pc = part[v];
        if (pc >= 0 && !in_sorted(ci, a0, a1, pc) && !(mi >= 0 && in_sorted(ci, b0, b1, pc))) ++extra;
    }
    if (!o) {
        cnt[i] = merged + extra;
        return;
    }
    int k = merged;
    for (int q = 0; q < merged; ++q) {
        const int pc = part[o[q]];
        if (pc >= 0 && !in_sorted(ci, a0, a1, pc) && !(mi >= 0 && in_sorted(ci, b0, b1, pc))) o[k++] = pc;
    }
    for (int q = merged; q < k; ++q) {   // insertion sort of the appended partners
        const int v = o[q];
        int w = q - 1;
        while (w >= 0 && o[w] > v) {
            o[w + 1] = o[w];
            --w;
        }
        o[w + 1] = v;
    }
}

// values of C on the closure (0 at the added positions) and the mirror positions there
// (the closure of a symmetric pattern is symmetric; a missing mirror is counted in bad
// and replaced by the entry itself, so no later read leaves the arrays)
__global__ void k_bpat_values(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ Cval, const int* __restrict__ brp,
                              const int* __restrict__ bci, double* bval, int* bmir, int* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = brp[i]; e < brp[i + 1]; ++e) {
        const int j = bci[e];
        const int q = find_sorted(ci, rp[i], rp[i + 1], j);
        bval[e] = q >= 0 ? Cval[q] : 0.0;
        const int m = find_sorted(bci, brp[j], brp[j + 1], i);
        if (m < 0) atomicAdd(bad, 1);
        bmir[e] = m >= 0 ? m : e;
    }
}

// D_{i,partner(i)} on entry: (C_ij + C_ji)/2 at the pair's position
__global__ void k_pair_offdiag(int n, const int* __restrict__ part, const int* __restrict__ brp,
                               const int* __restrict__ bci, const double* __restrict__ bval,
                               const int* __restrict__ bmir, double* doff) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int m = part[i];
    double v = 0.0;
    if (m >= 0) {
        const int q = find_sorted(bci, brp[i], brp[i + 1], m);
        if (q >= 0) v = 0.5 * (bval[q] + bval[bmir[q]]);
    }
    doff[i] = v;
}

// (L_r D)_a = l_ra d_a + l_{r,partner(a)} D_{a,partner(a)} over row r = lci[ra, rb)
__device__ __forceinline__ double lrow_d(const int* lci, const double* lv, int ra, int rb, int a, const int* part,
                                         const double* d, const double* doff) {
    const int q = find_sorted(lci, ra, rb, a);
    if (q < 0) return 0.0;
    double v = lv[q] * d[a];
    const int pa = part[a];
    if (pa >= 0) {
        const int q2 = find_sorted(lci, ra, rb, pa);
        if (q2 >= 0) v += lv[q2] * doff[a];
    }
    return v;
}

// Pivot blocks of colour c, one thread per block (its leader; the partner's row has the
// same lower columns by the closure).  For each lower block K = {k, partner(k)} of row i,
// colour by colour:  S_rk = m_rk - sum_{a in L(k)} (L_r D)_a l_ka  for the rows r of the
// block and the columns of K, then L_{.,K} = S D_K^-1;  finally D_I = M_II - L_I D L_I^T.
__global__ void k_ildl_level_bk(const int* __restrict__ lvl, int cnt, int c, const int* __restrict__ colour,
                                const int* __restrict__ part, const int* __restrict__ lrp, const int* __restrict__ lci,
                                double* lv, double* d, double* doff, double thr, double dmax, int* nzero, int* bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = lvl[t];
    const int mi = part[i];
    if (mi >= 0 && mi < i) return;
    const int nr = mi >= 0 ? 2 : 1;
    int ra[2] = {lrp[i], mi >= 0 ? lrp[mi] : 0};
    int rb[2] = {lrp[i + 1], mi >= 0 ? lrp[mi + 1] : 0};
    if (nr == 2 && rb[1] - ra[1] != rb[0] - ra[0]) {
        atomicAdd(bad, 1);
        return;
    }
    for (int cc = 0; cc < c; ++cc) {
        for (int q = ra[0]; q < rb[0]; ++q) {
            const int k = lci[q];
            if (colour[k] != cc) continue;
            const int pk = part[k];
            if (pk >= 0 && pk < k) continue;   // taken with its leader
            const int ncol = pk >= 0 ? 2 : 1;
            const int kc[2] = {k, pk};
            double S[2][2];
            int pos[2][2];
            for (int r = 0; r < nr; ++r) {
                for (int cix = 0; cix < ncol; ++cix) {
                    const int col = kc[cix];
                    const int p0 = find_sorted(lci, ra[r], rb[r], col);
                    pos[r][cix] = p0;
                    if (p0 < 0) {
                        atomicAdd(bad, 1);
                        return;
                    }
                    double sv = lv[p0];
                    for (int q2 = lrp[col]; q2 < lrp[col + 1]; ++q2)
                        sv -= lrow_d(lci, lv, ra[r], rb[r], lci[q2], part, d, doff) * lv[q2];
                    S[r][cix] = sv;
                }
            }
            for (int r = 0; r < nr; ++r) {
                if (ncol == 1) {
                    lv[pos[r][0]] = S[r][0] / d[k];
                } else {
                    const double o = doff[k];
                    const double det = d[k] * d[pk] - o * o;
                    lv[pos[r][0]] = (S[r][0] * d[pk] - S[r][1] * o) / det;
                    lv[pos[r][1]] = (S[r][1] * d[k] - S[r][0] * o) / det;
                }
            }
        }
    }
    const int rows[2] = {i, mi};
    double dd[2];
    for (int r = 0; r < nr; ++r) {
        double v = d[rows[r]];
        for (int q = ra[r]; q < rb[r]; ++q) v -= lv[q] * lrow_d(lci, lv, ra[r], rb[r], lci[q], part, d, doff);
        dd[r] = v;
    }
    if (nr == 1) {
        if (dd[0] == 0.0 || fabs(dd[0]) < thr) atomicAdd(nzero, 1);
        d[i] = dd[0];
        return;
    }
    double o = doff[i];
    for (int q = ra[1]; q < rb[1]; ++q) o -= lv[q] * lrow_d(lci, lv, ra[0], rb[0], lci[q], part, d, doff);
    const double det = dd[0] * dd[1] - o * o;
    if (det == 0.0 || fabs(det) < thr * dmax) atomicAdd(nzero, 1);
    d[i] = dd[0];
    d[mi] = dd[1];
    doff[i] = o;
    doff[mi] = o;
}

// |D|^-1/2 block by block (a 2x2 block [[a, b], [b, c]] as V |Lambda|^-1/2 V^T from its
// closed-form eigenpairs) and the number of U_r columns each vertex contributes:
// a negative 1x1 pivot one (e_i), a pair one per negative eigenvalue (at its leader)
__global__ void k_block_weights(int n, const int* __restrict__ part, const double* __restrict__ d,
                                const double* __restrict__ doff, double* wd, double* wo, int* ncols) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int m = part[i];
    if (m < 0) {
        wd[i] = 1.0 / sqrt(fabs(d[i]));
        wo[i] = 0.0;
        ncols[i] = d[i] < 0.0 ? 1 : 0;
        return;
    }
    if (m < i) {
        ncols[i] = 0;
        return;
    }
    const double a = d[i], b = doff[i], c = d[m];
    const double mid = 0.5 * (a + c), h = 0.5 * (a - c);
    const double rad = hypot(h, b);
    const double l1 = mid - rad, l2 = mid + rad;
    // eigenvector of l2 without cancellation, then v1 = its rotation by 90 degrees
    double x, y;
    if (h >= 0.0) {
        x = h + rad;
        y = b;
    } else {
        x = b;
        y = rad - h;
    }
    const double nv = hypot(x, y);
    if (nv > 0.0) {
        x /= nv;
        y /= nv;
    } else {
        x = 1.0;
        y = 0.0;
    }
    const double f1 = 1.0 / sqrt(fabs(l1)), f2 = 1.0 / sqrt(fabs(l2));
    wd[i] = f1 * y * y + f2 * x * x;
    wd[m] = f1 * x * x + f2 * y * y;
    wo[i] = wo[m] = (f2 - f1) * x * y;
    ncols[i] = (l1 < 0.0 ? 1 : 0) + (l2 < 0.0 ? 1 : 0);
}

__global__ void k_block_ur(int n, const int* __restrict__ part, const double* __restrict__ d,
                           const double* __restrict__ doff, const int* __restrict__ upos, int* i1, int* i2,
                           double* c1, double* c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int m = part[i];
    int q = upos[i];
    if (m < 0) {
        if (d[i] < 0.0) {
            i1[q] = i;
            i2[q] = -1;
            c1[q] = 1.0;
            c2[q] = 0.0;
        }
        return;
    }
    if (m < i) return;
    const double a = d[i], b = doff[i], c = d[m];
    const double mid = 0.5 * (a + c), h = 0.5 * (a - c);
    const double rad = hypot(h, b);
    const double l1 = mid - rad, l2 = mid + rad;
    double x, y;
    if (h >= 0.0) {
        x = h + rad;
        y = b;
    } else {
        x = b;
        y = rad - h;
    }
    const double nv = hypot(x, y);
    if (nv > 0.0) {
        x /= nv;
        y /= nv;
    } else {
        x = 1.0;
        y = 0.0;
    }
    if (l1 < 0.0) {   // v1 = (-y, x)
        i1[q] = i;
        i2[q] = m;
        c1[q] = -y;
        c2[q] = x;
        ++q;
    }
    if (l2 < 0.0) {   // v2 = (x, y)
        i1[q] = i;
        i2[q] = m;
        c1[q] = x;
        c2[q] = y;
    }
}

// y = W x with W = |D|^-1/2 (diagonal wd, and wo between the members of a pair)
__global__ void k_wmul(int n, const double* __restrict__ wd, const double* __restrict__ wo,
                       const int* __restrict__ part, const double* __restrict__ x, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = wd[i] * x[i];
    if (part) {
        const int m = part[i];
        if (m >= 0) v += wo[i] * x[m];
    }
    y[i] = v;
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


asss_status ildl_build(const Ctx& c, const DCsr& P0, const int* mirror0, const double* Cval0, double* d,
                       uint64_t seed, double zero_tol, bool fp32, IldlFactor& F, int* nzero, bool pivots2) {
    NvtxRange nv_("asss:ildl");
    cudaStream_t s = c.stream;
    const int n = P0.n;
    F.n = n;
    *nzero = 0;
    // 2x2 pivots: the pairs, then the block closure of the pattern with C on it
    const DCsr* Pp = &P0;
    const int* mirror = mirror0;
    const double* Cval = Cval0;
    DCsr Pb;
    DBuf<int> bmir;
    DBuf<double> bval;
    F.npairs = 0;
    F.nur = 0;
    if (pivots2 && n > 0) {
        DBuf<int> rbest, need, np;
        ASSS_TRY(rbest.alloc(n));
        ASSS_TRY(need.alloc(n));
        ASSS_TRY(np.alloc(1));
        ASSS_TRY(F.part.alloc(n));
        ASSS_CUDA(cudaMemsetAsync(np.p, 0, sizeof(int), s));
        k_bk_pick<<<cdiv(n, 256), 256, 0, s>>>(n, P0.rp.p, P0.ci.p, mirror0, Cval0, d, (1.0 + sqrt(17.0)) / 8.0,
                                               rbest.p, need.p);
        ASSS_CHECK_LAUNCH();
        k_bk_pair<<<cdiv(n, 256), 256, 0, s>>>(n, rbest.p, need.p, F.part.p, np.p);
        ASSS_CHECK_LAUNCH();
        int hnp = 0;
        ASSS_CUDA(cudaMemcpyAsync(&hnp, np.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        F.npairs = hnp / 2;
        if (F.npairs > 0) {
            DBuf<int> bcnt;
            ASSS_TRY(bcnt.alloc(n));
            k_bpat_row<<<cdiv(n, 128), 128, 0, s>>>(n, P0.rp.p, P0.ci.p, F.part.p, nullptr, bcnt.p, nullptr);
            ASSS_CHECK_LAUNCH();
            Pb.n = n;
            ASSS_TRY(Pb.rp.alloc(n + 1));
            int64_t tot = 0;
            ASSS_TRY(exclusive_scan(bcnt.p, Pb.rp.p, n, &tot, s));
            if (tot > 0x7fffffffLL) {
                set_error("the block pattern of the 2x2 pivots has too many entries (%lld)", (long long)tot);
                return ASSS_ERR_UNSUPPORTED;
            }
            Pb.nnz = (int)tot;
            ASSS_TRY(Pb.ci.alloc(tot > 0 ? tot : 1));
            k_bpat_row<<<cdiv(n, 128), 128, 0, s>>>(n, P0.rp.p, P0.ci.p, F.part.p, Pb.rp.p, nullptr, Pb.ci.p);
            ASSS_CHECK_LAUNCH();
            ASSS_TRY(bval.alloc(tot > 0 ? tot : 1));
            ASSS_TRY(bmir.alloc(tot > 0 ? tot : 1));
            ASSS_CUDA(cudaMemsetAsync(np.p, 0, sizeof(int), s));
            k_bpat_values<<<cdiv(n, 128), 128, 0, s>>>(n, P0.rp.p, P0.ci.p, Cval0, Pb.rp.p, Pb.ci.p, bval.p, bmir.p,
                                                       np.p);
            ASSS_CHECK_LAUNCH();
            int hbad = 0;
            ASSS_CUDA(cudaMemcpyAsync(&hbad, np.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            ASSS_CUDA(cudaStreamSynchronize(s));
            if (hbad) {
                set_error("the block closure of the pattern is not symmetric (%d entries)", hbad);
                return ASSS_ERR_PATTERN;
            }
            ASSS_TRY(F.doff.alloc(n));
            k_pair_offdiag<<<cdiv(n, 256), 256, 0, s>>>(n, F.part.p, Pb.rp.p, Pb.ci.p, bval.p, bmir.p, F.doff.p);
            ASSS_CHECK_LAUNCH();
            Pp = &Pb;
            mirror = bmir.p;
            Cval = bval.p;
        }
    }
    const DCsr& P = *Pp;
    const int* part = F.npairs > 0 ? F.part.p : nullptr;
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
        k_jp_round<<<cdiv(n, 256), 256, 0, s>>>(n, P.rp.p, P.ci.p, cseed, t, rnd.p, F.colour.p, left.p, ovf.p, part);
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
    ASSS_TRY(nz.alloc(2));
    ASSS_CUDA(cudaMemsetAsync(nz.p, 0, 2 * sizeof(int), s));
    for (int k = 0; k < F.ncol; ++k) {
        const int cnt = F.hls[k + 1] - F.hls[k];
        if (cnt == 0) continue;
        if (part)
            k_ildl_level_bk<<<cdiv(cnt, 128), 128, 0, s>>>(F.lvl.p + F.hls[k], cnt, k, F.colour.p, part, F.lrp.p,
                                                            F.lci.p, F.lv.p, d, F.doff.p, zero_tol * dmax, dmax, nz.p,
                                                            nz.p + 1);
        else
            k_ildl_level<<<cdiv(cnt, 128), 128, 0, s>>>(F.lvl.p + F.hls[k], cnt, k, F.colour.p, F.lrp.p, F.lci.p,
                                                         F.lv.p, d, zero_tol * dmax, nz.p);
        ASSS_CHECK_LAUNCH();
    }
    int hnz[2] = {0, 0};
    ASSS_CUDA(cudaMemcpyAsync(hnz, nz.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    k_fill_u<<<cdiv((int)(nu > 0 ? nu : 1), 256), 256, 0, s>>>((int)nu, umir.p, lpos.p, F.lv.p, F.uv.p);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(F.wd.alloc(n > 0 ? n : 1));
    if (part) {
        // |D|^-1/2 and U_r block by block
        DBuf<int> ncols, upos;
        ASSS_TRY(ncols.alloc(n));
        ASSS_TRY(upos.alloc(n + 1));
        ASSS_TRY(F.wo.alloc(n));
        k_block_weights<<<cdiv(n, 256), 256, 0, s>>>(n, part, d, F.doff.p, F.wd.p, F.wo.p, ncols.p);
        ASSS_CHECK_LAUNCH();
        int64_t nur = 0;
        ASSS_TRY(exclusive_scan(ncols.p, upos.p, n, &nur, s));
        F.nur = (int)nur;
        if (nur > 0) {
            ASSS_TRY(F.ur_i1.alloc(nur));
            ASSS_TRY(F.ur_i2.alloc(nur));
            ASSS_TRY(F.ur_c1.alloc(nur));
            ASSS_TRY(F.ur_c2.alloc(nur));
            k_block_ur<<<cdiv(n, 256), 256, 0, s>>>(n, part, d, F.doff.p, upos.p, F.ur_i1.p, F.ur_i2.p, F.ur_c1.p,
                                                     F.ur_c2.p);
            ASSS_CHECK_LAUNCH();
        }
    } else {
        k_inv_sqrt_abs<<<cdiv(n, 256), 256, 0, s>>>(n, d, F.wd.p);
        ASSS_CHECK_LAUNCH();
    }
    ASSS_CUDA(cudaStreamSynchronize(s));
    *nzero = hnz[0];
    if (hnz[1]) {
        set_error("the block pattern of the 2x2 pivots is not closed (%d blocks)", hnz[1]);
        return ASSS_ERR_BREAKDOWN;
    }
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
        if (part) {
            ASSS_TRY(F.wo32.alloc(n));
            k_d2f_n<<<cdiv(n, 256), 256, 0, s>>>(F.wo.p, n, F.wo32.p);
            ASSS_CHECK_LAUNCH();
        }
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
    k_wmul<<<cdiv(F.n, 256), 256, 0, s>>>(F.n, F.wd.p, F.wo.p, F.npairs ? F.part.p : nullptr, F.ft.p, out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// out = (I + L)^-T |D|^-1/2 v   (out != v)
asss_status ildl_G(const Ctx& c, IldlFactor& F, const double* v, double* out) {
    cudaStream_t s = c.stream;
    k_wmul<<<cdiv(F.n, 256), 256, 0, s>>>(F.n, F.wd.p, F.wo.p, F.npairs ? F.part.p : nullptr, v, F.ft.p);
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
