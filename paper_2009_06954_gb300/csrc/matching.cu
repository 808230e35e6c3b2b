// Maximum-product matching and scaling on the GPU: the role of MC64 in §2, Eq. mc64
// (a row permutation P and scalings D_r, D_c with |diag(P D_r A D_c)| = 1 and every
// other entry of modulus at most one).
//
// Formulation: cost c_ij = log(max_k |a_kj|) - log|a_ij| >= 0 on A's nonzeros, a
// perfect matching of minimum total cost (maximum product of the matched |a_ij|)
// and dual variables u_i + v_j <= c_ij.  The matching comes from Bertsekas' auction
// algorithm with epsilon-scaling, run in parallel (Jacobi) rounds:
//   bid:    every unassigned row i finds its best column j1 (largest -c_ij - p_j) and
//           the second best value; it bids p_j1 + (best - second) + eps for j1 and the
//           column keeps the largest bid (64-bit atomic max on the bid's bits: prices
//           are never negative, so their bit patterns order like the values);
//   win:    one of the rows that bid that largest value takes the column (CAS);
//   assign: the column's price becomes the winning bid, its former owner is unassigned.
// Each phase restarts the assignment with the prices of the last one and eps / 8,
// down to eps_final; every row then holds a column whose value is within eps_final of
// its best (eps-complementary slackness).  The duals v_j = -p_j, u_i = min_j (c_ij + p_j)
// are feasible; on the matching c_ij - u_i - v_j <= eps_final.  The scalings
// dr = exp(u), dc = exp(v) / colmax then give |entries| <= 1 and matched entries in
// [exp(-eps_final), 1]; the rows are finally divided by their matched entry, so the
// diagonal is exactly 1 in modulus and the rest at most exp(eps_final).
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asss {

__global__ void k_match_colmax(const int* rp, const int* ci, const double* v, int n, unsigned long long* cmax) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        double a = fabs(v[e]);
        unsigned long long bits;
        memcpy(&bits, &a, sizeof(bits));
        atomicMax(&cmax[ci[e]], bits);
    }
}

// cost of every nonzero; *bad counts explicit zeros (no finite cost) and empty columns
__global__ void k_match_costs(const int* rp, const int* ci, const double* v, const unsigned long long* cmax_bits, int n,
                              double* cost, unsigned long long* cmax_out, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        double cm;
        unsigned long long b = cmax_bits[ci[e]];
        memcpy(&cm, &b, sizeof(cm));
        const double a = fabs(v[e]);
        if (a > 0.0 && cm > 0.0) {
            cost[e] = fmax(log(cm) - log(a), 0.0);   // >= 0 (a <= cm); rounding kept non-negative
            atomicMax(cmax_out, (unsigned long long)__double_as_longlong(cost[e]));
        } else {
            cost[e] = INFINITY;
        }
    }
    double cm;
    unsigned long long b = cmax_bits[i];
    memcpy(&cm, &b, sizeof(cm));
    if (!(cm > 0.0)) atomicAdd(bad, 1);
}

__global__ void k_match_reset(int n, int* assigned, int* owner, unsigned long long* colbid, int* colwin,
                              unsigned* nassigned) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *nassigned = 0u;
    if (i >= n) return;
    assigned[i] = -1;
    owner[i] = -1;
    colbid[i] = 0ull;
    colwin[i] = -1;
}

__global__ void k_match_bid(const int* rp, const int* ci, const double* cost, int n, const double* price,
                            const int* assigned, double eps, double* bidval, int* bidcol,
                            unsigned long long* colbid) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bidcol[i] = -1;
    if (assigned[i] >= 0) return;
    double w1 = -INFINITY, w2 = -INFINITY;
    int j1 = -1;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const double c = cost[e];
        if (!(c < INFINITY)) continue;
        const int j = ci[e];
        const double val = -c - price[j];
        if (val > w1) {
            w2 = w1;
            w1 = val;
            j1 = j;
        } else if (val > w2) {
            w2 = val;
        }
    }
    if (j1 < 0) return;   // a row without finite entries: no perfect matching (caught by the round limit)
    // A row with one column has no second best.  Any bid of at least p + eps keeps
    // eps-complementary slackness for it; bidding just that (rather than an "infinite"
    // increment) keeps its column's price, and with it the range of the scalings, from
    // growing with every epsilon phase: such prices reached e^130 in tests, and scalings
    // that lopsided defeat the outer iteration in floating point.
    if (!(w2 > -INFINITY)) w2 = w1;
    const double bid = price[j1] + (w1 - w2) + eps;
    bidval[i] = bid;
    bidcol[i] = j1;
    atomicMax(&colbid[j1], (unsigned long long)__double_as_longlong(bid));
}

__global__ void k_match_win(int n, const double* bidval, const int* bidcol, const unsigned long long* colbid,
                            int* colwin) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = bidcol[i];
    if (j < 0) return;
    if ((unsigned long long)__double_as_longlong(bidval[i]) == colbid[j]) atomicCAS(&colwin[j], -1, i);
}

__global__ void k_match_assign(int n, int* owner, int* assigned, double* price, unsigned long long* colbid,
                               int* colwin, unsigned* nassigned) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int w = colwin[j];
    if (w < 0) return;
    const int old = owner[j];
    owner[j] = w;
    assigned[w] = j;
    if (old >= 0) assigned[old] = -1;
    else atomicAdd(nassigned, 1u);
    price[j] = __longlong_as_double((long long)colbid[j]);
    colbid[j] = 0ull;
    colwin[j] = -1;
}

// u_i = min_j (c_ij + p_j) (feasible row duals for v = -p), and the row's matched entry
__global__ void k_match_duals(const int* rp, const int* ci, const double* cost, int n, const double* price,
                              const int* assigned, double* u, double* cmatch) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = INFINITY, cm = INFINITY;
    const int ja = assigned[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const double c = cost[e];
        if (!(c < INFINITY)) continue;
        m = fmin(m, c + price[ci[e]]);
        if (ci[e] == ja) cm = c;
    }
    u[i] = m;
    cmatch[i] = cm;
}

// dr_i = exp(u_i - shift) / exp-slack of its match, dc_j = exp(v_j + shift) / colmax_j, perm[j] = owner[j]
__global__ void k_match_scale(int n, const double* u, const double* price, const double* cmatch, const int* assigned,
                              const unsigned long long* cmax_bits, double shift, double* dr, double* dc, int* perm,
                              const int* owner) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // row i: |a_ij d_r d_c| = exp(u_i + v_j - c_ij) on its matched column j; divide it out
    const int j = assigned[i];
    const double slack = cmatch[i] - (u[i] - price[j]);   // c_ij - u_i - v_j >= 0
    dr[i] = exp(u[i] - shift + slack);
    double cm;
    unsigned long long b = cmax_bits[i];
    memcpy(&cm, &b, sizeof(cm));
    dc[i] = exp(-price[i] + shift) / cm;
    perm[i] = owner[i];
}

asss_status matching_scaling(const Ctx& c, const DCsr& A, int* perm, double* dr, double* dc, int* rounds_out,
                             double* eps_out) {
    NvtxRange nv_("asss:matching");
    cudaStream_t s = c.stream;
    const int n = A.n;
    const int nb = cdiv(n, 256);
    DBuf<unsigned long long> cmax, colbid, cmaxc;
    DBuf<double> cost, price, bidval, u, cm;
    DBuf<int> assigned, owner, colwin, bidcol, bad;
    DBuf<unsigned> nas;
    ASSS_TRY(cmax.alloc(n));
    ASSS_TRY(cmaxc.alloc(1));
    ASSS_TRY(cost.alloc(A.nnz > 0 ? A.nnz : 1));
    ASSS_TRY(price.alloc(n));
    ASSS_TRY(bidval.alloc(n));
    ASSS_TRY(u.alloc(n));
    ASSS_TRY(cm.alloc(n));
    ASSS_TRY(assigned.alloc(n));
    ASSS_TRY(owner.alloc(n));
    ASSS_TRY(colwin.alloc(n));
    ASSS_TRY(bidcol.alloc(n));
    ASSS_TRY(colbid.alloc(n));
    ASSS_TRY(bad.alloc(1));
    ASSS_TRY(nas.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(cmax.p, 0, sizeof(unsigned long long) * n, s));
    ASSS_CUDA(cudaMemsetAsync(cmaxc.p, 0, sizeof(unsigned long long), s));
    ASSS_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    ASSS_CUDA(cudaMemsetAsync(price.p, 0, sizeof(double) * n, s));
    k_match_colmax<<<nb, 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, n, cmax.p);
    ASSS_CHECK_LAUNCH();
    k_match_costs<<<nb, 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, cmax.p, n, cost.p, cmaxc.p, bad.p);
    ASSS_CHECK_LAUNCH();
    int hbad = 0;
    unsigned long long hcm = 0;
    ASSS_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaMemcpyAsync(&hcm, cmaxc.p, sizeof(hcm), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        set_error("matching: A has an empty column");
        return ASSS_ERR_PATTERN;
    }
    double cmaxv;
    memcpy(&cmaxv, &hcm, sizeof(cmaxv));
    const double scale = cmaxv > 1.0 ? cmaxv : 1.0;
    const double eps_final = 1e-12 * scale;
    // rounds allowed in all (a structurally singular A never completes a phase)
    const long long max_rounds = 10000LL + 50LL * n;
    long long rounds = 0;
    unsigned hn = 0;
    for (double eps = scale / 4.0;; eps = fmax(eps / 8.0, eps_final)) {
        k_match_reset<<<nb, 256, 0, s>>>(n, assigned.p, owner.p, colbid.p, colwin.p, nas.p);
        ASSS_CHECK_LAUNCH();
        hn = 0;
        while (true) {
            // several rounds between read-backs of the assigned count
            for (int r = 0; r < 8; ++r) {
                k_match_bid<<<nb, 256, 0, s>>>(A.rp.p, A.ci.p, cost.p, n, price.p, assigned.p, eps, bidval.p,
                                               bidcol.p, colbid.p);
                ASSS_CHECK_LAUNCH();
                k_match_win<<<nb, 256, 0, s>>>(n, bidval.p, bidcol.p, colbid.p, colwin.p);
                ASSS_CHECK_LAUNCH();
                k_match_assign<<<nb, 256, 0, s>>>(n, owner.p, assigned.p, price.p, colbid.p, colwin.p, nas.p);
                ASSS_CHECK_LAUNCH();
            }
            rounds += 8;
            ASSS_CUDA(cudaMemcpyAsync(&hn, nas.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            ASSS_CUDA(cudaStreamSynchronize(s));
            if ((int)hn == n) break;
            if (rounds > max_rounds) {
                set_error("matching: no perfect matching after %lld auction rounds (A structurally singular?)",
                          rounds);
                return ASSS_ERR_PATTERN;
            }
        }
        if (eps <= eps_final) break;
    }
    k_match_duals<<<nb, 256, 0, s>>>(A.rp.p, A.ci.p, cost.p, n, price.p, assigned.p, u.p, cm.p);
    ASSS_CHECK_LAUNCH();
    // centre the duals (u + v is what matters) so that exp() stays in range
    std::vector<double> hu(n), hp(n);
    ASSS_CUDA(cudaMemcpyAsync(hu.data(), u.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaMemcpyAsync(hp.data(), price.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    double su = 0.0, sp = 0.0;
    for (int i = 0; i < n; ++i) {
        su += hu[i];
        sp += hp[i];
    }
    const double shift = 0.5 * (su + sp) / n;   // mean(u) - shift = -(mean(v) + shift)
    k_match_scale<<<nb, 256, 0, s>>>(n, u.p, price.p, cm.p, assigned.p, cmax.p, shift, dr, dc, perm, owner.p);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (rounds_out) *rounds_out = (int)(rounds < 2147483647LL ? rounds : 2147483647LL);
    if (eps_out) *eps_out = eps_final;
    return ASSS_OK;
}

}  // namespace asss
