// The least-squares problem for the shifted skew-symmetrizer S (paper §2,
// Eqs. eq1, eq2, regularized; App. A), solved on the device without forming B.
//
// Unknowns: the entries of S on its pattern (CSR order).  Constraint rows: one
// per upper entry (i < j) of the symmetric pattern P = pat(Abar S) + pat(Abar S)^T,
// stating (Abar S)_ij + (Abar S)_ji = 0, and one per diagonal entry,
// sqrt(gamma) (Abar S)_ii = sqrt(gamma).  With C = Abar S evaluated on P:
//   (B s)_ij = C_ij + C_ji  (i < j),    (B s)_ii = sqrt(gamma) C_ii
//   (B^T t)_lj = sum_i abar_il G_ij  with G symmetric on P, G_ij = t_{min,max}
//   (off-diagonal) and G_ii = sqrt(gamma) t_ii.
// Each output is one sorted-list intersection ("merge dot"), computed by one
// thread, so results do not depend on scheduling.
//
// The normal equations B^T B s = B^T v are solved by preconditioned conjugate
// gradients.  The preconditioner is block-Jacobi on the pairs {s_lj, s_jl}: when
// Abar is close to I a skew perturbation of S barely changes the objective, so
// the two entries of a pair are strongly coupled; the 2x2 Gram block of a pair is
//   [ sum_i abar_il^2 w_ij     abar_ll abar_jj ]
//   [ abar_ll abar_jj          sum_i abar_ij^2 w_il ]     (w = gamma on i = column)
// and is inverted in closed form.
#include "common.cuh"
#include "internal.h"

namespace asss {

__device__ __forceinline__ double merge_dot_s(const int* __restrict__ ac, const double* __restrict__ av, int alen,
                                              const int* __restrict__ bc, const int* __restrict__ bu, int blen,
                                              const double* __restrict__ s) {
    int x = 0, y = 0;
    double acc = 0.0;
    while (x < alen && y < blen) {
        int ca = ac[x], cb = bc[y];
        if (ca == cb) {
            acc += av[x] * s[bu[y]];
            ++x;
            ++y;
        } else if (ca < cb) {
            ++x;
        } else {
            ++y;
        }
    }
    return acc;
}

__global__ void k_row_of_entry(const int* rp, int n, int* row) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) row[e] = i;
}

// q = B s on the constraint entries of P (upper + diagonal); lower entries get 0
__global__ void k_lls_B(int nP, const int* __restrict__ prow, const int* __restrict__ pci,
                        const int* __restrict__ arp, const int* __restrict__ aci, const double* __restrict__ av,
                        const int* __restrict__ strp, const int* __restrict__ stci, const int* __restrict__ stsrc,
                        const double* __restrict__ s, double sg, double* q) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nP) return;
    int i = prow[k], j = pci[k];
    if (j < i) {
        q[k] = 0.0;
        return;
    }
    double cij = merge_dot_s(aci + arp[i], av + arp[i], arp[i + 1] - arp[i], stci + strp[j], stsrc + strp[j],
                             strp[j + 1] - strp[j], s);
    if (j == i) {
        q[k] = sg * cij;
        return;
    }
    double cji = merge_dot_s(aci + arp[j], av + arp[j], arp[j + 1] - arp[j], stci + strp[i], stsrc + strp[i],
                             strp[i + 1] - strp[i], s);
    q[k] = cij + cji;
}

// C = Abar S on every entry of P
__global__ void k_lls_C(int nP, const int* __restrict__ prow, const int* __restrict__ pci,
                        const int* __restrict__ arp, const int* __restrict__ aci, const double* __restrict__ av,
                        const int* __restrict__ strp, const int* __restrict__ stci, const int* __restrict__ stsrc,
                        const double* __restrict__ s, double* C) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nP) return;
    int i = prow[k], j = pci[k];
    C[k] = merge_dot_s(aci + arp[i], av + arp[i], arp[i + 1] - arp[i], stci + strp[j], stsrc + strp[j],
                       strp[j + 1] - strp[j], s);
}

// g = B^T t on the unknowns
__global__ void k_lls_BT(int nS, const int* __restrict__ srow, const int* __restrict__ sci,
                         const int* __restrict__ atrp, const int* __restrict__ atci, const double* __restrict__ atv,
                         const int* __restrict__ prp, const int* __restrict__ pci, const int* __restrict__ mirror,
                         const double* __restrict__ t, double sg, double* g) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nS) return;
    int l = srow[u], j = sci[u];
    int x = atrp[l], xe = atrp[l + 1];
    int y = prp[j], ye = prp[j + 1];
    double acc = 0.0;
    while (x < xe && y < ye) {
        int ia = atci[x], ib = pci[y];
        if (ia == ib) {
            double G;
            if (ia > j) G = t[y];
            else if (ia < j) G = (mirror[y] >= 0) ? t[mirror[y]] : 0.0;
            else G = sg * t[y];
            acc += atv[x] * G;
            ++x;
            ++y;
        } else if (ia < ib) {
            ++x;
        } else {
            ++y;
        }
    }
    g[u] = acc;
}

// ---------------------------------------------------------------------------
// B and B^T stored explicitly (when they fit a memory budget): the entries each merge
// above would visit, in the same order, so the products are bit for bit those of the
// merge kernels while each iteration streams two sparse matrices instead of redoing
// the intersections.  B row k: the C_ij terms (unknown, abar_il) then - off the
// diagonal - the C_ji terms from position bsplit[k]; B^T row u: (P position, abar_lj),
// a position stored as ~pos where the diagonal weight sqrt(gamma) applies.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int merge_list(const int* __restrict__ ac, const double* __restrict__ av, int alen,
                                          const int* __restrict__ bc, const int* __restrict__ bu, int blen,
                                          int* oc, double* ov) {
    int x = 0, y = 0, k = 0;
    while (x < alen && y < blen) {
        int ca = ac[x], cb = bc[y];
        if (ca == cb) {
            if (oc) {
                oc[k] = bu[y];
                ov[k] = av[x];
            }
            ++k;
            ++x;
            ++y;
        } else if (ca < cb) {
            ++x;
        } else {
            ++y;
        }
    }
    return k;
}

// count (bcol == nullptr) or fill row k of B
__global__ void k_bx_rows(int nP, const int* __restrict__ prow, const int* __restrict__ pci,
                          const int* __restrict__ arp, const int* __restrict__ aci, const double* __restrict__ av,
                          const int* __restrict__ strp, const int* __restrict__ stci, const int* __restrict__ stsrc,
                          const int* brp, int* bcnt, int* bsplit, int* bcol, double* bval) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nP) return;
    int i = prow[k], j = pci[k];
    if (j < i) {
        if (!bcol) bcnt[k] = 0;
        else bsplit[k] = 0;
        return;
    }
    int* oc = bcol ? bcol + brp[k] : nullptr;
    double* ov = bcol ? bval + brp[k] : nullptr;
    int a = merge_list(aci + arp[i], av + arp[i], arp[i + 1] - arp[i], stci + strp[j], stsrc + strp[j],
                       strp[j + 1] - strp[j], oc, ov);
    int b = 0;
    if (j != i)
        b = merge_list(aci + arp[j], av + arp[j], arp[j + 1] - arp[j], stci + strp[i], stsrc + strp[i],
                       strp[i + 1] - strp[i], oc ? oc + a : nullptr, ov ? ov + a : nullptr);
    if (!bcol) bcnt[k] = a + b;
    else bsplit[k] = a;
}

// q = B s, summed as the merge kernel does: C_ij and C_ji separately, then added
__global__ void k_bx_apply(int nP, const int* __restrict__ prow, const int* __restrict__ pci,
                           const int* __restrict__ brp, const int* __restrict__ bsplit,
                           const int* __restrict__ bcol, const double* __restrict__ bval,
                           const double* __restrict__ s, double sg, double* q) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nP) return;
    const int i = prow[k], j = pci[k];
    if (j < i) {
        q[k] = 0.0;
        return;
    }
    const int e0 = brp[k], e1 = brp[k + 1], em = e0 + bsplit[k];
    double cij = 0.0;
    for (int e = e0; e < em; ++e) cij += bval[e] * s[bcol[e]];
    if (j == i) {
        q[k] = sg * cij;
        return;
    }
    double cji = 0.0;
    for (int e = em; e < e1; ++e) cji += bval[e] * s[bcol[e]];
    q[k] = cij + cji;
}

// count (tcol == nullptr) or fill row u of B^T (same walk as k_lls_BT)
__global__ void k_btx_rows(int nS, const int* __restrict__ srow, const int* __restrict__ sci,
                           const int* __restrict__ atrp, const int* __restrict__ atci, const double* __restrict__ atv,
                           const int* __restrict__ prp, const int* __restrict__ pci, const int* __restrict__ mirror,
                           const int* trp, int* tcnt, int* tcol, double* tval) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nS) return;
    int l = srow[u], j = sci[u];
    int x = atrp[l], xe = atrp[l + 1];
    int y = prp[j], ye = prp[j + 1];
    int o = tcol ? trp[u] : 0;
    int k = 0;
    while (x < xe && y < ye) {
        int ia = atci[x], ib = pci[y];
        if (ia == ib) {
            int pos;
            if (ia > j) pos = y;
            else if (ia < j) pos = mirror[y] >= 0 ? mirror[y] : -1;   // none: a zero term, left out
            else pos = ~y;                                           // the diagonal: weight sqrt(gamma)
            if (ia == j || pos >= 0) {
                if (tcol) {
                    tcol[o + k] = pos;
                    tval[o + k] = atv[x];
                }
                ++k;
            }
            ++x;
            ++y;
        } else if (ia < ib) {
            ++x;
        } else {
            ++y;
        }
    }
    if (!tcol) tcnt[u] = k;
}

__global__ void k_btx_apply(int nS, const int* __restrict__ trp, const int* __restrict__ tcol,
                            const double* __restrict__ tval, const double* __restrict__ t, double sg, double* g) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nS) return;
    double acc = 0.0;
    for (int e = trp[u]; e < trp[u + 1]; ++e) {
        const int c = tcol[e];
        const double G = c >= 0 ? t[c] : sg * t[~c];
        acc += tval[e] * G;
    }
    g[u] = acc;
}

__global__ void k_diag_values(const int* rp, const int* ci, const double* v, int n, double* dv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == i) {
            d = v[e];
            break;
        }
    dv[i] = d;
}

__global__ void k_lls_prec_setup(int nS, const int* srow, const int* sci, const int* srp,
                                 const int* atrp, const int* atci, const double* atv, const double* adiag,
                                 double gamma, double* N, int* partner, double* cross) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nS) return;
    int l = srow[u], j = sci[u];
    double acc = 0.0;
    for (int e = atrp[l]; e < atrp[l + 1]; ++e) {
        double a = atv[e];
        acc += a * a * (atci[e] == j ? gamma : 1.0);
    }
    N[u] = acc;
    int p = -1;
    if (l != j) {
        int lo = srp[j], hi = srp[j + 1] - 1;
        while (lo <= hi) {
            int mid = lo + ((hi - lo) >> 1);   // no overflow for offsets near 2^31
            int c = sci[mid];
            if (c == l) {
                p = mid;
                break;
            }
            if (c < l) lo = mid + 1;
            else hi = mid - 1;
        }
    }
    partner[u] = p;
    cross[u] = (p >= 0) ? adiag[l] * adiag[j] : 0.0;
}

__global__ void k_lls_prec_apply(int nS, const double* N, const int* partner, const double* cross, const double* r,
                                 double* z) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nS) return;
    double nu = N[u];
    if (nu <= 0.0) {
        z[u] = 0.0;
        return;
    }
    int p = partner[u];
    if (p >= 0) {
        double np = N[p], c = cross[u];
        double det = nu * np - c * c;
        if (det > 1e-12 * nu * np) {
            z[u] = (np * r[u] - c * r[p]) / det;
            return;
        }
    }
    z[u] = r[u] / nu;
}

__global__ void k_lls_init_rho(int nP, const int* prow, const int* pci, double sg, double* rho) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nP) return;
    rho[k] = (prow[k] == pci[k]) ? sg : 0.0;
}

__global__ void k_cg_update(double* s, const double* p, int nS, double* rho, const double* q, int nP,
                            const double* rz, const double* qq) {
    double a = (*qq > 0.0) ? (*rz) / (*qq) : 0.0;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nS) s[t] += a * p[t];
    if (t < nP) rho[t] -= a * q[t];
}

__global__ void k_cg_newp(double* p, const double* z, int nS, const double* rz_new, const double* rz_old) {
    double b = (*rz_old != 0.0) ? (*rz_new) / (*rz_old) : 0.0;
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nS) p[u] = z[u] + b * p[u];
}

__global__ void k_sum_counts(const int* cnt, int n, unsigned long long* total) {
    unsigned long long a = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a += (unsigned)cnt[i];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, a);
}

// the sum of n counts in 64 bits (integer: the same whatever the order)
static asss_status sum_counts(const int* cnt, int n, int64_t* total, cudaStream_t s) {
    DBuf<unsigned long long> t;
    ASSS_TRY(t.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(t.p, 0, sizeof(unsigned long long), s));
    k_sum_counts<<<256, 256, 0, s>>>(cnt, n, t.p);
    ASSS_CHECK_LAUNCH();
    unsigned long long h = 0;
    ASSS_CUDA(cudaMemcpyAsync(&h, t.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    *total = (int64_t)h;
    return ASSS_OK;
}

asss_status lls_product_on_pattern(const Ctx& c, const DCsr& Abar, const DCsr& ST, const int* st_src,
                                   const double* s_val, const DCsr& P, const int* prow, double* Cval) {
    k_lls_C<<<cdiv(P.nnz, 256), 256, 0, c.stream>>>(P.nnz, prow, P.ci.p, Abar.rp.p, Abar.ci.p, Abar.v.p, ST.rp.p,
                                                      ST.ci.p, st_src, s_val, Cval);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

asss_status lls_fit(const Ctx& c, const DCsr& Abar, const DCsr& AbarT, const DCsr& Spat, double gamma, double tol,
                    int maxit, DBuf<double>& s_val, DCsr& P, DBuf<int>& mirror, DBuf<int>& diagpos,
                    DBuf<double>& Cval, LlsResult* res, const double* s0) {
    cudaStream_t s = c.stream;
    int n = Abar.n;
    int nS = Spat.nnz;
    // S^T pattern with the CSR position of every entry of S
    DCsr ST;
    DBuf<int> st_src;
    ASSS_TRY(transpose_csr(Spat, ST, &st_src, s));
    ASSS_TRY(build_pattern(Abar, AbarT, Spat, ST, P, mirror, diagpos, s));
    int nP = P.nnz;
    DBuf<int> prow, srow;
    ASSS_TRY(prow.alloc(nP));
    ASSS_TRY(srow.alloc(nS));
    k_row_of_entry<<<cdiv(n, 256), 256, 0, s>>>(P.rp.p, n, prow.p);
    ASSS_CHECK_LAUNCH();
    k_row_of_entry<<<cdiv(n, 256), 256, 0, s>>>(Spat.rp.p, n, srow.p);
    ASSS_CHECK_LAUNCH();

    // preconditioner
    DBuf<double> adiag, Nn, cross;
    DBuf<int> partner;
    ASSS_TRY(adiag.alloc(n));
    ASSS_TRY(Nn.alloc(nS));
    ASSS_TRY(cross.alloc(nS));
    ASSS_TRY(partner.alloc(nS));
    k_diag_values<<<cdiv(n, 256), 256, 0, s>>>(Abar.rp.p, Abar.ci.p, Abar.v.p, n, adiag.p);
    ASSS_CHECK_LAUNCH();
    k_lls_prec_setup<<<cdiv(nS, 256), 256, 0, s>>>(nS, srow.p, Spat.ci.p, Spat.rp.p, AbarT.rp.p, AbarT.ci.p,
                                                    AbarT.v.p, adiag.p, gamma, Nn.p, partner.p, cross.p);
    ASSS_CHECK_LAUNCH();

    const double sg = sqrt(gamma);
    DBuf<double> rho, q, r, z, p, sc;
    ASSS_TRY(s_val.alloc(nS));
    ASSS_TRY(rho.alloc(nP));
    ASSS_TRY(q.alloc(nP));
    ASSS_TRY(r.alloc(nS));
    ASSS_TRY(z.alloc(nS));
    ASSS_TRY(p.alloc(nS));
    ASSS_TRY(sc.alloc(8));  // 0: rz, 1: qq, 2: rr, 3: rz_new, 4: rr0
    double* d_rz = sc.p;
    double* d_qq = sc.p + 1;
    double* d_rr = sc.p + 2;
    double* d_rzn = sc.p + 3;
    ASSS_CUDA(cudaMemsetAsync(s_val.p, 0, sizeof(double) * nS, s));
    k_lls_init_rho<<<cdiv(nP, 256), 256, 0, s>>>(nP, prow.p, P.ci.p, sg, rho.p);
    ASSS_CHECK_LAUNCH();
    // B and B^T stored explicitly when they fit min(8 GiB, a quarter of the free device
    // memory): the same products, bit for bit, streamed instead of re-intersected each
    // iteration; otherwise the merge kernels apply them matrix-free
    DBuf<int> bcnt, brp, bsplit, bcol, tcnt, trp, tcol;
    DBuf<double> bval, tval;
    bool explicit_b = false;
    {
        ASSS_TRY(bcnt.alloc(nP > 0 ? nP : 1));
        ASSS_TRY(tcnt.alloc(nS > 0 ? nS : 1));
        k_bx_rows<<<cdiv(nP, 256), 256, 0, s>>>(nP, prow.p, P.ci.p, Abar.rp.p, Abar.ci.p, Abar.v.p, ST.rp.p, ST.ci.p,
                                                 st_src.p, nullptr, bcnt.p, nullptr, nullptr, nullptr);
        ASSS_CHECK_LAUNCH();
        k_btx_rows<<<cdiv(nS, 256), 256, 0, s>>>(nS, srow.p, Spat.ci.p, AbarT.rp.p, AbarT.ci.p, AbarT.v.p, P.rp.p,
                                                  P.ci.p, mirror.p, nullptr, tcnt.p, nullptr, nullptr);
        ASSS_CHECK_LAUNCH();
        int64_t nb = 0, nt = 0;
        ASSS_TRY(sum_counts(bcnt.p, nP, &nb, s));
        ASSS_TRY(sum_counts(tcnt.p, nS, &nt, s));
        size_t fr = 0, tot = 0;
        ASSS_CUDA(cudaMemGetInfo(&fr, &tot));
        const double need = 12.0 * (double)(nb + nt) + 8.0 * (double)(nP + nS);
        const double budget = fmin(8.0 * 1024 * 1024 * 1024, 0.25 * (double)fr);
        explicit_b = nb < 0x7fffffffLL && nt < 0x7fffffffLL && need <= budget;
        if (explicit_b) {
            ASSS_TRY(brp.alloc(nP + 1));
            ASSS_TRY(trp.alloc(nS + 1));
            ASSS_TRY(exclusive_scan(bcnt.p, brp.p, nP, nullptr, s));
            ASSS_TRY(exclusive_scan(tcnt.p, trp.p, nS, nullptr, s));
            ASSS_TRY(bsplit.alloc(nP > 0 ? nP : 1));
            ASSS_TRY(bcol.alloc(nb > 0 ? nb : 1));
            ASSS_TRY(bval.alloc(nb > 0 ? nb : 1));
            ASSS_TRY(tcol.alloc(nt > 0 ? nt : 1));
            ASSS_TRY(tval.alloc(nt > 0 ? nt : 1));
            k_bx_rows<<<cdiv(nP, 256), 256, 0, s>>>(nP, prow.p, P.ci.p, Abar.rp.p, Abar.ci.p, Abar.v.p, ST.rp.p,
                                                     ST.ci.p, st_src.p, brp.p, nullptr, bsplit.p, bcol.p, bval.p);
            ASSS_CHECK_LAUNCH();
            k_btx_rows<<<cdiv(nS, 256), 256, 0, s>>>(nS, srow.p, Spat.ci.p, AbarT.rp.p, AbarT.ci.p, AbarT.v.p,
                                                      P.rp.p, P.ci.p, mirror.p, trp.p, nullptr, tcol.p, tval.p);
            ASSS_CHECK_LAUNCH();
        }
    }
    auto applyBT = [&](const double* t, double* g) -> asss_status {
        if (explicit_b)
            k_btx_apply<<<cdiv(nS, 256), 256, 0, s>>>(nS, trp.p, tcol.p, tval.p, t, sg, g);
        else
            k_lls_BT<<<cdiv(nS, 256), 256, 0, s>>>(nS, srow.p, Spat.ci.p, AbarT.rp.p, AbarT.ci.p, AbarT.v.p, P.rp.p,
                                                    P.ci.p, mirror.p, t, sg, g);
        ASSS_CHECK_LAUNCH();
        return ASSS_OK;
    };
    auto applyB = [&](const double* sv, double* out) -> asss_status {
        if (explicit_b)
            k_bx_apply<<<cdiv(nP, 256), 256, 0, s>>>(nP, prow.p, P.ci.p, brp.p, bsplit.p, bcol.p, bval.p, sv, sg,
                                                      out);
        else
            k_lls_B<<<cdiv(nP, 256), 256, 0, s>>>(nP, prow.p, P.ci.p, Abar.rp.p, Abar.ci.p, Abar.v.p, ST.rp.p,
                                                   ST.ci.p, st_src.p, sv, sg, out);
        ASSS_CHECK_LAUNCH();
        return ASSS_OK;
    };
    auto precond = [&]() -> asss_status {
        k_lls_prec_apply<<<cdiv(nS, 256), 256, 0, s>>>(nS, Nn.p, partner.p, cross.p, r.p, z.p);
        ASSS_CHECK_LAUNCH();
        return ASSS_OK;
    };
    // the tolerance is relative to ||B^T v|| (the gradient at s = 0), also when the
    // iteration starts from given values s0 (a set-up resumed from saved S values)
    ASSS_TRY(applyBT(rho.p, r.p));
    ASSS_TRY(dot(r.p, r.p, nS, d_rr, s));
    double rr0 = 0.0;
    ASSS_CUDA(cudaMemcpyAsync(&rr0, d_rr, sizeof(double), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    double rel = rr0 > 0 ? 1.0 : 0.0;
    if (s0 && rr0 > 0) {
        ASSS_CUDA(cudaMemcpyAsync(s_val.p, s0, sizeof(double) * nS, cudaMemcpyDeviceToDevice, s));
        ASSS_TRY(applyB(s_val.p, q.p));
        ASSS_TRY(vaxpy(rho.p, q.p, -1.0, nP, s));  // rho = v - B s0
        ASSS_TRY(applyBT(rho.p, r.p));
        ASSS_TRY(dot(r.p, r.p, nS, d_rr, s));
        double rr = 0.0;
        ASSS_CUDA(cudaMemcpyAsync(&rr, d_rr, sizeof(double), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        rel = sqrt(rr / rr0);
    }
    ASSS_TRY(precond());
    ASSS_TRY(vcopy(p.p, z.p, nS, s));
    ASSS_TRY(dot(r.p, z.p, nS, d_rz, s));
    int its = 0;
    const int check_every = 8;
    int mx = nS > nP ? nS : nP;
    while (rr0 > 0 && rel > tol && its < maxit) {
        ASSS_TRY(applyB(p.p, q.p));
        ASSS_TRY(dot(q.p, q.p, nP, d_qq, s));
        k_cg_update<<<cdiv(mx, 256), 256, 0, s>>>(s_val.p, p.p, nS, rho.p, q.p, nP, d_rz, d_qq);
        ASSS_CHECK_LAUNCH();
        ASSS_TRY(applyBT(rho.p, r.p));
        ASSS_TRY(precond());
        ASSS_TRY(dot(r.p, z.p, nS, d_rzn, s));
        k_cg_newp<<<cdiv(nS, 256), 256, 0, s>>>(p.p, z.p, nS, d_rzn, d_rz);
        ASSS_CHECK_LAUNCH();
        ASSS_CUDA(cudaMemcpyAsync(d_rz, d_rzn, sizeof(double), cudaMemcpyDeviceToDevice, s));
        ++its;
        if (its % check_every == 0 || its == maxit) {
            ASSS_TRY(dot(r.p, r.p, nS, d_rr, s));
            double rr = 0.0;
            ASSS_CUDA(cudaMemcpyAsync(&rr, d_rr, sizeof(double), cudaMemcpyDeviceToHost, s));
            ASSS_CUDA(cudaStreamSynchronize(s));
            rel = sqrt(rr / rr0);
            if (rel <= tol) break;
        }
    }
    if (res) {
        res->its = its;
        res->relgrad = rel;
    }
    ASSS_TRY(Cval.alloc(nP));
    ASSS_TRY(lls_product_on_pattern(c, Abar, ST, st_src.p, s_val.p, P, prow.p, Cval.p));
    return ASSS_OK;
}

}  // namespace asss
