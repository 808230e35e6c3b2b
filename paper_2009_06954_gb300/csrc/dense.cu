// Small dense and tall-skinny kernels (FP64): the Lanczos start vector, Gram
// products for re-orthogonalisation and the SMW matrices, the small inverse of
// the SMW matrix, and vector updates.
#include "common.cuh"
#include "internal.h"

namespace asss {

// ---------------------------------------------------------------------------
// splitmix64 (Vigna): state_i = seed + (i+1)*golden, u = (mix >> 11) * 2^-53
// ---------------------------------------------------------------------------
__global__ void k_splitmix(uint64_t seed, int n, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    out[i] = 2.0 * u - 1.0;
}

asss_status splitmix64_fill(uint64_t seed, int n, double* out, cudaStream_t s) {
    k_splitmix<<<cdiv(n, 256), 256, 0, s>>>(seed, n, out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// G = A^T B (p x q, row-major), A n x p and B n x q column-major.
// Block b sums rows [b*CH, (b+1)*CH) for every (a, c) pair; partials are then
// added in block order (deterministic).
// ---------------------------------------------------------------------------
constexpr int GRAM_THREADS = 256;
constexpr int GRAM_BLOCKS = 296;

__global__ void k_gram_partial(const double* __restrict__ A, int lda, int p, const double* __restrict__ B, int ldb,
                               int q, int n, double* part) {
    const int pq = p * q;
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * chunk;
    const int r1 = min(n, r0 + chunk);
    for (int t = threadIdx.x; t < pq; t += blockDim.x) {
        int a = t / q, c = t % q;
        const double* pa = A + (size_t)a * lda;
        const double* pb = B + (size_t)c * ldb;
        double acc = 0.0;
        for (int r = r0; r < r1; ++r) acc += pa[r] * pb[r];
        part[(size_t)blockIdx.x * pq + t] = acc;
    }
}

// one warp per output, lanes stride over the block partials (fixed order)
__global__ void k_gram_final(const double* part, int nb, int pq, double* G) {
    int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (t >= pq) return;
    double acc = 0.0;
    for (int b = lane; b < nb; b += 32) acc += part[(size_t)b * pq + t];
    acc = warp_sum(acc);
    if (lane == 0) G[t] = acc;
}

// q == 1: part[b*p + a] = sum over the rows of block b of A[r, a] x[r].  Columns are
// taken eight at a time so each thread keeps eight independent loads in flight.
constexpr int GEMTV_CH = 8;
__global__ void k_gemtv_partial(const double* __restrict__ A, int lda, int p, const double* __restrict__ x, int n,
                                double* part) {
    __shared__ double sw[GRAM_THREADS / 32][GEMTV_CH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a0 = 0; a0 < p; a0 += GEMTV_CH) {
        double acc[GEMTV_CH];
#pragma unroll
        for (int t = 0; t < GEMTV_CH; ++t) acc[t] = 0.0;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            double xr = x[r];
#pragma unroll
            for (int t = 0; t < GEMTV_CH; ++t)
                if (a0 + t < p) acc[t] += A[(size_t)(a0 + t) * lda + r] * xr;
        }
#pragma unroll
        for (int t = 0; t < GEMTV_CH; ++t) {
            double v = warp_sum(acc[t]);
            if (lane == 0) sw[warp][t] = v;
        }
        __syncthreads();
        if (threadIdx.x < GEMTV_CH && a0 + threadIdx.x < p) {
            double v = 0.0;
            for (int w = 0; w < GRAM_THREADS / 32; ++w) v += sw[w][threadIdx.x];
            part[(size_t)blockIdx.x * p + a0 + threadIdx.x] = v;
        }
        __syncthreads();
    }
}

asss_status gram(const double* A, int lda, int p, const double* B, int ldb, int q, int n, double* G,
                 cudaStream_t s) {
    if (p == 0 || q == 0) return ASSS_OK;
    double* part = nullptr;
    ASSS_TRY(process_scratch(1, (int64_t)GRAM_BLOCKS * p * q, &part));
    if (q == 1) {
        k_gemtv_partial<<<GRAM_BLOCKS, GRAM_THREADS, 0, s>>>(A, lda, p, B, n, part);
    } else {
        k_gram_partial<<<GRAM_BLOCKS, GRAM_THREADS, 0, s>>>(A, lda, p, B, ldb, q, n, part);
    }
    ASSS_CHECK_LAUNCH();
    k_gram_final<<<cdiv(p * q, 4), 128, 0, s>>>(part, GRAM_BLOCKS, p * q, G);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// out = z - Y w  (Y n x m row-major)
__global__ void k_sub_rowmajor_gemv(const double* __restrict__ Y, int m, const double* __restrict__ w,
                                    const double* z, int n, double* out, const int* skip) {
    extern __shared__ double sw_[];
    if (skip && *skip) return;   // a speculative application the outer method did not need
    for (int t = threadIdx.x; t < m; t += blockDim.x) sw_[t] = w[t];
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* row = Y + (size_t)i * m;
    double acc = 0.0;
    for (int c = 0; c < m; ++c) acc += row[c] * sw_[c];
    out[i] = z[i] - acc;
}

asss_status sub_rowmajor_gemv(const double* Y, int m, const double* w, const double* z, int n, double* out,
                              cudaStream_t s, const int* skip) {
    k_sub_rowmajor_gemv<<<cdiv(n, 256), 256, sizeof(double) * (m > 0 ? m : 1), s>>>(Y, m, w, z, n, out, skip);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// out = A c + beta*out, A n x p column-major
__global__ void k_colmajor_gemv(const double* __restrict__ A, int lda, int p, const double* __restrict__ c, int n,
                                double beta, double* out) {
    extern __shared__ double sc_[];
    for (int t = threadIdx.x; t < p; t += blockDim.x) sc_[t] = c[t];
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int a = 0; a < p; ++a) acc += A[(size_t)a * lda + i] * sc_[a];
    out[i] = (beta == 0.0 ? 0.0 : beta * out[i]) + acc;
}

asss_status colmajor_gemv(const double* A, int lda, int p, const double* c, int n, double beta, double* out,
                          cudaStream_t s) {
    k_colmajor_gemv<<<cdiv(n, 256), 256, sizeof(double) * (p > 0 ? p : 1), s>>>(A, lda, p, c, n, beta, out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// in-place inverse of a row-major m x m matrix: Gauss-Jordan with partial
// pivoting in one block (m is at most a few hundred)
// ---------------------------------------------------------------------------
__global__ void k_gauss_jordan(double* K, double* W, int m, int* perm, int* singular) {
    // W: m x 2m augmented [K | I]
    for (int t = threadIdx.x; t < m * 2 * m; t += blockDim.x) {
        int r = t / (2 * m), c = t % (2 * m);
        W[t] = (c < m) ? K[r * m + c] : (c - m == r ? 1.0 : 0.0);
    }
    __shared__ int s_piv;
    __shared__ double s_best[32];
    __shared__ int s_bidx[32];
    __syncthreads();
    for (int col = 0; col < m; ++col) {
        // pivot search
        double best = -1.0;
        int bi = col;
        for (int r = col + threadIdx.x; r < m; r += blockDim.x) {
            double v = fabs(W[r * 2 * m + col]);
            if (v > best) {
                best = v;
                bi = r;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            s_best[threadIdx.x >> 5] = best;
            s_bidx[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int idx = col;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (s_best[w] > b || (s_best[w] == b && s_bidx[w] < idx)) {
                    b = s_best[w];
                    idx = s_bidx[w];
                }
            s_piv = idx;
            if (b <= 0.0) *singular = 1;
        }
        __syncthreads();
        int pr = s_piv;
        if (pr != col) {
            for (int c = threadIdx.x; c < 2 * m; c += blockDim.x) {
                double a = W[col * 2 * m + c];
                W[col * 2 * m + c] = W[pr * 2 * m + c];
                W[pr * 2 * m + c] = a;
            }
        }
        __syncthreads();
        double pv = W[col * 2 * m + col];
        __syncthreads();
        if (pv != 0.0) {
            for (int c = threadIdx.x; c < 2 * m; c += blockDim.x) W[col * 2 * m + c] /= pv;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m * 2 * m; t += blockDim.x) {
            int r = t / (2 * m), c = t % (2 * m);
            if (r == col) continue;
            double f = W[r * 2 * m + col];
            if (c != col) W[t] -= f * W[col * 2 * m + c];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            if (r != col) W[r * 2 * m + col] = 0.0;
        __syncthreads();
    }
    (void)perm;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        int r = t / m, c = t % m;
        K[t] = W[r * 2 * m + m + c];
    }
}

asss_status small_inverse(double* K, int m, int* singular, cudaStream_t s) {
    if (m == 0) return ASSS_OK;
    DBuf<double> W;
    DBuf<int> sg;
    ASSS_TRY(W.alloc((int64_t)2 * m * m));
    ASSS_TRY(sg.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(sg.p, 0, sizeof(int), s));
    k_gauss_jordan<<<1, 1024, 0, s>>>(K, W.p, m, nullptr, sg.p);
    ASSS_CHECK_LAUNCH();
    int h = 0;
    ASSS_CUDA(cudaMemcpyAsync(&h, sg.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (singular) *singular = h;
    return ASSS_OK;
}

// col-major n x p -> row-major n x kp (zero padded)
template <class T>
__global__ void k_to_rowmajor(const double* A, int lda, int p, int n, int kp, T* out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * kp) return;
    int i = (int)(t / kp), a = (int)(t % kp);
    out[t] = (a < p) ? (T)A[(size_t)a * lda + i] : (T)0;
}

asss_status to_rowmajor(const double* A, int lda, int p, int n, int kp, double* out, cudaStream_t s) {
    if (kp == 0) return ASSS_OK;
    k_to_rowmajor<double><<<cdiv((int64_t)n * kp, 256), 256, 0, s>>>(A, lda, p, n, kp, out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}
asss_status to_rowmajor_f(const double* A, int lda, int p, int n, int kp, float* out, cudaStream_t s) {
    if (kp == 0) return ASSS_OK;
    k_to_rowmajor<float><<<cdiv((int64_t)n * kp, 256), 256, 0, s>>>(A, lda, p, n, kp, out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// vector helpers
// ---------------------------------------------------------------------------
__global__ void k_vscale(double* y, const double* x, double a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}
__global__ void k_vaxpy(double* y, const double* x, double a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}
__global__ void k_vaxpy_dev(double* y, const double* x, const double* a, double sign, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += sign * (*a) * x[i];
}
__global__ void k_vmul(double* y, const double* a, const double* b, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] * b[i];
}
__global__ void k_vfill(double* y, double v, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = v;
}

asss_status vscale(double* y, const double* x, double a, int n, cudaStream_t s) {
    k_vscale<<<cdiv(n, 256), 256, 0, s>>>(y, x, a, n);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}
asss_status vaxpy(double* y, const double* x, double a, int n, cudaStream_t s) {
    k_vaxpy<<<cdiv(n, 256), 256, 0, s>>>(y, x, a, n);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}
asss_status vaxpy_dev(double* y, const double* x, const double* a, double sign, int n, cudaStream_t s) {
    k_vaxpy_dev<<<cdiv(n, 256), 256, 0, s>>>(y, x, a, sign, n);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}
asss_status vmul(double* y, const double* a, const double* b, int n, cudaStream_t s) {
    k_vmul<<<cdiv(n, 256), 256, 0, s>>>(y, a, b, n);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}
asss_status vcopy(double* y, const double* x, int n, cudaStream_t s) {
    ASSS_CUDA(cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return ASSS_OK;
}
asss_status vfill(double* y, double v, int n, cudaStream_t s) {
    k_vfill<<<cdiv(n, 256), 256, 0, s>>>(y, v, n);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

}  // namespace asss
