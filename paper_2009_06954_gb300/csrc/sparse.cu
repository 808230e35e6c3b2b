// Sparse-matrix plumbing: CSR upload/validation, transpose, SpMV, the pattern of
// Abar S + (Abar S)^T, SELL-C conversion, scans and deterministic dot products.
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asss {

// ---------------------------------------------------------------------------
// error text
// ---------------------------------------------------------------------------
static thread_local char g_err[1024] = {0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

// The dynamic shared-memory limit is an attribute of the kernel for the whole process, and
// set-ups may run on several host threads at once: the limit only ever grows (under a
// lock), so a launch sized for it never finds it lowered by another thread.
asss_status raise_dynamic_smem(const void* func, int bytes) {
    static std::mutex mu;
    static std::vector<std::tuple<const void*, int, int>> set;   // (kernel, device, limit)
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    ASSS_CUDA(cudaGetDevice(&dev));
    for (auto& f : set) {
        if (std::get<0>(f) == func && std::get<1>(f) == dev) {
            if (std::get<2>(f) >= bytes) return ASSS_OK;
            ASSS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            std::get<2>(f) = bytes;
            return ASSS_OK;
        }
    }
    ASSS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    set.emplace_back(func, dev, bytes);
    return ASSS_OK;
}

static unsigned long long g_launches = 0;
void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
unsigned long long launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

constexpr int SCRATCH_MAXDEV = 64, SCRATCH_SLOTS = 4;
static thread_local double* g_scratch[SCRATCH_MAXDEV][SCRATCH_SLOTS] = {};
static thread_local int64_t g_scratch_cap[SCRATCH_MAXDEV][SCRATCH_SLOTS] = {};

void release_thread_scratch() {
    for (int d = 0; d < SCRATCH_MAXDEV; ++d)
        for (int s = 0; s < SCRATCH_SLOTS; ++s)
            if (g_scratch[d][s]) {
                cudaFree(g_scratch[d][s]);
                g_scratch[d][s] = nullptr;
                g_scratch_cap[d][s] = 0;
            }
}

asss_status process_scratch(int slot, int64_t count, double** out) {
    constexpr int MAXDEV = SCRATCH_MAXDEV, SLOTS = SCRATCH_SLOTS;
    auto& buf = g_scratch;
    auto& cap = g_scratch_cap;
    int dev = 0;
    ASSS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAXDEV || slot < 0 || slot >= SLOTS) {
        set_error("scratch slot out of range");
        return ASSS_ERR_ARG;
    }
    if (cap[dev][slot] < count) {
        if (buf[dev][slot]) cudaFree(buf[dev][slot]);
        buf[dev][slot] = nullptr;
        cap[dev][slot] = 0;
        ASSS_CUDA(cudaMalloc((void**)&buf[dev][slot], sizeof(double) * (size_t)count));
        cap[dev][slot] = count;
    }
    *out = buf[dev][slot];
    return ASSS_OK;
}

asss_status make_ctx(Ctx& c, void* stream, double wait_timeout_ms) {
    c.stream = (cudaStream_t)stream;
    ASSS_CUDA(cudaGetDevice(&c.device));
    ASSS_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, c.device));
    ASSS_CUDA(cudaDeviceGetAttribute(&c.clock_khz, cudaDevAttrClockRate, c.device));
    if (c.clock_khz <= 0) c.clock_khz = 2000000;
    double ms = wait_timeout_ms > 0 ? wait_timeout_ms : 2000.0;
    // clock64 counts SM cycles; use the maximum clock so the budget is an upper bound in time
    c.wait_cycles = (long long)(ms * (double)c.clock_khz);
    int l2 = 0;
    ASSS_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c.device));
    c.l2_bytes = l2;
    const char* fe = getenv("ASSS_FORCE_EVICT_FIRST");
    c.force_stream = fe && fe[0] == '1';
    return ASSS_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long block_excl_scan_1024(long long v, long long* total) {
    __shared__ long long ws[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long y = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        ws[lane] = y;
    }
    __syncthreads();
    long long add = warp > 0 ? ws[warp - 1] : 0;
    *total = ws[31];
    long long r = x + add - v;
    __syncthreads();
    return r;
}

template <class TO>
__global__ void k_scan1(const int* in, TO* out, long long* bsum, int n) {
    int i = blockIdx.x * 1024 + threadIdx.x;
    long long v = (i < n) ? (long long)in[i] : 0;
    long long tot;
    long long ex = block_excl_scan_1024(v, &tot);
    if (i < n) out[i] = (TO)ex;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan2(long long* bsum, int nb, long long* total) {
    long long carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        long long v = (i < nb) ? bsum[i] : 0;
        long long tot;
        long long ex = block_excl_scan_1024(v, &tot);
        if (i < nb) bsum[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <class TO>
__global__ void k_scan3(TO* out, const long long* bsum, int n, const long long* total) {
    int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += (TO)bsum[blockIdx.x];
    if (i == 0) out[n] = (TO)(*total);
}

template <class TO>
static asss_status scan_impl(const int* cnt, TO* out, int n, long long* total_h, cudaStream_t s) {
    int nb = cdiv(n, 1024);
    if (nb == 0) nb = 1;
    DBuf<long long> bsum;
    ASSS_TRY(bsum.alloc(nb + 1));
    k_scan1<TO><<<nb, 1024, 0, s>>>(cnt, out, bsum.p, n);
    ASSS_CHECK_LAUNCH();
    k_scan2<<<1, 1024, 0, s>>>(bsum.p, nb, bsum.p + nb);
    ASSS_CHECK_LAUNCH();
    k_scan3<TO><<<nb, 1024, 0, s>>>(out, bsum.p, n, bsum.p + nb);
    ASSS_CHECK_LAUNCH();
    if (total_h) {
        ASSS_CUDA(cudaMemcpyAsync(total_h, bsum.p + nb, sizeof(long long), cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
    }
    return ASSS_OK;
}

asss_status exclusive_scan(const int* cnt, int* out, int n, int64_t* total, cudaStream_t s) {
    long long t = 0;
    ASSS_TRY(scan_impl<int>(cnt, out, n, &t, s));
    if (t >= (1LL << 31) - 1) {
        set_error("scan total %lld exceeds the 32-bit index range", t);
        return ASSS_ERR_UNSUPPORTED;
    }
    if (total) *total = t;
    return ASSS_OK;
}

asss_status exclusive_scan64(const int* cnt, long long* out, int n, long long* total, cudaStream_t s) {
    return scan_impl<long long>(cnt, out, n, total, s);
}

// ---------------------------------------------------------------------------
// deterministic dot products: fixed grid, per-block partials, ordered final sum
// ---------------------------------------------------------------------------
constexpr int DOT_BLOCKS = 296;
constexpr int DOT_THREADS = 512;

template <class T>
__global__ void k_dot_partial(const T* a, const T* b, int n, double* part) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    __shared__ double sw[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void k_sum_partials(const double* part, int np, double* out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += 32) acc += part[i];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

template <class T>
static asss_status dot_impl(const T* a, const T* b, int n, double* d_out, cudaStream_t s) {
    double* part = nullptr;
    ASSS_TRY(process_scratch(0, DOT_BLOCKS, &part));
    k_dot_partial<T><<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(a, b, n, part);
    ASSS_CHECK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(part, DOT_BLOCKS, d_out);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

asss_status dot(const double* a, const double* b, int n, double* d_out, cudaStream_t s) {
    return dot_impl<double>(a, b, n, d_out, s);
}
asss_status dot_f(const float* a, const float* b, int n, double* d_out, cudaStream_t s) {
    return dot_impl<float>(a, b, n, d_out, s);
}

// ---------------------------------------------------------------------------
// CSR upload and validation
// ---------------------------------------------------------------------------
__global__ void k_rowptr_check(const long long* rp64, int* rp32, int n, long long nnz, int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    long long v = rp64[i];
    if (i == 0 && v != 0) atomicOr(flag, 1);
    if (i == n && v != nnz) atomicOr(flag, 1);
    if (i < n && rp64[i + 1] < v) atomicOr(flag, 1);
    rp32[i] = (int)v;
}

__global__ void k_col_check(const int* rp, const int* ci, int n, int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int prev = -1;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int c = ci[e];
        if (c < 0 || c >= n || c <= prev) {
            atomicOr(flag, 2);
            return;
        }
        prev = c;
    }
}

asss_status upload_csr(const asss_csr* A, DCsr& out, bool need_values, cudaStream_t s) {
    if (!A || A->n <= 0 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && !A->col_idx)) {
        set_error("invalid CSR argument");
        return ASSS_ERR_ARG;
    }
    if (A->n >= (1LL << 31) - 1 || A->nnz >= (1LL << 31) - 1) {
        set_error("n or nnz beyond the 32-bit index range of this build");
        return ASSS_ERR_UNSUPPORTED;
    }
    if (need_values && A->nnz > 0 && !A->val) {
        set_error("CSR values required");
        return ASSS_ERR_ARG;
    }
    int n = (int)A->n, nnz = (int)A->nnz;
    out.n = n;
    out.nnz = nnz;
    DBuf<long long> rp64;
    ASSS_TRY(to_device(rp64, (const long long*)A->row_ptr, n + 1, s));
    ASSS_TRY(out.rp.alloc(n + 1));
    ASSS_TRY(to_device(out.ci, A->col_idx, nnz, s));
    if (A->val) ASSS_TRY(to_device(out.v, A->val, nnz, s));
    DBuf<int> flag;
    ASSS_TRY(flag.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    k_rowptr_check<<<cdiv(n + 1, 256), 256, 0, s>>>(rp64.p, out.rp.p, n, (long long)nnz, flag.p);
    ASSS_CHECK_LAUNCH();
    int hflag = 0;
    ASSS_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hflag) {
        set_error("row_ptr is not a valid CSR row pointer");
        return ASSS_ERR_PATTERN;
    }
    k_col_check<<<cdiv(n, 256), 256, 0, s>>>(out.rp.p, out.ci.p, n, flag.p);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hflag) {
        set_error("column indices out of range, unsorted or duplicated within a row");
        return ASSS_ERR_PATTERN;
    }
    return ASSS_OK;
}

asss_status copy_csr(const DCsr& a, DCsr& out, cudaStream_t s) {
    out.n = a.n;
    out.nnz = a.nnz;
    ASSS_TRY(out.rp.alloc(a.n + 1));
    ASSS_TRY(out.ci.alloc(a.nnz));
    ASSS_CUDA(cudaMemcpyAsync(out.rp.p, a.rp.p, sizeof(int) * (a.n + 1), cudaMemcpyDeviceToDevice, s));
    ASSS_CUDA(cudaMemcpyAsync(out.ci.p, a.ci.p, sizeof(int) * a.nnz, cudaMemcpyDeviceToDevice, s));
    if (a.v.p) {
        ASSS_TRY(out.v.alloc(a.nnz));
        ASSS_CUDA(cudaMemcpyAsync(out.v.p, a.v.p, sizeof(double) * a.nnz, cudaMemcpyDeviceToDevice, s));
    }
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// transpose (rows of the result sorted by column; deterministic)
// ---------------------------------------------------------------------------
__global__ void k_count_cols(const int* ci, int nnz, int* cnt) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(&cnt[ci[e]], 1);
}

__global__ void k_scatter_t(const int* rp, const int* ci, const double* v, int n, const int* rpT,
                            int* fill, int* ciT, double* vT, int* srcpos) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int c = ci[e];
        int pos = rpT[c] + atomicAdd(&fill[c], 1);
        ciT[pos] = i;
        if (v) vT[pos] = v[e];
        if (srcpos) srcpos[pos] = e;
    }
}

__global__ void k_sort_rows(const int* rp, int n, int* ci, double* v, int* aux) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = rp[i], e = rp[i + 1];
    for (int a = b + 1; a < e; ++a) {
        int key = ci[a];
        double kv = v ? v[a] : 0.0;
        int ka = aux ? aux[a] : 0;
        int t = a - 1;
        while (t >= b && ci[t] > key) {
            ci[t + 1] = ci[t];
            if (v) v[t + 1] = v[t];
            if (aux) aux[t + 1] = aux[t];
            --t;
        }
        ci[t + 1] = key;
        if (v) v[t + 1] = kv;
        if (aux) aux[t + 1] = ka;
    }
}

asss_status transpose_csr(const DCsr& a, DCsr& t, DBuf<int>* srcpos, cudaStream_t s) {
    int n = a.n, nnz = a.nnz;
    t.n = n;
    t.nnz = nnz;
    DBuf<int> cnt, fill;
    ASSS_TRY(cnt.alloc(n));
    ASSS_TRY(fill.alloc(n));
    ASSS_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * n, s));
    ASSS_CUDA(cudaMemsetAsync(fill.p, 0, sizeof(int) * n, s));
    if (nnz) k_count_cols<<<cdiv(nnz, 256), 256, 0, s>>>(a.ci.p, nnz, cnt.p);
    ASSS_CHECK_LAUNCH();
    ASSS_TRY(t.rp.alloc(n + 1));
    ASSS_TRY(exclusive_scan(cnt.p, t.rp.p, n, nullptr, s));
    ASSS_TRY(t.ci.alloc(nnz));
    if (a.v.p) ASSS_TRY(t.v.alloc(nnz));
    if (srcpos) ASSS_TRY(srcpos->alloc(nnz));
    k_scatter_t<<<cdiv(n, 256), 256, 0, s>>>(a.rp.p, a.ci.p, a.v.p, n, t.rp.p, fill.p, t.ci.p, t.v.p,
                                              srcpos ? srcpos->p : nullptr);
    ASSS_CHECK_LAUNCH();
    k_sort_rows<<<cdiv(n, 128), 128, 0, s>>>(t.rp.p, n, t.ci.p, t.v.p, srcpos ? srcpos->p : nullptr);
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// CSR SpMV (FP64): y = A x, LANES threads per row
// ---------------------------------------------------------------------------
template <int LANES>
__global__ void k_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ v, const double* __restrict__ x,
                       double* __restrict__ y, const double* __restrict__ lscale) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int row = gt / LANES;
    int sub = gt % LANES;
    // no early exit: every lane of the warp takes part in the shuffles below
    const bool live = row < n;
    double acc = 0.0;
    if (live)
        for (int e = rp[row] + sub; e < rp[row + 1]; e += LANES) acc += v[e] * __ldg(&x[ci[e]]);
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, LANES);
    if (live && sub == 0) y[row] = lscale ? lscale[row] * acc : acc;
}

// ---------------------------------------------------------------------------
// diagonal storage for stencil-like FP64 matrices: one thread per row, the
// diagonals read with unit stride (no column indices), offsets in shared memory
// ---------------------------------------------------------------------------
constexpr int DIA_MAX = 16;

// Every diagonal of a row is unrolled (ND >= ndiag, the extra ones predicated off), so
// the loads of a row - all its values, then all its x entries - are in flight together
// and the FP64 FMAs (the pipe this product shares with its loads on GB300) issue as soon
// as they land.
template <int ND, bool EF>
__global__ void __launch_bounds__(256) k_dia_spmv(int n, int ndiag, const int* __restrict__ off,
                                                  const double* __restrict__ val, const double* __restrict__ x,
                                                  double* __restrict__ y, const double* __restrict__ lscale) {
    __shared__ int s_off[ND];
    if (threadIdx.x < ND) s_off[threadIdx.x] = threadIdx.x < ndiag ? off[threadIdx.x] : 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[ND], xv[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const int j = i + s_off[d];
        const bool in = d < ndiag && j >= 0 && j < n;
        const double* vp = &val[(size_t)d * n + i];
        v[d] = in ? (EF ? __ldcs(vp) : __ldg(vp)) : 0.0;
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const int j = i + s_off[d];
        const bool in = d < ndiag && j >= 0 && j < n;
        xv[d] = in ? __ldg(&x[j]) : 0.0;
    }
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) acc += v[d] * xv[d];
    y[i] = lscale ? lscale[i] * acc : acc;
}

__global__ void k_dia_offsets(int n, const int* rp, const int* ci, unsigned* bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const unsigned b = (unsigned)(ci[e] - i + n - 1);  // 0 .. 2n-2
        atomicOr(&bits[b >> 5], 1u << (b & 31));
    }
}

__global__ void k_dia_fill(int n, const int* rp, const int* ci, const double* v, const int* off, int ndiag,
                           double* val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int o = ci[e] - i;
        int lo = 0, hi = ndiag - 1;
        while (lo < hi) {
            const int mid = lo + ((hi - lo) >> 1);   // no overflow for offsets near 2^31
            if (off[mid] < o) lo = mid + 1;
            else hi = mid;
        }
        val[(size_t)lo * n + i] = v[e];  // every offset of A is in the list
    }
}

asss_status attach_dia(DCsr& A, int max_diag, double min_fill, int* ok, cudaStream_t s) {
    *ok = A.dia.ndiag > 0;
    if (A.dia.tried) return ASSS_OK;
    A.dia.tried = true;
    const int n = A.n;
    if (n < 1 || !A.v.p || A.nnz < 1 || max_diag > DIA_MAX) return ASSS_OK;
    const long long nbits = 2LL * n - 1;
    const int words = (int)((nbits + 31) / 32);
    DBuf<unsigned> bits;
    ASSS_TRY(bits.alloc(words));
    ASSS_CUDA(cudaMemsetAsync(bits.p, 0, sizeof(unsigned) * words, s));
    k_dia_offsets<<<cdiv(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, bits.p);
    ASSS_CHECK_LAUNCH();
    std::vector<unsigned> hb(words);
    ASSS_CUDA(cudaMemcpyAsync(hb.data(), bits.p, sizeof(unsigned) * words, cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    std::vector<int> off;
    for (int w = 0; w < words; ++w) {
        unsigned b = hb[w];
        while (b) {
            const int t = __builtin_ctz(b);
            off.push_back(w * 32 + t - (n - 1));
            b &= b - 1;
            if ((int)off.size() > max_diag) return ASSS_OK;
        }
    }
    double stored = 0.0;
    for (int o : off) stored += (double)(n - (o < 0 ? -o : o));
    if ((double)A.nnz < min_fill * stored) return ASSS_OK;
    ASSS_TRY(to_device(A.dia.off, off.data(), (int64_t)off.size(), s));
    ASSS_TRY(A.dia.val.alloc((int64_t)off.size() * n));
    ASSS_CUDA(cudaMemsetAsync(A.dia.val.p, 0, sizeof(double) * off.size() * (size_t)n, s));
    k_dia_fill<<<cdiv(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, A.dia.off.p, (int)off.size(), A.dia.val.p);
    ASSS_CHECK_LAUNCH();
    A.dia.ndiag = (int)off.size();
    // the outer operator applies two such products back to back
    int dev = 0, l2 = 0;
    ASSS_CUDA(cudaGetDevice(&dev));
    ASSS_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const char* fe = getenv("ASSS_FORCE_EVICT_FIRST");
    A.dia.stream = (fe && fe[0] == '1') || 2LL * (long long)off.size() * n * (long long)sizeof(double) > (long long)l2 * 3 / 4;
    *ok = 1;
    return ASSS_OK;
}

asss_status spmv(const DCsr& A, const double* x, double* y, const double* lscale, cudaStream_t s) {
    int n = A.n;
    if (A.dia.ndiag > 0) {
        const int nb = cdiv(n, 256);
        const bool ef = A.dia.stream != 0;
        if (A.dia.ndiag <= 8) {
            if (ef) k_dia_spmv<8, true><<<nb, 256, 0, s>>>(n, A.dia.ndiag, A.dia.off.p, A.dia.val.p, x, y, lscale);
            else k_dia_spmv<8, false><<<nb, 256, 0, s>>>(n, A.dia.ndiag, A.dia.off.p, A.dia.val.p, x, y, lscale);
        } else {
            if (ef) k_dia_spmv<DIA_MAX, true><<<nb, 256, 0, s>>>(n, A.dia.ndiag, A.dia.off.p, A.dia.val.p, x, y, lscale);
            else k_dia_spmv<DIA_MAX, false><<<nb, 256, 0, s>>>(n, A.dia.ndiag, A.dia.off.p, A.dia.val.p, x, y, lscale);
        }
        ASSS_CHECK_LAUNCH();
        return ASSS_OK;
    }
    double mean = n ? (double)A.nnz / n : 0;
    int threads = 256;
    if (mean <= 6) {
        k_spmv<1><<<cdiv(n, threads), threads, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, x, y, lscale);
    } else if (mean <= 12) {
        k_spmv<2><<<cdiv((int64_t)n * 2, threads), threads, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, x, y, lscale);
    } else if (mean <= 24) {
        k_spmv<4><<<cdiv((int64_t)n * 4, threads), threads, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, x, y, lscale);
    } else if (mean <= 64) {
        k_spmv<8><<<cdiv((int64_t)n * 8, threads), threads, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, x, y, lscale);
    } else {
        k_spmv<32><<<cdiv((int64_t)n * 32, threads), threads, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, x, y, lscale);
    }
    ASSS_CHECK_LAUNCH();
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// the symmetric pattern P = pat(Abar S) + pat(Abar S)^T (+ diagonal), row by row:
// row i of P = {i} u U_{l in Abar_i} S_l u U_{l in S^T_i} Abar^T_l
// One warp per row gathers the candidates into shared memory, sorts them
// (bitonic network) and keeps the distinct values.
// ---------------------------------------------------------------------------
__global__ void k_pattern_cand_count(int n, const int* arp, const int* aci, const int* srp,
                                     const int* strp, const int* stci, const int* atrp, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 1;
    for (int e = arp[i]; e < arp[i + 1]; ++e) {
        int l = aci[e];
        c += srp[l + 1] - srp[l];
    }
    for (int e = strp[i]; e < strp[i + 1]; ++e) {
        int l = stci[e];
        c += atrp[l + 1] - atrp[l];
    }
    cnt[i] = c;
}

__global__ void k_max_int(const int* a, int n, int* out) {
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

constexpr int PAT_WARPS = 4;

__global__ void k_pattern_rows(int n, const int* arp, const int* aci, const int* srp, const int* sci,
                               const int* strp, const int* stci, const int* atrp, const int* atci,
                               int cap, const int* cand, const int* prp, int* counts, int* pci, int* chk) {
    extern __shared__ int smem[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* buf = smem + warp * cap;
    for (int i = blockIdx.x * PAT_WARPS + warp; i < n; i += gridDim.x * PAT_WARPS) {
        if (cand[i] > cap) continue;  // a heavy row: k_pattern_heavy handles it
        int pos = 0;
        if (lane == 0) buf[0] = i;
        pos = 1;
        for (int e = arp[i]; e < arp[i + 1]; ++e) {
            int l = aci[e];
            int b = srp[l], len = srp[l + 1] - b;
            for (int t = lane; t < len; t += 32) buf[pos + t] = sci[b + t];
            pos += len;
        }
        for (int e = strp[i]; e < strp[i + 1]; ++e) {
            int l = stci[e];
            int b = atrp[l], len = atrp[l + 1] - b;
            for (int t = lane; t < len; t += 32) buf[pos + t] = atci[b + t];
            pos += len;
        }
        int p2 = 32;
        while (p2 < pos) p2 <<= 1;
        for (int t = pos + lane; t < p2; t += 32) buf[t] = 0x7fffffff;
        __syncwarp();
        for (int size = 2; size <= p2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < (p2 >> 1); t += 32) {
                    int lo = 2 * stride * (t / stride) + (t % stride);
                    int hi = lo + stride;
                    bool up = ((lo & size) == 0);
                    int a = buf[lo], bb = buf[hi];
                    if ((a > bb) == up) {
                        buf[lo] = bb;
                        buf[hi] = a;
                    }
                }
                __syncwarp();
            }
        }
        int base = prp ? prp[i] : 0;
        const int end = prp ? prp[i + 1] : 0;
        int written = 0;
        for (int t0 = 0; t0 < pos; t0 += 32) {
            int t = t0 + lane;
            bool u = (t < pos) && (t == 0 || buf[t] != buf[t - 1]);
            unsigned m = __ballot_sync(0xffffffffu, u);
            if (pci && u) {
                // checked write: a row never writes past its own range
                const int at = base + written + __popc(m & ((1u << lane) - 1u));
                if (at < end) pci[at] = buf[t];
                else atomicOr(chk, 1);
            }
            written += __popc(m);
        }
        if (counts && lane == 0) counts[i] = written;
        if (pci && lane == 0 && base + written != end) atomicOr(chk, 8);
        __syncwarp();
    }
}

// Rows whose candidates do not fit the shared-memory sort: one block per row marks
// the candidate columns in a bitmap of n bits (global scratch, one per block), then
// counts them or writes them in ascending order (a block prefix sum over words).
constexpr int PATH_THREADS = 512;

__global__ void __launch_bounds__(PATH_THREADS) k_pattern_heavy(
    int n, const int* heavy, int nheavy, const int* arp, const int* aci, const int* srp, const int* sci,
    const int* strp, const int* stci, const int* atrp, const int* atci, unsigned* bitmaps, int words,
    const int* prp, int* counts, int* pci, int* chk) {
    __shared__ int s_warp[PATH_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = PATH_THREADS / 32;
    unsigned* bm = bitmaps + (size_t)blockIdx.x * words;
    const int per = (words + PATH_THREADS - 1) / PATH_THREADS;
    const int w0 = min(words, (int)threadIdx.x * per), w1 = min(words, w0 + per);
    for (int h = blockIdx.x; h < nheavy; h += gridDim.x) {
        const int i = heavy[h];
        for (int w = threadIdx.x; w < words; w += PATH_THREADS) bm[w] = 0u;
        __syncthreads();
        if (threadIdx.x == 0) atomicOr(&bm[i >> 5], 1u << (i & 31));
        for (int e = arp[i] + warp; e < arp[i + 1]; e += nw) {
            const int l = aci[e];
            for (int t = srp[l] + lane; t < srp[l + 1]; t += 32) {
                const int c = sci[t];
                atomicOr(&bm[c >> 5], 1u << (c & 31));
            }
        }
        for (int e = strp[i] + warp; e < strp[i + 1]; e += nw) {
            const int l = stci[e];
            for (int t = atrp[l] + lane; t < atrp[l + 1]; t += 32) {
                const int c = atci[t];
                atomicOr(&bm[c >> 5], 1u << (c & 31));
            }
        }
        __syncthreads();
        int cnt = 0;
        for (int w = w0; w < w1; ++w) cnt += __popc(bm[w]);
        // exclusive prefix of cnt over the block (threads own consecutive word ranges)
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int v = lane < nw ? s_warp[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (lane < nw) s_warp[lane] = v;  // inclusive totals per warp
        }
        __syncthreads();
        const int before = (warp > 0 ? s_warp[warp - 1] : 0) + incl - cnt;
        if (counts) {
            if (threadIdx.x == PATH_THREADS - 1) counts[i] = before + cnt;
        } else {
            int pos = prp[i] + before;
            const int end = prp[i + 1];
            for (int w = w0; w < w1; ++w) {
                unsigned bits = bm[w];
                while (bits) {
                    const int t = __ffs(bits) - 1;
                    if (pos < end) pci[pos] = w * 32 + t;   // checked write
                    else atomicOr(chk, 2);
                    ++pos;
                    bits &= bits - 1u;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_mirror(int n, const int* prp, const int* pci, int* mirror, int* diagpos, int* chk) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = prp[i]; k < prp[i + 1]; ++k) {
        int j = pci[k];
        if (j < 0 || j >= n) {   // checked read: a column outside the matrix is recorded, not followed
            atomicOr(chk, 4);
            mirror[k] = -1;
            continue;
        }
        int lo = prp[j], hi = prp[j + 1] - 1, f = -1;
        while (lo <= hi) {
            int mid = lo + ((hi - lo) >> 1);   // no overflow for offsets near 2^31
            int c = pci[mid];
            if (c == i) {
                f = mid;
                break;
            }
            if (c < i) lo = mid + 1;
            else hi = mid - 1;
        }
        mirror[k] = f;
        if (j == i) diagpos[i] = k;
    }
}

asss_status build_pattern(const DCsr& Abar, const DCsr& AbarT, const DCsr& S, const DCsr& ST, DCsr& P,
                          DBuf<int>& mirror, DBuf<int>& diagpos, cudaStream_t s) {
    int n = Abar.n;
    DBuf<int> cnt, mx;
    ASSS_TRY(cnt.alloc(n));
    ASSS_TRY(mx.alloc(1));
    k_pattern_cand_count<<<cdiv(n, 256), 256, 0, s>>>(n, Abar.rp.p, Abar.ci.p, S.rp.p, ST.rp.p, ST.ci.p,
                                                       AbarT.rp.p, cnt.p);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(int), s));
    k_max_int<<<256, 256, 0, s>>>(cnt.p, n, mx.p);
    ASSS_CHECK_LAUNCH();
    int hmax = 0;
    ASSS_CUDA(cudaMemcpyAsync(&hmax, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    // rows with at most PAT_LIGHT candidates are sorted in shared memory by one warp;
    // the rest (power-law rows) go through a bitmap per block
    constexpr int PAT_LIGHT = 8192;
    int cap = 32;
    while (cap < hmax && cap < PAT_LIGHT) cap <<= 1;
    std::vector<int> heavy;
    if (hmax > cap) {
        std::vector<int> hc(n);
        ASSS_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        ASSS_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i)
            if (hc[i] > cap) heavy.push_back(i);
    }
    DBuf<int> cand, hrows, chk;
    DBuf<unsigned> bitmaps;
    ASSS_TRY(chk.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(chk.p, 0, sizeof(int), s));
    const int words = (n + 31) / 32;
    int hblk = 0;
    ASSS_TRY(cand.alloc(n));
    ASSS_CUDA(cudaMemcpyAsync(cand.p, cnt.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    if (!heavy.empty()) {
        ASSS_TRY(to_device(hrows, heavy.data(), (int64_t)heavy.size(), s));
        hblk = (int)heavy.size() < 256 ? (int)heavy.size() : 256;
        ASSS_TRY(bitmaps.alloc((int64_t)hblk * words));
    }
    size_t smem = (size_t)cap * PAT_WARPS * sizeof(int);
    ASSS_TRY(raise_dynamic_smem((const void*)k_pattern_rows, (int)smem));
    int grid = cdiv(n, PAT_WARPS);
    if (grid > 65535 * 8) grid = 65535 * 8;
    k_pattern_rows<<<grid, PAT_WARPS * 32, smem, s>>>(n, Abar.rp.p, Abar.ci.p, S.rp.p, S.ci.p, ST.rp.p,
                                                      ST.ci.p, AbarT.rp.p, AbarT.ci.p, cap, cand.p, nullptr,
                                                      cnt.p, nullptr, chk.p);
    ASSS_CHECK_LAUNCH();
    if (hblk) {
        k_pattern_heavy<<<hblk, PATH_THREADS, 0, s>>>(n, hrows.p, (int)heavy.size(), Abar.rp.p, Abar.ci.p, S.rp.p,
                                                      S.ci.p, ST.rp.p, ST.ci.p, AbarT.rp.p, AbarT.ci.p, bitmaps.p,
                                                      words, nullptr, cnt.p, nullptr, chk.p);
        ASSS_CHECK_LAUNCH();
    }
    P.n = n;
    ASSS_TRY(P.rp.alloc(n + 1));
    int64_t tot = 0;
    ASSS_TRY(exclusive_scan(cnt.p, P.rp.p, n, &tot, s));
    if (tot > 0x7fffffffLL) {
        set_error("the pattern of Abar*S has %lld entries; this build indexes at most 2^31 - 1", (long long)tot);
        return ASSS_ERR_UNSUPPORTED;
    }
    P.nnz = (int)tot;
    ASSS_TRY(P.ci.alloc(tot));
    k_pattern_rows<<<grid, PAT_WARPS * 32, smem, s>>>(n, Abar.rp.p, Abar.ci.p, S.rp.p, S.ci.p, ST.rp.p,
                                                      ST.ci.p, AbarT.rp.p, AbarT.ci.p, cap, cand.p, P.rp.p,
                                                      nullptr, P.ci.p, chk.p);
    ASSS_CHECK_LAUNCH();
    if (hblk) {
        k_pattern_heavy<<<hblk, PATH_THREADS, 0, s>>>(n, hrows.p, (int)heavy.size(), Abar.rp.p, Abar.ci.p, S.rp.p,
                                                      S.ci.p, ST.rp.p, ST.ci.p, AbarT.rp.p, AbarT.ci.p, bitmaps.p,
                                                      words, P.rp.p, nullptr, P.ci.p, chk.p);
        ASSS_CHECK_LAUNCH();
    }
    int hchk = 0;
    ASSS_CUDA(cudaMemcpyAsync(&hchk, chk.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hchk) {
        set_error("pattern of Abar*S: a row's entries disagree with its count (check bits %d)", hchk);
        return ASSS_ERR_CUDA;
    }
    ASSS_TRY(mirror.alloc(tot));
    ASSS_TRY(diagpos.alloc(n));
    k_mirror<<<cdiv(n, 256), 256, 0, s>>>(n, P.rp.p, P.ci.p, mirror.p, diagpos.p, chk.p);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaMemcpyAsync(&hchk, chk.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hchk) {
        set_error("pattern of Abar*S: a column index outside the matrix (check bits %d)", hchk);
        return ASSS_ERR_CUDA;
    }
    return ASSS_OK;
}

// ---------------------------------------------------------------------------
// SELL-C (C = 32) from CSR, optionally leaving out diagonal entries
// ---------------------------------------------------------------------------
// length of each row as stored (the diagonal left out when skip_diag)
__global__ void k_sell_rowlen(int n, const int* rp, const int* ci, int skip_diag, int* len) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int l = rp[r + 1] - rp[r];
    if (skip_diag) {
        for (int e = rp[r]; e < rp[r + 1]; ++e)
            if (ci[e] == r) {
                --l;
                break;
            }
    }
    len[r] = l;
}

// SELL-C-sigma: one block per window of sigma rows sorts (length desc, row asc) with a
// bitonic network in shared memory (each of the 1024 threads holds sigma / 1024 keys;
// sigma a power of two from 1024 to SELL_SIGMA_MAX, the keys in dynamic shared memory)
// and writes slot -> row and row -> slot; slots past the last row map to row n
constexpr int SELL_SORT_THREADS = 1024;
__global__ void __launch_bounds__(SELL_SORT_THREADS) k_sell_sort_window(int n, int nslots, int sigma, const int* len,
                                                                          int* rowmap, int* rowpos) {
    extern __shared__ long long key[];
    const int w0 = blockIdx.x * sigma;
    for (int t = threadIdx.x; t < sigma; t += SELL_SORT_THREADS) {
        const int r = w0 + t;
        // length in the high word (complemented: descending), row in the low word
        key[t] = r < n ? ((long long)(0x7fffffff - len[r]) << 32) | (unsigned)r
                       : ((long long)0x7fffffff << 32) | 0x7fffffffu;
    }
    __syncthreads();
    for (int k = 2; k <= sigma; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < sigma; t += SELL_SORT_THREADS) {
                const int ixj = t ^ j;
                if (ixj > t) {
                    const long long a = key[t], b = key[ixj];
                    const bool up = (t & k) == 0;
                    if ((a > b) == up) {
                        key[t] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < sigma; t += SELL_SORT_THREADS) {
        const int slot = w0 + t;
        if (slot < nslots) {
            const int row = (int)(key[t] & 0xffffffffLL);
            const bool real = row < n;   // the padding key's row word is 0x7fffffff >= n
            rowmap[slot] = real ? row : n;
            if (real) rowpos[row] = slot;
        }
    }
}

__global__ void k_sell_width(int n, const int* len, const int* rowmap, int nslices, int* w, unsigned long long* nnz) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int m = 0;
    long long tot = 0;
    for (int slot = s * 32; slot < s * 32 + 32; ++slot) {
        const int r = rowmap ? rowmap[slot] : slot;
        if (r >= n) continue;
        const int l = len[r];
        m = max(m, l);
        tot += l;
    }
    w[s] = m * 32;
    atomicAdd(nnz, (unsigned long long)tot);
}

template <class T>
__global__ void k_sell_fill(int n, int nslices, const int* rp, const int* ci, const double* v, int skip_diag,
                            const int* rowmap, const int* sptr, int* scol, T* sval) {
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    int s = slot >> 5, lane = slot & 31;
    if (s >= nslices) return;
    const int r = rowmap ? rowmap[slot] : slot;
    int base = sptr[s], width = (sptr[s + 1] - base) >> 5;
    int kk = 0;
    if (r < n) {
        for (int e = rp[r]; e < rp[r + 1]; ++e) {
            if (skip_diag && ci[e] == r) continue;
            scol[base + kk * 32 + lane] = ci[e];
            sval[base + kk * 32 + lane] = (T)v[e];
            ++kk;
        }
    }
    int pad = r < n ? r : 0;
    for (; kk < width; ++kk) {
        scol[base + kk * 32 + lane] = pad;
        sval[base + kk * 32 + lane] = (T)0;
    }
}

// Slices of 32 rows in natural order; when that pads the stored entries by more than
// a fifth over the matrix's own (heavy-tailed row lengths), SELL-C-sigma instead (sigma:
// the window in rows, a power of two from 1024 to SELL_SIGMA_MAX; 0: SELL_SIGMA).  Slices
// wider than `split` entries per lane become several work units (0: SELL_SPLIT).
template <class T>
asss_status build_sell(const DCsr& A, bool skip_diag, DSell<T>& out, cudaStream_t s, int sigma, int split) {
    if (sigma <= 0) sigma = SELL_SIGMA;
    if (split <= 0) split = SELL_SPLIT;
    if (sigma < 1024 || sigma > SELL_SIGMA_MAX || (sigma & (sigma - 1))) {
        set_error("SELL-C-sigma window %d is not a power of two in [1024, %d]", sigma, SELL_SIGMA_MAX);
        return ASSS_ERR_ARG;
    }
    if (split < 64) {
        set_error("SELL-C work unit of %d entries per lane is below 64", split);
        return ASSS_ERR_ARG;
    }
    out.sigma = 0;
    out.split = split;
    out.rowmap.free();
    out.rowpos.free();
    int n = A.n;
    int ns = cdiv(n, 32);
    out.n = n;
    out.nslices = ns;
    DBuf<int> w, len;
    DBuf<unsigned long long> cnt;
    ASSS_TRY(w.alloc(ns));
    ASSS_TRY(len.alloc(n > 0 ? n : 1));
    ASSS_TRY(cnt.alloc(1));
    k_sell_rowlen<<<cdiv(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, skip_diag ? 1 : 0, len.p);
    ASSS_CHECK_LAUNCH();
    long long tot = 0;
    unsigned long long hn = 0;
    DBuf<long long> off64;
    ASSS_TRY(off64.alloc(ns + 1));
    for (int pass = 0; pass < 2; ++pass) {
        const int* rmap = pass ? out.rowmap.p : nullptr;
        ASSS_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
        k_sell_width<<<cdiv(ns, 128), 128, 0, s>>>(n, len.p, rmap, ns, w.p, cnt.p);
        ASSS_CHECK_LAUNCH();
        ASSS_CUDA(cudaMemcpyAsync(&hn, cnt.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
        ASSS_TRY(exclusive_scan64(w.p, off64.p, ns, &tot, s));   // 64-bit total (synchronises)
        if (pass == 1 || (double)tot <= 1.2 * (double)hn) break;
        // heavy-tailed rows: sort each window of sigma rows by length
        const int nslots = ns * 32;
        ASSS_TRY(out.rowmap.alloc(nslots));
        ASSS_TRY(out.rowpos.alloc(n));
        const size_t smem = sizeof(long long) * (size_t)sigma;
        ASSS_TRY(raise_dynamic_smem((const void*)k_sell_sort_window, (int)smem));
        k_sell_sort_window<<<cdiv(nslots, sigma), SELL_SORT_THREADS, smem, s>>>(n, nslots, sigma, len.p,
                                                                                out.rowmap.p, out.rowpos.p);
        ASSS_CHECK_LAUNCH();
        out.sigma = sigma;
    }
    out.nnz = (int64_t)hn;
    out.nstored = tot;
    if (tot >= (1LL << 31) - 1) {
        set_error("SELL-C storage of %lld entries exceeds 32-bit slice offsets", tot);
        return ASSS_ERR_UNSUPPORTED;
    }
    ASSS_TRY(out.sptr.alloc(ns + 1));
    ASSS_TRY(exclusive_scan(w.p, out.sptr.p, ns, nullptr, s));
    ASSS_TRY(out.col.alloc(tot > 0 ? tot : 1));
    ASSS_TRY(out.val.alloc(tot > 0 ? tot : 1));
    k_sell_fill<T><<<cdiv((int64_t)ns * 32, 256), 256, 0, s>>>(n, ns, A.rp.p, A.ci.p, A.v.p, skip_diag ? 1 : 0,
                                                               out.rowmap.p, out.sptr.p, out.col.p, out.val.p);
    ASSS_CHECK_LAUNCH();
    // work units: slices longer than `split` entries per lane are cut into parts
    std::vector<int> hsp(ns + 1);
    ASSS_CUDA(cudaMemcpyAsync(hsp.data(), out.sptr.p, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    std::vector<int4> units;
    std::vector<int> uoff(ns + 1);
    int nheavy = 0;
    units.reserve(ns + 64);
    for (int sl = 0; sl < ns; ++sl) {
        uoff[sl] = (int)units.size();
        const int width = (hsp[sl + 1] - hsp[sl]) >> 5;
        const int np = width > split ? (width + split - 1) / split : 1;
        const int hidx = np > 1 ? nheavy++ : -1;
        for (int pt = 0; pt < np; ++pt) units.push_back(make_int4(sl, pt, np, hidx));
    }
    uoff[ns] = (int)units.size();
    out.nunits = (int)units.size();
    out.nheavy = nheavy;
    ASSS_TRY(to_device(out.units, units.data(), (int64_t)units.size(), s));
    ASSS_TRY(to_device(out.uoff, uoff.data(), (int64_t)ns + 1, s));
    out.hacc.free();
    out.hcnt.free();
    if (nheavy) {
        ASSS_TRY(out.hacc.alloc((int64_t)nheavy * 32));
        ASSS_TRY(out.hcnt.alloc(nheavy));
        ASSS_CUDA(cudaMemsetAsync(out.hacc.p, 0, sizeof(T) * 32 * (size_t)nheavy, s));
        ASSS_CUDA(cudaMemsetAsync(out.hcnt.p, 0, sizeof(unsigned) * (size_t)nheavy, s));
    }
    ASSS_CUDA(cudaStreamSynchronize(s));
    return ASSS_OK;
}

template asss_status build_sell<double>(const DCsr&, bool, DSell<double>&, cudaStream_t, int, int);
template asss_status build_sell<float>(const DCsr&, bool, DSell<float>&, cudaStream_t, int, int);

}  // namespace asss

namespace asss {

// ---------------------------------------------------------------------------
// skew half-diagonal storage
// ---------------------------------------------------------------------------
// exact skew check (J_ij == -J_ji bit for bit, zero diagonal) and the offset set
__global__ void k_skew_offsets(int n, const int* rp, const int* ci, const double* v, unsigned* bits,
                               unsigned long long* nup, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long cnt = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int j = ci[e];
        if (j == i) {
            if (v[e] != 0.0) atomicOr(bad, 1);
            continue;
        }
        // mirror entry
        int lo = rp[j], hi = rp[j + 1] - 1, f = -1;
        while (lo <= hi) {
            int mid = lo + ((hi - lo) >> 1);   // no overflow for offsets near 2^31
            int c = ci[mid];
            if (c == i) {
                f = mid;
                break;
            }
            if (c < i) lo = mid + 1;
            else hi = mid - 1;
        }
        double mv = f >= 0 ? v[f] : 0.0;
        if (mv != -v[e]) atomicOr(bad, 1);
        if (j > i) {
            int off = j - i;
            atomicOr(&bits[off >> 5], 1u << (off & 31));
            ++cnt;
        }
    }
    if (cnt) atomicAdd(nup, (unsigned long long)cnt);
}

template <class T>
__global__ void k_fill_dia(int n, const int* rp, const int* ci, const double* v, const int* off, int ndiag,
                           int64_t ustride, T* U) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int j = ci[e];
        if (j <= i) continue;
        int m = j - i;
        int lo = 0, hi = ndiag - 1;
        while (lo < hi) {
            int mid = lo + ((hi - lo) >> 1);   // no overflow for offsets near 2^31
            if (off[mid] < m) lo = mid + 1;
            else hi = mid;
        }
        U[(size_t)lo * ustride + i] = (T)v[e];
    }
}

template <class T>
asss_status build_skew_dia(const DCsr& J, int max_diag, double min_fill, DSkewDia<T>& out, int* ok, cudaStream_t s) {
    *ok = 0;
    int n = J.n;
    if (n < 2 || !J.v.p) return ASSS_OK;
    int words = (n + 31) / 32;
    DBuf<unsigned> bits;
    DBuf<unsigned long long> nup;
    DBuf<int> bad;
    ASSS_TRY(bits.alloc(words));
    ASSS_TRY(nup.alloc(1));
    ASSS_TRY(bad.alloc(1));
    ASSS_CUDA(cudaMemsetAsync(bits.p, 0, sizeof(unsigned) * words, s));
    ASSS_CUDA(cudaMemsetAsync(nup.p, 0, sizeof(unsigned long long), s));
    ASSS_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_skew_offsets<<<cdiv(n, 256), 256, 0, s>>>(n, J.rp.p, J.ci.p, J.v.p, bits.p, nup.p, bad.p);
    ASSS_CHECK_LAUNCH();
    std::vector<unsigned> hb(words);
    unsigned long long hnup = 0;
    int hbad = 0;
    ASSS_CUDA(cudaMemcpyAsync(hb.data(), bits.p, sizeof(unsigned) * words, cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaMemcpyAsync(&hnup, nup.p, sizeof(hnup), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASSS_CUDA(cudaStreamSynchronize(s));
    if (hbad) return ASSS_OK;  // not exactly skew
    std::vector<int> off;
    for (int w = 0; w < words; ++w) {
        unsigned b = hb[w];
        while (b) {
            int t = __builtin_ctz(b);
            off.push_back(w * 32 + t);
            b &= b - 1;
            if ((int)off.size() > max_diag) return ASSS_OK;
        }
    }
    if (off.empty()) return ASSS_OK;
    double stored = 0.0;
    for (int m : off) stored += (double)(n - m);
    if ((double)hnup < min_fill * stored) return ASSS_OK;
    out.n = n;
    out.ndiag = (int)off.size();
    out.nnz = (int64_t)hnup;
    out.halo = off.back();
    out.ustride = (int64_t)n + out.halo;
    ASSS_TRY(to_device(out.off, off.data(), (int64_t)off.size(), s));
    ASSS_TRY(out.U.alloc((int64_t)out.ndiag * out.ustride));
    ASSS_CUDA(cudaMemsetAsync(out.U.p, 0, sizeof(T) * (size_t)out.ndiag * out.ustride, s));
    k_fill_dia<T><<<cdiv(n, 256), 256, 0, s>>>(n, J.rp.p, J.ci.p, J.v.p, out.off.p, out.ndiag, out.ustride,
                                               out.U.p + out.halo);
    ASSS_CHECK_LAUNCH();
    ASSS_CUDA(cudaStreamSynchronize(s));
    *ok = 1;
    return ASSS_OK;
}

template asss_status build_skew_dia<double>(const DCsr&, int, double, DSkewDia<double>&, int*, cudaStream_t);
template asss_status build_skew_dia<float>(const DCsr&, int, double, DSkewDia<float>&, int*, cudaStream_t);

}  // namespace asss
