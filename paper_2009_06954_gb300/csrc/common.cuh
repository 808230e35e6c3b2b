// Shared device helpers and host-side plumbing for the ASSS library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/asss.h"

namespace asss {

// ---------------------------------------------------------------------------
// host-side error handling: every internal function returns asss_status and
// records a message; nothing aborts.
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
const char* get_error();

#define ASSS_CUDA(call)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::asss::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,          \
                              cudaGetErrorString(e_));                             \
            return e_ == cudaErrorMemoryAllocation ? ASSS_ERR_OOM : ASSS_ERR_CUDA; \
        }                                                                          \
    } while (0)

#define ASSS_TRY(call)                     \
    do {                                   \
        asss_status s_ = (call);           \
        if (s_ != ASSS_OK) return s_;      \
    } while (0)

void count_launch();
#define ASSS_CHECK_LAUNCH()            \
    do {                               \
        ::asss::count_launch();        \
        ASSS_CUDA(cudaGetLastError()); \
    } while (0)

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// device buffers owned by the library
// ---------------------------------------------------------------------------
template <class T>
struct DBuf {
    T* p = nullptr;
    int64_t n = 0;
    asss_status alloc(int64_t count) {
        free();
        if (count <= 0) return ASSS_OK;
        cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * (size_t)count);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc of %lld bytes failed: %s", (long long)(sizeof(T) * count),
                      cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? ASSS_ERR_OOM : ASSS_ERR_CUDA;
        }
        n = count;
        return ASSS_OK;
    }
    void free() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DBuf() { free(); }
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
};

// Reduction scratch that lives as long as the process, one buffer per device and
// thread.  It is never freed by the library's own threads, so no CUDA call runs during
// process teardown; worker threads the library starts free theirs before they end
// (release_thread_scratch, after their streams are idle).
asss_status process_scratch(int slot, int64_t count, double** out);
void release_thread_scratch();
// raises a kernel's dynamic shared-memory limit to at least bytes (never lowers it)
asss_status raise_dynamic_smem(const void* func, int bytes);

// CSR with 32-bit row pointers (nnz < 2^31 is checked on entry).
// Optional diagonal copy of a CSR matrix whose entries sit on a few diagonals
// (stencils): val[d*n + i] = A(i, i + off[d]), 0 where absent or outside the matrix.
struct DDia {
    bool tried = false;  // attach_dia ran on this matrix (attached or not)
    bool stream = false; // values loaded evict-first (two products' values exceed L2)
    int ndiag = 0;
    DBuf<int> off;       // ascending signed offsets
    DBuf<double> val;
};

struct DCsr {
    int n = 0;
    int nnz = 0;
    DBuf<int> rp, ci;
    DBuf<double> v;
    DDia dia;            // used by spmv when present
};

// SELL-C (C = 32) storage: slot 32s + t (lane t of slice s) holds row rowmap[32s + t]
// (row 32s + t when rowmap is empty); entry kk of that lane sits at sptr[s] + kk*32 + t.
// With SELL-C-sigma the rows of each window of sigma consecutive rows are sorted
// by length (longest first) before they are cut into slices, so a slice holds rows
// of similar length and heavy-tailed row lengths do not pad every slice to its
// longest row.  Padding entries have value 0 and a valid column; slots past the
// last row map to row n (no row).
constexpr int SELL_SIGMA = 4096;          // default sorting window
constexpr int SELL_SIGMA_MAX = 16384;     // largest window the sort kernel takes
template <class T>
struct DSell {
    int n = 0;
    int nslices = 0;
    int64_t nstored = 0;  // including padding
    int64_t nnz = 0;      // stored entries that come from the matrix
    DBuf<int> sptr;   // nslices + 1
    DBuf<int> col;
    DBuf<T> val;
    DBuf<int> rowmap; // 32 * nslices slots -> row (empty: identity)
    DBuf<int> rowpos; // n rows -> slot (empty: identity)
    // Work units of a pass: a slice, or one part of `split` entries of a long slice
    // (x slice, y part, z parts of that slice, w its accumulator or -1); uoff[s] is the
    // first unit of slice s.  The parts of a long slice add their lanes' partial sums
    // into hacc (32 values per long slice) and the last one to finish carries on.
    int sigma = 0;        // sorting window in rows (0: natural order)
    int split = 0;        // entries per lane of one work unit
    int nunits = 0;
    int nheavy = 0;
    DBuf<int4> units;
    DBuf<int> uoff;
    DBuf<T> hacc;
    DBuf<unsigned> hcnt;
};
constexpr int SELL_SPLIT = 1024;

// Skew half-diagonal storage of an exactly skew matrix J whose entries lie on a
// few diagonals (stencil-like patterns): only the diagonals with positive offset
// are stored, U[d*n + i] = J[i, i + off[d]] (0 where absent), and the lower
// triangle is read from the same arrays shifted: J[i, i - off[d]] = -U[d*n + i - off[d]].
template <class T>
struct DSkewDia {
    int n = 0;
    int ndiag = 0;
    int64_t nnz = 0;          // stored upper entries that come from the matrix
    int halo = 0;             // largest offset: zero entries stored in front of each diagonal
    int64_t ustride = 0;      // n + halo
    DBuf<int> off;            // ndiag ascending positive offsets
    DBuf<T> U;                // diagonal d at U + d*ustride + halo, entries [-halo, n)
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  Every block calls
// it the same number of times.  The wait is bounded: after `budget` clock cycles
// the block records ASSS_ERR_TIMEOUT in *err and returns.
struct GridBarrier {
    unsigned* count;  // arrivals in the current phase
    unsigned* gen;    // phase counter
    int* err;         // device status word
};

__device__ __forceinline__ void grid_sync(const GridBarrier& gb, unsigned nblocks, long long budget) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g = ld_acquire(gb.gen);
        __threadfence();
        unsigned ticket = atomicAdd(gb.count, 1u);
        if (ticket == nblocks - 1) {
            atomicExch(gb.count, 0u);
            __threadfence();
            atomicAdd(gb.gen, 1u);
        } else {
            long long t0 = clock64();
            while (ld_acquire(gb.gen) == g) {
                if (clock64() - t0 > budget) {
                    atomicExch(gb.err, (int)ASSS_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Grid barrier on a counter that only grows during a launch (set to 0 before it):
// barrier number `phase` (0-based) is complete once the counter reaches
// (phase + 1) * nblocks.  One atomic per block and no reset on the critical path;
// the last block to arrive does not wait.  Waits are bounded like grid_sync.
__device__ __forceinline__ void grid_sync_phase(const GridBarrier& gb, unsigned nblocks, unsigned phase,
                                                long long budget) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = (phase + 1u) * nblocks;
        __threadfence();
        const unsigned arrived = atomicAdd(gb.count, 1u) + 1u;
        if (arrived != target) {
            long long t0 = clock64();
            while ((int)(ld_acquire(gb.count) - target) < 0) {
                if (clock64() - t0 > budget) {
                    atomicExch(gb.err, (int)ASSS_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// NVTX ranges (header-only NVTX 3: no library to link; a profiler that injects
// itself, e.g. ncu --nvtx, sees them, otherwise they cost a branch)
// ---------------------------------------------------------------------------
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// host helpers shared by the translation units
// ---------------------------------------------------------------------------
struct Ctx {
    cudaStream_t stream = 0;
    int device = 0;
    int sms = 0;
    int clock_khz = 0;
    long long wait_cycles = 0;
    long long l2_bytes = 0;
    bool force_stream = false;  // ASSS_FORCE_EVICT_FIRST=1: take the evict-first loads at any size
};

// Data read once per pass is loaded evict-first only when the pass's working set is
// larger than L2: then it would only push out the vectors that the next pass reuses;
// when everything fits, normal loads keep the streamed data in L2 for the next pass.
// The environment variable ASSS_FORCE_EVICT_FIRST=1 (read when a context is made)
// selects the evict-first loads at every size, so that small inputs exercise the code
// path that large ones take.
inline bool stream_evict_first(const Ctx& c, long long pass_bytes) {
    return c.force_stream || (c.l2_bytes > 0 && pass_bytes > c.l2_bytes * 3 / 4);
}
asss_status make_ctx(Ctx& c, void* stream, double wait_timeout_ms);

// pointer classification
bool is_device_ptr(const void* p);

// copy n elements from a host-or-device pointer into a device buffer
template <class T>
asss_status to_device(DBuf<T>& dst, const T* src, int64_t n, cudaStream_t s) {
    ASSS_TRY(dst.alloc(n));
    if (n == 0) return ASSS_OK;
    ASSS_CUDA(cudaMemcpyAsync(dst.p, src, sizeof(T) * n, cudaMemcpyDefault, s));
    return ASSS_OK;
}

// exclusive scan of int counts (n entries) into out (n+1 entries); returns total
asss_status exclusive_scan(const int* cnt, int* out, int n, int64_t* total, cudaStream_t s);
asss_status exclusive_scan64(const int* cnt, long long* out, int n, long long* total, cudaStream_t s);

// deterministic sum reductions: out[0] = sum a[i]*b[i] (b may be null: sum a^2 if a==b flagged)
asss_status dot(const double* a, const double* b, int n, double* d_out, cudaStream_t s);
asss_status dot_f(const float* a, const float* b, int n, double* d_out, cudaStream_t s);

}  // namespace asss
