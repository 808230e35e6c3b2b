// Device helpers shared by the single- and multi-right-hand-side mrs kernels.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace asss {

constexpr int MRS_THREADS = 512;
constexpr int MRS_WARPS = MRS_THREADS / 32;
constexpr int MRS_KPMAX = 64;
constexpr int MRS_MAXDIAG = 64;

// BF16 rows: KP a multiple of 8, 16-byte aligned, converted to T on load
template <class T, int KP>
__device__ __forceinline__ void load_qrow16(const __nv_bfloat16* __restrict__ Q, int i, T (&q)[KP > 0 ? KP : 1]) {
    if constexpr (KP > 0) {
        const __nv_bfloat16* row = Q + (size_t)i * KP;
#pragma unroll
        for (int m = 0; m < KP; m += 8) {
            uint4 v = *reinterpret_cast<const uint4*>(row + m);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                float2 f = __bfloat1622float2(h[t]);
                q[m + 2 * t] = (T)f.x;
                q[m + 2 * t + 1] = (T)f.y;
            }
        }
    }
}

// cs: Q is streamed once per step and the step's data exceed L2, so its rows are
// loaded evict-first to keep the reused vectors in L2 (see stream_evict_first)
template <class T, int KP>
__device__ __forceinline__ void load_qrow(const T* __restrict__ Q, int i, T (&q)[KP > 0 ? KP : 1],
                                          bool cs = false) {
    if constexpr (KP > 0) {
        const T* row = Q + (size_t)i * KP;
        if constexpr (sizeof(T) == 4 && (KP % 4) == 0) {
#pragma unroll
            for (int m = 0; m < KP; m += 4) {
                const float4* a = reinterpret_cast<const float4*>(row + m);
                float4 v = cs ? __ldcs(a) : __ldg(a);
                q[m] = v.x;
                q[m + 1] = v.y;
                q[m + 2] = v.z;
                q[m + 3] = v.w;
            }
        } else if constexpr (sizeof(T) == 8 && (KP % 2) == 0) {
#pragma unroll
            for (int m = 0; m < KP; m += 2) {
                double2 v = *reinterpret_cast<const double2*>(row + m);
                q[m] = v.x;
                q[m + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int m = 0; m < KP; ++m) q[m] = row[m];
        }
    }
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Error-free FP32 pair ("double-float") addition: TwoSum of the leading parts, the
// trailing parts added to the error, renormalised.  About 44 significant bits, so
// the FP32 solve's cross-block sums stay accurate without the (slow) FP64 pipe.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s = a.x + b.x;
    float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    float hi = s + e;
    float lo = e - (hi - s);
    return make_float2(hi, lo);
}

// Scalar state of the recurrence, kept in shared memory and advanced by one
// thread per block in the precision of the vectors (the FP32 solve keeps its
// whole synchronisation chain off the narrow FP64 pipe of this part; every block
// computes the same values from the same reduced sums, so all blocks agree bit
// for bit).
template <class S>
struct MrsScalars {
    S r0, rr0, nu, coef_old, theta_t, c_prev, s_prev, delta_prev, G;
    S nu_p, delta_pp, rtheta_p, xcoef_p;   // rtheta_p = 1 / theta of the previous step
    // final-pass coefficients when the iteration stops
    S fin_nu, fin_delta, fin_rtheta, fin_xcoef;
    S ratio;
    int its, stop;
};

// block b owns slices [blk[b], blk[b+1]), balanced by stored entries (SELL) or
// uniform (diagonal storage: every row carries the same work)
static __global__ void k_partition(const int* sptr, int nslices, int nblk, int* blk) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblk) return;
    if (b == nblk) {
        blk[b] = nslices;
        return;
    }
    if (!sptr) {
        blk[b] = (int)((long long)nslices * b / nblk);
        return;
    }
    long long total = sptr[nslices];
    // slices also carry fixed per-row work (Q row, vectors): weight = stored + 32*8
    long long wtot = total + (long long)nslices * 256;
    long long target = wtot * b / nblk;
    int lo = 0, hi = nslices;
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);   // no overflow for offsets near 2^31
        long long w = (long long)sptr[mid] + (long long)mid * 256;
        if (w < target) lo = mid + 1;
        else hi = mid;
    }
    blk[b] = lo;
}

}  // namespace asss
