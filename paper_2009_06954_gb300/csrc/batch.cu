// Batched solves (many matrices of uneven size, many right-hand sides): the work-space
// size and the dispatch to the kernel instantiations (batch_kernel.cuh holds the
// kernel, batch_p0..3.cu instantiate it).
#include "batch_kernel.cuh"

namespace asss {

long long batch_work_doubles(int n_max, int halo_max, int restart) {
    long long nd = (long long)(5 + 2 * restart + 1) * n_max;                  // r, rh, dy, t1, t2, V, Z
    long long nf = 3LL * ((long long)n_max + 2LL * halo_max) + 3LL * n_max;   // Y ring, P, z32 (floats)
    return nd + (nf + 1) / 2 + 64;
}

static asss_status batch_dispatch(const BatchLaunch* L, int kp, int qbf16, int nthreads, int minb, int nblk,
                                  cudaStream_t s, int* occ) {
    if (!qbf16) return kp <= 16 ? batch_part0(L, kp, nthreads, minb, nblk, s, occ)
                                : batch_part1(L, kp, nthreads, minb, nblk, s, occ);
    return kp <= 16 ? batch_part2(L, kp, nthreads, minb, nblk, s, occ) : batch_part3(L, kp, nthreads, minb, nblk, s, occ);
}

asss_status batch_launch(const BatchLaunch& L, int nthreads, int minb, int nblk, cudaStream_t s) {
    return batch_dispatch(&L, L.kp, L.qbf16, nthreads, minb, nblk, s, nullptr);
}

asss_status batch_occupancy(int kp, int qbf16, int nthreads, int minb, int* occ) {
    return batch_dispatch(nullptr, kp, qbf16, nthreads, minb, 0, 0, occ);
}

}  // namespace asss
