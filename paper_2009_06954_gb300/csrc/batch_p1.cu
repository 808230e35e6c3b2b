// Instantiations of the batched solver (batch_kernel.cuh): FP32 Q, padded widths 20, 24 and 32.
#include "batch_kernel.cuh"

namespace asss {

asss_status batch_part1(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ) {
    switch (kp) {
        case 20:
            return L ? launch_nt<20, false>(*L, nthreads, minb, nblk, s) : occ_nt<20, false>(nthreads, minb, occ);
        case 24:
            return L ? launch_nt<24, false>(*L, nthreads, minb, nblk, s) : occ_nt<24, false>(nthreads, minb, occ);
        case 32:
            return L ? launch_nt<32, false>(*L, nthreads, minb, nblk, s) : occ_nt<32, false>(nthreads, minb, occ);
    }
    set_error("batched solver: unsupported Lanczos width %d", kp);
    return ASSS_ERR_UNSUPPORTED;
}

}  // namespace asss
