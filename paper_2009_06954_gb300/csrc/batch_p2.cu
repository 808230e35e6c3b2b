// Instantiations of the batched solver (batch_kernel.cuh): BF16 Q, padded widths 8 and 16.
#include "batch_kernel.cuh"

namespace asss {

asss_status batch_part2(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ) {
    switch (kp) {
        case 8:
            return L ? launch_nt<8, true>(*L, nthreads, minb, nblk, s) : occ_nt<8, true>(nthreads, minb, occ);
        case 16:
            return L ? launch_nt<16, true>(*L, nthreads, minb, nblk, s) : occ_nt<16, true>(nthreads, minb, occ);
    }
    set_error("batched solver: unsupported Lanczos width %d", kp);
    return ASSS_ERR_UNSUPPORTED;
}

}  // namespace asss
