// Instantiations of the batched solver (batch_kernel.cuh): BF16 Q, padded widths 24 and 32.
#include "batch_kernel.cuh"

namespace asss {

asss_status batch_part3(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ) {
    switch (kp) {
        case 24:
            return L ? launch_nt<24, true>(*L, nthreads, minb, nblk, s) : occ_nt<24, true>(nthreads, minb, occ);
        case 32:
            return L ? launch_nt<32, true>(*L, nthreads, minb, nblk, s) : occ_nt<32, true>(nthreads, minb, occ);
    }
    set_error("batched solver: unsupported Lanczos width %d", kp);
    return ASSS_ERR_UNSUPPORTED;
}

}  // namespace asss
