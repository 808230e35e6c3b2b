// Instantiations of the batched solver (batch_kernel.cuh): FP32 Q, padded widths 0, 8 and 16.
#include "batch_kernel.cuh"

namespace asss {

asss_status batch_part0(const BatchLaunch* L, int kp, int nthreads, int minb, int nblk, cudaStream_t s, int* occ) {
    switch (kp) {
        case 0:
            return L ? launch_nt<0, false>(*L, nthreads, minb, nblk, s) : occ_nt<0, false>(nthreads, minb, occ);
        case 8:
            return L ? launch_nt<8, false>(*L, nthreads, minb, nblk, s) : occ_nt<8, false>(nthreads, minb, occ);
        case 16:
            return L ? launch_nt<16, false>(*L, nthreads, minb, nblk, s) : occ_nt<16, false>(nthreads, minb, occ);
    }
    set_error("batched solver: unsupported Lanczos width %d", kp);
    return ASSS_ERR_UNSUPPORTED;
}

}  // namespace asss
