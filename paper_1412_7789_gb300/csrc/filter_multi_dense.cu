// The multi-automaton batch kernel (filter_kernel.cuh, pfac_filter_multi) for
// dense ids, compiled apart so that the kernel forms build in parallel.
#include "filter_kernel.cuh"

namespace pfac {

cudaError_t launch_filter_multi_dense(const filt::MultiParams &mp, uint32_t grid, uint32_t smem, int max_smem,
                                      cudaStream_t stream) {
    return filt::launch_multi<OUT_DENSE>(mp, grid, smem, max_smem, stream);
}

}  // namespace pfac
