// The 8-bit-code forms of the filter kernel (filter_kernel.cuh, B = 8: the
// hashed root filter over windows of up to 4 codes and the state hash),
// compiled apart from the small-alphabet forms so that the sets build in
// parallel.
#include "filter_kernel.cuh"

namespace pfac {

cudaError_t launch_filter8(OutMode mode, const filt::FilterParams &p, uint32_t gbits, uint32_t grid, uint32_t block,
                           uint32_t smem, int max_smem, cudaStream_t stream) {
    using filt::launch_modes;
    return gbits == 16 ? launch_modes<8, int16_t, false>(mode, p, grid, block, smem, max_smem, stream)
                       : launch_modes<8, int32_t, false>(mode, p, grid, block, smem, max_smem, stream);
}

}  // namespace pfac
