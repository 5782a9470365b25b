// The forms of the small-alphabet kernel that share heavy tiles within the
// CTA (filter_kernel.cuh, HELP = true), compiled apart from the plain forms so
// that the two sets build in parallel.
#include "filter_kernel.cuh"

namespace pfac {

cudaError_t launch_filter_help(OutMode mode, const filt::FilterParams &p, uint32_t B, uint32_t gbits, uint32_t grid,
                               uint32_t block, uint32_t smem, int max_smem, cudaStream_t stream) {
    using filt::launch_modes;
    if (B == 2) {
        if (gbits == 16) return launch_modes<2, int16_t, true>(mode, p, grid, block, smem, max_smem, stream);
        return launch_modes<2, int32_t, true>(mode, p, grid, block, smem, max_smem, stream);
    }
    if (B == 4) {
        if (gbits == 16) return launch_modes<4, int16_t, true>(mode, p, grid, block, smem, max_smem, stream);
        return launch_modes<4, int32_t, true>(mode, p, grid, block, smem, max_smem, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pfac
