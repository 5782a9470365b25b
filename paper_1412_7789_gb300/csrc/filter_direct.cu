// The one-phase single-text forms of the small-alphabet kernel for 2-bit
// codes computed as (byte >> 1) & 3, at the widest launch (filter_kernel.cuh,
// DIRECT = true), compiled apart so that they build in parallel with the
// other forms.
#include "filter_kernel.cuh"

namespace pfac {
namespace filt {

cudaError_t launch_filter_direct(int mode, const FilterParams &p, uint32_t gbits, uint32_t grid, uint32_t block,
                                 uint32_t smem, int max_smem, cudaStream_t stream) {
    if (p.direct_shift != 1 || block > static_cast<uint32_t>(kMaxBlock))
        return cudaErrorInvalidValue;
    switch (mode) {
        case OUT_DENSE:
            return gbits == 16
                       ? launch_one_bounded<2, int16_t, OUT_DENSE, false, false, false, kMaxBlock, true>(
                             p, grid, block, smem, max_smem, stream)
                       : launch_one_bounded<2, int32_t, OUT_DENSE, false, false, false, kMaxBlock, true>(
                             p, grid, block, smem, max_smem, stream);
        case OUT_COUNT:
            return gbits == 16
                       ? launch_one_bounded<2, int16_t, OUT_COUNT, false, false, false, kMaxBlock, true>(
                             p, grid, block, smem, max_smem, stream)
                       : launch_one_bounded<2, int32_t, OUT_COUNT, false, false, false, kMaxBlock, true>(
                             p, grid, block, smem, max_smem, stream);
        case OUT_SLOTS:
            return gbits == 16
                       ? launch_one_bounded<2, int16_t, OUT_SLOTS, false, false, false, kMaxBlock, true>(
                             p, grid, block, smem, max_smem, stream)
                       : launch_one_bounded<2, int32_t, OUT_SLOTS, false, false, false, kMaxBlock, true>(
                             p, grid, block, smem, max_smem, stream);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace filt
}  // namespace pfac
