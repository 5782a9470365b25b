// The second and third steps of the filter kernel's phased form
// (filter_kernel.cuh): one thread per listed survivor, then one per listed
// walk, for every code width.
#include "filter_kernel.cuh"

namespace pfac {

cudaError_t launch_survivors(OutMode mode, const filt::FilterParams &p, uint32_t B, uint32_t gbits, uint32_t sms,
                             int per_thread, cudaStream_t stream) {
    using filt::launch_survivors;
    const bool g16 = gbits == 16;
    if (B == 8) {
        if (per_thread == 4)
            return g16 ? launch_survivors<8, int16_t, 4>(mode, p, sms, stream)
                       : launch_survivors<8, int32_t, 4>(mode, p, sms, stream);
        return g16 ? launch_survivors<8, int16_t, 2>(mode, p, sms, stream)
                   : launch_survivors<8, int32_t, 2>(mode, p, sms, stream);
    }
    if (B == 4)
        return g16 ? launch_survivors<4, int16_t, 2>(mode, p, sms, stream)
                   : launch_survivors<4, int32_t, 2>(mode, p, sms, stream);
    if (B == 2)
        return g16 ? launch_survivors<2, int16_t, 2>(mode, p, sms, stream)
                   : launch_survivors<2, int32_t, 2>(mode, p, sms, stream);
    return cudaErrorInvalidValue;
}

}  // namespace pfac
