// ac_match_compact_static: the compacted matching call without any device
// allocation.  Its scratch (tile counter, per-tile match counts, prefix sums and
// match slots of the compaction) lives in one file-scope device array that
// every call shares.
#include <cuda_runtime.h>

#include <mutex>

#include "ac.h"
#include "pfac_internal.h"


namespace {

// Scratch for texts of up to AC_STATIC_MAX_TEXT bytes, shared by all calls on a
// device.  The module holding it is loaded, and the array committed, on a
// device when the first handle is compiled there (static_scratch_address,
// called by ac_compile); it stays until the process exits.
__device__ __align__(256) unsigned char g_compact_scratch[AC_STATIC_SCRATCH_BYTES];

// A text of AC_STATIC_MAX_TEXT bytes at any alignment, cut into the shortest
// tiles of any matching kernel, must fit the array (no dense fallback).
static_assert(pfac::compact_dense_offset((AC_STATIC_MAX_TEXT + 15 + pfac::kMinTile - 1) / pfac::kMinTile) <=
                  AC_STATIC_SCRATCH_BYTES,
              "AC_STATIC_SCRATCH_BYTES does not hold the scratch of an AC_STATIC_MAX_TEXT text");

std::mutex g_mu;
void *g_scratch_ptr[64] = {nullptr};  // device address of g_compact_scratch, per device

}  // namespace

// The device address of the array on device `dev` (the current device),
// looked up once per device: host code sees only a host-side stand-in for the
// symbol, never its device address.
cudaError_t pfac::static_scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_compact_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

extern "C" ac_status ac_match_compact_static(ac_handle h, const uint8_t *d_text, uint64_t n, uint32_t *d_pos,
                                             uint32_t *d_ids, uint64_t cap, uint64_t *d_count, void *stream) {
    int device = 0;
    bool host_only = true;
    const pfac::DevTables *t = pfac::handle_tables(h, &device, &host_only);
    if (!t || host_only) return AC_ERR_INVALID_ARG;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return AC_ERR_CUDA;
    if (cur != device || cur < 0 || cur >= 64) return AC_ERR_INVALID_ARG;
    if (!d_count || (cap > 0 && (!d_pos || !d_ids))) return AC_ERR_INVALID_ARG;
    if (n > AC_STATIC_MAX_TEXT) return AC_ERR_BUDGET;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st) == cudaSuccess ? AC_OK : AC_ERR_CUDA;
    if (!d_text) return AC_ERR_INVALID_ARG;
    const uint32_t units = pfac::compact_units(*t, *pfac::handle_tuning(h), d_text, n);
    // no dense fallback here: a tile with many matches is matched again by the gather step
    const size_t bytes = pfac::compact_scratch_bytes(*t, units, false);
    if (bytes > AC_STATIC_SCRATCH_BYTES) return AC_ERR_BUDGET;
    void *scratch = nullptr;
    if (pfac::static_scratch_address(cur, &scratch) != cudaSuccess) return AC_ERR_CUDA;
    // enqueue_compact clears the counter and counts it uses: the array keeps
    // the previous call's contents
    pfac::CompactOut out{d_pos, d_ids, cap, reinterpret_cast<unsigned long long *>(d_count)};
    const cudaError_t e = pfac::enqueue_compact(*t, *pfac::handle_tuning(h), d_text, n, out, scratch, bytes, false, st);
    if (e == cudaSuccess) return AC_OK;
    if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) return AC_ERR_INVALID_ARG;
    return AC_ERR_CUDA;
}
