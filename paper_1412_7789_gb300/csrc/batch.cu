// Batch planning on the device.
//
// A batch is a list of (text, automaton) items in device memory.  The matching
// kernels take their work as tiles ("units"); for one automaton they need its
// texts in a list with, per text, the number of its first unit, so that a warp
// that claims unit u finds its text with a short search (find_item).  One CTA
// per automaton builds that list in item order with two passes over the items:
// the first counts the texts of earlier automata (where this automaton's part
// of the shared list starts), the second compacts this automaton's non-empty
// texts with a block-wide scan of their tile counts.  Nothing is read on the
// host, so a batch stays asynchronous and can be captured in a CUDA graph whose
// item contents change between replays.
#include <cuda_runtime.h>

#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

namespace {

constexpr int kPlanThreads = 1024;

struct PlanArgs {
    const ac_batch_item *items;
    uint32_t nitems, nh;
    const uint8_t *texts;
    BatchHead *heads;
    BatchItemDev *lists;
    unsigned int *err;
    uint32_t tile_len[kMaxBatchAutomata];
};

// Block-wide exclusive scan of (count, tiles) pairs; returns the block totals.
__device__ __forceinline__ void block_scan(uint32_t c, uint64_t t, uint32_t &c_ex, uint64_t &t_ex, uint32_t &c_tot,
                                           uint64_t &t_tot) {
    __shared__ uint32_t wc[32];
    __shared__ uint64_t wt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t ci = c;
    uint64_t ti = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t yc = __shfl_up_sync(0xffffffffu, ci, d);
        const uint64_t yt = __shfl_up_sync(0xffffffffu, ti, d);
        if (lane >= d) {
            ci += yc;
            ti += yt;
        }
    }
    if (lane == 31) {
        wc[warp] = ci;
        wt[warp] = ti;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t xc = lane < nw ? wc[lane] : 0u;
        uint64_t xt = lane < nw ? wt[lane] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t yc = __shfl_up_sync(0xffffffffu, xc, d);
            const uint64_t yt = __shfl_up_sync(0xffffffffu, xt, d);
            if (lane >= d) {
                xc += yc;
                xt += yt;
            }
        }
        if (lane < nw) {
            wc[lane] = xc;  // inclusive over warps
            wt[lane] = xt;
        }
    }
    __syncthreads();
    const uint32_t wbase_c = warp > 0 ? wc[warp - 1] : 0u;
    const uint64_t wbase_t = warp > 0 ? wt[warp - 1] : 0ull;
    c_ex = wbase_c + ci - c;
    t_ex = wbase_t + ti - t;
    c_tot = wc[nw - 1];
    t_tot = wt[nw - 1];
    __syncthreads();  // the shared words are reused by the next call
}

__global__ void __launch_bounds__(kPlanThreads) batch_plan(const PlanArgs a) {
    __shared__ uint32_t red[32];
    const uint32_t aut = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // 1. non-empty texts of earlier automata: the start of this one's list
    uint32_t before = 0;
    bool bad = false;
    for (uint32_t i = threadIdx.x; i < a.nitems; i += blockDim.x) {
        const ac_batch_item it = a.items[i];
        if (it.automaton >= a.nh) bad = true;
        else if (it.len > 0 && it.automaton < aut) ++before;
    }
    if (bad && aut == 0) atomicOr(a.err, static_cast<unsigned>(kErrBatchItem));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) before += __shfl_xor_sync(0xffffffffu, before, d);
    if (lane == 0) red[warp] = before;
    __syncthreads();
    uint32_t offset = 0;
    for (int w = 0; w < nw; ++w) offset += red[w];
    // 2. this automaton's texts in item order, numbered by their first unit
    const uint32_t T = a.tile_len[aut];
    uint32_t count = 0;
    uint64_t units = 0;
    for (uint32_t base = 0; base < a.nitems; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        ac_batch_item it{};
        bool mine = false;
        uint64_t tiles = 0;
        if (i < a.nitems) {
            it = a.items[i];
            mine = it.automaton == aut && it.len > 0;
            if (mine) {
                const uint64_t head = (reinterpret_cast<uintptr_t>(a.texts) + it.text_off) & 15u;
                tiles = (it.len + head + T - 1) / T;
            }
        }
        uint32_t c_ex, c_tot;
        uint64_t t_ex, t_tot;
        block_scan(mine ? 1u : 0u, tiles, c_ex, t_ex, c_tot, t_tot);
        if (mine) {
            BatchItemDev d;
            d.text_off = it.text_off;
            d.len = it.len;
            d.out_off = it.out_off;
            d.first_unit = static_cast<uint32_t>(units + t_ex);
            d.item = i;
            a.lists[offset + count + c_ex] = d;
        }
        count += c_tot;
        units += t_tot;
    }
    if (threadIdx.x == 0) {
        BatchHead h;
        h.count = count;
        h.offset = offset;
        h.pad = 0;
        if (units >= 0xFFFFFFFFull) {  // unit numbers are 32-bit: match nothing, report
            atomicOr(a.err, static_cast<unsigned>(kErrBatchItem));
            units = 0;
            h.count = 0;
        }
        h.units = static_cast<uint32_t>(units);
        a.heads[aut] = h;
    }
}

}  // namespace

cudaError_t launch_batch_plan(const ac_batch_item *items, uint32_t nitems, uint32_t nh, const uint8_t *texts,
                              const uint32_t *tile_len, BatchHead *heads, BatchItemDev *lists, cudaStream_t stream) {
    if (nh == 0 || nh > kMaxBatchAutomata || !heads || (nitems > 0 && (!items || !lists)))
        return cudaErrorInvalidValue;
    PlanArgs a{};
    a.items = items;
    a.nitems = nitems;
    a.nh = nh;
    a.texts = texts;
    a.heads = heads;
    a.lists = lists;
    for (uint32_t i = 0; i < nh; ++i) {
        if (tile_len[i] == 0 || (tile_len[i] & 15u)) return cudaErrorInvalidValue;
        a.tile_len[i] = tile_len[i];
    }
    cudaError_t e = device_error_word(&a.err);
    if (e != cudaSuccess) return e;
    batch_plan<<<nh, kPlanThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace pfac
