// Compacted output (the (pos, id) list in ascending position), in three steps
// after a matching kernel that ran in slot mode, i.e. wrote for every work
// unit (tile) u the number of matches counts[u] and the first kSlotCap of them,
// in any order, into slots[u]:
//   compact_reduce   the sum of counts over each of kScanCtas contiguous ranges
//                    of units;
//   compact_prefix   the exclusive prefix of counts at every unit (each CTA
//                    adds the partial sums before its range to a block scan of
//                    its own range);
//   compact_gather   one warp per unit with matches (grid stride; 32 units'
//                    counts read per warp round, the empty ones skipped): the unit's matches in
//                    ascending position at the unit's place in its text's
//                    list; then every text's total.  A unit with more than
//                    kSlotCap matches (a dense run of matches) is read from the
//                    dense ids the matching kernel kept for it, or, without
//                    them, matched again here, one plain walk per position.
// No step waits on another CTA, so no step can stall on a CTA that is not
// resident; each runs at the speed of its memory traffic (4 + 8 bytes per unit
// for the scan, 8 bytes per match for the gather).
#include <cuda_runtime.h>

#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

namespace {

constexpr int kScanThreads = 512;
constexpr int kGatherThreads = 256;
constexpr uint32_t kRows = 8;  // rows of 32 dense ids loaded together

// Block-wide sum; every thread gets the total.
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v) {
    __shared__ unsigned long long ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int w = 0; w < nw; ++w) t += ws[w];
    __syncthreads();
    return t;
}

// Block-wide exclusive scan; `total` receives the block's sum.
__device__ __forceinline__ unsigned long long block_excl(unsigned long long v, unsigned long long &total) {
    __shared__ unsigned long long ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) before += ws[w];
        all += ws[w];
    }
    __syncthreads();
    total = all;
    return before + inc - v;
}

__device__ __forceinline__ uint32_t scan_units(uint32_t units, const uint32_t *units_dev) {
    return units_dev ? __ldg(units_dev) : units;
}

__global__ void __launch_bounds__(kScanThreads) compact_reduce(const uint32_t *counts, uint32_t units,
                                                               const uint32_t *units_dev,
                                                               unsigned long long *partials) {
    const uint32_t U = scan_units(units, units_dev);
    const uint32_t R = (U + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = static_cast<uint64_t>(blockIdx.x) * R;
    const uint64_t hi = lo + R < U ? lo + R : U;
    unsigned long long s = 0;
    for (uint64_t u = lo + threadIdx.x; u < hi; u += blockDim.x) s += __ldg(counts + u);
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads) compact_prefix(const uint32_t *counts, uint32_t units,
                                                               const uint32_t *units_dev,
                                                               unsigned long long *prefix,
                                                               const unsigned long long *partials) {
    const uint32_t U = scan_units(units, units_dev);
    const uint32_t R = (U + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = static_cast<uint64_t>(blockIdx.x) * R;
    const uint64_t hi = lo + R < U ? lo + R : U;
    unsigned long long base = 0;
    for (uint32_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) base += partials[b];
    base = block_sum(base);
    for (uint64_t c0 = lo; c0 < hi; c0 += blockDim.x) {
        const uint64_t u = c0 + threadIdx.x;
        const unsigned long long v = u < hi ? __ldg(counts + u) : 0ull;
        unsigned long long tot = 0;
        const unsigned long long ex = block_excl(v, tot);
        if (u < hi) prefix[u] = base + ex;
        base += tot;
    }
}

// The gather's request and the tables to match a unit again (RootWalk).
struct GatherParams : RootWalk {
    GatherRequest g;
};

// One warp: unit u's matches in ascending position at the unit's place in its
// text's list.
template <typename GT>
__device__ __forceinline__ void gather_unit(const GatherParams &p, const Work &wk, uint32_t T, uint32_t u, int lane) {
    const uint8_t *text = p.g.text;
    uint64_t n = p.g.n;
    uint32_t first = 0;
    CompactOut out = p.g.out;
    if (wk.list) {
        const uint32_t item = find_item(wk, u, lane);
        const BatchItemDev it = wk.list[item];
        text = p.g.text + it.text_off;
        n = it.len;
        first = it.first_unit;
        out = p.g.outs[it.item];
    }
    const uint32_t head = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(text) & 15u);
    const uint32_t lu = u - first;  // the unit's tile within its text
    const int64_t gpb = static_cast<int64_t>(lu) * T - head;
    const uint64_t su = static_cast<uint64_t>(p.g.ubase) + u;
    const unsigned long long base = __ldg(p.g.prefix + p.g.ubase + first);
    const unsigned long long at = __ldg(p.g.prefix + su);
    const uint32_t c = __ldg(p.g.counts + su);
    unsigned long long o = at - base;
    if (c <= kSlotCap) {
        const unsigned long long e =
            static_cast<uint32_t>(lane) < c ? __ldg(p.g.slots + su * kSlotCap + lane) : ~0ull;
        const uint32_t mine = static_cast<uint32_t>(e);
        uint32_t rank = 0;
        for (uint32_t d = 0; d < c; ++d) {  // c is the same for the whole warp
            const uint32_t other = __shfl_sync(0xffffffffu, mine, static_cast<int>(d));
            rank += other < mine ? 1u : 0u;
        }
        if (static_cast<uint32_t>(lane) < c && o + rank < out.cap) {
            out.pos[o + rank] = mine;
            out.ids[o + rank] = static_cast<uint32_t>(e >> 32);
        }
    } else {
        // more matches than slots: the unit's dense ids if kept (eight rows of
        // 32 loaded at a time, so their loads overlap), else match it again
        const int32_t *dn = p.g.dense ? p.g.dense + su * kDenseStride : nullptr;
        for (uint32_t i0 = 0; i0 < T; i0 += 32 * kRows) {
            int id[kRows];
#pragma unroll
            for (uint32_t j = 0; j < kRows; ++j) {
                const int64_t gp = gpb + static_cast<int64_t>(i0 + 32 * j) + lane;
                id[j] = -1;
                if (i0 + 32 * j < T && gp >= 0 && static_cast<uint64_t>(gp) < n)
                    id[j] = dn ? __ldg(dn + i0 + 32 * j + lane) : walk_from_root<GT>(p, text, n, gp);
            }
#pragma unroll
            for (uint32_t j = 0; j < kRows; ++j) {
                const unsigned m = __ballot_sync(0xffffffffu, id[j] >= 0);
                const uint32_t r = __popc(m & ((1u << lane) - 1u));
                if (id[j] >= 0 && o + r < out.cap) {
                    out.pos[o + r] = static_cast<uint32_t>(gpb + static_cast<int64_t>(i0 + 32 * j) + lane);
                    out.ids[o + r] = static_cast<uint32_t>(id[j]);
                }
                o += __popc(m);
            }
        }
    }
}

template <typename GT>
__global__ void __launch_bounds__(kGatherThreads) compact_gather(const GatherParams p) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const Work wk = load_work(p.g.batch, p.g.lists, p.g.units);
    const uint32_t T = p.g.tile;
    // Units gw, gw + nwarps, ... (grid stride), 32 of them per round with one
    // count load per lane: only units with matches are visited (most have
    // none), and every warp keeps its share of the units.
    for (uint64_t u0 = gw; u0 < wk.units; u0 += 32ull * nwarps) {
        const uint64_t uu = u0 + static_cast<uint64_t>(lane) * nwarps;
        const uint32_t cu = uu < wk.units ? __ldg(p.g.counts + p.g.ubase + uu) : 0u;
        for (uint32_t todo = __ballot_sync(0xffffffffu, cu != 0); todo; todo &= todo - 1)
            gather_unit<GT>(p, wk, T, static_cast<uint32_t>(u0 + static_cast<uint64_t>(__ffs(todo) - 1) * nwarps), lane);
    }
    // each text's total: its last unit's prefix and count, less its first's prefix
    if (!wk.list) {
        if (gw == 0 && lane == 0 && wk.units > 0) {
            const uint64_t last = static_cast<uint64_t>(p.g.ubase) + wk.units - 1;
            *p.g.out.count = __ldg(p.g.prefix + last) + __ldg(p.g.counts + last) - __ldg(p.g.prefix + p.g.ubase);
        }
        return;
    }
    for (uint32_t i = gw * 32u + static_cast<uint32_t>(lane); i < wk.nlist; i += nwarps * 32u) {
        const BatchItemDev it = wk.list[i];
        const uint32_t head = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.g.text + it.text_off) & 15u);
        const uint64_t text_units = (it.len + head + T - 1) / T;
        const uint64_t first = static_cast<uint64_t>(p.g.ubase) + it.first_unit;
        const uint64_t last = first + text_units - 1;
        *p.g.outs[it.item].count = __ldg(p.g.prefix + last) + __ldg(p.g.counts + last) - __ldg(p.g.prefix + first);
    }
}

}  // namespace

cudaError_t launch_compact_scan(const uint32_t *counts, uint32_t units, const uint32_t *units_dev,
                                unsigned long long *prefix, unsigned long long *partials, cudaStream_t stream) {
    if (!counts || !prefix || !partials) return cudaErrorInvalidValue;
    compact_reduce<<<kScanCtas, kScanThreads, 0, stream>>>(counts, units, units_dev, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    compact_prefix<<<kScanCtas, kScanThreads, 0, stream>>>(counts, units, units_dev, prefix, partials);
    return cudaGetLastError();
}

cudaError_t launch_compact_gather(const DevTables &t, const GatherRequest &g, cudaStream_t stream) {
    if (!g.counts || !g.prefix || !g.slots || g.tile == 0) return cudaErrorInvalidValue;
    if (!g.batch && g.units == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    GatherParams p{};
    p.g = g;
    p.G = t.G;
    p.cls8 = t.cls8;
    p.W = t.W;
    p.C = t.C;
    p.maxlen = t.maxlen;
    p.skip = t.skip;
    p.chain = t.chain;
    p.s_chain = t.skip ? t.s_chain : 0xFFFFFFFFu;
    e = device_error_word(&p.err);
    if (e != cudaSuccess) return e;
    const uint32_t per_cta = kGatherThreads / 32;
    uint32_t grid = static_cast<uint32_t>(sms) * 8u;  // grid-stride over units
    if (!g.batch) {
        const uint32_t need = (g.units + per_cta - 1) / per_cta;
        if (grid > need) grid = need;
    }
    if (t.gbits == 16)
        compact_gather<int16_t><<<grid, kGatherThreads, 0, stream>>>(p);
    else
        compact_gather<int32_t><<<grid, kGatherThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

namespace {
inline size_t round16(size_t v) { return (v + 15u) & ~static_cast<size_t>(15u); }
}  // namespace

uint32_t compact_units(const DevTables &t, const Tuning &tu, const uint8_t *text, uint64_t n) {
    const uint64_t T = unit_positions(t, tu);
    const uint64_t head = reinterpret_cast<uintptr_t>(text) & 15u;
    const uint64_t u = (n + head + T - 1) / T;
    return u >= 0x7FFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(u);
}

size_t compact_scratch_bytes(const DevTables &t, uint32_t units, bool dense) {
    (void)t;
    return compact_dense_offset(units) + (dense ? 4 * static_cast<size_t>(kDenseStride) * units : 0);
}

cudaError_t enqueue_compact(const DevTables &t, const Tuning &tu, const uint8_t *text, uint64_t n,
                            const CompactOut &out, void *scratch, size_t scratch_bytes, bool dense,
                            cudaStream_t stream) {
    const uint32_t U = compact_units(t, tu, text, n);
    if (U == 0xFFFFFFFFu || n > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    if (!scratch || scratch_bytes < compact_scratch_bytes(t, U, dense)) return cudaErrorInvalidValue;
    uint8_t *b = static_cast<uint8_t *>(scratch);
    uint32_t *counts = reinterpret_cast<uint32_t *>(b + 16);
    unsigned long long *prefix = reinterpret_cast<unsigned long long *>(b + 16 + round16(4 * size_t(U)));
    unsigned long long *slots = prefix + U;
    unsigned long long *partials = slots + static_cast<size_t>(kSlotCap) * U;
    int32_t *dn = dense ? reinterpret_cast<int32_t *>(b + compact_dense_offset(U)) : nullptr;
    cudaError_t e = cudaMemsetAsync(b, 0, 16 + 4 * size_t(U), stream);
    if (e != cudaSuccess) return e;
    MatchRequest r;
    // room after the scratch for the phased form's lists: then its units
    // keep no dense fallback (the gather matches an overflowing unit again)
    const size_t lo = compact_scratch_bytes(t, U, dense);
    SurvivorLists sl;
    if (uses_filter(t, tu)) sl = survivor_lists(t, tu, n, true);
    if (sl.list_cap && scratch_bytes >= lo + sl.bytes()) {
        e = cudaMemsetAsync(b + lo, 0, 32, stream);
        if (e != cudaSuccess) return e;
        set_lists(r, b + lo, sl);
        dn = nullptr;
    }
    r.text = text;
    r.n = n;
    r.slots.counts = counts;
    r.slots.slots = slots;
    r.slots.ubase = 0;
    r.slots.dense = dn;
    r.scratch = b;
    r.scratch_bytes = 16;
    e = launch_match(t, r, OUT_SLOTS, tu, stream);
    if (e != cudaSuccess) return e;
    e = launch_compact_scan(counts, U, nullptr, prefix, partials, stream);
    if (e != cudaSuccess) return e;
    GatherRequest g;
    g.text = text;
    g.n = n;
    g.out = out;
    g.units = U;
    g.tile = unit_positions(t, tu);
    g.counts = counts;
    g.prefix = prefix;
    g.slots = slots;
    g.dense = dn;
    return launch_compact_gather(t, g, stream);
}

}  // namespace pfac
