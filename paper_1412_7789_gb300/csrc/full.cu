// Full Aho-Corasick output: every occurrence of every keyword, the
// sub-patterns included (paper section II: the serial machine's output
// function reports at each text position all keywords ending there; the
// failureless walk keeps only the longest keyword per start).
//
// A keyword occurs at start i exactly when it is a prefix of the longest
// keyword r that the failureless walk from i reports, so the full list is the
// walk's compacted results with each result r expanded into the keywords that
// are prefixes of r (the builder's full-output records: r's string, its equal
// keywords, and the chain of proper-prefix keywords).  After the slot-mode
// matching kernel (per tile its match count and first 32 matches, plus its
// dense ids when it has more; with the phased form's lists no tile keeps dense
// ids, and a tile with more than 32 matches is matched again here):
//   full_count   one warp per tile: the tile's occurrences, the sum of the
//                chain lengths of its results;
//   scan         the exclusive prefix of those counts over the tiles
//                (compact_reduce / compact_prefix of compact.cu);
//   full_gather  one warp per tile: its results in ascending position, each
//                written out as its occurrences (end = start + len - 1, id),
//                shortest first, equal strings in ascending id.
#include <cuda_runtime.h>

#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

namespace {

constexpr int kFullThreads = 256;
constexpr uint32_t kRows = 8;  // rows of 32 dense ids loaded together
constexpr unsigned kFull = 0xffffffffu;

struct FullParams : RootWalk {
    const uint8_t *text;
    uint64_t n;
    uint32_t units, tile, head, max_clen, nkw;
    const uint32_t *counts;
    const unsigned long long *slots;
    const int32_t *dense;
    uint32_t *fcounts;
    const unsigned long long *fprefix;
    const uint4 *rec;
    const uint32_t *dups;
    CompactOut out;
};

// Chain length of result id (an id outside the keyword set, which no matching
// kernel writes, latches kErrWalk and counts as none).
__device__ __forceinline__ uint32_t chain_len(const FullParams &p, uint32_t id) {
    if (id >= p.nkw) {
        atomicOr(p.err, static_cast<unsigned>(kErrWalk));
        return 0;
    }
    return __ldg(reinterpret_cast<const uint32_t *>(p.rec) + 4ull * id + 3u);
}

// The dense id of tile position i of unit u (-1 outside the text): kept by
// the matching kernel, or (no dense ids) the walk from the root again.
template <typename GT>
__device__ __forceinline__ int dense_id(const FullParams &p, uint32_t u, int64_t gpb, uint32_t i) {
    const int64_t gp = gpb + static_cast<int64_t>(i);
    if (gp < 0 || static_cast<uint64_t>(gp) >= p.n) return -1;
    if (!p.dense) return walk_from_root<GT>(p, p.text, p.n, static_cast<uint64_t>(gp));
    return __ldg(p.dense + static_cast<uint64_t>(u) * kDenseStride + i);
}

template <typename GT>
__global__ void __launch_bounds__(kFullThreads) full_count(const FullParams p) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    // units gw, gw + nwarps, ... (grid stride), 32 per round: the empty ones
    // get 0 from their lane, the others are summed by the whole warp
    for (uint64_t u0 = gw; u0 < p.units; u0 += 32ull * nwarps) {
        const uint64_t uu = u0 + static_cast<uint64_t>(lane) * nwarps;
        const uint32_t cu = uu < p.units ? __ldg(p.counts + uu) : 0u;
        if (uu < p.units && cu == 0) p.fcounts[uu] = 0;
        for (uint32_t todo = __ballot_sync(kFull, cu != 0); todo; todo &= todo - 1) {
            const uint32_t b = static_cast<uint32_t>(__ffs(todo) - 1);
            const uint32_t u = static_cast<uint32_t>(u0 + static_cast<uint64_t>(b) * nwarps);
            const uint32_t c = __shfl_sync(kFull, cu, static_cast<int>(b));
            uint32_t sum = 0;
            if (c <= kSlotCap) {
                if (static_cast<uint32_t>(lane) < c)
                    sum = chain_len(p, static_cast<uint32_t>(
                                           __ldg(p.slots + static_cast<uint64_t>(u) * kSlotCap + lane) >> 32));
            } else {
                // eight rows of 32 dense ids at a time, so their loads overlap
                const int64_t gpb = static_cast<int64_t>(u) * p.tile - p.head;
                for (uint32_t i0 = 0; i0 < p.tile; i0 += 32 * kRows) {
                    int id[kRows];
#pragma unroll
                    for (uint32_t j = 0; j < kRows; ++j)
                        id[j] = i0 + 32 * j < p.tile ? dense_id<GT>(p, u, gpb, i0 + 32 * j + lane) : -1;
#pragma unroll
                    for (uint32_t j = 0; j < kRows; ++j)
                        if (id[j] >= 0) sum += chain_len(p, static_cast<uint32_t>(id[j]));
                }
            }
            sum = __reduce_add_sync(kFull, sum);
            if (lane == 0) p.fcounts[u] = sum;
        }
    }
}

// One lane: the occurrences of result r at start `pos`, from list index `at`:
// the chain from r down to its shortest prefix keyword fills the range from
// its end backwards, each string's equal keywords in ascending id.
__device__ __forceinline__ void put_chain(const FullParams &p, unsigned long long at, uint32_t pos, uint32_t r) {
    if (r >= p.nkw) return;  // latched by chain_len
    uint4 rx = __ldg(p.rec + r);
    for (uint32_t guard = 0; guard < p.max_clen; ++guard) {  // a chain has at most max_clen strings
        uint4 ru = make_uint4(kNoKeyword, 0u, 0u, 0u);
        if (rx.x != kNoKeyword && rx.x < p.nkw) ru = __ldg(p.rec + rx.x);
        const uint32_t end = pos + rx.y - 1u;
        for (uint32_t j = ru.w; j < rx.w; ++j) {
            const unsigned long long o = at + j;
            if (o < p.out.cap) {
                p.out.pos[o] = end;
                p.out.ids[o] = __ldg(p.dups + rx.z + (j - ru.w));
            }
        }
        if (rx.x == kNoKeyword) break;
        rx = ru;
    }
}

template <typename GT>
__global__ void __launch_bounds__(kFullThreads) full_gather(const FullParams p) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    // units gw, gw + nwarps, ... (grid stride), 32 per round, only those with
    // results visited
    for (uint64_t u0 = gw; u0 < p.units; u0 += 32ull * nwarps) {
        const uint64_t uu = u0 + static_cast<uint64_t>(lane) * nwarps;
        const uint32_t cu = uu < p.units ? __ldg(p.counts + uu) : 0u;
        for (uint32_t todo = __ballot_sync(kFull, cu != 0); todo; todo &= todo - 1) {
            const uint32_t b = static_cast<uint32_t>(__ffs(todo) - 1);
            const uint32_t u = static_cast<uint32_t>(u0 + static_cast<uint64_t>(b) * nwarps);
            const uint32_t c = __shfl_sync(kFull, cu, static_cast<int>(b));
            unsigned long long o = __ldg(p.fprefix + u);
            if (c <= kSlotCap) {
                // the slots in any order: a result's place is the chain lengths
                // of the results at smaller positions
                const unsigned long long e = static_cast<uint32_t>(lane) < c
                                                 ? __ldg(p.slots + static_cast<uint64_t>(u) * kSlotCap + lane)
                                                 : ~0ull;
                const uint32_t pos = static_cast<uint32_t>(e), id = static_cast<uint32_t>(e >> 32);
                const uint32_t cl = static_cast<uint32_t>(lane) < c ? chain_len(p, id) : 0u;
                unsigned long long off = 0;
#pragma unroll 8
                for (int d = 0; d < 32; ++d) {
                    const uint32_t op = __shfl_sync(kFull, pos, d), oc = __shfl_sync(kFull, cl, d);
                    off += op < pos ? oc : 0u;
                }
                if (static_cast<uint32_t>(lane) < c) put_chain(p, o + off, pos, id);
            } else {
                // eight rows of 32 at a time: their id and chain-length loads
                // overlap, then each row is scanned and written
                const int64_t gpb = static_cast<int64_t>(u) * p.tile - p.head;
                for (uint32_t i0 = 0; i0 < p.tile; i0 += 32 * kRows) {
                    int id[kRows];
                    uint32_t cl[kRows];
#pragma unroll
                    for (uint32_t j = 0; j < kRows; ++j)
                        id[j] = i0 + 32 * j < p.tile ? dense_id<GT>(p, u, gpb, i0 + 32 * j + lane) : -1;
#pragma unroll
                    for (uint32_t j = 0; j < kRows; ++j)
                        cl[j] = id[j] >= 0 ? chain_len(p, static_cast<uint32_t>(id[j])) : 0u;
#pragma unroll
                    for (uint32_t j = 0; j < kRows; ++j) {
                        uint32_t inc = cl[j];
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, inc, d);
                            if (lane >= d) inc += y;
                        }
                        if (id[j] >= 0)
                            put_chain(p, o + (inc - cl[j]), static_cast<uint32_t>(gpb + i0 + 32 * j + lane),
                                      static_cast<uint32_t>(id[j]));
                        o += __shfl_sync(kFull, inc, 31);
                    }
                }
            }
        }
    }
    if (gw == 0 && lane == 0) *p.out.count = __ldg(p.fprefix + p.units - 1) + __ldg(p.fcounts + p.units - 1);
}

inline size_t round16(size_t v) { return (v + 15u) & ~static_cast<size_t>(15u); }

}  // namespace

// Layout: the compacted output's scratch (with its dense fallback, or without
// it when the phased form's lists follow) | occurrence counts (4 per unit) |
// their prefix (8 per unit) | partial sums (8 * kScanCtas) | the lists.
size_t full_scratch_bytes(const DevTables &t, const Tuning &tu, uint32_t units, uint64_t n) {
    const size_t U = units;
    SurvivorLists sl;
    if (uses_filter(t, tu)) sl = survivor_lists(t, tu, n, true);
    const bool dense = sl.list_cap == 0;
    return round16(round16(compact_scratch_bytes(t, units, dense)) + round16(4 * U) + 8 * U +
                   8 * static_cast<size_t>(kScanCtas)) +
           sl.bytes();
}

cudaError_t enqueue_full(const DevTables &t, const Tuning &tu, const uint8_t *text, uint64_t n,
                         const CompactOut &out, void *scratch, size_t scratch_bytes, cudaStream_t stream) {
    const uint32_t U = compact_units(t, tu, text, n);
    if (U == 0xFFFFFFFFu || n == 0 || n > 0xFFFFFFFFull || !t.full_rec || !t.full_dups)
        return cudaErrorInvalidValue;
    if (!scratch || scratch_bytes < full_scratch_bytes(t, tu, U, n)) return cudaErrorInvalidValue;
    SurvivorLists sl;
    if (uses_filter(t, tu)) sl = survivor_lists(t, tu, n, true);
    const bool dense = sl.list_cap == 0;
    uint8_t *b = static_cast<uint8_t *>(scratch);
    // the compacted output's layout (compact.cu): tile counter | counts | prefix | slots | partials | dense
    uint32_t *counts = reinterpret_cast<uint32_t *>(b + 16);
    unsigned long long *slots =
        reinterpret_cast<unsigned long long *>(b + 16 + round16(4 * size_t(U))) + static_cast<size_t>(U);
    int32_t *dn = dense ? reinterpret_cast<int32_t *>(b + compact_dense_offset(U)) : nullptr;
    uint8_t *f = b + round16(compact_scratch_bytes(t, U, dense));
    uint32_t *fcounts = reinterpret_cast<uint32_t *>(f);
    unsigned long long *fprefix = reinterpret_cast<unsigned long long *>(f + round16(4 * size_t(U)));
    unsigned long long *fpartials = fprefix + U;

    cudaError_t e = cudaMemsetAsync(b, 0, 16 + 4 * size_t(U), stream);
    if (e != cudaSuccess) return e;
    MatchRequest r;
    r.text = text;
    r.n = n;
    r.slots.counts = counts;
    r.slots.slots = slots;
    r.slots.ubase = 0;
    r.slots.dense = dn;
    r.scratch = b;
    r.scratch_bytes = 16;
    if (!dense) {  // the phased form's lists after the rest
        uint8_t *lb = f + round16(round16(4 * size_t(U)) + 8 * size_t(U) + 8 * static_cast<size_t>(kScanCtas));
        e = cudaMemsetAsync(lb, 0, 32, stream);
        if (e != cudaSuccess) return e;
        set_lists(r, lb, sl);
    }
    e = launch_match(t, r, OUT_SLOTS, tu, stream);
    if (e != cudaSuccess) return e;

    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    FullParams p{};
    p.G = t.G;
    p.cls8 = t.cls8;
    p.W = t.W;
    p.C = t.C;
    p.maxlen = t.maxlen;
    p.skip = t.skip;
    p.chain = t.chain;
    p.s_chain = t.skip ? t.s_chain : 0xFFFFFFFFu;
    p.text = text;
    p.n = n;
    p.units = U;
    p.tile = unit_positions(t, tu);
    p.head = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(text) & 15u);
    p.max_clen = t.full_max_clen;
    p.nkw = t.nkw;
    p.counts = counts;
    p.slots = slots;
    p.dense = dn;
    p.fcounts = fcounts;
    p.fprefix = fprefix;
    p.rec = t.full_rec;
    p.dups = t.full_dups;
    p.out = out;
    e = device_error_word(&p.err);
    if (e != cudaSuccess) return e;
    const uint32_t per_cta = kFullThreads / 32;
    uint32_t grid = static_cast<uint32_t>(sms) * 8u;  // grid-stride over units
    const uint32_t need = (U + per_cta - 1) / per_cta;
    if (grid > need) grid = need;
    if (t.gbits == 16)
        full_count<int16_t><<<grid, kFullThreads, 0, stream>>>(p);
    else
        full_count<int32_t><<<grid, kFullThreads, 0, stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_compact_scan(fcounts, U, nullptr, fprefix, fpartials, stream);
    if (e != cudaSuccess) return e;
    if (t.gbits == 16)
        full_gather<int16_t><<<grid, kFullThreads, 0, stream>>>(p);
    else
        full_gather<int32_t><<<grid, kFullThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace pfac
