// pfac_jump8 -- failureless Aho-Corasick for large alphabets (8-bit codes),
// one thread per start position at high occupancy, sm_103a.
//
// The GPU design of the paper (section I, Fig. 3: every position its own
// thread, walking the goto table) with three changes for GB300:
//   * the text is staged per warp tile (1024 positions + 16-byte halo) by one
//     bulk async copy (the TMA unit), two tiles in flight per warp, so the
//     windows and most walk bytes come from shared memory;
//   * the first two levels of every walk are one lookup in the root jump table
//     (2-byte windows, int16, resident in shared memory for the whole kernel);
//   * the walk continues through the goto table with the rows of the first
//     levels kept in L2 (evict-last loads); 32 warps per SM hide its latency,
//     and each thread carries two walks (positions i and i + 512 of the tile)
//     so their loads overlap.
// Output per position is written coalesced: dense ids, a count, or slots (per
// tile the number of matches and the first kSlotCap of them) for compact.cu.
// Work units are the tiles of one text, or of all texts of one automaton in a
// batch (the planned list), claimed from a global counter.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

namespace {

constexpr int kBlock = 1024;
constexpr int kWarps = kBlock / 32;
constexpr int kStages = 2;
constexpr uint32_t kTile = 1024;             // positions per warp tile
constexpr uint32_t kHalf = kTile / 2;        // the second walk of a thread is 512 positions on
constexpr uint32_t kStaged = kTile + 16;     // staged bytes per tile
constexpr uint32_t kOffBar = 0;              // kWarps * kStages mbarriers + the table barrier
constexpr uint32_t kOffTile = kOffBar + (kWarps * kStages + 1) * 8;   // stage unit + item
constexpr uint32_t kOffCls = 1152;                                    // after the stage descriptors
constexpr uint32_t kOffJ = 1408;
static_assert(kOffTile + kWarps * kStages * 8 <= kOffCls, "stage descriptors overlap the class map");
constexpr unsigned kFull = 0xffffffffu;

struct JumpParams {
    const uint8_t *text;    // batch: base of all texts
    uint64_t n;
    const BatchHead *batch;
    const BatchItemDev *lists;
    uint32_t ntiles;
    const void *G;
    const int16_t *Jg;
    const uint8_t *cls8g;
    uint32_t C, W, k, base_k, maxlen, jbytes;
    int32_t *out;
    unsigned long long *count;
    SlotOut sl;
    unsigned int *counter;
    unsigned int *err;
    uint32_t off_stage;     // first stage buffer
    uint32_t global;        // 1: pfac_jump8g (tables and text through L1)
    uint32_t sms;
    uint32_t rows;          // pfac_jump8g: rows of a tile per claim (1 or 16)
    unsigned long long wait_ns;  // bounded waits give up after this
};

__device__ __forceinline__ TileText tile_text(const JumpParams &p, const Work &wk, uint32_t u, uint32_t item) {
    if (!wk.list) return make_text(p.text, p.out, p.n, u);
    return batch_text(wk, p.text, p.out, item, u);
}

__device__ __forceinline__ void issue_unit(const JumpParams &p, const Work &wk, uint64_t *bar, uint32_t *stile,
                                           uint8_t *st, uint32_t u, int lane) {
    const uint32_t item = (wk.list && u < wk.units) ? find_item(wk, u, lane) : 0u;
    if (lane == 0) {
        stile[0] = u;
        stile[1] = item;
        if (u >= wk.units)
            mbar_arrive(bar);
        else
            issue_text_tile(tile_text(p, wk, u, item), kTile, kStaged, bar, st);
    }
}

template <bool INV>
__device__ __forceinline__ uint32_t column_of(const JumpParams &p, const uint8_t *cls8, uint32_t b) {
    if (!INV) return b;
    const uint32_t v = cls8[b];
    return v != 0xFFu ? v : p.C;
}

// The byte at tile index q: staged (STAGED, q inside the stage) or from global
// memory.
template <bool STAGED>
__device__ __forceinline__ uint32_t byte_at(const TileText &tt, const uint8_t *st, int64_t gpb, uint32_t q) {
    if (STAGED && q < kStaged) return st[q];
    return __ldg(tt.text + gpb + q);
}

// Root jump-table entry idx: from shared memory (STAGED) or through L1.
template <bool STAGED>
__device__ __forceinline__ int jump_load(const JumpParams &p, const uint8_t *jbase, uint32_t idx) {
    if (STAGED) return *reinterpret_cast<const int16_t *>(jbase + 2u * idx);
    return __ldg(p.Jg + idx);
}

// The result of the walk from position i of the tile (valid, inside the text).
// Two walks advance together so their goto loads overlap.
template <bool INV, typename GT, bool STAGED>
__device__ __forceinline__ void walk2(const JumpParams &p, const TileText &tt, const uint8_t *st,
                                      const uint8_t *cls8, const uint8_t *jbase, int64_t gpb, uint64_t keep,
                                      const uint32_t i[2], const bool ok[2], int r[2]) {
    const GT *G = static_cast<const GT *>(p.G);
    const int64_t n = static_cast<int64_t>(tt.n);
    uint32_t state[2], q[2];
    bool live[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        r[t] = -1;
        live[t] = false;
        state[t] = 0;
        q[t] = i[t];
        if (!ok[t]) continue;
        const int64_t gp = gpb + i[t];
        int v = kJumpSlow;
        if (p.k == 2 && gp + 2 <= n) {
            const uint32_t b0 = byte_at<STAGED>(tt, st, gpb, i[t]), b1 = byte_at<STAGED>(tt, st, gpb, i[t] + 1);
            const uint32_t c0 = INV ? cls8[b0] : b0;
            const uint32_t c1 = INV ? cls8[b1] : b1;
            v = jump_load<STAGED>(p, jbase, c0 | (c1 << 8));
        } else if (p.k == 1 && gp + 1 <= n) {
            const uint32_t b0 = byte_at<STAGED>(tt, st, gpb, i[t]);
            v = jump_load<STAGED>(p, jbase, INV ? cls8[b0] : b0);
        }
        if (v >= -1) {
            r[t] = v;
        } else {
            live[t] = true;
            if (v != kJumpSlow) {
                state[t] = p.base_k + static_cast<uint32_t>(-v - 2);
                q[t] = i[t] + p.k;
            }
        }
    }
    for (uint32_t step = 0; live[0] || live[1]; ++step) {
        int e[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (live[t]) {
                const int64_t gq = gpb + q[t];
                const uint32_t c = gq < n ? column_of<INV>(p, cls8, byte_at<STAGED>(tt, st, gpb, q[t])) : p.C;
                e[t] = goto_ld_hint(G, state[t], p.W, c, keep);
            }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (live[t]) {
                if (e[t] < 0 || static_cast<uint32_t>(e[t]) <= state[t] || step > p.maxlen + 1) {
                    if (e[t] >= 0) {
                        atomicOr(p.err, static_cast<unsigned>(kErrWalk));
                        r[t] = -1;
                    } else {
                        r[t] = decode_dead(e[t]);
                    }
                    live[t] = false;
                } else {
                    state[t] = static_cast<uint32_t>(e[t]);
                    q[t] += 1;
                }
            }
        }
    }
}

// walk2 for the full-occupancy form: bytes through L1 by pointer, 32-bit row
// offsets (the launcher checks S * W < 2^32), one signed compare per step to
// end a walk (a dead entry is negative; a live one must be a larger state).
template <bool INV, typename GT>
__device__ __forceinline__ void walk2g(const JumpParams &p, const TileText &tt, const uint8_t *cls8, int64_t gpb,
                                       uint64_t keep, const uint32_t i[2], const bool ok[2], int r[2]) {
    const GT *G = static_cast<const GT *>(p.G);
    uint32_t state[2], rem[2];
    const uint8_t *tp[2];
    uint32_t live = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        r[t] = -1;
        state[t] = 0;
        rem[t] = 0;
        tp[t] = tt.text;
        if (!ok[t]) continue;
        const uint64_t gp = static_cast<uint64_t>(gpb + i[t]);
        const uint64_t left = tt.n - gp;
        int v = kJumpSlow;
        if (p.k == 2 && left >= 2) {
            const uint32_t b0 = __ldg(tt.text + gp), b1 = __ldg(tt.text + gp + 1);
            v = __ldg(p.Jg + ((INV ? cls8[b0] : b0) | ((INV ? cls8[b1] : b1) << 8)));
        } else if (p.k == 1 && left >= 1) {
            const uint32_t b0 = __ldg(tt.text + gp);
            v = __ldg(p.Jg + (INV ? cls8[b0] : b0));
        }
        uint32_t d = 0;
        if (v >= -1) {
            r[t] = v;
        } else {
            live |= 1u << t;
            if (v != kJumpSlow) {
                state[t] = p.base_k + static_cast<uint32_t>(-v - 2);
                d = p.k;
            }
        }
        tp[t] = tt.text + gp + d;
        rem[t] = left - d > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(left - d);
    }
    while (live) {
        int e[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if ((live >> t) & 1u) {
                const uint32_t c = rem[t] ? column_of<INV>(p, cls8, __ldg(tp[t])) : p.C;
                int v;
                if (sizeof(GT) == 4) {
                    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;"
                        : "=r"(v)
                        : "l"(G + (state[t] * p.W + c)), "l"(keep));
                } else {
                    short h;
                    asm("ld.global.nc.L2::cache_hint.s16 %0, [%1], %2;"
                        : "=h"(h)
                        : "l"(G + (state[t] * p.W + c)), "l"(keep));
                    v = h;
                }
                e[t] = v;
            }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if ((live >> t) & 1u) {
                if (e[t] <= static_cast<int>(state[t])) {
                    if (e[t] >= 0) {
                        atomicOr(p.err, static_cast<unsigned>(kErrWalk));
                        r[t] = -1;
                    } else {
                        r[t] = decode_dead(e[t]);
                    }
                    live &= ~(1u << t);
                } else {
                    state[t] = static_cast<uint32_t>(e[t]);
                    tp[t] += 1;
                    rem[t] -= 1;
                }
            }
        }
    }
}

// The results of one row of a tile (positions i[0], i[1] of every lane):
// dense ids (coalesced), a count, or the tile's match slots.
template <int MODE>
__device__ __forceinline__ void put2(const JumpParams &p, const TileText &tt, int64_t gpb, uint32_t su,
                                     const uint32_t i[2], const bool in[2], const int r[2], int lane,
                                     unsigned long long &cnt) {
    if (MODE == OUT_DENSE) {
#pragma unroll
        for (int t = 0; t < 2; ++t)
            if (in[t]) __stcs(tt.out + gpb + i[t], r[t]);
    } else if (MODE == OUT_COUNT) {
        cnt += (in[0] && r[0] >= 0 ? 1u : 0u) + (in[1] && r[1] >= 0 ? 1u : 0u);
    } else {
        if (p.sl.dense) {  // the tile may overflow its slots: keep its dense ids
#pragma unroll
            for (int t = 0; t < 2; ++t)
                if (in[t]) __stcs(p.sl.dense + static_cast<uint64_t>(su) * kDenseStride + i[t], r[t]);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const bool hit = in[t] && r[t] >= 0;
            const unsigned m = __ballot_sync(kFull, hit);
            if (m) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(p.sl.counts + su, __popc(m));
                base = __shfl_sync(kFull, base, 0) + __popc(m & ((1u << lane) - 1u));
                if (hit && base < kSlotCap)
                    p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + base] =
                        (static_cast<unsigned long long>(static_cast<uint32_t>(r[t])) << 32) |
                        static_cast<uint32_t>(gpb + i[t]);
            }
        }
    }
}

template <bool INV, typename GT, int MODE, bool BATCH>
__global__ void __launch_bounds__(kBlock, 1) pfac_jump8(const JumpParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t *jbar = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint64_t *bars = jbar + 1 + warp * kStages;
    uint32_t *stile = reinterpret_cast<uint32_t *>(smem + kOffTile) + warp * kStages * 2;
    uint8_t *stages = smem + p.off_stage + static_cast<size_t>(warp) * kStages * kStaged;
    const uint8_t *cls8 = smem + kOffCls;
    const uint8_t *jbase = smem + kOffJ;
    const Work wk = BATCH ? load_work(p.batch, p.lists, p.ntiles) : load_work(nullptr, nullptr, p.ntiles);

    if (threadIdx.x == 0) {
        for (int i = 0; i < 1 + nw * kStages; ++i) mbar_init(&jbar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(jbar, 256u + p.jbytes);
        bulk_load(smem + kOffCls, p.cls8g, 256u, jbar);
        if (p.jbytes) bulk_load(smem + kOffJ, p.Jg, p.jbytes, jbar);
    }
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nw;
    UnitClaims claims = claims_start(gw, GW);
    auto next_tile = [&](uint32_t) -> uint32_t {  // all lanes
        uint32_t t = 0xFFFFFFFFu;
        if (lane == 0) {
            const uint64_t c = claims_next(claims, p.counter, wk.units);
            if (c < wk.units) t = static_cast<uint32_t>(c);
        }
        return __shfl_sync(kFull, t, 0);
    };
    for (uint32_t s = 0; s < kStages; ++s)
        issue_unit(p, wk, &bars[s], stile + 2 * s, stages + s * kStaged, next_tile(s), lane);

    const uint64_t keep = policy_evict_last();
    unsigned long long cnt = 0;
    bool ok = mbar_wait(jbar, 0, p.wait_ns);
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % kStages;
        ok = ok && mbar_wait(&bars[s], (it / kStages) & 1u, p.wait_ns);
        if (!__all_sync(kFull, ok)) {
            if (lane == 0) {
                atomicOr(p.err, static_cast<unsigned>(kErrTimeout));
                mbar_wait(jbar, 0, p.wait_ns);
                for (uint32_t j = it; j < it + kStages; ++j)
                    mbar_wait(&bars[j % kStages], (j / kStages) & 1u, p.wait_ns);
            }
            return;
        }
        const uint32_t tile = stile[2 * s];
        if (tile >= wk.units) break;
        const TileText tt = tile_text(p, wk, tile, stile[2 * s + 1]);
        uint8_t *st = stages + s * kStaged;
        const uint64_t tlo = static_cast<uint64_t>(tt.tile) * kTile;
        const int64_t gpb = static_cast<int64_t>(tlo) - tt.head;
        const int64_t n = static_cast<int64_t>(tt.n);
        const bool interior = gpb >= 0 && gpb + static_cast<int64_t>(kStaged) <= n;
        if (!interior) {
            load_text_fringe(tt, kStaged, st, tlo, lane);
            __syncwarp();
        }
        const uint32_t su = p.sl.ubase + tile;
        for (uint32_t j = 0; j < kHalf / 32; ++j) {
            uint32_t i[2];
            bool in[2];
            i[0] = 32u * j + static_cast<uint32_t>(lane);
            i[1] = i[0] + kHalf;
#pragma unroll
            for (int t = 0; t < 2; ++t) in[t] = gpb + static_cast<int64_t>(i[t]) >= 0 && gpb + static_cast<int64_t>(i[t]) < n;
            int r[2];
            walk2<INV, GT, true>(p, tt, st, cls8, jbase, gpb, keep, i, in, r);
            put2<MODE>(p, tt, gpb, su, i, in, r, lane, cnt);
        }
        __syncwarp();
        if (lane == 0) fence_proxy_async_smem();
        issue_unit(p, wk, &bars[s], stile + 2 * s, st, next_tile(it + kStages), lane);
    }
    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

// The same walks at full occupancy: no shared-memory tables or stages (the
// jump table and the text are read through L1), 256-thread CTAs, 8 per SM
// (32 registers a thread).  Chain records are not used here: their logic
// costs the registers of that occupancy, which measured the larger win.
constexpr int kBlockG = 256;
constexpr int kCtasG = 8;

template <bool INV, typename GT, int MODE, bool BATCH>
__global__ void __launch_bounds__(kBlockG, kCtasG) pfac_jump8g(const JumpParams p) {
    __shared__ uint8_t cls8[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const Work wk = BATCH ? load_work(p.batch, p.lists, p.ntiles) : load_work(nullptr, nullptr, p.ntiles);
    if (INV)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) cls8[i] = __ldg(p.cls8g + i);
    __syncthreads();
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nw;
    const uint64_t keep = policy_evict_last();
    unsigned long long cnt = 0;
    // A claim is p.rows rows (16 = a whole tile; 1 for small texts, so that
    // their few tiles spread over many warps).
    const uint32_t rows = p.rows;
    const uint64_t claims = static_cast<uint64_t>(wk.units) * (kHalf / 32) / rows;
    for (uint32_t it = 0;; ++it) {
        uint32_t claim = 0xFFFFFFFFu;
        if (lane == 0) {
            // no claims beyond the warps' first: the counter is not touched
            const uint64_t c = it == 0 ? gw : (GW >= claims || !p.counter ? claims : GW + atomicAdd(p.counter, 1u));
            if (c < claims) claim = static_cast<uint32_t>(c);
        }
        claim = __shfl_sync(kFull, claim, 0);
        if (claim == 0xFFFFFFFFu) break;
        const uint32_t row0 = claim * rows;
        const uint32_t tile = row0 / (kHalf / 32);
        const uint32_t item = wk.list ? find_item(wk, tile, lane) : 0u;
        const TileText tt = tile_text(p, wk, tile, item);
        const int64_t gpb = static_cast<int64_t>(tt.tile) * kTile - tt.head;
        const int64_t n = static_cast<int64_t>(tt.n);
        const uint32_t su = p.sl.ubase + tile;
        const uint32_t j0 = row0 % (kHalf / 32);
        for (uint32_t j = j0; j < j0 + rows; ++j) {
            uint32_t i[2];
            bool in[2];
            i[0] = 32u * j + static_cast<uint32_t>(lane);
            i[1] = i[0] + kHalf;
#pragma unroll
            for (int t = 0; t < 2; ++t)
                in[t] = gpb + static_cast<int64_t>(i[t]) >= 0 && gpb + static_cast<int64_t>(i[t]) < n;
            int r[2];
            walk2g<INV, GT>(p, tt, cls8, gpb, keep, i, in, r);
            put2<MODE>(p, tt, gpb, su, i, in, r, lane, cnt);
        }
    }
    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

template <bool INV, typename GT, int MODE, bool BATCH>
cudaError_t launch_one(const JumpParams &p, uint32_t grid, uint32_t smem, int max_smem, cudaStream_t stream) {
    if (p.global) {
        const uint32_t g = p.sms * static_cast<uint32_t>(kCtasG);
        pfac_jump8g<INV, GT, MODE, BATCH><<<grid < g ? grid : g, kBlockG, 0, stream>>>(p);
        return cudaGetLastError();
    }
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void (*kernel)(const JumpParams) = pfac_jump8<INV, GT, MODE, BATCH>;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    kernel<<<grid, kBlock, smem, stream>>>(p);
    return cudaGetLastError();
}

template <bool INV, typename GT>
cudaError_t launch_modes(OutMode mode, const JumpParams &p, uint32_t grid, uint32_t smem, int max_smem,
                         cudaStream_t stream) {
    switch (mode) {
        case OUT_DENSE:
            return p.batch ? launch_one<INV, GT, OUT_DENSE, true>(p, grid, smem, max_smem, stream)
                           : launch_one<INV, GT, OUT_DENSE, false>(p, grid, smem, max_smem, stream);
        case OUT_COUNT:
            return launch_one<INV, GT, OUT_COUNT, false>(p, grid, smem, max_smem, stream);
        case OUT_SLOTS:
            return p.batch ? launch_one<INV, GT, OUT_SLOTS, true>(p, grid, smem, max_smem, stream)
                           : launch_one<INV, GT, OUT_SLOTS, false>(p, grid, smem, max_smem, stream);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace

uint32_t jump8_tile_positions() { return kTile; }

cudaError_t launch_jump8(const DevTables &t, const MatchRequest &r, OutMode mode, bool global,
                         unsigned long long wait_ns, cudaStream_t stream) {
    if (t.B != 8 || t.k > 2) return cudaErrorInvalidValue;
    if (mode != OUT_DENSE && mode != OUT_COUNT && mode != OUT_SLOTS) return cudaErrorInvalidValue;
    const bool batch = r.batch != nullptr;
    if (batch && (mode == OUT_COUNT || !r.lists)) return cudaErrorInvalidValue;
    if (mode == OUT_SLOTS && (!r.slots.counts || !r.slots.slots)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    JumpParams p{};
    p.text = r.text;
    p.n = r.n;
    p.batch = r.batch;
    p.lists = r.lists;
    uint64_t tiles = 0;
    if (!batch) {
        const uint64_t head = reinterpret_cast<uintptr_t>(r.text) & 15u;
        tiles = (r.n + head + kTile - 1) / kTile;
        if (tiles >= 0x7FFFFFFFull) return cudaErrorInvalidValue;
    }
    p.ntiles = static_cast<uint32_t>(tiles);
    p.G = t.G;
    p.Jg = t.J;
    p.cls8g = t.cls8;
    p.C = t.C;
    p.W = t.W;
    p.k = t.k;
    p.base_k = t.base_k;
    p.maxlen = t.maxlen;
    p.jbytes = t.jbytes;
    p.wait_ns = wait_ns ? wait_ns : kWaitNs;
    p.out = r.out;
    p.count = r.count;
    p.sl = r.slots;
    // the claim counter; none is needed when every claim is some warp's first
    p.counter = r.scratch && r.scratch_bytes >= 16 ? static_cast<unsigned int *>(r.scratch) : nullptr;
    e = device_error_word(&p.err);
    if (e != cudaSuccess) return e;
    p.off_stage = (kOffJ + t.jbytes + 127u) & ~127u;
    const uint32_t smem = p.off_stage + kWarps * kStages * kStaged;
    if (static_cast<int>(smem) > max_smem) return cudaErrorInvalidConfiguration;
    if (global && static_cast<uint64_t>(t.S) * t.W >= (1ull << 31)) global = false;  // 32-bit row offsets
    p.global = global ? 1u : 0u;
    // small texts: one row per claim, so their few tiles spread over many warps
    p.rows = (!batch && static_cast<uint64_t>(p.ntiles) * (kHalf / 32) <= 4ull * sms * kCtasG * (kBlockG / 32u)) ? 1u
                                                                                                  : kHalf / 32;
    p.sms = static_cast<uint32_t>(sms);
    uint32_t grid = static_cast<uint32_t>(sms);
    if (global) grid = static_cast<uint32_t>(sms) * static_cast<uint32_t>(kCtasG);
    {
        const uint32_t per = global ? kBlockG / 32u : static_cast<uint32_t>(kWarps);
        const uint64_t work = global ? static_cast<uint64_t>(p.ntiles) * (kHalf / 32) / p.rows : p.ntiles;
        if (!batch) {
            const uint64_t need = (work + per - 1) / per;
            if (grid > need) grid = static_cast<uint32_t>(need);
        }
        if (!p.counter && (batch || work > static_cast<uint64_t>(grid) * per)) return cudaErrorInvalidValue;
    }
    if (grid == 0) return cudaSuccess;
    const bool inv = t.C < 256;
    if (t.gbits == 16) {
        if (inv) return launch_modes<true, int16_t>(mode, p, grid, smem, max_smem, stream);
        return launch_modes<false, int16_t>(mode, p, grid, smem, max_smem, stream);
    }
    if (inv) return launch_modes<true, int32_t>(mode, p, grid, smem, max_smem, stream);
    return launch_modes<false, int32_t>(mode, p, grid, smem, max_smem, stream);
}

}  // namespace pfac
