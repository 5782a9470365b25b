// Failureless Aho-Corasick matching kernels for sm_103a.
//
// pfac_tiled  -- the production kernel.  One persistent CTA per SM walks the
//                text tile by tile:
//   * each tile of T = 16 * blockDim positions plus a halo of max-keyword-length
//     bytes is bulk-copied (cp.async.bulk, TMA unit, no multicast) into one of
//     `stages` shared-memory buffers, tracked by an mbarrier per stage, so
//     several tiles are in flight while one is matched;
//   * the tile's bytes are mapped to class codes once and packed B bits each;
//   * every start position resolves its first k characters with ONE lookup in
//     the root jump table (the top k levels of the goto table flattened,
//     resident in shared memory for the whole kernel), survivors resolve k2
//     more with one lookup in the stride table (global, L2-resident), and the
//     rare walks that go deeper follow the goto table through L1, all walks of
//     a thread interleaved so their loads overlap;
//   * output: dense int32 ids (vectorised streaming stores), a count (one
//     atomic per warp), or the compacted (pos, id) list in ascending order
//     (block scan + decoupled look-back across tiles).
// pfac_simple -- one thread per position walking the goto table in global
//                memory: the design of the paper's GPU side (section I, Fig. 3),
//                kept as the comparison point.
#include <cuda_runtime.h>

#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

__device__ unsigned int g_dev_error = 0;

namespace {

constexpr int kPPT = 16;          // positions per thread per tile (4 groups of 4)
constexpr int kMaxStages = 8;
constexpr int kMaxBlock = 512;
constexpr uint32_t kHdrBytes = 1024;  // barriers, tile ids, scan scratch, class map

struct TiledParams {
    const uint8_t *text;
    const uint8_t *gbase;   // text rounded down to 16 bytes
    uint64_t n;
    uint32_t head;          // text - gbase
    uint32_t T, H, SL, nstages, ntiles;
    const void *G;
    const int16_t *Jg;
    const int32_t *J2;
    const int16_t *clsg;
    uint32_t C, W, k, k2, base_k, maxlen, jbytes;
    int32_t *out;
    int vec_ok;
    uint32_t *cpos;
    uint32_t *cids;
    unsigned long long cap;
    unsigned long long *count;
    unsigned long long *status;
    unsigned int *counter;
    uint32_t off_J, off_stage, off_packed, off_inv;
};

struct Smem {
    uint64_t *bars;          // [0, nstages): text stages; [kMaxStages]: tables
    uint32_t *stage_tile;
    unsigned long long *red; // 34 words: warp partials, block total, tile prefix
    int16_t *cls;
    int16_t *J;
    uint8_t *stages;
    uint32_t *packed;
    uint32_t *inv;
};

__device__ __forceinline__ Smem carve(uint8_t *smem, const TiledParams &p) {
    Smem s;
    s.bars = reinterpret_cast<uint64_t *>(smem);
    s.stage_tile = reinterpret_cast<uint32_t *>(smem + 128);
    s.red = reinterpret_cast<unsigned long long *>(smem + 192);
    s.cls = reinterpret_cast<int16_t *>(smem + 512);
    s.J = reinterpret_cast<int16_t *>(smem + p.off_J);
    s.stages = smem + p.off_stage;
    s.packed = reinterpret_cast<uint32_t *>(smem + p.off_packed);
    s.inv = reinterpret_cast<uint32_t *>(smem + p.off_inv);
    return s;
}

// Thread 0: start the bulk copy of `tile` (or mark the stage as the end).
__device__ __forceinline__ void issue_stage(const TiledParams &p, const Smem &sm, uint32_t s, uint32_t tile) {
    sm.stage_tile[s] = tile;
    uint64_t *bar = &sm.bars[s];
    if (tile >= p.ntiles) {
        mbar_arrive(bar);
        return;
    }
    const uint64_t tlo = static_cast<uint64_t>(tile) * p.T;
    const uint64_t a1 = (static_cast<uint64_t>(p.head) + 15ull) & ~15ull;
    const uint64_t a2 = (static_cast<uint64_t>(p.head) + p.n) & ~15ull;
    const uint64_t lo = tlo > a1 ? tlo : a1;
    const uint64_t hi = (tlo + p.SL) < a2 ? (tlo + p.SL) : a2;
    if (a1 < a2 && lo < hi) {
        const uint32_t bytes = static_cast<uint32_t>(hi - lo);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load(sm.stages + static_cast<size_t>(s) * p.SL + (lo - tlo), p.gbase + lo, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

// Warp 0: the unaligned head and tail bytes of the text that the bulk copy
// leaves out (at most 15 each).
__device__ __forceinline__ void load_fringe(const TiledParams &p, uint8_t *st, uint64_t tlo, int lane) {
    const uint64_t head = p.head, end = head + p.n;
    const uint64_t a1 = (head + 15ull) & ~15ull, a2 = end & ~15ull;
    uint64_t lo, hi;
    if (lane < 16) {
        lo = head;
        hi = a1 < end ? a1 : end;
    } else {
        lo = a1 > a2 ? a1 : a2;
        hi = end;
    }
    if (lo < tlo) lo = tlo;
    if (hi > tlo + p.SL) hi = tlo + p.SL;
    const uint64_t idx = lo + static_cast<uint64_t>(lane & 15);
    if (idx < hi) st[idx - tlo] = p.gbase[idx];
}

// Map the staged bytes to class codes (packed B bits per position) and record
// positions that cannot extend a walk (byte in no keyword, or outside the text).
template <int B>
__device__ __forceinline__ void convert_stage(const TiledParams &p, const Smem &sm, uint8_t *st, int64_t gpb,
                                              int tid, int nt) {
    uint16_t *inv16 = reinterpret_cast<uint16_t *>(sm.inv);
    const int64_t n = static_cast<int64_t>(p.n);
    const uint32_t chunks = p.SL / 16;
    for (uint32_t c = tid; c < chunks; c += nt) {
        const uint4 v = reinterpret_cast<const uint4 *>(st)[c];
        const int64_t gp0 = gpb + 16 * static_cast<int64_t>(c);
        const bool inside = gp0 >= 0 && gp0 + 16 <= n;
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t ib = 0;
        uint64_t pk = 0;
        uint32_t o[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const uint32_t byte = (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
            const int cv = sm.cls[byte];
            const bool valid = cv >= 0 && (inside || (gp0 + b >= 0 && gp0 + b < n));
            const uint32_t code = valid ? static_cast<uint32_t>(cv) : 0u;
            ib |= (valid ? 0u : 1u) << b;
            if (B == 8)
                o[b >> 2] |= code << (8 * (b & 3));
            else
                pk |= static_cast<uint64_t>(code) << (B * b);
        }
        if (B == 2) {
            sm.packed[c] = static_cast<uint32_t>(pk);
        } else if (B == 4) {
            sm.packed[2 * c] = static_cast<uint32_t>(pk);
            sm.packed[2 * c + 1] = static_cast<uint32_t>(pk >> 32);
        } else {
            reinterpret_cast<uint4 *>(st)[c] = make_uint4(o[0], o[1], o[2], o[3]);
        }
        inv16[c] = static_cast<uint16_t>(ib);
    }
}

// Code of stage position q, false when q cannot extend a walk.
template <int B, bool INV>
__device__ __forceinline__ bool fetch_code(const TiledParams &p, const Smem &sm, const uint8_t *st, int64_t gpb,
                                           uint32_t q, uint32_t &c) {
    if (q < p.SL) {
        if (INV) {
            if ((sm.inv[q >> 5] >> (q & 31u)) & 1u) return false;
        } else {
            if (gpb + static_cast<int64_t>(q) >= static_cast<int64_t>(p.n)) return false;
        }
        if (B == 8)
            c = st[q];
        else
            c = (sm.packed[(B * q) >> 5] >> ((B * q) & 31u)) & ((1u << B) - 1u);
        return true;
    }
    const int64_t gp = gpb + static_cast<int64_t>(q);
    if (gp >= static_cast<int64_t>(p.n)) return false;
    const int v = sm.cls[__ldg(p.text + gp)];
    if (v < 0) return false;
    c = static_cast<uint32_t>(v);
    return true;
}

__device__ __forceinline__ void block_exclusive_scan(unsigned long long v, unsigned long long &excl,
                                                     unsigned long long &total, unsigned long long *red, int tid,
                                                     int nt) {
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    unsigned long long inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) red[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < nw ? red[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < nw) red[lane] = wi - w;
        if (lane == nw - 1) red[32] = wi;
    }
    __syncthreads();
    excl = red[warp] + inc - v;
    total = red[32];
}

// Thread 0: decoupled look-back over the per-tile status words.  Returns the
// number of matches in all earlier tiles.
__device__ __forceinline__ unsigned long long lookback(unsigned long long *status, uint32_t tile,
                                                       unsigned long long total) {
    constexpr unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kVal = (1ull << 62) - 1ull;
    if (tile == 0) {
        st_relaxed(&status[0], kPre | total);
        return 0ull;
    }
    st_relaxed(&status[tile], kAgg | total);
    unsigned long long excl = 0;
    int64_t pred = static_cast<int64_t>(tile) - 1;
    unsigned long long t0 = 0;
    while (pred >= 0) {
        const unsigned long long v = ld_relaxed(&status[pred]);
        const unsigned long long f = v >> 62;
        if (f == 0) {
            const unsigned long long now = global_timer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitNs) {
                atomicOr(&g_dev_error, kErrLookback);
                break;
            }
            continue;
        }
        excl += v & kVal;
        if (f == 2) break;
        --pred;
        t0 = 0;
    }
    st_relaxed(&status[tile], kPre | (excl + total));
    return excl;
}

template <int B, bool INV, typename GT, int MODE>
__device__ __forceinline__ void match_tile(const TiledParams &p, const Smem &sm, const uint8_t *st, uint32_t tile,
                                           int tid, int nt, unsigned long long &cnt) {
    const GT *G = static_cast<const GT *>(p.G);
    const int64_t n = static_cast<int64_t>(p.n);
    const int64_t gpb = static_cast<int64_t>(tile) * p.T - p.head;  // text index of stage position 0
    const uint32_t k = p.k, k2 = p.k2;
    const uint32_t kmask = (1u << (B * k)) - 1u;
    const uint32_t kbits = (1u << k) - 1u;
    const uint32_t k2mask = (1u << (B * k2)) - 1u;
    const uint32_t k2bits = (1u << k2) - 1u;

    int res[kPPT];
    int stt[kPPT];       // >= 0: state still walking; -1: done
    uint32_t q[kPPT];    // stage position of the next character
    uint64_t x[4];       // codes of the group's window, position i0 in the low bits
    uint64_t ivx[4];     // "cannot extend" bits of the same window

    // 1. root jump table: first k characters in one shared-memory lookup
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint32_t i0 = 4u * static_cast<uint32_t>(g * nt + tid);
        if (B == 8) {
            const uint32_t *s32 = reinterpret_cast<const uint32_t *>(st);
            x[g] = static_cast<uint64_t>(s32[i0 >> 2]) | (static_cast<uint64_t>(s32[(i0 >> 2) + 1]) << 32);
        } else {
            const uint32_t bo = B * i0, w = bo >> 5, sh = bo & 31u;
            x[g] = (static_cast<uint64_t>(sm.packed[w]) | (static_cast<uint64_t>(sm.packed[w + 1]) << 32)) >> sh;
        }
        if (INV) {
            const uint32_t w = i0 >> 5, sh = i0 & 31u;
            ivx[g] = (static_cast<uint64_t>(sm.inv[w]) | (static_cast<uint64_t>(sm.inv[w + 1]) << 32)) >> sh;
        } else {
            ivx[g] = 0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = 4 * g + r;
            const int64_t gp = gpb + i0 + r;
            res[j] = -1;
            stt[j] = -1;
            q[j] = i0 + r;
            if (gp < 0 || gp >= n) continue;
            const bool wok = (k > 0) && (INV ? (((ivx[g] >> r) & kbits) == 0) : (gp + k <= n));
            if (!wok) {
                stt[j] = 0;
                continue;
            }
            const int e = sm.J[static_cast<uint32_t>(x[g] >> (B * r)) & kmask];
            if (e >= 0) {
                stt[j] = static_cast<int>(p.base_k) + e;
                q[j] += k;
            } else if (e == kJumpSlow) {
                stt[j] = 0;
            } else {
                res[j] = decode_dead(e);
            }
        }
    }

    // 2. stride table: k2 more characters for the starts still alive at depth k
    if (k2 > 0) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint32_t i0 = 4u * static_cast<uint32_t>(g * nt + tid);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int j = 4 * g + r;
                if (stt[j] > 0) {
                    const int64_t gp = gpb + i0 + r;
                    const bool wok =
                        INV ? (((ivx[g] >> (r + k)) & k2bits) == 0) : (gp + static_cast<int64_t>(k + k2) <= n);
                    if (wok) {
                        const uint32_t row = static_cast<uint32_t>(stt[j]) - p.base_k;
                        const uint32_t w2 = static_cast<uint32_t>(x[g] >> (B * (r + k))) & k2mask;
                        const int e2 = __ldg(p.J2 + ((static_cast<uint64_t>(row) << (B * k2)) | w2));
                        if (e2 >= 0) {
                            stt[j] = e2;
                            q[j] += k2;
                        } else {
                            res[j] = decode_dead(e2);
                            stt[j] = -1;
                        }
                    }
                }
            }
        }
    }

    // 3. deeper walks through the goto table, all of this thread's walks
    //    advanced together one character per round
    bool active = false;
#pragma unroll
    for (int j = 0; j < kPPT; ++j) active |= stt[j] >= 0;
    for (uint32_t round = 0; __any_sync(0xffffffffu, active); ++round) {
        if (round > p.maxlen + 1) {  // impossible for a well-formed table
            if (active) atomicOr(&g_dev_error, static_cast<unsigned>(kErrWalk));
#pragma unroll
            for (int j = 0; j < kPPT; ++j)
                if (stt[j] >= 0) stt[j] = -1;
            break;
        }
        active = false;
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            if (stt[j] >= 0) {
                const uint32_t s = static_cast<uint32_t>(stt[j]);
                uint32_t c = 0;
                if (!fetch_code<B, INV>(p, sm, st, gpb, q[j], c)) {
                    res[j] = decode_dead(goto_ld(G, s, p.W, p.C));
                    stt[j] = -1;
                } else {
                    const int t = goto_ld(G, s, p.W, c);
                    if (t < 0) {
                        res[j] = decode_dead(t);
                        stt[j] = -1;
                    } else {
                        stt[j] = t;
                        q[j] += 1;
                        active = true;
                    }
                }
            }
        }
    }

    // 4. output
    if (MODE == OUT_DENSE) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint32_t i0 = 4u * static_cast<uint32_t>(g * nt + tid);
            const int64_t gp0 = gpb + i0;
            if (p.vec_ok && gp0 >= 0 && gp0 + 4 <= n) {
                __stcs(reinterpret_cast<int4 *>(p.out + gp0),
                       make_int4(res[4 * g], res[4 * g + 1], res[4 * g + 2], res[4 * g + 3]));
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int64_t gp = gp0 + r;
                    if (gp >= 0 && gp < n) p.out[gp] = res[4 * g + r];
                }
            }
        }
    } else if (MODE == OUT_COUNT) {
#pragma unroll
        for (int j = 0; j < kPPT; ++j) cnt += res[j] >= 0 ? 1ull : 0ull;
    } else {
        unsigned long long mine = 0;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            unsigned long long c = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) c += res[4 * g + r] >= 0 ? 1ull : 0ull;
            mine |= c << (16 * g);
        }
        unsigned long long excl, total;
        block_exclusive_scan(mine, excl, total, sm.red, tid, nt);
        const unsigned long long tile_total =
            (total & 0xFFFFull) + ((total >> 16) & 0xFFFFull) + ((total >> 32) & 0xFFFFull) + (total >> 48);
        if (tid == 0) {
            const unsigned long long pre = lookback(p.status, tile, tile_total);
            sm.red[33] = pre;
            if (tile == p.ntiles - 1) *p.count = pre + tile_total;
        }
        __syncthreads();
        unsigned long long off = sm.red[33];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint32_t i0 = 4u * static_cast<uint32_t>(g * nt + tid);
            unsigned long long o = off + ((excl >> (16 * g)) & 0xFFFFull);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (res[4 * g + r] >= 0) {
                    if (o < p.cap) {
                        p.cpos[o] = static_cast<uint32_t>(gpb + i0 + r);
                        p.cids[o] = static_cast<uint32_t>(res[4 * g + r]);
                    }
                    ++o;
                }
            }
            off += (total >> (16 * g)) & 0xFFFFull;
        }
    }
}

template <int B, bool INV, typename GT, int MODE>
__global__ void __launch_bounds__(kMaxBlock, 1) pfac_tiled(const TiledParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const Smem sm = carve(smem, p);
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint32_t nst = p.nstages;

    if (tid == 0) {
        for (uint32_t s = 0; s < nst; ++s) mbar_init(&sm.bars[s], 1);
        mbar_init(&sm.bars[kMaxStages], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto next_tile = [&](uint32_t it) -> uint32_t {
        if (MODE == OUT_COMPACT) return atomicAdd(p.counter, 1u);
        const uint64_t t = static_cast<uint64_t>(blockIdx.x) + static_cast<uint64_t>(it) * gridDim.x;
        return t < p.ntiles ? static_cast<uint32_t>(t) : 0xFFFFFFFFu;
    };
    if (tid == 0) {
        mbar_arrive_expect_tx(&sm.bars[kMaxStages], 512u + p.jbytes);
        bulk_load(sm.cls, p.clsg, 512u, &sm.bars[kMaxStages]);
        if (p.jbytes) bulk_load(sm.J, p.Jg, p.jbytes, &sm.bars[kMaxStages]);
        for (uint32_t s = 0; s < nst; ++s) issue_stage(p, sm, s, next_tile(s));
    }

    unsigned long long cnt = 0;
    bool ok = mbar_wait(&sm.bars[kMaxStages], 0);
    uint32_t it = 0;
    for (;; ++it) {
        const uint32_t s = it % nst;
        ok = ok && mbar_wait(&sm.bars[s], (it / nst) & 1u);
        if (!__syncthreads_and(ok)) {
            // A copy never completed: latch the error, let the copies this CTA
            // still has in flight finish (bounded), and leave.
            if (tid == 0) {
                atomicOr(&g_dev_error, static_cast<unsigned>(kErrTimeout));
                mbar_wait(&sm.bars[kMaxStages], 0);
                for (uint32_t j = it; j < it + nst; ++j) mbar_wait(&sm.bars[j % nst], (j / nst) & 1u);
            }
            return;
        }
        const uint32_t tile = sm.stage_tile[s];
        if (tile >= p.ntiles) break;
        uint8_t *st = sm.stages + static_cast<size_t>(s) * p.SL;
        const uint64_t tlo = static_cast<uint64_t>(tile) * p.T;
        if (tid < 32) load_fringe(p, st, tlo, tid);
        __syncthreads();
        if (B < 8 || INV) {
            convert_stage<B>(p, sm, st, static_cast<int64_t>(tlo) - p.head, tid, nt);
            __syncthreads();
        }
        match_tile<B, INV, GT, MODE>(p, sm, st, tile, tid, nt, cnt);
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_smem();
            issue_stage(p, sm, s, next_tile(it + nst));
        }
    }

    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
        if ((tid & 31) == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

template <typename GT>
__global__ void __launch_bounds__(256) pfac_simple(const uint8_t *__restrict__ text, uint64_t n,
                                                   const GT *__restrict__ G, const int16_t *__restrict__ clsg,
                                                   uint32_t W, uint32_t C, int32_t *__restrict__ out) {
    __shared__ int16_t cls[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cls[i] = clsg[i];
    __syncthreads();
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t s = 0;
    int res;
    for (uint64_t j = i;; ++j) {
        if (j >= n) {
            res = decode_dead(goto_ld(G, s, W, C));
            break;
        }
        const int c = cls[text[j]];
        if (c < 0) {
            res = decode_dead(goto_ld(G, s, W, C));
            break;
        }
        const int t = goto_ld(G, s, W, static_cast<uint32_t>(c));
        if (t < 0) {
            res = decode_dead(t);
            break;
        }
        s = static_cast<uint32_t>(t);
    }
    out[i] = res;
}

// -------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------
inline uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

struct Geometry {
    uint32_t T, H, SL, nstages, ntiles, off_J, off_stage, off_packed, off_inv, smem;
};

bool make_geometry(const DevTables &t, uint64_t n, uint32_t head, const Tuning &tu, int max_smem, Geometry *g) {
    const uint32_t nt = static_cast<uint32_t>(tu.block);
    g->T = nt * kPPT;
    uint32_t H = t.maxlen < kHaloCap ? t.maxlen : kHaloCap;
    if (H < t.k + t.k2 + 4) H = t.k + t.k2 + 4;
    g->H = align16(H);
    g->SL = g->T + g->H;
    const uint64_t span = n + head;
    const uint64_t nt64 = (span + g->T - 1) / g->T;
    if (nt64 >= 0xFFFFFFFFull) return false;
    g->ntiles = static_cast<uint32_t>(nt64);
    const bool inv = t.B < 8 || t.C < 256;
    const uint32_t packed_bytes = t.B < 8 ? align16(g->SL * t.B / 8 + 16) : 0u;
    const uint32_t inv_bytes = inv ? align16(g->SL / 8 + 16) : 0u;
    for (int st = tu.stages; st >= 2; --st) {
        g->nstages = static_cast<uint32_t>(st);
        g->off_J = kHdrBytes;
        g->off_stage = align16(g->off_J + t.jbytes);
        g->off_packed = align16(g->off_stage + g->nstages * g->SL);
        g->off_inv = align16(g->off_packed + packed_bytes);
        g->smem = align16(g->off_inv + inv_bytes);
        if (static_cast<int>(g->smem) <= max_smem) return true;
    }
    return false;
}

template <int B, bool INV, typename GT, int MODE>
cudaError_t launch_one(const TiledParams &p, uint32_t grid, uint32_t block, uint32_t smem, int max_smem,
                       cudaStream_t stream) {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(pfac_tiled<B, INV, GT, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    pfac_tiled<B, INV, GT, MODE><<<grid, block, smem, stream>>>(p);
    return cudaGetLastError();
}

template <int B, bool INV, typename GT>
cudaError_t launch_modes(OutMode mode, const TiledParams &p, uint32_t grid, uint32_t block, uint32_t smem,
                         int max_smem, cudaStream_t stream) {
    switch (mode) {
        case OUT_DENSE:
            return launch_one<B, INV, GT, OUT_DENSE>(p, grid, block, smem, max_smem, stream);
        case OUT_COUNT:
            return launch_one<B, INV, GT, OUT_COUNT>(p, grid, block, smem, max_smem, stream);
        default:
            return launch_one<B, INV, GT, OUT_COMPACT>(p, grid, block, smem, max_smem, stream);
    }
}

template <typename GT>
cudaError_t launch_gt(const DevTables &t, OutMode mode, const TiledParams &p, uint32_t grid, uint32_t block,
                      uint32_t smem, int max_smem, cudaStream_t stream) {
    if (t.B == 2) return launch_modes<2, true, GT>(mode, p, grid, block, smem, max_smem, stream);
    if (t.B == 4) return launch_modes<4, true, GT>(mode, p, grid, block, smem, max_smem, stream);
    if (t.C < 256) return launch_modes<8, true, GT>(mode, p, grid, block, smem, max_smem, stream);
    return launch_modes<8, false, GT>(mode, p, grid, block, smem, max_smem, stream);
}

struct DeviceProps {
    int sms = 0;
    int max_smem = 0;
};

cudaError_t device_props(DeviceProps *out) {
    static DeviceProps cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cache[dev].sms == 0) {
        DeviceProps d;
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        cache[dev] = d;
    }
    *out = cache[dev];
    return cudaSuccess;
}

}  // namespace

size_t compact_scratch_bytes(const DevTables &t, uint64_t n, const Tuning &tu) {
    const uint64_t T = static_cast<uint64_t>(tu.block) * kPPT;
    const uint64_t tiles = (n + 15 + T - 1) / T;
    (void)t;
    return static_cast<size_t>(16 + 8 * (tiles + 1));
}

cudaError_t launch_tiled(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                         cudaStream_t stream) {
    if (tu.block < 32 || tu.block > kMaxBlock || (tu.block & 31) || tu.stages < 2 || tu.stages > kMaxStages)
        return cudaErrorInvalidValue;
    DeviceProps dp;
    cudaError_t e = device_props(&dp);
    if (e != cudaSuccess) return e;
    TiledParams p{};
    p.text = r.text;
    p.head = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(r.text) & 15u);
    p.gbase = r.text - p.head;
    p.n = r.n;
    Geometry g;
    if (!make_geometry(t, r.n, p.head, tu, dp.max_smem, &g)) return cudaErrorInvalidConfiguration;
    p.T = g.T;
    p.H = g.H;
    p.SL = g.SL;
    p.nstages = g.nstages;
    p.ntiles = g.ntiles;
    p.off_J = g.off_J;
    p.off_stage = g.off_stage;
    p.off_packed = g.off_packed;
    p.off_inv = g.off_inv;
    p.G = t.G;
    p.Jg = t.J;
    p.J2 = t.J2;
    p.clsg = t.cls;
    p.C = t.C;
    p.W = t.W;
    p.k = t.k;
    p.k2 = t.k2;
    p.base_k = t.base_k;
    p.maxlen = t.maxlen;
    p.jbytes = t.jbytes;
    p.out = r.out;
    p.vec_ok = ((reinterpret_cast<uintptr_t>(r.out) - 4u * p.head) & 15u) == 0;
    p.cpos = r.pos;
    p.cids = r.ids;
    p.cap = r.cap;
    p.count = r.count;
    if (mode == OUT_COMPACT) {
        if (!r.scratch || r.scratch_bytes < 16 + 8 * (static_cast<size_t>(g.ntiles) + 1))
            return cudaErrorInvalidValue;
        p.counter = static_cast<unsigned int *>(r.scratch);
        p.status = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(r.scratch) + 16);
    }
    uint32_t grid = tu.grid > 0 ? static_cast<uint32_t>(tu.grid) : static_cast<uint32_t>(dp.sms);
    if (grid > g.ntiles) grid = g.ntiles;
    if (grid == 0) return cudaSuccess;
    if (t.gbits == 16)
        return launch_gt<int16_t>(t, mode, p, grid, static_cast<uint32_t>(tu.block), g.smem, dp.max_smem, stream);
    return launch_gt<int32_t>(t, mode, p, grid, static_cast<uint32_t>(tu.block), g.smem, dp.max_smem, stream);
}

cudaError_t launch_simple(const DevTables &t, const MatchRequest &r, cudaStream_t stream) {
    const uint64_t blocks = (r.n + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    if (t.gbits == 16)
        pfac_simple<int16_t><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
            r.text, r.n, static_cast<const int16_t *>(t.G), t.cls, t.W, t.C, r.out);
    else
        pfac_simple<int32_t><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
            r.text, r.n, static_cast<const int32_t *>(t.G), t.cls, t.W, t.C, r.out);
    return cudaGetLastError();
}

cudaError_t read_device_error(unsigned int *value) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbol(value, g_dev_error, sizeof(unsigned int));
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_dev_error, &zero, sizeof(unsigned int));
}

}  // namespace pfac
