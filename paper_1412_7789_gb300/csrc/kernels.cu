// Failureless Aho-Corasick matching kernels for sm_103a.
//
// pfac_match -- the production kernel.  Persistent CTAs (one per SM); every
//   warp owns a private ring of `stages` text buffers in shared memory and
//   walks warp tiles of 1024 positions independently of the other warps (no
//   block-wide barrier after start-up):
//   * a warp tile plus a halo of up to max-keyword-length bytes is fetched with
//     one bulk async copy (cp.async.bulk, the TMA unit, no multicast) that
//     completes on the stage's mbarrier, several tiles ahead of use;
//   * the warp maps the tile's bytes to class codes once, packed B bits each,
//     with one "cannot extend a walk" bit per position (byte permutes on a
//     3-bit hash for alphabets of up to 8 keyword bytes, else a byte table);
//   * each lane takes groups of 4 consecutive positions; one shared-memory
//     lookup in the root jump table (the top k levels of the goto table
//     flattened; resident for the whole kernel) gives the result of most
//     positions outright;
//   * the positions whose walk is still alive at depth k (or whose window holds
//     an unknown byte or the text end) go to a per-warp queue and are spread
//     over all 32 lanes: one lookup in the stride table (k2 more levels,
//     global, L2-resident), then, rarely, the goto table one character at a
//     time through L1;
//   * results are staged per pass in shared memory; output is dense int32 ids
//     (one bulk async store per pass, or coalesced 16-byte stores at the text
//     edges), a count (one atomic per warp), or
//     the compacted (pos, id) list in ascending order (warp scan + decoupled
//     look-back across half-tiles).
// pfac_simple -- one thread per position walking the goto table in global
//   memory: the design of the paper's GPU side (section I, Fig. 3), kept as the
//   comparison point.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

__device__ unsigned int g_dev_error = 0;

namespace {

constexpr int kMaxBlock = 512;
constexpr int kMaxWarps = kMaxBlock / 32;
constexpr int kMaxStages = 4;
constexpr uint32_t kPass = 512;          // positions per pass: 32 lanes x 4 groups x 4
constexpr uint32_t kTW = 2 * kPass;      // positions per warp tile
// shared-memory header
constexpr uint32_t kOffJBar = 0;
constexpr uint32_t kOffStageBar = 64;                                   // kMaxWarps * kMaxStages * 8
constexpr uint32_t kOffStageTile = kOffStageBar + kMaxWarps * kMaxStages * 8;
constexpr uint32_t kOffCls = 1024;                                      // 256 x uint8
constexpr uint32_t kOffJ = 1280;                                        // root jump table
constexpr unsigned kFull = 0xffffffffu;
// per-warp region: [stages][packed codes][cannot-extend bits][pass results][survivor queue]
constexpr uint32_t kResBytes = kPass * 4;
constexpr uint32_t kQueueBytes = kPass * 2;

struct WarpParams {
    const uint8_t *text;    // batch: base of all texts
    uint64_t n;
    const BatchHead *batch; // batch: this automaton's head and the planned list
    const BatchItemDev *lists;
    uint32_t SLW;           // staged bytes per warp tile (tile + halo)
    uint32_t tw;            // positions per warp tile (kTW, or kPass for the compacted output)
    uint32_t nstages, ntiles;
    const void *G;
    const int16_t *Jg;
    const int32_t *J2;
    const uint8_t *cls8g;
    uint32_t C, W, k, k2, base_k, maxlen, jbytes;
    int jslow;
    int hash_shift;          // >= 0: classify with the 3-bit hash
    uint32_t hcode_lo, hcode_hi, hbyte_lo, hbyte_hi;
    int32_t *out;           // batch: base of all outputs
    uint32_t *cpos;
    uint32_t *cids;
    unsigned long long cap;
    unsigned long long *count;
    unsigned long long *status;  // compact: one word per half tile
    unsigned int *counter;       // compact: next tile to claim
    uint32_t off_warp, warp_bytes, off_packed, off_inv, off_res, off_queue, off_meta;
};

struct WarpSmem {
    const uint8_t *cls8;
    const uint8_t *jbase;   // root jump table (byte addressed)
    uint8_t *st;            // current stage
    uint32_t *packed;
    uint32_t *inv;
    int32_t *res;
    uint16_t *queue;
};

// The text and tile of work unit u (entry `item` of the planned list in a batch).
__device__ __forceinline__ TileText tile_text(const WarpParams &p, const Work &wk, uint32_t u, uint32_t item) {
    if (!wk.list) return make_text(p.text, p.out, p.n, u);
    return batch_text(wk, p.text, p.out, item, u);
}

// All lanes: point stage s at unit u (>= wk.units: the end of this warp's
// work) and start its bulk copy.
__device__ __forceinline__ void issue_unit(const WarpParams &p, const Work &wk, uint64_t *bar, uint32_t *stile,
                                           uint32_t *sitem, uint8_t *st, uint32_t u, int lane) {
    const uint32_t item = (wk.list && u < wk.units) ? find_item(wk, u, lane) : 0u;
    if (lane == 0) {
        *stile = u;
        *sitem = item;
        if (u >= wk.units)
            mbar_arrive(bar);
        else
            issue_text_tile(tile_text(p, wk, u, item), p.tw, p.SLW, bar, st);
    }
}

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int b) {
    return __byte_perm(w, 0u, 0x4440u | static_cast<uint32_t>(b));
}

// Four class-table values (bytes, 0xFF = unknown byte) of the bytes of w, as one word.
__device__ __forceinline__ uint32_t classify4(const uint8_t *cls8, uint32_t w) {
    const uint32_t t0 = cls8[byte_of(w, 0)], t1 = cls8[byte_of(w, 1)];
    const uint32_t t2 = cls8[byte_of(w, 2)], t3 = cls8[byte_of(w, 3)];
    return __byte_perm(__byte_perm(t0, t1, 0x0040u), __byte_perm(t2, t3, 0x0040u), 0x5410u);
}

// Map the staged bytes to class codes (B bits each, position order) and set a
// bit for each position that cannot extend a walk (byte in no keyword, or
// outside the text).  Returns true when no staged position has that bit.
template <int B>
__device__ __forceinline__ bool convert_stage(const WarpParams &p, const TileText &tt, const WarpSmem &w, int64_t gpb,
                                              bool interior, int lane) {
    const int64_t n = static_cast<int64_t>(tt.n);
    const uint32_t items = p.SLW / 8;
    uint8_t *inv8 = reinterpret_cast<uint8_t *>(w.inv);
    uint32_t any = 0;
    const bool hashed = (B < 8) && p.hash_shift >= 0;
    for (uint32_t c = lane; c < items; c += 32) {
        const uint2 v = reinterpret_cast<const uint2 *>(w.st)[c];
        uint32_t lo, hi, ib;
        if (hashed) {
            // per byte h = (byte >> s) & 7 selects, with byte permutes, its code
            // and the one keyword byte with that hash; a mismatch is an unknown byte
            const uint32_t sh = static_cast<uint32_t>(p.hash_shift);
            const uint32_t hl = (v.x >> sh) & 0x07070707u, hh = (v.y >> sh) & 0x07070707u;
            const uint32_t sl = __byte_perm(hl | (hl >> 4), 0u, 0x4420u);
            const uint32_t sg = __byte_perm(hh | (hh >> 4), 0u, 0x4420u);
            lo = __byte_perm(p.hcode_lo, p.hcode_hi, sl);
            hi = __byte_perm(p.hcode_lo, p.hcode_hi, sg);
            const uint32_t xl = v.x ^ __byte_perm(p.hbyte_lo, p.hbyte_hi, sl);
            const uint32_t xh = v.y ^ __byte_perm(p.hbyte_lo, p.hbyte_hi, sg);
            // bit 7 of each byte of t set iff that byte of x is non-zero
            const uint32_t tl = ((xl & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | xl;
            const uint32_t th = ((xh & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | xh;
            ib = (((tl & 0x80808080u) * 0x00204081u) >> 28) | ((((th & 0x80808080u) * 0x00204081u) >> 28) << 4);
        } else {
            lo = classify4(w.cls8, v.x);
            hi = classify4(w.cls8, v.y);
            // gather one flag per unknown byte (class value 0xFF): bit 7 of each
            // byte flag, moved to bits 0-3 by one multiply.  Codes below 16 never
            // have bit 7 set; 8-bit codes compare the whole byte with 0xFF.
            uint32_t fl = lo, fh = hi;
            if (B == 8) {
                fl = __vcmpeq4(lo, 0xFFFFFFFFu);
                fh = __vcmpeq4(hi, 0xFFFFFFFFu);
            }
            ib = (((fl & 0x80808080u) * 0x00204081u) >> 28) | ((((fh & 0x80808080u) * 0x00204081u) >> 28) << 4);
        }
        if (!interior) {
            const int64_t gp0 = gpb + 8 * static_cast<int64_t>(c);
            if (!(gp0 >= 0 && gp0 + 8 <= n)) {
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    if (gp0 + b < 0 || gp0 + b >= n) ib |= 1u << b;
            }
        }
        any |= ib;
        if (B == 2) {
            const uint32_t cl = ((lo & 0x03030303u) * 0x01041040u) >> 24;
            const uint32_t ch = ((hi & 0x03030303u) * 0x01041040u) >> 24;
            reinterpret_cast<uint16_t *>(w.packed)[c] = static_cast<uint16_t>(cl | (ch << 8));
        } else if (B == 4) {
            uint32_t xl = lo & 0x0F0F0F0Fu, xh = hi & 0x0F0F0F0Fu;
            xl = (xl | (xl >> 4)) & 0x00FF00FFu;
            xh = (xh | (xh >> 4)) & 0x00FF00FFu;
            xl = (xl | (xl >> 8)) & 0xFFFFu;
            xh = (xh | (xh >> 8)) & 0xFFFFu;
            w.packed[c] = xl | (xh << 16);
        } else {
            reinterpret_cast<uint2 *>(w.st)[c] = make_uint2(lo, hi);
        }
        inv8[c] = static_cast<uint8_t>(ib);
    }
    return __any_sync(kFull, any != 0) == 0;
}

// Codes of positions i.. in the low bits (16 codes for B = 2, 8 for B = 4 and
// B = 8).
template <int B>
__device__ __forceinline__ uint64_t code_window(const uint8_t *st, const uint32_t *packed, uint32_t i) {
    if (B == 8) {
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(st);
        const uint32_t w = i >> 2, sh = 8u * (i & 3u);
        const uint32_t a = s32[w], b = s32[w + 1], c = s32[w + 2];
        return static_cast<uint64_t>(__funnelshift_r(a, b, sh)) |
               (static_cast<uint64_t>(__funnelshift_r(b, c, sh)) << 32);
    } else {
        const uint32_t bo = B * i, w = bo >> 5;
        return __funnelshift_r(packed[w], packed[w + 1], bo & 31u);
    }
}

__device__ __forceinline__ uint32_t inv_window(const uint32_t *inv, uint32_t i) {
    const uint32_t w = i >> 5;
    return __funnelshift_r(inv[w], inv[w + 1], i & 31u);
}

__device__ __forceinline__ int jump_at(const uint8_t *jbase, uint32_t idx) {
    return *reinterpret_cast<const int16_t *>(jbase + 2u * idx);
}

// Code of staged position q; false when q cannot extend a walk.
template <int B, bool INV>
__device__ __forceinline__ bool fetch_code(const WarpParams &p, const TileText &tt, const WarpSmem &w, int64_t gpb,
                                           uint32_t q, uint32_t &c) {
    if (q < p.SLW) {
        if (INV) {
            if ((w.inv[q >> 5] >> (q & 31u)) & 1u) return false;
        } else {
            if (gpb + static_cast<int64_t>(q) >= static_cast<int64_t>(tt.n)) return false;
        }
        if (B == 8)
            c = w.st[q];
        else
            c = (w.packed[(B * q) >> 5] >> ((B * q) & 31u)) & ((1u << B) - 1u);
        return true;
    }
    const int64_t gp = gpb + static_cast<int64_t>(q);
    if (gp >= static_cast<int64_t>(tt.n)) return false;
    const uint32_t b = __ldg(tt.text + gp);
    if (!INV) {
        c = b;
        return true;
    }
    const uint32_t v = w.cls8[b];
    if (v == 0xFFu) return false;
    c = v;
    return true;
}

// Finish up to SLOTS * 32 queued survivors (entries base.. of the queue, `avail`
// of them): each lane takes SLOTS entries and advances their walks together.
template <int B, bool INV, typename GT, int MODE, int SLOTS>
__device__ __forceinline__ void finish_survivors(const WarpParams &p, const TileText &tt, const WarpSmem &w,
                                                 int64_t gpb, bool interior, bool clean, uint32_t avail, uint32_t h,
                                                 int lane, unsigned long long &cnt, uint32_t base = 0) {
    const int64_t n = static_cast<int64_t>(tt.n);
    const uint32_t k = p.k, k2 = p.k2;
    const uint32_t kmask = (1u << (B * k)) - 1u;
    const GT *G = static_cast<const GT *>(p.G);
    uint32_t st4[SLOTS], q4[SLOTS], i4[SLOTS];
    int v4[SLOTS];
    uint32_t walking = 0, act = 0;
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        const uint32_t qi = lane + 32u * t;
        v4[t] = INT_MIN;
        st4[t] = 0;
        q4[t] = 0;
        i4[t] = 0;
        if (qi < avail) {
            act |= 1u << t;
            const uint32_t e16 = w.queue[base + qi];
            const uint32_t i = e16 & 0x7FFFu;
            i4[t] = i;
            q4[t] = i;
            if (!(e16 >> 15)) {
                const uint64_t x = code_window<B>(w.st, w.packed, i);
                const uint32_t off = static_cast<uint32_t>(-jump_at(w.jbase, static_cast<uint32_t>(x) & kmask) - 2);
                st4[t] = p.base_k + off;
                q4[t] = i + k;
                if (k2 > 0) {
                    bool ok2 = interior || gpb + static_cast<int64_t>(i + k + k2) <= n;
                    if (INV && !clean) ok2 = ok2 && ((inv_window(w.inv, i + k) & ((1u << k2) - 1u)) == 0);
                    if (ok2) {
                        const uint32_t w2 = static_cast<uint32_t>(x >> (B * k)) & ((1u << (B * k2)) - 1u);
                        v4[t] = __ldg(p.J2 + ((static_cast<uint64_t>(off) << (B * k2)) | w2));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        if ((act >> t) & 1u) {
            if (v4[t] == INT_MIN) {
                walking |= 1u << t;
            } else if (v4[t] < 0) {
                v4[t] = decode_dead(v4[t]);
            } else {
                st4[t] = static_cast<uint32_t>(v4[t]);
                q4[t] += k2;
                v4[t] = INT_MIN;
                walking |= 1u << t;
            }
        }
    }
    for (uint32_t step = 0; walking; ++step) {
        if (step > p.maxlen + 1) {  // impossible for a well-formed table
            atomicOr(&g_dev_error, static_cast<unsigned>(kErrWalk));
#pragma unroll
            for (int t = 0; t < SLOTS; ++t)
                if ((walking >> t) & 1u) v4[t] = -1;
            break;
        }
        int e4[SLOTS];
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            if ((walking >> t) & 1u) {
                uint32_t c = 0;
                const bool okc = fetch_code<B, INV>(p, tt, w, gpb, q4[t], c);
                // an unknown byte or the text end reads the row's end column,
                // which always holds the result of stopping there
                e4[t] = goto_ld(G, st4[t], p.W, okc ? c : p.C);
            }
        }
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            if ((walking >> t) & 1u) {
                if (e4[t] < 0) {
                    v4[t] = decode_dead(e4[t]);
                    walking &= ~(1u << t);
                } else {
                    st4[t] = static_cast<uint32_t>(e4[t]);
                    q4[t] += 1;
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        if ((act >> t) & 1u) {
            if (MODE == OUT_COUNT)
                cnt += v4[t] >= 0 ? 1ull : 0ull;
            else
                w.res[i4[t] - h * kPass] = v4[t];
        }
    }
}

// Flags describing a warp tile.
enum : uint32_t { kInterior = 1u, kClean = 2u };

template <int B, bool INV, typename GT, int MODE>
__device__ __forceinline__ void match_pass(const WarpParams &p, const TileText &tt, const WarpSmem &w, int64_t gpb,
                                           uint32_t flags, uint32_t h, int lane, unsigned long long &cnt) {
    const int64_t n = static_cast<int64_t>(tt.n);
    const uint32_t k = p.k;
    const uint32_t kmask = (1u << (B * k)) - 1u;
    const bool interior = flags & kInterior;
    const bool clean = !INV || (flags & kClean);
    const uint32_t ibase = h * kPass + 4u * static_cast<uint32_t>(lane);

    // 1. one root-jump lookup per position: the result, or (<= -2) a walk that
    //    continues past depth k, or kJumpSlow
    int res[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint64_t x = code_window<B>(w.st, w.packed, ibase + 128u * g);
#pragma unroll
        for (int r = 0; r < 4; ++r) res[4 * g + r] = jump_at(w.jbase, static_cast<uint32_t>(x >> (B * r)) & kmask);
    }
    uint32_t valid = 0xFFFFu;
    const bool fixups = !interior || !clean || k == 0;
    if (fixups) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint32_t i0 = ibase + 128u * g;
            uint32_t wi = 0;
            if (INV) wi = inv_window(w.inv, i0);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int j = 4 * g + r;
                const int64_t gp = gpb + i0 + r;
                if (gp < 0 || gp >= n) {
                    res[j] = -1;
                    valid &= ~(1u << j);
                } else if (k == 0 || gp + static_cast<int64_t>(k) > n || ((wi >> r) & ((1u << k) - 1u))) {
                    res[j] = kJumpSlow;
                }
            }
        }
    }
    uint32_t sv = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) sv |= (res[j] < -1 ? 1u : 0u) << j;
    uint32_t slowm = 0;
    if (fixups || p.jslow) {
#pragma unroll
        for (int j = 0; j < 16; ++j) slowm |= (res[j] == kJumpSlow ? 1u : 0u) << j;
    }

    // 2. survivors into the warp's queue (position, slow flag), in lane order
    const uint32_t c = __popc(sv);
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    {
        uint32_t o = inc - c, m = sv;
        while (m) {
            const uint32_t j = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t i = ibase + ((j >> 2) << 7) + (j & 3u);
            w.queue[o++] = static_cast<uint16_t>(i | (((slowm >> j) & 1u) << 15));
        }
    }
    if (MODE == OUT_COUNT) {
        uint32_t hit = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) hit |= (res[j] >= 0 ? 1u : 0u) << j;
        cnt += __popc(hit & valid);
    } else {
        if (MODE == OUT_DENSE) {
            // the previous pass's bulk store must have read the staging buffer
            if (lane == 0) bulk_wait_read();
            __syncwarp();
        }
#pragma unroll
        for (int g = 0; g < 4; ++g)
            reinterpret_cast<int4 *>(w.res)[32 * g + lane] =
                make_int4(res[4 * g], res[4 * g + 1], res[4 * g + 2], res[4 * g + 3]);
    }
    __syncwarp();

    // 3. the survivors, spread over the lanes (several per lane at a time so
    //    their dependent loads overlap): stride table, then (rarely) the goto
    //    table one character at a time
    if (total <= 64) {
        finish_survivors<B, INV, GT, MODE, 2>(p, tt, w, gpb, interior, clean, total, h, lane, cnt);
    } else {
        for (uint32_t base = 0; base < total; base += 256)
            finish_survivors<B, INV, GT, MODE, 8>(p, tt, w, gpb, interior, clean, total - base, h, lane, cnt,
                                                  base);
    }
    __syncwarp();

    // 4. output
    if (MODE == OUT_DENSE && interior && tt.vec_ok) {
        // the whole pass is inside the text: one bulk store of the staged ids
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            bulk_store(tt.out + gpb + h * kPass, w.res, kResBytes);
            bulk_commit();
        }
    } else if (MODE == OUT_DENSE) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int4 r4 = reinterpret_cast<const int4 *>(w.res)[32 * g + lane];
            const int64_t gp0 = gpb + ibase + 128u * g;
            if (tt.vec_ok && ((valid >> (4 * g)) & 0xFu) == 0xFu) {
                __stcs(reinterpret_cast<int4 *>(tt.out + gp0), r4);
            } else {
                const int rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if ((valid >> (4 * g + r)) & 1u) tt.out[gp0 + r] = rr[r];
            }
        }
    }
    // compacted output: the staged results are ranked per CTA round (pfac_match_compact)
    __syncwarp();
}

template <int B, bool INV, typename GT, int MODE>
__global__ void __launch_bounds__(kMaxBlock, 1) pfac_match(const WarpParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t *jbar = reinterpret_cast<uint64_t *>(smem + kOffJBar);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffStageBar) + warp * kMaxStages;
    uint32_t *stile = reinterpret_cast<uint32_t *>(smem + kOffStageTile) + warp * kMaxStages;
    uint8_t *wreg = smem + p.off_warp + static_cast<size_t>(warp) * p.warp_bytes;
    WarpSmem w;
    w.cls8 = smem + kOffCls;
    w.jbase = smem + kOffJ;
    w.st = wreg;
    w.packed = reinterpret_cast<uint32_t *>(wreg + p.off_packed);
    w.inv = reinterpret_cast<uint32_t *>(wreg + p.off_inv);
    w.res = reinterpret_cast<int32_t *>(wreg + p.off_res);
    w.queue = reinterpret_cast<uint16_t *>(wreg + p.off_queue);
    uint32_t *sitem = reinterpret_cast<uint32_t *>(wreg + p.off_meta);
    const uint32_t nst = p.nstages;
    const Work wk = load_work(p.batch, p.lists, p.ntiles);

    if (threadIdx.x == 0) {
        mbar_init(jbar, 1);
        uint64_t *all = reinterpret_cast<uint64_t *>(smem + kOffStageBar);
        for (int i = 0; i < nw * kMaxStages; ++i) mbar_init(&all[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(jbar, 256u + p.jbytes);
        bulk_load(smem + kOffCls, p.cls8g, 256u, jbar);
        if (p.jbytes) bulk_load(smem + kOffJ, p.Jg, p.jbytes, jbar);
    }
    // consecutive tiles go to different SMs (warp-major, CTA-minor numbering)
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nw;
    // Tiles are claimed from a global counter, so a warp that meets an
    // expensive tile (long walks) stops taking work while the others go on;
    // each warp's first tile is handed out statically.
    auto next_tile = [&](uint32_t it) -> uint32_t {  // all lanes
        uint32_t t = 0xFFFFFFFFu;
        if (lane == 0) {
            const uint64_t c = it == 0 ? gw : GW + atomicAdd(p.counter, 1u);
            if (c < wk.units) t = static_cast<uint32_t>(c);
        }
        return __shfl_sync(kFull, t, 0);
    };
    for (uint32_t s = 0; s < nst; ++s)
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], wreg + s * p.SLW, next_tile(s), lane);

    unsigned long long cnt = 0;
    bool ok = mbar_wait(jbar, 0);
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % nst;
        ok = ok && mbar_wait(&bars[s], (it / nst) & 1u);
        if (!__all_sync(kFull, ok)) {
            // A copy never completed: latch the error, let this warp's copies in
            // flight finish (bounded), and leave.
            if (lane == 0) {
                bulk_wait_all();
                atomicOr(&g_dev_error, static_cast<unsigned>(kErrTimeout));
                mbar_wait(jbar, 0);
                for (uint32_t j = it; j < it + nst; ++j) mbar_wait(&bars[j % nst], (j / nst) & 1u);
            }
            return;
        }
        const uint32_t tile = stile[s];
        if (tile >= wk.units) break;
        const TileText tt = tile_text(p, wk, tile, sitem[s]);
        w.st = wreg + s * p.SLW;
        const uint64_t tlo = static_cast<uint64_t>(tt.tile) * p.tw;
        const int64_t gpb = static_cast<int64_t>(tlo) - tt.head;
        const bool interior = gpb >= 0 && gpb + static_cast<int64_t>(p.SLW) <= static_cast<int64_t>(tt.n);
        if (!interior) {
            load_text_fringe(tt, p.SLW, w.st, tlo, lane);
            __syncwarp();
        }
        uint32_t flags = interior ? kInterior : 0u;
        if (B < 8 || INV) {
            if (convert_stage<B>(p, tt, w, gpb, interior, lane)) flags |= kClean;
            __syncwarp();
        }
#pragma unroll 1
        for (uint32_t h = 0; h < kTW / kPass; ++h) match_pass<B, INV, GT, MODE>(p, tt, w, gpb, flags, h, lane, cnt);
        if (lane == 0) fence_proxy_async_smem();
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], w.st, next_tile(it + nst), lane);
    }

    if (MODE == OUT_DENSE && lane == 0) bulk_wait_all();
    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

// ---------------------------------------------------------------------------
// Compacted output.  The ascending (pos, id) list needs every match's rank, so
// the unit of ordering is a CTA round: the CTA claims a chunk of nw
// consecutive one-pass tiles (one per warp), each warp matches its tile into
// shared memory and counts its matches, then one warp scans the counts and
// places the chunk with a warp-wide decoupled look-back, and every warp writes
// its matches.  Chunks are claimed in increasing order by running CTAs, so the
// look-back always ends; with one chunk per CTA in flight it stays short.
// ---------------------------------------------------------------------------
constexpr uint32_t kOffChunk = 832;   // 2 x uint32: chunk held by each stage
constexpr uint32_t kOffCounts = 840;  // kMaxWarps x uint32: matches per warp
constexpr uint32_t kOffBase = 904;    // kMaxWarps x uint32: output offset per warp (n < 2^32)
constexpr uint32_t kOffAbort = kOffBase + kMaxWarps * 4;
static_assert(kOffAbort + 4 <= kOffCls, "compaction header overlaps the class map");

// Matches among the staged results of a pass (positions outside the text hold -1).
__device__ __forceinline__ uint32_t count_staged(const int32_t *res, int lane) {
    uint32_t c = 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const int4 r4 = reinterpret_cast<const int4 *>(res)[32 * g + lane];
        c += (r4.x >= 0) + (r4.y >= 0) + (r4.z >= 0) + (r4.w >= 0);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
    return c;
}

// Write the staged matches of a pass, in ascending position, from output offset base.
__device__ __forceinline__ void write_staged(const WarpParams &p, const int32_t *res, int64_t gpb,
                                             unsigned long long base, int lane) {
    int rr[16];
    uint32_t mine = 0;  // 4 fields of 8 bits: matches per group of 4 (<= 4)
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const int4 r4 = reinterpret_cast<const int4 *>(res)[32 * g + lane];
        rr[4 * g] = r4.x;
        rr[4 * g + 1] = r4.y;
        rr[4 * g + 2] = r4.z;
        rr[4 * g + 3] = r4.w;
        const uint32_t cg = (r4.x >= 0) + (r4.y >= 0) + (r4.z >= 0) + (r4.w >= 0);
        mine |= cg << (8 * g);
    }
    uint32_t sc = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, sc, d);
        if (lane >= d) sc += y;
    }
    const uint32_t tot = __shfl_sync(kFull, sc, 31);  // fields <= 128: no carries
    const uint32_t excl = sc - mine;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint32_t i0 = 4u * (32u * g + lane);
        unsigned long long o = base + ((excl >> (8 * g)) & 0xFFu);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (rr[4 * g + r] >= 0) {
                if (o < p.cap) {
                    p.cpos[o] = static_cast<uint32_t>(gpb + i0 + r);
                    p.cids[o] = static_cast<uint32_t>(rr[4 * g + r]);
                }
                ++o;
            }
        }
        base += (tot >> (8 * g)) & 0xFFu;
    }
}

template <int B, bool INV, typename GT>
__global__ void __launch_bounds__(kMaxBlock, 1) pfac_match_compact(const WarpParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t *jbar = reinterpret_cast<uint64_t *>(smem + kOffJBar);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffStageBar) + warp * kMaxStages;
    uint32_t *stile = reinterpret_cast<uint32_t *>(smem + kOffStageTile) + warp * kMaxStages;
    volatile uint32_t *chunk = reinterpret_cast<uint32_t *>(smem + kOffChunk);
    uint32_t *counts = reinterpret_cast<uint32_t *>(smem + kOffCounts);
    uint32_t *bases = reinterpret_cast<uint32_t *>(smem + kOffBase);
    volatile uint32_t *abort_flag = reinterpret_cast<uint32_t *>(smem + kOffAbort);
    uint8_t *wreg = smem + p.off_warp + static_cast<size_t>(warp) * p.warp_bytes;
    WarpSmem w;
    w.cls8 = smem + kOffCls;
    w.jbase = smem + kOffJ;
    w.st = wreg;
    w.packed = reinterpret_cast<uint32_t *>(wreg + p.off_packed);
    w.inv = reinterpret_cast<uint32_t *>(wreg + p.off_inv);
    w.res = reinterpret_cast<int32_t *>(wreg + p.off_res);
    w.queue = reinterpret_cast<uint16_t *>(wreg + p.off_queue);
    uint32_t *sitem = reinterpret_cast<uint32_t *>(wreg + p.off_meta);
    const Work wk = load_work(nullptr, nullptr, p.ntiles);  // one text
    const uint32_t nchunks = (wk.units + nw - 1) / nw;

    if (threadIdx.x == 0) {
        mbar_init(jbar, 1);
        uint64_t *all = reinterpret_cast<uint64_t *>(smem + kOffStageBar);
        for (int i = 0; i < nw * kMaxStages; ++i) mbar_init(&all[i], 1);
        fence_mbar_init();
        *abort_flag = 0;
        chunk[0] = atomicAdd(p.counter, 1u);
        chunk[1] = atomicAdd(p.counter, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(jbar, 256u + p.jbytes);
        bulk_load(smem + kOffCls, p.cls8g, 256u, jbar);
        if (p.jbytes) bulk_load(smem + kOffJ, p.Jg, p.jbytes, jbar);
    }
    auto tile_of = [&](uint32_t c) -> uint32_t {
        const uint64_t t = static_cast<uint64_t>(c) * nw + warp;
        return (c < nchunks && t < wk.units) ? static_cast<uint32_t>(t) : 0xFFFFFFFFu;
    };
    for (uint32_t s = 0; s < 2; ++s)
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], wreg + s * p.SLW, tile_of(chunk[s]), lane);

    unsigned long long unused = 0;
    bool ok = mbar_wait(jbar, 0);
    for (uint32_t r = 0;; ++r) {
        const uint32_t s = r & 1u;
        const uint32_t c = chunk[s];
        if (c >= nchunks) break;  // the same value for every warp of the CTA
        ok = ok && mbar_wait(&bars[s], (r >> 1) & 1u);
        ok = __all_sync(kFull, ok);
        const uint32_t tile = stile[s];
        uint32_t m = 0;
        int64_t gpb = 0;
        if (ok && tile < wk.units) {
            const TileText tt = tile_text(p, wk, tile, sitem[s]);
            w.st = wreg + s * p.SLW;
            const uint64_t tlo = static_cast<uint64_t>(tt.tile) * p.tw;
            gpb = static_cast<int64_t>(tlo) - tt.head;
            const bool interior = gpb >= 0 && gpb + static_cast<int64_t>(p.SLW) <= static_cast<int64_t>(tt.n);
            if (!interior) {
                load_text_fringe(tt, p.SLW, w.st, tlo, lane);
                __syncwarp();
            }
            uint32_t flags = interior ? kInterior : 0u;
            if (B < 8 || INV) {
                if (convert_stage<B>(p, tt, w, gpb, interior, lane)) flags |= kClean;
                __syncwarp();
            }
            match_pass<B, INV, GT, OUT_COMPACT>(p, tt, w, gpb, flags, 0, lane, unused);
            m = count_staged(w.res, lane);
        }
        if (lane == 0) {
            counts[warp] = m;
            if (!ok) *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) {
            // A copy never completed: latch the error, let this warp's copies in
            // flight finish (bounded), and leave (every warp of the CTA does).
            if (lane == 0) {
                atomicOr(&g_dev_error, static_cast<unsigned>(kErrTimeout));
                mbar_wait(jbar, 0);
                for (uint32_t j = r; j < r + 2; ++j) mbar_wait(&bars[j & 1u], (j >> 1) & 1u);
            }
            return;
        }
        if (warp == 0) {
            const uint32_t mine = lane < nw ? counts[lane] : 0u;
            uint32_t inc = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, d);
                if (lane >= d) inc += y;
            }
            const uint32_t total = __shfl_sync(kFull, inc, 31);
            const unsigned long long pre = lookback_warp(p.status, c, total, &g_dev_error, lane);
            if (lane < nw) bases[lane] = static_cast<uint32_t>(pre + (inc - mine));
            if (lane == 0) {
                if (c == nchunks - 1) *p.count = pre + total;
                chunk[s] = atomicAdd(p.counter, 1u);  // this stage's next chunk
            }
        }
        __syncthreads();
        if (tile < wk.units) write_staged(p, w.res, gpb, bases[warp], lane);
        __syncwarp();
        if (lane == 0) fence_proxy_async_smem();
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], wreg + s * p.SLW, tile_of(chunk[s]), lane);
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
    uint32_t SLW, nstages, ntiles, off_warp, warp_bytes, off_packed, off_inv, off_res, off_queue, off_meta, smem;
};

// Warp tile: two passes, or one for the compacted output (a warp keeps one
// pass of results staged until its CTA round is placed).
inline uint32_t tile_len(OutMode mode) { return mode == OUT_COMPACT ? kPass : kTW; }

bool make_geometry(const DevTables &t, uint64_t n, uint32_t head, OutMode mode, const Tuning &tu, int max_smem,
                   Geometry *g) {
    const uint32_t nw = static_cast<uint32_t>(tu.block) / 32u;
    const uint32_t tw = tile_len(mode);
    uint32_t H = t.maxlen < kHaloCap ? t.maxlen : kHaloCap;
    if (H < t.k + t.k2 + 8) H = t.k + t.k2 + 8;
    H = align16(H);
    g->SLW = tw + H;
    const uint64_t tiles = (n + head + tw - 1) / tw;
    if (tiles >= 0x7FFFFFFFull) return false;
    g->ntiles = static_cast<uint32_t>(tiles);
    const bool inv = t.B < 8 || t.C < 256;
    const uint32_t packed_bytes = t.B < 8 ? align16(g->SLW * t.B / 8 + 16) : 0u;
    const uint32_t inv_bytes = inv ? align16(g->SLW / 8 + 16) : 0u;
    for (int st = (mode == OUT_COMPACT || tu.stages == 0) ? 2 : tu.stages; st >= 2; --st) {
        g->nstages = static_cast<uint32_t>(st);
        g->off_packed = g->nstages * g->SLW;
        g->off_inv = align16(g->off_packed + packed_bytes);
        g->off_res = align16(g->off_inv + inv_bytes);
        g->off_queue = g->off_res + kResBytes;
        g->off_meta = g->off_queue + kQueueBytes;
        g->warp_bytes = align16(g->off_meta + 16u);
        g->off_warp = align16(kOffJ + t.jbytes);
        g->smem = g->off_warp + nw * g->warp_bytes;
        if (static_cast<int>(g->smem) <= max_smem) return true;
    }
    return false;
}

template <int B, bool INV, typename GT, int MODE>
cudaError_t launch_one(const WarpParams &p, uint32_t grid, uint32_t block, uint32_t smem, int max_smem,
                       cudaStream_t stream) {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void (*kernel)(const WarpParams);
    if constexpr (MODE == OUT_COMPACT)
        kernel = pfac_match_compact<B, INV, GT>;
    else
        kernel = pfac_match<B, INV, GT, MODE>;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    kernel<<<grid, block, smem, stream>>>(p);
    return cudaGetLastError();
}

template <int B, bool INV, typename GT>
cudaError_t launch_modes(OutMode mode, const WarpParams &p, uint32_t grid, uint32_t block, uint32_t smem,
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
cudaError_t launch_gt(const DevTables &t, OutMode mode, const WarpParams &p, uint32_t grid, uint32_t block,
                      uint32_t smem, int max_smem, cudaStream_t stream) {
    if (t.B != 8) return cudaErrorInvalidValue;  // small alphabets use the filter kernel
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

uint32_t tiled_tile_positions() { return kTW; }

size_t scratch_bytes(const DevTables &t, uint64_t n, OutMode mode, const Tuning &tu) {
    (void)t;
    if (mode != OUT_COMPACT) return 16;
    const uint64_t nw = static_cast<uint64_t>(tu.block) / 32u;
    const uint64_t tiles = (n + 15 + kPass - 1) / kPass;
    const uint64_t chunks = (tiles + nw - 1) / nw;
    return static_cast<size_t>(16 + 8 * (chunks + 2));  // tile counter, one look-back word per chunk
}

cudaError_t launch_tiled(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                         cudaStream_t stream) {
    if (tu.block < 32 || tu.block > kMaxBlock || (tu.block & 31) || (tu.stages != 0 && tu.stages < 2) ||
        tu.stages > kMaxStages)
        return cudaErrorInvalidValue;
    DeviceProps dp;
    cudaError_t e = device_props(&dp);
    if (e != cudaSuccess) return e;
    const bool batch = r.batch != nullptr;
    if (batch && (mode != OUT_DENSE || !r.lists)) return cudaErrorInvalidValue;
    WarpParams p{};
    p.text = r.text;
    p.n = r.n;
    p.batch = r.batch;
    p.lists = r.lists;
    const uint32_t head = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(r.text) & 15u);
    Geometry g;
    if (!make_geometry(t, batch ? 0 : r.n, head, mode, tu, dp.max_smem, &g)) return cudaErrorInvalidConfiguration;
    p.tw = tile_len(mode);
    p.SLW = g.SLW;
    p.nstages = g.nstages;
    p.ntiles = g.ntiles;
    p.off_warp = g.off_warp;
    p.warp_bytes = g.warp_bytes;
    p.off_packed = g.off_packed;
    p.off_inv = g.off_inv;
    p.off_res = g.off_res;
    p.off_queue = g.off_queue;
    p.off_meta = g.off_meta;
    p.G = t.G;
    p.Jg = t.J;
    p.J2 = t.J2;
    p.cls8g = t.cls8;
    p.C = t.C;
    p.W = t.W;
    p.k = t.k;
    p.k2 = t.k2;
    p.base_k = t.base_k;
    p.maxlen = t.maxlen;
    p.jbytes = t.jbytes;
    p.jslow = t.jslow ? 1 : 0;
    p.hash_shift = t.hash_shift;
    p.hcode_lo = t.hash_code[0];
    p.hcode_hi = t.hash_code[1];
    p.hbyte_lo = t.hash_byte[0];
    p.hbyte_hi = t.hash_byte[1];
    p.out = r.out;
    p.cpos = r.pos;
    p.cids = r.ids;
    p.cap = r.cap;
    p.count = r.count;
    const size_t need_scratch = scratch_bytes(t, r.n, mode, tu);
    if (!r.scratch || r.scratch_bytes < need_scratch) return cudaErrorInvalidValue;
    p.counter = static_cast<unsigned int *>(r.scratch);
    if (mode == OUT_COMPACT)
        p.status = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(r.scratch) + 16);
    const uint32_t nw = static_cast<uint32_t>(tu.block) / 32u;
    uint32_t grid = tu.grid > 0 ? static_cast<uint32_t>(tu.grid) : static_cast<uint32_t>(dp.sms);
    if (!batch) {  // a batch's units are counted on the device: every CTA starts
        const uint32_t need = (g.ntiles + nw - 1) / nw;
        if (grid > need) grid = need;
    }
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

cudaError_t device_error_word(unsigned int **ptr) {
    static unsigned int *cache[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!cache[dev]) {
        void *a = nullptr;
        e = cudaGetSymbolAddress(&a, g_dev_error);
        if (e != cudaSuccess) return e;
        cache[dev] = static_cast<unsigned int *>(a);
    }
    *ptr = cache[dev];
    return cudaSuccess;
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
