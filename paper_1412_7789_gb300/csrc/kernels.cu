// Failureless Aho-Corasick matching kernels for large alphabets (8-bit codes:
// more than 16 distinct keyword bytes), sm_103a.
//
// pfac_walk8 -- the production kernel.  Persistent CTAs (one per SM); every
//   warp owns a private ring of `stages` text buffers in shared memory and
//   works on tiles of 1024 positions (two passes of 512) independently of the
//   other warps (no block-wide barrier after start-up):
//   * a tile plus a 16-byte halo is fetched with one bulk async copy
//     (cp.async.bulk, the TMA unit, no multicast) that completes on the stage's
//     mbarrier, several tiles ahead of use;
//   * each lane takes 16 positions of a pass and maps the bytes of their
//     windows to class codes (byte table in shared memory) when keywords use
//     fewer than 256 byte values; one shared-memory lookup per position in the
//     root jump table (the goto table's top k levels flattened, resident for
//     the whole kernel) gives the result of every position whose walk ends
//     within k characters, and the depth-k state of the others;
//   * the others ("survivors") go to the warp's queue and from there into the
//     warp's short walk slots (8 per lane, in registers), refilled as walks
//     end; all slots advance together one character per step (the next byte
//     from the stage, one goto-table entry), and each result goes to the
//     pass's buffer in shared memory, so a pass is written out with coalesced
//     16-byte stores;
//   * the few walks still alive a few steps after the queue empties move to
//     long slots (2 per lane) that follow them across passes and tiles,
//     reading bytes from global memory, so the warp never waits for its
//     longest walk; a long walk writes its own result;
//   * output: dense ids, a count (one atomic per warp), or slots (per tile
//     the number of matches and the first kSlotCap of them) from which
//     compact.cu makes the compacted list.
//   Work units are the tiles of one text, or of all texts of one automaton in
//   a batch (the planned list), claimed from a global counter.
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
constexpr uint32_t kTW = 2 * kPass;      // positions per tile
constexpr uint32_t kHalo = 16;           // staged bytes past the tile (jump windows read up to 12)
constexpr uint32_t kSLW = kTW + kHalo;   // staged bytes per tile
// shared-memory header
constexpr uint32_t kOffJBar = 0;
constexpr uint32_t kOffStageBar = 64;                                   // kMaxWarps * kMaxStages * 8
constexpr uint32_t kOffStageTile = kOffStageBar + kMaxWarps * kMaxStages * 8;
constexpr uint32_t kOffCls = 1024;                                      // 256 x uint8
constexpr uint32_t kOffJ = 1280;                                        // root jump table
constexpr unsigned kFull = 0xffffffffu;
// queue entry: tile position (10 bits), walk-from-the-root flag (bit 10),
// depth-k state offset (bits 11-25)
constexpr uint32_t kQPos = 0x3FFu;
constexpr uint32_t kQSlow = 1u << 10;
constexpr uint32_t kQOffShift = 11;

struct WarpParams {
    const uint8_t *text;    // batch: base of all texts
    uint64_t n;
    const BatchHead *batch; // batch: this automaton's head and the planned list
    const BatchItemDev *lists;
    uint32_t nstages, ntiles;
    const void *G;
    const int16_t *Jg;
    const uint8_t *cls8g;
    uint32_t C, W, k, base_k, maxlen, jbytes;
    int32_t *out;           // batch: base of all outputs
    unsigned long long *count;
    SlotOut sl;
    unsigned int *counter;  // next tile to claim
    uint32_t off_warp, warp_bytes, off_queue, off_pass, off_meta;
    unsigned long long wait_ns;  // bounded waits give up after this
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
            issue_text_tile(tile_text(p, wk, u, item), kTW, kSLW, bar, st);
    }
}

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int b) {
    return __byte_perm(w, 0u, 0x4440u | static_cast<uint32_t>(b));
}

// Four class-table values (bytes, 0xFF = byte in no keyword) of the bytes of w.
__device__ __forceinline__ uint32_t classify4(const uint8_t *cls8, uint32_t w) {
    const uint32_t t0 = cls8[byte_of(w, 0)], t1 = cls8[byte_of(w, 1)];
    const uint32_t t2 = cls8[byte_of(w, 2)], t3 = cls8[byte_of(w, 3)];
    return __byte_perm(__byte_perm(t0, t1, 0x0040u), __byte_perm(t2, t3, 0x0040u), 0x5410u);
}

// Codes of positions i..i+7 of the stage, first in the low byte.
__device__ __forceinline__ uint64_t code_window(const uint8_t *st, uint32_t i) {
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(st);
    const uint32_t w = i >> 2, sh = 8u * (i & 3u);
    const uint32_t a = s32[w], b = s32[w + 1], c = s32[w + 2];
    return static_cast<uint64_t>(__funnelshift_r(a, b, sh)) | (static_cast<uint64_t>(__funnelshift_r(b, c, sh)) << 32);
}

__device__ __forceinline__ int jump_at(const uint8_t *jbase, uint32_t idx) {
    return *reinterpret_cast<const int16_t *>(jbase + 2u * idx);
}

// Walks that outlive their pass ("long" walks), SL per lane, carried across
// passes and tiles.  A walk is at goto state `state`; `tp` points at its next
// text byte, of which `rem` remain in its text (clamped), and `nb` is that
// byte, loaded one step ahead.  Its result goes to `op` (dense) or to slot
// unit `su` at text position `pos` (slots).
template <int SL>
struct LongWalks {
    uint32_t act;  // bit t: slot t holds a walk
    uint32_t state[SL];
    const uint8_t *tp[SL];
    uint32_t rem[SL];
    uint32_t nb[SL];
    int32_t *op[SL];
    uint32_t pos[SL];
    uint32_t su[SL];
};

// Walks of the current pass ("short" walks), SS per lane: state, stage index
// of the next byte, that byte (loaded one step ahead), pass position.
template <int SS>
struct ShortWalks {
    uint32_t act;
    uint32_t state[SS];
    uint32_t q[SS];
    uint32_t nb[SS];
    uint32_t i[SS];
};

template <int MODE>
__device__ __forceinline__ void emit(const WarpParams &p, int32_t *op, uint32_t su, uint32_t pos, int r,
                                     unsigned long long &cnt) {
    if (MODE == OUT_DENSE) {
        __stcs(op, r);
    } else if (MODE == OUT_COUNT) {
        cnt += r >= 0 ? 1ull : 0ull;
    } else {
        if (op) __stcs(op, r);  // the tile's dense fallback
        if (r < 0) return;
        const uint32_t idx = atomicAdd(p.sl.counts + su, 1u);
        if (idx < kSlotCap)
            p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + idx] =
                (static_cast<unsigned long long>(static_cast<uint32_t>(r)) << 32) | pos;
    }
}

// The goto column of byte b: its class, or the end column C for a byte in no
// keyword (whose entry always holds the result of stopping there).
template <bool INV>
__device__ __forceinline__ uint32_t column_of(const WarpParams &p, const uint8_t *cls8, uint32_t b) {
    if (!INV) return b;
    const uint32_t v = cls8[b];
    return v != 0xFFu ? v : p.C;
}

// States are numbered in breadth-first order, so a live goto entry is always a
// larger state than the one it leaves: a table that breaks this ends the walk
// with the error latched instead of looping.
__device__ __forceinline__ bool walk_ends(int e, uint32_t state) {
    return e < 0 || static_cast<uint32_t>(e) <= state;
}

__device__ __forceinline__ int walk_result(int e) {
    if (e >= 0) {
        atomicOr(&g_dev_error, static_cast<unsigned>(kErrWalk));
        return -1;
    }
    return decode_dead(e);
}

// One step of every long walk of the lane (text bytes from global memory).
template <bool INV, typename GT, int MODE, int SL>
__device__ __forceinline__ void step_long(const WarpParams &p, const uint8_t *cls8, LongWalks<SL> &w,
                                          unsigned long long &cnt) {
    const GT *G = static_cast<const GT *>(p.G);
    int e[SL];
#pragma unroll
    for (int t = 0; t < SL; ++t) {
        if ((w.act >> t) & 1u) {
            const uint32_t c = w.rem[t] ? column_of<INV>(p, cls8, w.nb[t]) : p.C;
            e[t] = goto_ld(G, w.state[t], p.W, c);
            if (w.rem[t] > 1) w.nb[t] = __ldg(w.tp[t] + 1);
        }
    }
#pragma unroll
    for (int t = 0; t < SL; ++t) {
        if ((w.act >> t) & 1u) {
            if (walk_ends(e[t], w.state[t])) {
                emit<MODE>(p, w.op[t], w.su[t], w.pos[t], walk_result(e[t]), cnt);
                w.act &= ~(1u << t);
            } else {
                w.state[t] = static_cast<uint32_t>(e[t]);
                w.tp[t] += 1;
                w.rem[t] -= 1;
            }
        }
    }
}

// One step of every short walk of the lane: bytes from the stage (from global
// memory past the staged bytes), results into the pass buffer.
template <bool INV, typename GT, int SS>
__device__ __forceinline__ void step_short(const WarpParams &p, const TileText &tt, const uint8_t *st,
                                           const uint8_t *cls8, int64_t gpb, ShortWalks<SS> &w, int32_t *pb) {
    const GT *G = static_cast<const GT *>(p.G);
    const int64_t n = static_cast<int64_t>(tt.n);
    int e[SS];
    uint32_t nx[SS];
#pragma unroll
    for (int t = 0; t < SS; ++t) {
        if ((w.act >> t) & 1u) {
            const int64_t gp = gpb + w.q[t];
            const uint32_t c = gp < n ? column_of<INV>(p, cls8, w.nb[t]) : p.C;
            e[t] = goto_ld(G, w.state[t], p.W, c);
            const uint32_t q1 = w.q[t] + 1;
            nx[t] = 0;
            if (q1 < kSLW)
                nx[t] = st[q1];
            else if (gp + 1 < n)
                nx[t] = __ldg(tt.text + gp + 1);
        }
    }
#pragma unroll
    for (int t = 0; t < SS; ++t) {
        if ((w.act >> t) & 1u) {
            if (walk_ends(e[t], w.state[t])) {
                pb[w.i[t]] = walk_result(e[t]);
                w.act &= ~(1u << t);
            } else {
                w.state[t] = static_cast<uint32_t>(e[t]);
                w.q[t] += 1;
                w.nb[t] = nx[t];
            }
        }
    }
}

// All lanes: give the queued survivors [head, qn) of the current pass to free
// short slots, in lane order (a warp scan of the free-slot counts).  Returns
// the new head.
template <int SS>
__device__ __forceinline__ uint32_t refill(const WarpParams &p, const uint8_t *st, uint32_t pbase,
                                           const uint32_t *queue, uint32_t head, uint32_t qn, ShortWalks<SS> &w,
                                           int lane) {
    const uint32_t freem = ~w.act & ((1u << SS) - 1u);
    const uint32_t nf = __popc(freem);
    uint32_t inc = nf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    const uint32_t tot = __shfl_sync(kFull, inc, 31);
    uint32_t qi = head + inc - nf;
#pragma unroll
    for (int t = 0; t < SS; ++t) {
        if (((freem >> t) & 1u) && qi < qn) {
            const uint32_t e = queue[qi++];
            const uint32_t i = e & kQPos;
            const bool slow = (e & kQSlow) != 0;
            w.state[t] = slow ? 0u : p.base_k + (e >> kQOffShift);
            w.q[t] = i + (slow ? 0u : p.k);
            w.nb[t] = st[w.q[t]];  // i + k < kSLW
            w.i[t] = i - pbase;
            w.act |= 1u << t;
        }
    }
    const uint32_t nh = head + tot;
    return nh < qn ? nh : qn;
}

// Pass-buffer mark of a position whose walk moved to a long slot: the pass
// does not write it, the long walk does.
constexpr int kLongMark = INT_MIN;

// Move the lane's short walks into free long slots (as many as fit).
template <int SS, int SL>
__device__ __forceinline__ void spill(const WarpParams &p, const TileText &tt, int64_t gpb, uint32_t pbase,
                                      uint32_t su, ShortWalks<SS> &s, LongWalks<SL> &l, int32_t *pb,
                                      bool slots_mode, int32_t *tile_dense) {
#pragma unroll
    for (int t = 0; t < SS; ++t) {
        if ((s.act >> t) & 1u) {
#pragma unroll
            for (int u = 0; u < SL; ++u) {
                if (((s.act >> t) & 1u) && !((l.act >> u) & 1u)) {
                    const uint64_t gq = static_cast<uint64_t>(gpb + s.q[t]);
                    const uint64_t gpos = static_cast<uint64_t>(gpb + pbase + s.i[t]);
                    const uint64_t left = tt.n > gq ? tt.n - gq : 0;
                    l.state[u] = s.state[t];
                    l.tp[u] = tt.text + gq;
                    l.rem[u] = left > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(left);
                    l.nb[u] = s.nb[t];
                    // dense: the id's place; slots: the tile's dense fallback, if kept
                    l.op[u] = !slots_mode ? tt.out + gpos : (tile_dense ? tile_dense + pbase + s.i[t] : nullptr);
                    l.pos[u] = static_cast<uint32_t>(gpos);
                    l.su[u] = su;
                    l.act |= 1u << u;
                    s.act &= ~(1u << t);
                    pb[s.i[t]] = kLongMark;
                }
            }
        }
    }
}

// Rounds a pass keeps stepping its short walks after its queue is empty,
// before the walks still alive move to long slots.
constexpr uint32_t kExtraRounds = 4;

// One pass of 512 positions: root jump table per position; the positions it
// resolves go to the pass buffer, the others are walked in short slots
// (refilled from the queue as walks end) into the pass buffer; walks still
// alive a few rounds after the queue empties move to long slots; then the
// pass buffer is written out (dense: coalesced 16-byte stores), counted, or
// its matches are appended to the tile's slots.  su: the slot unit of the tile.
template <bool INV, typename GT, int MODE, int SS, int SL>
__device__ __forceinline__ void walk_pass(const WarpParams &p, const TileText &tt, const uint8_t *st,
                                          const uint8_t *cls8, const uint8_t *jbase, uint32_t *queue, int32_t *pb,
                                          int64_t gpb, bool interior, uint32_t su, uint32_t h, int lane,
                                          ShortWalks<SS> &sw, LongWalks<SL> &lw, unsigned long long &cnt) {
    const int64_t n = static_cast<int64_t>(tt.n);
    const uint32_t k = p.k;
    const uint32_t kmask = (1u << (8u * k)) - 1u;
    const uint32_t pbase = h * kPass;
    const uint32_t ibase = pbase + 4u * static_cast<uint32_t>(lane);

    // 1. one root-jump lookup per position: the result (>= -1), the depth-k
    //    state (<= -2), or kJumpSlow (walk from the root)
    int res[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint64_t x = code_window(st, ibase + 128u * g);
        if (INV)  // class codes of the window's bytes (0xFF: a byte in no keyword stops the walk)
            x = static_cast<uint64_t>(classify4(cls8, static_cast<uint32_t>(x))) |
                (static_cast<uint64_t>(classify4(cls8, static_cast<uint32_t>(x >> 32))) << 32);
#pragma unroll
        for (int r = 0; r < 4; ++r)
            res[4 * g + r] = k ? jump_at(jbase, static_cast<uint32_t>(x >> (8 * r)) & kmask) : kJumpSlow;
    }
    uint32_t valid = 0xFFFFu;
    if (!interior) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int j = 4 * g + r;
                const int64_t gp = gpb + ibase + 128u * g + r;
                if (gp < 0 || gp >= n) {
                    res[j] = -1;
                    valid &= ~(1u << j);
                } else if (gp + static_cast<int64_t>(k) > n) {
                    res[j] = kJumpSlow;  // the window runs past the text end
                }
            }
        }
    }
    uint32_t sv = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) sv |= (res[j] < -1 ? 1u : 0u) << j;

    // 2. resolved results (survivors: -1 until their walk ends) into the pass
    //    buffer; survivors into the queue
#pragma unroll
    for (int g = 0; g < 4; ++g)
        reinterpret_cast<int4 *>(pb)[32 * g + lane] =
            make_int4(res[4 * g] < -1 ? -1 : res[4 * g], res[4 * g + 1] < -1 ? -1 : res[4 * g + 1],
                      res[4 * g + 2] < -1 ? -1 : res[4 * g + 2], res[4 * g + 3] < -1 ? -1 : res[4 * g + 3]);
    const uint32_t c = __popc(sv);
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    const uint32_t qn = __shfl_sync(kFull, inc, 31);
    {
        uint32_t o = inc - c, m = sv;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t i = ibase + 128u * (j >> 2) + (j & 3);
            const int v = res[j];
            queue[o++] = v == kJumpSlow ? (i | kQSlow) : (i | (static_cast<uint32_t>(-v - 2) << kQOffShift));
        }
    }
    __syncwarp();

    // 3. the walks
    uint32_t head = 0, extra = 0;
    for (;;) {
        head = refill<SS>(p, st, pbase, queue, head, qn, sw, lane);
        if (head >= qn) {
            if (extra >= kExtraRounds)
                spill<SS, SL>(p, tt, gpb, pbase, su, sw, lw, pb, MODE == OUT_SLOTS,
                              MODE == OUT_SLOTS && p.sl.dense ? p.sl.dense + static_cast<uint64_t>(su) * kDenseStride
                                                              : nullptr);
            if (!__any_sync(kFull, sw.act != 0)) break;
            ++extra;
        }
        step_short<INV, GT, SS>(p, tt, st, cls8, gpb, sw, pb);
        if (lw.act) step_long<INV, GT, MODE, SL>(p, cls8, lw, cnt);
    }
    __syncwarp();  // the pass buffer is complete (long walks hold kLongMark)

    // 4. out
    if (MODE == OUT_DENSE) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int4 v = reinterpret_cast<const int4 *>(pb)[32 * g + lane];
            const int64_t gp0 = gpb + ibase + 128u * g;
            const uint32_t vm = (valid >> (4 * g)) & 0xFu;
            const bool marked = v.x == kLongMark || v.y == kLongMark || v.z == kLongMark || v.w == kLongMark;
            if (tt.vec_ok && vm == 0xFu && !marked) {
                __stcs(reinterpret_cast<int4 *>(tt.out + gp0), v);
            } else {
                const int rr[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (((vm >> r) & 1u) && rr[r] != kLongMark) __stcs(tt.out + gp0 + r, rr[r]);
            }
        }
    } else {
        int rr[16];
        uint32_t hit = 0;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int4 v = reinterpret_cast<const int4 *>(pb)[32 * g + lane];
            rr[4 * g] = v.x;
            rr[4 * g + 1] = v.y;
            rr[4 * g + 2] = v.z;
            rr[4 * g + 3] = v.w;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) hit |= (rr[j] >= 0 ? 1u : 0u) << j;
        hit &= valid;
        if (MODE == OUT_COUNT) {
            cnt += __popc(hit);
        } else {
            if (p.sl.dense) {  // the tile may overflow its slots: keep its dense ids
                int32_t *dn = p.sl.dense + static_cast<uint64_t>(su) * kDenseStride;
#pragma unroll
                for (int g = 0; g < 4; ++g)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (((valid >> (4 * g + r)) & 1u) && rr[4 * g + r] != kLongMark)
                            __stcs(dn + ibase + 128u * g + r, rr[4 * g + r]);
            }
            const uint32_t mine = __popc(hit);
            uint32_t sc = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, sc, d);
                if (lane >= d) sc += y;
            }
            const uint32_t tot = __shfl_sync(kFull, sc, 31);
            uint32_t base = 0;
            if (lane == 0 && tot) base = atomicAdd(p.sl.counts + su, tot);
            base = __shfl_sync(kFull, base, 0) + sc - mine;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if ((hit >> j) & 1u) {
                    if (base < kSlotCap) {
                        const uint32_t pos = static_cast<uint32_t>(gpb + ibase + 128u * (j >> 2) + (j & 3));
                        p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + base] =
                            (static_cast<unsigned long long>(static_cast<uint32_t>(rr[j])) << 32) | pos;
                    }
                    ++base;
                }
            }
        }
    }
    __syncwarp();  // the pass buffer and queue are reused by the next pass
}

template <bool INV, typename GT, int MODE, int SS, int SL, bool BATCH>
__global__ void __launch_bounds__(kMaxBlock, 1) pfac_walk8(const WarpParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t *jbar = reinterpret_cast<uint64_t *>(smem + kOffJBar);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffStageBar) + warp * kMaxStages;
    uint32_t *stile = reinterpret_cast<uint32_t *>(smem + kOffStageTile) + warp * kMaxStages;
    uint8_t *wreg = smem + p.off_warp + static_cast<size_t>(warp) * p.warp_bytes;
    uint32_t *queue = reinterpret_cast<uint32_t *>(wreg + p.off_queue);
    int32_t *pb = reinterpret_cast<int32_t *>(wreg + p.off_pass);
    uint32_t *sitem = reinterpret_cast<uint32_t *>(wreg + p.off_meta);
    const uint8_t *cls8 = smem + kOffCls;
    const uint8_t *jbase = smem + kOffJ;
    const uint32_t nst = p.nstages;
    // one text: a null list the compiler sees, so the batch lookups fold away
    const Work wk = BATCH ? load_work(p.batch, p.lists, p.ntiles) : load_work(nullptr, nullptr, p.ntiles);

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
    // Tiles: the first one per warp statically (warp-major numbering, so
    // neighbouring tiles land on different SMs), the rest from a global counter.
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
    for (uint32_t s = 0; s < nst; ++s)
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], wreg + s * kSLW, next_tile(s), lane);

    ShortWalks<SS> sw;
    sw.act = 0;
    LongWalks<SL> lw;
    lw.act = 0;
    unsigned long long cnt = 0;
    bool ok = mbar_wait(jbar, 0, p.wait_ns);
    // stage s of iteration it is it % nst, its phase parity (it / nst) & 1
    for (uint32_t it = 0, s = 0, par = 0;; ++it, s = s + 1 == nst ? 0u : s + 1, par ^= s == 0 ? 1u : 0u) {
        ok = ok && mbar_wait(&bars[s], par, p.wait_ns);
        if (!__all_sync(kFull, ok)) {
            // A copy never completed: latch the error, let this warp's copies in
            // flight finish (bounded), and leave.
            if (lane == 0) {
                atomicOr(&g_dev_error, static_cast<unsigned>(kErrTimeout));
                mbar_wait(jbar, 0, p.wait_ns);
                for (uint32_t j = it; j < it + nst; ++j) mbar_wait(&bars[j % nst], (j / nst) & 1u, p.wait_ns);
            }
            return;
        }
        const uint32_t tile = stile[s];
        if (tile >= wk.units) break;
        const TileText tt = tile_text(p, wk, tile, sitem[s]);
        uint8_t *st = wreg + s * kSLW;
        const uint64_t tlo = static_cast<uint64_t>(tt.tile) * kTW;
        const int64_t gpb = static_cast<int64_t>(tlo) - tt.head;
        const bool interior = gpb >= 0 && gpb + static_cast<int64_t>(kSLW) <= static_cast<int64_t>(tt.n);
        if (!interior) {
            load_text_fringe(tt, kSLW, st, tlo, lane);
            __syncwarp();
        }
        const uint32_t su = p.sl.ubase + tile;
#pragma unroll 1
        for (uint32_t h = 0; h < kTW / kPass; ++h)
            walk_pass<INV, GT, MODE, SS, SL>(p, tt, st, cls8, jbase, queue, pb, gpb, interior, su, h, lane, sw, lw,
                                             cnt);
        if (lane == 0) fence_proxy_async_smem();
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], st, next_tile(it + nst), lane);
    }
    // the walks still in the slots
    while (__any_sync(kFull, lw.act != 0)) step_long<INV, GT, MODE, SL>(p, cls8, lw, cnt);

    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
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
constexpr int kShortSlots = 8;
constexpr int kLongSlots = 2;

inline uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

template <bool INV, typename GT, int MODE, bool BATCH>
cudaError_t launch_one(const WarpParams &p, uint32_t grid, uint32_t block, uint32_t smem, int max_smem,
                       cudaStream_t stream) {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void (*kernel)(const WarpParams) = pfac_walk8<INV, GT, MODE, kShortSlots, kLongSlots, BATCH>;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    kernel<<<grid, block, smem, stream>>>(p);
    return cudaGetLastError();
}

template <bool INV, typename GT>
cudaError_t launch_modes(OutMode mode, const WarpParams &p, uint32_t grid, uint32_t block, uint32_t smem,
                         int max_smem, cudaStream_t stream) {
    switch (mode) {
        case OUT_DENSE:
            return p.batch ? launch_one<INV, GT, OUT_DENSE, true>(p, grid, block, smem, max_smem, stream)
                           : launch_one<INV, GT, OUT_DENSE, false>(p, grid, block, smem, max_smem, stream);
        case OUT_COUNT:
            return launch_one<INV, GT, OUT_COUNT, false>(p, grid, block, smem, max_smem, stream);
        case OUT_SLOTS:
            return p.batch ? launch_one<INV, GT, OUT_SLOTS, true>(p, grid, block, smem, max_smem, stream)
                           : launch_one<INV, GT, OUT_SLOTS, false>(p, grid, block, smem, max_smem, stream);
        default:
            return cudaErrorInvalidValue;
    }
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

cudaError_t launch_tiled(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                         cudaStream_t stream) {
    const int blk = tu.block > 0 ? tu.block : kMaxBlock;  // 0: the default, 512
    if (blk < 32 || blk > kMaxBlock || (blk & 31) || (tu.stages != 0 && tu.stages < 2) || tu.stages > kMaxStages)
        return cudaErrorInvalidValue;
    if (t.B != 8) return cudaErrorInvalidValue;  // small alphabets use the filter kernel
    // default (variant 0): the full-occupancy one-thread-per-position kernel,
    // the fastest of the three on the 256-value Zipf workloads
    if (tu.variant != 1) return launch_jump8(t, r, mode, tu.variant != 2, tu.wait_ns, stream);
    if (mode != OUT_DENSE && mode != OUT_COUNT && mode != OUT_SLOTS) return cudaErrorInvalidValue;
    const bool batch = r.batch != nullptr;
    if (batch && (mode == OUT_COUNT || !r.lists)) return cudaErrorInvalidValue;
    if (mode == OUT_SLOTS && (!r.slots.counts || !r.slots.slots)) return cudaErrorInvalidValue;
    if (t.k > 2 || t.base_k + kJumpMaxStates < t.base_k) return cudaErrorInvalidValue;
    DeviceProps dp;
    cudaError_t e = device_props(&dp);
    if (e != cudaSuccess) return e;
    WarpParams p{};
    p.text = r.text;
    p.n = r.n;
    p.batch = r.batch;
    p.lists = r.lists;
    uint64_t tiles = 0;
    if (!batch) {
        const uint64_t head = reinterpret_cast<uintptr_t>(r.text) & 15u;
        tiles = (r.n + head + kTW - 1) / kTW;
        if (tiles >= 0x7FFFFFFFull) return cudaErrorInvalidValue;
    }
    p.ntiles = static_cast<uint32_t>(tiles);
    // per warp: stages, survivor queue, pass buffer, stage descriptors
    const uint32_t nw = static_cast<uint32_t>(blk) / 32u;
    uint32_t smem = 0;
    bool fits = false;
    for (int st = tu.stages ? tu.stages : 3; st >= 2 && !fits; --st) {
        p.nstages = static_cast<uint32_t>(st);
        p.off_queue = p.nstages * kSLW;
        p.off_pass = p.off_queue + kPass * 4u;
        p.off_meta = p.off_pass + kPass * 4u;
        p.warp_bytes = align16(p.off_meta + 16u);
        p.off_warp = align16(kOffJ + t.jbytes);
        smem = p.off_warp + nw * p.warp_bytes;
        fits = static_cast<int>(smem) <= dp.max_smem;
    }
    if (!fits) return cudaErrorInvalidConfiguration;
    p.G = t.G;
    p.Jg = t.J;
    p.cls8g = t.cls8;
    p.C = t.C;
    p.W = t.W;
    p.k = t.k;
    p.base_k = t.base_k;
    p.maxlen = t.maxlen;
    p.jbytes = t.jbytes;
    p.wait_ns = tu.wait_ns ? tu.wait_ns : kWaitNs;
    p.out = r.out;
    p.count = r.count;
    p.sl = r.slots;
    // the tile counter; none is needed when every tile is some warp's first
    p.counter = r.scratch && r.scratch_bytes >= 16 ? static_cast<unsigned int *>(r.scratch) : nullptr;
    uint32_t grid = tu.grid > 0 ? static_cast<uint32_t>(tu.grid) : static_cast<uint32_t>(dp.sms);
    if (!batch) {  // a batch's units are counted on the device: every CTA starts
        const uint32_t need = (p.ntiles + nw - 1) / nw;
        if (grid > need) grid = need;
    }
    if (!p.counter && (batch || static_cast<uint64_t>(p.ntiles) > static_cast<uint64_t>(grid) * nw))
        return cudaErrorInvalidValue;
    if (grid == 0) return cudaSuccess;
    const uint32_t block = static_cast<uint32_t>(blk);
    const bool inv = t.C < 256;
    if (t.gbits == 16) {
        if (inv) return launch_modes<true, int16_t>(mode, p, grid, block, smem, dp.max_smem, stream);
        return launch_modes<false, int16_t>(mode, p, grid, block, smem, dp.max_smem, stream);
    }
    if (inv) return launch_modes<true, int32_t>(mode, p, grid, block, smem, dp.max_smem, stream);
    return launch_modes<false, int32_t>(mode, p, grid, block, smem, dp.max_smem, stream);
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
