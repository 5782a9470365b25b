// Failureless Aho-Corasick matching with a root filter, sm_103a: keyword
// bytes mapped to 2- or 4-bit codes (small alphabets: the filter is exact over
// windows of k codes), or 8-bit codes (any alphabet: the filter is hashed over
// windows of kh = min(4, shortest keyword) codes, and survivors find their
// depth-kh state in a hash of those states).
//
// pfac_filter_pipe -- persistent CTAs (one per SM), every warp on its own tiles
// of 992 positions (two halves of 496), no block-wide barrier after start-up:
//   * a tile plus a halo is fetched with one bulk async copy (cp.async.bulk,
//     the TMA unit, no multicast) into one of the warp's shared-memory stages,
//     completing on that stage's mbarrier, `stages` tiles ahead of use;
//   * lane l classifies the 16 bytes at 16 l of each half once (byte permutes
//     on a 3-bit hash, or the byte table), packs their codes into one word (two
//     for 4-bit codes) and gets the next lane's word with one shuffle, so each
//     of its start positions has its window of codes in registers; lane 31
//     only supplies the look-ahead word;
//   * one bit per position from the root filter (resident in shared memory for
//     the whole kernel): clear means the walk from the root stops within the
//     first k characters with no keyword, i.e. the result is -1 -- almost every
//     position of a text whose keywords are longer than k;
//   * the other positions ("survivors") are resolved by one load from the
//     window table (depth-k state or result; with 8-bit codes one bucket of
//     the state hash), one from the stride table (k2 more characters), and
//     the goto table one character at a time (chain records for the long
//     unbranched runs of deep states).  A
//     tile with at most one survivor per lane keeps them "in flight" across the
//     next two tiles, so their dependent loads overlap other work; a tile with
//     more finishes them at once, eight walks per lane per round of 256 (in the
//     HELP forms, used for short texts, the rounds of such a tile are shared
//     with the CTA's warps that have run out of tiles);
//   * output: dense ids (one bulk async store of a constant -1 buffer when no
//     survivor found a keyword, else -1 stores and the survivors' ids), a count
//     (one atomic per warp), or slots (per tile the number of matches and the
//     first kSlotCap of them) from which compact.cu makes the compacted list.
// Work units are the tiles of one text, or of all texts of one automaton in a
// batch (the planned list), claimed from a global counter.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "pfac_device.cuh"

namespace pfac {

// The kernel and its launch templates; filter.cu launches the plain forms,
// filter_help.cu the forms whose heavy tiles are shared within the CTA.
namespace filt {

// Threads per CTA: up to 512 for every form (128 registers a thread), up to
// 640 for the one-phase single-text forms of 2- and 4-bit codes, compiled
// apart at 96 registers (20 warps per SM measured faster than 16 there).
constexpr int kStdBlock = 512;
constexpr int kMaxBlock = 640;
constexpr int kMaxWarps = kMaxBlock / 32;
constexpr int kMaxStages = 4;
constexpr uint32_t kOwnLanes = 31;            // lanes that own start positions in a pass
constexpr uint32_t kPass = 16 * kOwnLanes;    // 496 positions per pass
constexpr uint32_t kTile = 2 * kPass;         // 992 positions per warp tile
constexpr uint32_t kCodeSpan = kTile + 16;    // positions classified per tile
// shared-memory header
constexpr uint32_t kOffJBar = 0;
constexpr uint32_t kOffStageBar = 64;
constexpr uint32_t kOffStageTile = kOffStageBar + kMaxWarps * kMaxStages * 8;
constexpr uint32_t kOffRetired = 1024;  // warps of the CTA done with their own tiles
constexpr uint32_t kOffOffers = 1028;   // heavy tiles offered and not yet finished
static_assert(kOffStageTile + kMaxWarps * kMaxStages * 4 <= kOffRetired && kOffOffers + 4 <= 1152,
              "CTA counters overlap the stage descriptors or the class map");
constexpr uint32_t kOffCls = 1152;  // 256 x uint8
constexpr uint32_t kOffF = 1408;    // root filter bits
constexpr unsigned kFull = 0xffffffffu;
// Texts of at most this many tiles per warp of the grid take the forms that
// share heavy tiles within the CTA.
constexpr uint32_t kHelpTilesPerWarp = 16;
// Entries of the phased form's lists a warp reserves at a time.
constexpr uint32_t kListChunk = 1024;
constexpr uint32_t kWalkChunk = kWalkChunkEntries;

// Walks per lane in one round of a tile with many survivors: 8 (rounds of
// 256); with 8-bit codes, whose tiles hold about a hundred survivors each and
// whose window lookups hold a 16-byte bucket per walk, 4 (rounds of 128).
template <int B>
__host__ __device__ constexpr int heavy_slots() { return B == 8 ? 4 : 8; }

struct FilterParams {
    const uint8_t *text;
    uint64_t n;
    uint32_t tile;    // positions per tile (multiple of 16)
    uint32_t staged;  // bytes staged per tile (tile + halo, multiple of 16)
    uint32_t ntiles;  // single text: its tiles
    uint32_t nstages;
    const void *G;
    const uint32_t *Fg;
    const int32_t *JK;
    const int32_t *J2;
    const uint8_t *cls8g;
    uint32_t C, W, k, k2, base_k, maxlen, fbytes;
    uint32_t famask;  // byte offsets of the root filter's words reached by a window
    int hash_shift;
    uint32_t hcode_lo, hcode_hi, hbyte_lo, hbyte_hi;
    int direct_shift;            // 1: 2-bit codes (byte >> 1) & 3, else -1
    uint32_t dsel_lo, dsel_hi;   // byte 2c of the pair: the keyword byte of code c
    uint32_t dfill;              // a byte in no keyword
    int32_t *out;
    unsigned long long *count;
    SlotOut sl;
    unsigned int *counter;
    unsigned int *err;
    uint32_t off_neg1, off_warp, warp_bytes, off_packed, off_inv, off_queue, off_meta, off_help;
    // batch: the automaton's head and the planned list (text and out are then
    // the bases of all texts and outputs)
    const BatchHead *batch;
    const BatchItemDev *lists;
    // one text: its 16-byte aligned base, the tile starts whose staged bytes
    // lie wholly in its aligned part [a1, a2), and whether its output takes
    // 16-byte stores
    const uint8_t *gbase;
    uint64_t a1, a2;
    uint32_t vec_ok;
    // chain records from state s_chain on (0xFFFFFFFF: none)
    const uint4 *skip;
    const uint8_t *chain;
    uint32_t s_chain;
    // bounded waits give up after wait_ns; stall_help: an owner waits for one
    // more finished chunk than its offered tile has (a test of that wait)
    unsigned long long wait_ns;
    uint32_t stall_help;
    uint32_t kind;  // (B << 8) | goto-entry bits, for the multi-automaton launch
    // the lists of the phased form (null: one phase); list_count[0]
    // survivors, list_count[1] walks.  One text: walks {(tile << 10) |
    // position, state | d << 31}, the next byte at position + k + k2 + d.  A
    // batch (8-bit codes; one list for the launch's automata): survivors carry
    // aidx << 16 in their third word and the unit's planned-list entry in the
    // fourth, walks4 {(unit << 10) | position, state | d << 31, aidx, entry}.
    uint4 *list;
    unsigned int *list_count;
    uint32_t list_cap;
    uint2 *walks;
    uint4 *walks4;
    uint32_t walk_cap;
    uint32_t aidx;  // the automaton's index in a multi-automaton launch
    // 8-bit codes: the codes are the bytes (256 columns), or classes from the
    // byte table; the filter index is the top bits of (window & wmask) *
    // kFilterHashMul (32 - fshift of them), the state hash's bucket the top
    // hk_bits of (window & wmask) * kStateHashMul, probed over hk_probes buckets
    uint32_t identity;
    uint32_t wmask;
    uint32_t fshift;
    const uint4 *HK;
    uint32_t hk_shift, hk_mask, hk_probes;
};

struct WarpSmem {
    const uint8_t *cls8;
    const uint32_t *F;
    uint8_t *st;
    uint32_t *packed;  // codes of the tile's kCodeSpan positions, B bits each
    uint16_t *inv;     // 16 "cannot extend a walk" bits per 16 positions
    uint16_t *queue;
    const int32_t *neg1;  // kTile x -1, shared by the CTA's warps
};

// A warp's tile with more survivors than one round of walks, offered to the
// CTA's other warps once they have no tiles of their own: chunks of 256 queued
// survivors, claimed by an atomic on `ticket` ((publication << 32) | next
// chunk).  The fields are written before the ticket is reset for a new
// publication, and a claim is valid only for the publication it names and a
// chunk below nchunks, so a stale claim never touches a new tile.  The owner
// reuses its queue and codes only after `done` reaches nchunks.
struct HelpSlot {
    unsigned long long ticket;
    uint32_t pub;      // publication the fields belong to (0: none yet)
    uint32_t nchunks;
    uint32_t done;     // chunks finished, this publication
    uint32_t tile, item, total;
    long long gpb;
    uint32_t flags;    // bit 0: interior, bit 1: clean, bit 2: results to the dense fallback too
    uint32_t su;       // slot-mode unit
};

// The text and tile of work unit u (entry `item` of the planned list in a batch).
__device__ __forceinline__ TileText tile_text(const FilterParams &p, const Work &wk, uint32_t u, uint32_t item) {
    if (!wk.list) return make_text(p.text, p.out, p.n, u);
    return batch_text(wk, p.text, p.out, item, u);
}

// All lanes: point stage s at unit u (>= wk.units: the end of this warp's
// work) and start its bulk copy.
__device__ __forceinline__ void issue_unit(const FilterParams &p, const Work &wk, uint64_t *bar, uint32_t *stile,
                                           uint32_t *sitem, uint8_t *st, uint32_t u, int lane) {
    const uint32_t item = (wk.list && u < wk.units) ? find_item(wk, u, lane) : 0u;
    if (lane == 0) {
        *stile = u;
        *sitem = item;
        const uint64_t tlo = static_cast<uint64_t>(u) * p.tile;
        if (u >= wk.units) {
            mbar_arrive(bar);
        } else if (!wk.list && tlo >= p.a1 && tlo + p.staged <= p.a2) {
            // one text, a tile inside its aligned part: the whole stage
            mbar_arrive_expect_tx(bar, p.staged);
            bulk_load_hint(st, p.gbase + tlo, p.staged, bar, policy_evict_first());
        } else {
            issue_text_tile(tile_text(p, wk, u, item), p.tile, p.staged, bar, st);
        }
    }
}

// Classify the 4 bytes of w: their class codes (one per byte) and a word whose
// non-zero bytes mark bytes in no keyword.
__device__ __forceinline__ void classify_word(const FilterParams &p, const uint8_t *cls8, uint32_t w,
                                              uint32_t &codes, uint32_t &unknown) {
    if (p.hash_shift >= 0) {
        // h = (byte >> s) & 7 selects, with byte permutes, the code of the one
        // keyword byte with that hash and the byte itself; a mismatch is a byte
        // in no keyword
        const uint32_t sh = static_cast<uint32_t>(p.hash_shift);
        const uint32_t hv = (w >> sh) & 0x07070707u;
        const uint32_t sel = __byte_perm(hv | (hv >> 4), 0u, 0x4420u);
        codes = __byte_perm(p.hcode_lo, p.hcode_hi, sel);
        unknown = w ^ __byte_perm(p.hbyte_lo, p.hbyte_hi, sel);
    } else {
        const uint32_t t0 = cls8[__byte_perm(w, 0u, 0x4440u)], t1 = cls8[__byte_perm(w, 0u, 0x4441u)];
        const uint32_t t2 = cls8[__byte_perm(w, 0u, 0x4442u)], t3 = cls8[__byte_perm(w, 0u, 0x4443u)];
        codes = __byte_perm(__byte_perm(t0, t1, 0x0040u), __byte_perm(t2, t3, 0x0040u), 0x5410u);
        unknown = codes & 0x80808080u;  // class value 0xFF marks a byte in no keyword
    }
}

// 8-bit codes: the codes of the 4 bytes of w (the bytes themselves with 256
// columns, else their classes from the byte table, 0xFF for a byte in no
// keyword) and a word whose non-zero bytes mark bytes in no keyword.
__device__ __forceinline__ void classify_word8(const FilterParams &p, const uint8_t *cls8, uint32_t w,
                                               uint32_t &codes, uint32_t &unknown) {
    if (p.identity) {
        codes = w;
        unknown = 0;
        return;
    }
    const uint32_t t0 = cls8[__byte_perm(w, 0u, 0x4440u)], t1 = cls8[__byte_perm(w, 0u, 0x4441u)];
    const uint32_t t2 = cls8[__byte_perm(w, 0u, 0x4442u)], t3 = cls8[__byte_perm(w, 0u, 0x4443u)];
    codes = __byte_perm(__byte_perm(t0, t1, 0x0040u), __byte_perm(t2, t3, 0x0040u), 0x5410u);
    const uint32_t x = ~codes;  // a zero byte: code 0xFF
    unknown = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
}

// 8-bit codes: the state hash.  Entry slot of window w (masked to kh codes),
// and the entry of w given the entry e at that slot (loaded by the caller, so
// that several lookups overlap): linear probing up to an empty entry (state
// 0) or hk_probes entries; an entry with state 0 when no depth-kh state has
// window w (a walk that does not reach depth kh finds no keyword).
__device__ __forceinline__ uint32_t hk_slot(const FilterParams &p, uint32_t w) {
    return (w * kStateHashMul) >> p.hk_shift;
}

__device__ __forceinline__ uint4 hk_find(const FilterParams &p, uint32_t w, uint4 e) {
    uint32_t b = hk_slot(p, w);
    for (uint32_t i = 1; e.y != 0u && e.x != w; ++i) {
        if (i >= p.hk_probes) return make_uint4(0u, 0u, 0u, 0u);
        b = (b + 1u) & p.hk_mask;
        e = __ldg(p.HK + b);
    }
    return e;
}

// A survivor at tile position i from its state-hash entry e and the code c of
// the character after its window (c_ok: one is there, in a keyword byte):
// true with its result r, or false with its walk to go on from state s at
// tile position q.  A depth-kh state with one child: the walk stops there
// (result: the state's) unless c is the child's code; a leaf: it stops; with
// several children: its goto row decides.
__device__ __forceinline__ bool hk_outcome(const FilterParams &p, const uint4 e, uint32_t i, uint32_t c, bool c_ok,
                                           int &r, uint32_t &s, uint32_t &q) {
    if (e.y == 0u) {
        r = -1;
        return true;
    }
    if (e.z == kHkBranch) {
        s = e.y;
        q = i + p.k;
        return false;
    }
    r = static_cast<int>(e.w & 0xFFFFFFu) - 1;
    if (e.z == 0u || !c_ok || c != (e.w >> 24)) return true;
    s = e.z;
    q = i + p.k + 1;
    return false;
}

// The window-table entry of window x (codes from the first position on), 2-
// and 4-bit codes: the depth-k state, or the encoded result where the walk
// stops inside the window.
template <int B>
__device__ __forceinline__ int window_entry(const FilterParams &p, uint32_t x) {
    return __ldg(p.JK + (x & ((1u << (B * p.k)) - 1u)));
}

// One flag per non-zero byte of x (bit i for byte i).
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t x) {
    const uint32_t t = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;  // bit 7 of each byte: that byte != 0
    return ((t & 0x80808080u) * 0x00204081u) >> 28;
}


// Flags (bit b) of the 16 positions g0 + b outside the text [0, n).
__device__ __forceinline__ uint32_t outside_marks(int64_t g0, int64_t n) {
    uint32_t iv = 0;
    if (!(g0 >= 0 && g0 + 16 <= n)) {
#pragma unroll
        for (int b = 0; b < 16; ++b)
            if (g0 + b < 0 || g0 + b >= n) iv |= 1u << b;
    }
    return iv;
}

// A warp: the staged bytes st[q] at text positions gpb + q outside the text
// [0, n) become `fill`.  Out of line (fringe tiles only): inlined, it cost
// the kernel it sits in registers on every tile.
static __device__ __noinline__ void fill_outside(uint8_t *st, int64_t gpb, int64_t n, uint32_t staged, uint32_t fill,
                                                 int lane) {
    for (uint32_t q = static_cast<uint32_t>(lane); q < staged; q += 32u) {
        const int64_t g = gpb + static_cast<int64_t>(q);
        if (g < 0 || g >= n) st[q] = static_cast<uint8_t>(fill);
    }
}

// Flags (bit b) of the 16 bytes of raw in no keyword (class table entry
// 0xFF).  Out of line: the kernels that call it do so rarely.
static __device__ __noinline__ uint32_t unknown_flags16(const uint8_t *cls8, const uint4 raw) {
    const uint32_t v[4] = {raw.x, raw.y, raw.z, raw.w};
    uint32_t iv = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j)
        if (cls8[(v[j >> 2] >> (8 * (j & 3))) & 0xFFu] == 0xFFu) iv |= 1u << j;
    return iv;
}

// Pack the low B bits of the 4 byte codes of `codes` (4 B bits, first byte lowest).
template <int B>
__device__ __forceinline__ uint32_t pack4(uint32_t codes) {
    if (B == 2) return ((codes & 0x03030303u) * 0x01041040u) >> 24;
    uint32_t x = codes & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    return (x | (x >> 8)) & 0xFFFFu;
}

// Codes of positions i.. (16 for B = 2, 8 for B = 4, 4 for B = 8) from the
// packed stream.
template <int B>
__device__ __forceinline__ uint32_t code_window(const uint32_t *packed, uint32_t i) {
    const uint32_t bo = B * i, w = bo >> 5;
    return __funnelshift_r(packed[w], packed[w + 1], bo & 31u);
}

// The "cannot extend a walk" flags of tile positions j, j + 1, ... (bit 0
// for j; at least 17 of them): two 16-bit entries joined, then shifted.
__device__ __forceinline__ uint32_t inv_flags(const WarpSmem &w, uint32_t j) {
    return (static_cast<uint32_t>(w.inv[j >> 4]) | (static_cast<uint32_t>(w.inv[(j >> 4) + 1]) << 16)) >> (j & 15u);
}

// Code of tile position q; false when q cannot extend a walk.  Positions below
// `coded` have their codes in the packed stream already; later ones are read
// from the text in global memory (the stage may already hold the next tile).
// identity: 256 columns, the code is the byte (the byte table's 0xFF would
// read as "in no keyword").
template <int B>
__device__ __forceinline__ bool fetch_code(const TileText &tt, const WarpSmem &w, int64_t gpb, uint32_t coded,
                                           uint32_t q, uint32_t &c, bool identity) {
    if (q < coded) {
        if ((w.inv[q >> 4] >> (q & 15u)) & 1u) return false;
        c = (w.packed[(B * q) >> 5] >> ((B * q) & 31u)) & ((1u << B) - 1u);
        return true;
    }
    const int64_t gp = gpb + static_cast<int64_t>(q);
    if (gp >= static_cast<int64_t>(tt.n)) return false;
    const uint32_t b = __ldg(tt.text + gp);
    if (B == 8 && identity) {
        c = b;
        return true;
    }
    const uint32_t v = w.cls8[b];
    if (v == 0xFFu) return false;
    c = v;
    return true;
}

// A walk at state s (>= p.s_chain) whose next byte is at tile index q: its
// chain record decides.  Returns 1 when the state's whole run of forced
// transitions matched the text (s and q moved to the run's end), 0 when the
// walk stops in the run or at a leaf (result in r), 2 when s branches (take its
// goto row).  The text bytes come from global memory (L1/L2: the tile was
// just read).
__device__ __forceinline__ int chain_step(const FilterParams &p, const TileText &tt, int64_t gpb, uint32_t &s,
                                          uint32_t &q, int &r) {
    const uint4 rc = __ldg(p.skip + (s - p.s_chain));
    if (rc.x == kSkipBranch) return 2;
    const int64_t gq = gpb + static_cast<int64_t>(q);
    const bool ok = rc.x > 0 && gq + static_cast<int64_t>(rc.x) <= static_cast<int64_t>(tt.n) &&
                    run_equal(tt.text + gq, p.chain + rc.y, rc.x);
    if (ok) {
        s = rc.z;
        q += rc.x;
        return 1;
    }
    r = static_cast<int>(rc.w);
    return 0;
}

// The walk from state s at tile position q, text bytes from global memory;
// out of line, for the few walks of 8-bit codes that the state hash leaves
// open (a copy per call site would crowd the instruction cache).
// (The structures go by value: a reference to the caller's would keep them in
// local memory for the caller's whole run.)
template <typename GT>
__device__ __noinline__ int walk_far(const FilterParams &p, const uint8_t *cls8, const TileText tt, int64_t gpb,
                                     uint32_t s, uint32_t q);

// Finish up to SLOTS * 32 queued survivors (queue[base .. base + avail)) of a
// tile whose dense ids were set to -1 first: the ids found go to the dense
// output (MODE == OUT_DENSE; with FALLBACK to the unit's dense fallback
// instead), are counted, or go to the unit's slots (dense_all: every result
// also to the unit's dense fallback, set to -1 first).  Returns true when this
// lane found a keyword.
template <int B, typename GT, int MODE, int SLOTS, bool DIRECT = false, bool FALLBACK = false>
__device__ __forceinline__ bool finish_survivors(const FilterParams &p, const TileText &tt, const WarpSmem &w,
                                                 int64_t gpb, bool interior, bool clean, uint32_t avail,
                                                 uint32_t pbase, int lane, unsigned long long &cnt, uint32_t base,
                                                 uint32_t coded = 0, uint32_t su = 0, bool dense_all = false) {
    const int64_t n = static_cast<int64_t>(tt.n);
    const uint32_t k = p.k, k2 = p.k2;
    const GT *G = static_cast<const GT *>(p.G);
    uint32_t st[SLOTS], q[SLOTS], ii[SLOTS];
    int v[SLOTS];
    uint32_t act = 0, pend = 0, walking = 0;
    uint32_t x[SLOTS];
    uint4 he[B == 8 ? SLOTS : 1];  // 8-bit codes: each window's first state-hash entry
    // window table (8-bit codes: state hash): depth-k state or result; all
    // loads first
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        const uint32_t qi = lane + 32u * t;
        v[t] = INT_MIN;
        st[t] = 0;
        q[t] = 0;
        ii[t] = 0;
        x[t] = 0;
        if (qi < avail) {
            act |= 1u << t;
            const uint32_t e16 = w.queue[base + qi];
            const uint32_t i = e16 & 0x7FFFu;
            ii[t] = i;
            q[t] = i;
            if (!(e16 >> 15)) {
                x[t] = code_window<B>(w.packed, i);
                if constexpr (B == 8) {
                    x[t] &= p.wmask;
                    he[t] = __ldg(p.HK + hk_slot(p, x[t]));
                } else {
                    v[t] = __ldg(p.JK + (x[t] & ((1u << (B * k)) - 1u)));
                }
                pend |= 1u << t;
            }
        }
    }
    if constexpr (B == 8) {
        // the entry settles most survivors; the others walk on from the state
        // or its child (no stride table)
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            if ((pend >> t) & 1u) {
                const uint4 f = hk_find(p, x[t], he[t]);
                const uint32_t j = ii[t] + k;  // the character after the window (j < kCodeSpan)
                const bool c_ok = !((w.inv[j >> 4] >> (j & 15u)) & 1u);
                const uint32_t c = (w.packed[j >> 2] >> (8u * (j & 3u))) & 0xFFu;
                int r = -1;
                if (!hk_outcome(p, f, ii[t], c, c_ok, r, st[t], q[t])) {
                    v[t] = INT_MIN;  // walking
                } else {
                    v[t] = r;
                }
            }
        }
        pend = 0;
    }
    // stride table for the walks still alive at depth k
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        if ((pend >> t) & 1u) {
            const int e = v[t];
            if (e < 0) {
                v[t] = decode_dead(e);
                pend &= ~(1u << t);
            } else {
                st[t] = static_cast<uint32_t>(e);
                q[t] = ii[t] + k;
                v[t] = INT_MIN;
                bool ok2 = k2 > 0 && (interior || gpb + static_cast<int64_t>(ii[t] + k + k2) <= n);
                if (ok2 && !clean) {
                    const uint32_t j = ii[t] + k;
                    const uint32_t wi = inv_flags(w, j);
                    ok2 = (wi & ((1u << k2) - 1u)) == 0;
                }
                if (ok2) {
                    const uint32_t w2 = (x[t] >> (B * k)) & ((1u << (B * k2)) - 1u);
                    v[t] = __ldg(p.J2 + ((static_cast<uint64_t>(st[t] - p.base_k) << (B * k2)) | w2));
                } else {
                    pend &= ~(1u << t);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        if ((act >> t) & 1u) {
            if ((pend >> t) & 1u) {
                if (v[t] < 0) {
                    v[t] = decode_dead(v[t]);
                } else {
                    st[t] = static_cast<uint32_t>(v[t]);
                    q[t] += k2;
                    v[t] = INT_MIN;
                    walking |= 1u << t;
                }
            } else if (v[t] == INT_MIN) {
                walking |= 1u << t;
            }
        }
    }
    // the goto table, one character at a time
    for (uint32_t step = 0; walking; ++step) {
        if (step > p.maxlen + 1) {  // impossible for a well-formed table
            atomicOr(p.err, static_cast<unsigned>(kErrWalk));
#pragma unroll
            for (int t = 0; t < SLOTS; ++t)
                if ((walking >> t) & 1u) v[t] = -1;
            break;
        }
        int e[SLOTS];
        uint32_t loaded = 0;
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            if ((walking >> t) & 1u) {
                if (st[t] >= p.s_chain) {  // a run of forced transitions, a leaf, or a branch
                    int rr = -1;
                    // text bytes from global memory: the tile's stage already
                    // takes the next bulk copy while its survivors are walked
                    const int k3 = chain_step(p, tt, gpb, st[t], q[t], rr);
                    if (k3 == 1) continue;
                    if (k3 == 0) {
                        v[t] = rr;
                        walking &= ~(1u << t);
                        continue;
                    }
                }
                uint32_t c = 0;
                const bool okc =
                    fetch_code<B>(tt, w, gpb, DIRECT ? coded : pbase + kPass + 16u, q[t], c, p.identity != 0);
                // an unknown byte or the text end reads the row's end column,
                // which always holds the result of stopping there
                e[t] = goto_ld(G, st[t], p.W, okc ? c : p.C);
                loaded |= 1u << t;
            }
        }
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            if ((loaded >> t) & 1u) {
                if (e[t] < 0) {
                    v[t] = decode_dead(e[t]);
                    walking &= ~(1u << t);
                } else {
                    st[t] = static_cast<uint32_t>(e[t]);
                    q[t] += 1;
                }
            }
        }
    }
    bool found = false;
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
        const bool mine = (act >> t) & 1u;
        if (MODE == OUT_SLOTS) {
            // one atomic per warp and slot index, ranks by ballot (all lanes)
            const bool hit = mine && v[t] >= 0;
            const unsigned m = __ballot_sync(kFull, hit);
            if (hit && dense_all) p.sl.dense[static_cast<uint64_t>(su) * kDenseStride + ii[t]] = v[t];
            if (m) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(p.sl.counts + su, static_cast<uint32_t>(__popc(m)));
                base = __shfl_sync(kFull, base, 0) + __popc(m & ((1u << lane) - 1u));
                if (hit && base < kSlotCap)
                    p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + base] =
                        (static_cast<unsigned long long>(static_cast<uint32_t>(v[t])) << 32) |
                        static_cast<uint32_t>(gpb + ii[t]);
            }
            found |= hit;
            continue;
        }
        if (mine) {
            found |= v[t] >= 0;
            if (MODE == OUT_COUNT)
                cnt += v[t] >= 0 ? 1ull : 0ull;
            else if (v[t] >= 0 && FALLBACK)
                p.sl.dense[static_cast<uint64_t>(su) * kDenseStride + ii[t]] = v[t];
            else if (v[t] >= 0)  // the -1 of every other position is written already
                tt.out[gpb + ii[t]] = v[t];
        }
    }
    return found;
}

// One warp, a tile whose matches overflowed its slots: the survivors walked
// again, 64 at a time (rare, so with few registers), the ids found written to
// the unit's dense fallback (set to -1 by the caller).  The structures go by
// value (references would keep the caller's in local memory).
template <int B, typename GT>
__device__ __noinline__ void refill_fallback(const FilterParams &p, const TileText tt, const WarpSmem w,
                                                int64_t gpb, bool interior, bool clean, uint32_t total, int lane,
                                                uint32_t su) {
    unsigned long long none = 0;
    for (uint32_t c = 0; 64u * c < total; ++c) {
        finish_survivors<B, GT, OUT_DENSE, 2, true, true>(p, tt, w, gpb, interior, clean, total - 64u * c, 0, lane,
                                                          none, 64u * c, kCodeSpan, su);
        __syncwarp();
    }
}

// One warp: claim a chunk of the tile offered in slot hs.  True (with the
// chunk) when the claim names the slot's current publication and a chunk it
// has; any other claim is void and changes nothing.
__device__ __forceinline__ bool claim_chunk(HelpSlot *hs, int lane, uint32_t &chunk) {
    uint32_t ok = 0, c = 0;
    // a plain look first: no atomic on a slot with nothing left to claim
    bool open = false;
    if (lane == 0) {
        const unsigned long long t = *reinterpret_cast<volatile unsigned long long *>(&hs->ticket);
        const uint32_t pub = *reinterpret_cast<volatile uint32_t *>(&hs->pub);
        const uint32_t nch = *reinterpret_cast<volatile uint32_t *>(&hs->nchunks);
        open = static_cast<uint32_t>(t >> 32) != 0u && static_cast<uint32_t>(t >> 32) == pub &&
               static_cast<uint32_t>(t) < nch;
    }
    if (lane == 0 && open) {
        const unsigned long long t = atomicAdd(&hs->ticket, 1ull);
        __threadfence_block();
        const uint32_t gen = static_cast<uint32_t>(t >> 32);
        c = static_cast<uint32_t>(t);
        const uint32_t pub = *reinterpret_cast<volatile uint32_t *>(&hs->pub);
        const uint32_t nch = *reinterpret_cast<volatile uint32_t *>(&hs->nchunks);
        ok = (gen != 0u && gen == pub && c < nch) ? 1u : 0u;
    }
    chunk = __shfl_sync(kFull, c, 0);
    return __shfl_sync(kFull, ok, 0) != 0u;
}

// One warp: finish chunk c of the tile offered by warp s (its queue and codes
// stay in place until every chunk is done), then report it done.
template <int B, typename GT, int MODE>
__device__ __forceinline__ void help_chunk(const FilterParams &p, const Work &wk, uint8_t *smem, HelpSlot *hs,
                                           uint32_t s, uint32_t c, int lane, unsigned long long &cnt) {
    uint32_t tile = 0, item = 0, total = 0, flags = 0, su = 0, glo = 0, ghi = 0;
    if (lane == 0) {
        tile = hs->tile;
        item = hs->item;
        total = hs->total;
        flags = hs->flags;
        su = hs->su;
        const unsigned long long g = static_cast<unsigned long long>(hs->gpb);
        glo = static_cast<uint32_t>(g);
        ghi = static_cast<uint32_t>(g >> 32);
    }
    tile = __shfl_sync(kFull, tile, 0);
    item = __shfl_sync(kFull, item, 0);
    total = __shfl_sync(kFull, total, 0);
    flags = __shfl_sync(kFull, flags, 0);
    su = __shfl_sync(kFull, su, 0);
    glo = __shfl_sync(kFull, glo, 0);
    ghi = __shfl_sync(kFull, ghi, 0);
    const int64_t gpb = static_cast<int64_t>((static_cast<uint64_t>(ghi) << 32) | glo);
    uint8_t *ws = smem + p.off_warp + static_cast<size_t>(s) * p.warp_bytes;
    WarpSmem v;
    v.cls8 = smem + kOffCls;
    v.F = reinterpret_cast<const uint32_t *>(smem + kOffF);
    v.st = ws;
    v.packed = reinterpret_cast<uint32_t *>(ws + p.off_packed);
    v.inv = reinterpret_cast<uint16_t *>(ws + p.off_inv);
    v.queue = reinterpret_cast<uint16_t *>(ws + p.off_queue);
    v.neg1 = reinterpret_cast<const int32_t *>(smem + p.off_neg1);
    const TileText tt = tile_text(p, wk, tile, item);
    constexpr uint32_t kRound = 32u * heavy_slots<B>();
    finish_survivors<B, GT, MODE, heavy_slots<B>(), true>(p, tt, v, gpb, (flags & 1u) != 0, (flags & 2u) != 0,
                                                          total - kRound * c, 0, lane, cnt, kRound * c, kCodeSpan, su,
                                                          (flags & 4u) != 0);
    __threadfence_block();
    __syncwarp();
    if (lane == 0) atomicAdd(&hs->done, 1u);
}

// ---------------------------------------------------------------------------
// Pipelined variant (dense ids and counts).  A tile's survivors (at most one
// per lane) stay in flight while the warp works on the next tiles: the window
// table load is issued when the tile is filtered, the stride table load one
// tile later, and the tile is finished and written two tiles later, so the
// two dependent L2 round trips overlap the classification and filtering of
// the next tiles.  A tile with more survivors than lanes (long walks) drains
// the pipeline and is finished at once.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoPos = 0xFFFFu;
enum : uint32_t { kPhJK = 0, kPhJ2 = 1, kPhWalk = 2, kPhDone = 3 };

struct Flight {
    int64_t gpb;      // text index of the tile's position 0
    uint32_t tile;    // work unit; 0xFFFFFFFF: empty
    uint32_t item;    // batch: its entry in the planned list
    uint32_t interior;
    uint32_t pos;     // this lane's survivor (tile position) or kNoPos
    uint32_t phase;
    uint32_t state;   // goto state of the walk
    uint32_t q;       // tile position of the walk's next character
    uint32_t w2;      // stride-table codes
    uint32_t ok2;     // the stride window is usable
    int val;          // load in flight, or the result when done
};

__device__ __forceinline__ Flight empty_flight() {
    Flight f;
    f.gpb = 0;
    f.tile = 0xFFFFFFFFu;
    f.item = 0;
    f.interior = 0;
    f.pos = kNoPos;
    f.phase = kPhDone;
    f.state = 0;
    f.q = 0;
    f.w2 = 0;
    f.ok2 = 0;
    f.val = -1;
    return f;
}

// Walk the goto table from state s, reading the text from global memory.
template <typename GT>
__device__ __forceinline__ int walk_global(const FilterParams &p, const uint8_t *cls8, const TileText &tt,
                                           int64_t gpb, uint32_t s, uint32_t q) {
    const GT *G = static_cast<const GT *>(p.G);
    for (uint32_t step = 0; step <= p.maxlen + 1; ++step) {
        if (s >= p.s_chain) {  // a run of forced transitions, a leaf, or a branch
            int rr = -1;
            const int k3 = chain_step(p, tt, gpb, s, q, rr);
            if (k3 == 1) continue;
            if (k3 == 0) return rr;
        }
        const int64_t gp = gpb + static_cast<int64_t>(q);
        uint32_t c = p.C;  // the end column: stop here
        if (gp < static_cast<int64_t>(tt.n)) {
            const uint32_t b = __ldg(tt.text + gp);
            const uint32_t v = p.identity ? b : cls8[b];  // 256 columns: the byte itself
            if (p.identity || v != 0xFFu) c = v;
        }
        const int t = goto_ld(G, s, p.W, c);
        if (t < 0) return decode_dead(t);
        s = static_cast<uint32_t>(t);
        ++q;
    }
    atomicOr(p.err, static_cast<unsigned>(kErrWalk));
    return -1;
}

template <typename GT>
__device__ __noinline__ int walk_far(const FilterParams &p, const uint8_t *cls8, const TileText tt, int64_t gpb,
                                     uint32_t s, uint32_t q) {
    return walk_global<GT>(p, cls8, tt, gpb, s, q);
}

// Second stage: the window-table result has arrived; issue the stride load.
template <int B>
__device__ __forceinline__ void flight_advance(const FilterParams &p, Flight &f) {
    if (f.pos == kNoPos || f.phase != kPhJK) return;
    const int e = f.val;
    if (e < 0) {
        f.val = decode_dead(e);
        f.phase = kPhDone;
        return;
    }
    f.state = static_cast<uint32_t>(e);
    f.q = f.pos + p.k;
    if (f.ok2) {
        f.val = __ldg(p.J2 + ((static_cast<uint64_t>(f.state - p.base_k) << (B * p.k2)) | f.w2));
        f.phase = kPhJ2;
    } else {
        f.phase = kPhWalk;
    }
}

// Last stage: the stride-table result has arrived; finish the walk if needed
// (8-bit codes: out of line).
template <int B, typename GT>
__device__ __forceinline__ void flight_finish(const FilterParams &p, const Work &wk, const uint8_t *cls8, Flight &f) {
    if (f.pos == kNoPos) return;
    if (f.phase == kPhJ2) {
        const int e = f.val;
        if (e < 0) {
            f.val = decode_dead(e);
            f.phase = kPhDone;
            return;
        }
        f.state = static_cast<uint32_t>(e);
        f.q += p.k2;
        f.phase = kPhWalk;
    }
    if (f.phase == kPhWalk) {
        if constexpr (B == 8)
            f.val = walk_far<GT>(p, cls8, tile_text(p, wk, f.tile, f.item), f.gpb, f.state, f.q);
        else
            f.val = walk_global<GT>(p, cls8, tile_text(p, wk, f.tile, f.item), f.gpb, f.state, f.q);
        f.phase = kPhDone;
    }
}

// Write (or count) a finished tile: one bulk store of -1 when no survivor
// found a keyword, else -1 from the position owners and the survivors' ids.
template <int MODE>
__device__ __forceinline__ void flight_output(const FilterParams &p, const Work &wk, const WarpSmem &w, const Flight &f,
                                              int lane, unsigned long long &cnt) {
    if (f.tile == 0xFFFFFFFFu) return;
    const bool mine = f.pos != kNoPos && f.val >= 0;
    if (MODE == OUT_COUNT) {
        cnt += mine ? 1ull : 0ull;
        return;
    }
    if (MODE == OUT_SLOTS) {
        // at most one survivor per lane: rank by lane (ascending position)
        const unsigned m = __ballot_sync(kFull, mine);
        const uint32_t su = p.sl.ubase + f.tile;
        const uint32_t r = __popc(m & ((1u << lane) - 1u));
        if (mine && r < kSlotCap)
            p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + r] =
                (static_cast<unsigned long long>(static_cast<uint32_t>(f.val)) << 32) |
                static_cast<uint32_t>(f.gpb + f.pos);
        if (lane == 0 && m) p.sl.counts[su] = __popc(m);  // the unit's only writer
        return;
    }
    const bool found = __any_sync(kFull, mine);
    if (!found && f.interior && !wk.list && p.vec_ok) {  // one text: no lookup of its output
        if (lane == 0) {
            bulk_store(p.out + f.gpb, w.neg1, kTile * 4);
            bulk_commit();
            bulk_wait_read_keep8();  // bound the groups in flight
        }
        return;
    }
    const TileText tt = tile_text(p, wk, f.tile, f.item);
    const int64_t n = static_cast<int64_t>(tt.n);
    if (!found && f.interior && tt.vec_ok) {
        if (lane == 0) {
            bulk_store(tt.out + f.gpb, w.neg1, kTile * 4);
            bulk_commit();
            bulk_wait_read_keep8();  // bound the groups in flight
        }
        return;
    }
    if (lane < static_cast<int>(kOwnLanes)) {
        const int4 none = make_int4(-1, -1, -1, -1);
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
#pragma unroll
            for (uint32_t g = 0; g < 4; ++g) {
                const int64_t g0 = f.gpb + h * kPass + 16u * lane + 4u * g;
                if (tt.vec_ok && g0 >= 0 && g0 + 4 <= n) {
                    *reinterpret_cast<int4 *>(tt.out + g0) = none;
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (g0 + r >= 0 && g0 + r < n) tt.out[g0 + r] = -1;
                }
            }
        }
    }
    __syncwarp();  // the -1 stores of the owners come before the survivors' ids
    if (mine) tt.out[f.gpb + f.pos] = f.val;
}

// The CTA's start: the constant -1 buffer, the help slots and CTA counters,
// and the mbarriers (p: the launch's shared-memory layout).  Ends with a
// CTA barrier.
__device__ __forceinline__ void filter_setup(const FilterParams &p, uint8_t *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint8_t *wreg = smem + p.off_warp + static_cast<size_t>(warp) * p.warp_bytes;
    HelpSlot *my_help = reinterpret_cast<HelpSlot *>(wreg + p.off_help);
    for (uint32_t i = threadIdx.x; i < kTile; i += blockDim.x) reinterpret_cast<int32_t *>(smem + p.off_neg1)[i] = -1;
    fence_proxy_async_smem();  // the constant buffer is read by bulk stores
    if (lane == 0) {
        my_help->ticket = 0;
        my_help->pub = 0;
        my_help->nchunks = 0;
        my_help->done = 0;
    }
    if (threadIdx.x == 0) {
        *reinterpret_cast<uint32_t *>(smem + kOffRetired) = 0;
        *reinterpret_cast<uint32_t *>(smem + kOffOffers) = 0;
        mbar_init(reinterpret_cast<uint64_t *>(smem + kOffJBar), 1);
        uint64_t *all = reinterpret_cast<uint64_t *>(smem + kOffStageBar);
        for (int i = 0; i < nw * kMaxStages; ++i) mbar_init(&all[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// One thread: fetch an automaton's byte table and root filter into shared
// memory, completing on the table mbarrier.  The CTA must be done reading
// the previous ones (a CTA barrier before).
__device__ __forceinline__ void filter_load_tables(const FilterParams &p, uint8_t *smem) {
    uint64_t *jbar = reinterpret_cast<uint64_t *>(smem + kOffJBar);
    fence_proxy_async_smem();  // earlier generic reads of these bytes before the async writes
    mbar_arrive_expect_tx(jbar, 256u + p.fbytes);
    bulk_load(smem + kOffCls, p.cls8g, 256u, jbar);
    bulk_load(smem + kOffF, p.Fg, p.fbytes, jbar);
}

// One warp: every work unit of the launch's automaton that this warp takes,
// through the pipeline below.  Stage barriers are used in a running order:
// iteration it uses stage it % nstages with phase parity (it / nstages) & 1;
// the warp starts at iteration it0 and returns in *it_next where the next
// automaton's units start.  jpar: the phase parity of the table barrier that
// the automaton's tables complete.  False when a bounded wait ran out (the
// error is latched; the warp's copies in flight have landed or been waited
// for, within the limit).
// HELP: share heavy tiles within the CTA (the forms for one text that is short
// next to the grid; see the heavy path below).  LISTED: the first phase of the
// phased form (p.list set; the forms without it carry none of its code).
template <int B, typename GT, int MODE, bool BATCH, bool HELP, bool LISTED = false, bool DIRECT = false>
__device__ __forceinline__ bool filter_units(const FilterParams &p, uint8_t *smem, uint32_t it0, uint32_t jpar,
                                             unsigned long long &cnt, uint32_t *it_next) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t *jbar = reinterpret_cast<uint64_t *>(smem + kOffJBar);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffStageBar) + warp * kMaxStages;
    uint32_t *stile = reinterpret_cast<uint32_t *>(smem + kOffStageTile) + warp * kMaxStages;
    uint8_t *wreg = smem + p.off_warp + static_cast<size_t>(warp) * p.warp_bytes;
    WarpSmem w;
    w.cls8 = smem + kOffCls;
    w.F = reinterpret_cast<const uint32_t *>(smem + kOffF);
    w.st = wreg;
    w.packed = reinterpret_cast<uint32_t *>(wreg + p.off_packed);
    w.inv = reinterpret_cast<uint16_t *>(wreg + p.off_inv);
    w.queue = reinterpret_cast<uint16_t *>(wreg + p.off_queue);
    w.neg1 = reinterpret_cast<const int32_t *>(smem + p.off_neg1);
    uint32_t *sitem = reinterpret_cast<uint32_t *>(wreg + p.off_meta);
    HelpSlot *my_help = reinterpret_cast<HelpSlot *>(wreg + p.off_help);
    uint32_t *retired = reinterpret_cast<uint32_t *>(smem + kOffRetired);
    uint32_t *offers = reinterpret_cast<uint32_t *>(smem + kOffOffers);
    const uint32_t nst = p.nstages;
    // one text: a null list the compiler sees, so the batch lookups fold away
    const Work wk = BATCH ? load_work(p.batch, p.lists, p.ntiles) : load_work(nullptr, nullptr, p.ntiles);
    const uint32_t k = p.k, k2 = p.k2;
    const bool owner = lane < static_cast<int>(kOwnLanes);

    // Tiles: the first one per warp statically, the rest claimed from a global
    // counter so that a warp held up by an expensive tile stops taking work.
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nw;
    UnitClaims claims = claims_start(gw, GW);
    auto next_tile = [&](uint32_t) -> uint32_t {
        uint32_t t = 0xFFFFFFFFu;
        if (lane == 0) {
            const uint64_t c = claims_next(claims, p.counter, wk.units);
            if (c < wk.units) t = static_cast<uint32_t>(c);
        }
        return __shfl_sync(kFull, t, 0);
    };
    for (uint32_t j = it0; j < it0 + nst; ++j) {
        const uint32_t s = j % nst;
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], wreg + s * p.staged, next_tile(j), lane);
    }

    Flight f1 = empty_flight(), f2 = empty_flight();  // one and two tiles back
    // phased form: the part [lnext, lend) of the survivor list this warp
    // reserved and has not filled yet (lfull: no more room)
    uint32_t lnext = 0, lend = 0;
    bool lfull = false;
    bool ok = mbar_wait(jbar, jpar, p.wait_ns);
    // stage s of iteration it is it % nst, its phase parity (it / nst) & 1
    uint32_t it = it0;
    for (uint32_t s = it0 % nst, par = (it0 / nst) & 1u;; ++it, s = s + 1 == nst ? 0u : s + 1, par ^= s == 0 ? 1u : 0u) {
        ok = ok && mbar_wait(&bars[s], par, p.wait_ns);
        if (!__all_sync(kFull, ok)) {
            // A copy never completed: latch the error, let this warp's copies in
            // flight finish (bounded), and leave.
            if (lane == 0) {
                bulk_wait_all();
                atomicOr(p.err, static_cast<unsigned>(kErrTimeout));
                atomicAdd(retired, 1u);
                mbar_wait(jbar, jpar, p.wait_ns);
                for (uint32_t j = it; j < it + nst; ++j) mbar_wait(&bars[j % nst], (j / nst) & 1u, p.wait_ns);
            }
            return false;
        }
        const uint32_t tile = stile[s];
        if (tile >= wk.units) break;
        const uint32_t item = sitem[s];
        const TileText tt = tile_text(p, wk, tile, item);
        const int64_t n = static_cast<int64_t>(tt.n);
        uint8_t *st = wreg + s * p.staged;
        const uint64_t tlo = static_cast<uint64_t>(tt.tile) * kTile;
        const int64_t gpb = static_cast<int64_t>(tlo) - tt.head;
        const bool interior = gpb >= 0 && gpb + static_cast<int64_t>(p.staged) <= n;
        if (!interior) {
            load_text_fringe(tt, p.staged, st, tlo, lane);
            if constexpr (B == 2 && DIRECT) {
                // the staged bytes outside the text become a byte in no
                // keyword, so the classification flags them as it does those
                __syncwarp();
                fill_outside(st, gpb, n, p.staged, p.dfill, lane);
            }
            __syncwarp();
        }

        // 1. classify the tile's bytes (both halves), once per byte
        uint32_t plo[2], phi[2], inv[2];
        uint32_t p8[2][4];  // 8-bit codes: the lane's 16 codes of each half
        if constexpr (B == 2 && DIRECT) {
            // Class codes (byte >> 1) & 3: masked in place, one multiply
            // gathers a word's four codes into its top byte (code j, at bit
            // 8j + 1, times 2^(23 - 6j) lands at bit 24 + 2j; the other
            // products land below bit 24 without carrying into it), and
            // byte permutes join the four top bytes.  A byte is a keyword
            // byte exactly when the keyword byte of its code equals it: a
            // byte permute selected by 2 x code (the masked word with the
            // next byte's bits moved to the high nibble, bytes 0 and 2
            // joined) picks it from p.dsel_lo/hi.  Only a word pair that
            // differs somewhere has its bytes flagged one by one (through
            // the class table); positions outside the text hold p.dfill,
            // a byte in no keyword.
            constexpr uint32_t dmask = 0x06060606u, dmul = 0x01041040u >> 1;
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const uint32_t i0 = h * kPass + 16u * static_cast<uint32_t>(lane);
                const uint4 raw = *reinterpret_cast<const uint4 *>(st + i0);
                const uint32_t x0 = raw.x & dmask, x1 = raw.y & dmask, x2 = raw.z & dmask, x3 = raw.w & dmask;
                plo[h] = __byte_perm(__byte_perm(x0 * dmul, x1 * dmul, 0x0073u),
                                     __byte_perm(x2 * dmul, x3 * dmul, 0x0073u), 0x5410u);
                phi[h] = 0;
                const uint32_t any =
                    (raw.x ^ __byte_perm(p.dsel_lo, p.dsel_hi, __byte_perm(x0 | (x0 >> 4), 0u, 0x4420u))) |
                    (raw.y ^ __byte_perm(p.dsel_lo, p.dsel_hi, __byte_perm(x1 | (x1 >> 4), 0u, 0x4420u))) |
                    (raw.z ^ __byte_perm(p.dsel_lo, p.dsel_hi, __byte_perm(x2 | (x2 >> 4), 0u, 0x4420u))) |
                    (raw.w ^ __byte_perm(p.dsel_lo, p.dsel_hi, __byte_perm(x3 | (x3 >> 4), 0u, 0x4420u)));
                uint32_t iv = 0;
                if (any) iv = unknown_flags16(w.cls8, raw);
                inv[h] = iv;
                w.packed[i0 >> 4] = plo[h];
                w.inv[i0 >> 4] = static_cast<uint16_t>(iv);
            }
        } else {
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const uint32_t i0 = h * kPass + 16u * static_cast<uint32_t>(lane);
                const uint4 raw = *reinterpret_cast<const uint4 *>(st + i0);
                uint32_t c0, c1, c2, c3, u0, u1, u2, u3;
                if constexpr (B == 8) {
                    classify_word8(p, w.cls8, raw.x, c0, u0);
                    classify_word8(p, w.cls8, raw.y, c1, u1);
                    classify_word8(p, w.cls8, raw.z, c2, u2);
                    classify_word8(p, w.cls8, raw.w, c3, u3);
                } else {
                    classify_word(p, w.cls8, raw.x, c0, u0);
                    classify_word(p, w.cls8, raw.y, c1, u1);
                    classify_word(p, w.cls8, raw.z, c2, u2);
                    classify_word(p, w.cls8, raw.w, c3, u3);
                }
                uint32_t iv = 0;
                if (u0 | u1 | u2 | u3)
                    iv = nonzero_bytes(u0) | (nonzero_bytes(u1) << 4) | (nonzero_bytes(u2) << 8) |
                         (nonzero_bytes(u3) << 12);
                if (!interior) iv |= outside_marks(gpb + i0, n);
                inv[h] = iv;
                if constexpr (B == 2) {
                    plo[h] = pack4<2>(c0) | (pack4<2>(c1) << 8) | (pack4<2>(c2) << 16) | (pack4<2>(c3) << 24);
                    phi[h] = 0;
                    w.packed[i0 >> 4] = plo[h];
                } else if constexpr (B == 4) {
                    plo[h] = pack4<4>(c0) | (pack4<4>(c1) << 16);
                    phi[h] = pack4<4>(c2) | (pack4<4>(c3) << 16);
                    w.packed[i0 >> 3] = plo[h];
                    w.packed[(i0 >> 3) + 1] = phi[h];
                } else {
                    p8[h][0] = c0;
                    p8[h][1] = c1;
                    p8[h][2] = c2;
                    p8[h][3] = c3;
                    plo[h] = c0;
                    phi[h] = 0;
                    *reinterpret_cast<uint4 *>(w.packed + (i0 >> 2)) = make_uint4(c0, c1, c2, c3);
                }
                w.inv[i0 >> 4] = static_cast<uint16_t>(iv);
            }
        }
        const bool clean = !__any_sync(kFull, (inv[0] | inv[1]) != 0);
        __syncwarp();
        // the stage is consumed: start fetching a later tile into it
        if (lane == 0) fence_proxy_async_smem();
        issue_unit(p, wk, &bars[s], &stile[s], &sitem[s], st, next_tile(it + nst), lane);

        // 2. root filter, one bit per start position (bits 0-15: first half)
        uint32_t sv = 0, slowm = 0;
        uint32_t nlo[2];  // the next lane's first codes (lane 31 supplies the look-ahead)
        nlo[0] = __shfl_down_sync(kFull, plo[0], 1);
        nlo[1] = __shfl_down_sync(kFull, plo[1], 1);
        if (owner) {
            // The bit of window value v is bit 31 - (v & 31) of filter word
            // v >> 5: rotating the word left by v's low five bits brings it to
            // bit 31, and a funnel shift appends it to an accumulator (first
            // position ends highest, hence the bit reversal).  Four
            // accumulators of 8 positions each keep the appends out of one
            // 32-long dependency chain.
            const uint8_t *fb = reinterpret_cast<const uint8_t *>(w.F);
            uint32_t acc4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    uint32_t win;
                    if constexpr (B == 2) {
                        win = __funnelshift_r(plo[h], nlo[h], 2 * r);
                    } else if constexpr (B == 4) {
                        win = r < 8 ? __funnelshift_r(plo[h], phi[h], 4 * r)
                                    : __funnelshift_r(phi[h], nlo[h], 4 * (r - 8));
                    } else {
                        // 8-bit codes: the filter bit's index is a hash of the window
                        const uint32_t lo = p8[h][r >> 2], hi = (r >> 2) < 3 ? p8[h][(r >> 2) + 1] : nlo[h];
                        win = ((__funnelshift_r(lo, hi, 8 * (r & 3)) & p.wmask) * kFilterHashMul) >> p.fshift;
                    }
                    const uint32_t word = *reinterpret_cast<const uint32_t *>(fb + ((win >> 3) & p.famask));
                    uint32_t &acc = acc4[2 * h + (r >> 3)];
                    acc = __funnelshift_l(__funnelshift_l(word, word, win), acc, 1);
                }
            }
            // positions 0-7, 8-15, 16-23, 24-31 from the highest byte down
            sv = __brev((acc4[0] << 24) | (acc4[1] << 16) | (acc4[2] << 8) | acc4[3]);
        }
        if (!interior || !clean) {
            const uint32_t kbits = (1u << k) - 1u;
            uint32_t valid = 0;
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const uint32_t ninv = __shfl_down_sync(kFull, inv[h], 1);
                const uint32_t iw = inv[h] | (ninv << 16);
                const uint32_t i0 = h * kPass + 16u * static_cast<uint32_t>(lane);
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int64_t gp = gpb + i0 + r;
                    if (owner && gp >= 0 && gp < n) {
                        valid |= 1u << (16 * h + r);
                        // a window past the text end; with small alphabets also one
                        // holding a byte in no keyword (a shorter keyword may end
                        // before it; with 8-bit codes such a window has no state
                        // in the hash, and no keyword ends before depth k)
                        if (gp + static_cast<int64_t>(k) > n || (B != 8 && ((iw >> r) & kbits)))
                            slowm |= 1u << (16 * h + r);
                    }
                }
            }
            sv = (sv | slowm) & valid;
        }

        // 3. survivors into the warp's queue in ascending position
        const uint32_t c = __popc(sv & 0xFFFFu) | (__popc(sv >> 16) << 16);
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += y;
        }
        const uint32_t tot2 = __shfl_sync(kFull, inc, 31);
        uint32_t total = (tot2 & 0xFFFFu) + (tot2 >> 16);
        {
            const uint32_t excl = inc - c;
            uint32_t o0 = excl & 0xFFFFu, o1 = (tot2 & 0xFFFFu) + (excl >> 16);
            uint32_t m = sv;
            while (m) {
                const uint32_t b = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t h = b >> 4;
                const uint32_t i = h * kPass + 16u * static_cast<uint32_t>(lane) + (b & 15u);
                const uint16_t e = static_cast<uint16_t>(i | (((slowm >> b) & 1u) << 15));
                if (h == 0)
                    w.queue[o0++] = e;
                else
                    w.queue[o1++] = e;
            }
        }
        __syncwarp();

        bool listed = false;
        if constexpr (LISTED) {
            // phased form: the tile's survivors go to the list (their windows
            // with them; consecutive lanes write consecutive entries) and the
            // tile counts as one without survivors here.  With 8-bit codes a
            // window past the text end keeps them here; with 2- and 4-bit codes
            // any tile but an interior one of keyword bytes only (whose windows
            // and stride windows are all known); and so do no room and, in a
            // batch, unit numbers past 22 bits.  (Each lane writing its own
            // survivors' entries straight from its filter bits, without the
            // queue, measured slower: the stores no longer coalesce.)
            const bool listable = (B == 8 ? !__any_sync(kFull, (slowm & sv) != 0u) : interior && clean) &&
                                  (!BATCH || wk.units < (1u << 22));
            if (p.list && !lfull && total > 0 && listable) {
                if (lend - lnext < total) {
                    // a new chunk of list space (the rest of the old one: empty)
                    for (uint32_t j = lnext + static_cast<uint32_t>(lane); j < lend; j += 32u)
                        p.list[j] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
                    const uint32_t want = total > kListChunk ? total : kListChunk;
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(p.list_count, want);
                    base = __shfl_sync(kFull, base, 0);
                    lnext = base;
                    lend = base + want;
                    if (static_cast<uint64_t>(base) + want > p.list_cap) {
                        // no room: what was reserved below the capacity is empty
                        for (uint32_t j = base + static_cast<uint32_t>(lane); j < p.list_cap && j < lend; j += 32u)
                            p.list[j] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
                        lnext = lend = 0;
                        lfull = true;
                    }
                }
                if (!lfull) {
                    for (uint32_t j = static_cast<uint32_t>(lane); j < total; j += 32u) {
                        const uint32_t i = w.queue[j] & 0x7FFFu;
                        if constexpr (B == 8) {
                            // the code after the window (0x100: the text ends, or a
                            // byte in no keyword); i + k < kCodeSpan
                            const uint32_t ja = i + k;
                            const uint32_t ca = ((w.inv[ja >> 4] >> (ja & 15u)) & 1u)
                                                    ? 0x100u
                                                    : (w.packed[ja >> 2] >> (8u * (ja & 3u))) & 0xFFu;
                            p.list[lnext + j] = make_uint4((tile << 10) | i, code_window<8>(w.packed, i) & p.wmask,
                                                           ca | (BATCH ? p.aidx << 16 : 0u), BATCH ? item : 0u);
                        } else {
                            // the window's and the stride window's codes (i + k + k2 < kCodeSpan)
                            p.list[lnext + j] = make_uint4((tile << 10) | i, code_window<B>(w.packed, i),
                                                           BATCH ? p.aidx << 16 : 0u, BATCH ? item : 0u);
                        }
                    }
                    lnext += total;
                    total = 0;
                    listed = true;
                }
            }
        }
        if (LISTED && listed && f1.tile == 0xFFFFFFFFu && f2.tile == 0xFFFFFFFFu) {
            // a listed tile and none in flight: write (or count) it now
            Flight fo = empty_flight();
            fo.tile = tile;
            fo.item = item;
            fo.gpb = gpb;
            fo.interior = interior ? 1u : 0u;
            flight_output<MODE>(p, wk, w, fo, lane, cnt);
            continue;
        }

        if (total > 32) {
            // 4a. many survivors: finish the tiles in flight, then this one
            flight_advance<B>(p, f1);
            flight_finish<B, GT>(p, wk, w.cls8, f2);
            flight_output<MODE>(p, wk, w, f2, lane, cnt);
            flight_finish<B, GT>(p, wk, w.cls8, f1);
            flight_output<MODE>(p, wk, w, f1, lane, cnt);
            f1 = empty_flight();
            f2 = empty_flight();
            if (MODE == OUT_DENSE) {
                // -1 from the position owners first, then every survivor's id
                if (owner) {
                    const int4 none = make_int4(-1, -1, -1, -1);
#pragma unroll
                    for (uint32_t h = 0; h < 2; ++h) {
#pragma unroll
                        for (uint32_t g = 0; g < 4; ++g) {
                            const int64_t g0 = gpb + h * kPass + 16u * lane + 4u * g;
                            if (tt.vec_ok && g0 >= 0 && g0 + 4 <= n) {
                                *reinterpret_cast<int4 *>(tt.out + g0) = none;
                            } else {
#pragma unroll
                                for (int r = 0; r < 4; ++r)
                                    if (g0 + r >= 0 && g0 + r < n) tt.out[g0 + r] = -1;
                            }
                        }
                    }
                }
                __syncwarp();
            }
            // slots: a tile whose survivors are most of its positions will
            // likely hold more matches than its slots, so its dense ids are
            // kept as they are found (-1 first); the others keep them only if
            // their matches do overflow (a second pass below)
            const bool dense_all = MODE == OUT_SLOTS && p.sl.dense && total > kTile / 2;
            int32_t *const fdn =
                MODE == OUT_SLOTS && p.sl.dense ? p.sl.dense + static_cast<uint64_t>(p.sl.ubase + tile) * kDenseStride
                                                : nullptr;
            if (dense_all) {
                if (owner) {
#pragma unroll
                    for (uint32_t h = 0; h < 2; ++h)
#pragma unroll
                        for (uint32_t g = 0; g < 4; ++g)
                            *reinterpret_cast<int4 *>(fdn + h * kPass + 16u * lane + 4u * g) = make_int4(-1, -1, -1, -1);
                }
                __syncwarp();
            }
            constexpr uint32_t kRound = 32u * heavy_slots<B>();
            const uint32_t nchunks = (total + kRound - 1u) / kRound;
            // more than one round (HELP forms): offer the rounds to the CTA's
            // warps that run out of tiles (now or while this warp works), take
            // rounds too, then wait until the helpers are done with this warp's
            // queue and codes
            const bool offer = HELP && nchunks > 1;
            if (offer) {
                __threadfence_block();  // the -1 prefill before the offer
                __syncwarp();
                if (lane == 0) {
                    const uint32_t pub = my_help->pub + 1u;
                    my_help->tile = tile;
                    my_help->item = item;
                    my_help->total = total;
                    my_help->gpb = gpb;
                    my_help->flags = (interior ? 1u : 0u) | (clean ? 2u : 0u) | (dense_all ? 4u : 0u);
                    my_help->su = p.sl.ubase + tile;
                    my_help->nchunks = nchunks;
                    my_help->done = 0;
                    my_help->pub = pub;
                    __threadfence_block();
                    atomicExch(&my_help->ticket, static_cast<unsigned long long>(pub) << 32);
                    atomicAdd(offers, 1u);
                }
                __syncwarp();
            }
            for (uint32_t next = 0;;) {
                uint32_t c = next++;
                if (offer ? !claim_chunk(my_help, lane, c) : c >= nchunks) break;
                finish_survivors<B, GT, MODE, heavy_slots<B>(), true>(p, tt, w, gpb, interior, clean,
                                                                      total - kRound * c, 0, lane, cnt, kRound * c,
                                                                      kCodeSpan, p.sl.ubase + tile, dense_all);
                __syncwarp();
                if (offer && lane == 0) atomicAdd(&my_help->done, 1u);
            }
            if (offer && lane == 0) {
                const unsigned long long t0 = global_timer();
                const uint32_t need = nchunks + (p.stall_help ? 1u : 0u);
                while (*reinterpret_cast<volatile uint32_t *>(&my_help->done) < need) {
                    if (global_timer() - t0 > p.wait_ns) {
                        atomicOr(p.err, static_cast<unsigned>(kErrTimeout));
                        break;
                    }
                    __nanosleep(128);
                }
                atomicSub(offers, 1u);
            }
            __syncwarp();
            if (MODE == OUT_SLOTS && fdn && !dense_all) {
                // every round is done: when the tile's matches overflow its
                // slots after all, keep its dense ids (-1, then a second pass
                // over the survivors writing the ids found)
                uint32_t found_all = 0;
                if (lane == 0) found_all = atomicAdd(p.sl.counts + p.sl.ubase + tile, 0u);
                if (__shfl_sync(kFull, found_all, 0) > kSlotCap) {
                    if (owner) {
#pragma unroll
                        for (uint32_t h = 0; h < 2; ++h)
#pragma unroll
                            for (uint32_t g = 0; g < 4; ++g)
                                *reinterpret_cast<int4 *>(fdn + h * kPass + 16u * lane + 4u * g) =
                                    make_int4(-1, -1, -1, -1);
                    }
                    __syncwarp();
                    refill_fallback<B, GT>(p, tt, w, gpb, interior, clean, total, lane, p.sl.ubase + tile);
                }
            }
            continue;
        }

        // 4b. at most one survivor per lane: issue its window-table load now
        Flight f0 = empty_flight();
        f0.tile = tile;
        f0.item = item;
        f0.gpb = gpb;
        f0.interior = interior ? 1u : 0u;
        if (static_cast<uint32_t>(lane) < total) {
            const uint32_t e16 = w.queue[lane];
            const uint32_t i = e16 & 0x7FFFu;
            f0.pos = i;
            if (e16 >> 15) {
                f0.phase = kPhWalk;  // walk from the root
                f0.state = 0;
                f0.q = i;
            } else {
                const uint32_t x = code_window<B>(w.packed, i);
                if constexpr (B == 8) {
                    // the state hash settles the survivor, or names where its walk goes on
                    const uint32_t wx = x & p.wmask;
                    const uint4 fe = hk_find(p, wx, __ldg(p.HK + hk_slot(p, wx)));
                    const uint32_t j = i + k;
                    const bool c_ok = !((w.inv[j >> 4] >> (j & 15u)) & 1u);
                    const uint32_t c = (w.packed[j >> 2] >> (8u * (j & 3u))) & 0xFFu;
                    int r = -1;
                    uint32_t s2 = 0, q2 = 0;
                    if (hk_outcome(p, fe, i, c, c_ok, r, s2, q2)) {
                        f0.val = r;
                        f0.phase = kPhDone;
                    } else {
                        f0.state = s2;
                        f0.q = q2;
                        f0.phase = kPhWalk;
                    }
                } else {
                    f0.val = window_entry<B>(p, x);
                    f0.phase = kPhJK;
                    f0.w2 = (x >> (B * k)) & ((1u << (B * k2)) - 1u);
                    bool ok2 = k2 > 0 && (interior || gpb + static_cast<int64_t>(i + k + k2) <= n);
                    if (ok2 && !clean) {
                        const uint32_t j = i + k;
                        const uint32_t wi = inv_flags(w, j);
                        ok2 = (wi & ((1u << k2) - 1u)) == 0;
                    }
                    f0.ok2 = ok2 ? 1u : 0u;
                }
            }
        }
        // 5. the tile one back: issue its stride-table loads
        flight_advance<B>(p, f1);
        // 6. the tile two back: finish and write it
        flight_finish<B, GT>(p, wk, w.cls8, f2);
        flight_output<MODE>(p, wk, w, f2, lane, cnt);
        f2 = f1;
        f1 = f0;
    }
    // drain
    flight_advance<B>(p, f1);
    flight_finish<B, GT>(p, wk, w.cls8, f2);
    flight_output<MODE>(p, wk, w, f2, lane, cnt);
    flight_finish<B, GT>(p, wk, w.cls8, f1);
    flight_output<MODE>(p, wk, w, f1, lane, cnt);
    // phased form: the unfilled rest of this warp's list chunk is empty
    if (LISTED && p.list)
        for (uint32_t j = lnext + static_cast<uint32_t>(lane); j < lend; j += 32u)
            p.list[j] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    // the stages issued past this warp's last unit hold end marks (an arrival
    // without a copy): complete their phases, so the next automaton's units
    // start on fresh ones
    for (uint32_t j = it + 1; j < it + nst; ++j) mbar_wait(&bars[j % nst], (j / nst) & 1u, p.wait_ns);
    *it_next = it + nst;

    // no tiles left: help with the CTA's heavy tiles until every warp is done
    // with its own (no tile is offered after that, and every offer is then
    // finished: its owner waits for its chunks before going on)
    if (HELP && lane == 0) {
        __threadfence_block();
        atomicAdd(retired, 1u);
    }
    if (HELP) {
        unsigned long long t0 = 0;
        if (lane == 0) t0 = global_timer();
        for (;;) {
            bool any = false;
            uint32_t open = 0;
            if (lane == 0) open = *reinterpret_cast<volatile uint32_t *>(offers);
            open = __shfl_sync(kFull, open, 0);
            for (int s = 0; open != 0 && s < nw; ++s) {
                if (s == warp) continue;
                HelpSlot *hs = reinterpret_cast<HelpSlot *>(smem + p.off_warp + static_cast<size_t>(s) * p.warp_bytes +
                                                            p.off_help);
                uint32_t c = 0;
                while (claim_chunk(hs, lane, c)) {
                    any = true;
                    help_chunk<B, GT, MODE>(p, wk, smem, hs, static_cast<uint32_t>(s), c, lane, cnt);
                }
            }
            if (any) continue;
            uint32_t stop = 0;
            if (lane == 0) {
                if (*reinterpret_cast<volatile uint32_t *>(retired) >= static_cast<uint32_t>(nw)) {
                    stop = 1;
                } else if (global_timer() - t0 > p.wait_ns) {
                    atomicOr(p.err, static_cast<unsigned>(kErrTimeout));
                    stop = 1;
                } else {
                    __nanosleep(256);
                }
            }
            if (__shfl_sync(kFull, stop, 0)) break;
        }
    }

    return true;
}

template <int B, typename GT, int MODE, bool BATCH, bool HELP, bool LISTED, int MAXT, bool DIRECT>
__global__ void __launch_bounds__(MAXT, 1) pfac_filter_pipe(const __grid_constant__ FilterParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    filter_setup(p, smem);
    if (threadIdx.x == 0) filter_load_tables(p, smem);
    unsigned long long cnt = 0;
    uint32_t it = 0;
    if (!filter_units<B, GT, MODE, BATCH, HELP, LISTED, DIRECT>(p, smem, 0, 0, cnt, &it)) return;
    if (MODE == OUT_DENSE && lane == 0) bulk_wait_all();
    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

// The second phase of the phased form (one long text): one thread per listed
// survivor, SPT at a time so that their loads overlap, at high occupancy (48
// warps per SM with 2 at a time, 32 with 4).  8-bit codes: the survivor's
// state-hash entry settles most survivors; a walk from a depth-k state with
// several children takes its first goto step here (the code after the window
// is in the entry), which ends most of them.  2- and 4-bit codes: the window
// table, then the stride table (the codes of both windows are in the entry).
// The walks left go to the walk list for the third step (it has room for all
// of them; were it ever full, the error word says so).  Ids found go to the
// dense output (its -1 are written by the first phase), the count, or the
// unit's slots (no dense fallback: the gather step matches a unit with more
// matches than slots again).
constexpr int kSurvBlock = 256;
template <int SPT>
__host__ __device__ constexpr int surv_ctas() { return SPT <= 2 ? 6 : 4; }
static_assert(surv_ctas<2>() * kSurvBlock / 32 <= static_cast<int>(kSurvWarpsPerSm) &&
                  surv_ctas<4>() * kSurvBlock / 32 <= static_cast<int>(kSurvWarpsPerSm),
              "the walk list's room assumes at most kSurvWarpsPerSm warps of step 2 per SM");

template <int B, typename GT, int MODE, int SPT>
__global__ void __launch_bounds__(kSurvBlock, surv_ctas<SPT>()) pfac_survivors(const __grid_constant__ FilterParams p) {
    const int lane = threadIdx.x & 31;
    const GT *G = static_cast<const GT *>(p.G);
    const uint32_t listed = *reinterpret_cast<volatile const unsigned int *>(p.list_count);
    const uint32_t m = listed < p.list_cap ? listed : p.list_cap;
    const uint32_t stride = gridDim.x * blockDim.x;
    const int64_t head = static_cast<int64_t>(reinterpret_cast<uintptr_t>(p.text) & 15u);
    unsigned long long cnt = 0;
    // the part [wnext, wend) of the walk list this warp reserved
    uint32_t wnext = 0, wend = 0;
    // all lanes of a warp take part in every round (the walk list is filled
    // warp-wide): the loop runs on the warp's first index
    for (uint32_t wb = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wb < m; wb += SPT * stride) {
        const uint32_t b0 = wb + static_cast<uint32_t>(lane);
        uint4 e[SPT];
        int r[SPT];
        uint32_t s[SPT], q[SPT];
        bool walk[SPT];
        if constexpr (B == 8) {
            uint4 he[SPT];
#pragma unroll
            for (int t = 0; t < SPT; ++t) {
                const uint32_t idx = b0 + static_cast<uint32_t>(t) * stride;
                e[t] = idx < m ? __ldg(p.list + idx) : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
                he[t] = make_uint4(0u, 0u, 0u, 0u);
                if (e[t].x != 0xFFFFFFFFu) he[t] = __ldg(p.HK + hk_slot(p, e[t].y));
            }
            // outcomes; the first step of the walks from a branching state
            int g[SPT];
#pragma unroll
            for (int t = 0; t < SPT; ++t) {
                const bool on = e[t].x != 0xFFFFFFFFu;
                const uint32_t i = e[t].x & 1023u, c = e[t].z;  // c: the code after the window (0x100: none)
                r[t] = -1;
                s[t] = 0;
                q[t] = 0;
                walk[t] = on && !hk_outcome(p, hk_find(p, e[t].y, he[t]), i, c & 0xFFu, c < 0x100u, r[t], s[t], q[t]);
                if (walk[t]) r[t] = -1;  // its id comes from the walk
                // (every state has its goto row; the chain records only shortcut runs)
                g[t] = 0;
                if (walk[t] && q[t] == i + p.k) g[t] = goto_ld(G, s[t], p.W, c < 0x100u ? c : p.C);
            }
#pragma unroll
            for (int t = 0; t < SPT; ++t) {
                const uint32_t i = e[t].x & 1023u;
                if (walk[t] && q[t] == i + p.k) {
                    if (g[t] < 0) {
                        r[t] = decode_dead(g[t]);
                        walk[t] = false;
                    } else {
                        s[t] = static_cast<uint32_t>(g[t]);
                        ++q[t];
                    }
                }
            }
        } else {
            // the window table, then the stride table
            const uint32_t kmask = (1u << (B * p.k)) - 1u, k2mask = (1u << (B * p.k2)) - 1u;
            int j1[SPT], j2[SPT];
#pragma unroll
            for (int t = 0; t < SPT; ++t) {
                const uint32_t idx = b0 + static_cast<uint32_t>(t) * stride;
                e[t] = idx < m ? __ldg(p.list + idx) : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
                j1[t] = e[t].x != 0xFFFFFFFFu ? __ldg(p.JK + (e[t].y & kmask)) : -1;
            }
#pragma unroll
            for (int t = 0; t < SPT; ++t) {
                const uint32_t i = e[t].x & 1023u;
                r[t] = -1;
                s[t] = 0;
                q[t] = 0;
                walk[t] = false;
                j2[t] = -1;
                if (e[t].x == 0xFFFFFFFFu) continue;
                if (j1[t] < 0) {
                    r[t] = decode_dead(j1[t]);
                } else if (p.k2) {
                    j2[t] = __ldg(p.J2 + ((static_cast<uint64_t>(static_cast<uint32_t>(j1[t]) - p.base_k) << (B * p.k2)) |
                                          ((e[t].y >> (B * p.k)) & k2mask)));
                } else {
                    walk[t] = true;
                    s[t] = static_cast<uint32_t>(j1[t]);
                    q[t] = i + p.k;
                }
            }
#pragma unroll
            for (int t = 0; t < SPT; ++t) {
                if (e[t].x == 0xFFFFFFFFu || j1[t] < 0 || !p.k2) continue;
                if (j2[t] < 0) {
                    r[t] = decode_dead(j2[t]);
                } else {
                    walk[t] = true;
                    s[t] = static_cast<uint32_t>(j2[t]);
                    q[t] = (e[t].x & 1023u) + p.k + p.k2;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const uint32_t unit = e[t].x >> 10, i = e[t].x & 1023u;
            const int64_t gpb = static_cast<int64_t>(unit) * kTile - head;
            // walks that go on: to the walk list (warp-wide, in the warp's
            // chunk; when it runs out, its rest takes the first walks and a
            // new chunk the others, so that only each warp's last chunk has
            // unused entries)
            const unsigned wm = __ballot_sync(kFull, walk[t]);
            if (wm) {
                const uint32_t need = __popc(wm), rank = __popc(wm & ((1u << lane) - 1u));
                uint32_t slot = wnext + rank;
                if (wend - wnext < need) {
                    const uint32_t rest = wend - wnext;
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(p.list_count + 1, kWalkChunk);
                    base = __shfl_sync(kFull, base, 0);
                    if (rank >= rest) slot = base + (rank - rest);
                    wnext = base + (need - rest);
                    wend = base + kWalkChunk;
                    // the list has room for every walk and each warp's last chunk
                    if (static_cast<uint64_t>(base) + kWalkChunk > p.walk_cap) {  // so this cannot happen
                        if (lane == 0) atomicOr(p.err, static_cast<unsigned>(kErrWalk));
                        wnext = wend = 0;
                    }
                } else {
                    wnext += need;
                }
                if (walk[t] && wend != 0 && slot < p.walk_cap)
                    p.walks[slot] = make_uint2(e[t].x, s[t] | ((q[t] - i - p.k - p.k2) << 31));
            }
            const int rr = r[t];
            if (e[t].x == 0xFFFFFFFFu || rr < 0) continue;
            if (MODE == OUT_DENSE) {
                p.out[gpb + i] = rr;
            } else if (MODE == OUT_COUNT) {
                ++cnt;
            } else {
                const uint32_t su = p.sl.ubase + unit;
                const uint32_t k = atomicAdd(p.sl.counts + su, 1u);
                if (k < kSlotCap)
                    p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + k] =
                        (static_cast<unsigned long long>(static_cast<uint32_t>(rr)) << 32) |
                        static_cast<uint32_t>(gpb + i);
            }
        }
    }
    for (uint32_t j = wnext + static_cast<uint32_t>(lane); j < wend; j += 32u) p.walks[j] = make_uint2(0xFFFFFFFFu, 0u);
    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

// The third step of the phased form: one thread per listed walk (state, next
// byte) at high occupancy; the ids found go out as in the second step.
template <typename GT, int MODE>
__global__ void __launch_bounds__(kSurvBlock, surv_ctas<2>()) pfac_walks(const __grid_constant__ FilterParams p) {
    __shared__ uint8_t cls8[256];
    const int lane = threadIdx.x & 31;
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) cls8[i] = __ldg(p.cls8g + i);
    __syncthreads();
    const uint32_t listed = *reinterpret_cast<volatile const unsigned int *>(p.list_count + 1);
    const uint32_t m = listed < p.walk_cap ? listed : p.walk_cap;
    const int64_t head = static_cast<int64_t>(reinterpret_cast<uintptr_t>(p.text) & 15u);
    unsigned long long cnt = 0;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint2 e = __ldg(p.walks + j);
        if (e.x == 0xFFFFFFFFu) continue;
        const uint32_t unit = e.x >> 10, i = e.x & 1023u;
        const int64_t gpb = static_cast<int64_t>(unit) * kTile - head;
        const int r = walk_global<GT>(p, cls8, make_text(p.text, p.out, p.n, unit), gpb, e.y & 0x7FFFFFFFu,
                                      i + p.k + p.k2 + (e.y >> 31));
        if (r < 0) continue;
        if (MODE == OUT_DENSE) {
            p.out[gpb + i] = r;
        } else if (MODE == OUT_COUNT) {
            ++cnt;
        } else {
            const uint32_t su = p.sl.ubase + unit;
            const uint32_t k = atomicAdd(p.sl.counts + su, 1u);
            if (k < kSlotCap)
                p.sl.slots[static_cast<uint64_t>(su) * kSlotCap + k] =
                    (static_cast<unsigned long long>(static_cast<uint32_t>(r)) << 32) | static_cast<uint32_t>(gpb + i);
        }
    }
    if (MODE == OUT_COUNT) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(kFull, cnt, d);
        if (lane == 0 && cnt) atomicAdd(p.count, cnt);
    }
}

template <int B, typename GT, int SPT>
cudaError_t launch_survivors(OutMode mode, const FilterParams &p, uint32_t sms, cudaStream_t stream) {
    const uint32_t grid = sms * static_cast<uint32_t>(surv_ctas<SPT>());
    switch (mode) {
        case OUT_DENSE: pfac_survivors<B, GT, OUT_DENSE, SPT><<<grid, kSurvBlock, 0, stream>>>(p); break;
        case OUT_COUNT: pfac_survivors<B, GT, OUT_COUNT, SPT><<<grid, kSurvBlock, 0, stream>>>(p); break;
        case OUT_SLOTS: pfac_survivors<B, GT, OUT_SLOTS, SPT><<<grid, kSurvBlock, 0, stream>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !p.walks) return e;
    const uint32_t wgrid = sms * static_cast<uint32_t>(surv_ctas<2>());
    switch (mode) {
        case OUT_DENSE: pfac_walks<GT, OUT_DENSE><<<wgrid, kSurvBlock, 0, stream>>>(p); break;
        case OUT_COUNT: pfac_walks<GT, OUT_COUNT><<<wgrid, kSurvBlock, 0, stream>>>(p); break;
        default: pfac_walks<GT, OUT_SLOTS><<<wgrid, kSurvBlock, 0, stream>>>(p); break;
    }
    return cudaGetLastError();
}

// Batches: every automaton of the batch (at most kMultiMax) in one persistent
// launch.  Each CTA takes the automata in order: it fetches an automaton's
// tables into shared memory, its warps take that automaton's units through
// filter_units (the units of all its texts, from its own counter), and once
// all of the CTA's warps are done with it the CTA moves to the next.  CTAs
// move on independently, so the automata overlap on the GPU and no launch
// boundary drains the grid between them.  Every automaton of the launch
// shares one shared-memory layout (offsets from a[0]); the automaton being
// matched has its parameters copied to shared memory at params_off.
constexpr uint32_t kMultiMax = 32;
// Threads per CTA of the multi-automaton kernel: 12 warps, which leaves room
// for the automaton loop's registers around the largest form with few spills.
constexpr int kMultiBlock = 384;

struct MultiParams {
    FilterParams a[kMultiMax];
    uint32_t nh;
    uint32_t params_off;
    // the phased form of the 8-bit-code automata (list null: none); the same
    // lists are in their a[].list / walks4
    uint4 *list;
    unsigned int *list_count;
    uint32_t list_cap;
    uint4 *walks4;
    uint32_t walk_cap;
};
static_assert(sizeof(FilterParams) % 4 == 0, "parameters are copied as words");
static_assert(sizeof(MultiParams) <= 32764, "kernel parameters are limited to 32764 bytes");

// FilterParams::kind of a form: (B << 8) | goto-entry bits.
__host__ __device__ constexpr uint32_t filter_kind(uint32_t B, uint32_t gbits) { return (B << 8) | gbits; }

template <int MODE, bool LISTED>
__global__ void __launch_bounds__(kMultiBlock, 1) pfac_filter_multi(const __grid_constant__ MultiParams mp) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    filter_setup(mp.a[0], smem);
    FilterParams &p = *reinterpret_cast<FilterParams *>(smem + mp.params_off);
    uint32_t it = 0, loads = 0;
    int bad = 0;
    for (uint32_t a = 0; a < mp.nh; ++a) {
        if (__ldg(&mp.a[a].batch->units) == 0) continue;  // the same for every thread
        // the CTA is done with the previous automaton (and leaves together
        // when a warp's bounded wait ran out)
        if (__syncthreads_or(bad)) break;
        for (uint32_t i = threadIdx.x; i < sizeof(FilterParams) / 4; i += blockDim.x)
            reinterpret_cast<uint32_t *>(&p)[i] = reinterpret_cast<const uint32_t *>(&mp.a[a])[i];
        __syncthreads();
        if (threadIdx.x == 0) filter_load_tables(p, smem);
        unsigned long long cnt = 0;  // batches have no count mode
        bool ok = true;
        switch (p.kind) {
            case filter_kind(2, 16): ok = filter_units<2, int16_t, MODE, true, false, LISTED>(p, smem, it, loads & 1u, cnt, &it); break;
            case filter_kind(2, 32): ok = filter_units<2, int32_t, MODE, true, false, LISTED>(p, smem, it, loads & 1u, cnt, &it); break;
            case filter_kind(4, 16): ok = filter_units<4, int16_t, MODE, true, false, LISTED>(p, smem, it, loads & 1u, cnt, &it); break;
            case filter_kind(4, 32): ok = filter_units<4, int32_t, MODE, true, false, LISTED>(p, smem, it, loads & 1u, cnt, &it); break;
            case filter_kind(8, 16): ok = filter_units<8, int16_t, MODE, true, false, LISTED>(p, smem, it, loads & 1u, cnt, &it); break;
            default: ok = filter_units<8, int32_t, MODE, true, false, LISTED>(p, smem, it, loads & 1u, cnt, &it); break;
        }
        ++loads;
        bad |= ok ? 0 : 1;
    }
    if (MODE == OUT_DENSE && lane == 0) bulk_wait_all();
}

// The second and third steps of a batch's phased form: the survivors that
// the first phase (pfac_filter_multi) listed for the launch's 8-bit-code
// automata, each with its automaton (third word, from bit 16) and its unit's
// planned-list entry (fourth word); then the walks they leave.  Each CTA
// copies the automata's parameters (and, for the walks, their byte tables)
// to shared memory.  Results go out as the single-text steps write them, at
// the unit's text.
__device__ __forceinline__ void multi_params_to_smem(const MultiParams &mp, FilterParams *ps) {
    for (uint32_t i = threadIdx.x; i < mp.nh * static_cast<uint32_t>(sizeof(FilterParams) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(ps)[i] = reinterpret_cast<const uint32_t *>(mp.a)[i];
}

// The text of a listed unit (its planned-list entry `item`) and the tile's
// first position in it.
__device__ __forceinline__ TileText listed_text(const FilterParams &P, uint32_t unit, uint32_t item, int64_t &gpb) {
    const Work wk = load_work(P.batch, P.lists, 0);
    const TileText tt = batch_text(wk, P.text, P.out, item, unit);
    gpb = static_cast<int64_t>(static_cast<uint64_t>(tt.tile) * kTile) - tt.head;
    return tt;
}

template <int MODE>
__device__ __forceinline__ void listed_output(const FilterParams &P, const TileText &tt, int64_t gpb, uint32_t unit,
                                              uint32_t i, int r) {
    if (MODE == OUT_DENSE) {
        tt.out[gpb + i] = r;
    } else {
        const uint32_t su = P.sl.ubase + unit;
        const uint32_t k = atomicAdd(P.sl.counts + su, 1u);
        if (k < kSlotCap)
            P.sl.slots[static_cast<uint64_t>(su) * kSlotCap + k] =
                (static_cast<unsigned long long>(static_cast<uint32_t>(r)) << 32) | static_cast<uint32_t>(gpb + i);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kSurvBlock, surv_ctas<2>()) pfac_survivors_multi(const __grid_constant__ MultiParams mp) {
    extern __shared__ __align__(16) uint8_t msm[];
    FilterParams *ps = reinterpret_cast<FilterParams *>(msm);
    multi_params_to_smem(mp, ps);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t listed = *reinterpret_cast<volatile const unsigned int *>(mp.list_count);
    const uint32_t m = listed < mp.list_cap ? listed : mp.list_cap;
    const uint32_t stride = gridDim.x * blockDim.x;
    constexpr int SPT = 2;
    uint32_t wnext = 0, wend = 0;
    for (uint32_t wb = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wb < m; wb += SPT * stride) {
        const uint32_t b0 = wb + static_cast<uint32_t>(lane);
        uint4 e[SPT], he[SPT];
        // first loads: 8-bit codes the state-hash bucket, small alphabets the
        // window table (he[].x)
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const uint32_t idx = b0 + static_cast<uint32_t>(t) * stride;
            e[t] = idx < m ? __ldg(mp.list + idx) : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
            he[t] = make_uint4(0u, 0u, 0u, 0u);
            if (e[t].x != 0xFFFFFFFFu) {
                const FilterParams &P = ps[(e[t].z >> 16) & (kMultiMax - 1u)];
                if ((P.kind >> 8) == 8u)
                    he[t] = __ldg(P.HK + hk_slot(P, e[t].y));
                else
                    he[t].x = static_cast<uint32_t>(__ldg(P.JK + (e[t].y & ((1u << ((P.kind >> 8) * P.k)) - 1u))));
            }
        }
        int r[SPT], g[SPT];
        uint32_t s[SPT], q[SPT];
        bool walk[SPT];
        // second loads: 8-bit codes the first goto step of a branching state,
        // small alphabets the stride table
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const bool on = e[t].x != 0xFFFFFFFFu;
            const FilterParams &P = ps[(e[t].z >> 16) & (kMultiMax - 1u)];
            const uint32_t i = e[t].x & 1023u, c = e[t].z & 0x1FFu, Bq = P.kind >> 8;
            r[t] = -1;
            s[t] = 0;
            q[t] = 0;
            g[t] = 0;
            if (Bq == 8u) {
                walk[t] = on && !hk_outcome(P, hk_find(P, e[t].y, he[t]), i, c & 0xFFu, c < 0x100u, r[t], s[t], q[t]);
                if (walk[t]) r[t] = -1;
                if (walk[t] && q[t] == i + P.k) {
                    const uint32_t col = c < 0x100u ? c : P.C;
                    g[t] = (P.kind & 0xFFu) == 16u ? goto_ld(static_cast<const int16_t *>(P.G), s[t], P.W, col)
                                                   : goto_ld(static_cast<const int32_t *>(P.G), s[t], P.W, col);
                }
            } else {
                walk[t] = false;
                if (!on) continue;
                const int j1 = static_cast<int>(he[t].x);
                if (j1 < 0) {
                    r[t] = decode_dead(j1);
                } else if (P.k2) {
                    g[t] = __ldg(P.J2 + ((static_cast<uint64_t>(static_cast<uint32_t>(j1) - P.base_k) << (Bq * P.k2)) |
                                         ((e[t].y >> (Bq * P.k)) & ((1u << (Bq * P.k2)) - 1u))));
                    walk[t] = true;  // settled below by the stride entry
                    s[t] = 0xFFFFFFFFu;
                } else {
                    walk[t] = true;
                    s[t] = static_cast<uint32_t>(j1);
                    q[t] = i + P.k;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const FilterParams &P = ps[(e[t].z >> 16) & (kMultiMax - 1u)];
            const uint32_t i = e[t].x & 1023u;
            if ((P.kind >> 8) == 8u) {
                if (walk[t] && q[t] == i + P.k) {
                    if (g[t] < 0) {
                        r[t] = decode_dead(g[t]);
                        walk[t] = false;
                    } else {
                        s[t] = static_cast<uint32_t>(g[t]);
                        ++q[t];
                    }
                }
            } else if (walk[t] && s[t] == 0xFFFFFFFFu) {  // the stride entry
                if (g[t] < 0) {
                    r[t] = decode_dead(g[t]);
                    walk[t] = false;
                } else {
                    s[t] = static_cast<uint32_t>(g[t]);
                    q[t] = i + P.k + P.k2;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const uint32_t a = (e[t].z >> 16) & (kMultiMax - 1u);
            const FilterParams &P = ps[a];
            const uint32_t unit = e[t].x >> 10, i = e[t].x & 1023u;
            const unsigned wm = __ballot_sync(kFull, walk[t]);
            if (wm) {  // to the walk list, as in the single-text step
                const uint32_t need = __popc(wm), rank = __popc(wm & ((1u << lane) - 1u));
                uint32_t slot = wnext + rank;
                if (wend - wnext < need) {
                    const uint32_t rest = wend - wnext;
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(mp.list_count + 1, kWalkChunk);
                    base = __shfl_sync(kFull, base, 0);
                    if (rank >= rest) slot = base + (rank - rest);
                    wnext = base + (need - rest);
                    wend = base + kWalkChunk;
                    if (static_cast<uint64_t>(base) + kWalkChunk > mp.walk_cap) {  // cannot happen (room for all)
                        if (lane == 0) atomicOr(P.err, static_cast<unsigned>(kErrWalk));
                        wnext = wend = 0;
                    }
                } else {
                    wnext += need;
                }
                if (walk[t] && wend != 0 && slot < mp.walk_cap)
                    mp.walks4[slot] = make_uint4(e[t].x, s[t] | ((q[t] - i - P.k - P.k2) << 31), a, e[t].w);
            }
            if (e[t].x == 0xFFFFFFFFu || r[t] < 0) continue;
            int64_t gpb = 0;
            const TileText tt = listed_text(P, unit, e[t].w, gpb);
            listed_output<MODE>(P, tt, gpb, unit, i, r[t]);
        }
    }
    for (uint32_t j = wnext + static_cast<uint32_t>(lane); j < wend; j += 32u)
        mp.walks4[j] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
}

template <int MODE>
__global__ void __launch_bounds__(kSurvBlock, surv_ctas<2>()) pfac_walks_multi(const __grid_constant__ MultiParams mp) {
    extern __shared__ __align__(16) uint8_t msm[];
    FilterParams *ps = reinterpret_cast<FilterParams *>(msm);
    uint8_t *cls = msm + mp.nh * sizeof(FilterParams);
    multi_params_to_smem(mp, ps);
    for (uint32_t i = threadIdx.x; i < mp.nh * 256u; i += blockDim.x) cls[i] = __ldg(mp.a[i >> 8].cls8g + (i & 255u));
    __syncthreads();
    const uint32_t listed = *reinterpret_cast<volatile const unsigned int *>(mp.list_count + 1);
    const uint32_t m = listed < mp.walk_cap ? listed : mp.walk_cap;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint4 e = __ldg(mp.walks4 + j);
        if (e.x == 0xFFFFFFFFu) continue;
        const uint32_t a = e.z & (kMultiMax - 1u);
        const FilterParams &P = ps[a];
        const uint32_t unit = e.x >> 10, i = e.x & 1023u;
        int64_t gpb = 0;
        const TileText tt = listed_text(P, unit, e.w, gpb);
        const uint32_t st = e.y & 0x7FFFFFFFu, q = i + P.k + P.k2 + (e.y >> 31);
        const int r = (P.kind & 0xFFu) == 16u ? walk_global<int16_t>(P, cls + 256u * a, tt, gpb, st, q)
                                              : walk_global<int32_t>(P, cls + 256u * a, tt, gpb, st, q);
        if (r >= 0) listed_output<MODE>(P, tt, gpb, unit, i, r);
    }
}

inline uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

template <int B, typename GT, int MODE, bool BATCH, bool HELP, bool LISTED = false, int MAXT = kStdBlock,
          bool DIRECT = false>
cudaError_t launch_one_bounded(const FilterParams &p, uint32_t grid, uint32_t block, uint32_t smem, int max_smem,
                               cudaStream_t stream) {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void (*kernel)(const FilterParams) = pfac_filter_pipe<B, GT, MODE, BATCH, HELP, LISTED, MAXT, DIRECT>;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    kernel<<<grid, block, smem, stream>>>(p);
    return cudaGetLastError();
}

// The one-phase single-text forms of 2-bit codes at more than 512 threads
// whose codes come from (byte >> 1) & 3 (DIRECT), filter_direct.cu.
cudaError_t launch_filter_direct(int mode, const FilterParams &p, uint32_t gbits, uint32_t grid, uint32_t block,
                                 uint32_t smem, int max_smem, cudaStream_t stream);

// The forms at up to 512 threads; more only for the one-phase single-text
// forms of 2- and 4-bit codes (2-bit codes with p.direct_shift set: the
// DIRECT forms).
template <int B, typename GT, int MODE, bool BATCH, bool HELP, bool LISTED = false>
cudaError_t launch_one(const FilterParams &p, uint32_t grid, uint32_t block, uint32_t smem, int max_smem,
                       cudaStream_t stream) {
    if (block <= static_cast<uint32_t>(kStdBlock))
        return launch_one_bounded<B, GT, MODE, BATCH, HELP, LISTED>(p, grid, block, smem, max_smem, stream);
    if constexpr (B <= 4 && !BATCH && !HELP && !LISTED) {
        if (B == 2 && p.direct_shift == 1)
            return launch_filter_direct(MODE, p, 8u * sizeof(GT), grid, block, smem, max_smem, stream);
        return launch_one_bounded<B, GT, MODE, false, false, false, kMaxBlock>(p, grid, block, smem, max_smem,
                                                                             stream);
    }
    return cudaErrorInvalidConfiguration;
}

template <int B, typename GT, bool HELP>
cudaError_t launch_modes(OutMode mode, const FilterParams &p, uint32_t grid, uint32_t block, uint32_t smem,
                         int max_smem, cudaStream_t stream) {
    if constexpr (HELP) {  // one text only
        switch (mode) {
            case OUT_DENSE:
                return launch_one<B, GT, OUT_DENSE, false, true>(p, grid, block, smem, max_smem, stream);
            case OUT_COUNT:
                return launch_one<B, GT, OUT_COUNT, false, true>(p, grid, block, smem, max_smem, stream);
            case OUT_SLOTS:
                return launch_one<B, GT, OUT_SLOTS, false, true>(p, grid, block, smem, max_smem, stream);
            default:
                return cudaErrorInvalidValue;
        }
    } else if (p.list && !p.batch) {  // the first phase of the phased form
        switch (mode) {
            case OUT_DENSE:
                return launch_one<B, GT, OUT_DENSE, false, false, true>(p, grid, block, smem, max_smem, stream);
            case OUT_COUNT:
                return launch_one<B, GT, OUT_COUNT, false, false, true>(p, grid, block, smem, max_smem, stream);
            case OUT_SLOTS:
                return launch_one<B, GT, OUT_SLOTS, false, false, true>(p, grid, block, smem, max_smem, stream);
            default:
                return cudaErrorInvalidValue;
        }
    } else {
        switch (mode) {
            case OUT_DENSE:
                return p.batch ? launch_one<B, GT, OUT_DENSE, true, false>(p, grid, block, smem, max_smem, stream)
                               : launch_one<B, GT, OUT_DENSE, false, false>(p, grid, block, smem, max_smem, stream);
            case OUT_COUNT:
                return launch_one<B, GT, OUT_COUNT, false, false>(p, grid, block, smem, max_smem, stream);
            case OUT_SLOTS:
                return p.batch ? launch_one<B, GT, OUT_SLOTS, true, false>(p, grid, block, smem, max_smem, stream)
                               : launch_one<B, GT, OUT_SLOTS, false, false>(p, grid, block, smem, max_smem, stream);
            default:
                return cudaErrorInvalidValue;
        }
    }
}

}  // namespace filt

// Launch of the forms that share heavy tiles (one text only), filter_help.cu.
cudaError_t launch_filter_help(OutMode mode, const filt::FilterParams &p, uint32_t B, uint32_t gbits, uint32_t grid,
                               uint32_t block, uint32_t smem, int max_smem, cudaStream_t stream);
// Launch of the 8-bit-code forms (hashed filter) and of the second phase of
// their two-phase form, filter8.cu.
cudaError_t launch_filter8(OutMode mode, const filt::FilterParams &p, uint32_t gbits, uint32_t grid, uint32_t block,
                           uint32_t smem, int max_smem, cudaStream_t stream);
// The second and third steps of the phased form (survivors.cu); per_thread:
// survivors a thread of the second step takes at a time (2 or 4; 8-bit codes).
cudaError_t launch_survivors(OutMode mode, const filt::FilterParams &p, uint32_t B, uint32_t gbits, uint32_t sms,
                             int per_thread, cudaStream_t stream);

namespace filt {
template <int MODE, bool LISTED>
cudaError_t launch_multi_one(const MultiParams &mp, uint32_t grid, uint32_t smem, int max_smem, cudaStream_t stream) {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(pfac_filter_multi<MODE, LISTED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    pfac_filter_multi<MODE, LISTED><<<grid, kMultiBlock, smem, stream>>>(mp);
    return cudaGetLastError();
}

// The multi-automaton launch, and with lists the second and third steps.
template <int MODE>
cudaError_t launch_multi(const MultiParams &mp, uint32_t sms, uint32_t smem, int max_smem, cudaStream_t stream) {
    if (!mp.list) return launch_multi_one<MODE, false>(mp, sms, smem, max_smem, stream);
    cudaError_t e = launch_multi_one<MODE, true>(mp, sms, smem, max_smem, stream);
    if (e != cudaSuccess) return e;
    const uint32_t grid = sms * static_cast<uint32_t>(surv_ctas<2>());
    const uint32_t ps = mp.nh * static_cast<uint32_t>(sizeof(FilterParams));
    pfac_survivors_multi<MODE><<<grid, kSurvBlock, ps, stream>>>(mp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pfac_walks_multi<MODE><<<grid, kSurvBlock, ps + 256u * mp.nh, stream>>>(mp);
    return cudaGetLastError();
}
}  // namespace filt

// Launches of the multi-automaton kernel (grid: the SM count; with lists also
// the second and third steps), filter_multi_dense.cu and filter_multi_slots.cu.
cudaError_t launch_filter_multi_dense(const filt::MultiParams &mp, uint32_t grid, uint32_t smem, int max_smem,
                                      cudaStream_t stream);
cudaError_t launch_filter_multi_slots(const filt::MultiParams &mp, uint32_t grid, uint32_t smem, int max_smem,
                                      cudaStream_t stream);
inline cudaError_t launch_filter_multi_modes(OutMode mode, const filt::MultiParams &mp, uint32_t grid, uint32_t smem,
                                             int max_smem, cudaStream_t stream) {
    return mode == OUT_DENSE ? launch_filter_multi_dense(mp, grid, smem, max_smem, stream)
                             : launch_filter_multi_slots(mp, grid, smem, max_smem, stream);
}

}  // namespace pfac
