// Internal declarations shared by the builder, the kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>

#include <cuda_runtime_api.h>

#include "ac.h"

namespace pfac {

// A dead goto entry encodes the result of a walk that stops at its row:
// entry = -(id + 2), id = keyword id or -1.  Live entries are child ids > 0
// (the root, state 0, is never a child).
inline int32_t encode_dead(int32_t id) { return -(id + 2); }

// Root jump-table entries are int16: a result (>= -1) when the walk stops
// within the window, -(2 + r) for the r-th state at depth k when it is still
// alive there (r < kJumpMaxStates), or kJumpSlow to send the start to the
// plain walk (a result that does not fit 15 bits).
constexpr int16_t kJumpSlow = -32768;

// Chain record of a state with two or more children: take its goto row.
constexpr uint32_t kSkipBranch = 0xFFFFFFFFu;

// Full-output record field `up` of a keyword with no keyword as a proper prefix.
constexpr uint32_t kNoKeyword = 0xFFFFFFFFu;
constexpr uint32_t kJumpMaxStates = 32766;

// Bits of the per-device kernel error word.
enum : unsigned { kErrTimeout = 1u, kErrWalk = 2u, kErrBatchItem = 8u };

// Window bits of the root filter (2- and 4-bit codes): 2^20 bits = 128 KiB.
constexpr uint32_t kFilterBits = 20;

// 8-bit codes: the hashed root filter and the hash of the depth-kh states
// index a window w of kh codes (first code lowest) by the top bits of
// w * kFilterHashMul and w * kStateHashMul (mod 2^32).
constexpr uint32_t kFilterHashMul = 0x9E3779B1u;
constexpr uint32_t kStateHashMul = 0x85EBCA77u;
constexpr uint32_t kHashWindow = 4;  // codes per hashed window (at most)
// State-hash entry field `child` of a depth-kh state with several children.
constexpr uint32_t kHkBranch = 0xFFFFFFFFu;

// Longest halo staged in shared memory; walks that run past it read global memory.
constexpr uint32_t kHaloCap = 256;

struct BuildOptions {
    int index_width = 0;        // 0 = auto, 16, 32
    int class_compress = 1;     // 1 = distinct keyword bytes, 0 = 256 columns
    uint32_t jump_bytes = 128u << 10;
    uint64_t stride_bytes = 16ull << 20;
    bool chains = true;         // chain records for the deep states
};

// A byte buffer sized without a fill: its owner writes every byte (the
// builder fills the goto table's rows in parallel, so a zero fill first would
// be one more serial pass over up to a gigabyte).
struct RawBytes {
    std::unique_ptr<uint8_t[]> p;
    size_t n = 0;
    uint8_t *data() { return p.get(); }
    const uint8_t *data() const { return p.get(); }
    size_t size() const { return n; }
    void resize_unfilled(size_t m) {  // throws std::bad_alloc
        p.reset(new uint8_t[m]);
        n = m;
    }
};

// Host-side automaton: everything the kernels need, in the layout they use.
struct HostTables {
    uint32_t nkw = 0;        // keywords
    uint32_t S = 0;          // states (BFS order, root = 0)
    uint32_t C = 0;          // classes (distinct keyword bytes, or 256)
    uint32_t W = 0;          // row width: C goto columns + 1 end column, padded
    uint32_t gbits = 32;     // goto entry width (16 or 32)
    uint32_t B = 8;          // bits per character code in the packed stream (2, 4, 8)
    uint32_t k = 0;          // root jump depth (0 = no jump table)
    uint32_t k2 = 0;         // stride depth after the jump (0 = none)
    uint32_t base_k = 0;     // first state at depth k
    uint32_t count_k = 0;    // states at depth k
    uint32_t minlen = 0, maxlen = 0;
    std::vector<int16_t> cls;        // 256: byte -> code or -1
    std::vector<uint8_t> cls8;       // 256: byte -> code, 0xFF = in no keyword (identity when C = 256)
    bool jslow = false;              // some jump entry is kJumpSlow
    // Small alphabets (at most 8 keyword bytes): a shift s such that
    // (byte >> s) & 7 differs for every keyword byte, or -1.  hash_code[h] is
    // the class code of the keyword byte with hash h, hash_byte[h] that byte
    // (or a byte whose hash is not h, for unused h).
    int hash_shift = -1;
    uint8_t hash_code[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint8_t hash_byte[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // Exactly four keyword bytes that (byte >> 1) & 3 tells apart (the DNA
    // letters, either case): their class codes are that value, so the kernel
    // computes four codes with one multiply (direct_shift = 1); direct_byte[c]
    // is the keyword byte of code c.  Else direct_shift = -1.
    int direct_shift = -1;
    uint8_t direct_byte[4] = {0, 0, 0, 0};
    RawBytes G;                      // S * W entries of gbits
    bool filter = false;             // B <= 4: root filter + window table instead of J
    std::vector<uint32_t> F;         // filter bits, 2^(B*k) (at least 4 words)
    std::vector<int32_t> JK;         // window table, 2^(B*k) entries
    uint32_t match_windows_ppm = 0;  // windows of JK whose walk found a keyword, per million
    std::vector<int16_t> J;          // 2^(B*k) (padded to 8 entries)
    std::vector<int32_t> J2;         // count_k << (B*k2)
    std::vector<uint32_t> depth_count;  // maxlen + 1
    // Chain records, one per state from s_chain on (4 words: run length or
    // kSkipBranch, offset of the run's bytes in `chain`, the run's end state,
    // the state's result), and the runs' raw bytes.
    uint32_t s_chain = 0;
    std::vector<uint32_t> skip;
    std::vector<uint8_t> chain;
    // 8-bit codes: a hashed root filter over windows of kh = min(4, shortest
    // keyword) codes, in F (2^fbits bits, the same bit layout as the small
    // alphabets' filter): the bit of the window of every depth-kh state is
    // set, so a clear bit means the walk stops before depth kh, where no
    // keyword ends (result -1).  HK: the depth-kh states by their window, in
    // 2^hk_bits entries of four words {window, state (0: empty), child,
    // (child code << 24) | (result + 1)}, linear probing over at most
    // hk_probes entries; child: the state's one child, 0 for a leaf, or
    // kHkBranch (several children: take the goto row).
    bool hashed = false;
    uint32_t kh = 0, fbits = 0, hk_bits = 0, hk_probes = 0;
    std::vector<uint32_t> HK;
    // Full output: 4 words per keyword id {up, len, dup_off, clen} (set for
    // the lowest id of each keyword string, the id a walk reports), the ids
    // grouped by string, and the largest clen.
    std::vector<uint32_t> full_rec;
    std::vector<uint32_t> full_dups;
    uint32_t full_max_clen = 0;
    bool identity_classes() const { return C == 256; }
};

// Returns an ac_status value.
int build_tables(const uint8_t *const *patterns, const uint32_t *lens, uint32_t k,
                 const BuildOptions &opt, HostTables *out);

// Largest k + k2 the kernel's code window allows for a code width (one 32-bit
// window of 2- or 4-bit codes, one 64-bit window of 8-bit codes).
inline uint32_t window_limit(uint32_t B) { return B == 2 ? 16u : 8u; }

// The tables of the root filter kernel that depend on how much of it sits in
// shared memory (its depth): computed by the builder, and again by the
// autotuner for other depths from the goto table alone.
struct RootTables {
    uint32_t k = 0, k2 = 0, base_k = 0, count_k = 0;  // 2- and 4-bit codes
    uint32_t fbits = 0;                                // 8-bit codes
    std::vector<uint32_t> F;
    std::vector<int32_t> JK, J2;
    // 2- and 4-bit codes: the windows whose walk already found a keyword, per
    // million windows (the share of positions where a match ends inside the
    // window on uniform text)
    uint32_t match_windows_ppm = 0;
};
// Windows with a match inside, per million, from which small-alphabet
// automata resolve survivors in the phased form by default: with matches that
// common the warps' in-tile pipeline writes ids position by position and
// falls behind the listed form (1 GiB sweep set: 0 ppm, in the warps 1.11 ms
// against 1.24 listed; 256 MiB batch sets with 8-byte keywords: 1,100-9,000
// ppm, listed 8-66 % faster; 290 ppm, in the warps 6 % faster).
constexpr uint32_t kListMatchWindowsPpm = 500;
// 2- and 4-bit codes: the root filter and window table over windows of k codes
// (1 <= k, B k <= kFilterBits), and the stride table from the depth-k states
// (at most stride_bytes; none when 0 or 1).
void window_tables(const HostTables &h, uint32_t k, uint64_t stride_bytes, RootTables *out);
// 8-bit codes with the state hash: the hashed filter at 2^fbits bits (5 <=
// fbits <= kFilterBits), from the windows in the state hash.
void hashed_filter(const HostTables &h, uint32_t fbits, RootTables *out);
// The widest window of B-bit codes whose filter fits `bytes`.
uint32_t filter_window(uint32_t B, uint32_t maxlen, uint32_t bytes);

// Device view of a compiled automaton.
struct DevTables {
    const void *G = nullptr;         // goto table
    const int16_t *J = nullptr;      // root jump table (device copy, for the bulk load)
    const uint32_t *F = nullptr;     // root filter bits (device copy, for the bulk load)
    const int32_t *JK = nullptr;     // window table (filter mode)
    uint32_t fbytes = 0;             // bytes of F
    bool filter = false;             // 2- and 4-bit codes: root filter + window table
    bool list_prefer = false;        // small alphabets: the phased form by default (kListMatchWindowsPpm)
    bool hashed = false;             // 8-bit codes: hashed root filter + state hash
    const uint4 *HK = nullptr;       // state hash buckets (hashed)
    uint32_t kh = 0, fbits = 0, hk_bits = 0, hk_probes = 0;
    const int32_t *J2 = nullptr;     // stride table
    const uint4 *skip = nullptr;     // chain records (states from s_chain on), or none
    const uint8_t *chain = nullptr;  // chain bytes
    uint32_t s_chain = 0xFFFFFFFFu;  // first state with a chain record
    const uint4 *full_rec = nullptr;    // full-output records (one per keyword id)
    const uint32_t *full_dups = nullptr;
    uint32_t full_max_clen = 0;
    uint32_t nkw = 0;
    const int16_t *cls = nullptr;    // class map (256 entries)
    const uint8_t *cls8 = nullptr;   // byte class map (256 entries, 0xFF = unknown byte)
    uint32_t S = 0, C = 0, W = 0, gbits = 32, B = 8, k = 0, k2 = 0, base_k = 0, maxlen = 0;
    uint32_t jbytes = 0;             // bytes of J (multiple of 16)
    bool jslow = false;
    int hash_shift = -1;             // see HostTables
    uint32_t hash_code[2] = {0, 0};  // hash_code bytes, little-endian
    uint32_t hash_byte[2] = {0, 0};
    int direct_shift = -1;           // see HostTables
    uint32_t direct_sel[2] = {0, 0}; // byte 2c of the pair: the keyword byte of code c
    uint32_t direct_fill = 0;        // a byte in no keyword
};

// OUT_SLOTS: per work unit, the number of matches and the first kSlotCap of
// them in any order (SlotOut); the compacted list is then made by the scan
// and gather steps (compact.cu).  OUT_COMPACT names that whole sequence.
enum OutMode : int { OUT_DENSE = 0, OUT_COUNT = 1, OUT_COMPACT = 2, OUT_SLOTS = 3 };

// Matches a unit keeps in its slots; for a unit with more, the gather step
// reads the unit's dense ids (SlotOut::dense), or matches it again.
constexpr uint32_t kSlotCap = 32;

// Entries per unit in SlotOut::dense (every kernel's tile is at most this long).
constexpr uint32_t kDenseStride = 1024;

struct SlotOut {
    uint32_t *counts = nullptr;              // per unit, zeroed before the launch
    unsigned long long *slots = nullptr;     // per unit kSlotCap entries: (id << 32) | position in its text
    uint32_t ubase = 0;                      // counts / slots index of the launch's unit 0
    // Optional, per unit kDenseStride entries: the dense ids of the unit's
    // positions (entry i: tile position i), written where a unit may hold more
    // than kSlotCap matches, so the gather step reads them instead of matching
    // the unit again.
    int32_t *dense = nullptr;
};

// Where one text's compacted list goes (ac_match_compact's arguments).
struct CompactOut {
    uint32_t *pos;
    uint32_t *ids;
    unsigned long long cap;
    unsigned long long *count;
};

// One text of a batch as the matching kernels read it: its bytes at
// texts + text_off, its dense ids at outs + out_off, its tiles numbered from
// first_unit among the texts of its automaton.  Written on the device by the
// batch planning kernel; `item` is the text's index in the caller's list.
struct alignas(16) BatchItemDev {
    uint64_t text_off, len, out_off;
    uint32_t first_unit, item;
};
static_assert(sizeof(BatchItemDev) == 32, "BatchItemDev is read as two 16-byte words");

// Per automaton of a batch: its tiles (work units), its non-empty texts and
// where they start in the planned list (ascending first_unit).
struct BatchHead {
    uint32_t units, count, offset, pad;
};

struct MatchRequest {
    const uint8_t *text = nullptr;           // batch: base of all texts
    uint64_t n = 0;                          // batch: unused
    int32_t *out = nullptr;                  // dense (batch: base of all outputs)
    const BatchHead *batch = nullptr;        // batch: this automaton's head (device)
    const BatchItemDev *lists = nullptr;     // batch: the planned list (device)
    unsigned long long *count = nullptr;     // count
    SlotOut slots;                           // OUT_SLOTS
    void *scratch = nullptr;                 // zeroed: tile counter (16 bytes)
    size_t scratch_bytes = 0;
    // One long text: the lists of the phased form (survivor_lists); list =
    // nullptr: every tile's survivors are resolved by the warp that filtered
    // it.
    uint4 *list = nullptr;
    unsigned int *list_count = nullptr;      // zeroed, two words: survivors, walks
    uint32_t list_cap = 0;
    uint2 *walks = nullptr;
    uint32_t walk_cap = 0;
};

// The phased form of the filter kernel for one long text:
//   1. the filter kernel stages, filters and writes the -1 of every tile, and
//      appends each survivor to a list instead of resolving it -- 8-bit
//      codes: {(tile << 10) | tile position, window, code of the character
//      after it (0x100: none), 0}; 2- and 4-bit codes: {(tile << 10) |
//      position, the codes from the position on (window and stride
//      window), 0, 0};
//   2. one thread per survivor at full occupancy resolves it -- 8-bit codes:
//      its state-hash entry, and for a branching state the first goto step;
//      2- and 4-bit codes: the window table, then the stride table -- and
//      writes the ids found; a survivor whose walk goes on is appended to a
//      second list -- {(tile << 10) | position, state | d << 31}, the walk's
//      next byte at tile index position + k + k2 + d;
//   3. one thread per walk, at full occupancy, finishes the walks.
// Warps reserve list space in chunks (entries they leave unused are marked
// empty: x = 0xFFFFFFFF).  A tile whose survivors do not fit -- or, with
// 8-bit codes, that holds a window past the text end; with 2- and 4-bit
// codes, any tile but an interior one of keyword bytes only -- is resolved
// by its warp as in the one-phase form.  The walk list has room for one walk
// per listed survivor plus a chunk per warp of step 2 (a warp leaves entries
// unused only in its last chunk), so every walk fits.
constexpr uint32_t kWalkChunkEntries = 64;   // walk-list entries a warp of step 2 reserves at a time
constexpr uint32_t kSurvWarpsPerSm = 48;     // most warps of step 2 resident on one SM
uint32_t device_sm_count();                  // of the current device (cached; 0 on error)
struct Tuning;
// Whether the filter kernel takes the phased form for a text of n bytes
// (filter.cu): 8-bit codes from 4 MiB on; 2- and 4-bit codes, when the
// tuning asks for it or, for dense ids and counts (not slots), when the
// automaton prefers it (list_prefer), beyond the texts short enough for the
// forms that share heavy tiles within the CTA.  Never for texts of more
// tiles than the entries can name, nor when the tuning says never.  (Listed
// units keep no dense fallback, and the sets that prefer listing have tiles
// of many matches, which the gather would then match again.)
bool filter_phased(const DevTables &t, const Tuning &tu, uint64_t n, bool slots = false);
struct SurvivorLists {
    uint32_t list_cap = 0, walk_cap = 0;
    size_t bytes() const { return list_cap ? 32 + 16ull * list_cap + 8ull * walk_cap : 0; }
};
// The lists of a text of n bytes (none: the one-phase form).  Scratch
// layout: two counters (32 bytes, zeroed) | list_cap uint4 | walk_cap uint2.
inline SurvivorLists survivor_lists(const DevTables &t, const Tuning &tu, uint64_t n, bool slots = false) {
    SurvivorLists s;
    if (!filter_phased(t, tu, n, slots)) return s;
    const uint64_t sms = device_sm_count();
    if (sms == 0) return s;
    s.list_cap = static_cast<uint32_t>(n / 8);  // 12.5 % of the positions
    s.walk_cap = static_cast<uint32_t>(s.list_cap + sms * kSurvWarpsPerSm * kWalkChunkEntries);
    return s;
}
inline void set_lists(MatchRequest &r, void *scratch, const SurvivorLists &s) {
    uint8_t *b = static_cast<uint8_t *>(scratch);
    r.list_count = reinterpret_cast<unsigned int *>(b);
    r.list = reinterpret_cast<uint4 *>(b + 32);
    r.list_cap = s.list_cap;
    r.walks = reinterpret_cast<uint2 *>(b + 32 + 16ull * s.list_cap);
    r.walk_cap = s.walk_cap;
}


struct Tuning {
    int block = 0;        // threads per CTA (multiple of 32, <= 640; 0 = the kernel's choice:
                          // 640 for the one-phase single-text filter forms of 2- and
                          // 4-bit codes, 512 elsewhere; above 512 only those forms)
    int stages = 0;       // text stages in flight per warp (2..4, 0 = the kernel's default;
                          // fewer when shared memory is short)
    int grid = 0;         // 0 = one CTA per SM
    int variant = 0;      // 8-bit codes: 1 = warp tiles with walk slots (kernels.cu),
                          // 2 = one thread per position with the jump table in shared
                          // memory (jump8.cu), 0 or 3 = the same at full occupancy with
                          // the table read through L1 (the default)
    int per_thread = 0;   // 8-bit codes, long texts: survivors a thread of the second
                          // step takes at a time (2, or 4 with fewer threads; 0 = 2)
    int halo = 0;         // bytes staged after each tile: 0 = the 16 the filter reads,
                          // or up to kHaloCap (a wider halo reaches L2 ahead of the walks)
    int survivor_list = 0;  // long single texts: 0 = the phased form for 8-bit codes and for
                            // small alphabets with list_prefer, 1 = for every code width, 2 = never
    unsigned long long wait_ns = 0;  // bounded waits give up after this (0 = kWaitNs)
    int stall_help = 0;   // test aid: owners wait for one chunk more than their heavy tile has
};

// The scan and gather steps of the compacted output (compact.cu).
//   units: launch units (host count), or, when units_dev is set, read there.
//   partials: kScanCtas words of scratch.
constexpr uint32_t kScanCtas = 256;
cudaError_t launch_compact_scan(const uint32_t *counts, uint32_t units, const uint32_t *units_dev,
                                unsigned long long *prefix, unsigned long long *partials, cudaStream_t stream);
// Gather: for every unit of one automaton's launch (one text, or the planned
// list of a batch with per-text outputs outs[item]), its matches in ascending
// position at its place in its text's list; *count of each text from its last
// unit.  tile = positions per unit.
struct GatherRequest {
    const uint8_t *text = nullptr;           // one text (or batch base)
    uint64_t n = 0;
    CompactOut out{};                        // one text
    const BatchHead *batch = nullptr;        // batch
    const BatchItemDev *lists = nullptr;
    const CompactOut *outs = nullptr;        // batch: per caller item
    uint32_t units = 0;                      // one text: its units
    uint32_t tile = 0;
    const uint32_t *counts = nullptr;
    const unsigned long long *prefix = nullptr;
    const unsigned long long *slots = nullptr;
    const int32_t *dense = nullptr;          // optional, as SlotOut::dense
    uint32_t ubase = 0;
};
cudaError_t launch_compact_gather(const DevTables &t, const GatherRequest &g, cudaStream_t stream);

// The whole compacted match of one text (slot-mode matching kernel, scan,
// gather) on `stream`, with `scratch` of compact_scratch_bytes(t, units, dense)
// bytes (cleared here), units = compact_units(t, text, n).  dense: keep the
// per-unit dense fallback (4 bytes per position) so that units with many
// matches are copied, not matched again.
uint32_t compact_units(const DevTables &t, const Tuning &tu, const uint8_t *text, uint64_t n);
size_t compact_scratch_bytes(const DevTables &t, uint32_t units, bool dense);
cudaError_t enqueue_compact(const DevTables &t, const Tuning &tu, const uint8_t *text, uint64_t n,
                            const CompactOut &out, void *scratch, size_t scratch_bytes, bool dense,
                            cudaStream_t stream);
// Byte offset of the dense fallback in that scratch (16-byte aligned).
// Layout: tile counter (16) | counts (4 per unit) | prefix (8 per unit) |
// slots (8 * kSlotCap per unit) | partial sums (8 * kScanCtas) | dense
// fallback (4 per position of every unit, optional).
constexpr size_t round16c(size_t v) { return (v + 15u) & ~static_cast<size_t>(15u); }
constexpr size_t compact_dense_offset(uint64_t units) {
    return round16c(16 + round16c(4 * units) + 8 * units + 8 * static_cast<size_t>(kSlotCap) * units +
                    8 * static_cast<size_t>(kScanCtas));
}
// Fewest positions per work unit of any matching kernel (the filter kernel's
// tile); a text of n bytes at any alignment has at most
// (n + 15 + kMinTile - 1) / kMinTile units.
constexpr uint32_t kMinTile = 992;

// Full output of one text (full.cu): every keyword occurrence as (end, id)
// into out.pos / out.ids, ordered by start, end, id; the slot-mode matching
// kernel, per-unit occurrence counts, their scan, and the expansion.  Scratch:
// full_scratch_bytes(t, tu, units, n) bytes, units = compact_units(t, tu,
// text, n) (with the phased form's lists when the text takes that form).
size_t full_scratch_bytes(const DevTables &t, const Tuning &tu, uint32_t units, uint64_t n);
cudaError_t enqueue_full(const DevTables &t, const Tuning &tu, const uint8_t *text, uint64_t n,
                         const CompactOut &out, void *scratch, size_t scratch_bytes, cudaStream_t stream);

// 8-bit-code kernel (kernels.cu).  Modes: dense, count, slots; 16 bytes of
// zeroed scratch (tile counter).
cudaError_t launch_tiled(const DevTables &t, const MatchRequest &r, OutMode mode,
                         const Tuning &tu, cudaStream_t stream);
cudaError_t launch_simple(const DevTables &t, const MatchRequest &r, cudaStream_t stream);

// The library's stream-ordered pool for per-call scratch on device `dev`.
cudaError_t scratch_pool(int dev, cudaMemPool_t *out);

// Device address of the static scratch of ac_match_compact_static on device
// `dev` (the current device); the first call on a device loads the module that
// holds the array, which commits its memory (noalloc.cu).
cudaError_t static_scratch_address(int dev, void **out);

// Handle internals for entry points outside api.cpp.
const DevTables *handle_tables(ac_handle h, int *device, bool *host_only);
const Tuning *handle_tuning(ac_handle h);

// Read and clear the device error word of the current device.
cudaError_t read_device_error(unsigned int *value);

// Device address of the current device's kernel error word.
cudaError_t device_error_word(unsigned int **ptr);

// Batch planning (batch.cu): from the caller's item list (device), one
// BatchHead per automaton and the non-empty texts of each automaton in item
// order with their first work unit.  tile_len: host array of nh entries, the
// dense tile length of each automaton's kernel (filter_tile_positions or
// tiled_tile_positions).  An item whose automaton is >= nh, or an automaton
// with 2^32 or more units, latches kErrBatchItem.
constexpr uint32_t kMaxBatchAutomata = 256;
cudaError_t launch_batch_plan(const ac_batch_item *items, uint32_t nitems, uint32_t nh, const uint8_t *texts,
                              const uint32_t *tile_len, BatchHead *heads, BatchItemDev *lists, cudaStream_t stream);

// Filter-mode kernel (2- and 4-bit codes; 8-bit codes with the hashed
// filter), in filter.cu.  Modes: dense, count, slots.  Every launch takes 16
// bytes of zeroed scratch (tile counter).
cudaError_t launch_filter(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                          cudaStream_t stream);
// Positions per work unit (tile) of the dense filter kernel and of the dense
// 8-bit kernels: the tile lengths a batch is planned with.
uint32_t filter_tile_positions();
uint32_t tiled_tile_positions();

// The filter kernel serves an automaton: always for 2- and 4-bit codes; for
// 8-bit codes (hashed filter) unless another kernel was chosen (Tuning::variant).
inline bool uses_filter(const DevTables &t, const Tuning &tu) { return t.filter || (t.hashed && tu.variant == 0); }
// Positions per work unit of the kernel that serves the automaton.
inline uint32_t unit_positions(const DevTables &t, const Tuning &tu) {
    return uses_filter(t, tu) ? filter_tile_positions() : tiled_tile_positions();
}
// A batch of nh automata in one persistent launch of the filter kernel
// (filter.cu): whether it serves them all (every automaton has a root filter
// and nh is small enough for the launch's parameters), and the launch.  rs[a]:
// automaton a's request (batch head, planned list, its tile counter as
// scratch, dense output or slots).  Every automaton runs the filter kernel,
// whatever kernel its tuning names for single texts.  lists (optional, null:
// none): scratch of multi_lists_bytes(list_cap) bytes whose first 32 are
// zeroed, for the phased form of the batch's 8-bit-code automata: their
// survivors go to one list of up to list_cap entries (tiles past that are
// resolved in their warps), resolved by a second launch and a third for the
// walks.  With slot output the units then keep no dense fallback (the gather
// matches a unit with more matches than slots again).
bool filter_multi_serves(const DevTables *const *ts, uint32_t nh);
size_t multi_lists_bytes(uint32_t list_cap);
cudaError_t launch_filter_multi(const DevTables *const *ts, const MatchRequest *rs, uint32_t nh, OutMode mode,
                                unsigned long long wait_ns, cudaStream_t stream, void *lists = nullptr,
                                uint32_t list_cap = 0);

// A matching launch on the kernel that serves the automaton.
inline cudaError_t launch_match(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                                cudaStream_t stream) {
    return uses_filter(t, tu) ? launch_filter(t, r, mode, tu, stream) : launch_tiled(t, r, mode, tu, stream);
}

// One-thread-per-position 8-bit kernel (jump8.cu); same modes, scratch and
// tile length as launch_tiled, which hands over to it for Tuning::variant 2.
// global: the full-occupancy form that reads the jump table and the text
// through L1 (Tuning::variant 3).
cudaError_t launch_jump8(const DevTables &t, const MatchRequest &r, OutMode mode, bool global,
                         unsigned long long wait_ns, cudaStream_t stream);

}  // namespace pfac
