// Failureless Aho-Corasick matching with a root filter, sm_103a: the launchers
// (2- and 4-bit codes with the exact filter, 8-bit codes with the hashed
// filter and state hash; one text, one automaton's batch texts, or a whole
// batch of automata in one launch).  The kernel is in filter_kernel.cuh.
#include <mutex>

#include "filter_kernel.cuh"

namespace pfac {

using namespace filt;

uint32_t filter_tile_positions() { return kTile; }

namespace {

bool served(const DevTables &t) { return ((t.B == 2 || t.B == 4) && t.filter) || (t.B == 8 && t.hashed && t.HK); }

// Bytes staged per tile: the tile and the 16 bytes after it (the windows'
// look-ahead; kCodeSpan positions are classified), or a wider halo (tuning:
// up to kHaloCap bytes, at most the longest keyword).  The filter reads no
// further; a walk past the classified span reads its bytes through L1/L2,
// where a wider halo has brought them.
uint32_t staged_bytes(const DevTables &t, const Tuning &tu) {
    uint32_t h = tu.halo > 16 ? static_cast<uint32_t>(tu.halo) : 16u;
    if (h > kHaloCap) h = kHaloCap;
    if (h > t.maxlen && t.maxlen > 16) h = t.maxlen;
    return align16(kTile + h);
}

// The launch parameters of automaton t and request r, all but the shared-
// memory layout.
cudaError_t fill_params(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu, FilterParams &p) {
    if (!served(t)) return cudaErrorInvalidValue;
    const bool hashed = t.B == 8;
    if (mode != OUT_DENSE && mode != OUT_COUNT && mode != OUT_SLOTS) return cudaErrorInvalidValue;
    const bool batch = r.batch != nullptr;
    if (batch && (mode == OUT_COUNT || !r.lists)) return cudaErrorInvalidValue;
    if (mode == OUT_SLOTS && (!r.slots.counts || !r.slots.slots)) return cudaErrorInvalidValue;
    p = FilterParams{};
    p.text = r.text;
    p.n = r.n;
    p.tile = kTile;
    p.staged = staged_bytes(t, tu);
    uint64_t tiles = 0;
    if (!batch) {
        const uint64_t head = reinterpret_cast<uintptr_t>(r.text) & 15u;
        tiles = (r.n + head + kTile - 1) / kTile;
        if (tiles >= 0x7FFFFFFFull) return cudaErrorInvalidValue;
        p.gbase = r.text - head;
        p.a1 = (head + 15u) & ~15ull;
        p.a2 = (head + r.n) & ~15ull;
        p.vec_ok = ((reinterpret_cast<uintptr_t>(r.out) - 4u * head) & 15u) == 0 ? 1u : 0u;
    }
    p.ntiles = static_cast<uint32_t>(tiles);
    p.batch = r.batch;
    p.lists = r.lists;
    p.G = t.G;
    p.Fg = t.F;
    p.JK = t.JK;
    p.J2 = t.J2;
    p.cls8g = t.cls8;
    p.C = t.C;
    p.W = t.W;
    p.k = hashed ? t.kh : t.k;
    p.k2 = hashed ? 0u : t.k2;
    p.base_k = t.base_k;
    p.maxlen = t.maxlen;
    p.fbytes = t.fbytes;
    {
        // filter index bits: the window's (windows below 32 bits are
        // replicated to 32), or the hash's
        const uint32_t wb = hashed ? t.fbits : t.B * t.k;
        const uint32_t nb = (wb >= 5 ? (1u << wb) : 32u) / 8u;
        if (nb > t.fbytes || (hashed && (t.fbits < 5 || t.fbits > 31 || t.kh < 1 || t.kh > kHashWindow)))
            return cudaErrorInvalidValue;
        p.famask = (nb - 1u) & ~3u;
    }
    p.identity = t.C >= 256 ? 1u : 0u;
    p.wmask = hashed ? (t.kh >= 4 ? 0xFFFFFFFFu : (1u << (8u * t.kh)) - 1u) : 0u;
    p.fshift = hashed ? 32u - t.fbits : 0u;
    p.HK = hashed ? t.HK : nullptr;
    p.hk_shift = hashed ? 32u - t.hk_bits : 0u;
    p.hk_mask = hashed ? (1u << t.hk_bits) - 1u : 0u;
    p.hk_probes = hashed ? t.hk_probes : 0u;
    p.wait_ns = tu.wait_ns ? tu.wait_ns : kWaitNs;
    p.stall_help = tu.stall_help ? 1u : 0u;
    p.kind = filter_kind(t.B, t.gbits);
    p.skip = t.skip;
    p.chain = t.chain;
    p.s_chain = t.skip ? t.s_chain : 0xFFFFFFFFu;
    p.hash_shift = t.hash_shift;
    p.hcode_lo = t.hash_code[0];
    p.hcode_hi = t.hash_code[1];
    p.hbyte_lo = t.hash_byte[0];
    p.hbyte_hi = t.hash_byte[1];
    p.direct_shift = t.B == 2 ? t.direct_shift : -1;
    p.dsel_lo = t.direct_sel[0];
    p.dsel_hi = t.direct_sel[1];
    p.dfill = t.direct_fill;
    p.out = r.out;
    p.count = r.count;
    p.sl = r.slots;
    if (!batch && r.list && r.list_count && r.list_cap && p.ntiles < (1u << 22)) {
        p.list = r.list;
        p.list_count = r.list_count;
        p.list_cap = r.list_cap;
        p.walks = r.walks;
        p.walk_cap = r.walks ? r.walk_cap : 0u;
    }
    // the tile counter; none is needed when every tile is some warp's first
    p.counter = r.scratch && r.scratch_bytes >= 16 ? static_cast<unsigned int *>(r.scratch) : nullptr;
    return device_error_word(&p.err);
}

// The shared-memory layout of a launch of nw warps whose automata stage up to
// `staged` bytes per tile, take up to B bits per code and have filters of up
// to fbytes: per warp the stages, packed codes, unknown-byte bits, survivor
// queue, stage descriptors and help slot; a CTA-wide -1 buffer for the bulk
// stores.  The most stages (want, down to 2) that fit max_smem; false if none.
bool layout(FilterParams &p, uint32_t staged, uint32_t B, uint32_t fbytes, uint32_t nw, int want, int max_smem,
            uint32_t *smem) {
    const uint32_t packed_bytes = align16(kCodeSpan * B / 8 + 16);
    const uint32_t inv_bytes = align16(kCodeSpan / 8 + 16);
    const uint32_t queue_bytes = align16(kTile * 2);
    const uint32_t neg1_bytes = kTile * 4;
    for (int st = want; st >= 2; --st) {
        p.nstages = static_cast<uint32_t>(st);
        p.off_packed = p.nstages * staged;
        p.off_inv = p.off_packed + packed_bytes;
        p.off_queue = p.off_inv + inv_bytes;
        p.off_meta = p.off_queue + queue_bytes;
        p.off_help = p.off_meta + 16u;
        p.warp_bytes = p.off_help + align16(static_cast<uint32_t>(sizeof(HelpSlot)));
        p.off_neg1 = align16(kOffF + fbytes);
        p.off_warp = align16(p.off_neg1 + neg1_bytes);
        *smem = p.off_warp + nw * p.warp_bytes;
        if (static_cast<int>(*smem) <= max_smem) return true;
    }
    return false;
}

struct DeviceShape {
    int sms = 0;
    int max_smem = 0;
};

cudaError_t device_shape(DeviceShape *out) {
    static DeviceShape cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cache[dev].sms == 0) {
        DeviceShape d;
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        cache[dev] = d;
    }
    *out = cache[dev];
    return cudaSuccess;
}

}  // namespace

bool filter_phased(const DevTables &t, const Tuning &tu, uint64_t n, bool slots) {
    if (!served(t) || n / kTile >= (1ull << 22) - 1 || tu.survivor_list == 2) return false;
    if (t.B == 8) return n >= (4ull << 20);
    if (tu.survivor_list != 1 && (slots || !t.list_prefer)) return false;
    // small alphabets: beyond the texts that take the forms sharing heavy
    // tiles within the CTA (the launcher's test, with the most tiles the
    // text's alignment can give)
    const uint64_t sms = device_sm_count();
    if (sms == 0) return false;
    // the launcher's test for the forms that share heavy tiles (at most 512 threads)
    const uint64_t grid = tu.grid > 0 ? static_cast<uint64_t>(tu.grid) : sms;
    const uint64_t nw = static_cast<uint64_t>(tu.block > 0 && tu.block < kStdBlock ? tu.block : kStdBlock) / 32;
    return n / kTile > static_cast<uint64_t>(kHelpTilesPerWarp) * grid * nw;
}

uint32_t device_sm_count() {
    DeviceShape ds;
    if (device_shape(&ds) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return static_cast<uint32_t>(ds.sms);
}

cudaError_t launch_filter(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                          cudaStream_t stream) {
    if (tu.block < 0 || tu.block > kMaxBlock || (tu.block & 31) || (tu.stages != 0 && tu.stages < 2) ||
        tu.stages > kMaxStages)
        return cudaErrorInvalidValue;
    DeviceShape ds;
    cudaError_t e = device_shape(&ds);
    if (e != cudaSuccess) return e;
    FilterParams p;
    e = fill_params(t, r, mode, tu, p);
    if (e != cudaSuccess) return e;
    const bool batch = r.batch != nullptr;
    const uint32_t grid0 = tu.grid > 0 ? static_cast<uint32_t>(tu.grid) : static_cast<uint32_t>(ds.sms);
    // a text short next to the grid: its heavy tiles (many survivors, long
    // walks) would be one warp's work each while most warps have run out of
    // tiles, so those forms share them within the CTA (small alphabets; the
    // phased form lists heavy tiles like any other)
    const uint32_t nw_std = static_cast<uint32_t>(tu.block > 0 && tu.block < kStdBlock ? tu.block : kStdBlock) / 32u;
    const bool help = !batch && t.B <= 4 && !p.list &&
                      static_cast<uint64_t>(p.ntiles) <= static_cast<uint64_t>(kHelpTilesPerWarp) * grid0 * nw_std;
    // threads per CTA: the tuning's (0: 640 for the one-phase single-text
    // forms of 2- and 4-bit codes, 512 elsewhere); the other forms run at
    // most 512
    const bool wide_form = t.B <= 4 && !batch && !help && !p.list;
    uint32_t block = tu.block > 0 ? static_cast<uint32_t>(tu.block) : (wide_form ? kMaxBlock : kStdBlock);
    if (!wide_form && block > static_cast<uint32_t>(kStdBlock)) block = kStdBlock;
    const uint32_t nw = block / 32u;
    uint32_t smem = 0;
    if (!layout(p, p.staged, t.B, t.fbytes, nw, tu.stages ? tu.stages : 3, ds.max_smem, &smem))
        return cudaErrorInvalidConfiguration;
    uint32_t grid = grid0;
    if (!batch) {  // a batch's units are counted on the device: every CTA starts
        const uint32_t need_ctas = (p.ntiles + nw - 1) / nw;
        if (grid > need_ctas) grid = need_ctas;
    }
    if (!p.counter && (batch || static_cast<uint64_t>(p.ntiles) > static_cast<uint64_t>(grid) * nw))
        return cudaErrorInvalidValue;
    if (grid == 0) return cudaSuccess;
    if (help) return launch_filter_help(mode, p, t.B, t.gbits, grid, block, smem, ds.max_smem, stream);
    if (t.B == 8)
        e = launch_filter8(mode, p, t.gbits, grid, block, smem, ds.max_smem, stream);
    else if (t.B == 2)
        e = t.gbits == 16 ? launch_modes<2, int16_t, false>(mode, p, grid, block, smem, ds.max_smem, stream)
                          : launch_modes<2, int32_t, false>(mode, p, grid, block, smem, ds.max_smem, stream);
    else
        e = t.gbits == 16 ? launch_modes<4, int16_t, false>(mode, p, grid, block, smem, ds.max_smem, stream)
                          : launch_modes<4, int32_t, false>(mode, p, grid, block, smem, ds.max_smem, stream);
    if (e == cudaSuccess && p.list)
        e = launch_survivors(mode, p, t.B, t.gbits, static_cast<uint32_t>(ds.sms), tu.per_thread, stream);
    return e;
}

bool filter_multi_serves(const DevTables *const *ts, uint32_t nh) {
    if (nh == 0 || nh > kMultiMax) return false;
    for (uint32_t a = 0; a < nh; ++a)
        if (!served(*ts[a])) return false;
    return true;
}

size_t multi_lists_bytes(uint32_t list_cap) {
    const uint64_t walk_cap = static_cast<uint64_t>(list_cap) + static_cast<uint64_t>(device_sm_count()) *
                                                                    kSurvWarpsPerSm * kWalkChunkEntries;
    return 32 + 16ull * list_cap + 16ull * walk_cap;
}

cudaError_t launch_filter_multi(const DevTables *const *ts, const MatchRequest *rs, uint32_t nh, OutMode mode,
                                unsigned long long wait_ns, cudaStream_t stream, void *lists, uint32_t list_cap) {
    if (!filter_multi_serves(ts, nh) || (mode != OUT_DENSE && mode != OUT_SLOTS)) return cudaErrorInvalidValue;
    DeviceShape ds;
    cudaError_t e = device_shape(&ds);
    if (e != cudaSuccess) return e;
    // 11 KiB of parameters: kept off the stack, filled and launched under a lock
    static MultiParams mp;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    mp.nh = nh;
    uint32_t staged = 0, B = 0, fbytes = 0;
    Tuning tu;
    tu.wait_ns = wait_ns;
    // the phased form's lists, when given
    mp.list = nullptr;
    mp.list_count = nullptr;
    mp.list_cap = mp.walk_cap = 0;
    mp.walks4 = nullptr;
    // the automata that list: 8-bit codes, and small alphabets that prefer it;
    // with slots only those without a dense fallback (the listed survivors
    // write none of it: the gather matches an overflowing unit again)
    auto lists_for = [&](uint32_t a) {
        return (ts[a]->B == 8 || ts[a]->list_prefer) && (mode == OUT_DENSE || !rs[a].slots.dense);
    };
    bool listed = false;
    for (uint32_t a = 0; a < nh; ++a) listed = listed || lists_for(a);
    if (lists && list_cap && listed) {
        uint8_t *b = static_cast<uint8_t *>(lists);
        mp.list_count = reinterpret_cast<unsigned int *>(b);
        mp.list = reinterpret_cast<uint4 *>(b + 32);
        mp.list_cap = list_cap;
        mp.walks4 = reinterpret_cast<uint4 *>(b + 32 + 16ull * list_cap);
        mp.walk_cap = static_cast<uint32_t>((multi_lists_bytes(list_cap) - 32 - 16ull * list_cap) / 16);
    }
    for (uint32_t a = 0; a < nh; ++a) {
        if (!rs[a].batch || !rs[a].lists || !rs[a].scratch || rs[a].scratch_bytes < 16) return cudaErrorInvalidValue;
        e = fill_params(*ts[a], rs[a], mode, tu, mp.a[a]);
        if (e != cudaSuccess) return e;
        mp.a[a].aidx = a;
        if (mp.list && lists_for(a)) {
            mp.a[a].list = mp.list;
            mp.a[a].list_count = mp.list_count;
            mp.a[a].list_cap = mp.list_cap;
            mp.a[a].walks4 = mp.walks4;
            mp.a[a].walk_cap = mp.walk_cap;
        }
        staged = staged > mp.a[a].staged ? staged : mp.a[a].staged;
        B = B > ts[a]->B ? B : ts[a]->B;
        fbytes = fbytes > ts[a]->fbytes ? fbytes : ts[a]->fbytes;
    }
    // one layout for all: the largest stages, codes and filter; the active
    // automaton's parameters after it
    FilterParams shape{};
    uint32_t smem = 0;
    const uint32_t pbytes = align16(static_cast<uint32_t>(sizeof(FilterParams)));
    if (!layout(shape, staged, B, fbytes, kMultiBlock / 32, 3, ds.max_smem - static_cast<int>(pbytes), &smem))
        return cudaErrorInvalidConfiguration;
    mp.params_off = smem;
    smem += pbytes;
    for (uint32_t a = 0; a < nh; ++a) {
        FilterParams &p = mp.a[a];
        p.nstages = shape.nstages;
        p.off_packed = shape.off_packed;
        p.off_inv = shape.off_inv;
        p.off_queue = shape.off_queue;
        p.off_meta = shape.off_meta;
        p.off_help = shape.off_help;
        p.warp_bytes = shape.warp_bytes;
        p.off_neg1 = shape.off_neg1;
        p.off_warp = shape.off_warp;
    }
    return launch_filter_multi_modes(mode, mp, static_cast<uint32_t>(ds.sms), smem, ds.max_smem, stream);
}

}  // namespace pfac
