// Failureless Aho-Corasick matching with a root filter, sm_103a: the launcher
// (2- and 4-bit codes with the exact filter, 8-bit codes with the hashed
// filter and state hash).  The kernel is in filter_kernel.cuh.
#include "filter_kernel.cuh"

namespace pfac {

using namespace filt;

uint32_t filter_tile_positions() { return kTile; }

cudaError_t launch_filter(const DevTables &t, const MatchRequest &r, OutMode mode, const Tuning &tu,
                          cudaStream_t stream) {
    if (tu.block < 32 || tu.block > kMaxBlock || (tu.block & 31) || (tu.stages != 0 && tu.stages < 2) ||
        tu.stages > kMaxStages)
        return cudaErrorInvalidValue;
    const bool hashed = t.B == 8 && t.hashed && t.HK != nullptr;
    if (!((t.B == 2 || t.B == 4) && t.filter) && !hashed) return cudaErrorInvalidValue;
    if (mode != OUT_DENSE && mode != OUT_COUNT && mode != OUT_SLOTS) return cudaErrorInvalidValue;
    const bool batch = r.batch != nullptr;
    if (batch && (mode == OUT_COUNT || !r.lists)) return cudaErrorInvalidValue;
    if (mode == OUT_SLOTS && (!r.slots.counts || !r.slots.slots)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    FilterParams p{};
    p.text = r.text;
    p.n = r.n;
    p.tile = kTile;
    const uint32_t H = t.maxlen < kHaloCap ? t.maxlen : kHaloCap;
    p.staged = align16(kTile + H) > align16(kTile + 16) ? align16(kTile + H) : align16(kTile + 16);
    uint64_t tiles = 0;
    if (!batch) {
        const uint64_t head = reinterpret_cast<uintptr_t>(r.text) & 15u;
        tiles = (r.n + head + kTile - 1) / kTile;
        if (tiles >= 0x7FFFFFFFull) return cudaErrorInvalidValue;
    }
    p.ntiles = static_cast<uint32_t>(tiles);
    if (!batch) {
        const uint64_t head = reinterpret_cast<uintptr_t>(r.text) & 15u;
        p.gbase = r.text - head;
        p.a1 = (head + 15u) & ~15ull;
        p.a2 = (head + r.n) & ~15ull;
        p.vec_ok = ((reinterpret_cast<uintptr_t>(r.out) - 4u * head) & 15u) == 0 ? 1u : 0u;
    }
    p.batch = r.batch;
    p.lists = r.lists;
    // per-warp layout: stages, packed codes, unknown-byte bits, survivor
    // queue, stage descriptors; a CTA-wide -1 buffer for the bulk stores
    const uint32_t packed_bytes = align16(kCodeSpan * t.B / 8 + 16);
    const uint32_t inv_bytes = align16(kCodeSpan / 8 + 16);
    const uint32_t queue_bytes = align16(kTile * 2);
    const uint32_t neg1_bytes = kTile * 4;
    const uint32_t nw = static_cast<uint32_t>(tu.block) / 32u;
    uint32_t smem = 0;
    bool fits = false;
    const int want = tu.stages ? tu.stages : 3;
    for (int st = want; st >= 2 && !fits; --st) {
        p.nstages = static_cast<uint32_t>(st);
        p.off_packed = p.nstages * p.staged;
        p.off_inv = p.off_packed + packed_bytes;
        p.off_queue = p.off_inv + inv_bytes;
        p.off_meta = p.off_queue + queue_bytes;
        p.off_help = p.off_meta + 16u;
        p.warp_bytes = p.off_help + align16(static_cast<uint32_t>(sizeof(HelpSlot)));
        p.off_neg1 = align16(kOffF + t.fbytes);
        p.off_warp = align16(p.off_neg1 + neg1_bytes);
        smem = p.off_warp + nw * p.warp_bytes;
        fits = static_cast<int>(smem) <= max_smem;
    }
    if (!fits) return cudaErrorInvalidConfiguration;
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
    p.skip = t.skip;
    p.chain = t.chain;
    p.s_chain = t.skip ? t.s_chain : 0xFFFFFFFFu;
    p.wait_ns = tu.wait_ns ? tu.wait_ns : kWaitNs;
    p.stall_help = tu.stall_help ? 1u : 0u;
    p.hash_shift = t.hash_shift;
    p.hcode_lo = t.hash_code[0];
    p.hcode_hi = t.hash_code[1];
    p.hbyte_lo = t.hash_byte[0];
    p.hbyte_hi = t.hash_byte[1];
    p.out = r.out;
    p.count = r.count;
    p.sl = r.slots;
    // the tile counter; none is needed when every tile is some warp's first
    p.counter = r.scratch && r.scratch_bytes >= 16 ? static_cast<unsigned int *>(r.scratch) : nullptr;
    e = device_error_word(&p.err);
    if (e != cudaSuccess) return e;
    uint32_t grid = tu.grid > 0 ? static_cast<uint32_t>(tu.grid) : static_cast<uint32_t>(sms);
    if (!batch) {  // a batch's units are counted on the device: every CTA starts
        const uint32_t need_ctas = (p.ntiles + nw - 1) / nw;
        if (grid > need_ctas) grid = need_ctas;
    }
    if (!p.counter && (batch || static_cast<uint64_t>(p.ntiles) > static_cast<uint64_t>(grid) * nw))
        return cudaErrorInvalidValue;
    if (grid == 0) return cudaSuccess;
    // a text short next to the grid: its heavy tiles (many survivors, long
    // walks) would be one warp's work each while most warps have run out of
    // tiles, so those forms share them within the CTA (small alphabets)
    if (!batch && t.B <= 4 &&
        static_cast<uint64_t>(p.ntiles) <= static_cast<uint64_t>(kHelpTilesPerWarp) * grid * nw)
        return launch_filter_help(mode, p, t.B, t.gbits, grid, tu.block, smem, max_smem, stream);
    if (t.B == 8) return launch_filter8(mode, p, t.gbits, grid, tu.block, smem, max_smem, stream);
    if (t.B == 2) {
        if (t.gbits == 16) return launch_modes<2, int16_t, false>(mode, p, grid, tu.block, smem, max_smem, stream);
        return launch_modes<2, int32_t, false>(mode, p, grid, tu.block, smem, max_smem, stream);
    }
    if (t.gbits == 16) return launch_modes<4, int16_t, false>(mode, p, grid, tu.block, smem, max_smem, stream);
    return launch_modes<4, int32_t, false>(mode, p, grid, tu.block, smem, max_smem, stream);
}

}  // namespace pfac
