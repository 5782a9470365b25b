// Device building blocks of the failureless Aho-Corasick kernels (sm_103a).
//
// The walk (paper section II, Fig. 5; section I, Fig. 3): every text position
// starts at the root of the goto-only machine, follows the transitions of the
// bytes that follow it and stops at the first missing transition; the result
// is the longest keyword on the path (encoded in the dead entry where it
// stops, or in the row's end column when the text or an unknown byte ends it).
#pragma once

#include <cstdint>

#include "pfac_internal.h"

namespace pfac {


// Every bounded wait gives up after this many nanoseconds of %globaltimer
// unless the launch names another limit (ac_set_wait_limit).
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier + bulk async copy (TMA unit, 1-D, no multicast) --------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// L2 eviction policies: streamed data (the text) leaves L2 first, the hot
// rows of the goto table stay.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bulk_load with an L2 eviction policy.
__device__ __forceinline__ void bulk_load_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                               uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Shared -> global bulk copy (bulk-group completion); dst, src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Wait until all but the 8 most recent bulk-store groups have read shared memory.
__device__ __forceinline__ void bulk_wait_read_keep8() {
    asm volatile("cp.async.bulk.wait_group.read 8;" ::: "memory");
}

// Wait until every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for a phase with a time limit (ns of %globaltimer); false when the
// limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer() - t0 > limit) return false;
    }
}

__device__ __forceinline__ int decode_dead(int e) { return -e - 2; }

// The text a work unit (one tile) belongs to.  The text is gbase + head with
// gbase 16-byte aligned; tile t covers text positions [t * tile_len - head,
// (t + 1) * tile_len - head) and stages bytes [t * tile_len, t * tile_len +
// staged) of gbase, the part of them inside the text.
struct TileText {
    const uint8_t *text;   // first byte of the text
    const uint8_t *gbase;  // text rounded down to 16 bytes
    int32_t *out;          // its dense ids (out[i] for text position i)
    uint64_t n;            // its length
    uint32_t head;         // text - gbase
    uint32_t tile;         // the unit's tile within the text
    uint32_t vec_ok;       // out - 4 * head is 16-byte aligned (tiles store 16-byte groups)
};

__device__ __forceinline__ TileText make_text(const uint8_t *text, int32_t *out, uint64_t n, uint32_t tile) {
    TileText t;
    t.text = text;
    t.head = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(text) & 15u);
    t.gbase = text - t.head;
    t.out = out;
    t.n = n;
    t.tile = tile;
    t.vec_ok = ((reinterpret_cast<uintptr_t>(out) - 4u * t.head) & 15u) == 0 ? 1u : 0u;
    return t;
}

// Where a launch's work units come from: the tiles of one text (list ==
// nullptr), or the tiles of a batch's texts (the planned list of one
// automaton, ascending in first_unit).
struct Work {
    uint32_t units;
    uint32_t nlist;
    const BatchItemDev *list;
};

__device__ __forceinline__ Work load_work(const BatchHead *head, const BatchItemDev *lists, uint32_t single_units) {
    Work w;
    if (!head) {
        w.units = single_units;
        w.nlist = 0;
        w.list = nullptr;
        return w;
    }
    const uint4 h = __ldg(reinterpret_cast<const uint4 *>(head));
    w.units = h.x;
    w.nlist = h.y;
    w.list = lists + h.z;
    return w;
}

// The batch text of entry `item` of the planned list, for its unit u.
__device__ __forceinline__ TileText batch_text(const Work &wk, const uint8_t *texts, int32_t *outs, uint32_t item,
                                               uint32_t u) {
    const uint4 *e = reinterpret_cast<const uint4 *>(wk.list + item);
    const uint4 a = __ldg(e), b = __ldg(e + 1);
    const uint64_t text_off = static_cast<uint64_t>(a.x) | (static_cast<uint64_t>(a.y) << 32);
    const uint64_t len = static_cast<uint64_t>(a.z) | (static_cast<uint64_t>(a.w) << 32);
    const uint64_t out_off = static_cast<uint64_t>(b.x) | (static_cast<uint64_t>(b.y) << 32);
    return make_text(texts + text_off, outs + out_off, len, u - b.z);
}

// All lanes of a warp, u warp-uniform: the index of the last entry of the
// planned list whose first_unit <= u, i.e. the text that unit u belongs to
// (list[0].first_unit == 0; empty texts are not in the list).  32 entries are
// sampled per round, so three rounds cover 32768 texts.
__device__ __forceinline__ uint32_t find_item(const Work &wk, uint32_t u, int lane) {
    uint32_t lo = 0, hi = wk.nlist;
    while (hi - lo > 32u) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t idx = lo + static_cast<uint32_t>(lane) * step;
        const bool le = idx < hi && __ldg(&wk.list[idx].first_unit) <= u;
        const unsigned b = __ballot_sync(0xffffffffu, le);  // bit 0 set: list[lo] <= u
        lo += static_cast<uint32_t>(31 - __clz(b)) * step;
        hi = (lo + step) < hi ? (lo + step) : hi;
    }
    const uint32_t idx = lo + static_cast<uint32_t>(lane);
    const bool le = idx < hi && __ldg(&wk.list[idx].first_unit) <= u;
    const unsigned b = __ballot_sync(0xffffffffu, le);
    return lo + static_cast<uint32_t>(31 - __clz(b));
}

// Lane 0 of a warp: the warp's work units in the order it takes them.  The
// first is static (warp-major numbering, so neighbouring units land on
// different SMs); the rest come from a global counter in blocks of
// consecutive units whose size shrinks with the work left: a quarter of one
// warp's share of it, at most kClaimMax and at least 1.  Early claims are
// large, so the counter sees few atomics; the last units still go out one at
// a time, so a warp held up by an expensive unit leaves the rest to others.
constexpr uint32_t kClaimMax = 8;

struct UnitClaims {
    uint64_t first;  // the static unit (~0: taken)
    uint32_t skip;   // units before the counter's first: warps in the grid
    uint32_t next;   // the current block's next unit (counter numbering)
    uint32_t left;   // its units not yet taken
    uint32_t seen;   // the counter after this warp's last claim
};

__device__ __forceinline__ UnitClaims claims_start(uint64_t first, uint64_t grid_warps) {
    UnitClaims c;
    c.first = first;
    c.skip = static_cast<uint32_t>(grid_warps);
    c.next = 0;
    c.left = 0;
    c.seen = 0;
    return c;
}

// Lane 0: the next unit, or ~0 once the units are used up (then ~0 for good).
// units < 2^31.
__device__ __forceinline__ uint64_t claims_next(UnitClaims &c, unsigned int *counter, uint64_t units) {
    if (c.first != ~0ull) {
        const uint64_t u = c.first;
        c.first = ~0ull;
        return u;
    }
    if (c.left == 0) {
        if (units <= c.skip || !counter) return ~0ull;  // no counter: the launcher saw units <= skip
        const uint32_t dyn = static_cast<uint32_t>(units) - c.skip;  // units the counter hands out
        if (c.seen >= dyn) return ~0ull;
        uint32_t blk = (dyn - c.seen) / (4u * c.skip);
        blk = blk < 1u ? 1u : (blk > kClaimMax ? kClaimMax : blk);
        const uint32_t at = atomicAdd(counter, blk);
        c.seen = at + blk < at ? 0xFFFFFFFFu : at + blk;
        if (at >= dyn) return ~0ull;
        c.next = at;
        c.left = dyn - at < blk ? dyn - at : blk;
    }
    --c.left;
    return static_cast<uint64_t>(c.skip) + c.next++;
}

// One thread: start the bulk copy of tile t.tile into shared buffer st (text
// lines marked to leave L2 first: the text is read once).  Only the 16-byte
// aligned part inside the text is copied; load_text_fringe fetches the rest.
__device__ __forceinline__ void issue_text_tile(const TileText &t, uint32_t tile_len, uint32_t staged,
                                                uint64_t *bar, uint8_t *st) {
    const uint64_t tlo = static_cast<uint64_t>(t.tile) * tile_len;
    const uint64_t a1 = (static_cast<uint64_t>(t.head) + 15ull) & ~15ull;
    const uint64_t a2 = (static_cast<uint64_t>(t.head) + t.n) & ~15ull;
    const uint64_t lo = tlo > a1 ? tlo : a1;
    const uint64_t hi = (tlo + staged) < a2 ? (tlo + staged) : a2;
    if (a1 < a2 && lo < hi) {
        const uint32_t bytes = static_cast<uint32_t>(hi - lo);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load_hint(st + (lo - tlo), t.gbase + lo, bytes, bar, policy_evict_first());
    } else {
        mbar_arrive(bar);
    }
}

// A warp: the unaligned head and tail bytes of the text that the bulk copy
// leaves out (at most 15 each): lanes 0-15 the head, 16-31 the tail.
__device__ __forceinline__ void load_text_fringe(const TileText &t, uint32_t staged, uint8_t *st, uint64_t tlo,
                                                 int lane) {
    const uint64_t head = t.head, end = head + t.n;
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
    if (hi > tlo + staged) hi = tlo + staged;
    const uint64_t idx = lo + static_cast<uint64_t>(lane & 15);
    if (idx < hi) st[idx - tlo] = t.gbase[idx];
}

// True when the L bytes at t equal the L bytes at c (any alignment): aligned
// 4-byte words, 16 bytes per round with all of a round's loads issued before
// any compare.  Only words holding at least one of the L bytes are read.
__device__ __forceinline__ bool run_equal(const uint8_t *t, const uint8_t *c, uint32_t L) {
    const uint32_t ta = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(t) & 3u);
    const uint32_t ca = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(c) & 3u);
    const uint32_t *tw = reinterpret_cast<const uint32_t *>(t - ta);
    const uint32_t *cw = reinterpret_cast<const uint32_t *>(c - ca);
    const uint32_t tn = (ta + L + 3u) >> 2, cn = (ca + L + 3u) >> 2;  // words holding the bytes
    uint32_t tp = __ldg(tw), cp = __ldg(cw);
    for (uint32_t j = 0; j < L; j += 16) {
        const uint32_t w0 = (j >> 2) + 1;
        uint32_t tx[4], cx[4];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            tx[k] = w0 + k < tn ? __ldg(tw + w0 + k) : 0u;
            cx[k] = w0 + k < cn ? __ldg(cw + w0 + k) : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t done = j + 4u * k;
            if (done < L) {
                const uint32_t a = __funnelshift_r(tp, tx[k], 8u * ta);
                const uint32_t b = __funnelshift_r(cp, cx[k], 8u * ca);
                const uint32_t left = L - done;
                const uint32_t mask = left >= 4u ? 0xFFFFFFFFu : ((1u << (8u * left)) - 1u);
                if ((a ^ b) & mask) return false;
            }
            tp = tx[k];
            cp = cx[k];
        }
    }
    return true;
}

template <typename GT>
__device__ __forceinline__ int goto_ld(const GT *G, uint32_t s, uint32_t W, uint32_t c) {
    return static_cast<int>(__ldg(G + static_cast<uint64_t>(s) * W + c));
}

// goto_ld with an L2 eviction policy (read-only path).
__device__ __forceinline__ int goto_ld_hint(const int32_t *G, uint32_t s, uint32_t W, uint32_t c, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;"
                 : "=r"(v)
                 : "l"(G + static_cast<uint64_t>(s) * W + c), "l"(pol));
    return v;
}

__device__ __forceinline__ int goto_ld_hint(const int16_t *G, uint32_t s, uint32_t W, uint32_t c, uint64_t pol) {
    short v;
    asm("ld.global.nc.L2::cache_hint.s16 %0, [%1], %2;"
                 : "=h"(v)
                 : "l"(G + static_cast<uint64_t>(s) * W + c), "l"(pol));
    return static_cast<int>(v);
}

// The tables a plain walk from the root needs (the compaction and full-output
// steps match a unit again with it when it has no dense fallback).
struct RootWalk {
    const void *G;
    const uint8_t *cls8;
    uint32_t W, C, maxlen;
    unsigned int *err;
    const uint4 *skip;      // chain records from state s_chain on
    const uint8_t *chain;
    uint32_t s_chain;       // 0xFFFFFFFF: none
};

// The id of the longest keyword starting at text position gp: the walk from
// the root through the goto table (and the chain records).
template <typename GT>
__device__ int walk_from_root(const RootWalk &p, const uint8_t *text, uint64_t n, uint64_t gp) {
    const GT *G = static_cast<const GT *>(p.G);
    uint32_t s = 0;
    uint64_t q = gp;
    for (uint32_t step = 0; step <= p.maxlen + 1; ++step, ++q) {
        if (s >= p.s_chain) {  // a run of forced transitions, a leaf, or a branch
            const uint4 rc = __ldg(p.skip + (s - p.s_chain));
            if (rc.x != kSkipBranch) {
                const bool ok = rc.x > 0 && q + rc.x <= n && run_equal(text + q, p.chain + rc.y, rc.x);
                if (!ok) return static_cast<int>(rc.w);
                s = rc.z;
                q += rc.x - 1;  // the loop adds one
                continue;
            }
        }
        uint32_t c = p.C;
        if (q < n) {
            const uint32_t b = __ldg(text + q);
            if (p.C >= 256) {
                c = b;  // one column per byte value: every byte is a keyword byte
            } else {
                const uint32_t v = __ldg(p.cls8 + b);
                if (v != 0xFFu) c = v;
            }
        }
        const int e = goto_ld(G, s, p.W, c);
        if (e < 0) return decode_dead(e);
        s = static_cast<uint32_t>(e);
    }
    atomicOr(p.err, static_cast<unsigned>(kErrWalk));
    return -1;
}

}  // namespace pfac
