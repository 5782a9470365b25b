// The C ABI declared in include/ac.h: handle lifetime, device residency of the
// compiled tables, argument checks and dispatch to the kernels.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime_api.h>

#include "ac.h"
#include "pfac_internal.h"

struct ac_automaton {
    pfac::HostTables host;
    pfac::DevTables dev;
    bool host_only = false;
    int device = 0;
    ac_kernel kernel = AC_KERNEL_TILED;
    pfac::Tuning tuning;
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    std::vector<void *> owned;  // device allocations of the tables
    uint64_t stride_bytes = 0;  // the build's stride-table budget
    // Root filter tables by shared-table depth (key: the window k, or the
    // hashed filter's bits), once a depth other than the built one is asked
    // for: the built tables first.  Replaced tables stay allocated (launches
    // captured before may read them) until ac_destroy, or until the autotuner
    // drops the depths it did not choose.
    struct RootSet {
        uint32_t key = 0;
        pfac::RootTables t;
        const uint32_t *F = nullptr;
        const int32_t *JK = nullptr, *J2 = nullptr;
    };
    std::vector<RootSet> roots;

    // staging for ac_match_host (allocated on first use)
    std::mutex host_mu;
    uint8_t *h2d_text[2] = {nullptr, nullptr};
    int32_t *h2d_out[2] = {nullptr, nullptr};
    size_t chunk = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
};

struct ac_batch_plan {
    std::vector<ac_handle> hs;
    int device = 0;
    uint32_t max_items = 0;
    void *scratch = nullptr;
    void *lists = nullptr;  // the phased form's lists (ac_batch_reserve_lists)
    uint32_t list_cap = 0;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void *dev_malloc(ac_automaton *h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (h->dev_alloc) return h->dev_alloc(bytes, h->alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_release(ac_automaton *h, void *p) {
    if (!p) return;
    if (h->dev_free)
        h->dev_free(p, h->alloc_ctx);
    else
        cudaFree(p);
}

ac_status upload(ac_automaton *h, const void *src, size_t bytes, const void **dst) {
    void *p = dev_malloc(h, bytes);
    if (!p) return AC_ERR_OOM;
    h->owned.push_back(p);
    if (bytes && cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return AC_ERR_CUDA;
    *dst = p;
    return AC_OK;
}

void release_owned(ac_automaton *h, const void *p) {
    if (!p) return;
    for (size_t i = 0; i < h->owned.size(); ++i)
        if (h->owned[i] == p) {
            dev_release(h, h->owned[i]);
            h->owned.erase(h->owned.begin() + static_cast<std::ptrdiff_t>(i));
            return;
        }
}

// ---- shared-table depth: the root filter tables rebuilt at another size ----

bool has_root(const pfac::HostTables &t) { return t.filter || t.hashed; }
uint32_t root_key(const pfac::HostTables &t) { return t.filter ? t.k : t.fbits; }

// The depth of the largest root filter within `bytes` (0: none fits).
uint32_t root_key_for(const pfac::HostTables &t, uint32_t bytes) {
    if (t.filter) return bytes >= 16 ? pfac::filter_window(t.B, t.maxlen, bytes) : 0u;
    uint32_t fb = 0;
    while (fb < pfac::kFilterBits && (2ull << fb) <= 8ull * bytes) ++fb;
    return fb >= 5 ? fb : 0u;
}

// Make depth `key` the handle's (host and device tables), building and
// uploading its tables the first time.
ac_status use_root(ac_automaton *h, uint32_t key) {
    pfac::HostTables &t = h->host;
    pfac::DevTables &d = h->dev;
    if (!has_root(t)) return AC_ERR_INVALID_ARG;
    if (key == root_key(t)) return AC_OK;
    if (h->roots.empty()) {  // the built tables, as they are
        ac_automaton::RootSet b;
        b.key = root_key(t);
        b.t.k = t.k;
        b.t.k2 = t.k2;
        b.t.base_k = t.base_k;
        b.t.count_k = t.count_k;
        b.t.fbits = t.fbits;
        b.t.match_windows_ppm = t.match_windows_ppm;
        b.t.F = t.F;
        if (t.filter) {
            b.t.JK = t.JK;
            b.t.J2 = t.J2;
        }
        b.F = d.F;
        b.JK = d.JK;
        b.J2 = d.J2;
        h->roots.push_back(std::move(b));
    }
    size_t at = h->roots.size();
    for (size_t i = 0; i < h->roots.size(); ++i)
        if (h->roots[i].key == key) at = i;
    if (at == h->roots.size()) {
        ac_automaton::RootSet rs;
        rs.key = key;
        try {
            if (t.filter)
                pfac::window_tables(t, key, h->stride_bytes, &rs.t);
            else
                pfac::hashed_filter(t, key, &rs.t);
        } catch (const std::bad_alloc &) {
            return AC_ERR_OOM;
        }
        if (!h->host_only) {
            ac_status s = upload(h, rs.t.F.data(), rs.t.F.size() * sizeof(uint32_t),
                                 reinterpret_cast<const void **>(&rs.F));
            if (s == AC_OK && t.filter)
                s = upload(h, rs.t.JK.data(), rs.t.JK.size() * sizeof(int32_t), reinterpret_cast<const void **>(&rs.JK));
            if (s == AC_OK && t.filter && !rs.t.J2.empty())
                s = upload(h, rs.t.J2.data(), rs.t.J2.size() * sizeof(int32_t), reinterpret_cast<const void **>(&rs.J2));
            if (s != AC_OK) {
                release_owned(h, rs.F);
                release_owned(h, rs.JK);
                release_owned(h, rs.J2);
                return s;
            }
        }
        h->roots.push_back(std::move(rs));
    }
    const ac_automaton::RootSet &rs = h->roots[at];
    t.F = rs.t.F;
    d.F = rs.F;
    d.fbytes = static_cast<uint32_t>(rs.t.F.size() * sizeof(uint32_t));
    if (t.filter) {
        t.k = d.k = rs.t.k;
        t.k2 = d.k2 = rs.t.k2;
        t.base_k = d.base_k = rs.t.base_k;
        t.count_k = rs.t.count_k;
        t.JK = rs.t.JK;
        t.J2 = rs.t.J2;
        t.match_windows_ppm = rs.t.match_windows_ppm;
        d.list_prefer = t.match_windows_ppm >= pfac::kListMatchWindowsPpm;
        d.JK = rs.JK;
        d.J2 = rs.J2;
    } else {
        t.fbits = d.fbits = rs.t.fbits;
    }
    return AC_OK;
}

// Free the root tables of every depth but the built one and the current one.
void drop_roots(ac_automaton *h) {
    const uint32_t cur = root_key(h->host);
    for (size_t i = h->roots.size(); i-- > 1;) {
        if (h->roots[i].key == cur) continue;
        release_owned(h, h->roots[i].F);
        release_owned(h, h->roots[i].JK);
        release_owned(h, h->roots[i].J2);
        h->roots.erase(h->roots.begin() + static_cast<std::ptrdiff_t>(i));
    }
}

void release_host_path(ac_automaton *h) {
    for (int i = 0; i < 2; ++i) {
        dev_release(h, h->h2d_text[i]);
        dev_release(h, h->h2d_out[i]);
        h->h2d_text[i] = nullptr;
        h->h2d_out[i] = nullptr;
        if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
        if (h->ev_comp[i]) cudaEventDestroy(h->ev_comp[i]);
        if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
        h->ev_in[i] = h->ev_comp[i] = h->ev_out[i] = nullptr;
    }
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    h->s_in = h->s_out = nullptr;
    h->chunk = 0;
}

ac_status check_device(ac_automaton *h) {
    if (!h) return AC_ERR_INVALID_ARG;
    if (h->host_only) return AC_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return AC_ERR_CUDA;
    if (dev != h->device) return AC_ERR_INVALID_ARG;
    return AC_OK;
}

}  // namespace

// The library's stream-ordered pool for per-call scratch on `dev`.  It keeps
// the memory it has grown to (release threshold: unlimited), so a call does
// not map fresh device memory after every synchronisation, as the default
// pool (threshold 0) would.
cudaError_t pfac::scratch_pool(int dev, cudaMemPool_t *out) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

namespace {

using pfac::scratch_pool;

// A tiled launch (dense ids or count) with its zeroed scratch (the tile
// counter) in stream-ordered memory, so calls on different streams never share it.
// A text short enough that every tile is some warp's first needs no counter:
// the launchers accept no scratch then, which saves the allocation and the
// clearing of small calls.
cudaError_t run_tiled(ac_automaton *h, pfac::MatchRequest r, pfac::OutMode mode, cudaStream_t st) {
    // 8-bit codes, long text: the phased form's lists after the counter
    pfac::SurvivorLists sl;
    if (!r.batch && pfac::uses_filter(h->dev, h->tuning)) sl = pfac::survivor_lists(h->dev, h->tuning, r.n);
    const bool le = sl.list_cap != 0;
    if (!r.batch && r.n <= (16u << 20) && !le) {
        pfac::MatchRequest r0 = r;
        r0.scratch = nullptr;
        r0.scratch_bytes = 0;
        const cudaError_t e0 = pfac::launch_match(h->dev, r0, mode, h->tuning, st);
        if (e0 == cudaSuccess) return e0;  // else: a counter is needed (or a real error, reported below)
    }
    const size_t bytes = 16 + sl.bytes();
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(h->device, &pool);
    if (e != cudaSuccess) return e;
    void *scratch = nullptr;
    e = cudaMallocFromPoolAsync(&scratch, bytes, pool, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(scratch, 0, le ? 48 : 16, st);
    if (e == cudaSuccess) {
        r.scratch = scratch;
        r.scratch_bytes = 16;
        if (le) pfac::set_lists(r, static_cast<uint8_t *>(scratch) + 16, sl);
        e = pfac::launch_match(h->dev, r, mode, h->tuning, st);
    }
    const cudaError_t e2 = cudaFreeAsync(scratch, st);
    return e != cudaSuccess ? e : e2;
}

// The compacted match of one text with its scratch from the pool.
cudaError_t run_compact(ac_automaton *h, const uint8_t *text, uint64_t n, const pfac::CompactOut &out,
                        cudaStream_t st) {
    const uint32_t units = pfac::compact_units(h->dev, h->tuning, text, n);
    if (units == 0xFFFFFFFFu) return cudaErrorInvalidValue;
    // the phased form's lists instead of the dense fallback when it applies
    // (the gather then matches an overflowing unit again)
    pfac::SurvivorLists sl;
    if (pfac::uses_filter(h->dev, h->tuning)) sl = pfac::survivor_lists(h->dev, h->tuning, n, true);
    const bool dense = sl.list_cap == 0;
    const size_t bytes = pfac::compact_scratch_bytes(h->dev, units, dense) + sl.bytes();
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(h->device, &pool);
    if (e != cudaSuccess) return e;
    void *scratch = nullptr;
    e = cudaMallocFromPoolAsync(&scratch, bytes, pool, st);
    if (e != cudaSuccess) return e;
    e = pfac::enqueue_compact(h->dev, h->tuning, text, n, out, scratch, bytes, dense, st);
    const cudaError_t e2 = cudaFreeAsync(scratch, st);
    return e != cudaSuccess ? e : e2;
}

// The full output of one text with its scratch from the pool.
cudaError_t run_full(ac_automaton *h, const uint8_t *text, uint64_t n, const pfac::CompactOut &out,
                     cudaStream_t st) {
    const uint32_t units = pfac::compact_units(h->dev, h->tuning, text, n);
    if (units == 0xFFFFFFFFu) return cudaErrorInvalidValue;
    const size_t bytes = pfac::full_scratch_bytes(h->dev, h->tuning, units, n);
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(h->device, &pool);
    if (e != cudaSuccess) return e;
    void *scratch = nullptr;
    e = cudaMallocFromPoolAsync(&scratch, bytes, pool, st);
    if (e != cudaSuccess) return e;
    e = pfac::enqueue_full(h->dev, h->tuning, text, n, out, scratch, bytes, st);
    const cudaError_t e2 = cudaFreeAsync(scratch, st);
    return e != cudaSuccess ? e : e2;
}

ac_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return AC_OK;
    if (e == cudaErrorMemoryAllocation) return AC_ERR_OOM;
    if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) return AC_ERR_INVALID_ARG;
    return AC_ERR_CUDA;
}

// Bytes of a batch's scratch: per automaton a head and a tile counter
// (16 bytes each), then the planned list (32 bytes per text).
size_t batch_scratch_bytes(uint32_t nh, uint32_t nitems) {
    return static_cast<size_t>(nh) * 32u + static_cast<size_t>(nitems) * sizeof(pfac::BatchItemDev);
}

ac_status check_handles(const ac_handle *hs, uint32_t nh) {
    if (!hs || nh == 0 || nh > pfac::kMaxBatchAutomata) return AC_ERR_INVALID_ARG;
    for (uint32_t a = 0; a < nh; ++a) {
        const ac_status s = check_device(hs[a]);
        if (s != AC_OK) return s;
    }
    return AC_OK;
}

// Enqueue a batch on `st`: clear the tile counters, plan on the device, then
// match: when the filter kernel serves every automaton, one persistent launch
// for all of them (each CTA takes the automata in turn, so they overlap and no
// launch boundary drains the GPU between them); otherwise one persistent
// launch per automaton, one after another.
cudaError_t enqueue_batch(const ac_handle *hs, uint32_t nh, void *scratch, const uint8_t *texts,
                          const ac_batch_item *items, uint32_t nitems, int32_t *out, cudaStream_t st,
                          void *surv_lists = nullptr, uint32_t list_cap = 0) {
    uint8_t *base = static_cast<uint8_t *>(scratch);
    pfac::BatchHead *heads = reinterpret_cast<pfac::BatchHead *>(base);
    uint8_t *counters = base + static_cast<size_t>(nh) * 16u;
    pfac::BatchItemDev *lists = reinterpret_cast<pfac::BatchItemDev *>(base + static_cast<size_t>(nh) * 32u);
    std::vector<const pfac::DevTables *> ts(nh);
    for (uint32_t a = 0; a < nh; ++a) ts[a] = &hs[a]->dev;
    const bool multi = pfac::filter_multi_serves(ts.data(), nh);
    std::vector<uint32_t> tile_len(nh);
    for (uint32_t a = 0; a < nh; ++a)
        tile_len[a] = multi ? pfac::filter_tile_positions() : pfac::unit_positions(hs[a]->dev, hs[a]->tuning);
    cudaError_t e = cudaMemsetAsync(counters, 0, static_cast<size_t>(nh) * 16u, st);
    if (e == cudaSuccess) e = pfac::launch_batch_plan(items, nitems, nh, texts, tile_len.data(), heads, lists, st);
    if (multi) {
        std::vector<pfac::MatchRequest> rs(nh);
        for (uint32_t a = 0; a < nh; ++a) {
            rs[a].text = texts;
            rs[a].out = out;
            rs[a].batch = heads + a;
            rs[a].lists = lists;
            rs[a].scratch = counters + 16u * a;
            rs[a].scratch_bytes = 16;
        }
        if (e == cudaSuccess && surv_lists && list_cap) e = cudaMemsetAsync(surv_lists, 0, 32, st);
        if (e == cudaSuccess)
            e = pfac::launch_filter_multi(ts.data(), rs.data(), nh, pfac::OUT_DENSE, hs[0]->tuning.wait_ns, st,
                                          list_cap ? surv_lists : nullptr, list_cap);
        return e;
    }
    for (uint32_t a = 0; a < nh && e == cudaSuccess; ++a) {
        cudaStream_t sa = st;
        pfac::MatchRequest r;
        r.text = texts;
        r.out = out;
        r.batch = heads + a;
        r.lists = lists;
        r.scratch = counters + 16u * a;
        r.scratch_bytes = 16;
        ac_automaton *h = hs[a];
        e = pfac::launch_match(h->dev, r, pfac::OUT_DENSE, h->tuning, sa);
    }
    return e;
}

}  // namespace

namespace pfac {
// The device tables of a handle, for entry points outside this file.
const DevTables *handle_tables(ac_handle h, int *device, bool *host_only) {
    if (!h) return nullptr;
    *device = h->device;
    *host_only = h->host_only;
    return &h->dev;
}

const Tuning *handle_tuning(ac_handle h) { return h ? &h->tuning : nullptr; }
}  // namespace pfac

extern "C" {

void ac_default_options(ac_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->class_compress = 1;
}

ac_status ac_compile(const uint8_t *const *patterns, const uint32_t *lens, uint32_t k, const ac_options *opt,
                     ac_handle *out) {
    if (!out) return AC_ERR_INVALID_ARG;
    *out = nullptr;
    if (k == 0) return AC_ERR_EMPTY_PATTERN;
    if (!patterns || !lens) return AC_ERR_INVALID_ARG;
    ac_options o;
    ac_default_options(&o);
    if (opt) o = *opt;
    if (o.index_width != 0 && o.index_width != 16 && o.index_width != 32) return AC_ERR_INVALID_ARG;
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr)) return AC_ERR_INVALID_ARG;

    ac_automaton *h = new (std::nothrow) ac_automaton();
    if (!h) return AC_ERR_OOM;
    pfac::BuildOptions bo;
    bo.index_width = o.index_width;
    bo.class_compress = o.class_compress ? 1 : 0;
    if (o.jump_bytes) bo.jump_bytes = o.jump_bytes;
    if (o.stride_bytes) bo.stride_bytes = o.stride_bytes;
    bo.chains = o.no_chains == 0;
    h->stride_bytes = bo.stride_bytes;
    int st = pfac::build_tables(patterns, lens, k, bo, &h->host);
    if (st != AC_OK) {
        delete h;
        return static_cast<ac_status>(st);
    }
    h->host_only = o.host_only != 0;
    h->dev_alloc = o.dev_alloc;
    h->dev_free = o.dev_free;
    h->alloc_ctx = o.alloc_ctx;
    const pfac::HostTables &t = h->host;
    pfac::DevTables &d = h->dev;
    d.S = t.S;
    d.C = t.C;
    d.W = t.W;
    d.gbits = t.gbits;
    d.B = t.B;
    d.k = t.k;
    d.k2 = t.k2;
    d.base_k = t.base_k;
    d.maxlen = t.maxlen;
    d.jbytes = static_cast<uint32_t>(t.J.size() * sizeof(int16_t));
    d.jslow = t.jslow;
    d.filter = t.filter;
    d.list_prefer = t.filter && t.match_windows_ppm >= pfac::kListMatchWindowsPpm;
    d.hashed = t.hashed;
    d.kh = t.kh;
    d.fbits = t.fbits;
    d.hk_bits = t.hk_bits;
    d.hk_probes = t.hk_probes;
    d.fbytes = static_cast<uint32_t>(t.F.size() * sizeof(uint32_t));
    d.hash_shift = t.hash_shift;
    d.full_max_clen = t.full_max_clen;
    d.nkw = t.nkw;
    std::memcpy(d.hash_code, t.hash_code, 8);
    std::memcpy(d.hash_byte, t.hash_byte, 8);
    d.direct_shift = t.direct_shift;
    if (t.direct_shift == 1) {  // byte 2c of the pair
        d.direct_sel[0] = t.direct_byte[0] | (static_cast<uint32_t>(t.direct_byte[1]) << 16);
        d.direct_sel[1] = t.direct_byte[2] | (static_cast<uint32_t>(t.direct_byte[3]) << 16);
        for (uint32_t b = 0; b < 256; ++b)
            if (t.cls8[b] == 0xFF) {
                d.direct_fill = b;
                break;
            }
    }
    if (!h->host_only) {
        if (cudaGetDevice(&h->device) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return AC_ERR_CUDA;
        }
        ac_status s = upload(h, t.G.data(), t.G.size(), &d.G);
        if (s == AC_OK) s = upload(h, t.cls.data(), 512, reinterpret_cast<const void **>(&d.cls));
        if (s == AC_OK) s = upload(h, t.cls8.data(), 256, reinterpret_cast<const void **>(&d.cls8));
        if (s == AC_OK && !t.J.empty())
            s = upload(h, t.J.data(), t.J.size() * sizeof(int16_t), reinterpret_cast<const void **>(&d.J));
        if (s == AC_OK && !t.F.empty())
            s = upload(h, t.F.data(), t.F.size() * sizeof(uint32_t), reinterpret_cast<const void **>(&d.F));
        if (s == AC_OK && !t.JK.empty())
            s = upload(h, t.JK.data(), t.JK.size() * sizeof(int32_t), reinterpret_cast<const void **>(&d.JK));
        if (s == AC_OK && !t.HK.empty())
            s = upload(h, t.HK.data(), t.HK.size() * sizeof(uint32_t), reinterpret_cast<const void **>(&d.HK));
        if (s == AC_OK && !t.J2.empty())
            s = upload(h, t.J2.data(), t.J2.size() * sizeof(int32_t), reinterpret_cast<const void **>(&d.J2));
        if (s == AC_OK && !t.skip.empty()) {
            s = upload(h, t.skip.data(), t.skip.size() * sizeof(uint32_t), reinterpret_cast<const void **>(&d.skip));
            if (s == AC_OK)
                s = upload(h, t.chain.data(), t.chain.size(), reinterpret_cast<const void **>(&d.chain));
            d.s_chain = t.s_chain;
        }
        if (s == AC_OK)
            s = upload(h, t.full_rec.data(), t.full_rec.size() * sizeof(uint32_t),
                       reinterpret_cast<const void **>(&d.full_rec));
        if (s == AC_OK)
            s = upload(h, t.full_dups.data(), t.full_dups.size() * sizeof(uint32_t),
                       reinterpret_cast<const void **>(&d.full_dups));
        // commit the static scratch of ac_match_compact_static on this device
        // now, while device memory can still be had, rather than at its first call
        void *stat = nullptr;
        if (s == AC_OK && pfac::static_scratch_address(h->device, &stat) != cudaSuccess) {
            cudaGetLastError();
            s = AC_ERR_CUDA;
        }
        if (s != AC_OK) {
            ac_destroy(h);
            return s;
        }
    }
    *out = h;
    return AC_OK;
}

ac_status ac_destroy(ac_handle h) {
    if (!h) return AC_OK;
    release_host_path(h);
    for (void *p : h->owned) dev_release(h, p);
    delete h;
    return AC_OK;
}

ac_status ac_info(ac_handle h, ac_info_t *info) {
    if (!h || !info) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    std::memset(info, 0, sizeof(*info));
    info->n_keywords = t.nkw;
    info->n_states = t.S;
    info->n_classes = t.C;
    info->row_width = t.W;
    info->index_width = t.gbits;
    info->code_bits = t.B;
    info->jump_depth = t.k;
    info->stride_depth = t.k2;
    info->min_len = t.minlen;
    info->max_len = t.maxlen;
    info->table_bytes = t.G.size() + t.J.size() * sizeof(int16_t) + t.J2.size() * sizeof(int32_t) +
                        t.F.size() * sizeof(uint32_t) + t.JK.size() * sizeof(int32_t) +
                        t.skip.size() * sizeof(uint32_t) + t.chain.size() + 768 +
                        (t.full_rec.size() + t.full_dups.size()) * sizeof(uint32_t);
    info->depth_base_jump = t.base_k;
    info->count_jump = t.count_k;
    info->class_hash_shift = t.hash_shift;
    info->match_windows_ppm = t.B <= 4 ? t.match_windows_ppm : 0u;
    info->class_direct_shift = t.direct_shift;
    return AC_OK;
}

ac_status ac_export_tables(ac_handle h, int16_t *cls, void *goto_, uint32_t *depth) {
    if (!h) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    if (cls) std::memcpy(cls, t.cls.data(), 256 * sizeof(int16_t));
    if (goto_) std::memcpy(goto_, t.G.data(), t.G.size());
    if (depth) std::memcpy(depth, t.depth_count.data(), t.depth_count.size() * sizeof(uint32_t));
    return AC_OK;
}

ac_status ac_export_chains(ac_handle h, uint32_t *s_chain, uint32_t *records, uint8_t *bytes, uint64_t *n_records,
                           uint64_t *n_bytes) {
    if (!h || !s_chain || !n_records || !n_bytes) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    *s_chain = t.skip.empty() ? t.S : t.s_chain;
    *n_records = t.skip.size() / 4;
    *n_bytes = t.chain.size();
    if (records && !t.skip.empty()) std::memcpy(records, t.skip.data(), t.skip.size() * sizeof(uint32_t));
    if (bytes && !t.chain.empty()) std::memcpy(bytes, t.chain.data(), t.chain.size());
    return AC_OK;
}

ac_status ac_export_full(ac_handle h, uint32_t *records, uint32_t *dups, uint32_t *max_chain) {
    if (!h) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    if (records) std::memcpy(records, t.full_rec.data(), t.full_rec.size() * sizeof(uint32_t));
    if (dups) std::memcpy(dups, t.full_dups.data(), t.full_dups.size() * sizeof(uint32_t));
    if (max_chain) *max_chain = t.full_max_clen;
    return AC_OK;
}

ac_status ac_export_filter(ac_handle h, uint32_t *F, int32_t *JK, uint32_t *B, uint32_t *k, uint64_t *f_words,
                           uint64_t *jk_entries) {
    if (!h || !B || !k || !f_words || !jk_entries) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    *B = t.filter ? t.B : 0u;
    *k = t.filter ? t.k : 0u;
    *f_words = t.filter ? t.F.size() : 0u;
    *jk_entries = t.filter ? t.JK.size() : 0u;
    if (t.filter && F) std::memcpy(F, t.F.data(), t.F.size() * sizeof(uint32_t));
    if (t.filter && JK) std::memcpy(JK, t.JK.data(), t.JK.size() * sizeof(int32_t));
    return AC_OK;
}

ac_status ac_export_hash(ac_handle h, uint32_t *F, uint32_t *HK, uint32_t *kh, uint32_t *fbits, uint32_t *hk_bits,
                         uint32_t *probes) {
    if (!h || !kh || !fbits || !hk_bits || !probes) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    *kh = t.hashed ? t.kh : 0u;
    *fbits = t.hashed ? t.fbits : 0u;
    *hk_bits = t.hashed ? t.hk_bits : 0u;
    *probes = t.hashed ? t.hk_probes : 0u;
    if (t.hashed && F) std::memcpy(F, t.F.data(), t.F.size() * sizeof(uint32_t));
    if (t.hashed && HK) std::memcpy(HK, t.HK.data(), t.HK.size() * sizeof(uint32_t));
    return AC_OK;
}

ac_status ac_export_stride(ac_handle h, int32_t *J2, uint32_t *k2, uint32_t *base_k, uint32_t *count_k,
                           uint64_t *entries) {
    if (!h || !k2 || !base_k || !count_k || !entries) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    *k2 = t.J2.empty() ? 0u : t.k2;
    *base_k = t.base_k;
    *count_k = t.count_k;
    *entries = t.J2.size();
    if (J2 && !t.J2.empty()) std::memcpy(J2, t.J2.data(), t.J2.size() * sizeof(int32_t));
    return AC_OK;
}

ac_status ac_export_jump(ac_handle h, int16_t *J, uint32_t *k, uint32_t *base_k, uint64_t *entries) {
    if (!h || !k || !base_k || !entries) return AC_ERR_INVALID_ARG;
    const pfac::HostTables &t = h->host;
    const bool has = t.B == 8 && t.k > 0 && !t.J.empty();
    *k = has ? t.k : 0u;
    *base_k = t.base_k;
    *entries = has ? (1ull << (t.B * t.k)) : 0u;  // J is padded to at least 8 entries
    if (has && J) std::memcpy(J, t.J.data(), static_cast<size_t>(*entries) * sizeof(int16_t));
    return AC_OK;
}

ac_status ac_set_kernel(ac_handle h, ac_kernel kernel) {
    if (!h) return AC_ERR_INVALID_ARG;
    switch (kernel) {
        case AC_KERNEL_TILED:
        case AC_KERNEL_SIMPLE:
            h->tuning.variant = 0;
            break;
        case AC_KERNEL_WALK_SLOTS:
            h->tuning.variant = 1;
            break;
        case AC_KERNEL_THREAD_JUMP:
            h->tuning.variant = 2;
            break;
        case AC_KERNEL_THREAD_JUMP_L1:
            h->tuning.variant = 3;
            break;
        default:
            return AC_ERR_INVALID_ARG;
    }
    h->kernel = kernel == AC_KERNEL_SIMPLE ? AC_KERNEL_SIMPLE : AC_KERNEL_TILED;
    return AC_OK;
}

ac_status ac_get_tuning(ac_handle h, ac_tuning *out) {
    if (!h || !out) return AC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->block = static_cast<uint32_t>(h->tuning.block);
    out->stages = static_cast<uint32_t>(h->tuning.stages);
    out->halo = h->tuning.halo > 16 ? static_cast<uint32_t>(h->tuning.halo) : 16u;
    out->per_thread = h->tuning.per_thread == 4 ? 4u : 2u;
    out->filter_bytes = has_root(h->host) ? static_cast<uint32_t>(h->host.F.size() * sizeof(uint32_t)) : 0u;
    out->survivor_list = static_cast<uint32_t>(h->tuning.survivor_list);
    return AC_OK;
}

ac_status ac_set_tuning(ac_handle h, const ac_tuning *tu) {
    if (!h || !tu) return AC_ERR_INVALID_ARG;
    if ((tu->block != 0 && tu->block < 32) || tu->block > 640 || (tu->block & 31u) ||
        (tu->stages != 0 && (tu->stages < 2 || tu->stages > 4)) ||
        tu->halo > pfac::kHaloCap || (tu->per_thread != 0 && tu->per_thread != 2 && tu->per_thread != 4) ||
        tu->survivor_list > 2)
        return AC_ERR_INVALID_ARG;
    if (tu->filter_bytes != 0) {
        if (!has_root(h->host)) return AC_ERR_INVALID_ARG;
        const uint32_t key = root_key_for(h->host, tu->filter_bytes);
        if (key == 0) return AC_ERR_INVALID_ARG;
        const ac_status s = use_root(h, key);
        if (s != AC_OK) return s;
    }
    h->tuning.block = static_cast<int>(tu->block);
    h->tuning.stages = static_cast<int>(tu->stages);
    h->tuning.halo = static_cast<int>(tu->halo);
    h->tuning.per_thread = static_cast<int>(tu->per_thread);
    h->tuning.survivor_list = static_cast<int>(tu->survivor_list);
    return AC_OK;
}

ac_status ac_set_wait_limit(ac_handle h, uint64_t limit_ns, int32_t stall_help) {
    if (!h) return AC_ERR_INVALID_ARG;
    h->tuning.wait_ns = limit_ns;
    h->tuning.stall_help = stall_help ? 1 : 0;
    return AC_OK;
}

ac_status ac_match(ac_handle h, const uint8_t *d_text, uint64_t n, int32_t *d_out_ids, void *stream) {
    ac_status s = check_device(h);
    if (s != AC_OK) return s;
    if (n == 0) return AC_OK;
    if (!d_text || !d_out_ids) return AC_ERR_INVALID_ARG;
    pfac::MatchRequest r;
    r.text = d_text;
    r.n = n;
    r.out = d_out_ids;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (h->kernel == AC_KERNEL_SIMPLE) return cuda_status(pfac::launch_simple(h->dev, r, st));
    return cuda_status(run_tiled(h, r, pfac::OUT_DENSE, st));
}

ac_status ac_count(ac_handle h, const uint8_t *d_text, uint64_t n, uint64_t *d_count, void *stream) {
    ac_status s = check_device(h);
    if (s != AC_OK) return s;
    if (!d_count) return AC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st);
    if (e != cudaSuccess || n == 0) return cuda_status(e);
    if (!d_text) return AC_ERR_INVALID_ARG;
    pfac::MatchRequest r;
    r.text = d_text;
    r.n = n;
    r.count = reinterpret_cast<unsigned long long *>(d_count);
    return cuda_status(run_tiled(h, r, pfac::OUT_COUNT, st));
}

ac_status ac_match_compact(ac_handle h, const uint8_t *d_text, uint64_t n, uint32_t *d_pos, uint32_t *d_ids,
                           uint64_t cap, uint64_t *d_count, void *stream) {
    ac_status s = check_device(h);
    if (s != AC_OK) return s;
    if (!d_count || (cap > 0 && (!d_pos || !d_ids))) return AC_ERR_INVALID_ARG;
    if (n > 0xFFFFFFFFull) return AC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st));
    if (!d_text) return AC_ERR_INVALID_ARG;
    const pfac::CompactOut out{d_pos, d_ids, cap, reinterpret_cast<unsigned long long *>(d_count)};
    return cuda_status(run_compact(h, d_text, n, out, st));
}

ac_status ac_match_full(ac_handle h, const uint8_t *d_text, uint64_t n, uint32_t *d_end, uint32_t *d_ids,
                        uint64_t cap, uint64_t *d_count, void *stream) {
    ac_status s = check_device(h);
    if (s != AC_OK) return s;
    if (!d_count || (cap > 0 && (!d_end || !d_ids))) return AC_ERR_INVALID_ARG;
    if (n > 0xFFFFFFFFull) return AC_ERR_INVALID_ARG;
    // a unit's occurrence count (at most kDenseStride results, each with up to
    // full_max_clen occurrences) must fit 32 bits
    if (static_cast<uint64_t>(h->dev.full_max_clen) * pfac::kDenseStride > 0xFFFFFFFFull) return AC_ERR_OVERFLOW;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st));
    if (!d_text) return AC_ERR_INVALID_ARG;
    const pfac::CompactOut out{d_end, d_ids, cap, reinterpret_cast<unsigned long long *>(d_count)};
    return cuda_status(run_full(h, d_text, n, out, st));
}

ac_status ac_match_host(ac_handle h, const uint8_t *h_text, uint64_t n, int32_t *h_out_ids, void *stream) {
    ac_status s = check_device(h);
    if (s != AC_OK) return s;
    if (n == 0) return AC_OK;
    if (!h_text || !h_out_ids) return AC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(h->host_mu);
    cudaStream_t sc = static_cast<cudaStream_t>(stream);
    const size_t chunk = 64u << 20;
    const size_t halo = h->host.maxlen;
    if (h->chunk == 0) {
        for (int i = 0; i < 2; ++i) {
            h->h2d_text[i] = static_cast<uint8_t *>(dev_malloc(h, chunk + halo + 16));
            h->h2d_out[i] = static_cast<int32_t *>(dev_malloc(h, (chunk + halo + 16) * sizeof(int32_t)));
            if (!h->h2d_text[i] || !h->h2d_out[i]) {
                release_host_path(h);
                return AC_ERR_OOM;
            }
            if (cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_comp[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming) != cudaSuccess) {
                release_host_path(h);
                return AC_ERR_CUDA;
            }
        }
        if (cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking) != cudaSuccess) {
            release_host_path(h);
            return AC_ERR_CUDA;
        }
        h->chunk = chunk;
    }
    // Every call ends with all three streams synchronised, so the events only
    // order the chunks of this call.
    cudaError_t e = cudaSuccess;
    const uint64_t nchunks = (n + chunk - 1) / chunk;
    for (uint64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int slot = static_cast<int>(c & 1);
        const uint64_t lo = c * chunk;
        const uint64_t hi = std::min<uint64_t>(n, lo + chunk);
        const uint64_t hi_halo = std::min<uint64_t>(n, hi + halo);
        // text slot is free once the kernel two chunks back has read it
        if (c >= 2) e = cudaStreamWaitEvent(h->s_in, h->ev_comp[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->h2d_text[slot], h_text + lo, hi_halo - lo, cudaMemcpyHostToDevice, h->s_in);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[slot], h->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, h->ev_in[slot], 0);
        // output slot is free once the copy-out two chunks back has finished
        if (e == cudaSuccess && c >= 2) e = cudaStreamWaitEvent(sc, h->ev_out[slot], 0);
        if (e == cudaSuccess) {
            pfac::MatchRequest r;
            r.text = h->h2d_text[slot];
            r.n = hi_halo - lo;
            r.out = h->h2d_out[slot];
            e = (h->kernel == AC_KERNEL_SIMPLE) ? pfac::launch_simple(h->dev, r, sc)
                                                : run_tiled(h, r, pfac::OUT_DENSE, sc);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_comp[slot], sc);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_comp[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out_ids + lo, h->h2d_out[slot], (hi - lo) * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, h->s_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[slot], h->s_out);
    }
    cudaError_t e1 = cudaStreamSynchronize(h->s_out);
    cudaError_t e2 = cudaStreamSynchronize(sc);
    cudaError_t e3 = cudaStreamSynchronize(h->s_in);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    return cuda_status(e);
}

ac_status ac_match_batch(const ac_handle *hs, uint32_t nh, const uint8_t *d_texts, const ac_batch_item *d_items,
                         uint32_t nitems, int32_t *d_out, void *stream) {
    ac_status s = check_handles(hs, nh);
    if (s != AC_OK) return s;
    if (nitems == 0) return AC_OK;
    if (!d_texts || !d_items || !d_out) return AC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(hs[0]->device, &pool);
    if (e != cudaSuccess) return cuda_status(e);
    void *scratch = nullptr;
    e = cudaMallocFromPoolAsync(&scratch, batch_scratch_bytes(nh, nitems), pool, st);
    if (e != cudaSuccess) return cuda_status(e);
    e = enqueue_batch(hs, nh, scratch, d_texts, d_items, nitems, d_out, st);
    const cudaError_t e2 = cudaFreeAsync(scratch, st);
    return cuda_status(e != cudaSuccess ? e : e2);
}

ac_status ac_batch_destroy(ac_batch b) {
    if (!b) return AC_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->scratch) cudaFree(b->scratch);
    if (b->lists) cudaFree(b->lists);
    delete b;
    return AC_OK;
}

ac_status ac_batch_create(const ac_handle *hs, uint32_t nh, uint32_t max_items, ac_batch *out) {
    if (!out) return AC_ERR_INVALID_ARG;
    *out = nullptr;
    ac_status s = check_handles(hs, nh);
    if (s != AC_OK) return s;
    if (max_items == 0) return AC_ERR_INVALID_ARG;
    ac_batch b = new (std::nothrow) ac_batch_plan();
    if (!b) return AC_ERR_OOM;
    b->hs.assign(hs, hs + nh);
    b->device = hs[0]->device;
    b->max_items = max_items;
    cudaError_t e = cudaMalloc(&b->scratch, batch_scratch_bytes(nh, max_items));
    if (e != cudaSuccess) b->scratch = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ac_batch_destroy(b);
        return cuda_status(e);
    }
    *out = b;
    return AC_OK;
}

ac_status ac_batch_reserve_lists(ac_batch b, uint64_t text_bytes) {
    if (!b) return AC_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return AC_ERR_CUDA;
    if (dev != b->device) return AC_ERR_INVALID_ARG;
    const uint64_t cap = text_bytes / 8;
    if (cap >= 0x7FFFFFFFull) return AC_ERR_INVALID_ARG;
    // a graph captured with the old lists would read freed memory: it goes
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->lists) {
        cudaError_t e = cudaFree(b->lists);
        b->lists = nullptr;
        b->list_cap = 0;
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (cap == 0) return AC_OK;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, pfac::multi_lists_bytes(static_cast<uint32_t>(cap)));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? AC_ERR_OOM : cuda_status(e);
    }
    b->lists = p;
    b->list_cap = static_cast<uint32_t>(cap);
    return AC_OK;
}

namespace {
ac_status batch_enqueue(ac_batch b, const uint8_t *d_texts, const ac_batch_item *d_items, uint32_t nitems,
                        int32_t *d_out, cudaStream_t st) {
    return cuda_status(enqueue_batch(b->hs.data(), static_cast<uint32_t>(b->hs.size()), b->scratch, d_texts, d_items,
                                     nitems, d_out, st, b->lists, b->list_cap));
}

ac_status check_plan_args(ac_batch b, const uint8_t *d_texts, const ac_batch_item *d_items, uint32_t nitems,
                          int32_t *d_out) {
    if (!b || nitems > b->max_items) return AC_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return AC_ERR_CUDA;
    if (dev != b->device) return AC_ERR_INVALID_ARG;
    if (nitems > 0 && (!d_texts || !d_items || !d_out)) return AC_ERR_INVALID_ARG;
    return AC_OK;
}
}  // namespace

ac_status ac_batch_run(ac_batch b, const uint8_t *d_texts, const ac_batch_item *d_items, uint32_t nitems,
                       int32_t *d_out, void *stream) {
    ac_status s = check_plan_args(b, d_texts, d_items, nitems, d_out);
    if (s != AC_OK || nitems == 0) return s;
    return batch_enqueue(b, d_texts, d_items, nitems, d_out, static_cast<cudaStream_t>(stream));
}

ac_status ac_batch_capture(ac_batch b, const uint8_t *d_texts, const ac_batch_item *d_items, uint32_t nitems,
                           int32_t *d_out) {
    ac_status s = check_plan_args(b, d_texts, d_items, nitems, d_out);
    if (s != AC_OK) return s;
    if (nitems == 0) return AC_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e);
    s = batch_enqueue(b, d_texts, d_items, nitems, d_out, b->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (s == AC_OK && e != cudaSuccess) s = cuda_status(e);
    cudaGraphExec_t x = nullptr;
    if (s == AC_OK) {
        e = cudaGraphInstantiate(&x, g, 0);
        if (e != cudaSuccess) s = cuda_status(e);
    }
    if (s != AC_OK) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph = g;
    b->exec = x;
    return AC_OK;
}

ac_status ac_batch_replay(ac_batch b, void *stream) {
    if (!b || !b->exec) return AC_ERR_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
}

ac_status ac_autotune(ac_handle h, const uint8_t *d_sample, uint64_t n, uint32_t reps, void *stream,
                      uint32_t *block, uint32_t *stages, uint32_t *kernel) {
    ac_status s = check_device(h);
    if (s != AC_OK) return s;
    if (!d_sample || n == 0) return AC_ERR_INVALID_ARG;
    if (reps == 0) reps = 5;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(h->device, &pool);
    if (e != cudaSuccess) return cuda_status(e);
    void *out = nullptr;
    e = cudaMallocFromPoolAsync(&out, n * sizeof(int32_t), pool, st);
    if (e != cudaSuccess) return cuda_status(e);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const pfac::Tuning keep = h->tuning;
    const ac_kernel keep_kernel = h->kernel;
    const bool root = has_root(h->host);
    const uint32_t keep_key = root ? root_key(h->host) : 0u;
    h->kernel = AC_KERNEL_TILED;
    pfac::Tuning best = keep;
    uint32_t best_key = keep_key;
    float best_ms = -1.0f;
    pfac::MatchRequest r;
    r.text = d_sample;
    r.n = n;
    r.out = static_cast<int32_t *>(out);
    ac_status fail = AC_OK;
    // time one candidate (at the current depth); one that does not fit shared
    // memory is skipped
    auto time_one = [&](const pfac::Tuning &tu) {
        if (e != cudaSuccess) return;
        h->tuning = tu;
        cudaError_t le = run_tiled(h, r, pfac::OUT_DENSE, st);  // warm-up
        if (le == cudaErrorInvalidConfiguration) {
            cudaGetLastError();
            return;
        }
        if (le != cudaSuccess) {
            e = le;
            return;
        }
        std::vector<float> ms;
        for (uint32_t i = 0; i < reps && e == cudaSuccess; ++i) {
            e = cudaEventRecord(t0, st);
            if (e == cudaSuccess) e = run_tiled(h, r, pfac::OUT_DENSE, st);
            if (e == cudaSuccess) e = cudaEventRecord(t1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float v = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t0, t1);
            ms.push_back(v);
        }
        if (e != cudaSuccess) return;
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if (best_ms < 0.0f || med < best_ms) {
            best_ms = med;
            best = tu;
            best_key = root && tu.variant == 0 ? root_key(h->host) : keep_key;
        }
    };
    // shared-table depths: as built (or set), and two smaller
    std::vector<uint32_t> depths{keep_key};
    if (root) {
        const uint32_t step = h->host.filter ? 1u : 2u, lo = h->host.filter ? 1u : 5u;
        for (uint32_t i = 1; i <= 2; ++i)
            if (keep_key >= lo + i * step) depths.push_back(keep_key - i * step);
    }
    static const int kBlocks[4] = {256, 384, 512, 640};  // 640: small alphabets' one-phase forms only
    // small alphabets: the filter kernel only; 8-bit codes: the filter kernel
    // with the hashed filter (when built) and the three 8-bit kernels
    std::vector<int> variants{0};
    if (!h->dev.filter) variants = h->dev.hashed ? std::vector<int>{0, 3, 2, 1} : std::vector<int>{3, 2, 1};
    for (int v : variants) {
        pfac::Tuning tu = keep;
        tu.variant = v;
        tu.grid = 0;
        tu.halo = 0;
        tu.per_thread = 0;
        tu.survivor_list = 0;
        if (v == 2 || v == 3) {
            time_one(tu);
            continue;
        }
        const bool filtered = v == 0 && root;
        for (size_t di = 0; di < (filtered ? depths.size() : 1u) && e == cudaSuccess && fail == AC_OK; ++di) {
            if (filtered) fail = use_root(h, depths[di]);
            for (int bi = 0; bi < 4 && fail == AC_OK; ++bi)
                for (int sg = 2; sg <= 4; ++sg) {
                    if (kBlocks[bi] > 512 && (v != 0 || !h->host.filter)) continue;  // a form of 512 at most
                    tu.block = kBlocks[bi];
                    tu.stages = sg;
                    time_one(tu);
                }
        }
    }
    // at the best shape: the halo, how survivors are resolved on long texts
    // (listed for a second kernel or in the warp), and chars per thread of
    // that second kernel
    if (e == cudaSuccess && fail == AC_OK && best.variant == 0 && root) {
        fail = use_root(h, best_key);
        const pfac::Tuning base = best;
        const int hmax = static_cast<int>(std::min<uint32_t>(pfac::kHaloCap, (h->host.maxlen + 15u) & ~15u));
        std::vector<int> halos{0};
        if (hmax > 16) halos.push_back(hmax);
        pfac::Tuning listed = base;
        listed.survivor_list = 1;
        const bool can_list = pfac::filter_phased(h->dev, listed, n);
        // 8-bit codes list by default, small alphabets try it
        std::vector<int> lists{0};
        if (can_list) lists.push_back(h->host.hashed ? 2 : 1);
        for (int hv : halos)
            for (int sl : lists)
                for (int pt : {0, 4}) {
                    if (hv == 0 && sl == 0 && pt == 0) continue;  // timed above
                    if (pt == 4 && !(can_list && (h->host.hashed ? sl == 0 : sl == 1))) continue;  // no second kernel
                    if (fail != AC_OK) break;
                    pfac::Tuning tu = base;
                    tu.halo = hv;
                    tu.survivor_list = sl;
                    tu.per_thread = pt;
                    time_one(tu);
                }
    }
    if (e == cudaSuccess && fail == AC_OK) {
        if (root) fail = use_root(h, best_key);
        h->tuning = best;
    } else {
        if (root) use_root(h, keep_key);
        h->tuning = keep;
    }
    if (root) drop_roots(h);
    h->kernel = keep_kernel == AC_KERNEL_SIMPLE ? AC_KERNEL_TILED : keep_kernel;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    const cudaError_t e2 = cudaFreeAsync(out, st);
    const cudaError_t e3 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return cuda_status(e);
    if (fail != AC_OK) return fail;
    if (block) *block = static_cast<uint32_t>(h->tuning.block);
    if (stages) *stages = static_cast<uint32_t>(h->tuning.stages);
    if (kernel) {
        static const uint32_t kByVariant[4] = {AC_KERNEL_TILED, AC_KERNEL_WALK_SLOTS, AC_KERNEL_THREAD_JUMP,
                                               AC_KERNEL_THREAD_JUMP_L1};
        *kernel = pfac::uses_filter(h->dev, h->tuning) ? AC_KERNEL_TILED : kByVariant[h->tuning.variant & 3];
    }
    return AC_OK;
}

ac_status ac_scratch_pool_usage(uint64_t *used_now, uint64_t *used_high, int32_t reset_high) {
    if (!used_now || !used_high) return AC_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return AC_ERR_CUDA;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(dev, &pool);
    uint64_t now = 0, high = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &now);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high);
    if (e == cudaSuccess && reset_high) {
        uint64_t zero = 0;  // resets the high-water mark to the current use
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
    }
    if (e != cudaSuccess) return cuda_status(e);
    *used_now = now;
    *used_high = high;
    return AC_OK;
}

ac_status ac_device_status(void) {
    unsigned int v = 0;
    cudaError_t e = pfac::read_device_error(&v);
    if (e != cudaSuccess) return AC_ERR_CUDA;
    if (v & (pfac::kErrTimeout | pfac::kErrWalk)) return AC_ERR_TIMEOUT;
    return v ? AC_ERR_INVALID_ARG : AC_OK;
}

const char *ac_status_string(ac_status s) {
    switch (s) {
        case AC_OK: return "ok";
        case AC_ERR_INVALID_ARG: return "invalid argument";
        case AC_ERR_EMPTY_PATTERN: return "empty keyword or empty keyword set";
        case AC_ERR_TOO_MANY_STATES: return "too many automaton states";
        case AC_ERR_OOM: return "out of memory";
        case AC_ERR_CUDA: return "CUDA runtime error";
        case AC_ERR_OVERFLOW: return "more matches than output capacity";
        case AC_ERR_BUDGET: return "request exceeds the memory budget";
        case AC_ERR_TIMEOUT: return "a bounded device wait ran out";
        case AC_ERR_NOT_FOUND: return "unknown id";
        case AC_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

}  // extern "C"
