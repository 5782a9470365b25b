// The serving loop declared in include/ac.h (ac_server_*): continuous batching
// of compacted-match requests over device-resident automata.
//
// One worker thread owns the GPU side.  Submissions go to a pending queue; the
// worker admits them in arrival order while the HBM budget allows, builds a
// wave from every admitted request not yet launched (at most max_wave), and
// enqueues it on the next free wave stream:
//   clear the per-unit match counts and tile counters; copy the wave's plan
//   (per automaton a head, the list of its texts with their first tile, each
//   text's output buffers) from pinned host memory; per automaton one
//   persistent matching launch in slot mode over all its texts' tiles; one
//   scan over all tiles of the wave; per automaton one gather launch that
//   writes each text's compacted list and count; an event.
// The worker polls the events of the waves in flight; a finished wave's
// requests move to the completion queue and give their budget back.  Up to
// waves_in_flight waves run at once, so a wave launched while another is on
// the GPU fills the SMs the other frees.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime_api.h>

#include "ac.h"
#include "pfac_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    ac_server_request r{};
    uint64_t bytes = 0;  // budget held while admitted
    double t_submit = 0.0, t_launch = 0.0;
};

// A wave slot: its stream, completion event, pinned staging for the plan
// (grown on demand), the requests of the wave it runs, and the wave's device
// scratch when it came from the caller's allocator (freed at completion).
struct WaveSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void *host = nullptr;
    size_t host_bytes = 0;
    bool busy = false;
    std::vector<Request> reqs;
    void *user_scratch = nullptr;
};

constexpr uint32_t kMaxWaves = 8;

size_t round256(size_t v) { return (v + 255u) & ~static_cast<size_t>(255u); }

}  // namespace

struct ac_server_impl {
    std::vector<ac_handle> hs;
    std::vector<const pfac::DevTables *> tabs;
    std::vector<pfac::Tuning> tune;
    int device = 0;
    bool multi = false;          // waves match all automata in one launch (filter kernel for all)
    uint64_t budget = 0;         // for requests: the option's budget less the automata's tables
    uint64_t table_bytes = 0;    // the resident automata (each handle once)
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    uint32_t max_wave = 0;
    uint32_t nslots = 0;
    bool fifo = false;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work;  // worker: new requests or stop
    std::condition_variable cv_done;  // pollers / drain: completions
    std::deque<Request> pending;
    std::deque<ac_server_completion> completed;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, finished = 0;
    bool stop = false;

    // worker-only state
    uint64_t inflight_bytes = 0;
    std::vector<WaveSlot> slots;
    std::thread worker;

    double now_us() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }
};

namespace {

// Positions per work unit of automaton a in the server's waves.
uint32_t tile_of(const ac_server_impl *s, uint32_t a) {
    return s->multi ? pfac::filter_tile_positions() : pfac::unit_positions(*s->tabs[a], s->tune[a]);
}

bool host_text(const ac_server_request &r) { return (r.flags & AC_REQ_HOST_TEXT) != 0; }

// The text's offset from a 16-byte boundary on the device: a host text is
// copied to a 16-byte aligned place.
uint64_t text_head(const ac_server_request &r) {
    return host_text(r) ? 0u : (reinterpret_cast<uintptr_t>(r.d_text) & 15u);
}

uint64_t units_of(const ac_server_impl *s, const ac_server_request &r) {
    if (r.n == 0) return 0;
    const uint64_t T = tile_of(s, r.automaton);
    return (r.n + text_head(r) + T - 1) / T;
}

// Whether automaton a's texts may take survivor lists for the phased form:
// 8-bit codes in one-launch waves, or (FIFO) as ac_match_compact takes them.
// (Small alphabets keep their dense fallback: the sets whose windows often
// end a keyword have tiles of many matches, which the gather would otherwise
// match again.)
bool wave_lists(const ac_server_impl *s, uint32_t a) { return (s->multi || s->fifo) && s->tabs[a]->B == 8; }

// Device bytes a request holds while admitted: its text (a host text's device
// copy), its output and the scratch of its tiles (counts, prefix, slots,
// dense fallback), and with 8-bit codes in one-launch waves its share of the
// wave's survivor lists (about 4 bytes per text byte).
uint64_t request_bytes(const ac_server_impl *s, const ac_server_request &r) {
    const uint64_t per_unit = 4 + 8 + 8ull * pfac::kSlotCap + 4ull * pfac::kDenseStride;
    const uint64_t lists = wave_lists(s, r.automaton) ? 32ull * (r.n / 8) + 32 : 0;
    return r.n + 8ull * r.cap + units_of(s, r) * per_unit + lists + 64;
}

// Device scratch of a wave: from the caller's allocator (freed when the wave
// completes) or the library pool (freed in stream order after the wave).
cudaError_t wave_alloc(ac_server_impl *s, WaveSlot &w, size_t bytes, void **out) {
    *out = nullptr;
    if (s->dev_alloc) {
        void *p = s->dev_alloc(bytes, s->alloc_ctx);
        if (!p) return cudaErrorMemoryAllocation;
        w.user_scratch = p;
        *out = p;
        return cudaSuccess;
    }
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pfac::scratch_pool(s->device, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(out, bytes, pool, w.stream);
}

cudaError_t wave_release(ac_server_impl *s, WaveSlot &w, void *p) {
    if (!p || s->dev_alloc) return cudaSuccess;  // caller's memory: freed at completion
    return cudaFreeAsync(p, w.stream);
}

inline size_t round16(size_t v) { return (v + 15u) & ~static_cast<size_t>(15u); }

cudaError_t ensure_host(WaveSlot &w, size_t bytes) {
    if (w.host_bytes >= bytes) return cudaSuccess;
    if (w.host) cudaFreeHost(w.host);
    w.host = nullptr;
    w.host_bytes = 0;
    const size_t want = std::max<size_t>(bytes, 1u << 20);
    cudaError_t e = cudaMallocHost(&w.host, want);
    if (e != cudaSuccess) return e;
    w.host_bytes = want;
    return cudaSuccess;
}

// Enqueue the wave in w.reqs on w's stream (worker thread).
cudaError_t launch_wave(ac_server_impl *s, WaveSlot &w) {
    const uint32_t nh = static_cast<uint32_t>(s->hs.size());
    const uint32_t R = static_cast<uint32_t>(w.reqs.size());
    cudaError_t e = cudaSuccess;

    if (s->fifo) {  // the comparison point: the single-text compacted path
        const Request &q = w.reqs[0];
        if (q.r.n == 0) return cudaMemsetAsync(q.r.d_count, 0, sizeof(uint64_t), w.stream);
        const pfac::DevTables &t = *s->tabs[q.r.automaton];
        const pfac::Tuning &tu = s->tune[q.r.automaton];
        // a host text: its copy at the front of the scratch (16-byte aligned)
        const size_t tb = host_text(q.r) ? round16(q.r.n) : 0;
        const uint32_t units = pfac::compact_units(t, tu, tb ? nullptr : q.r.d_text, q.r.n);
        // as ac_match_compact: the phased form's lists instead of the dense fallback when it applies
        pfac::SurvivorLists sl;
        if (pfac::uses_filter(t, tu)) sl = pfac::survivor_lists(t, tu, q.r.n, true);
        const bool dense = sl.list_cap == 0;
        const size_t bytes = tb + pfac::compact_scratch_bytes(t, units, dense) + sl.bytes();
        void *scratch = nullptr;
        e = wave_alloc(s, w, bytes, &scratch);
        if (e != cudaSuccess) return e;
        const uint8_t *text = q.r.d_text;
        if (tb) {
            e = cudaMemcpyAsync(scratch, q.r.d_text, q.r.n, cudaMemcpyHostToDevice, w.stream);
            text = static_cast<const uint8_t *>(scratch);
        }
        const pfac::CompactOut out{q.r.d_pos, q.r.d_ids, q.r.cap, reinterpret_cast<unsigned long long *>(q.r.d_count)};
        if (e == cudaSuccess)
            e = pfac::enqueue_compact(t, tu, text, q.r.n, out, static_cast<uint8_t *>(scratch) + tb, bytes - tb, dense,
                                      w.stream);
        const cudaError_t e2 = wave_release(s, w, scratch);
        return e != cudaSuccess ? e : e2;
    }

    // plan on the host: per automaton its texts in arrival order, their first
    // tile, and the automaton's first tile in the wave's numbering; host texts
    // get a 16-byte aligned place in the wave's scratch for their copies
    std::vector<uint32_t> order;
    order.reserve(R);
    std::vector<size_t> stage_off(R, 0);
    size_t staged = 0;
    for (uint32_t i = 0; i < R; ++i) {
        const ac_server_request &r = w.reqs[i].r;
        if (r.n == 0) {
            e = cudaMemsetAsync(r.d_count, 0, sizeof(uint64_t), w.stream);
            if (e != cudaSuccess) return e;
            continue;
        }
        order.push_back(i);
        if (host_text(r)) {
            stage_off[i] = staged;
            staged += round16(r.n);
        }
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return w.reqs[a].r.automaton < w.reqs[b].r.automaton; });
    const uint32_t L = static_cast<uint32_t>(order.size());
    if (L == 0) return cudaSuccess;
    std::vector<pfac::BatchHead> heads(nh);
    std::vector<uint32_t> ubase(nh, 0);
    std::vector<pfac::BatchItemDev> list(L);
    std::vector<pfac::CompactOut> outs(R);
    uint64_t U = 0;
    uint32_t j = 0;
    for (uint32_t a = 0; a < nh; ++a) {
        heads[a].offset = j;
        heads[a].pad = 0;
        ubase[a] = static_cast<uint32_t>(U);
        uint64_t units = 0;
        while (j < L && w.reqs[order[j]].r.automaton == a) {
            const ac_server_request &r = w.reqs[order[j]].r;
            pfac::BatchItemDev &d = list[j];
            d.len = r.n;
            d.out_off = 0;
            d.first_unit = static_cast<uint32_t>(units);
            d.item = order[j];
            units += units_of(s, r);
            ++j;
        }
        heads[a].count = j - heads[a].offset;
        heads[a].units = static_cast<uint32_t>(units);
        U += units;
    }
    if (U >= 0xFFFFFFFFull) return cudaErrorInvalidValue;
    for (uint32_t i = 0; i < R; ++i) {
        const ac_server_request &r = w.reqs[i].r;
        outs[i] = pfac::CompactOut{r.d_pos, r.d_ids, r.cap, reinterpret_cast<unsigned long long *>(r.d_count)};
    }

    // the survivor lists of the wave's 8-bit-code texts (the phased form of
    // the one launch), when they hold 4 MiB or more (below that the two extra
    // launches cost more than they save); with them those automata's units
    // keep no dense fallback (the gather matches a unit with more matches
    // than slots again), the others' do (and so list nothing)
    uint64_t list_text = 0;
    for (uint32_t k = 0; k < L; ++k)
        if (s->multi && wave_lists(s, w.reqs[order[k]].r.automaton)) list_text += w.reqs[order[k]].r.n;
    const uint32_t list_cap =
        list_text >= (4ull << 20) ? static_cast<uint32_t>(std::min<uint64_t>(list_text / 8, 0x7FFFFFF0ull)) : 0u;
    const size_t lsb = list_cap ? round256(pfac::multi_lists_bytes(list_cap)) : 0;
    auto dense_for = [&](uint32_t a, int32_t *d) -> int32_t * { return list_cap && wave_lists(s, a) ? nullptr : d; };

    // device: plan (heads | list | outs) | tile counters | counts | prefix |
    // slots | partial sums | dense fallback | host-text copies | survivor lists
    const size_t hb = sizeof(pfac::BatchHead) * nh, lb = sizeof(pfac::BatchItemDev) * L,
                 ob = sizeof(pfac::CompactOut) * R;
    const size_t plan_bytes = round256(hb) + round256(lb) + round256(ob);
    const size_t cb = round256(16ull * nh), nb = round256(4 * U), pb = 8 * U, sb = 8ull * pfac::kSlotCap * U;
    const size_t db = round256(plan_bytes + cb + nb + pb + sb + 8ull * pfac::kScanCtas);  // dense fallback: aligned
    const size_t stb = round256(db + 4ull * pfac::kDenseStride * U);
    void *dev = nullptr;
    e = wave_alloc(s, w, stb + round256(staged) + lsb, &dev);
    if (e != cudaSuccess) return e;
    uint8_t *dp = static_cast<uint8_t *>(dev);

    // the texts as the kernels see them: offsets from the lowest text address
    std::vector<const uint8_t *> ptr(L);
    const uint8_t *base = nullptr;
    for (uint32_t k = 0; k < L; ++k) {
        const ac_server_request &r = w.reqs[order[k]].r;
        ptr[k] = host_text(r) ? dp + stb + stage_off[order[k]] : r.d_text;
        if (!base || ptr[k] < base) base = ptr[k];
    }
    for (uint32_t k = 0; k < L; ++k)
        list[k].text_off = static_cast<uint64_t>(reinterpret_cast<uintptr_t>(ptr[k]) - reinterpret_cast<uintptr_t>(base));

    e = ensure_host(w, plan_bytes);
    if (e != cudaSuccess) {
        wave_release(s, w, dev);
        return e;
    }
    uint8_t *hp = static_cast<uint8_t *>(w.host);
    std::memcpy(hp, heads.data(), hb);
    std::memcpy(hp + round256(hb), list.data(), lb);
    std::memcpy(hp + round256(hb) + round256(lb), outs.data(), ob);

    const pfac::BatchHead *d_heads = reinterpret_cast<const pfac::BatchHead *>(dp);
    const pfac::BatchItemDev *d_list = reinterpret_cast<const pfac::BatchItemDev *>(dp + round256(hb));
    const pfac::CompactOut *d_outs = reinterpret_cast<const pfac::CompactOut *>(dp + round256(hb) + round256(lb));
    uint8_t *counters = dp + plan_bytes;
    uint32_t *counts = reinterpret_cast<uint32_t *>(counters + cb);
    unsigned long long *prefix = reinterpret_cast<unsigned long long *>(counters + cb + nb);
    unsigned long long *slots = prefix + U;
    unsigned long long *partials = slots + static_cast<size_t>(pfac::kSlotCap) * U;
    int32_t *dense = reinterpret_cast<int32_t *>(dp + db);
    void *surv_lists = list_cap ? static_cast<void *>(dp + stb + round256(staged)) : nullptr;

    e = cudaMemcpyAsync(dp, hp, plan_bytes, cudaMemcpyHostToDevice, w.stream);
    for (uint32_t k = 0; k < L && e == cudaSuccess; ++k) {  // host texts: one copy each
        const ac_server_request &r = w.reqs[order[k]].r;
        if (host_text(r)) e = cudaMemcpyAsync(const_cast<uint8_t *>(ptr[k]), r.d_text, r.n, cudaMemcpyHostToDevice,
                                              w.stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, cb + 4 * U, w.stream);
    if (e == cudaSuccess && surv_lists) e = cudaMemsetAsync(surv_lists, 0, 32, w.stream);
    if (s->multi && e == cudaSuccess) {  // every automaton of the wave in one launch
        std::vector<pfac::MatchRequest> rs(nh);
        for (uint32_t a = 0; a < nh; ++a) {
            pfac::MatchRequest &m = rs[a];
            m.text = base;
            m.batch = d_heads + a;
            m.lists = d_list;
            m.slots.counts = counts;
            m.slots.slots = slots;
            m.slots.ubase = ubase[a];
            m.slots.dense = dense_for(a, dense);
            m.scratch = counters + 16u * a;
            m.scratch_bytes = 16;
        }
        e = pfac::launch_filter_multi(s->tabs.data(), rs.data(), nh, pfac::OUT_SLOTS, s->tune[0].wait_ns, w.stream,
                                      surv_lists, list_cap);
    }
    for (uint32_t a = 0; a < nh && e == cudaSuccess && !s->multi; ++a) {
        if (heads[a].units == 0) continue;
        pfac::MatchRequest m;
        m.text = base;
        m.out = nullptr;
        m.batch = d_heads + a;
        m.lists = d_list;
        m.slots.counts = counts;
        m.slots.slots = slots;
        m.slots.ubase = ubase[a];
        m.slots.dense = dense;
        m.scratch = counters + 16u * a;
        m.scratch_bytes = 16;
        e = pfac::launch_match(*s->tabs[a], m, pfac::OUT_SLOTS, s->tune[a], w.stream);
    }
    if (e == cudaSuccess)
        e = pfac::launch_compact_scan(counts, static_cast<uint32_t>(U), nullptr, prefix, partials, w.stream);
    for (uint32_t a = 0; a < nh && e == cudaSuccess; ++a) {
        if (heads[a].units == 0) continue;
        pfac::GatherRequest g;
        g.text = base;
        g.batch = d_heads + a;
        g.lists = d_list;
        g.outs = d_outs;
        g.tile = tile_of(s, a);
        g.counts = counts;
        g.prefix = prefix;
        g.slots = slots;
        g.ubase = ubase[a];
        g.dense = dense_for(a, dense);
        e = pfac::launch_compact_gather(*s->tabs[a], g, w.stream);
    }
    const cudaError_t e2 = wave_release(s, w, dev);
    return e != cudaSuccess ? e : e2;
}

ac_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return AC_OK;
    if (e == cudaErrorMemoryAllocation) return AC_ERR_OOM;
    if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) return AC_ERR_INVALID_ARG;
    return AC_ERR_CUDA;
}

void complete_wave(ac_server_impl *s, WaveSlot &w, ac_status st, std::vector<ac_server_completion> &out) {
    if (w.user_scratch) {  // the wave's work is done: its scratch goes back to the caller's allocator
        s->dev_free(w.user_scratch, s->alloc_ctx);
        w.user_scratch = nullptr;
    }
    const double t = s->now_us();
    for (const Request &q : w.reqs) {
        ac_server_completion c;
        c.ticket = q.ticket;
        c.status = st;
        c.wave_size = static_cast<uint32_t>(w.reqs.size());
        c.t_submit_us = q.t_submit;
        c.t_launch_us = q.t_launch;
        c.t_done_us = t;
        out.push_back(c);
        s->inflight_bytes -= q.bytes;
    }
    w.reqs.clear();
    w.busy = false;
}

void worker_main(ac_server_impl *s) {
    cudaSetDevice(s->device);
    std::vector<ac_server_completion> done;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // 1. waves that finished
        lk.unlock();
        done.clear();
        bool busy = false;
        for (WaveSlot &w : s->slots) {
            if (!w.busy) continue;
            const cudaError_t q = cudaEventQuery(w.done);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            complete_wave(s, w, to_status(q), done);
        }
        lk.lock();
        if (!done.empty()) {
            for (const ac_server_completion &c : done) s->completed.push_back(c);
            s->finished += done.size();
            s->cv_done.notify_all();
        }
        // 2. admit and launch while a wave slot is free
        for (;;) {
            WaveSlot *w = nullptr;
            for (WaveSlot &x : s->slots)
                if (!x.busy) {
                    w = &x;
                    break;
                }
            if (!w || s->pending.empty()) break;
            const uint32_t cap = s->fifo ? 1u : s->max_wave;
            while (!s->pending.empty() && w->reqs.size() < cap &&
                   s->inflight_bytes + s->pending.front().bytes <= s->budget) {
                s->inflight_bytes += s->pending.front().bytes;
                w->reqs.push_back(s->pending.front());
                s->pending.pop_front();
            }
            if (w->reqs.empty()) break;  // the next request waits for budget
            lk.unlock();
            const double t = s->now_us();
            for (Request &q : w->reqs) q.t_launch = t;
            cudaError_t e = launch_wave(s, *w);
            if (e == cudaSuccess) e = cudaEventRecord(w->done, w->stream);
            w->busy = true;
            busy = true;
            if (e != cudaSuccess) {
                cudaGetLastError();
                cudaStreamSynchronize(w->stream);  // what was enqueued ends before its scratch is freed
                done.clear();
                complete_wave(s, *w, to_status(e), done);
                lk.lock();
                for (const ac_server_completion &c : done) s->completed.push_back(c);
                s->finished += done.size();
                s->cv_done.notify_all();
                continue;
            }
            lk.lock();
        }
        // 3. stop, sleep, or poll the GPU again
        if (s->stop && s->pending.empty() && !busy) break;
        if (!busy) {
            if (s->pending.empty()) s->cv_work.wait(lk);
            continue;
        }
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
    }
}

}  // namespace

extern "C" {

ac_status ac_server_destroy(ac_server s) {
    if (!s) return AC_OK;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    for (WaveSlot &w : s->slots) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        if (w.done) cudaEventDestroy(w.done);
        if (w.stream) cudaStreamDestroy(w.stream);
        if (w.host) cudaFreeHost(w.host);
    }
    delete s;
    return AC_OK;
}

ac_status ac_server_create(const ac_handle *hs, uint32_t nh, const ac_server_options *opt, ac_server *out) {
    if (!out) return AC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!hs || nh == 0 || nh > pfac::kMaxBatchAutomata) return AC_ERR_INVALID_ARG;
    ac_server_options o;
    std::memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return AC_ERR_CUDA;
    ac_server s = new (std::nothrow) ac_server_impl();
    if (!s) return AC_ERR_OOM;
    s->device = cur;
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr) || o.reserved != 0) {
        delete s;
        return AC_ERR_INVALID_ARG;
    }
    s->dev_alloc = o.dev_alloc;
    s->dev_free = o.dev_free;
    s->alloc_ctx = o.alloc_ctx;
    for (uint32_t a = 0; a < nh; ++a) {
        int dev = -1;
        bool host_only = true;
        const pfac::DevTables *t = pfac::handle_tables(hs[a], &dev, &host_only);
        if (!t || host_only || dev != cur) {
            delete s;
            return AC_ERR_INVALID_ARG;
        }
        bool seen = false;  // a handle named twice is resident once
        for (uint32_t b = 0; b < a; ++b) seen = seen || hs[b] == hs[a];
        if (!seen) {
            ac_info_t info;
            ac_info(hs[a], &info);
            s->table_bytes += info.table_bytes;
        }
        s->hs.push_back(hs[a]);
        s->tabs.push_back(t);
        s->tune.push_back(*pfac::handle_tuning(hs[a]));
    }
    const uint64_t budget = o.hbm_budget ? o.hbm_budget : (40ull << 30);
    if (s->table_bytes >= budget) {
        delete s;
        return AC_ERR_BUDGET;
    }
    s->budget = budget - s->table_bytes;
    s->max_wave = o.max_wave ? o.max_wave : 4096u;
    s->fifo = o.fifo != 0;
    s->multi = !s->fifo && pfac::filter_multi_serves(s->tabs.data(), nh);
    uint32_t nw = o.waves_in_flight ? o.waves_in_flight : 2u;
    if (nw > kMaxWaves) nw = kMaxWaves;
    if (s->fifo) nw = 1;
    s->nslots = nw;
    s->slots.resize(nw);
    for (WaveSlot &w : s->slots) {
        if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ac_server_destroy(s);
            return AC_ERR_CUDA;
        }
    }
    s->t0 = Clock::now();
    s->worker = std::thread(worker_main, s);
    *out = s;
    return AC_OK;
}

ac_status ac_server_submit(ac_server s, const ac_server_request *req, uint64_t *ticket) {
    if (!s || !req) return AC_ERR_INVALID_ARG;
    const ac_server_request &r = *req;
    if (r.automaton >= s->hs.size() || !r.d_count || r.n > 0xFFFFFFFFull || (r.flags & ~AC_REQ_HOST_TEXT))
        return AC_ERR_INVALID_ARG;
    if (r.n > 0 && !r.d_text) return AC_ERR_INVALID_ARG;
    if (r.cap > 0 && (!r.d_pos || !r.d_ids)) return AC_ERR_INVALID_ARG;
    Request q;
    q.r = r;
    q.bytes = request_bytes(s, r);
    if (q.bytes > s->budget) return AC_ERR_BUDGET;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q.ticket = s->next_ticket++;
        q.t_submit = s->now_us();
        s->pending.push_back(q);
        ++s->submitted;
    }
    s->cv_work.notify_one();
    if (ticket) *ticket = q.ticket;
    return AC_OK;
}

ac_status ac_server_replay(ac_server s, const ac_server_request *reqs, uint32_t n, const double *arrival_us,
                           uint64_t *tickets) {
    if (!s || (n > 0 && (!reqs || !arrival_us))) return AC_ERR_INVALID_ARG;
    const Clock::time_point start = Clock::now();
    for (uint32_t i = 0; i < n; ++i) {
        const Clock::time_point due =
            start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double, std::micro>(arrival_us[i]));
        while (Clock::now() < due) {
        }
        const ac_status st = ac_server_submit(s, &reqs[i], tickets ? &tickets[i] : nullptr);
        if (st != AC_OK) return st;
    }
    return AC_OK;
}

ac_status ac_server_poll(ac_server s, ac_server_completion *out, uint32_t max, uint32_t *n_out, uint32_t wait_us) {
    if (!s || !n_out || (max > 0 && !out)) return AC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->completed.empty() && wait_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !s->completed.empty(); });
    uint32_t k = 0;
    while (k < max && !s->completed.empty()) {
        out[k++] = s->completed.front();
        s->completed.pop_front();
    }
    *n_out = k;
    return AC_OK;
}

ac_status ac_server_drain(ac_server s) {
    if (!s) return AC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->finished >= s->submitted; });
    return AC_OK;
}

ac_status ac_server_cancel(ac_server s, uint64_t ticket) {
    if (!s) return AC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if (it->ticket != ticket) continue;
        ac_server_completion c;
        c.ticket = ticket;
        c.status = AC_ERR_CANCELLED;
        c.wave_size = 0;
        c.t_submit_us = it->t_submit;
        c.t_launch_us = c.t_done_us = s->now_us();
        s->pending.erase(it);
        s->completed.push_back(c);
        ++s->finished;
        s->cv_done.notify_all();
        return AC_OK;
    }
    return AC_ERR_NOT_FOUND;
}

}  // extern "C"
