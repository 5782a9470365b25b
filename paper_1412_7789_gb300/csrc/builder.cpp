// Host automaton builder: keyword set -> failureless goto table (paper section
// II: the goto function of the pattern matching machine, stored as a matrix
// for the GPU and used without failure transitions, Fig. 5).
//
// Steps, in order:
//   1. class map: each byte that occurs in a keyword gets a code 0..C-1 (in byte
//      order); other bytes can never extend a walk.
//   2. trie insertion of every keyword (the goto function), one subtrie per
//      first code on the host's threads;
//   3. breadth-first renumbering, children in code order, so depth d occupies
//      a contiguous id range and the hot upper levels form a prefix (each
//      subtrie's BFS on its own thread, then joined depth by depth);
//   4. per state, the longest keyword that is a prefix of the state's string
//      (the output a walk ending there reports; equal strings -> lowest id);
//   5. the dense table, one row per state: C goto columns plus one end column,
//      where a missing transition holds the encoded result of stopping there;
//   6. the top k levels of the table flattened, for the kernels' first lookup:
//      for small alphabets (2- or 4-bit codes) a filter bit per window of k
//      codes (clear: the walk stops inside the window with no keyword) plus
//      the window table (depth-k state reached, or the encoded result); for
//      8-bit codes the root jump table (result, or depth-k state, per window),
//      and a hashed filter over windows of kh codes with a hash of the
//      depth-kh states by their window;
//   7. the stride table: the depth-(k+k2) state or the result, for k2 more
//      codes from every depth-k state;
//   8. chain records for the deep, mostly unbranched states;
//   9. the full-output records: for each keyword, the keywords that are
//      prefixes of it (its sub-patterns on any walk that reaches it).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <thread>

#include "ac.h"
#include "pfac_internal.h"

namespace pfac {

namespace {

struct Edge {
    uint32_t parent;
    uint32_t code;
    uint32_t child;
};

inline uint32_t code_bits_for(uint32_t C) { return C <= 4 ? 2u : (C <= 16 ? 4u : 8u); }

template <typename T>
inline int32_t g_at(const HostTables &h, uint64_t idx) {
    return static_cast<int32_t>(reinterpret_cast<const T *>(h.G.data())[idx]);
}

// The children of the trie under construction: open addressing over keys
// (state << 8) | code with linear probing, Knuth's multiplicative hash, and a
// doubling of the table once it is half full.
class ChildTable {
public:
    explicit ChildTable(uint64_t expect) {
        uint32_t bits = 6;
        while ((1ull << bits) < 2 * expect) ++bits;
        rebuild(bits);
    }
    // The child stored under key; if none, t is stored and *inserted set.
    uint32_t find_or_insert(uint64_t key, uint32_t t, bool *inserted) {
        if ((used_ + 1) * 2 > keys_.size()) rebuild(bits_ + 1);
        const uint64_t mask = keys_.size() - 1;
        for (uint64_t i = slot(key);; i = (i + 1) & mask) {
            if (keys_[i] == kEmpty) {
                keys_[i] = key;
                vals_[i] = t;
                ++used_;
                *inserted = true;
                return t;
            }
            if (keys_[i] == key) {
                *inserted = false;
                return vals_[i];
            }
        }
    }

private:
    static constexpr uint64_t kEmpty = ~0ull;  // keys are below 2^39
    uint64_t slot(uint64_t key) const { return (key * 0x9E3779B97F4A7C15ull) >> (64 - bits_); }
    void rebuild(uint32_t bits) {
        std::vector<uint64_t> ok;
        std::vector<uint32_t> ov;
        ok.swap(keys_);
        ov.swap(vals_);
        bits_ = bits;
        keys_.assign(1ull << bits, kEmpty);
        vals_.assign(1ull << bits, 0u);
        used_ = 0;
        const uint64_t mask = keys_.size() - 1;
        for (uint64_t j = 0; j < ok.size(); ++j) {
            if (ok[j] == kEmpty) continue;
            uint64_t i = slot(ok[j]);
            while (keys_[i] != kEmpty) i = (i + 1) & mask;
            keys_[i] = ok[j];
            vals_[i] = ov[j];
            ++used_;
        }
    }
    std::vector<uint64_t> keys_;
    std::vector<uint32_t> vals_;
    uint64_t used_ = 0;
    uint32_t bits_ = 0;
};

// body(lo, hi) over [0, n) in contiguous ranges on up to the machine's
// hardware threads (at least min_per_thread items each).  Callers write
// disjoint parts of their outputs, so results never depend on the split; a
// range whose thread cannot be started runs on the calling thread.
template <typename F>
void parallel_ranges(uint64_t n, uint64_t min_per_thread, F body) {
    uint64_t t = std::thread::hardware_concurrency();
    t = std::min<uint64_t>(std::max<uint64_t>(t, 1), 32);
    t = std::min<uint64_t>(t, std::max<uint64_t>(1, n / std::max<uint64_t>(min_per_thread, 1)));
    if (t <= 1) {
        body(uint64_t{0}, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(t);
    for (uint64_t i = 0; i < t; ++i) {
        const uint64_t lo = n * i / t, hi = n * (i + 1) / t;
        try {
            th.emplace_back(body, lo, hi);
        } catch (...) {
            body(lo, hi);
        }
    }
    for (std::thread &x : th) x.join();
}

// body(i) for every task i in [0, n), the tasks taken in order by up to the
// host's thread count (at most 32) through a shared counter.
template <typename F>
void parallel_tasks(uint32_t n, F body) {
    uint64_t t = std::thread::hardware_concurrency();
    t = std::min<uint64_t>(std::min<uint64_t>(std::max<uint64_t>(t, 1), 32), n);
    std::atomic<uint32_t> next{0};
    auto run = [&]() {
        for (uint32_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) body(i);
    };
    if (t <= 1) {
        run();
        return;
    }
    std::vector<std::thread> th;
    th.reserve(t);
    for (uint64_t i = 0; i < t; ++i) {
        try {
            th.emplace_back(run);
        } catch (...) {
            break;  // the threads started (or this one, below) take the rest
        }
    }
    run();
    for (std::thread &x : th) x.join();
}

inline int32_t goto_entry(const HostTables &h, uint32_t s, uint32_t c) {
    uint64_t idx = static_cast<uint64_t>(s) * h.W + c;
    return h.gbits == 16 ? g_at<int16_t>(h, idx) : g_at<int32_t>(h, idx);
}

// Walk `len` codes of window w (first code in the low bits) from state s:
// true with the state reached, or false with the encoded result where the
// walk stopped.  A code >= C (a byte in no keyword) reads the end column,
// which holds every state's encoded result.
bool walk_window(const HostTables &h, uint32_t s, uint32_t w, uint32_t len, int32_t *out) {
    const uint32_t cmask = (1u << h.B) - 1u;
    for (uint32_t i = 0; i < len; ++i) {
        const uint32_t c = (w >> (h.B * i)) & cmask;
        const int32_t t = goto_entry(h, s, c < h.C ? c : h.C);
        if (t < 0) {
            *out = t;
            return false;
        }
        s = static_cast<uint32_t>(t);
    }
    *out = static_cast<int32_t>(s);
    return true;
}

uint32_t first_state_at(const HostTables &h, uint32_t d) {
    uint32_t b = 0;
    for (uint32_t i = 0; i < d && i < h.depth_count.size(); ++i) b += h.depth_count[i];
    return b;
}

// Step 7: the stride table from the depth-k states: the deepest k2 >= 2 whose
// table fits stride_bytes (k + k2 codes in the kernel's window), each entry
// the walk of its k2 codes from its state.
void stride_rows(const HostTables &h, RootTables *rt, uint64_t stride_bytes) {
    rt->k2 = 0;
    rt->J2.clear();
    if (rt->k == 0 || stride_bytes <= 1 || rt->k >= h.maxlen) return;
    const uint32_t wl = window_limit(h.B);
    if (rt->k >= wl) return;
    const uint32_t top = std::min(h.maxlen - rt->k, wl - rt->k);
    for (uint32_t cand = top; cand >= 2; --cand) {
        if (h.B * cand >= 32) continue;
        const uint64_t bytes = (static_cast<uint64_t>(rt->count_k) << (h.B * cand)) * 4ull;
        if (bytes <= stride_bytes) {
            rt->k2 = cand;
            break;
        }
    }
    if (rt->k2 == 0) return;
    const uint32_t cols = 1u << (h.B * rt->k2);
    rt->J2.assign(static_cast<size_t>(rt->count_k) * cols, 0);
    for (uint32_t r = 0; r < rt->count_k; ++r)
        for (uint32_t w = 0; w < cols; ++w) {
            int32_t e = 0;
            walk_window(h, rt->base_k + r, w, rt->k2, &e);
            rt->J2[static_cast<size_t>(r) * cols + w] = e;
        }
}

}  // namespace

uint32_t filter_window(uint32_t B, uint32_t maxlen, uint32_t bytes) {
    uint32_t fbits = 0;  // largest filter (in bits) that fits the budget
    while (fbits < kFilterBits && (2ull << fbits) <= 8ull * bytes) ++fbits;
    return std::max<uint32_t>(1u, std::min<uint32_t>(maxlen, fbits / B));
}

void window_tables(const HostTables &h, uint32_t k, uint64_t stride_bytes, RootTables *rt) {
    // Step 6a: for every window of k codes, one filter bit that is clear when
    // the walk from the root stops inside the window with no keyword found
    // (the start's result is -1), and the window table: the depth-k state
    // reached, or the encoded result where the walk stopped.
    rt->k = k;
    rt->base_k = first_state_at(h, k);
    rt->count_k = k < h.depth_count.size() ? h.depth_count[k] : 0u;
    rt->fbits = 0;
    const uint32_t nwin = 1u << (h.B * k);
    // The bit of window w is bit 31 - (w & 31) of word w >> 5 (the kernel
    // rotates it to bit 31); windows of fewer than 5 bits are repeated over
    // the 32 bits of word 0, as the kernel indexes by the low 5 bits of the
    // code stream.
    rt->F.assign(std::max<uint32_t>(nwin / 32u, 4u), 0u);
    rt->JK.assign(nwin, 0);
    uint64_t found = 0;
    for (uint32_t w = 0; w < nwin; ++w) {
        int32_t e = 0;
        const bool alive = walk_window(h, 0, w, k, &e);
        rt->JK[w] = e;
        found += e < -1 ? 1u : 0u;
        if (alive || e < -1)
            for (uint32_t v = w; v < std::max<uint32_t>(nwin, 32u); v += nwin) rt->F[v >> 5] |= 1u << (31u - (v & 31u));
    }
    rt->match_windows_ppm = static_cast<uint32_t>(found * 1000000ull / nwin);
    stride_rows(h, rt, stride_bytes);
}

void hashed_filter(const HostTables &h, uint32_t fbits, RootTables *rt) {
    rt->fbits = fbits;
    rt->F.assign((1u << fbits) / 32u, 0u);
    for (size_t b = 0; b + 3 < h.HK.size(); b += 4) {
        if (h.HK[b + 1] == 0u) continue;  // an empty entry
        const uint32_t f = (h.HK[b] * kFilterHashMul) >> (32u - fbits);
        rt->F[f >> 5] |= 1u << (31u - (f & 31u));
    }
}

int build_tables(const uint8_t *const *patterns, const uint32_t *lens, uint32_t nkw,
                 const BuildOptions &opt, HostTables *out) {
    if (!out || !patterns || !lens) return AC_ERR_INVALID_ARG;
    if (nkw == 0) return AC_ERR_EMPTY_PATTERN;
    if (nkw > 0x7FFFFFF0u) return AC_ERR_INVALID_ARG;
    HostTables h;
    h.nkw = nkw;
    uint64_t total = 0;
    h.minlen = UINT32_MAX;
    for (uint32_t i = 0; i < nkw; ++i) {
        if (lens[i] == 0) return AC_ERR_EMPTY_PATTERN;
        if (!patterns[i]) return AC_ERR_INVALID_ARG;
        total += lens[i];
        h.minlen = std::min(h.minlen, lens[i]);
        h.maxlen = std::max(h.maxlen, lens[i]);
    }
    if (total + 1 > 0x7FFFFFFFull) return AC_ERR_TOO_MANY_STATES;

    try {
        // 1. class map
        h.cls.assign(256, -1);
        if (opt.class_compress) {
            bool present[256] = {false};
            for (uint32_t i = 0; i < nkw; ++i)
                for (uint32_t j = 0; j < lens[i]; ++j) present[patterns[i][j]] = true;
            int16_t c = 0;
            for (int b = 0; b < 256; ++b)
                if (present[b]) h.cls[b] = c++;
            h.C = static_cast<uint32_t>(c);
        } else {
            for (int b = 0; b < 256; ++b) h.cls[b] = static_cast<int16_t>(b);
            h.C = 256;
        }
        // four keyword bytes that (byte >> 1) & 3 tells apart (the DNA
        // letters in either case): that value becomes their class code
        h.direct_shift = -1;
        if (h.C == 4) {
            int seen[4] = {-1, -1, -1, -1};
            bool ok = true;
            for (int b = 0; b < 256 && ok; ++b) {
                if (h.cls[b] < 0) continue;
                const int v = (b >> 1) & 3;
                if (seen[v] >= 0) ok = false;
                seen[v] = b;
            }
            if (ok) {
                h.direct_shift = 1;
                for (int v = 0; v < 4; ++v) {
                    h.direct_byte[v] = static_cast<uint8_t>(seen[v]);
                    h.cls[seen[v]] = static_cast<int16_t>(v);
                }
            }
        }
        h.cls8.assign(256, 0xFF);
        for (int b = 0; b < 256; ++b)
            if (h.cls[b] >= 0) h.cls8[b] = static_cast<uint8_t>(h.cls[b]);
        // a 3-bit hash of the byte that separates the keyword bytes lets the
        // kernel classify four bytes at a time with byte permutes
        h.hash_shift = -1;
        if (h.C <= 8) {
            for (int sh = 0; sh <= 5 && h.hash_shift < 0; ++sh) {
                int seen[8];
                for (int v = 0; v < 8; ++v) seen[v] = -1;
                bool ok = true;
                for (int b = 0; b < 256 && ok; ++b) {
                    if (h.cls[b] < 0) continue;
                    const int hv = (b >> sh) & 7;
                    if (seen[hv] >= 0) ok = false;
                    seen[hv] = b;
                }
                if (!ok) continue;
                h.hash_shift = sh;
                for (int v = 0; v < 8; ++v) {
                    if (seen[v] >= 0) {
                        h.hash_code[v] = static_cast<uint8_t>(h.cls[seen[v]]);
                        h.hash_byte[v] = static_cast<uint8_t>(seen[v]);
                    } else {
                        h.hash_code[v] = 0;
                        h.hash_byte[v] = static_cast<uint8_t>((v ^ 1) << sh);  // hashes to v ^ 1
                    }
                }
            }
        }

        // 2. trie insertion.  The keywords are grouped by their first code:
        //    the subtries below the root's children are disjoint, so each
        //    group's subtrie is built by one thread, its keywords in increasing
        //    id (so a state's first keyword is its lowest).  Provisional ids:
        //    the root, then one block per group in code order, a group's
        //    depth-1 state first.
        std::vector<uint32_t> gstart(h.C + 1, 0);  // keywords of first code c: gids[gstart[c] .. gstart[c + 1])
        for (uint32_t id = 0; id < nkw; ++id) gstart[static_cast<uint32_t>(h.cls[patterns[id][0]]) + 1]++;
        for (uint32_t c = 0; c < h.C; ++c) gstart[c + 1] += gstart[c];
        std::vector<uint32_t> gids(nkw);
        {
            std::vector<uint32_t> fill(gstart.begin(), gstart.end() - 1);
            for (uint32_t id = 0; id < nkw; ++id) gids[fill[static_cast<uint32_t>(h.cls[patterns[id][0]])]++] = id;
        }
        std::vector<uint32_t> groups;  // first codes that start a keyword, largest group first
        std::vector<uint64_t> glen(h.C, 0);
        for (uint32_t c = 0; c < h.C; ++c) {
            for (uint32_t i = gstart[c]; i < gstart[c + 1]; ++i) glen[c] += lens[gids[i]];
            if (gstart[c + 1] > gstart[c]) groups.push_back(c);
        }
        std::sort(groups.begin(), groups.end(), [&](uint32_t a, uint32_t b) {
            return glen[a] != glen[b] ? glen[a] > glen[b] : a < b;
        });
        struct Subtrie {
            std::vector<int32_t> kw_at;  // local id -> lowest keyword id ending there (local 0: the depth-1 state)
            std::vector<Edge> edges;     // local ids
        };
        std::vector<Subtrie> sub(h.C);
        std::vector<uint32_t> kw_state(nkw);  // each keyword's state: local id first, then provisional
        std::atomic<bool> oom{false};
        parallel_tasks(static_cast<uint32_t>(groups.size()), [&](uint32_t gi) {
            const uint32_t c0 = groups[gi];
            try {
                Subtrie &t = sub[c0];
                const uint64_t expect = std::min<uint64_t>(glen[c0], 1ull << 26) + 16;
                ChildTable child(expect);
                t.kw_at.assign(1, -1);
                t.edges.reserve(static_cast<size_t>(expect));
                for (uint32_t i = gstart[c0]; i < gstart[c0 + 1]; ++i) {
                    const uint32_t id = gids[i];
                    uint32_t s = 0;
                    for (uint32_t j = 1; j < lens[id]; ++j) {
                        const uint32_t c = static_cast<uint32_t>(h.cls[patterns[id][j]]);
                        const uint64_t key = (static_cast<uint64_t>(s) << 8) | c;
                        bool inserted = false;
                        const uint32_t u = child.find_or_insert(key, static_cast<uint32_t>(t.kw_at.size()), &inserted);
                        if (inserted) {
                            t.kw_at.push_back(-1);
                            t.edges.push_back({s, c, u});
                        }
                        s = u;
                    }
                    if (t.kw_at[s] < 0) t.kw_at[s] = static_cast<int32_t>(id);
                    kw_state[id] = s;
                }
            } catch (const std::bad_alloc &) {
                oom = true;
            }
        });
        if (oom) return AC_ERR_OOM;
        std::vector<uint32_t> goff(h.C, 0), eoff(h.C, 0);  // each group's first provisional id, first edge
        uint64_t S64 = 1, E64 = 0;
        for (uint32_t c = 0; c < h.C; ++c) {
            if (gstart[c + 1] == gstart[c]) continue;
            goff[c] = static_cast<uint32_t>(S64);
            eoff[c] = static_cast<uint32_t>(E64);
            S64 += sub[c].kw_at.size();
            E64 += sub[c].edges.size() + 1;  // its edges and the root's edge into it
        }
        if (S64 > 0x7FFFFFF0ull) return AC_ERR_TOO_MANY_STATES;
        const uint32_t S = static_cast<uint32_t>(S64);
        h.S = S;
        std::vector<int32_t> kw_at(S, -1);  // lowest keyword id ending at each provisional state
        std::vector<Edge> edges(static_cast<size_t>(E64));
        parallel_tasks(static_cast<uint32_t>(groups.size()), [&](uint32_t gi) {
            const uint32_t c0 = groups[gi], o = goff[c0];
            Subtrie &t = sub[c0];
            std::copy(t.kw_at.begin(), t.kw_at.end(), kw_at.begin() + o);
            Edge *e = edges.data() + eoff[c0];
            e[0] = {0u, c0, o};
            for (size_t i = 0; i < t.edges.size(); ++i) e[i + 1] = {t.edges[i].parent + o, t.edges[i].code, t.edges[i].child + o};
            for (uint32_t i = gstart[c0]; i < gstart[c0 + 1]; ++i) kw_state[gids[i]] += o;
            std::vector<int32_t>().swap(t.kw_at);
            std::vector<Edge>().swap(t.edges);
        });

        // 3. breadth-first renumbering with children in code order.  At every
        //    depth the states of group c come after those of every group of a
        //    lower code (a BFS keeps its parents' order, and the depth-1 states
        //    are in code order), so each group's BFS runs on its own thread and
        //    a state's new id is: the states above its depth, those of the
        //    lower groups at its depth, then its rank in its group's BFS at
        //    that depth.
        std::vector<uint32_t> first(S + 1, 0);
        for (const Edge &e : edges) first[e.parent + 1]++;
        for (uint32_t s = 0; s < S; ++s) first[s + 1] += first[s];
        std::vector<uint32_t> adj(edges.size());
        {
            std::vector<uint32_t> fill(first.begin(), first.end() - 1);
            for (uint32_t i = 0; i < edges.size(); ++i) adj[fill[edges[i].parent]++] = i;
        }
        parallel_ranges(S, 16384, [&](uint64_t s0, uint64_t s1) {
            for (uint64_t s = s0; s < s1; ++s)
                if (first[s + 1] - first[s] > 1)
                    std::sort(adj.begin() + first[s], adj.begin() + first[s + 1],
                              [&](uint32_t a, uint32_t b) { return edges[a].code < edges[b].code; });
        });
        const uint32_t D = h.maxlen + 1;
        std::vector<std::vector<uint32_t>> seq(h.C);     // each group's BFS: edge index into each state
        std::vector<std::vector<uint32_t>> level(h.C);   // ... and where each depth starts in it (D + 1 entries)
        parallel_tasks(static_cast<uint32_t>(groups.size()), [&](uint32_t gi) {
            const uint32_t c0 = groups[gi];
            std::vector<uint32_t> &q = seq[c0];
            std::vector<uint32_t> &lv = level[c0];
            try {
                q.push_back(eoff[c0]);  // the root's edge into the group
                lv.assign(D + 1, 0);
                uint32_t d = 1;
                size_t end_of_level = 1;
                for (size_t qi = 0; qi < q.size(); ++qi) {
                    if (qi == end_of_level) {  // every state of the next depth is queued
                        ++d;
                        lv[d] = static_cast<uint32_t>(qi);
                        end_of_level = q.size();
                    }
                    const uint32_t old = edges[q[qi]].child;
                    for (uint32_t a = first[old]; a < first[old + 1]; ++a) q.push_back(adj[a]);
                }
                for (uint32_t e = d + 1; e <= D; ++e) lv[e] = static_cast<uint32_t>(q.size());
            } catch (const std::bad_alloc &) {
                oom = true;
            }
        });
        if (oom) return AC_ERR_OOM;
        // states per depth, and each group's first rank at each depth
        h.depth_count.assign(D, 0);
        h.depth_count[0] = 1;
        std::vector<uint32_t> gbase(static_cast<size_t>(h.C) * D, 0);
        {
            std::vector<uint64_t> run(D, 0);
            for (uint32_t c = 0; c < h.C; ++c) {
                if (gstart[c + 1] == gstart[c]) continue;
                const std::vector<uint32_t> &lv = level[c];
                for (uint32_t d = 1; d < D; ++d) {
                    const uint32_t n_at = (d + 1 <= D ? lv[d + 1] : static_cast<uint32_t>(seq[c].size())) - lv[d];
                    gbase[static_cast<size_t>(c) * D + d] = static_cast<uint32_t>(run[d]);
                    run[d] += n_at;
                }
            }
            for (uint32_t d = 1; d < D; ++d) h.depth_count[d] = static_cast<uint32_t>(run[d]);
        }
        std::vector<uint32_t> dbase(D + 1, 0);  // first new id at each depth
        for (uint32_t d = 0; d < D; ++d) dbase[d + 1] = dbase[d] + h.depth_count[d];
        std::vector<uint32_t> order(S);        // new id -> provisional id
        std::vector<uint32_t> newid(S, 0);
        std::vector<uint32_t> depth(S, 0);     // by new id
        std::vector<uint32_t> parent(S, 0);    // by new id
        std::vector<uint32_t> incode(S, 0);    // by new id: the code of the edge into the state
        order[0] = 0;
        parallel_tasks(static_cast<uint32_t>(groups.size()), [&](uint32_t gi) {
            const uint32_t c0 = groups[gi];
            const std::vector<uint32_t> &q = seq[c0];
            const std::vector<uint32_t> &lv = level[c0];
            uint32_t d = 1;
            for (size_t qi = 0; qi < q.size(); ++qi) {
                while (d + 1 < D && qi >= lv[d + 1]) ++d;
                const Edge &e = edges[q[qi]];
                const uint32_t nid = dbase[d] + gbase[static_cast<size_t>(c0) * D + d] + static_cast<uint32_t>(qi - lv[d]);
                newid[e.child] = nid;  // a parent's new id is set before its children's (BFS order)
                order[nid] = e.child;
                depth[nid] = d;
                parent[nid] = newid[e.parent];
                incode[nid] = e.code;
            }
            std::vector<uint32_t>().swap(seq[c0]);
        });

        // 4. longest keyword on the path to each state (BFS order: parents first)
        std::vector<int32_t> pathbest(S, -1);
        for (uint32_t s = 1; s < S; ++s) {
            int32_t own = kw_at[order[s]];
            pathbest[s] = own >= 0 ? own : pathbest[parent[s]];
        }

        // 5. dense goto table
        h.W = (h.C + 1 <= 8) ? 8u : h.C + 1;
        bool fits16 = (S <= 32768u) && (nkw <= 32767u);
        if (opt.index_width == 16 && !fits16) return AC_ERR_INVALID_ARG;
        h.gbits = (opt.index_width == 32 || !fits16) ? 32u : 16u;
        const uint64_t cells = static_cast<uint64_t>(S) * h.W;
        h.G.resize_unfilled(cells * (h.gbits / 8));  // every row is filled below
        auto put = [&](uint64_t idx, int32_t v) {
            if (h.gbits == 16)
                reinterpret_cast<int16_t *>(h.G.data())[idx] = static_cast<int16_t>(v);
            else
                reinterpret_cast<int32_t *>(h.G.data())[idx] = v;
        };
        std::vector<uint32_t> kids(S, 0), child1(S, 0);  // children; the first child
        std::vector<uint8_t> code1(S, 0);                 // its code
        // rows in parallel (each range writes its own rows and entries)
        parallel_ranges(S, 4096, [&](uint64_t s0, uint64_t s1) {
            for (uint64_t s = s0; s < s1; ++s) {
                const int32_t dead = encode_dead(pathbest[s]);
                const uint64_t row = s * h.W;
                if (h.gbits == 16)
                    std::fill_n(reinterpret_cast<int16_t *>(h.G.data()) + row, h.W, static_cast<int16_t>(dead));
                else
                    std::fill_n(reinterpret_cast<int32_t *>(h.G.data()) + row, h.W, dead);
                const uint32_t old = order[s];
                kids[s] = first[old + 1] - first[old];
                for (uint32_t a = first[old]; a < first[old + 1]; ++a) {
                    const Edge &e = edges[adj[a]];
                    put(row + e.code, static_cast<int32_t>(newid[e.child]));
                    if (a == first[old]) {
                        child1[s] = newid[e.child];
                        code1[s] = static_cast<uint8_t>(e.code);
                    }
                }
            }
        });
        std::vector<Edge>().swap(edges);

        h.B = code_bits_for(h.C);
        const uint32_t wl = window_limit(h.B);
        const uint32_t cmask = (1u << h.B) - 1u;
        std::vector<uint32_t> depth_base(h.maxlen + 2, 0);
        for (uint32_t d = 0; d <= h.maxlen; ++d) depth_base[d + 1] = depth_base[d] + h.depth_count[d];
        // Walk `len` codes of window w (first code in the low bits) from state s:
        // true with the state reached, or false with the encoded result where the
        // walk stopped (codes >= C stop it like a byte in no keyword).
        auto walk_codes = [&](uint32_t s, uint32_t w, uint32_t len, int32_t *out) -> bool {
            for (uint32_t i = 0; i < len; ++i) {
                const uint32_t c = (w >> (h.B * i)) & cmask;
                const int32_t t = c < h.C ? goto_entry(h, s, c) : encode_dead(pathbest[s]);
                if (t < 0) {
                    *out = t;
                    return false;
                }
                s = static_cast<uint32_t>(t);
            }
            *out = static_cast<int32_t>(s);
            return true;
        };

        if (h.B <= 4) {
            // 6a. root filter (2- and 4-bit codes): for every window of kf codes,
            //     one bit that is clear when the walk from the root stops inside
            //     the window with no keyword found (the start's result is -1), and
            //     the window table: the depth-kf state reached, or the encoded
            //     result where the walk stopped.
            //     (window_tables; step 7 with it)
            h.filter = true;
            RootTables rt;
            window_tables(h, filter_window(h.B, h.maxlen, opt.jump_bytes), opt.stride_bytes, &rt);
            h.k = rt.k;
            h.base_k = rt.base_k;
            h.count_k = rt.count_k;
            h.k2 = rt.k2;
            h.match_windows_ppm = rt.match_windows_ppm;
            h.F = std::move(rt.F);
            h.JK = std::move(rt.JK);
            h.J2 = std::move(rt.J2);
        } else {
            // 6b. root jump table (8-bit codes).  Entry for a window of k codes:
            //     the walk's result (>= -1) when it stops inside the window, else
            //     -(2 + s - base_k) for the depth-k state s reached; kJumpSlow
            //     when a result does not fit 15 bits.
            uint32_t jentries = std::max<uint32_t>(opt.jump_bytes, 2u) / 2u;
            uint32_t kj = 0;
            while (kj + 1 <= h.maxlen && kj + 1 <= wl && h.B * (kj + 1) <= 16 &&
                   (1ull << (h.B * (kj + 1))) <= jentries)
                ++kj;
            while (kj > 0 && h.depth_count[kj] > kJumpMaxStates) --kj;
            h.k = kj;
            h.base_k = depth_base[kj];
            h.count_k = h.depth_count[kj];
            if (kj > 0) {
                const uint32_t nj = 1u << (h.B * kj);
                h.J.assign(std::max<uint32_t>(nj, 8u), kJumpSlow);
                for (uint32_t w = 0; w < nj; ++w) {
                    int32_t e = 0;
                    if (walk_codes(0, w, kj, &e)) {
                        h.J[w] = static_cast<int16_t>(-2 - (e - static_cast<int32_t>(h.base_k)));
                    } else {
                        const int32_t v = -e - 2;  // result of the walk
                        h.J[w] = (v <= 32767) ? static_cast<int16_t>(v) : kJumpSlow;
                        if (v > 32767) h.jslow = true;
                    }
                }
            }
        }
        if (h.B == 8) {
            // 6c. hashed root filter and state hash (8-bit codes).  Windows of
            //     kh = min(4, shortest keyword) codes: a walk that does not
            //     reach depth kh stops before any keyword ends, so its result is
            //     -1.  The filter bit of the window of every depth-kh state is
            //     set (a clear bit: result -1); HK holds each depth-kh state
            //     under its window, one 16-byte entry {window, state, child,
            //     (child code << 24) | (result + 1)} per slot, linear probing:
            //     child is the state's one child, 0 for a leaf, or kHkBranch
            //     when it has several children (or a result of 2^24 - 1 or more).
            const uint32_t kh = std::min<uint32_t>(kHashWindow, h.minlen);
            uint32_t fb = 0;
            while (fb < kFilterBits && (2ull << fb) <= 8ull * opt.jump_bytes) ++fb;
            if (fb >= 5) {
                const uint32_t b0 = depth_base[kh], cnt = h.depth_count[kh];
                std::vector<uint32_t> key(static_cast<size_t>(b0) + cnt, 0);  // codes of the path, first lowest
                for (uint32_t s = 1; s < b0 + cnt; ++s)
                    key[s] = key[parent[s]] | (incode[s] << (8u * (depth[s] - 1u)));
                uint32_t hb = 6;
                while ((1ull << hb) < 4ull * cnt) ++hb;
                if (hb > 30) return AC_ERR_TOO_MANY_STATES;
                h.hashed = true;
                h.kh = kh;
                h.fbits = fb;
                h.hk_bits = hb;
                h.F.assign((1u << fb) / 32u, 0u);
                h.HK.assign((1ull << hb) * 4ull, 0u);
                const uint32_t emask = (1u << hb) - 1u;
                uint32_t probes = 1;
                for (uint32_t s = b0; s < b0 + cnt; ++s) {
                    const uint32_t w = key[s];
                    const uint32_t f = (w * kFilterHashMul) >> (32u - fb);
                    h.F[f >> 5] |= 1u << (31u - (f & 31u));
                    const uint32_t r1 = static_cast<uint32_t>(pathbest[s] + 1);
                    uint32_t child = kHkBranch, info = r1;
                    if (r1 < (1u << 24) && kids[s] <= 1) {
                        child = kids[s] == 0 ? 0u : child1[s];
                        info |= kids[s] == 0 ? 0u : (static_cast<uint32_t>(code1[s]) << 24);
                    }
                    uint32_t b = (w * kStateHashMul) >> (32u - hb);
                    for (uint32_t p = 1;; ++p, b = (b + 1u) & emask) {
                        uint32_t *e = &h.HK[4ull * b];
                        if (e[1] != 0u) continue;
                        e[0] = w;
                        e[1] = s;
                        e[2] = child;
                        e[3] = info;
                        probes = std::max(probes, p);
                        break;
                    }
                }
                h.hk_probes = probes;
            }
        }
        const uint32_t kj = h.k;

        // 7. stride table from the depth-k states (with 2- and 4-bit codes
        //    window_tables made it)
        if (h.B == 8) {
            RootTables rt;
            rt.k = kj;
            rt.base_k = h.base_k;
            rt.count_k = h.count_k;
            stride_rows(h, &rt, opt.stride_bytes);
            h.k2 = rt.k2;
            h.J2 = std::move(rt.J2);
        }

        // 8. chain records for the states from the first mostly-unbranched
        //    depth on: a state with one child starts a run of forced
        //    transitions through non-terminal one-child states; a walk that
        //    matches the run's bytes jumps to its end, one that does not stops
        //    with the state's result (no state inside the run has its own
        //    keyword, so every stop inside it has that result).
        uint32_t dc = h.maxlen + 1;
        {
            std::vector<uint64_t> single(h.maxlen + 1, 0);
            for (uint32_t s2 = 0; s2 < S; ++s2)
                if (kids[s2] <= 1) single[depth[s2]]++;
            for (uint32_t d = 2; d <= h.maxlen; ++d)
                if (h.depth_count[d] && single[d] * 100 >= 85ull * h.depth_count[d]) {
                    dc = d;
                    break;
                }
        }
        h.s_chain = (opt.chains && dc <= h.maxlen) ? depth_base[dc] : S;
        if (h.s_chain < S) {
            std::vector<uint8_t> byte_of(256, 0);
            for (int b = 0; b < 256; ++b)
                if (h.cls[b] >= 0) byte_of[static_cast<uint32_t>(h.cls[b])] = static_cast<uint8_t>(b);
            const uint32_t R = S - h.s_chain;
            h.skip.assign(static_cast<size_t>(R) * 4, 0);
            // A one-child state starts a run unless its parent is a one-child
            // state of the records (so in a run) and it has no keyword of its
            // own (then the parent's run goes through it).  Runs are found and
            // measured in parallel, their bytes laid out in the order of their
            // first states, then written in parallel.
            std::vector<uint32_t> runlen(R, 0);  // a run's length at its first state, else 0
            parallel_ranges(R, 16384, [&](uint64_t r0, uint64_t r1) {
                for (uint64_t r = r0; r < r1; ++r) {
                    const uint32_t s2 = h.s_chain + static_cast<uint32_t>(r);
                    uint32_t *rec = &h.skip[r * 4];
                    rec[3] = static_cast<uint32_t>(pathbest[s2]);
                    if (kids[s2] >= 2) {
                        rec[0] = kSkipBranch;
                        continue;
                    }
                    if (kids[s2] == 0) {  // a leaf: the walk stops here
                        rec[0] = 0;
                        rec[2] = s2;
                        continue;
                    }
                    const uint32_t p = parent[s2];
                    if (p >= h.s_chain && kids[p] == 1 && kw_at[order[s2]] < 0) continue;  // inside a run
                    uint32_t v = s2, L = 0;
                    do {
                        v = child1[v];
                        ++L;
                    } while (kids[v] == 1 && kw_at[order[v]] < 0);
                    runlen[r] = L;
                }
            });
            std::vector<uint32_t> runoff(R, 0);
            uint64_t total_bytes = 0;
            for (uint32_t r = 0; r < R; ++r) {
                runoff[r] = static_cast<uint32_t>(total_bytes);
                total_bytes += runlen[r];
            }
            if (total_bytes > 0xFFFFFFF0ull) return AC_ERR_TOO_MANY_STATES;
            h.chain.assign(std::max<size_t>(16, (static_cast<size_t>(total_bytes) + 15) & ~static_cast<size_t>(15)), 0);
            parallel_ranges(R, 16384, [&](uint64_t r0, uint64_t r1) {
                for (uint64_t r = r0; r < r1; ++r) {
                    const uint32_t L = runlen[r];
                    if (L == 0) continue;
                    const uint32_t s2 = h.s_chain + static_cast<uint32_t>(r), off = runoff[r];
                    uint32_t v = s2;
                    for (uint32_t j = 0; j < L; ++j) {
                        h.chain[off + j] = byte_of[code1[v]];
                        v = child1[v];
                    }
                    // the run's states: s2 and the one-child states inside it
                    uint32_t u = s2;
                    for (uint32_t j = 0; j < L; ++j) {
                        uint32_t *rc = &h.skip[static_cast<size_t>(u - h.s_chain) * 4];
                        rc[0] = L - j;
                        rc[1] = off + j;
                        rc[2] = v;
                        rc[3] = static_cast<uint32_t>(pathbest[u]);
                        u = child1[u];
                    }
                }
            });
        }

        // 9. full output (every keyword occurrence on a walk's path, the
        //    sub-patterns included): for the lowest id r of each keyword
        //    string, a record {up, len, dup_off, clen}.  up: the lowest id of
        //    the longest keyword that is a proper prefix of r's string
        //    (kNoKeyword: none); len = |r|; dups[dup_off ..) the ids of r's
        //    string, ascending; clen: the ids of r's string and of every
        //    keyword that is a proper prefix of it.  States in BFS order come
        //    after their prefixes, so up's clen is known when r's is set.
        {
            std::vector<uint64_t> by_state(nkw);  // (state << 32) | id
            for (uint32_t id = 0; id < nkw; ++id)
                by_state[id] = (static_cast<uint64_t>(newid[kw_state[id]]) << 32) | id;
            std::sort(by_state.begin(), by_state.end());
            h.full_rec.assign(4ull * nkw, 0);
            h.full_dups.resize(nkw);
            h.full_max_clen = 0;
            for (uint32_t i = 0; i < nkw;) {
                const uint32_t st = static_cast<uint32_t>(by_state[i] >> 32);
                uint32_t j = i;
                while (j < nkw && (by_state[j] >> 32) == st) {
                    h.full_dups[j] = static_cast<uint32_t>(by_state[j]);
                    ++j;
                }
                const uint32_t r = static_cast<uint32_t>(by_state[i]);  // lowest id of the string
                const int32_t up = pathbest[parent[st]];
                uint32_t *rec = &h.full_rec[4ull * r];
                rec[0] = up >= 0 ? static_cast<uint32_t>(up) : kNoKeyword;
                rec[1] = depth[st];
                rec[2] = i;
                rec[3] = (j - i) + (up >= 0 ? h.full_rec[4ull * static_cast<uint32_t>(up) + 3] : 0u);
                h.full_max_clen = std::max(h.full_max_clen, rec[3]);
                i = j;
            }
        }
    } catch (const std::bad_alloc &) {
        return AC_ERR_OOM;
    }
    *out = std::move(h);
    return AC_OK;
}

}  // namespace pfac
