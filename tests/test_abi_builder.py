"""CPU checks of the C ABI and the host automaton builder (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1412_7789_gb300 import api, build, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(ac_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "ac_compile" in names and "ac_match" in names and len(names) >= 12
    raw = ctypes.CDLL(api.library_path())
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(api, "_LIB", None)
    monkeypatch.setattr(api, "library_path", lambda: "/nonexistent/libpfac.so")
    with pytest.raises(RuntimeError):
        api.lib()


def test_status_strings(lib):
    assert api.ac_status_string(0) == "ok"
    assert "empty" in api.ac_status_string(api.AC_ERR_EMPTY_PATTERN)


def test_rejects_bad_keyword_sets(lib):
    with pytest.raises(api.AcError) as e:
        api.ac_compile([b"ab", b""], host_only=True)
    assert e.value.status == api.AC_ERR_EMPTY_PATTERN
    with pytest.raises(api.AcError) as e:
        api.ac_compile([], host_only=True)
    assert e.value.status == api.AC_ERR_EMPTY_PATTERN
    big = [bytes([i % 256, i // 256, 7]) for i in range(40000)]
    with pytest.raises(api.AcError) as e:
        api.ac_compile(big, index_width=16, host_only=True)
    assert e.value.status == api.AC_ERR_INVALID_ARG


def test_host_only_handle_refuses_matching(lib):
    h = api.ac_compile([b"ab"], host_only=True)
    try:
        st = lib.ac_match(h, 1, 10, 1, 0)
        assert st == api.AC_ERR_INVALID_ARG
    finally:
        api.ac_destroy(h)


def walk_table(cls, G, C, text):
    """Debug walker over the builder's exported table (not an oracle): follow
    the goto entries from every start, stop at the first dead entry."""
    n = len(text)
    out = np.empty(n, dtype=np.int32)
    for i in range(n):
        s = 0
        j = i
        while True:
            if j >= n or cls[text[j]] < 0:
                e = int(G[s, C])
                break
            e = int(G[s, cls[text[j]]])
            if e < 0:
                break
            s = e
            j += 1
        out[i] = -e - 2
    return out


CASES = [
    ([b"he", b"she", b"his", b"hers"], b"ushers"),
    ([b"AB", b"ABG", b"BEDE", b"ED"], b"ABEDEABGED"),
]


@pytest.mark.parametrize("seed", range(6))
def test_builder_structure_against_oracle(lib, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    alphabet = [b"ACGT", b"ab", bytes(range(256)), b"abcdefghij"][seed % 4]
    a = np.frombuffer(alphabet, dtype=np.uint8)
    text = a[g.integers(0, a.size, size=3000)]
    pats = [bytes(text[o:o + L]) for o, L in zip(g.integers(0, 2900, 30), g.integers(1, 20, 30))]
    pats += [bytes(a[g.integers(0, a.size, size=int(L))]) for L in g.integers(1, 12, 30)]
    pats += [pats[3], pats[7]]  # duplicates
    h = api.ac_compile(pats, host_only=True)
    try:
        info = api.ac_info(h)
        cls, G, depth = api.ac_export_tables(h)
        with oracle.Machine(pats) as m:
            assert info["n_states"] == m.n_states
            assert np.array_equal(depth.astype(np.uint64), m.depth_counts()[: depth.size])
            want = m.pfac_ids(text)
        # class map: distinct keyword bytes, in byte order (four that
        # (byte >> s) & 3 tells apart: that value)
        present = sorted(set(b"".join(pats)))
        assert info["n_classes"] == len(present)
        s = _direct_shift(present)
        assert info["class_direct_shift"] == s
        if s >= 0:
            assert [int(cls[b]) for b in present] == [(b >> s) & 3 for b in present]
        else:
            assert [int(cls[b]) for b in present] == list(range(len(present)))
        assert all(cls[b] == -1 for b in range(256) if b not in present)
        # 16-bit entries exactly when every state id and keyword id fits
        fits = info["n_states"] <= 32768 and len(pats) <= 32767
        assert info["index_width"] == (16 if fits else 32)
        # BFS order: children have larger ids, depth is non-decreasing in id
        C = info["n_classes"]
        starts = np.concatenate([[0], np.cumsum(depth)])
        dep = np.repeat(np.arange(depth.size), depth)
        child = G[:, :C]
        for s in range(info["n_states"]):
            kids = child[s][child[s] > 0]
            assert np.all(dep[kids] == dep[s] + 1)
            assert np.all(np.diff(kids) > 0)
        assert starts[-1] == info["n_states"]
        # every keyword's final state reports the lowest id of its string
        assert np.array_equal(walk_table(cls, G, C, text), want)
    finally:
        api.ac_destroy(h)


def test_builder_jump_and_stride_shapes(lib):
    text, pats = workloads.sweep_acgt(1 << 14)
    h = api.ac_compile(pats, host_only=True)
    info = api.ac_info(h)
    api.ac_destroy(h)
    # ACGT: 2-bit codes, a root filter over 10 characters (2^20 bits), and a
    # stride table of 4 more characters from the depth-10 states
    assert info["code_bits"] == 2 and info["jump_depth"] == 10
    assert info["stride_depth"] == 4
    h = api.ac_compile(pats, host_only=True, stride_bytes=1, jump_bytes=64)
    info = api.ac_info(h)
    api.ac_destroy(h)
    assert info["stride_depth"] == 0 and info["jump_depth"] == 4  # 512 filter bits
    text, pats = workloads.zipf_byte(1 << 16, n_keywords=2000)
    h = api.ac_compile(pats, host_only=True)
    info = api.ac_info(h)
    api.ac_destroy(h)
    assert info["code_bits"] == 8 and info["jump_depth"] == 2  # 2^16 int16 jump entries


def _direct_shift(present):
    """1 when (byte >> 1) & 3 tells four keyword bytes apart, else -1."""
    return 1 if len(present) == 4 and len({(b >> 1) & 3 for b in present}) == 4 else -1


@pytest.mark.parametrize("alphabet,shift", [
    (b"ACGT", 1),
    (b"acgt", 1),
    (bytes([0x00, 0x02, 0x04, 0x06]), 1),
    (bytes([0x10, 0x11, 0x12, 0x13]), -1),
    (bytes([0x00, 0x01, 0x80, 0x81]), -1),
    (b"AC", -1),
    (b"ACGTN", -1),
])
def test_direct_class_codes(lib, alphabet, shift):
    """Four keyword bytes that (byte >> 1) & 3 tells apart (the DNA letters
    in either case) take that value as their class code; the tables built on
    it walk as the oracle does."""
    g = np.random.Generator(np.random.PCG64(len(alphabet) * 31 + shift + 1))
    a = np.frombuffer(alphabet, dtype=np.uint8)
    pats = [bytes(a[g.integers(0, a.size, size=int(g.integers(1, 9)))]) for _ in range(80)]
    pats += [bytes([b]) for b in alphabet]
    text = np.concatenate([a, np.frombuffer(b"NxE\x00\xff", dtype=np.uint8)])[g.integers(0, a.size + 5, size=4000)]
    h = api.ac_compile(pats, host_only=True)
    try:
        info = api.ac_info(h)
        cls, G, _ = api.ac_export_tables(h)
        assert info["class_direct_shift"] == shift
        if shift >= 0:
            assert info["code_bits"] == 2
            assert sorted(int(cls[b]) for b in alphabet) == [0, 1, 2, 3]
            assert all(int(cls[b]) == (b >> shift) & 3 for b in alphabet)
        assert np.array_equal(walk_table(cls, G, info["n_classes"], text), oracle.pfac_ids(pats, text))
    finally:
        api.ac_destroy(h)


@pytest.mark.parametrize("alphabet,shift,bits", [
    (b"ACGT", 0, 2),
    (bytes([0x00, 0x01, 0x80, 0x81]), -1, 2),
    (b"abcdefg", 0, 4),
    (bytes([0x00, 0x08, 0x10, 0x18]), 2, 2),  # the smallest shift that separates them
    (bytes([0x00, 0x01, 0x02, 0x80, 0x81]), -1, 4),
    (b"abcdefghij", -1, 4),
])
def test_class_hash_choice(lib, alphabet, shift, bits):
    """Alphabets of at most 8 keyword bytes get a 3-bit hash (byte >> s) & 7
    that separates them, when one exists; the hash must be injective."""
    pats = [bytes([b]) * 3 for b in alphabet]
    h = api.ac_compile(pats, host_only=True)
    info = api.ac_info(h)
    api.ac_destroy(h)
    assert info["class_hash_shift"] == shift and info["code_bits"] == bits
    if shift >= 0:
        assert len({(b >> shift) & 7 for b in alphabet}) == len(alphabet)


def test_struct_layouts_match_the_header(tmp_path):
    """The Python mirrors of the C structs (ctypes and numpy) have the sizes
    and field offsets a C compiler gives them from ac.h."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {
        "ac_batch_item": api.BATCH_ITEM,
        "ac_server_request": api.SERVER_REQUEST,
        "ac_server_completion": api.SERVER_COMPLETION,
        "ac_server_options": api.ac_server_options,
        "ac_options": api.ac_options,
        "ac_info_t": api.ac_info_t,
        "ac_tuning": api.ac_tuning,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ac.h"', "int main(void) {"]
    for name, m in mirrors.items():
        fields = m.names if isinstance(m, np.dtype) else [f[0] for f in m._fields_]
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in fields:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for name, m in mirrors.items():
        if isinstance(m, np.dtype):
            assert int(got[name]) == m.itemsize, name
            for f in m.names:
                assert int(got["%s.%s" % (name, f)]) == m.fields[f][1], (name, f)
        else:
            assert int(got[name]) == ctypes.sizeof(m), name
            for f, _ in m._fields_:
                assert int(got["%s.%s" % (name, f)]) == getattr(m, f).offset, (name, f)


def _walk_with_chains(cls, G, s_chain, rec, byt, text, i):
    """The walk from position i using the goto table above s_chain and the
    chain records from s_chain on (the kernels' rule, written out plainly)."""
    C = G.shape[1] - 1
    n = text.size
    s, q = 0, i
    while True:
        if s >= s_chain:
            L, off, end, res = (int(x) for x in rec[s - s_chain])
            res = res - (1 << 32) if res >= (1 << 31) else res
            if L != 0xFFFFFFFF:
                if L > 0 and q + L <= n and bytes(text[q:q + L]) == bytes(byt[off:off + L]):
                    s, q = end, q + L
                    continue
                return res
        c = int(cls[text[q]]) if q < n else C
        if c < 0:
            c = C
        e = int(G[s, c])
        if e < 0:
            return -e - 2
        s, q = e, q + 1


@pytest.mark.parametrize("alpha", [b"ACGT", bytes(range(40, 80)), bytes(range(256))])
def test_chain_records_reproduce_the_walk(lib, alpha):
    """Walking with the chain records gives the oracle's ids (brute force over
    every position of random texts with long, partly copied keywords)."""
    g = np.random.Generator(np.random.PCG64(len(alpha)))
    a = np.frombuffer(alpha, dtype=np.uint8)
    for case in range(3):
        text = a[g.integers(0, a.size, size=3000)]
        pats = []
        for _ in range(60):
            L = int(g.integers(1, 40))
            if g.random() < 0.6:
                o = int(g.integers(0, text.size - L))
                pats.append(bytes(text[o:o + L]))
            else:
                pats.append(bytes(a[g.integers(0, a.size, size=L)]))
        h = api.ac_compile(pats, host_only=True)
        try:
            cls, G, depth = api.ac_export_tables(h)
            s_chain, rec, byt = api.ac_export_chains(h)
        finally:
            api.ac_destroy(h)
        assert s_chain < G.shape[0] and rec.shape[0] == G.shape[0] - s_chain
        runs = rec[:, 0][rec[:, 0] != 0xFFFFFFFF]
        assert runs.max() >= 2  # long runs exist, so the test exercises them
        want = oracle.pfac_ids(pats, text)
        got = np.array([_walk_with_chains(cls, G, s_chain, rec, byt, text, i) for i in range(text.size)])
        assert np.array_equal(got, want), case


def _nested_keywords(g, alpha: bytes, k: int, maxlen: int):
    """Keywords with many prefix relations and equal strings: prefixes of a few
    stems, random short words and repeats."""
    a = np.frombuffer(alpha, dtype=np.uint8)
    stems = [bytes(a[g.integers(0, a.size, size=maxlen)]) for _ in range(4)]
    pats = []
    for _ in range(k):
        u = g.random()
        if u < 0.5:
            s = stems[int(g.integers(0, len(stems)))]
            pats.append(s[:int(g.integers(1, maxlen + 1))])
        elif u < 0.8:
            pats.append(bytes(a[g.integers(0, a.size, size=int(g.integers(1, 5)))]))
        else:
            pats.append(pats[int(g.integers(0, len(pats)))] if pats else b"x")
    return pats


def full_chain_brute(pats, r: int):
    """Ids of every keyword that is a prefix of keyword r (equal strings
    included), ordered by length, then id -- from the definition."""
    p = pats[r]
    return sorted((len(q), i) for i, q in enumerate(pats) if p[:len(q)] == q)


@pytest.mark.parametrize("alpha", [b"ACGT", b"abcdefghijkl", bytes(range(256))])
def test_full_records_match_definition(lib, alpha):
    """The builder's full-output records: for the lowest id of each keyword
    string, its proper-prefix link, length, equal keywords and chain length,
    checked against brute force over the keyword list."""
    g = np.random.Generator(np.random.PCG64(7 + len(alpha)))
    for case in range(4):
        pats = _nested_keywords(g, alpha, 120, 12)
        h = api.ac_compile(pats, host_only=True)
        try:
            rec, dups, max_chain = api.ac_export_full(h, len(pats))
        finally:
            api.ac_destroy(h)
        lowest = {}
        for i, p in enumerate(pats):
            lowest.setdefault(p, i)
        clens = []
        for p, r in lowest.items():
            chain = full_chain_brute(pats, r)
            up_cands = [q for q in lowest if len(q) < len(p) and p[:len(q)] == q]
            up = lowest[max(up_cands, key=len)] if up_cands else 0xFFFFFFFF
            equal = sorted(i for i, q in enumerate(pats) if q == p)
            assert rec[r, 0] == up and rec[r, 1] == len(p) and rec[r, 3] == len(chain), (case, p)
            assert dups[rec[r, 2]:rec[r, 2] + len(equal)].tolist() == equal, (case, p)
            # following the links reproduces the whole chain, shortest first
            got, x = [], r
            while x != 0xFFFFFFFF:
                below = rec[rec[x, 0], 3] if rec[x, 0] != 0xFFFFFFFF else 0
                got = [(int(rec[x, 1]), int(i)) for i in dups[rec[x, 2]:rec[x, 2] + rec[x, 3] - below]] + got
                x = rec[x, 0]
            assert got == chain, (case, p)
            clens.append(len(chain))
        for i, p in enumerate(pats):
            if lowest[p] != i:
                assert not rec[i].any()
        assert max_chain == max(clens)


def test_full_expansion_equals_serial_machine(lib):
    """Each per-start longest result expanded through the records gives exactly
    the serial machine's occurrences (section II's output function), in the
    order start, end, id."""
    g = np.random.Generator(np.random.PCG64(31))
    for alpha in (b"ACGT", b"abcdef"):
        a = np.frombuffer(alpha, dtype=np.uint8)
        for case in range(3):
            pats = _nested_keywords(g, alpha, 80, 10)
            text = a[g.integers(0, a.size, size=4000)]
            for _ in range(30):  # plant the long stems
                p = pats[int(g.integers(0, len(pats)))]
                o = int(g.integers(0, text.size - len(p)))
                text[o:o + len(p)] = np.frombuffer(p, dtype=np.uint8)
            h = api.ac_compile(pats, host_only=True)
            try:
                rec, dups, _ = api.ac_export_full(h, len(pats))
            finally:
                api.ac_destroy(h)
            ids = oracle.pfac_ids(pats, text)
            got = []
            for i in np.nonzero(ids >= 0)[0]:
                x, chain = int(ids[i]), []
                while x != 0xFFFFFFFF:
                    below = rec[rec[x, 0], 3] if rec[x, 0] != 0xFFFFFFFF else 0
                    chain = [(int(i) + int(rec[x, 1]) - 1, int(d)) for d in dups[rec[x, 2]:rec[x, 2] + rec[x, 3] - below]] + chain
                    x = int(rec[x, 0])
                got += chain
            ends, fids = oracle.full_occurrences(pats, text)
            want = sorted(((int(e) - len(pats[d]) + 1, int(e), int(d)) for e, d in zip(ends, fids)))
            assert got == [(e, d) for _, e, d in want], (alpha, case)


def test_parallel_build_is_deterministic(lib):
    """The trie, its numbering, the goto table's rows and the chain records
    are built on several host threads: two builds of the same large keyword
    set export byte-identical tables and records, and every entry is either
    a larger child state or an encoded result."""
    text, pats = workloads.zipf_byte(1 << 20, seed=5, n_keywords=3000)
    tabs, chains = [], []
    for _ in range(2):
        h = api.ac_compile(pats, host_only=True)
        try:
            tabs.append(api.ac_export_tables(h))
            chains.append(api.ac_export_chains(h))
            info = api.ac_info(h)
        finally:
            api.ac_destroy(h)
    (c0, g0, d0), (c1, g1, d1) = tabs
    assert np.array_equal(c0, c1) and np.array_equal(d0, d1) and np.array_equal(g0, g1)
    for x, y in zip(chains[0], chains[1]):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    G = g0.reshape(info["n_states"], info["row_width"]).astype(np.int64)
    rows = np.arange(info["n_states"])[:, None]
    live = G > 0
    assert np.all(G[live] > np.broadcast_to(rows, G.shape)[live])  # BFS order: children after parents
    assert np.all(G[~live] <= -1)  # encoded results -(id + 2), id >= -1
    assert np.all(-G[~live] - 2 < len(pats))


@pytest.mark.parametrize("shape", ["one_group", "all_first_bytes", "skewed", "short_and_dups"])
def test_parallel_build_group_shapes(lib, shape):
    """The trie is built one subtrie per first byte class on the host's
    threads and numbered depth by depth across them: keyword sets whose
    first bytes form one group, all 256 groups, one group holding nine tenths
    of the keywords, and keywords of one or two bytes with duplicates across
    groups.  The exported goto table walks as the oracle does, BFS order
    holds (depths contiguous and non-decreasing, children after parents and
    in code order), and so do walks that take the chain records."""
    g = np.random.Generator(np.random.PCG64(["one_group", "all_first_bytes", "skewed", "short_and_dups"].index(shape) + 90))
    if shape == "one_group":
        pats = [b"Q" + bytes(g.integers(0, 256, size=int(g.integers(0, 30)), dtype=np.uint8)) for _ in range(800)]
    elif shape == "all_first_bytes":
        pats = [bytes([b]) + bytes(g.integers(0, 256, size=int(g.integers(0, 20)), dtype=np.uint8)) for b in range(256)
                for _ in range(3)]
    elif shape == "skewed":
        pats = [(b"e" if g.random() < 0.9 else bytes([int(g.integers(0, 256))])) +
                bytes(g.integers(97, 101, size=int(g.integers(0, 25)), dtype=np.uint8)) for _ in range(1500)]
    else:
        pats = [bytes(g.integers(0, 6, size=int(g.integers(1, 3)), dtype=np.uint8)) for _ in range(200)]
        pats += pats[::7]
    alphabet = np.array(sorted(set(b"".join(pats))), dtype=np.uint8)
    text = alphabet[g.integers(0, alphabet.size, size=6000)]
    for o in g.integers(0, 5900, size=40):  # plant keywords
        p = pats[int(g.integers(0, len(pats)))]
        text[o:o + len(p)] = np.frombuffer(p, dtype=np.uint8)[:max(0, min(len(p), text.size - o))]
    h = api.ac_compile(pats, host_only=True, class_compress=shape != "all_first_bytes")
    try:
        info = api.ac_info(h)
        cls, G, depth = api.ac_export_tables(h)
        s_chain, rec, byt = api.ac_export_chains(h)
        want = oracle.pfac_ids(pats, text)
        C = info["n_classes"]
        assert np.array_equal(walk_table(cls, G, C, text), want)
        starts = np.concatenate([[0], np.cumsum(depth)])
        assert starts[-1] == info["n_states"] and depth[0] == 1
        dep = np.repeat(np.arange(depth.size), depth)
        for s in range(info["n_states"]):
            kids = G[s, :C][G[s, :C] > 0]
            assert np.all(dep[kids] == dep[s] + 1) and np.all(np.diff(kids) > 0)
        got = np.array([_walk_with_chains(cls, G, s_chain, rec, byt, text, i) for i in range(text.size)], dtype=np.int32)
        assert np.array_equal(got, want)
    finally:
        api.ac_destroy(h)


@pytest.mark.parametrize("alpha,lmin,lmax", [(b"ACGT", 4, 40), (b"abcdefghijkl", 2, 12), (b"ACGT", 1, 2),
                                             (b"ACG", 3, 9)])
def test_root_filter_and_window_table(lib, alpha, lmin, lmax):
    """Every window of k codes: the window table holds the state the goto
    table's walk reaches (or its encoded result), and the filter bit read the
    way the kernel reads it -- the word at byte offset (w >> 3) & mask rotated
    left by w's low five bits, bit 31 -- is set exactly when that walk is
    alive or found a keyword, whatever codes follow the window in w."""
    g = np.random.Generator(np.random.PCG64(len(alpha) * 100 + lmax))
    a = np.frombuffer(alpha, dtype=np.uint8)
    pats = [bytes(a[g.integers(0, a.size, size=int(g.integers(lmin, lmax + 1)))]) for _ in range(300)]
    h = api.ac_compile(pats, host_only=True)
    try:
        _check_window_tables(h)
    finally:
        api.ac_destroy(h)


def _check_window_tables(h):
    B, k, F, JK = api.ac_export_filter(h)
    cls, G, depth = api.ac_export_tables(h)
    info = api.ac_info(h)
    assert B in (2, 4) and k >= 1 and JK.size == 1 << (B * k)
    C, W = info["n_classes"], info["row_width"]
    G = G.reshape(info["n_states"], W).astype(np.int64)
    v = np.arange(1 << (B * k), dtype=np.int64)
    s = np.zeros(v.size, dtype=np.int64)
    res = np.full(v.size, -2, dtype=np.int64)  # -2: still alive
    for i in range(k):
        c = (v >> (B * i)) & ((1 << B) - 1)
        e = G[s, np.where(c < C, c, C)]  # codes no keyword byte takes read the end column
        live = res == -2
        stop = live & (e < 0)
        res[stop] = -e[stop] - 2
        s = np.where(live & (e > 0), e, s)
    alive = res == -2
    assert np.array_equal(JK, np.where(alive, s, -(res + 2)))
    assert info["match_windows_ppm"] == int((res >= 0).sum()) * 10**6 // v.size
    want = alive | (res >= 0)
    wb = B * k
    famask = (((1 << wb) if wb >= 5 else 32) // 8 - 1) & ~3
    for garbage in (0, 1, 0x5A5A5A5A, 0xFFFFFFFF):
        win = (v | (garbage << wb)) & 0xFFFFFFFF
        words = F[((win >> 3) & famask) >> 2].astype(np.int64)
        r = win & 31
        rot = ((words << r) | (words >> ((32 - r) & 31))) & 0xFFFFFFFF
        rot = np.where(r == 0, words, rot)
        assert np.array_equal((rot >> 31) & 1, want.astype(np.int64)), garbage
    return k


@pytest.mark.parametrize("alpha,lmin,lmax", [(b"ACGT", 12, 40), (b"abcdefghijkl", 6, 20)])
def test_stride_table(lib, alpha, lmin, lmax):
    """Every stride-table entry equals the goto table's walk of its k2 codes
    from its depth-k state."""
    g = np.random.Generator(np.random.PCG64(len(alpha) * 7 + lmin))
    a = np.frombuffer(alpha, dtype=np.uint8)
    pats = [bytes(a[g.integers(0, a.size, size=int(g.integers(lmin, lmax + 1)))]) for _ in range(400)]
    h = api.ac_compile(pats, host_only=True)
    try:
        assert _check_stride_table(h) >= 2
    finally:
        api.ac_destroy(h)


def _check_stride_table(h):
    B, k, F, JK = api.ac_export_filter(h)
    k2, base_k, count_k, J2 = api.ac_export_stride(h)
    cls, G, depth = api.ac_export_tables(h)
    info = api.ac_info(h)
    if k2 == 0:
        assert J2.size == 0
        return 0
    assert J2.size == count_k << (B * k2)
    assert base_k == int(depth[:k].sum()) and count_k == int(depth[k])
    C, W = info["n_classes"], info["row_width"]
    G = G.reshape(info["n_states"], W).astype(np.int64)
    idx = np.arange(J2.size, dtype=np.int64)
    v = idx & ((1 << (B * k2)) - 1)
    s = base_k + (idx >> (B * k2))
    res = np.full(idx.size, -2, dtype=np.int64)
    for i in range(k2):
        c = (v >> (B * i)) & ((1 << B) - 1)
        e = G[s, np.where(c < C, c, C)]
        live = res == -2
        stop = live & (e < 0)
        res[stop] = -e[stop] - 2
        s = np.where(live & (e > 0), e, s)
    assert np.array_equal(J2, np.where(res == -2, s, -(res + 2)))
    return k2


@pytest.mark.parametrize("alpha,lmin,lmax", [(b"ACGT", 12, 40), (b"abcdefghijkl", 4, 20)])
def test_shared_table_depth(lib, alpha, lmin, lmax):
    """ac_set_tuning(filter_bytes) rebuilds the root filter, window table and
    stride table for the largest window whose filter fits, from the goto table
    alone: at every size they pass the same checks against goto-table walks,
    the window shrinks with the budget, and a size that fits no filter, or a
    bad field, is refused without changing anything."""
    g = np.random.Generator(np.random.PCG64(len(alpha) * 11 + lmin))
    a = np.frombuffer(alpha, dtype=np.uint8)
    pats = [bytes(a[g.integers(0, a.size, size=int(g.integers(lmin, lmax + 1)))]) for _ in range(400)]
    with api.Automaton(pats, host_only=True) as au:
        B, k0, F0, JK0 = api.ac_export_filter(au.handle)
        assert au.tuning()["filter_bytes"] == F0.nbytes
        seen = []
        for fb in (F0.nbytes // (1 << B), F0.nbytes // (1 << (2 * B)), 16, F0.nbytes):
            au.set_tuning(filter_bytes=fb)
            k = _check_window_tables(au.handle)
            _check_stride_table(au.handle)
            # the widest window whose filter (2^(B k) bits, at least 16 bytes) fits
            assert max(4, (1 << (B * k)) // 32) * 4 <= max(fb, 16)
            assert (1 << (B * (k + 1))) // 8 > fb or k == au.info()["max_len"]
            assert au.tuning()["filter_bytes"] == max(16, (1 << (B * k)) // 8)
            seen.append(k)
        assert seen[-1] == k0 and seen[0] == k0 - 1 and len(set(seen)) >= 3
        before = au.tuning()
        for bad in ({"filter_bytes": 8}, {"block": 48}, {"stages": 5}, {"per_thread": 3}, {"halo": 512},
                    {"survivor_list": 3}):
            with pytest.raises(api.AcError):
                au.set_tuning(**bad)
            assert au.tuning() == before
        au.set_tuning(block=256, stages=2, halo=64, per_thread=4, survivor_list=1)
        t = au.tuning()
        assert (t["block"], t["stages"], t["halo"], t["per_thread"], t["survivor_list"]) == (256, 2, 64, 4, 1)


def test_shared_table_depth_hashed(lib):
    """8-bit codes: the hashed filter rebuilt at 2^fbits bits from the state
    hash sets exactly the bits of the depth-kh states' windows."""
    _, pats = workloads.zipf_byte(1 << 18, seed=5, n_keywords=2000)
    with api.Automaton(pats, host_only=True) as au:
        kh, fbits0, hk_bits, probes, F0, HK = api.ac_export_hash(au.handle)
        assert fbits0 == 20
        wins = HK[HK[:, 1] != 0, 0].astype(np.int64)
        for fb in (1 << 15, 1 << 13, 4, 1 << 17):
            au.set_tuning(filter_bytes=fb)
            kh2, fbits, _, _, F, HK2 = api.ac_export_hash(au.handle)
            assert kh2 == kh and np.array_equal(HK2, HK)
            assert (1 << fbits) // 8 <= fb < (1 << (fbits + 1)) // 8 or fbits == 20
            f = ((wins * 0x9E3779B1) & 0xFFFFFFFF) >> (32 - fbits)
            want = np.zeros(F.size * 32, dtype=bool)
            want[f] = True
            bits = np.unpackbits(F.view(np.uint8).reshape(-1, 4)[:, ::-1], axis=1).reshape(-1).astype(bool)
            assert np.array_equal(bits, want), fb
            assert au.tuning()["filter_bytes"] == F.nbytes
        with pytest.raises(api.AcError):
            au.set_tuning(filter_bytes=3)


@pytest.mark.parametrize("kw", [{}, {"class_compress": False}])
def test_root_jump_table(lib, kw):
    """Every entry of the 8-bit root jump table equals the goto table's walk of
    its two bytes: the result where the walk stopped, or the index of the
    depth-2 state it reached."""
    text, pats = workloads.zipf_byte(1 << 18, seed=9, n_keywords=2000)
    h = api.ac_compile(pats, host_only=True, **kw)
    try:
        k, base_k, J = api.ac_export_jump(h)
        cls, G, depth = api.ac_export_tables(h)
        info = api.ac_info(h)
    finally:
        api.ac_destroy(h)
    assert info["code_bits"] == 8 and k == 2 and J.size == 1 << 16
    C, W = info["n_classes"], info["row_width"]
    G = G.reshape(info["n_states"], W).astype(np.int64)
    v = np.arange(J.size, dtype=np.int64)
    s = np.zeros(v.size, dtype=np.int64)
    res = np.full(v.size, -2, dtype=np.int64)
    for i in range(k):
        c = (v >> (8 * i)) & 0xFF  # class codes (identity when 256 columns)
        e = G[s, np.where(c < C, c, C)]
        live = res == -2
        stop = live & (e < 0)
        res[stop] = -e[stop] - 2
        s = np.where(live & (e > 0), e, s)
    want = np.where(res == -2, -(2 + (s - base_k)), res)
    slow = J == -32768
    assert np.array_equal(J[~slow].astype(np.int64), want[~slow])
    assert np.all(want[slow] > 32767) and np.all((res[slow] > 32767))


def _hk_find(HK, hk_bits, probes, w):
    """Lookup in the state hash as ac.h documents it: from entry
    (w * 0x85EBCA77 mod 2^32) >> (32 - hk_bits), at most `probes` entries,
    stopping at an empty one; returns the entry's index, or -1."""
    b = ((w * 0x85EBCA77) & 0xFFFFFFFF) >> (32 - hk_bits)
    for _ in range(probes):
        e = HK[b]
        if e[1] == 0:
            return -1
        if e[0] == w:
            return b
        b = (b + 1) % HK.shape[0]
    return -1


@pytest.mark.parametrize("case", ["zipf", "zipf_256cols", "short_keywords", "long_only"])
def test_hashed_filter_and_state_hash(lib, case):
    """8-bit codes: for every state at depth kh (= min(4, shortest keyword)),
    the walk of its kh codes through the goto table reaches it, its window's
    filter bit is set and the state hash finds it, with the state's child
    (none, the only one with its code, or several) and result as its goto row
    has them; windows whose walk does not reach depth kh (random ones, and
    every depth-kh window with one code changed) are not found."""
    g = np.random.default_rng(3)
    kw = {}
    if case.startswith("zipf"):
        _, pats = workloads.zipf_byte(1 << 18, seed=9, n_keywords=3000)
        if case == "zipf_256cols":
            kw = {"class_compress": False}
    elif case == "short_keywords":
        pats = [bytes(g.integers(0, 256, size=int(g.integers(2, 9)), dtype=np.uint8)) for _ in range(700)]
    else:
        pats = [bytes(g.integers(30, 90, size=int(g.integers(6, 40)), dtype=np.uint8)) for _ in range(500)]
    h = api.ac_compile(pats, host_only=True, **kw)
    try:
        kh, fbits, hk_bits, probes, F, HK = api.ac_export_hash(h)
        cls, G, depth = api.ac_export_tables(h)
        info = api.ac_info(h)
    finally:
        api.ac_destroy(h)
    assert info["code_bits"] == 8
    assert kh == min(4, min(len(p) for p in pats)) and fbits == 20 and probes >= 1
    C = info["n_classes"]
    G = G.reshape(info["n_states"], info["row_width"]).astype(np.int64)
    base = int(depth[:kh].sum())
    states = np.arange(base, base + int(depth[kh]))

    def walk(wins):
        s = np.zeros(wins.size, dtype=np.int64)
        alive = np.ones(wins.size, dtype=bool)
        for i in range(kh):
            c = (wins >> np.int64(8 * i)) & 0xFF
            e = G[s, np.where(c < C, c, C)]
            alive &= e > 0
            s = np.where(alive, e, 0)
        return np.where(alive, s, 0)

    # the window of every depth-kh state: the codes along its path, from the
    # goto table (BFS order: a state's parent is the row holding it)
    par = np.zeros(G.shape[0], dtype=np.int64)
    code = np.zeros(G.shape[0], dtype=np.int64)
    rows, cols = np.nonzero(G[:, :C] > 0)
    par[G[rows, cols]] = rows
    code[G[rows, cols]] = cols
    wins = np.zeros(states.size, dtype=np.int64)
    for j in range(kh):
        anc = states.copy()
        for _ in range(kh - 1 - j):
            anc = par[anc]
        wins |= code[anc] << np.int64(8 * j)
    assert np.array_equal(walk(wins), states)
    f = ((wins * 0x9E3779B1) & 0xFFFFFFFF) >> (32 - fbits)
    assert np.all((F[f >> 5] >> (31 - (f & 31))) & 1)
    live = G[:, :C] > 0
    for w, s in zip(wins, states):
        b = _hk_find(HK, hk_bits, probes, int(w))
        assert b >= 0 and HK[b, 1] == s
        kids = np.nonzero(live[s])[0]
        res = -int(G[s, C]) - 2  # the end column holds the result of stopping at s
        child, info = int(HK[b, 2]), int(HK[b, 3])
        if kids.size >= 2:
            assert child == 0xFFFFFFFF
        else:
            assert (info & 0xFFFFFF) == res + 1
            if kids.size == 0:
                assert child == 0
            else:
                assert child == int(G[s, kids[0]]) and (info >> 24) == int(kids[0])
    # windows whose walk stops before depth kh are not in the hash
    rnd = g.integers(0, 1 << (8 * kh), size=4000, dtype=np.int64)
    mutated = wins ^ (np.int64(1) << np.int64(8 * g.integers(0, kh, size=wins.size)))
    for cand in (rnd, mutated):
        reach = walk(cand)
        for w, s in zip(cand[:3000], reach[:3000]):
            b = _hk_find(HK, hk_bits, probes, int(w))
            assert (b < 0 and s == 0) or (b >= 0 and HK[b, 1] == s)
    # the filter keeps few windows: at most one bit per depth-kh state
    assert int(np.unpackbits(F.view(np.uint8)).sum()) <= states.size


def test_c_program_uses_the_library(lib, tmp_path):
    """A plain C program (no Python) compiles against ac.h, links the shared
    library and builds a host-only automaton: he/she/his/hers gives 10 states,
    5 classes (h, e, s, i, r) in 4-bit codes, and the exported goto table takes
    the walk "she" to a state whose end column reports keyword 1."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "ac.h"
int main(void) {
    const char *kw[4] = {"he", "she", "his", "hers"};
    const uint8_t *p[4];
    uint32_t len[4];
    for (int i = 0; i < 4; ++i) { p[i] = (const uint8_t *)kw[i]; len[i] = (uint32_t)strlen(kw[i]); }
    ac_options o;
    ac_default_options(&o);
    o.host_only = 1;
    ac_handle h = NULL;
    if (ac_compile(p, len, 4, &o, &h) != AC_OK) return 2;
    ac_info_t info;
    if (ac_info(h, &info) != AC_OK) return 3;
    int16_t cls[256];
    size_t cells = (size_t)info.n_states * info.row_width;
    int32_t *g = malloc(cells * sizeof(int32_t));
    if (info.index_width != 16 && info.index_width != 32) return 4;
    void *raw = malloc(cells * (info.index_width / 8));
    uint32_t *depth = malloc((info.max_len + 1) * sizeof(uint32_t));
    if (ac_export_tables(h, cls, raw, depth) != AC_OK) return 5;
    for (size_t i = 0; i < cells; ++i)
        g[i] = info.index_width == 16 ? ((int16_t *)raw)[i] : ((int32_t *)raw)[i];
    int32_t s = 0;
    const char *w = "she";
    for (int i = 0; i < 3; ++i) s = g[(size_t)s * info.row_width + cls[(uint8_t)w[i]]];
    int32_t end = g[(size_t)s * info.row_width + info.n_classes];  /* end column: stop here */
    printf("%u %u %u %d\n", info.n_states, info.n_classes, info.code_bits, -end - 2);
    ac_destroy(h);
    free(g); free(raw); free(depth);
    return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(api.library_path())
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lpfac",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out == ["10", "5", "4", "1"], out
