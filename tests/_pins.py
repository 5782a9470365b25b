"""The oracle's pin battery: checks of the CPU oracle against what the paper and
the mathematics fix, independent of the oracle's own code.  Each ``pin_*``
function takes the loaded oracle library (so a deliberately broken copy can be
run through the same checks) and raises AssertionError on a mismatch."""
from __future__ import annotations

import os

import numpy as np

import oracle
from paper_1412_7789_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------------------
# golden fixtures
# ----------------------------------------------------------------------------
def read_golden(name: str):
    """Parse a fixture: keyword lines, then (text, ids, full) groups."""
    keywords, cases = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.rstrip("\n")
            if not line or line.startswith("#"):
                continue
            tag, _, rest = line.partition(" ")
            if tag == "keyword":
                keywords.append(rest.encode())
            elif tag == "text":
                cases.append({"text": rest.encode()})
            elif tag == "ids":
                cases[-1]["ids"] = [int(x) for x in rest.split()]
            elif tag == "full":
                cases[-1]["full"] = sorted(tuple(int(v) for v in x.split(":")) for x in rest.split())
    return keywords, cases


def pin_golden(lib, name: str):
    keywords, cases = read_golden(name)
    assert cases
    for c in cases:
        got = oracle.pfac_ids(keywords, c["text"], lib)
        assert got.tolist() == c["ids"], (name, c["text"], got.tolist(), c["ids"])
        ends, ids = oracle.full_occurrences(keywords, c["text"], lib)
        pairs = sorted(zip(ends.tolist(), ids.tolist()))
        assert pairs == c["full"], (name, c["text"], pairs, c["full"])


# ----------------------------------------------------------------------------
# definitions written out (independent of the oracle's algorithm)
# ----------------------------------------------------------------------------
def brute_ids(patterns, text) -> list[int]:
    """Per start: the longest keyword equal to text[i:i+len]; ties -> lowest id."""
    t = bytes(text)
    n = len(t)
    out = [-1] * n
    for i in range(n):
        best = -1
        for pid, p in enumerate(patterns):
            L = len(p)
            if i + L <= n and t[i:i + L] == p:
                if best < 0 or L > len(patterns[best]):
                    best = pid
        out[i] = best
    return out


def brute_full(patterns, text) -> list[tuple[int, int]]:
    """Every (end, id) with text[end-len+1 : end+1] == keyword id."""
    t = bytes(text)
    out = []
    for pid, p in enumerate(patterns):
        L = len(p)
        start = t.find(p)
        while start >= 0:
            out.append((start + L - 1, pid))
            start = t.find(p, start + 1)
    return sorted(out)


def _tiny_case(g, alphabet: bytes):
    n = int(g.integers(0, 65))
    k = int(g.integers(1, 9))
    a = np.frombuffer(alphabet, dtype=np.uint8)
    text = bytes(a[g.integers(0, a.size, size=n)])
    pats = []
    for _ in range(k):
        if n and g.random() < 0.4:
            L = int(g.integers(1, min(n, 8) + 1))
            off = int(g.integers(0, n - L + 1))
            pats.append(text[off:off + L])
        else:
            L = int(g.integers(1, 7))
            pats.append(bytes(a[g.integers(0, a.size, size=L)]))
    return pats, text


TINY_ALPHABETS = [b"ab", b"ACGT", b"abc", bytes([0x00, 0x7F, 0x80, 0xFF]), bytes(range(256))]


def pin_bruteforce(lib, cases: int = 10_000, seed: int = 12345):
    g = np.random.Generator(np.random.PCG64(seed))
    for c in range(cases):
        alphabet = TINY_ALPHABETS[c % len(TINY_ALPHABETS)]
        pats, text = _tiny_case(g, alphabet)
        want = brute_ids(pats, text)
        with oracle.Machine(pats, lib) as m:
            got = m.pfac_ids(text).tolist()
            assert got == want, ("pfac", pats, text, got, want)
            if c % 4 == 0:
                ends, ids = m.full_occurrences(text)
                assert sorted(zip(ends.tolist(), ids.tolist())) == brute_full(pats, text), ("full", pats, text)


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------
def paper_closed_form(n: int) -> np.ndarray:
    """Paper-mode workload (section III): the alphabet repeated, keywords that
    are 26-letter permutations with keyword 0 = a..z and no other keyword a
    rotation of it.  Every 26-byte window of the text is a rotation of a..z, so
    only keyword 0 can occur, exactly at i = 0 mod 26 with i + 26 <= n."""
    ids = np.full(n, -1, dtype=np.int32)
    i = np.arange(n)
    ids[(i % 26 == 0) & (i + 26 <= n)] = 0
    return ids


def pin_paper_mode(lib):
    for count in (5, 10):
        pats = workloads.paper_keywords(count, seed=0)
        assert pats[0] == b"abcdefghijklmnopqrstuvwxyz"
        for p in pats[1:]:
            assert sorted(p) == sorted(pats[0]) and p not in pats[0] + pats[0]
        for n in (0, 1, 25, 26, 27, 1310, 16375, 53710):
            got = oracle.pfac_ids(pats, workloads.paper_text(n), lib)
            assert np.array_equal(got, paper_closed_form(n)), (count, n)


def pin_single_keyword(lib, seed: int = 7):
    """One keyword: the result is the naive find-all (every overlapping hit)."""
    g = np.random.Generator(np.random.PCG64(seed))
    for trial in range(200):
        alphabet = TINY_ALPHABETS[trial % 4]
        a = np.frombuffer(alphabet, dtype=np.uint8)
        n = int(g.integers(0, 3000))
        text = bytes(a[g.integers(0, a.size, size=n)])
        p = bytes(a[g.integers(0, a.size, size=int(g.integers(1, 6)))])
        want = np.full(n, -1, dtype=np.int32)
        j = text.find(p)
        while j >= 0:
            want[j] = 0
            j = text.find(p, j + 1)
        assert np.array_equal(oracle.pfac_ids([p], text, lib), want), (p, n)


def pin_length_one(lib, seed: int = 8):
    """All keywords of length 1: ids[i] = lowest id whose byte is text[i]."""
    g = np.random.Generator(np.random.PCG64(seed))
    for _ in range(50):
        k = int(g.integers(1, 40))
        bs = g.integers(0, 256, size=k).astype(np.uint8)
        pats = [bytes([int(b)]) for b in bs]
        lut = np.full(256, -1, dtype=np.int32)
        for pid in range(k - 1, -1, -1):
            lut[bs[pid]] = pid
        text = g.integers(0, 256, size=5000).astype(np.uint8)
        assert np.array_equal(oracle.pfac_ids(pats, text, lib), lut[text])


def pin_all_grams(lib, seed: int = 9):
    """Keyword set = all 4**L ACGT strings of length L (id = base-4 value):
    every i <= n-L matches, with id = base-4 value of text[i:i+L]."""
    code = np.zeros(256, dtype=np.int64)
    for v, ch in enumerate(b"ACGT"):
        code[ch] = v
    for L in (1, 2, 3, 5):
        pats = []
        for v in range(4 ** L):
            digits = [(v >> (2 * (L - 1 - j))) & 3 for j in range(L)]
            pats.append(bytes(b"ACGT"[d] for d in digits))
        text = workloads.acgt_text(4096, seed + L)
        n = text.size
        want = np.full(n, -1, dtype=np.int64)
        val = np.zeros(n - L + 1, dtype=np.int64)
        for j in range(L):
            val = val * 4 + code[text[j:n - L + 1 + j]]
        want[: n - L + 1] = val
        assert np.array_equal(oracle.pfac_ids(pats, text, lib), want.astype(np.int32)), L


# ----------------------------------------------------------------------------
# invariants on larger random inputs
# ----------------------------------------------------------------------------
def check_sound_and_maximal(patterns, text, ids):
    """I1: each reported keyword occurs at its start; I2: no longer keyword
    occurs there (all keyword strings hashed per length)."""
    t = bytes(text)
    by_len: dict[int, dict[bytes, int]] = {}
    for pid, p in enumerate(patterns):
        d = by_len.setdefault(len(p), {})
        if p not in d:
            d[p] = pid
    lengths = sorted(by_len)
    n = len(t)
    for i in range(n):
        r = int(ids[i])
        cur = len(patterns[r]) if r >= 0 else 0
        if r >= 0:
            assert t[i:i + cur] == patterns[r], ("unsound", i, r)
            assert by_len[cur][patterns[r]] == r, ("tie not lowest", i, r)
        for L in lengths:
            if L > cur and i + L <= n:
                assert t[i:i + L] not in by_len[L], ("not maximal", i, L)


def pin_invariants(lib, seed: int = 10):
    g = np.random.Generator(np.random.PCG64(seed))
    text = workloads.acgt_text(20_000, seed)
    pats = workloads.keywords_acgt(text, 60, 2, 12, 0.5, seed + 1)
    ids = oracle.pfac_ids(pats, text, lib)
    check_sound_and_maximal(pats, text, ids)
    # I3: a superset keyword set never unmatches a start nor shortens its match
    extra = workloads.keywords_acgt(text, 60, 2, 12, 0.5, seed + 2)
    ids2 = oracle.pfac_ids(pats + extra, text, lib)
    allp = pats + extra
    assert np.all((ids < 0) | (ids2 >= 0))
    l1 = np.array([len(pats[i]) if i >= 0 else 0 for i in ids])
    l2 = np.array([len(allp[i]) if i >= 0 else 0 for i in ids2])
    assert np.all(l2 >= l1)
    assert oracle.count(ids2) >= oracle.count(ids)
    # I6: the per-start pairs are a subset of the full machine's occurrences
    ends, fids = oracle.full_occurrences(pats, text, lib)
    full = set(zip((ends.astype(np.int64) + 1 - np.array([len(pats[i]) for i in fids])).tolist(), fids.tolist()))
    for i in np.nonzero(ids >= 0)[0].tolist():
        assert (i, int(ids[i])) in full
    # I4: count == |compact| == #{ids >= 0}, compact == filtered dense
    pos, cid = oracle.compact(ids)
    assert pos.size == oracle.count(ids) == int((ids >= 0).sum())
    assert np.array_equal(ids[pos], cid.astype(np.int32)) and np.all(np.diff(pos.astype(np.int64)) > 0)
    del g


ALL_PINS = {
    "w1": lambda lib: pin_golden(lib, "w1_ushers.txt"),
    "w2": lambda lib: pin_golden(lib, "w2_fig45.txt"),
    "paper_mode": pin_paper_mode,
    "single_keyword": pin_single_keyword,
    "length_one": pin_length_one,
    "all_grams": pin_all_grams,
    "bruteforce": pin_bruteforce,
    "invariants": pin_invariants,
}
