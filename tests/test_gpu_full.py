"""Full Aho-Corasick output (ac_match_full) through the C ABI against the CPU
oracle's serial machine (section II's output function), bit-exact: every
occurrence (end, id) of every keyword, sub-patterns and equal keywords
included, ordered by start, end, id."""
import numpy as np
import pytest

import oracle
from paper_1412_7789_gb300 import api, workloads
from tests import _gpu, _pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1412_7789_gb300 import build

    build.build()
    api.lib()
    yield
    assert api.ac_device_status() == api.AC_OK


def want_full(pats, text):
    """The oracle's occurrences in the order start, end, id."""
    ends, ids = oracle.full_occurrences(pats, text)
    order = sorted(((int(e) - len(pats[d]) + 1, int(e), int(d)) for e, d in zip(ends, ids)))
    return (np.array([e for _, e, _ in order], dtype=np.uint32), np.array([d for _, _, d in order], dtype=np.uint32))


def got_full(h, t, cap):
    import torch

    end = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=t.device)
    ids = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=t.device)
    c = torch.full((1,), 12345, dtype=torch.int64, device=t.device)
    api.ac_match_full(h, t, t.numel(), end, ids, cap, c)
    total = int(c.item())
    m = min(total, cap)
    return end[:m].cpu().numpy().astype(np.uint32), ids[:m].cpu().numpy().astype(np.uint32), total, end, ids


def check(h, pats, text, t=None, cap=None):
    we, wi = want_full(pats, text)
    t = _gpu.to_dev(text) if t is None else t
    cap = max(1, we.size) if cap is None else cap
    ge, gi, total, end, ids = got_full(h, t, cap)
    assert total == we.size, (total, we.size)
    m = min(total, cap)
    if not (np.array_equal(ge, we[:m]) and np.array_equal(gi, wi[:m])):
        bad = np.nonzero((ge != we[:m]) | (gi != wi[:m]))[0]
        raise AssertionError("full mismatch at %d entries, first %s: got %s / %s want %s / %s" % (
            bad.size, bad[:6].tolist(), ge[bad[:6]].tolist(), gi[bad[:6]].tolist(), we[bad[:6]].tolist(),
            wi[bad[:6]].tolist()))
    if cap > m:  # nothing written past the total
        assert np.all(end[m:].cpu().numpy() == -7) and np.all(ids[m:].cpu().numpy() == -7)


@pytest.mark.parametrize("name", ["w1_ushers.txt", "w2_fig45.txt"])
def test_golden_full(name):
    keywords, cases = _pins.read_golden(name)
    with api.Automaton(keywords) as a:
        for c in cases:
            text = np.frombuffer(c["text"], dtype=np.uint8)
            ge, gi, total, _, _ = got_full(a.handle, _gpu.to_dev(text), 64)
            got = sorted(zip(ge.tolist(), gi.tolist()))
            assert got == c["full"], (c["text"], got, c["full"])


def nested(g, alpha: bytes, k: int, maxlen: int):
    """Keywords with many prefix relations: prefixes of a few stems, short
    random words and repeats of earlier keywords (equal strings)."""
    a = np.frombuffer(alpha, dtype=np.uint8)
    stems = [bytes(a[g.integers(0, a.size, size=maxlen)]) for _ in range(6)]
    pats = []
    for _ in range(k):
        u = g.random()
        if u < 0.5:
            s = stems[int(g.integers(0, len(stems)))]
            pats.append(s[:int(g.integers(1, maxlen + 1))])
        elif u < 0.85 or not pats:
            pats.append(bytes(a[g.integers(0, a.size, size=int(g.integers(1, 6)))]))
        else:
            pats.append(pats[int(g.integers(0, len(pats)))])
    return pats, stems


def planted_text(g, alpha: bytes, n: int, stems):
    a = np.frombuffer(alpha, dtype=np.uint8)
    text = a[g.integers(0, a.size, size=n)].copy()
    for _ in range(max(1, n // 300)):
        s = stems[int(g.integers(0, len(stems)))]
        if len(s) < n:
            o = int(g.integers(0, n - len(s) + 1))
            text[o:o + len(s)] = np.frombuffer(s, dtype=np.uint8)
    return text


SIZES = [1, 2, 15, 16, 17, 991, 992, 993, 1023, 1024, 1025, 4000, 65537, 300001]


@pytest.mark.parametrize("alpha,kw", [(b"ACGT", {}), (b"abcdefghijkl", {}), (bytes(range(40, 120)), {}),
                                      (bytes(range(256)), {"class_compress": False})])
def test_full_random_sizes(alpha, kw):
    """Nested keyword sets with equal strings on planted random texts: ragged
    sizes around the tile lengths and unaligned starts (views at offsets)."""
    g = np.random.Generator(np.random.PCG64(len(alpha) * 7 + len(kw)))
    pats, stems = nested(g, alpha, 300, 40)
    with api.Automaton(pats, **kw) as a:
        for n in SIZES:
            text = planted_text(g, alpha, n + 5, stems)
            t = _gpu.to_dev(text)
            for off in (0, 3):
                if n + off <= text.size:
                    check(a.handle, pats, text[off:off + n], t=t[off:off + n])


@pytest.mark.parametrize("kernel", ["walk_slots", "thread_jump", "thread_jump_l1"])
def test_full_8bit_kernels(kernel):
    """The byte-alphabet kernels' slot modes feed the expansion alike."""
    text = workloads.zipf_text(200_000, 11)
    pats = workloads.keywords_zipf(text, 3000, 1, 12, 0.5, seed=12)
    pats = pats + [p[:max(1, len(p) // 2)] for p in pats[:500]]  # prefixes of keywords
    with api.Automaton(pats) as a:
        a.set_kernel(kernel)
        check(a.handle, pats, text)


@pytest.mark.parametrize("kind", ["zipf", "dense_bytes"])
def test_full_phased_form(kind):
    """Texts long enough for the phased form (8-bit codes, 5 MiB): its second
    and third steps feed the expansion, and with no dense fallback a tile with
    more than 32 matches is matched again by the expansion kernels.  Zipf
    keywords with their prefixes; and every string of 1-2 bytes over a few
    byte values (every position matches several times, so nearly every tile
    is matched again)."""
    g = np.random.default_rng(21)
    if kind == "zipf":
        text = workloads.zipf_text(5 << 20, 23)
        pats = workloads.keywords_zipf(text[:1 << 20], 3000, 3, 40, 0.5, seed=24)
        pats = pats + [p[:max(1, len(p) // 2)] for p in pats[:500]]
    else:
        vals = np.frombuffer(bytes(range(60, 80)), dtype=np.uint8)
        text = vals[g.integers(0, vals.size, size=5 << 20)].copy()
        text[g.integers(0, text.size, size=1000)] = 200  # bytes in no keyword
        pats = [bytes([a]) for a in vals] + [bytes([a, b]) for a in vals[:8] for b in vals[:8]]  # 20 keyword bytes
    with api.Automaton(pats) as a:
        assert a.info()["code_bits"] == 8
        check(a.handle, pats, text)


def test_full_dense_tiles():
    """Every string of length 1..3 over ACGT is a keyword (with repeats): every
    position starts three occurrences, so every tile has more matches than its
    slots and goes through the dense fallback."""
    import itertools

    pats = [bytes(p) for L in (1, 2, 3) for p in itertools.product(b"ACGT", repeat=L)]
    pats += pats[:20]
    text = workloads.acgt_text(50_000, 5)
    with api.Automaton(pats) as a:
        check(a.handle, pats, text)
        check(a.handle, pats, text[7:7 + 30_001])


def test_full_small_cap():
    """Room for only some occurrences: the first cap entries and the true total."""
    g = np.random.Generator(np.random.PCG64(3))
    pats, stems = nested(g, b"ACGT", 200, 30)
    text = planted_text(g, b"ACGT", 200_000, stems)
    with api.Automaton(pats) as a:
        total = want_full(pats, text)[0].size
        assert total > 100
        for cap in (1, 7, total // 3, total - 1):
            check(a.handle, pats, text, cap=cap)


def test_full_workload_sample():
    """The ACGT sweep set (10,000 keywords of 16-64 bytes plus their 8-byte
    prefixes as extra keywords) on a 4 MiB text: sub-patterns of every match."""
    text, pats = workloads.sweep_acgt(4 << 20, seed=0)
    pats = list(pats) + [p[:8] for p in pats[:2000]]
    with api.Automaton(pats) as a:
        check(a.handle, pats, text)


def test_full_empty_text():
    import torch

    with api.Automaton([b"ab", b"a"]) as a:
        c = torch.full((1,), 5, dtype=torch.int64, device="cuda")
        e = torch.zeros(1, dtype=torch.int32, device="cuda")
        api.ac_match_full(a.handle, e, 0, e, e, 1, c)
        assert int(c.item()) == 0
