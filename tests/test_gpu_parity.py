"""CUDA path against the CPU oracle, bit-exact, through the C ABI."""
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


def compile_(pats, **kw):
    return api.Automaton(pats, **kw)


@pytest.mark.parametrize("name", ["w1_ushers.txt", "w2_fig45.txt"])
@pytest.mark.parametrize("kernel", ["tiled", "simple"])
def test_golden(name, kernel):
    keywords, cases = _pins.read_golden(name)
    with compile_(keywords) as a:
        a.set_kernel(kernel)
        for c in cases:
            want = np.array(c["ids"], dtype=np.int32)
            text = np.frombuffer(c["text"], dtype=np.uint8)
            modes = ("dense", "count", "compact") if kernel == "tiled" else ("dense",)
            _gpu.check_all_modes(a.handle, text, want, modes=modes)


@pytest.mark.parametrize("count", [5, 10])
def test_paper_mode(count):
    pats = workloads.paper_keywords(count, seed=0)
    with compile_(pats) as a:
        for n in (26, 1310, 16375, 40000, 53710, 671375):
            text = workloads.paper_text(n)
            want = _pins.paper_closed_form(n)
            assert np.array_equal(oracle.pfac_ids(pats, text), want)
            _gpu.check_all_modes(a.handle, text, want)


def test_single_text_acgt_1mib():
    text, pats = workloads.single_text_acgt(seed=0)
    want = oracle.pfac_ids(pats, text)
    assert oracle.count(want) > 0
    with compile_(pats) as a:
        _gpu.check_all_modes(a.handle, text, want)
        a.set_kernel("simple")
        _gpu.check_all_modes(a.handle, text, want, modes=("dense",))


SIZES = [0, 1, 15, 16, 17, 63, 8191, 8192, 8193, 3 * 8192 + 77, 100_003]
ALPHABETS = {
    "ab": b"ab",                              # 2 classes   -> 2-bit codes, hashed
    "acgt": b"ACGT",                          # 4 classes   -> 2-bit codes, hashed
    "nohash4": bytes([0x00, 0x01, 0x80, 0x81]),  # 2-bit codes, class table
    "seven": b"abcdefg",                      # 7 classes   -> 4-bit codes, hashed
    "nohash5": bytes([0x00, 0x01, 0x02, 0x80, 0x81]),  # 4-bit codes, class table
    "ten": b"abcdefghij",                     # 10 classes  -> 4-bit codes, class table
    "forty": bytes(range(40, 80)),            # 40 classes  -> 8-bit codes, unknown bytes possible
    "many": bytes(range(0, 250)),             # 250 classes -> 8-bit codes above 127
    "bytes": bytes(range(256)),               # 256 classes -> raw bytes
}


def random_case(g, alphabet: bytes, n: int, kw: int, lmax: int):
    a = np.frombuffer(alphabet, dtype=np.uint8)
    text = a[g.integers(0, a.size, size=n)] if n else np.zeros(0, np.uint8)
    pats = []
    for _ in range(kw):
        L = int(g.integers(1, lmax + 1))
        if n > L and g.random() < 0.5:
            o = int(g.integers(0, n - L))
            pats.append(bytes(text[o:o + L]))
        else:
            pats.append(bytes(a[g.integers(0, a.size, size=L)]))
    return text, pats


@pytest.mark.parametrize("kernel", ["tiled", "walk_slots", "thread_jump", "thread_jump_l1"])
@pytest.mark.parametrize("alpha", sorted(ALPHABETS))
def test_random_sizes(alpha, kernel):
    """Every kernel variant (the 8-bit ones differ; small alphabets always use
    the filter kernel) on every code width and many sizes."""
    g = np.random.Generator(np.random.PCG64(sorted(ALPHABETS).index(alpha) + 1000))
    for n in SIZES:
        text, pats = random_case(g, ALPHABETS[alpha], max(n, 40), 50, 24)
        text = text[:n]
        want = oracle.pfac_ids(pats, text)
        with compile_(pats) as a:
            a.set_kernel(kernel)
            _gpu.check_all_modes(a.handle, text, want)


@pytest.mark.parametrize("opts", [
    dict(class_compress=False),
    dict(index_width=32),
    dict(jump_bytes=64, stride_bytes=1),
    dict(jump_bytes=1024),
    dict(stride_bytes=1),
])
def test_build_options_keep_results(opts):
    g = np.random.Generator(np.random.PCG64(99))
    text, pats = random_case(g, b"ACGT", 200_000, 400, 40)
    text2, pats2 = random_case(g, bytes(range(0, 256, 3)), 50_000, 300, 30)
    for t, p in ((text, pats), (text2, pats2)):
        want = oracle.pfac_ids(p, t)
        with compile_(p, **opts) as a:
            _gpu.check_all_modes(a.handle, t, want)


@pytest.mark.parametrize("kernel", ["tiled", "walk_slots", "thread_jump", "thread_jump_l1"])
def test_longest_walk_and_edges(kernel):
    """A run of one byte with keywords of that byte x1..x100: every start walks
    to the end of its run (the longest walks the method has)."""
    pats = [b"\x00" * L for L in range(1, 101)] + [b"\xff\x00", b"\x00\xff", b"\xff" * 3]
    for n in (5, 99, 100, 101, 4096, 20_000):
        text = np.zeros(n, dtype=np.uint8)
        text[n // 2] = 0xFF
        text[-1] = 0xFF
        want = oracle.pfac_ids(pats, text)
        with compile_(pats) as a:
            a.set_kernel(kernel)
            _gpu.check_all_modes(a.handle, text, want)


def test_keyword_longer_than_text_and_duplicates():
    pats = [b"ACGTACGTACGTACGTACGT" * 4, b"ACG", b"ACG", b"A", b"ACGTA", b"CGTAC" * 30]
    text = np.frombuffer(b"ACGTACGTAC", dtype=np.uint8)
    want = oracle.pfac_ids(pats, text)
    assert want.tolist()[:2] == [4, -1]
    with compile_(pats) as a:
        _gpu.check_all_modes(a.handle, text, want)


@pytest.mark.parametrize("kernel", ["tiled", "walk_slots", "thread_jump", "thread_jump_l1"])
def test_many_keywords_over_15_bits(kernel):
    """More than 32767 keywords: 32-bit goto entries, and jump-table results
    that do not fit 15 bits go to the plain walk."""
    g = np.random.Generator(np.random.PCG64(5))
    two = [bytes([a, b]) for a in range(256) for b in range(256)]
    order = g.permutation(len(two))[:40_000]
    pats = [two[i] for i in order] + [bytes(g.integers(0, 256, size=5).astype(np.uint8)) for _ in range(100)]
    text = workloads.zipf_text(300_000, 3)
    want = oracle.pfac_ids(pats, text)
    with compile_(pats) as a:
        assert a.info()["index_width"] == 32
        a.set_kernel(kernel)
        _gpu.check_all_modes(a.handle, text, want)


def _other_bytes(alphabet: bytes) -> np.ndarray:
    """Bytes in no keyword: each keyword byte with a bit above its code bits
    (bits 1-2) flipped (same code, another byte), 'N', 0x00 and 0xFF."""
    extra = {b ^ 0x10 for b in alphabet} | {b ^ 0x01 for b in alphabet} | {ord("N"), 0x00, 0xFF}
    return np.array(sorted(extra - set(alphabet)), dtype=np.uint8)


@pytest.mark.parametrize("alphabet,shift", [(b"ACGT", 1), (b"acgt", 1), (bytes([0x00, 0x02, 0x04, 0x06]), 1),
                                            (bytes([0x00, 0x01, 0x80, 0x81]), -1)])
def test_direct_codes_and_other_bytes(alphabet, shift):
    """2-bit codes computed as (byte >> 1) & 3 (and, for comparison, a
    four-byte alphabet without them) on texts of the four keyword
    bytes with other bytes mixed in (some with a keyword byte's code bits),
    from none to one in three, at sizes across tiles with ragged ends and at
    unaligned pointers: dense ids, count and compacted list against the
    oracle."""
    g = np.random.Generator(np.random.PCG64(shift * 7 + alphabet[0] + 10))
    others = _other_bytes(alphabet)
    for n, rate in ((5000, 0.3), (3 * 8192 + 77, 0.01), (100_003, 1e-4), (100_003, 0.0), (250_001, 0.002)):
        text, pats = random_case(g, alphabet, n, 120, 24)
        hit = g.random(n) < rate
        text[hit] = others[g.integers(0, others.size, size=int(hit.sum()))]
        want = oracle.pfac_ids(pats, text)
        with compile_(pats) as a:
            assert a.info()["class_direct_shift"] == shift and a.info()["code_bits"] == 2
            _gpu.check_all_modes(a.handle, text, want)
            base = _gpu.to_dev(text)
            for off in (3, 13):
                sub_want = oracle.pfac_ids(pats, text[off:])
                _gpu.check_all_modes(a.handle, text[off:], sub_want, t=base[off:])


def test_unaligned_pointers():
    import torch

    g = np.random.Generator(np.random.PCG64(11))
    text, pats = random_case(g, b"ACGT", 70_000, 200, 30)
    with compile_(pats) as a:
        base = _gpu.to_dev(text)
        for off in (1, 3, 7, 13, 16):
            for n in (0, 1, 17, 40_000, text.size - off):
                t = base[off:off + n]
                want = oracle.pfac_ids(pats, text[off:off + n])
                out = torch.full((n + 8,), -7, dtype=torch.int32, device="cuda")
                for oo in (0, 1, 2, 3):
                    o = out[oo:oo + n]
                    api.ac_match(a.handle, t, n, o)
                    assert np.array_equal(o.cpu().numpy(), want), (off, n, oo)
                _gpu.check_all_modes(a.handle, text[off:off + n], want, t=t, modes=("count", "compact"))


@pytest.mark.parametrize("n", [4096, 65536, 1 << 20])
def test_sweep_keywords_full(n):
    text, pats = workloads.sweep_acgt(n)
    want = oracle.pfac_ids(pats, text)
    with compile_(pats) as a:
        _gpu.check_all_modes(a.handle, text, want)


@pytest.mark.parametrize("kernel", ["tiled", "walk_slots", "thread_jump", "thread_jump_l1"])
def test_zipf_compact_and_overflow(kernel):
    text, pats = workloads.zipf_byte(1 << 22, n_keywords=20_000)
    want = oracle.pfac_ids(pats, text)
    wpos, wid = oracle.compact(want)
    assert wpos.size > 100
    with compile_(pats) as a:
        a.set_kernel(kernel)
        _gpu.check_all_modes(a.handle, text, want)
        t = _gpu.to_dev(text)
        cap = wpos.size // 3
        pos, ids, total = _gpu.compact(a.handle, t, cap)
        assert total == wpos.size and pos.size == cap
        assert np.array_equal(pos, wpos[:cap]) and np.array_equal(ids, wid[:cap])
        pos, ids, total = _gpu.compact(a.handle, t, 0)
        assert total == wpos.size and pos.size == 0


@pytest.mark.parametrize("kernel", ["tiled", "walk_slots", "thread_jump", "thread_jump_l1"])
@pytest.mark.parametrize("alpha", ["acgt", "bytes"])
def test_dense_matches_compact(alpha, kernel):
    """Nearly every position matches (one-byte keywords), so every tile holds
    more matches than its slots and the compacted list comes from the tiles'
    dense ids; the static-scratch call matches such tiles again instead."""
    import torch

    g = np.random.Generator(np.random.PCG64(77))
    text, pats = random_case(g, ALPHABETS[alpha], 300_001, 60, 12)
    pats += [bytes([b]) for b in ALPHABETS[alpha][::3]]
    want = oracle.pfac_ids(pats, text)
    assert (want >= 0).mean() > 0.2
    with compile_(pats) as a:
        a.set_kernel(kernel)
        _gpu.check_all_modes(a.handle, text, want, modes=("compact", "count"))
        wpos, wid = oracle.compact(want)
        t = _gpu.to_dev(text)
        pos = torch.full((wpos.size,), -7, dtype=torch.int32, device="cuda")
        ids = torch.full((wpos.size,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        api.ac_match_compact_static(a.handle, t, text.size, pos, ids, wpos.size, cnt)
        assert int(cnt.item()) == wpos.size
        assert np.array_equal(pos.cpu().numpy().astype(np.uint32), wpos)
        assert np.array_equal(ids.cpu().numpy().astype(np.uint32), wid)


@pytest.mark.parametrize("alpha,kernel", [(b"ACGT", "tiled"), (b"abcdefghijklmnopqrstuvwxyz", "tiled"),
                                          (b"abcdefghijklmnopqrstuvwxyz", "thread_jump"),
                                          (b"abcdefghijklmnopqrstuvwxyz", "walk_slots")])
def test_counter_free_boundary(alpha, kernel):
    """Dense ids and counts of texts just below and above the largest text
    whose tiles (or rows) all go to the warps' first claims -- launched
    without a tile counter -- and of two calls in a row on the same handle."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    g = np.random.Generator(np.random.PCG64(len(alpha) + len(kernel)))
    a = np.frombuffer(alpha, dtype=np.uint8)
    base = a[g.integers(0, a.size, size=1 << 22)]
    pats = [bytes(base[o:o + int(L)]) for o, L in zip(g.integers(0, 1 << 20, size=300), g.integers(3, 20, size=300))]
    if alpha == b"ACGT":
        edge = sms * 16 * 992  # filter kernel: 16 warps per CTA, 992 positions per tile
    elif kernel == "tiled":
        edge = sms * 4 * 1024  # full-occupancy 8-bit kernel: 64-position rows, 8 warps x 8 CTAs per SM
    elif kernel == "thread_jump":
        edge = sms * 32 * 1024  # one CTA of 32 warps per SM, 1024-position tiles
    else:
        edge = sms * 16 * 1024
    with compile_(pats) as h:
        h.set_kernel(kernel)
        for n in (edge - 4096, edge - 1, edge, edge + 1, edge + 4096):
            text = base[:n]
            want = oracle.pfac_ids(pats, text)
            _gpu.check_all_modes(h.handle, text, want, modes=("dense", "count"))
