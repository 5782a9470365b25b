"""Parity at full size, every position: the CUDA path through the C ABI against
the CPU oracle run over the whole text on every host core (tests/_par.py: the
id at start i depends only on text[i : i + max_len], so stretches with a
max_len - 1 halo reproduce one serial pass exactly).

* the benchmark's workload in its launch configuration: 1 GiB of ACGT text,
  the 10,000-keyword sweep set, dense ids (plus count and compacted list);
* every other size of the input-size sweep (4 KiB .. 256 MiB, prefixes of the
  same text);
* texts on both sides of the launcher's switch between the kernel forms that
  share heavy tiles within the CTA and the plain forms;
* the byte-alphabet workload at 256 MiB (Zipf(1.1) bytes, its own 20,000
  keywords): compacted list, count and dense ids, every 8-bit kernel;
* the host-buffer call across its 64 MiB chunk seams.
"""
import numpy as np
import pytest

from paper_1412_7789_gb300 import api, workloads
from tests import _par

pytestmark = pytest.mark.gpu

TILE = 992            # positions per tile of the small-alphabet kernel
HELP_TILES_PER_WARP = 16
WARPS_PER_CTA = 16    # default launch: 512 threads


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1412_7789_gb300 import build

    build.build()
    api.lib()
    yield
    assert api.ac_device_status() == api.AC_OK


@pytest.fixture(scope="module")
def sweep():
    import torch

    text, pats = workloads.sweep_acgt(1 << 30)
    wpos, wids = _par.oracle_compact(pats, text)
    t = torch.from_numpy(text).cuda()
    a = api.Automaton(pats)
    yield text, pats, wpos, wids, t, a
    a.close()
    del t
    torch.cuda.empty_cache()


def _all_outputs(a, t, n, wpos, wids, what):
    """Dense ids, count and compacted list of text t[:n] against the oracle's list."""
    _par.check_outputs(a.handle, t, n, wpos, wids, what)


def test_sweep_1gib_every_position(sweep):
    """The benchmark's step (ac_match on the 1 GiB text, default launch:
    survivors resolved in the warps), and the same with the survivors listed
    for the second kernel."""
    text, pats, wpos, wids, t, a = sweep
    assert wpos.size > 1000
    _all_outputs(a, t, text.size, wpos, wids, "1 GiB")
    a.set_tuning(survivor_list=1)
    try:
        _all_outputs(a, t, text.size, wpos, wids, "1 GiB, survivors listed")
    finally:
        a.set_tuning(survivor_list=0)


def test_sweep_sizes_every_position(sweep):
    text, pats, wpos, wids, t, a = sweep
    for n in workloads.SWEEP_SIZES[:-1]:
        p, i = _par.window_compact(wpos, wids, pats, text, 0, n)
        _all_outputs(a, t[:n], n, p, i, "%d B" % n)


def test_shared_and_plain_forms_boundary(sweep):
    """Texts of exactly the largest tile count that takes the forms sharing
    heavy tiles within the CTA (16 tiles per warp of the grid), one tile
    fewer, one and two more (plain forms; with the survivor list asked for,
    two more is the first that lists them for the second kernel), each with a
    ragged last tile; the heavy tiles of the sweep set's first 4 KiB run in
    every form."""
    import torch

    text, pats, wpos, wids, t, a = sweep
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    edge = HELP_TILES_PER_WARP * sms * WARPS_PER_CTA
    for tiles, listed in ((edge - 1, 0), (edge, 0), (edge + 1, 0), (edge + 2, 0), (edge + 1, 1), (edge + 2, 1)):
        n = tiles * TILE - 37
        p, i = _par.window_compact(wpos, wids, pats, text, 0, n)
        a.set_tuning(survivor_list=listed)
        try:
            _all_outputs(a, t[:n], n, p, i, "%d tiles, survivor list %d" % (tiles, listed))
        finally:
            a.set_tuning(survivor_list=0)


@pytest.fixture(scope="module")
def zipf():
    import torch

    text, pats = workloads.zipf_byte(256 << 20)
    wpos, wids = _par.oracle_compact(pats, text)
    t = torch.from_numpy(text).cuda()
    yield text, pats, wpos, wids, t
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kernel", ["tiled", "walk_slots", "thread_jump", "thread_jump_l1"])
def test_zipf_256mib_every_match(zipf, kernel):
    text, pats, wpos, wids, t = zipf
    assert wpos.size > 10000
    with api.Automaton(pats) as a:
        a.set_kernel(kernel)
        _all_outputs(a, t, text.size, wpos, wids, "zipf 256 MiB " + kernel)


def test_match_host_every_position():
    """ac_match_host: 64 MiB chunks with a max_len halo each, pinned host
    buffers, a text ending 12,345 bytes into its second chunk."""
    import torch

    n = (64 << 20) + 12_345
    text, pats = workloads.sweep_acgt(n, seed=4)
    wpos, wids = _par.oracle_compact(pats, text)
    with api.Automaton(pats) as a:
        ht = torch.from_numpy(text).pin_memory()
        got = a.match_host(ht)
        _par.check_dense(got, wpos, wids, "host")
        small = text[:5000]
        p, i = _par.window_compact(wpos, wids, pats, text, 0, small.size)
        got = a.match_host(torch.from_numpy(small.copy()))
        _par.check_dense(got, p, i, "host small")


@pytest.mark.parametrize("listed", [0, 1])
@pytest.mark.parametrize("kind", ["short_keywords", "dense_matches"])
def test_phased_small_alphabet_and_list_overflow(kind, listed):
    """2- and 4-bit codes on texts long enough for the phased form (by
    default for dense ids and counts, as both sets' root windows often end a
    keyword, and for every output when the survivor_list knob asks): ACGT
    keywords of 1-3 bytes (nearly every position survives, so the survivor
    list fills and most tiles fall back to their warps), and a 12-letter set
    whose windows often reach the stride table and beyond (the walk list),
    with non-keyword bytes sprinkled in (tiles that stay with their warps).
    Dense ids, count and compacted list, every position, against the oracle."""
    import torch

    g = np.random.default_rng(31)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = (HELP_TILES_PER_WARP * sms * WARPS_PER_CTA + 300) * TILE + 77
    if kind == "short_keywords":
        text = workloads.acgt_text(n, 32)
        acgt = np.frombuffer(b"ACGT", dtype=np.uint8)
        pats = [bytes(acgt[g.integers(0, 4, size=int(g.integers(1, 4)))]) for _ in range(60)]
    else:
        alpha = np.frombuffer(b"abcdefghijkl", dtype=np.uint8)
        text = alpha[g.integers(0, 3, size=n)].copy()  # three letters: long walks
        text[g.integers(0, n, size=n // 5000)] = ord("z")
        pats = [bytes(alpha[g.integers(0, 3, size=int(g.integers(6, 30)))]) for _ in range(2000)]
        pats += [bytes(alpha[g.integers(0, 12, size=int(g.integers(2, 9)))]) for _ in range(500)]
    wpos, wids = _par.oracle_compact(pats, text)
    t = _gpu_tensor(text)
    with api.Automaton(pats) as a:
        info = a.info()
        assert info["code_bits"] in (2, 4) and info["match_windows_ppm"] >= 500
        a.set_tuning(survivor_list=listed)
        _all_outputs(a, t, text.size, wpos, wids, kind)


def test_direct_codes_long_text_with_other_bytes(sweep):
    """Codes taken as (byte >> 1) & 3 in the one-phase forms at the widest
    launch (texts beyond the forms that share heavy tiles): the sweep set on
    48 MiB of its text with one byte in a thousand replaced by a byte in no
    keyword ('N', or a keyword byte with a bit above its code bits flipped,
    so the same code); and lowercase DNA keywords of 1-20 letters (nearly
    every position survives the filter, most tiles are heavy) on 40 MiB with
    one byte in a hundred replaced.  Dense ids, count and compacted list,
    every position, against the oracle."""
    import torch

    text, pats, _, _, _, a = sweep
    assert a.info()["class_direct_shift"] == 1
    g = np.random.default_rng(41)
    n = 48 << 20
    t = text[:n].copy()
    hit = np.nonzero(g.random(n) < 1e-3)[0]
    t[hit] = np.frombuffer(b"NIKOV", dtype=np.uint8)[g.integers(0, 5, size=hit.size)]
    wpos, wids = _par.oracle_compact(pats, t)
    d = torch.from_numpy(t).cuda()
    _all_outputs(a, d, n, wpos, wids, "48 MiB with other bytes")
    # an unaligned start and a ragged end: fringe tiles at both ends
    off, m = 5, n - 5 - 777
    p, i = _par.window_compact(wpos, wids, pats, t, off, m)
    _all_outputs(a, d[off:off + m], m, p, i, "48 MiB at offset 5")
    del d

    low = np.frombuffer(b"acgt", dtype=np.uint8)
    n = 40 << 20
    t = low[g.integers(0, 4, size=n)]
    hit = np.nonzero(g.random(n) < 1e-2)[0]
    t[hit] = np.frombuffer(b"qswdNbfu\x00\xff", dtype=np.uint8)[g.integers(0, 10, size=hit.size)]
    kws = [bytes(low[g.integers(0, 4, size=int(g.integers(1, 21)))]) for _ in range(300)]
    wpos, wids = _par.oracle_compact(kws, t)
    d = torch.from_numpy(t).cuda()
    with api.Automaton(kws) as b:
        assert b.info()["class_direct_shift"] == 1
        b.set_tuning(survivor_list=2)  # one phase for every output
        _all_outputs(b, d, n, wpos, wids, "40 MiB lowercase with other bytes")


@pytest.mark.parametrize("kind", ["short_keywords", "zipf_sparse"])
def test_two_phase_byte_form_and_list_overflow(kind):
    """8-bit codes on texts long enough for the two-phase form: a keyword set
    whose windows nearly all survive the filter (keywords of 1-3 bytes) fills
    the survivor list, so most tiles fall back to their warps; a sparse set
    lists nearly every tile.  Dense ids, count and compacted list, every
    position, against the oracle."""
    g = np.random.default_rng(17)
    text = workloads.zipf_text(6 << 20, 21)
    if kind == "short_keywords":
        pats = [bytes(g.integers(0, 64, size=int(g.integers(1, 4)), dtype=np.uint8)) for _ in range(3000)]
    else:
        pats = workloads.keywords_zipf(text[:1 << 20], 5000, 4, 60, 0.3, seed=22)
    wpos, wids = _par.oracle_compact(pats, text)
    t = _gpu_tensor(text)
    with api.Automaton(pats) as a:
        assert a.info()["code_bits"] == 8
        _all_outputs(a, t, text.size, wpos, wids, kind)


def _gpu_tensor(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
