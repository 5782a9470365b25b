"""Batches through the C ABI against the CPU oracle, bit-exact: every text of a
batch must get exactly the ids the oracle gives for that text alone (walks stop
at the end of their own text), and nothing outside the texts' output ranges
may be written."""
import numpy as np
import pytest

import oracle
from paper_1412_7789_gb300 import api, workloads
from tests import _gpu

pytestmark = pytest.mark.gpu

SENTINEL = -7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1412_7789_gb300 import build

    build.build()
    api.lib()
    yield
    assert api.ac_device_status() == api.AC_OK


@pytest.fixture(scope="module")
def automata():
    """Five automata of the kinds a batch mixes: 2-bit (ACGT filter), 4-bit
    (filter, 12 keyword bytes), 8-bit with class compression (Zipf), 8-bit
    with 256 columns, and a 16-bit-index ACGT set with long keywords."""
    g = np.random.default_rng(5)
    acgt = workloads.keywords_acgt(workloads.acgt_text(1 << 16, 1), 300, 4, 40, 0.5, seed=2)
    alpha12 = np.frombuffer(b"abcdefghijkl", dtype=np.uint8)
    four = [bytes(alpha12[g.integers(0, 12, size=int(g.integers(2, 12)))]) for _ in range(200)]
    zipf = workloads.keywords_zipf(workloads.zipf_text(1 << 16, 3), 400, 2, 30, 0.3, seed=4)
    full = [bytes(g.integers(0, 256, size=int(g.integers(1, 6)), dtype=np.uint8)) for _ in range(150)]
    longk = workloads.keywords_acgt(workloads.acgt_text(1 << 16, 6), 40, 60, 200, 1.0, seed=7)
    sets = [acgt, four, zipf, full, longk]
    hs = [api.Automaton(acgt), api.Automaton(four), api.Automaton(zipf), api.Automaton(full, class_compress=False),
          api.Automaton(longk)]
    yield sets, hs
    for a in hs:
        a.close()


def _text_for(kind: int, n: int, seed: int, sets) -> np.ndarray:
    g = np.random.default_rng(seed)
    if kind in (0, 4):
        t = workloads.acgt_text(n, seed)
    elif kind == 1:
        t = np.frombuffer(b"abcdefghijklmn", dtype=np.uint8)[g.integers(0, 14, size=n)]
    else:
        t = workloads.zipf_text(n, seed)
    t = np.array(t, dtype=np.uint8)
    # plant a few keywords of the text's own set
    pats = sets[kind]
    for _ in range(min(8, n // 64)):
        p = pats[int(g.integers(0, len(pats)))]
        if len(p) < n:
            o = int(g.integers(0, n - len(p) + 1))
            t[o:o + len(p)] = np.frombuffer(p, dtype=np.uint8)
    return t


def _run_and_check(hs, sets, texts, kinds, text_off, out_off, buf_len, out_len, runner):
    import torch

    buf = np.zeros(buf_len, dtype=np.uint8)
    for t, o in zip(texts, text_off):
        buf[o:o + t.size] = t
    items = api.batch_items(text_off, [t.size for t in texts], out_off, kinds)
    d_buf = _gpu.to_dev(buf)
    d_items = api.items_to_device(items)
    out = torch.full((out_len,), SENTINEL, dtype=torch.int32, device="cuda")
    runner(d_buf, d_items, len(texts), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    written = np.zeros(out_len, dtype=bool)
    for i, (t, o) in enumerate(zip(texts, out_off)):
        want = oracle.pfac_ids(sets[kinds[i]], t) if t.size else np.zeros(0, dtype=np.int32)
        g = got[o:o + t.size]
        if not np.array_equal(g, want):
            bad = np.nonzero(g != want)[0]
            raise AssertionError("text %d (len %d, set %d): %d mismatches, first %s got %s want %s" % (
                i, t.size, kinds[i], bad.size, bad[:6].tolist(), g[bad[:6]].tolist(), want[bad[:6]].tolist()))
        written[o:o + t.size] = True
    assert np.all(got[~written] == SENTINEL), "a batch wrote outside its texts' output ranges"


EDGE_LENGTHS = [0, 1, 2, 15, 16, 17, 31, 63, 64, 65, 495, 496, 497, 991, 992, 993, 1023, 1024, 1025, 2047,
                2048, 3000, 5000, 20000]


def _edge_batch(sets, seed):
    g = np.random.default_rng(seed)
    lens = EDGE_LENGTHS * 2 + [int(x) for x in g.integers(1, 70000, size=20)]
    kinds = [int(x) for x in g.integers(0, len(sets), size=len(lens))]
    texts = [_text_for(k, n, seed * 1000 + i, sets) for i, (k, n) in enumerate(zip(kinds, lens))]
    # texts at random, mostly unaligned offsets with gaps; outputs in another order
    text_off, pos = [], 3
    for t in texts:
        pos += int(g.integers(0, 40))
        text_off.append(pos)
        pos += t.size
    buf_len = pos + 64
    order = g.permutation(len(texts))
    out_off = [0] * len(texts)
    opos = 1
    for j in order:
        opos += int(g.integers(0, 9))
        out_off[j] = opos
        opos += texts[j].size
    return texts, kinds, text_off, out_off, buf_len, opos + 16


@pytest.mark.parametrize("seed", [1, 2])
def test_batch_edges_match_oracle(automata, seed):
    sets, hs = automata
    texts, kinds, text_off, out_off, buf_len, out_len = _edge_batch(sets, seed)
    handles = [a.handle for a in hs]
    _run_and_check(hs, sets, texts, kinds, text_off, out_off, buf_len, out_len,
                   lambda b, it, k, o: api.ac_match_batch(handles, b, it, k, o))


def test_batch_plan_run_capture_replay(automata):
    import torch

    sets, hs = automata
    handles = [a.handle for a in hs]
    texts, kinds, text_off, out_off, buf_len, out_len = _edge_batch(sets, 3)
    with api.BatchPlan(handles, max_items=len(texts) + 5) as plan:
        _run_and_check(hs, sets, texts, kinds, text_off, out_off, buf_len, out_len,
                       lambda b, it, k, o: plan.run(b, it, k, o))

        # capture once, then replay with changed item contents (same buffers)
        buf = np.zeros(buf_len, dtype=np.uint8)
        d_buf = _gpu.to_dev(buf)
        d_items = api.items_to_device(api.batch_items(text_off, [t.size for t in texts], out_off, kinds))
        out = torch.full((out_len,), SENTINEL, dtype=torch.int32, device="cuda")
        plan.capture(d_buf, d_items, len(texts), out)
        g = np.random.default_rng(11)
        for rep in range(3):
            # new lengths (no longer than the slots) and automata for each text
            kinds2 = [int(x) for x in g.integers(0, len(sets), size=len(texts))]
            texts2 = [_text_for(k, int(g.integers(0, t.size + 1)), 50_000 + 100 * rep + i, sets)
                      for i, (k, t) in enumerate(zip(kinds2, texts))]
            for t, o in zip(texts2, text_off):
                buf[o:o + t.size] = t
            d_buf.copy_(torch.from_numpy(buf))
            items2 = api.batch_items(text_off, [t.size for t in texts2], out_off, kinds2)
            d_items.copy_(api.items_to_device(items2))
            out.fill_(SENTINEL)
            plan.replay()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            written = np.zeros(out_len, dtype=bool)
            for i, (t, o) in enumerate(zip(texts2, out_off)):
                want = oracle.pfac_ids(sets[kinds2[i]], t) if t.size else np.zeros(0, dtype=np.int32)
                assert np.array_equal(got[o:o + t.size], want), (rep, i, t.size, kinds2[i])
                written[o:o + t.size] = True
            assert np.all(got[~written] == SENTINEL)


@pytest.mark.parametrize("reserve", [64 << 20, 4096])
def test_batch_plan_survivor_lists(automata, reserve):
    """The phased form inside the one persistent launch: the plan's 8-bit-code
    automata, and the 2- and 4-bit ones whose root windows often end a
    keyword (the first two sets; not the long-keyword one), list their
    survivors for the second and third launches.  The
    edge batch and a batch of longer texts (every kind, Zipf ones up to 1.5
    MB), run and captured: every text's ids are the oracle's, nothing outside
    the output ranges is written.  A 4 KiB reservation (512 entries) overflows
    at once, so nearly every tile falls back to its warp; reserving again
    drops the captured graph."""
    import torch

    sets, hs = automata
    handles = [a.handle for a in hs]
    ppm = [a.info()["match_windows_ppm"] for a in hs]
    assert ppm[0] >= 500 and ppm[1] >= 500 and ppm[4] < 500
    g = np.random.default_rng(77)
    texts, kinds, text_off, out_off, buf_len, out_len = _edge_batch(sets, 5)
    lens = [int(x) for x in g.integers(100_000, 1_500_000, size=10)]
    kinds2 = [2, 3, 2, 3, 0, 1, 2, 4, 2, 3]
    long_texts = [_text_for(k, n, 500 + i, sets) for i, (k, n) in enumerate(zip(kinds2, lens))]
    text_off2 = list(np.cumsum([0] + lens[:-1]) + 5)
    out_off2 = list(np.cumsum([0] + lens[:-1]) + 3)
    with api.BatchPlan(handles, max_items=len(texts) + 5) as plan:
        plan.reserve_lists(reserve)
        for args in ((texts, kinds, text_off, out_off, buf_len, out_len),
                     (long_texts, kinds2, text_off2, out_off2, sum(lens) + 64, sum(lens) + 64)):
            _run_and_check(hs, sets, *args[:2], *args[2:],
                           runner=lambda b, it, k, o: plan.run(b, it, k, o))
        # capture with the lists, replay
        buf = np.zeros(sum(lens) + 64, dtype=np.uint8)
        for t, o in zip(long_texts, text_off2):
            buf[o:o + t.size] = t
        d_buf = _gpu.to_dev(buf)
        d_items = api.items_to_device(api.batch_items(text_off2, lens, out_off2, kinds2))
        out = torch.full((sum(lens) + 64,), SENTINEL, dtype=torch.int32, device="cuda")
        plan.capture(d_buf, d_items, len(long_texts), out)
        plan.replay()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, (t, o) in enumerate(zip(long_texts, out_off2)):
            assert np.array_equal(got[o:o + t.size], oracle.pfac_ids(sets[kinds2[i]], t)), i
        plan.reserve_lists(reserve // 2)
        with pytest.raises(api.AcError):
            plan.replay()


def test_batch_bad_automaton_is_reported(automata):
    import torch

    sets, hs = automata
    handles = [a.handle for a in hs[:2]]
    texts = [_text_for(0, 5000, 1, sets), _text_for(1, 3000, 2, sets), _text_for(0, 100, 3, sets)]
    kinds = [0, 1, 7]  # the last names no handle: skipped, error latched
    offs = [0, 5000, 8000]
    items = api.batch_items(offs, [t.size for t in texts], offs, kinds)
    d_buf = _gpu.to_dev(np.concatenate(texts))
    out = torch.full((8100,), SENTINEL, dtype=torch.int32, device="cuda")
    api.ac_match_batch(handles, d_buf, api.items_to_device(items), 3, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got[:5000], oracle.pfac_ids(sets[0], texts[0]))
    assert np.array_equal(got[5000:8000], oracle.pfac_ids(sets[1], texts[1]))
    assert np.all(got[8000:] == SENTINEL)
    assert api.ac_device_status() == api.AC_ERR_INVALID_ARG
    assert api.ac_device_status() == api.AC_OK  # read and cleared


def test_batch_shared_text_two_automata(automata):
    """Two items reading the same bytes with different automata."""
    import torch

    sets, hs = automata
    text = _text_for(0, 40000, 9, sets)
    handles = [hs[0].handle, hs[4].handle]
    items = api.batch_items([0, 0, 17], [40000, 40000, 39000], [0, 40000, 80000], [0, 1, 0])
    out = torch.full((119000,), SENTINEL, dtype=torch.int32, device="cuda")
    api.ac_match_batch(handles, _gpu.to_dev(text), api.items_to_device(items), 3, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got[:40000], oracle.pfac_ids(sets[0], text))
    assert np.array_equal(got[40000:80000], oracle.pfac_ids(sets[4], text))
    assert np.array_equal(got[80000:119000], oracle.pfac_ids(sets[0], text[17:17 + 39000]))


def test_batch_workload_sample(automata):
    """The batched workload's shape (log-uniform lengths, ACGT / Zipf mix,
    eight keyword sets of 8-64 bytes) at a size the oracle checks in full."""
    import torch

    counts = (100, 175, 300, 550, 950, 1650, 2900, 5000)
    sets = workloads.batch_pattern_sets(seed=0, counts=counts)
    texts, kinds = workloads.batch_texts(96, 1024, 256 << 10, seed=0)
    buf, offs, lens, which = workloads.batch_layout(texts, kinds, n_sets=8, seed=0)
    hs = [api.Automaton(p) for p in sets]
    try:
        items = api.batch_items(offs, lens, offs, which)
        out = torch.full((buf.size,), SENTINEL, dtype=torch.int32, device="cuda")
        api.ac_match_batch([a.handle for a in hs], _gpu.to_dev(buf), api.items_to_device(items), len(texts), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, t in enumerate(texts):
            want = oracle.pfac_ids(sets[which[i]], t)
            assert np.array_equal(got[offs[i]:offs[i] + lens[i]], want), i
    finally:
        for a in hs:
            a.close()


def test_autotune_keeps_results(automata):
    """Every knob the autotuner searches changes only the time: at each
    shared-table depth it tries, threads per CTA and stages, the halo and
    chars per thread, and then with the shape it chose, dense ids, count and
    compacted list of a 6 MiB text (long enough for the phased form of 8-bit
    codes) are the oracle's."""
    from tests import _par

    sets, hs = automata
    for j in (0, 1, 2):
        a = hs[j]
        text = _text_for(j, 6 << 20, 40 + j, sets)
        t = _gpu.to_dev(text)
        wpos, wids = _par.oracle_compact(sets[j], text)
        base = a.tuning()
        fb = base["filter_bytes"]
        # the autotuner's smaller depths: one and two window codes fewer (8-bit
        # codes: a hashed filter of 2 and 4 bits fewer)
        shrink = 4 if j == 2 else 1 << a.info()["code_bits"]
        for knobs in ({"filter_bytes": fb // shrink}, {"filter_bytes": fb // (shrink * shrink)},
                      {"block": 256, "stages": 2}, {"block": 384, "stages": 4}, {"halo": 256}, {"per_thread": 4},
                      {"survivor_list": 2}, {"survivor_list": 1},
                      {"block": 640, "stages": 2},
                      {"filter_bytes": fb, "block": base["block"], "stages": base["stages"], "halo": 0, "per_thread": 0,
                       "survivor_list": 0}):
            a.set_tuning(**knobs)
            _par.check_outputs(a.handle, t, text.size, wpos, wids, "automaton %d %s" % (j, knobs))
        assert a.tuning() == base
        block, stages, kernel = a.autotune(t, reps=2)
        assert block in (0, 256, 384, 512, 640) and stages in (0, 2, 3, 4)  # 0: the kernel's choice
        assert kernel in (("tiled",) if j < 2 else ("tiled", "thread_jump_l1", "thread_jump", "walk_slots"))
        tuned = a.tuning()
        assert tuned["filter_bytes"] in (fb, fb // shrink, fb // (shrink * shrink))
        _par.check_outputs(a.handle, t, text.size, wpos, wids, "automaton %d autotuned %s" % (j, tuned))
