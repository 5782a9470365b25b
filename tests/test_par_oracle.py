"""The parallel oracle used by the full-size parity tests against one serial
pass of the oracle (CPU only): stretches with a max_len - 1 halo give exactly
the serial result, and so does a window's list cut from a longer text's."""
import numpy as np

import oracle
from paper_1412_7789_gb300 import workloads
from tests import _par


def _serial(pats, text):
    ids = oracle.pfac_ids(pats, text)
    nz = np.nonzero(ids >= 0)[0]
    return nz.astype(np.int64), ids[nz]


def test_stretches_equal_one_serial_pass():
    text, pats = workloads.sweep_acgt(3 << 20, seed=2)
    # plant keywords across the stretch seams so walks cross them
    text = text.copy()
    g = np.random.default_rng(0)
    stretch = 1 << 16
    for s in range(stretch, text.size, stretch):
        p = pats[int(g.integers(0, len(pats)))]
        o = s - int(g.integers(1, len(p)))
        text[o:o + len(p)] = np.frombuffer(p, dtype=np.uint8)
    wpos, wids = _serial(pats, text)
    pos, ids = _par.oracle_compact(pats, text, procs=4, stretch=stretch)
    assert wpos.size > 40
    assert np.array_equal(pos, wpos) and np.array_equal(ids, wids)


def test_window_lists_from_a_longer_text():
    text, pats = workloads.zipf_byte(1 << 18, seed=4, n_keywords=2000)
    pos, ids = _serial(pats, text)
    g = np.random.default_rng(1)
    for _ in range(20):
        off = int(g.integers(0, text.size))
        n = int(g.integers(0, text.size - off + 1))
        wp, wi = _serial(pats, text[off:off + n])
        gp, gi = _par.window_compact(pos, ids, pats, text, off, n)
        assert np.array_equal(gp, wp) and np.array_equal(gi, wi), (off, n)
    # prefixes (the sweep sizes are prefixes of one text)
    for n in (0, 1, 99, 100, 101, 4096, text.size):
        wp, wi = _serial(pats, text[:n])
        gp, gi = _par.window_compact(pos, ids, pats, text, 0, n)
        assert np.array_equal(gp, wp) and np.array_equal(gi, wi), n
