"""The CPU oracle over long texts, on every host core, for element-by-element
parity at full size.

Exactness: the failureless result at start i depends only on
text[i : i + max_len] (a walk reads at most max_len bytes and stops at the
text end).  So a long text is cut into contiguous stretches; each worker runs
the serial oracle on its stretch plus the max_len - 1 bytes after it (or up to
the text end) and keeps the results of its own stretch.  Together they equal
one serial pass over the whole text.  Workers are spawned processes (never
forked after CUDA is up) that read the text from shared memory and return the
matched starts only: (position, id) in ascending position.

The same argument gives the results of any window text[off : off + n] from
the list of the whole text: starts i with i + max_len <= off + n keep their
result, and the last max_len - 1 starts of the window (whose walks the window
end can cut) are recomputed by the serial oracle on the window's tail.
"""
from __future__ import annotations

import os

import numpy as np

import oracle

_W: dict = {}


def _init(pats, shm_name, size):
    from multiprocessing import shared_memory

    _W["m"] = oracle.Machine(pats)
    _W["shm"] = shared_memory.SharedMemory(name=shm_name)
    _W["text"] = np.ndarray((size,), dtype=np.uint8, buffer=_W["shm"].buf)


def _scan(job):
    a, b, halo = job
    text = _W["text"]
    ids = _W["m"].pfac_ids(text[a:min(b + halo, text.size)])[: b - a]
    nz = np.nonzero(ids >= 0)[0]
    return (nz + a).astype(np.int64), ids[nz].astype(np.int32)


def oracle_compact(pats, text: np.ndarray, procs: int = 0, stretch: int = 0):
    """(pos int64, ids int32): every start of ``text`` with a keyword, ascending,
    with the oracle's id -- one serial pass's result, computed in parallel."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    n = int(text.size)
    if n == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int32)
    procs = procs or (os.cpu_count() or 1)
    halo = max(len(p) for p in pats) - 1
    if not stretch:
        stretch = max(1 << 16, -(-n // (4 * procs)))  # about four stretches per process
    jobs = [(a, min(a + stretch, n), halo) for a in range(0, n, stretch)]
    shm = shared_memory.SharedMemory(create=True, size=n)
    try:
        np.ndarray((n,), dtype=np.uint8, buffer=shm.buf)[:] = text
        with mp.get_context("spawn").Pool(min(procs, len(jobs)), initializer=_init,
                                          initargs=(list(pats), shm.name, n)) as pool:
            parts = pool.map(_scan, jobs, chunksize=1)
    finally:
        shm.close()
        shm.unlink()
    pos = np.concatenate([p for p, _ in parts])
    ids = np.concatenate([i for _, i in parts])
    return pos, ids


def window_compact(pos: np.ndarray, ids: np.ndarray, pats, text: np.ndarray, off: int, n: int):
    """(pos int64 relative to off, ids int32) of the window text[off : off + n],
    from the list (pos, ids) of the whole text and the serial oracle on the
    window's last max_len - 1 starts."""
    maxlen = max(len(p) for p in pats)
    end = off + n
    cut = max(off, end - maxlen + 1)  # starts from here on may reach the window end
    lo, hi = np.searchsorted(pos, [off, cut])
    head_pos = pos[lo:hi] - off
    head_ids = ids[lo:hi]
    tail = oracle.pfac_ids(pats, text[cut:end]) if end > cut else np.zeros(0, np.int32)
    nz = np.nonzero(tail >= 0)[0]
    return (np.concatenate([head_pos, nz + (cut - off)]).astype(np.int64),
            np.concatenate([head_ids, tail[nz]]).astype(np.int32))


def check_dense(out_dev, wpos: np.ndarray, wids: np.ndarray, what: str = ""):
    """Dense ids on the device against the oracle's list, every position:
    out[wpos] == wids and out == -1 everywhere else."""
    import torch

    got_pos = torch.nonzero(out_dev >= 0).flatten()
    gp = got_pos.cpu().numpy()
    if gp.size != wpos.size or not np.array_equal(gp, wpos):
        extra = np.setdiff1d(gp, wpos)[:8].tolist()
        missing = np.setdiff1d(wpos, gp)[:8].tolist()
        raise AssertionError("%s dense: %d matched starts, oracle %d; extra %s missing %s" % (
            what, gp.size, wpos.size, extra, missing))
    gi = out_dev[got_pos].cpu().numpy() if gp.size else np.zeros(0, np.int32)
    if not np.array_equal(gi, wids):
        bad = np.nonzero(gi != wids)[0][:8]
        raise AssertionError("%s dense ids differ at %s: got %s want %s" % (
            what, wpos[bad].tolist(), gi[bad].tolist(), wids[bad].tolist()))
    below = int((out_dev < -1).sum().item())
    if below:
        raise AssertionError("%s dense: %d entries below -1" % (what, below))


def check_compact(pos_dev, ids_dev, total: int, wpos: np.ndarray, wids: np.ndarray, what: str = ""):
    """A compacted list (uint32 pos / ids, ``total`` the reported count)
    against the oracle's."""
    if total != wpos.size:
        raise AssertionError("%s compact: count %d, oracle %d" % (what, total, wpos.size))
    gp = pos_dev[:total].cpu().numpy().astype(np.uint32)
    gi = ids_dev[:total].cpu().numpy().astype(np.uint32)
    if not (np.array_equal(gp, wpos.astype(np.uint32)) and np.array_equal(gi, wids.astype(np.uint32))):
        bad = np.nonzero((gp != wpos.astype(np.uint32)) | (gi != wids.astype(np.uint32)))[0][:6]
        raise AssertionError("%s compact differs at entries %s: got %s / %s want %s / %s" % (
            what, bad.tolist(), gp[bad].tolist(), gi[bad].tolist(), wpos[bad].tolist(), wids[bad].tolist()))


def check_outputs(h: int, t, n: int, wpos: np.ndarray, wids: np.ndarray, what: str = ""):
    """Dense ids, count and compacted list of handle h on device text t[:n]
    through the C ABI, against the oracle's list (wpos, wids)."""
    import torch

    from paper_1412_7789_gb300 import api

    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    api.ac_match(h, t, n, out)
    check_dense(out[:n], wpos, wids, what)
    del out
    cnt = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    api.ac_count(h, t, n, cnt)
    assert int(cnt.item()) == wpos.size, (what, int(cnt.item()), wpos.size)
    cap = max(1, wpos.size)
    pos = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    ids = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    api.ac_match_compact(h, t, n, pos, ids, cap, cnt)
    check_compact(pos, ids, int(cnt.item()), wpos, wids, what)
