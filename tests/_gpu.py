"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the CPU oracle element by element (integers: bit-exact)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1412_7789_gb300 import api


def to_dev(a: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dense(h: int, t, n: int | None = None):
    import torch

    n = t.numel() if n is None else n
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device=t.device)
    api.ac_match(h, t, n, out)
    return out[:n]


def count(h: int, t) -> int:
    import torch

    c = torch.full((1,), 12345, dtype=torch.int64, device=t.device)
    api.ac_count(h, t, t.numel(), c)
    return int(c.item())


def compact(h: int, t, cap: int):
    import torch

    pos = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=t.device)
    ids = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=t.device)
    c = torch.full((1,), 12345, dtype=torch.int64, device=t.device)
    api.ac_match_compact(h, t, t.numel(), pos, ids, cap, c)
    total = int(c.item())
    m = min(total, cap)
    return pos[:m].cpu().numpy().astype(np.uint32), ids[:m].cpu().numpy().astype(np.uint32), total


def check_all_modes(h: int, text: np.ndarray, want: np.ndarray, t=None, modes=("dense", "count", "compact")):
    """Dense ids, count and compacted list of the CUDA path against the
    oracle's per-start ids ``want``."""
    t = to_dev(text) if t is None else t
    if "dense" in modes:
        got = dense(h, t).cpu().numpy()
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0]
            raise AssertionError("dense mismatch at %d positions, first %s: got %s want %s" % (
                bad.size, bad[:8].tolist(), got[bad[:8]].tolist(), want[bad[:8]].tolist()))
    if "count" in modes:
        assert count(h, t) == oracle.count(want)
    if "compact" in modes:
        wpos, wid = oracle.compact(want)
        pos, ids, total = compact(h, t, max(1, wpos.size))
        assert total == wpos.size, (total, wpos.size)
        if not (np.array_equal(pos, wpos) and np.array_equal(ids, wid)):
            bad = np.nonzero((pos != wpos) | (ids != wid))[0]
            raise AssertionError("compact mismatch at %d entries, first %s: got %s / %s want %s / %s" % (
                bad.size, bad[:6].tolist(), pos[bad[:6]].tolist(), ids[bad[:6]].tolist(),
                wpos[bad[:6]].tolist(), wid[bad[:6]].tolist()))
