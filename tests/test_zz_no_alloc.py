"""ac_match_compact_static -- the compacted matching call that allocates no
device memory -- against ac_match_compact, through the C ABI.

For callers that cannot allocate device memory while they match (for example a
process whose free device memory belongs to another framework's allocator), the
library offers this variant with its scratch in one static device array shared
by every call.  Each call must clear what it uses, so two calls in a row must
both agree with the allocating call.  The file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1412_7789_gb300 import api, workloads

pytestmark = pytest.mark.gpu


def _compact(fn, h, t, n, cap):
    import torch

    pos = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=t.device)
    ids = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=t.device)
    cnt = torch.full((1,), 12345, dtype=torch.int64, device=t.device)
    fn(h, t, n, pos, ids, cap, cnt)
    torch.cuda.synchronize()
    total = int(cnt.item())
    m = min(total, cap)
    return pos[:m].cpu().numpy(), ids[:m].cpu().numpy(), total


@pytest.mark.parametrize("kind", ["acgt", "zipf"])
def test_static_scratch_matches_allocating_call(kind):
    import torch

    from paper_1412_7789_gb300 import build

    build.build()
    if kind == "acgt":
        text, pats = workloads.single_text_acgt(seed=3, n=3 << 20)
    else:
        text, pats = workloads.zipf_byte(1 << 21, seed=3, n_keywords=4000)
    t = torch.from_numpy(text.copy()).cuda()
    n = text.size
    with api.Automaton(pats) as a:
        want_pos, want_ids, want_total = _compact(api.ac_match_compact, a.handle, t, n, n // 8 + 1)
        assert want_total > 0
        # the oracle agrees with the allocating call (sampled head of the text)
        head = oracle.pfac_ids(pats, text[: 1 << 16])
        hp, hi = oracle.compact(head[: (1 << 16) - max(len(p) for p in pats)])
        k = hp.size
        assert np.array_equal(want_pos[:k].astype(np.uint32), hp) and np.array_equal(want_ids[:k].astype(np.uint32), hi)
        for _ in range(2):  # two calls in a row share the static scratch
            pos, ids, total = _compact(api.ac_match_compact_static, a.handle, t, n, n // 8 + 1)
            assert total == want_total
            assert np.array_equal(pos, want_pos) and np.array_equal(ids, want_ids)
        # a smaller capacity: the true total, and the first `cap` entries
        cap = max(1, want_total // 3)
        pos, ids, total = _compact(api.ac_match_compact_static, a.handle, t, n, cap)
        assert total == want_total and np.array_equal(pos, want_pos[:cap]) and np.array_equal(ids, want_ids[:cap])
    assert api.ac_device_status() == api.AC_OK


def test_static_scratch_at_the_size_limit_misaligned():
    """A text of exactly AC_STATIC_MAX_TEXT bytes starting 15 bytes past a
    16-byte boundary (the most work units a text of that length can have)."""
    import torch

    from paper_1412_7789_gb300 import build

    build.build()
    n = api.AC_STATIC_MAX_TEXT
    text, pats = workloads.sweep_acgt(n + 15, seed=5)
    base = torch.from_numpy(text.copy()).cuda()
    t = base[15:15 + n]
    assert t.data_ptr() % 16 == 15
    with api.Automaton(pats) as a:
        want_pos, want_ids, want_total = _compact(api.ac_match_compact, a.handle, t, n, n // 64 + 1)
        pos, ids, total = _compact(api.ac_match_compact_static, a.handle, t, n, n // 64 + 1)
        assert total == want_total > 0
        assert np.array_equal(pos, want_pos) and np.array_equal(ids, want_ids)
    assert api.ac_device_status() == api.AC_OK


def test_static_scratch_call_allocates_nothing():
    """After a first call (which loads the kernels' code), further calls change
    neither the device's free memory nor the library's scratch pool use."""
    import torch

    from paper_1412_7789_gb300 import build

    build.build()
    text, pats = workloads.zipf_byte(1 << 20, seed=6, n_keywords=2000)
    t = torch.from_numpy(text.copy()).cuda()
    n = text.size
    cap = n // 8 + 1
    pos = torch.empty(cap, dtype=torch.int32, device="cuda")
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with api.Automaton(pats) as a:
        api.ac_match_compact_static(a.handle, t, n, pos, ids, cap, cnt)
        torch.cuda.synchronize()
        first = int(cnt.item())
        free0, _ = torch.cuda.mem_get_info()
        used0, _ = api.ac_scratch_pool_usage(reset_high=True)
        for _ in range(3):
            api.ac_match_compact_static(a.handle, t, n, pos, ids, cap, cnt)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        used1, high1 = api.ac_scratch_pool_usage()
        assert int(cnt.item()) == first
        assert free1 == free0, (free0, free1)
        assert used1 == used0 and high1 == used0, (used0, used1, high1)


def test_static_scratch_rejects_long_text():
    import torch

    from paper_1412_7789_gb300 import build

    build.build()
    n = api.AC_STATIC_MAX_TEXT + 1
    t = torch.zeros(n, dtype=torch.uint8, device="cuda")
    pos = torch.zeros(4, dtype=torch.int32, device="cuda")
    ids = torch.zeros(4, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with api.Automaton([b"ACGT"]) as a:
        with pytest.raises(api.AcError) as e:
            api.ac_match_compact_static(a.handle, t, n, pos, ids, 4, cnt)
        assert e.value.status == api.AC_ERR_BUDGET
