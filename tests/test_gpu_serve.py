"""The serving loop (ac_server_*) through the C ABI: every request's compacted
list must equal the CPU oracle's for its text, alone (ac_match_compact on its
text) and inside a mix of requests of other sizes and automata batched into
shared waves, under any admission budget, wave size or arrival pattern.  The
oracle's list of a request is cut from the list of its whole pool (tests/_par.py:
exact, with the window's last max_len - 1 starts recomputed)."""
import numpy as np
import pytest

from paper_1412_7789_gb300 import api, workloads
from tests import _gpu, _par

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1412_7789_gb300 import build

    build.build()
    api.lib()
    yield
    assert api.ac_device_status() == api.AC_OK


@pytest.fixture(scope="module")
def setup():
    """Three automata (2-bit filter, 8-bit with class compression, 4-bit
    filter; the 2- and 4-bit ones' root windows often end a keyword, yet
    their units keep the dense fallback and list nothing), a device pool of
    texts of each alphabet, and 160 requests of lengths 0 B - 1.5 MiB
    (log-uniform) at random offsets of their alphabet's pool."""
    import torch

    g = np.random.default_rng(21)
    pool_acgt = workloads.acgt_text(4 << 20, 31)
    pool_zipf = workloads.zipf_text(4 << 20, 32)
    pool_abc = np.frombuffer(b"abcdefghijklmn", dtype=np.uint8)[g.integers(0, 14, size=4 << 20)].copy()
    sets = [
        workloads.keywords_acgt(pool_acgt[:1 << 16], 2000, 6, 40, 0.6, seed=33),
        workloads.keywords_zipf(pool_zipf[:1 << 16], 3000, 2, 40, 0.4, seed=34),
        [bytes(np.frombuffer(b"abcdefghijkl", dtype=np.uint8)[g.integers(0, 12, size=int(g.integers(2, 9)))])
         for _ in range(500)],
    ]
    pools = [pool_acgt, pool_zipf, pool_abc]
    d_pools = [_gpu.to_dev(p) for p in pools]
    autos = [api.Automaton(p) for p in sets]
    assert all(autos[a].info()["match_windows_ppm"] >= 500 for a in (0, 2))
    reqs = []
    for i in range(160):
        a = int(g.integers(0, 3))
        n = 0 if i % 37 == 5 else int(np.exp(g.uniform(0, np.log(1.5 * (1 << 20)))))
        off = int(g.integers(0, pools[a].size - n + 1))
        reqs.append((a, off, n))
    # expected: the oracle's list of every request; the single-text compacted
    # path (the request alone) must give it too
    lists = [_par.oracle_compact(sets[a], pools[a]) for a in range(3)]
    want = []
    for a, off, n in reqs:
        wp, wi = _par.window_compact(*lists[a], sets[a], pools[a], off, n)
        want.append((wp.astype(np.uint32), wi.astype(np.uint32), wp.size))
        if n == 0:
            continue
        pos, ids, total = _gpu.compact(autos[a].handle, d_pools[a][off:off + n], max(1, n))  # room for every match
        assert total == wp.size and np.array_equal(pos, wp) and np.array_equal(ids, wi), (a, off, n)
    yield sets, pools, d_pools, autos, reqs, want
    for x in autos:
        x.close()


def _buffers(reqs, cap_div=1):
    import torch

    out = []
    for a, off, n in reqs:
        cap = max(1, n // cap_div)
        out.append((torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
                    torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
                    torch.full((1,), 12345, dtype=torch.int64, device="cuda"), cap))
    return out


def _request_array(d_pools, reqs, bufs, h_pools=None):
    """Request records; with h_pools (pinned host copies of the pools) every
    third request names its text in host memory (the secondary path)."""
    arr = np.zeros(len(reqs), dtype=api.SERVER_REQUEST)
    for i, ((a, off, n), (pos, ids, cnt, cap)) in enumerate(zip(reqs, bufs)):
        src = h_pools[a] if (h_pools is not None and i % 3 == 1) else d_pools[a]
        arr[i] = api.Server.request(a, src[off:off + n], n, pos, ids, cap, cnt)[0]
    return arr


def _check_results(reqs, bufs, want):
    import torch

    torch.cuda.synchronize()
    for i, ((a, off, n), (pos, ids, cnt, cap), (wp, wi, wt)) in enumerate(zip(reqs, bufs, want)):
        total = int(cnt.item())
        assert total == wt, (i, a, n, total, wt)
        m = min(total, cap)
        assert np.array_equal(pos[:m].cpu().numpy().astype(np.uint32), wp[:m]), (i, a, n)
        assert np.array_equal(ids[:m].cpu().numpy().astype(np.uint32), wi[:m]), (i, a, n)


@pytest.fixture(scope="module")
def h_pools(setup):
    import torch

    sets, pools, d_pools, autos, reqs, want = setup
    return [torch.from_numpy(p.copy()).pin_memory() for p in pools]


def _tables(autos):
    return sum(a.info()["table_bytes"] for a in autos)


@pytest.mark.parametrize("opts", [
    dict(),                                   # defaults: everything in as few waves as possible
    dict(max_wave=7, waves_in_flight=3),      # many small waves overlapping
    dict(hbm_budget=24 << 20, max_wave=64),   # admission held back by the budget (beyond the automata)
    dict(fifo=True),                          # one request per launch, in order
    dict(host=True),                          # every third text from pinned host memory
    dict(host=True, fifo=True),
])
def test_alone_equals_mixed(setup, h_pools, opts):
    sets, pools, d_pools, autos, reqs, want = setup
    bufs = _buffers(reqs)
    opts = dict(opts)
    host = opts.pop("host", False)
    if "hbm_budget" in opts:
        opts["hbm_budget"] += _tables(autos)
    with api.Server([a.handle for a in autos], **opts) as srv:
        tickets = [srv.submit(r) for r in _request_array(d_pools, reqs, bufs, h_pools if host else None)]
        srv.drain()
        done = srv.poll(len(reqs) + 10)
    assert len(done) == len(reqs)
    assert sorted(int(t) for t in done["ticket"]) == sorted(tickets)
    assert np.all(done["status"] == api.AC_OK)
    assert np.all(done["t_done_us"] >= done["t_launch_us"]) and np.all(done["t_launch_us"] >= done["t_submit_us"])
    if opts.get("fifo"):
        assert np.all(done["wave_size"] == 1)
    _check_results(reqs, bufs, want)


def test_replayed_arrivals_and_small_caps(setup):
    """Poisson arrivals played by the library's trace player, outputs with
    room for only some matches (count stays the true total)."""
    sets, pools, d_pools, autos, reqs, want = setup
    bufs = _buffers(reqs, cap_div=4096)
    g = np.random.default_rng(5)
    arrivals = np.cumsum(g.exponential(50.0, size=len(reqs)))  # 20k requests/s
    with api.Server([a.handle for a in autos], max_wave=32) as srv:
        srv.replay(_request_array(d_pools, reqs, bufs), arrivals)
        srv.drain()
        done = srv.poll(len(reqs) + 10)
    assert len(done) == len(reqs) and np.all(done["status"] == api.AC_OK)
    _check_results(reqs, bufs, want)


def test_submit_rejects(setup):
    import torch

    sets, pools, d_pools, autos, reqs, want = setup
    pos = torch.zeros(4, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    # the automata alone exceed the budget: no server
    with pytest.raises(api.AcError) as e:
        api.Server([a.handle for a in autos], hbm_budget=_tables(autos))
    assert e.value.status == api.AC_ERR_BUDGET
    with api.Server([a.handle for a in autos], hbm_budget=_tables(autos) + (1 << 20)) as srv:
        big = api.Server.request(0, d_pools[0], 4 << 20, pos, pos, 4, cnt)
        with pytest.raises(api.AcError) as e:
            srv.submit(big)
        assert e.value.status == api.AC_ERR_BUDGET
        bad = api.Server.request(7, d_pools[0], 100, pos, pos, 4, cnt)
        with pytest.raises(api.AcError) as e:
            srv.submit(bad)
        assert e.value.status == api.AC_ERR_INVALID_ARG


def test_scratch_allocation_failure_is_reported(setup):
    """Host-side fault injection: the waves' scratch comes from a caller
    allocator that fails its first calls; those waves' requests complete with
    AC_ERR_OOM, later waves succeed with exact results, and every block handed
    out is given back."""
    import threading

    import torch

    sets, pools, d_pools, autos, reqs, want = setup
    sub = [r for r in reqs if r[2] > 0][:40]
    sub_want = [want[reqs.index(r)] for r in sub]
    lock = threading.Lock()
    state = {"calls": 0, "live": {}}

    def alloc(nbytes):
        with lock:
            state["calls"] += 1
            if state["calls"] <= 3:
                return 0  # injected failure
            t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            state["live"][t.data_ptr()] = t
            return t.data_ptr()

    def free(ptr):
        with lock:
            state["live"].pop(ptr)

    bufs = _buffers(sub)
    arr = _request_array(d_pools, sub, bufs)
    with api.Server([a.handle for a in autos], max_wave=4, waves_in_flight=1, dev_alloc=alloc,
                    dev_free=free) as srv:
        tickets = [srv.submit(r) for r in arr]
        srv.drain()
        done = srv.poll(len(sub) + 10)
    assert len(done) == len(sub)
    by_ticket = {int(d["ticket"]): int(d["status"]) for d in done}
    failed = [i for i, t in enumerate(tickets) if by_ticket[t] != api.AC_OK]
    assert failed and all(by_ticket[tickets[i]] == api.AC_ERR_OOM for i in failed)
    assert len(failed) < len(sub)
    assert not state["live"]
    ok = [i for i in range(len(sub)) if i not in failed]
    _check_results([sub[i] for i in ok], [bufs[i] for i in ok], [sub_want[i] for i in ok])

    # the same server settings again with a working allocator: all exact
    state["calls"] = 100
    bufs = _buffers(sub)
    with api.Server([a.handle for a in autos], max_wave=4, dev_alloc=alloc, dev_free=free) as srv:
        for r in _request_array(d_pools, sub, bufs):
            srv.submit(r)
        srv.drain()
        done = srv.poll(len(sub) + 10)
    assert np.all(done["status"] == api.AC_OK) and not state["live"]
    _check_results(sub, bufs, sub_want)


def test_cancel_pending_request(setup):
    """A request that waits for budget can be cancelled: it completes with
    AC_ERR_CANCELLED and leaves its outputs alone; the others complete exactly;
    a request already done cannot be cancelled."""
    sets, pools, d_pools, autos, reqs, want = setup
    sub = sorted([r for r in reqs if r[2] > (256 << 10)], key=lambda r: -r[2])[:6]
    sub_want = [want[reqs.index(r)] for r in sub]
    bufs = _buffers(sub)
    arr = _request_array(d_pools, sub, bufs)
    import torch

    # room for about one request at a time (one holds its text, 8 bytes of
    # output room and about 4.4 bytes of scratch per text byte): the later
    # ones wait in the queue
    per = max(int(r["n"]) for r in arr) * 16
    with api.Server([a.handle for a in autos], hbm_budget=_tables(autos) + per, waves_in_flight=1) as srv:
        tickets = [srv.submit(r) for r in arr]
        srv.cancel(tickets[-1])
        with pytest.raises(api.AcError) as e:
            srv.cancel(tickets[-1])
        assert e.value.status == api.AC_ERR_NOT_FOUND
        srv.drain()
        done = srv.poll(len(sub) + 10)
        with pytest.raises(api.AcError) as e:
            srv.cancel(tickets[0])
        assert e.value.status == api.AC_ERR_NOT_FOUND
    st = {int(d["ticket"]): int(d["status"]) for d in done}
    assert st[tickets[-1]] == api.AC_ERR_CANCELLED
    assert all(st[t] == api.AC_OK for t in tickets[:-1])
    _check_results(sub[:-1], bufs[:-1], sub_want[:-1])
    pos, ids, cnt, cap = bufs[-1]
    torch.cuda.synchronize()
    assert int(cnt.item()) == 12345 and int(pos[0].item()) == -7
