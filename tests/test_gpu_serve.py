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
    filter), a device pool of texts of each alphabet, and 160 requests of
    lengths 0 B - 1.5 MiB (log-uniform) at random offsets of their alphabet's
    pool."""
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


def _request_array(d_pools, reqs, bufs):
    arr = np.zeros(len(reqs), dtype=api.SERVER_REQUEST)
    for i, ((a, off, n), (pos, ids, cnt, cap)) in enumerate(zip(reqs, bufs)):
        arr[i] = api.Server.request(a, d_pools[a][off:off + n], n, pos, ids, cap, cnt)[0]
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


@pytest.mark.parametrize("opts", [
    dict(),                                   # defaults: everything in as few waves as possible
    dict(max_wave=7, waves_in_flight=3),      # many small waves overlapping
    dict(hbm_budget=24 << 20, max_wave=64),   # admission held back by the budget
    dict(fifo=True),                          # one request per launch, in order
])
def test_alone_equals_mixed(setup, opts):
    sets, pools, d_pools, autos, reqs, want = setup
    bufs = _buffers(reqs)
    with api.Server([a.handle for a in autos], **opts) as srv:
        tickets = [srv.submit(r) for r in _request_array(d_pools, reqs, bufs)]
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
    with api.Server([a.handle for a in autos], hbm_budget=1 << 20) as srv:
        big = api.Server.request(0, d_pools[0], 4 << 20, pos, pos, 4, cnt)
        with pytest.raises(api.AcError) as e:
            srv.submit(big)
        assert e.value.status == api.AC_ERR_BUDGET
        bad = api.Server.request(7, d_pools[0], 100, pos, pos, 4, cnt)
        with pytest.raises(api.AcError) as e:
            srv.submit(bad)
        assert e.value.status == api.AC_ERR_INVALID_ARG
