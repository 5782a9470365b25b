"""Bounded device-side waits (failure detection without a GPU fault).

No wait in the kernels spins without a limit: after the limit (ac_set_wait_limit,
default 2 s of %globaltimer) a wait gives up, latches AC_ERR_TIMEOUT in the
device error word and the kernel goes on.  Here the wait of an owner warp for
the warps of its CTA that share its heavy tile is made to wait for a count
nothing reaches (one round more than the tile has), with a short limit: the
wait runs out, ac_device_status() reports the timeout, the results are still
exact (every round was done), the context stays usable, and the next call with
the default limit is exact with a clean status.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1412_7789_gb300 import api, workloads
from tests import _gpu

pytestmark = pytest.mark.gpu

LIMIT_NS = 20_000_000  # 20 ms


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1412_7789_gb300 import build

    build.build()
    api.lib()
    api.ac_device_status()  # start from a clean error word
    yield
    assert api.ac_device_status() == api.AC_OK


def test_shared_tile_wait_runs_out_and_reports():
    import torch

    # the sweep set's first 4 KiB: keywords copied from there start at nearly
    # every position, so its tiles are heavy (hundreds of survivors: several
    # rounds, shared with the idle warps of the one CTA a 4 KiB text gets)
    text, pats = workloads.sweep_acgt(4096)
    want = oracle.pfac_ids(pats, text)
    assert (want >= 0).sum() > 1000
    t = _gpu.to_dev(text)
    with api.Automaton(pats) as a:
        _gpu.check_all_modes(a.handle, text, want, t=t)
        assert api.ac_device_status() == api.AC_OK

        api.ac_set_wait_limit(a.handle, LIMIT_NS, stall_help=True)
        out = torch.full((text.size,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.ac_match(a.handle, t, text.size, out)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert api.ac_device_status() == api.AC_ERR_TIMEOUT
        # the owner gave up after the short limit, not the default 2 s
        assert LIMIT_NS * 1e-9 <= dt < 1.5, dt
        assert np.array_equal(out.cpu().numpy(), want)

        # every output kind takes the same wait
        _gpu.check_all_modes(a.handle, text, want, t=t, modes=("count", "compact"))
        assert api.ac_device_status() == api.AC_ERR_TIMEOUT

        api.ac_set_wait_limit(a.handle, 0, stall_help=False)
        _gpu.check_all_modes(a.handle, text, want, t=t)
        assert api.ac_device_status() == api.AC_OK


def test_default_limit_never_trips_on_long_walks():
    """A short limit alone (no stalled count) changes nothing on a text whose
    walks are the longest the method has."""
    pats = [b"A" * L for L in range(1, 65)]
    text = np.full(50_000, ord("A"), dtype=np.uint8)
    want = oracle.pfac_ids(pats, text)
    with api.Automaton(pats) as a:
        api.ac_set_wait_limit(a.handle, LIMIT_NS, stall_help=False)
        _gpu.check_all_modes(a.handle, text, want)
    assert api.ac_device_status() == api.AC_OK
