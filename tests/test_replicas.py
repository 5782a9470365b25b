"""The multi-GPU path of bench.py on CPU: N independent replicas (no data
exchange), timed by the slowest rank, reported as whole-job throughput.  Run
as world-size-2 gloo process groups on 127.0.0.1."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]  # the second replica is slower
    t = bench.slowest(local_ms, dist, "cpu")
    q.put((rank, t, bench.replica_gbs(1 << 30, 10, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [150.0, 150.0]
    want = 2 * (1 << 30) * 10 / 0.150 / 1e9
    assert all(abs(g[2] - want) < 1e-9 * want for g in got)


def test_single_process_is_its_own_slowest():
    import bench

    assert bench.slowest(3.5) == 3.5
    assert bench.replica_gbs(1e9, 2, 1, 1000.0) == pytest.approx(2.0)


def test_cpu_all_cores_context_matches_single_pass():
    """The all-cores oracle figure of bench.py: contiguous stretches with
    max-length halos in spawned processes give the same match count as one
    serial pass over the same sample."""
    import numpy as np

    import bench
    import oracle
    from paper_1412_7789_gb300 import workloads

    text, pats = workloads.sweep_acgt(1 << 21, seed=3, n_keywords=300)
    # plant keywords across the stretch boundaries of a two-process split
    g = np.random.default_rng(4)
    text = text.copy()
    for o in list(g.integers(0, text.size - 64, size=200)) + [text.size // 2 - 10, text.size // 2 - 1]:
        p = pats[int(g.integers(0, len(pats)))]
        text[o:o + len(p)] = np.frombuffer(p, dtype=np.uint8)
    r = bench.cpu_parallel(text, pats, single_gbs=4e-3, budget_s=1.0, cores=2)
    size = int(r["sample"].split()[1])
    assert size == text.size
    want = int(np.count_nonzero(oracle.pfac_ids(pats, text[:size]) >= 0))
    assert r["matches"] == want and r["cores"] == 2
