"""Benchmark: failureless Aho-Corasick matching throughput on one GB300.

Default workload (the top point of the input-size sweep): a 1 GiB text i.i.d.
uniform over {A,C,G,T}, 10,000 keywords of length 16-64 (half copied from the
text's first 4 KiB, half random ACGT), dense int32 per-position ids.  One step
= one ac_match call over the whole text (text staging, walks, dense output).

Prints one JSON line (rank 0).  Under torchrun each rank matches its own copy
of the workload on its own GPU (replicas; weak scaling) and the slowest rank's
time counts.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                  [--workload sweep|zipf|single] [--sweep]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s text scanned (1 GB300) & % HBM roofline; batch/serve p50/p99 vs plain PFAC"
GIB = 1 << 30
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from an
# ncu capture of the kernel as it stands, keyed by (workload, text bytes,
# kernel): a capture of a 256 MiB launch of the same workload and launch
# form, scaled by 4 to the 1 GiB launch (the traffic grows with the positions;
# the 256 MiB capture read 343.8 MB and wrote 1020.3 MB).  Drop an entry
# whenever its kernel changes.
KNOWN_TRAFFIC: dict = {
    ("sweep", GIB, "pfac_filter_pipe"): 4 * (343.750144e6 + 1020.311e6),
}


def kernel_name(info: dict, out_kind: str, kernel: str, phased: bool = False) -> str:
    if kernel == "simple":
        return "pfac_simple"
    if info["code_bits"] <= 4 or kernel == "tiled":
        name = "pfac_filter_pipe"  # 8-bit codes: its hashed-filter form
        if phased:  # long texts: the survivor and walk steps of the phased form after it
            name += "+pfac_survivors+pfac_walks"
    else:
        name = {"thread_jump": "pfac_jump8", "walk_slots": "pfac_walk8"}.get(kernel, "pfac_jump8g")
    # the compacted list: the matcher in slot mode, then scan and gather; the
    # full output: the matcher in slot mode, occurrence counts, scan, expansion
    return name + {"compact": "+compact", "full": "+full"}.get(out_kind, "")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def make_workload(name: str, n: int | None):
    from paper_1412_7789_gb300 import workloads as W

    if name == "sweep":
        n = n or GIB
        text, pats = W.sweep_acgt(n)
        desc = ("ACGT input-size sweep, top point: %d B i.i.d. uniform ACGT text, 10,000 keywords "
                "length 16-64 (50%% copied from the first 4 KiB, 50%% random ACGT), dense int32 ids" % n)
        out_kind = "dense"
    elif name == "zipf":
        n = n or GIB
        text, pats = W.zipf_byte(n)
        desc = ("byte alphabet: %d B Zipf(1.1) text over 256 byte values, 20,000 keywords length 4-100 "
                "(30%% copied, 70%% Zipf-random), dense 256-wide int32 goto table, compacted (pos,id) output" % n)
        out_kind = "compact"
    elif name == "single":
        text, pats = W.single_text_acgt(0, n or (1 << 20))
        desc = "single text: %d B ACGT, 100 keywords length 8-32, dense int32 ids" % text.size
        out_kind = "dense"
    else:
        raise SystemExit("unknown workload %r" % name)
    return text, pats, desc, out_kind


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self) -> int:
        return len(self.lines)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self, lo: int, hi: int):
        rows = []
        for line in self.lines[lo:hi] or self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, one core, bounded sample
# ----------------------------------------------------------------------------
def cpu_baseline(text: np.ndarray, pats, budget_s: float = 12.0, full: bool = False):
    import oracle

    with oracle.Machine(pats) as m:
        # the full output: the serial pass listing every occurrence
        run = m.full_occurrences if full else m.pfac_ids
        probe = min(text.size, 1 << 18)
        t0 = time.perf_counter()
        run(text[:probe])
        dt = max(time.perf_counter() - t0, 1e-6)
        size = int(min(text.size, max(probe, probe * budget_s / dt)))
        t0 = time.perf_counter()
        run(text[:size])
        dt = time.perf_counter() - t0
        wprobe = min(size, 1 << 22)
        steps, longest = m.walk_steps(text[:wprobe])
    return {"value": size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": ("first %d B of the same text, one serial pass (goto/failure/output, every occurrence "
                       "listed) on one host core" % size) if full else
                      ("first %d B of the same text, one serial pass (goto/failure/output, then per-start "
                       "longest conversion) on one host core" % size),
            "seconds": dt, "walk_steps_per_position": steps / max(wprobe, 1), "longest_walk": longest}


# the same oracle on every host core (context: the paper notes that a parallel
# CPU matcher would move the crossover): each process takes one contiguous
# stretch of a sample plus a halo of max_len - 1 bytes, so no start position's
# walk is cut; processes are spawned (never forked after CUDA is up)
_PAR = {}


def _par_init(pats, shm_name, size):
    from multiprocessing import shared_memory

    import oracle

    _PAR["m"] = oracle.Machine(pats)
    _PAR["shm"] = shared_memory.SharedMemory(name=shm_name)
    _PAR["text"] = np.ndarray((size,), dtype=np.uint8, buffer=_PAR["shm"].buf)


def _par_scan(rng):
    a, b, halo = rng
    ids = _PAR["m"].pfac_ids(_PAR["text"][a:min(b + halo, _PAR["text"].size)])
    return int(np.count_nonzero(ids[:b - a] >= 0))


def cpu_parallel(text: np.ndarray, pats, single_gbs: float, budget_s: float = 6.0, cores: int = 0):
    import multiprocessing as mp
    from multiprocessing import shared_memory

    cores = cores or (os.cpu_count() or 1)
    halo = max(len(p) for p in pats) - 1
    size = int(min(text.size, max(1 << 20, single_gbs * 1e9 * budget_s * cores)))
    shm = shared_memory.SharedMemory(create=True, size=size)
    try:
        np.ndarray((size,), dtype=np.uint8, buffer=shm.buf)[:] = text[:size]
        step = (size + cores - 1) // cores
        ranges = [(a, min(a + step, size), halo) for a in range(0, size, step)]
        with mp.get_context("spawn").Pool(cores, initializer=_par_init, initargs=(pats, shm.name, size)) as pool:
            pool.map(_par_scan, [(0, 1, 0)] * (4 * cores))  # every worker has built its machine
            t0 = time.perf_counter()
            matches = sum(pool.map(_par_scan, ranges, chunksize=1))
            dt = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    return {"value": size / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle, all host cores",
            "sample": "first %d B of the same text in %d contiguous stretches (plus a %d-byte halo each), one "
                      "process per core" % (size, len(ranges), halo), "seconds": dt, "matches": matches}


# ----------------------------------------------------------------------------
# the reference arm: the oracle, timed on the host cores
# ----------------------------------------------------------------------------
def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    text, pats, desc, _ = make_workload(args.workload, args.n)
    import oracle

    with oracle.Machine(pats) as m:
        probe = min(text.size, 1 << 18)
        t0 = time.perf_counter()
        m.pfac_ids(text[:probe])
        dt = max(time.perf_counter() - t0, 1e-6)
        # whole --steps K --warmup W run within about two minutes
        per_step = 100.0 / max(1, args.steps + args.warmup)
        size = int(min(text.size, max(probe, probe * per_step / dt)))
        sample = text[:size]
        for _ in range(args.warmup):
            m.pfac_ids(sample)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            m.pfac_ids(sample)
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = size * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": desc, "sample_bytes": size},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "first %d B of the workload's text per step" % size},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# replicas: every rank matches its own copy of the workload on its own GPU
# ----------------------------------------------------------------------------
def slowest(x: float, dist=None, device=None) -> float:
    """The largest value of x over the ranks (the job ends with its slowest
    replica); x itself with one process."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_gbs(bytes_per_rank: float, steps: int, world: int, t_ms: float) -> float:
    """Whole-job GB/s: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank * steps / (t_ms * 1e-3) / 1e9


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def matching_launches(a, n: int, kernel: str, out_kind: str) -> int:
    """Kernels one matching call launches before any compaction: the filter
    kernel, plus the survivor and walk steps of its phased form (single texts
    with dense, count or compacted output: 8-bit codes from 4 MiB on unless
    the tuning says never; 2- and 4-bit codes when the tuning asks for it or,
    by default for dense ids and counts, when 500 per million or more of their
    root windows end a keyword, beyond the texts whose heavy tiles are shared
    within the CTA)."""
    import torch

    info, tun = a.info(), a.tuning()
    if kernel != "tiled" or out_kind not in ("dense", "count", "compact") or tun["filter_bytes"] == 0:
        return 1
    if n // 992 >= (1 << 22) - 1 or tun["survivor_list"] == 2:
        return 1
    if info["code_bits"] == 8:
        return 3 if n >= (4 << 20) else 1
    if tun["survivor_list"] != 1 and (info["match_windows_ppm"] < 500 or out_kind == "compact"):
        return 1
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return 3 if n // 992 > 16 * sms * (min(tun["block"] or 512, 512) // 32) else 1


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_1412_7789_gb300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

    text_np, pats, desc, out_kind = make_workload(args.workload, args.n)
    if args.out:
        out_kind = args.out
        desc += " [output: %s]" % out_kind
    n = text_np.size
    t_build = time.perf_counter()
    a = api.Automaton(pats, chains=not args.no_chains)  # host build + upload, outside the timed region
    build_s = time.perf_counter() - t_build
    a.set_kernel(args.kernel)
    if args.tune:
        a.set_tuning(**{k: int(v) for k, v in (kv.split("=", 1) for kv in args.tune)})
    info = a.info()
    text = torch.from_numpy(text_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    if out_kind == "dense":
        out = torch.empty(n, dtype=torch.int32, device=dev)

        def step():
            api.ac_match(a.handle, text, n, out, stream)

        out_bytes_per_pos = 4.0
    elif out_kind == "count":
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)

        def step():
            api.ac_count(a.handle, text, n, cnt, stream)

        out_bytes_per_pos = 0.0
    else:
        cap = max(1, n // 256)
        pos = torch.empty(cap, dtype=torch.int32, device=dev)
        ids = torch.empty(cap, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        call = api.ac_match_full if out_kind == "full" else api.ac_match_compact

        def step():
            call(a.handle, text, n, pos, ids, cap, cnt, stream)

        out_bytes_per_pos = None
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    if out_kind in ("compact", "full"):
        matches = int(cnt.item())
        if matches > cap:
            raise SystemExit("%s capacity too small: %d > %d" % (out_kind, matches, cap))
        algo_bytes = n + 8 * matches
    elif out_kind == "count":
        matches = int(cnt.item())
        algo_bytes = n
    else:
        matches = None
        algo_bytes = n * (1 + out_bytes_per_pos)

    sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", local_rank)))
    sampler.start()
    time.sleep(0.3)
    # warm the clocks up under load before the timed region
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    m0 = sampler.mark()
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    m1 = sampler.mark()
    if dist is not None:
        dist.barrier()
    time.sleep(0.25)
    sampler.stop()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    t_ms = slowest(evs[0].elapsed_time(evs[-1]), dist, dev)
    clocks = sampler.summary(m0, m1)

    # end to end through the host-buffer C-ABI call (copies inside the timed region)
    e2e = None
    if out_kind == "dense" and not args.no_e2e:
        ht = torch.from_numpy(text_np).pin_memory()
        ho = torch.empty(n, dtype=torch.int32).pin_memory()
        api.ac_match_host(a.handle, int(ht.data_ptr()), n, int(ho.data_ptr()), stream)
        reps = max(1, min(args.steps, 3))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            api.ac_match_host(a.handle, int(ht.data_ptr()), n, int(ho.data_ptr()), stream)
        e2e_s = slowest((time.perf_counter() - t0) / reps, dist, dev)
        # the legs alone, for the bound a perfect overlap would reach: the text
        # in (pinned host -> device), the kernel, the ids out (device -> pinned host)
        legs = {}
        for name, fn in (("h2d", lambda: text.copy_(ht, non_blocking=True)),
                         ("d2h", lambda: ho.copy_(out, non_blocking=True))):
            fn()
            ms = statistics.median(_event_ms(stream, fn, 3))
            legs[name + "_ms"] = ms
            legs[name + "_gbs"] = (n if name == "h2d" else 4 * n) / (ms * 1e-3) / 1e9
        legs["kernel_ms"] = statistics.mean(per)
        legs["overlap_bound_ms"] = max(legs["h2d_ms"], legs["d2h_ms"], legs["kernel_ms"])
        e2e = {"value": replica_gbs(n, 1, world, 1e3 * e2e_s), "unit": "GB/s", "h2d_bytes_per_step": n,
               "d2h_bytes_per_step": 4 * n, "ms_per_step": 1e3 * e2e_s, "legs": legs,
               "api": "ac_match_host (pinned host text in, ids out, 64 MiB chunks on three streams)"}
        del ht, ho

    peak, peak_kind = load_peaks()
    launch_ms = statistics.mean(per)
    achieved = algo_bytes / (launch_ms * 1e-3) / 1e9
    value = replica_gbs(n, args.steps, world, t_ms)
    kname = kernel_name(info, out_kind, args.kernel, matching_launches(a, n, args.kernel, out_kind) > 1)
    traffic = args.traffic
    if traffic is None:
        # the captured launch form: the default tuning only
        traffic = None if args.tune else KNOWN_TRAFFIC.get((args.workload, n, kname))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind,
            # context: the nominal HBM3e figure (7.9 TB/s) beside the measured copy peak
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
            "algorithmic_bytes_per_launch": algo_bytes, "kernel": kname}

    extra = {"automaton": {k: info[k] for k in ("n_states", "n_classes", "index_width", "code_bits",
                                                  "jump_depth", "stride_depth", "max_len", "table_bytes")},
             "launch_ms_median": statistics.median(per), "launch_ms_min": min(per),
             "automaton_build_s": build_s}
    if matches is not None:
        extra["matches"] = matches
    if args.compare_simple and out_kind == "dense" and args.kernel != "simple":
        a.set_kernel("simple")
        api.ac_match(a.handle, text, n, out, stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            api.ac_match(a.handle, text, n, out, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        extra["simple_kernel_gbs"] = n * 3 / (e0.elapsed_time(e1) * 1e-3) / 1e9
        a.set_kernel(args.kernel)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(text_np, pats, args.cpu_seconds, full=out_kind == "full")
        extra["lookups_per_s"] = cpu["walk_steps_per_position"] * n * args.steps / (t_ms * 1e-3)
        if out_kind != "full" and not args.no_cpu_parallel:
            extra["cpu_all_cores"] = cpu_parallel(text_np, pats, cpu["value"], args.cpu_seconds / 2)

    if rank == 0 and world == 1 and args.workload == "sweep" and out_kind == "dense" and not args.no_extras:
        # the rest of the metric, after the headline's timed region
        del text, out
        torch.cuda.empty_cache()
        extra.update(extra_figures(args))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": desc, "n_bytes": n, "keywords": len(pats),
                       "l2": "inputs larger than L2 (%.1f GB text + output per step)" % (algo_bytes / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU", "tuning": a.tuning()},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * (matching_launches(a, n, args.kernel, out_kind)
                                          + {"compact": 3, "full": 4}.get(out_kind, 0)),
            "extra": extra,
        }
        print(json.dumps(line), flush=True)



def zipf_summary(steps: int, warmup: int) -> dict:
    """The byte-alphabet workload (1 GiB Zipf(1.1) bytes, 20,000 keywords of
    length 4-100) with compacted output, timed like the headline line."""
    import torch

    from paper_1412_7789_gb300 import api
    from paper_1412_7789_gb300 import workloads as W

    text_np, pats = W.zipf_byte(GIB)
    n = text_np.size
    stream = torch.cuda.current_stream()
    with api.Automaton(pats) as a:
        text = torch.from_numpy(text_np).cuda()
        cap = n // 256
        pos = torch.empty(cap, dtype=torch.int32, device="cuda")
        ids = torch.empty(cap, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")

        def step():
            api.ac_match_compact(a.handle, text, n, pos, ids, cap, cnt, stream)

        for _ in range(max(3, warmup)):
            step()
        torch.cuda.synchronize()
        per = _event_ms(stream, step, steps)
        matches = int(cnt.item())
        del text, pos, ids
    ms = statistics.mean(per)
    peak, peak_kind = load_peaks()
    achieved = (n + 8 * matches) / (ms * 1e-3) / 1e9
    return {"workload": "1 GiB Zipf(1.1) bytes, 20,000 keywords length 4-100, compacted (pos,id) output",
            "value": n / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms, "steps": steps, "matches": matches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "frac": achieved / peak, "algorithmic_bytes_per_step": n + 8 * matches},
            "kernels": "pfac_filter_pipe (hashed filter, survivors listed) + pfac_survivors + pfac_walks + scan + gather"}


def extra_figures(args) -> dict:
    """The metric's other parts beside the headline: the byte-alphabet
    workload (compacted), the batch of 4,096 texts and eight automata against
    one launch per text, and the served workload at one arrival rate against
    FIFO one-launch-per-request (p50/p99)."""
    import argparse

    out = {}
    try:
        out["zipf"] = zipf_summary(args.extra_steps, args.warmup)
    except Exception as e:  # reported, not fatal to the headline line
        out["zipf"] = {"error": repr(e)}
    ns = argparse.Namespace(**vars(args))
    ns.steps, ns.warmup, ns.autotune, ns.no_e2e, ns.no_cpu = args.extra_steps, args.warmup, False, True, True
    try:
        b = batch_line(ns)
        keep = ("graph_ms_median", "graph_gbs", "per_text_tiled_ms_median", "per_text_tiled_gbs",
                "speedup_vs_per_text_tiled", "text_done_ms_p50", "text_done_ms_p99", "per_text_done_ms_p50",
                "per_text_done_ms_p99", "parity_texts_checked")
        out["batch"] = {"workload": b["config"]["workload"], "value": b["value"], "unit": "GB/s",
                        "roofline_frac": b["roofline"]["frac"], **{k: b["batch"][k] for k in keep}}
    except Exception as e:
        out["batch"] = {"error": repr(e)}
    ns.serve_rates, ns.serve_requests, ns.serve_pool = [10000.0], [3000], 256 << 20
    try:
        s = serve_line(ns)
        out["serve"] = {"workload": s["config"]["workload"], **s["serve"][0],
                        "parity_requests_checked": s["extra"]["parity_requests_checked"]}
    except Exception as e:
        out["serve"] = {"error": repr(e)}
    return out


# ----------------------------------------------------------------------------
# input-size sweep and CPU/GPU crossover (the paper's section IV experiment)
# ----------------------------------------------------------------------------
def _median(xs):
    return float(statistics.median(xs))


class SweepTimer:
    """Times one automaton on text prefixes: three GPU scopes against the
    serial oracle on one host core."""

    def __init__(self, pats, text_np, max_n):
        import torch

        import oracle
        from paper_1412_7789_gb300 import api

        self.torch, self.api = torch, api
        self.text = text_np
        self.a = api.Automaton(pats)
        self.m = oracle.Machine(pats)
        self.dev_text = torch.from_numpy(text_np[:max_n]).cuda()
        self.dev_out = torch.empty(max(max_n, 1), dtype=torch.int32, device="cuda")
        self.host_text = torch.from_numpy(text_np[:max_n]).pin_memory()
        self.host_out = torch.empty(max(max_n, 1), dtype=torch.int32).pin_memory()
        self.stream = torch.cuda.current_stream()

    def gpu(self, n, reps):
        torch, api = self.torch, self.api
        t, o, h = self.dev_text[:n], self.dev_out[:n], self.a.handle
        for _ in range(3):
            api.ac_match(h, t, n, o, self.stream)
        torch.cuda.synchronize()
        # (i) kernel only: CUDA events around each call on its stream
        ks = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            api.ac_match(h, t, n, o, self.stream)
            e1.record(self.stream)
            e1.synchronize()
            ks.append(e0.elapsed_time(e1) * 1e-3)
        # (ii) host call -> stream synchronised
        cs = []
        for _ in range(reps):
            t0 = time.perf_counter()
            api.ac_match(h, t, n, o, self.stream)
            self.stream.synchronize()
            cs.append(time.perf_counter() - t0)
        # (iii) (ii) plus the text copied in from pinned host memory and the ids copied out
        hs = []
        ht, ho = int(self.host_text.data_ptr()), int(self.host_out.data_ptr())
        api.ac_match_host(h, ht, n, ho, self.stream)
        for _ in range(max(3, reps // 4)):
            t0 = time.perf_counter()
            api.ac_match_host(h, ht, n, ho, self.stream)
            hs.append(time.perf_counter() - t0)
        return _median(ks), _median(cs), _median(hs)

    def cpu(self, n, reps):
        sample = self.text[:n]
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            self.m.pfac_ids(sample)
            ts.append(time.perf_counter() - t0)
        return _median(ts)

    def point(self, n, cpu_reps=None):
        reps = 100 if n <= (1 << 20) else 20
        if cpu_reps is None:
            cpu_reps = 5 if n <= (64 << 20) else (3 if n <= (256 << 20) else 1)
        k, c, e = self.gpu(n, reps)
        cs = self.cpu(n, cpu_reps)
        return {"n": n, "gpu_kernel_s": k, "gpu_call_s": c, "gpu_e2e_s": e, "cpu_s": cs,
                "gpu_kernel_gbs": n / k / 1e9, "gpu_e2e_gbs": n / e / 1e9, "cpu_gbs": n / cs / 1e9}

    def close(self):
        self.a.close()
        self.m.close()


def _crossing(points, key):
    """Smallest n where the GPU scope is no slower than the CPU, log-interpolated
    between the two sizes that bracket it (None if the GPU never wins; the
    smallest size if it always does)."""
    prev = None
    for p in points:
        d = p[key] - p["cpu_s"]
        if d <= 0:
            if prev is None:
                return {"n": p["n"], "bracket": [None, p["n"]], "below_range": True}
            pd = prev[key] - prev["cpu_s"]
            f = pd / (pd - d) if pd != d else 0.0
            import math

            x = math.exp(math.log(prev["n"]) + (math.log(p["n"]) - math.log(prev["n"])) * f)
            return {"n": x, "bracket": [prev["n"], p["n"]], "below_range": False}
        prev = p
    return None


def _refine(timer, lo, hi, key, count=20):
    """The paper's second, finer sweep between the bracketing sizes."""
    import math

    sizes = sorted({int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * j / (count - 1))))
                    for j in range(count)})
    pts = [timer.point(n) for n in sizes]
    return pts, _crossing(pts, key)


def run_sweep(args):
    from paper_1412_7789_gb300 import build, workloads as W

    build.build()
    import torch

    torch.cuda.set_device(0)
    res = {"metric": "CPU/GPU crossover text size and GB/s over the input-size sweep", "unit": "bytes",
           "cpu": "oracle, one host core (serial Aho-Corasick, paper section II)",
           "gpu_scopes": {"gpu_kernel_s": "kernel only (CUDA events)",
                          "gpu_call_s": "host call to stream synchronised (includes the launch)",
                          "gpu_e2e_s": "call with the text copied in from pinned host memory and ids out"}}
    try:
        import multiprocessing

        res["host_cores"] = multiprocessing.cpu_count()
        res["host_cpu"] = subprocess.run(["lscpu"], capture_output=True, text=True).stdout.split("Model name:")[1].split("\n")[0].strip()
    except Exception:
        pass
    max_n = args.sweep_max
    text, pats = W.sweep_acgt(max_n)
    timer = SweepTimer(pats, text, max_n)
    coarse = []
    for n in [4096 * 4 ** j for j in range(10) if 4096 * 4 ** j <= max_n]:
        coarse.append(timer.point(n))
        print("sweep n=%d %s" % (n, json.dumps(coarse[-1])), file=sys.stderr, flush=True)
    res["sweep"] = coarse
    res["crossover"] = {}
    for key in ("gpu_kernel_s", "gpu_call_s", "gpu_e2e_s"):
        c = _crossing(coarse, key)
        if c is not None and c["below_range"]:
            # extend below the smallest coarse size (if the GPU loses there
            # in every new point, keep the coarse answer: at or below 4 KiB)
            c0 = c
            pts = [timer.point(n) for n in (16, 64, 256, 1024, 4096)]
            c = _crossing(pts, key)
            if c is not None and not c["below_range"]:
                _, c2 = _refine(timer, c["bracket"][0], c["bracket"][1], key)
                c = c2 or c
            elif c is None:
                c = c0
        elif c is not None:
            _, c2 = _refine(timer, c["bracket"][0], c["bracket"][1], key)
            c = c2 or c
        res["crossover"][key] = c
    timer.close()
    # paper mode: the alphabet text with 5 and 10 permutation keywords, at the
    # paper's sizes (section IV: 16,375..671,375 and 1,310..53,710 bytes)
    paper = {}
    sizes = sorted(set([16375 + 32750 * j for j in range(21)] + [1310 + 2620 * j for j in range(21)]))
    ptext = W.paper_text(max(sizes))
    for count in (5, 10):
        pt = SweepTimer(W.paper_keywords(count, seed=0), ptext, max(sizes))
        pts = [pt.point(n) for n in sizes]
        paper[str(count)] = {"points": pts,
                             "crossover": {key: _crossing(pts, key) for key in ("gpu_kernel_s", "gpu_call_s", "gpu_e2e_s")}}
        pt.close()
    res["paper_mode"] = paper
    print(json.dumps(res), flush=True)


def _crossovers(timer, sizes, refine: bool):
    """Coarse points and, per GPU scope, the crossover (refined between the
    bracketing sizes with the paper's 20-point second sweep)."""
    pts = [timer.point(n) for n in sizes]
    cross = {}
    for key in ("gpu_kernel_s", "gpu_call_s", "gpu_e2e_s"):
        c = _crossing(pts, key)
        if refine and c is not None and not c["below_range"]:
            _, c2 = _refine(timer, c["bracket"][0], c["bracket"][1], key)
            c = c2 or c
        cross[key] = c
    return pts, cross


def run_sweep_keywords(args):
    """The crossover against the keyword count (the paper's Fig. 8: ten
    keywords against five move it): on the paper-mode workload (the alphabet
    text, permutations of the 26 letters) and on the ACGT sweep workload
    (keywords of 16-64 characters, half copied from the first 4 KiB)."""
    from paper_1412_7789_gb300 import build, workloads as W

    build.build()
    import torch

    torch.cuda.set_device(0)
    counts = [int(c) for c in args.sweep_keyword_counts]
    res = {"metric": "CPU/GPU crossover text size against the keyword count", "unit": "bytes",
           "cpu": "oracle, one host core (serial Aho-Corasick, paper section II)", "counts": counts}
    try:
        import multiprocessing

        res["host_cores"] = multiprocessing.cpu_count()
    except Exception:
        pass
    psizes = sorted(set([16375 + 32750 * j for j in range(21)] + [1310 + 2620 * j for j in range(21)]))
    ptext = W.paper_text(max(psizes))
    asizes = [1024 * 2 ** j for j in range(13)]  # 1 KiB .. 4 MiB
    atext, _ = W.sweep_acgt(max(asizes), seed=0, n_keywords=10)
    out = {"paper_mode": {}, "acgt": {}}
    for count in counts:
        pt = SweepTimer(W.paper_keywords(count, seed=0), ptext, max(psizes))
        pts, cross = _crossovers(pt, psizes, refine=False)
        out["paper_mode"][str(count)] = {"crossover": cross, "states": pt.a.info()["n_states"],
                                         "points": pts}
        pt.close()
        _, pats = W.sweep_acgt(max(asizes), seed=0, n_keywords=count)
        at = SweepTimer(pats, atext, max(asizes))
        pts, cross = _crossovers(at, asizes, refine=True)
        out["acgt"][str(count)] = {"crossover": cross, "states": at.a.info()["n_states"], "points": pts}
        at.close()
        print("keywords %d: paper %s acgt %s" % (
            count, {k: (v or {}).get("n") for k, v in out["paper_mode"][str(count)]["crossover"].items()},
            {k: (v or {}).get("n") for k, v in cross.items()}), file=sys.stderr, flush=True)
    res.update(out)
    print(json.dumps(res), flush=True)


# ----------------------------------------------------------------------------
# batched workload: thousands of texts of uneven length, eight automata
# ----------------------------------------------------------------------------
def _event_ms(stream, fn, reps):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = []
    for _ in range(reps):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))
    return per


def _completion_ms(stream, launches):
    """Run launches[i]() in order on `stream`, each followed by an event: the
    time from the start to each one's completion (ms), and the total."""
    import torch

    start = torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in launches]
    start.record(stream)
    for f, e in zip(launches, evs):
        f()
        e.record(stream)
    evs[-1].synchronize()
    done = [start.elapsed_time(e) for e in evs]
    return done, done[-1]


def run_batch(args):
    print(json.dumps(batch_line(args)), flush=True)


def batch_line(args) -> dict:
    """Config: 4,096 texts, lengths log-uniform 1 KiB-4 MiB, half ACGT and half
    Zipf(1.1) over 256 bytes, each matched against a uniformly chosen keyword
    set of its own alphabet among eight (1k-50k keywords of length 8-64,
    counts geometric), dense int32 ids per text.  One step = the whole batch.
    Timed: the captured CUDA graph of the batch plan (planning kernel + one
    persistent matching launch for all eight automata), the same plan run
    eagerly, the one-shot ac_match_batch, and the comparison the batch is for:
    one ac_match launch per text on one stream (no graph), with the default
    kernel and with the one-thread-per-position kernel; per text, the time
    from the step's start to its ids being complete (p50/p99): in the batch
    every text completes with the graph, one launch per text completes them
    one after another."""
    import torch

    from paper_1412_7789_gb300 import api, build
    from paper_1412_7789_gb300 import workloads as W

    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    counts = (1000, 1750, 3000, 5500, 9500, 16500, 29000, 50000)
    sets = W.batch_pattern_sets(seed=0, counts=counts)
    texts, kinds = W.batch_texts(args.batch_texts, 1 << 10, 4 << 20, seed=0)
    buf, offs, lens, which = W.batch_layout(texts, kinds, n_sets=8, seed=0)
    gen_s = time.perf_counter() - t0
    total = int(buf.size)
    t0 = time.perf_counter()
    autos = [api.Automaton(p) for p in sets]
    build_s = time.perf_counter() - t0
    handles = [a.handle for a in autos]
    d_buf = torch.from_numpy(buf).to(dev)
    items = api.batch_items(offs, lens, offs, which)
    d_items = api.items_to_device(items, dev)
    out = torch.empty(total, dtype=torch.int32, device=dev)

    tuned = []
    if args.autotune:
        for j, a in enumerate(autos):
            idx = np.nonzero(which == j)[0]
            if idx.size == 0:
                tuned.append(None)
                continue
            # the set's own texts, up to 64 MiB of them, as the tuning sample
            take, acc = [], 0
            for i in idx:
                take.append(i)
                acc += int(lens[i])
                if acc >= 64 << 20:
                    break
            sample = torch.from_numpy(np.concatenate([texts[i] for i in take])).to(dev)
            tuned.append(a.autotune(sample, reps=3))
            del sample

    plan = api.BatchPlan(handles, max_items=len(texts))
    nitems = len(texts)
    # the phased form for the sets that list (8-bit codes; 2- and 4-bit codes
    # whose root windows often end a keyword): lists sized for all their text
    list_bytes = 0
    if not args.no_batch_lists:
        infos = [a.info() for a in autos]
        lists = [f["code_bits"] == 8 or f["match_windows_ppm"] >= 500 for f in infos]
        list_bytes = int(sum(int(lens[i]) for i in range(nitems) if lists[which[i]]))
        plan.reserve_lists(list_bytes)

    def graph_step():
        plan.replay(stream)

    def eager_step():
        plan.run(d_buf, d_items, nitems, out, stream)

    def oneshot_step():
        api.ac_match_batch(handles, d_buf, d_items, nitems, out, stream)

    views = [(d_buf[int(o):int(o) + int(n)], out[int(o):int(o) + int(n)], int(n), int(w))
             for o, n, w in zip(offs, lens, which)]

    def per_text_step():
        for tv, ov, n, w in views:
            api.ac_match(handles[w], tv, n, ov, stream)

    plan.capture(d_buf, d_items, nitems, out)
    # parity spot check against the oracle: a few texts of every set
    import oracle

    replays = max(3, args.warmup)
    for _ in range(replays):
        graph_step()
    torch.cuda.synchronize(dev)
    got = out.cpu().numpy()
    checked = 0
    for j in range(8):
        idx = [i for i in np.nonzero(which == j)[0] if lens[i] <= (256 << 10)][:2]
        for i in idx:
            want = oracle.pfac_ids(sets[j], texts[i])
            if not np.array_equal(got[offs[i]:offs[i] + lens[i]], want):
                raise SystemExit("batch parity failure: text %d (set %d)" % (i, j))
            checked += 1

    sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", 0)))
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        graph_step()
    torch.cuda.synchronize(dev)
    m0 = sampler.mark()
    g_ms = _event_ms(stream, graph_step, args.steps)
    m1 = sampler.mark()
    e_ms = _event_ms(stream, eager_step, max(3, args.steps // 2))
    o_ms = _event_ms(stream, oneshot_step, max(3, args.steps // 2))
    per_text_step()
    torch.cuda.synchronize(dev)
    p_ms = _event_ms(stream, per_text_step, max(3, args.steps // 2))
    done_ms, _ = _completion_ms(stream, [(lambda tv=tv, ov=ov, n=n, w=w: api.ac_match(handles[w], tv, n, ov, stream))
                                         for tv, ov, n, w in views])
    for a in autos:
        a.set_kernel("simple")
    per_text_step()
    torch.cuda.synchronize(dev)
    s_ms = _event_ms(stream, per_text_step, 3)
    for a in autos:
        a.set_kernel("tiled")
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(m0, m1)

    # end to end: pinned host texts in, ids out, around one graph replay
    e2e = None
    if not args.no_e2e:
        hb = torch.from_numpy(buf).pin_memory()
        ho = torch.empty(total, dtype=torch.int32).pin_memory()

        def e2e_step():
            d_buf.copy_(hb, non_blocking=True)
            plan.replay(stream)
            ho.copy_(out, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e2e_s = (time.perf_counter() - t0) / reps
        e2e = {"value": total / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": total,
               "d2h_bytes_per_step": 4 * total, "ms_per_step": 1e3 * e2e_s}
        del hb, ho

    cpu = None
    if not args.no_cpu:
        # the oracle on the first texts of the batch, about cpu_seconds of
        # matching (its eight machines built first, outside the timing)
        machines = [oracle.Machine(p) for p in sets]
        try:
            t0 = time.perf_counter()
            done_b = 0
            for i in range(len(texts)):
                machines[which[i]].pfac_ids(texts[i])
                done_b += int(lens[i])
                if time.perf_counter() - t0 > args.cpu_seconds:
                    break
            dt = time.perf_counter() - t0
        finally:
            for m in machines:
                m.close()
        cpu = {"value": done_b / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "first %d texts of the batch (%d B), serially, one machine per keyword set" % (
                   i + 1, done_b)}

    peak, peak_kind = load_peaks()
    gm = statistics.median(g_ms)
    line = {
        "metric": "batched GB/s text scanned (1 GB300)", "value": total / (statistics.mean(g_ms) * 1e-3) / 1e9,
        "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(g_ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": {"workload": "batch: %d texts log-uniform 1 KiB-4 MiB (%d B), 50%% ACGT / 50%% Zipf-256, "
                               "8 keyword sets %s of length 8-64, dense int32 ids" % (nitems, total, list(counts)),
                   "l2": "inputs larger than L2 (%.1f GB per step)" % (5 * total / 1e9),
                   "survivor_lists_for_bytes": list_bytes},
        "roofline": {"bound": "hbm", "achieved": 5 * total / (gm * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": 5 * total / (gm * 1e-3) / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": 5 * total, "kernel": "batch graph (all launches)"},
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        # the planning kernel and the one matching launch (with survivor lists
        # also the survivor and walk steps)
        "gpu_launches": args.steps * (4 if list_bytes else 2),
        "batch": {
            "graph_ms_median": gm, "graph_gbs": total / (gm * 1e-3) / 1e9,
            "text_done_ms_p50": gm, "text_done_ms_p99": gm,
            "per_text_done_ms_p50": float(np.percentile(done_ms, 50)),
            "per_text_done_ms_p99": float(np.percentile(done_ms, 99)),
            "plan_eager_ms_median": statistics.median(e_ms),
            "match_batch_ms_median": statistics.median(o_ms),
            "per_text_tiled_ms_median": statistics.median(p_ms),
            "per_text_tiled_gbs": total / (statistics.median(p_ms) * 1e-3) / 1e9,
            "per_text_simple_ms_median": statistics.median(s_ms),
            "per_text_simple_gbs": total / (statistics.median(s_ms) * 1e-3) / 1e9,
            "speedup_vs_per_text_tiled": statistics.median(p_ms) / gm,
            "speedup_vs_per_text_simple": statistics.median(s_ms) / gm,
            "texts_per_set": [int((which == j).sum()) for j in range(8)],
            "bytes_per_set": [int(lens[which == j].sum()) for j in range(8)],
            "autotuned": tuned, "parity_texts_checked": checked,
            "host_build_s": build_s, "generate_s": gen_s,
        },
    }
    plan.close()
    for a in autos:
        a.close()
    return line


# ----------------------------------------------------------------------------
# served workload: Poisson arrivals, 16 resident automata, continuous batching
# ----------------------------------------------------------------------------
def _serve_run(api, handles, reqs, arrivals, fifo, budget):
    with api.Server(handles, hbm_budget=budget, fifo=fifo) as srv:
        srv.replay(reqs, arrivals)
        srv.drain()
        done = srv.poll(len(reqs) + 16)
    if len(done) != len(reqs) or not np.all(done["status"] == 0):
        raise SystemExit("serve: %d of %d requests completed, statuses %s" % (
            len(done), len(reqs), sorted(set(done["status"].tolist()))))
    lat = done["t_done_us"] - done["t_submit_us"]
    span_s = (done["t_done_us"].max() - done["t_submit_us"].min()) * 1e-6
    return {"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
            "mean_us": float(lat.mean()), "span_s": span_s, "mean_wave": float(done["wave_size"].mean())}


def run_serve(args):
    print(json.dumps(serve_line(args)), flush=True)


def serve_line(args) -> dict:
    """Config: Poisson arrivals at several rates of requests for the compacted
    match of a text of log-uniform length 256 B - 64 MiB (mean 5.4 MB) taken
    from a device-resident pool (1 GiB ACGT, 1 GiB Zipf(1.1) bytes), each
    naming one of 16 resident automata (1k-50k keywords of length 4-100; 8
    ACGT, 8 Zipf), admitted under a 40 GB HBM budget (automata + requests in
    flight).  Per rate: p50/p99 latency (submission to observed completion)
    and aggregate GB/s, for the continuous-batching server and for FIFO
    one-launch-per-request through the same harness."""
    import torch

    from paper_1412_7789_gb300 import api, build
    from paper_1412_7789_gb300 import workloads as W

    build.build()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    sets = W.serve_pattern_sets(seed=0)
    pool_bytes = args.serve_pool
    pools = [W.acgt_text(pool_bytes, 11), W.zipf_text(pool_bytes, 12)]
    d_pools = [torch.from_numpy(p).to(dev) for p in pools]
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    autos = [api.Automaton(p) for p in sets]
    build_s = time.perf_counter() - t0
    handles = [a.handle for a in autos]
    table_bytes = sum(a.info()["table_bytes"] for a in autos)
    budget = int(40e9)  # the server counts the resident automata in it

    n_max = max(args.serve_requests)
    which, offs, lens = W.serve_requests(n_max, pool_bytes, seed=0)
    caps = np.maximum(1, lens // 64)
    cap_off = np.concatenate([[0], np.cumsum(caps)[:-1]])
    out_pos = torch.empty(int(caps.sum()), dtype=torch.int32, device=dev)
    out_ids = torch.empty(int(caps.sum()), dtype=torch.int32, device=dev)
    counts = torch.zeros(n_max, dtype=torch.int64, device=dev)
    reqs = np.zeros(n_max, dtype=api.SERVER_REQUEST)
    reqs["automaton"] = which
    alpha = (which >= 8).astype(np.int64)
    base = np.array([d_pools[0].data_ptr(), d_pools[1].data_ptr()], dtype=np.uint64)
    reqs["d_text"] = base[alpha] + offs.astype(np.uint64)
    reqs["n"] = lens
    reqs["d_pos"] = np.uint64(out_pos.data_ptr()) + 4 * cap_off.astype(np.uint64)
    reqs["d_ids"] = np.uint64(out_ids.data_ptr()) + 4 * cap_off.astype(np.uint64)
    reqs["cap"] = caps
    reqs["d_count"] = np.uint64(counts.data_ptr()) + 8 * np.arange(n_max, dtype=np.uint64)

    # warm-up (module loading, pool growth), then a parity spot check
    _serve_run(api, handles, reqs[:64], W.poisson_arrivals(64, 1000.0, seed=99), False, budget)
    torch.cuda.synchronize(dev)
    import oracle

    got_counts = counts.cpu().numpy()
    checked = 0
    for i in range(64):
        if lens[i] > (256 << 10) or checked >= 8:
            continue
        text = pools[alpha[i]][offs[i]:offs[i] + lens[i]]
        wp, wi = oracle.compact(oracle.pfac_ids(sets[which[i]], text))
        m = min(wp.size, caps[i])
        gp = out_pos[cap_off[i]:cap_off[i] + m].cpu().numpy().astype(np.uint32)
        gi = out_ids[cap_off[i]:cap_off[i] + m].cpu().numpy().astype(np.uint32)
        if got_counts[i] != wp.size or not (np.array_equal(gp, wp[:m]) and np.array_equal(gi, wi[:m])):
            raise SystemExit("serve parity failure: request %d" % i)
        checked += 1

    sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", 0)))
    sampler.start()
    time.sleep(0.3)
    rows = []
    m0 = sampler.mark()
    for rate, n in zip(args.serve_rates, args.serve_requests):
        arr = W.poisson_arrivals(n, rate, seed=int(rate))
        total = int(lens[:n].sum())
        cb = _serve_run(api, handles, reqs[:n], arr, False, budget)
        ff = _serve_run(api, handles, reqs[:n], arr, True, budget)
        rows.append({"rate_per_s": rate, "requests": n, "bytes": total,
                     "offered_gbs": total / (arr[-1] * 1e-6) / 1e9,
                     "gbs": total / cb["span_s"] / 1e9, "p50_us": cb["p50_us"], "p99_us": cb["p99_us"],
                     "mean_wave": cb["mean_wave"],
                     "fifo_gbs": total / ff["span_s"] / 1e9, "fifo_p50_us": ff["p50_us"],
                     "fifo_p99_us": ff["p99_us"]})
    m1 = sampler.mark()
    time.sleep(0.25)
    sampler.stop()
    top = rows[-1]
    line = {
        "metric": "served GB/s and p50/p99 latency (1 GB300)", "value": top["gbs"], "unit": "GB/s", "n_gpus": 1,
        "steps": len(rows), "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "serve: Poisson arrivals at %s req/s, texts log-uniform 256 B-64 MiB from a device "
                               "pool (%d B ACGT + %d B Zipf), 16 resident automata (1k-50k keywords, length "
                               "4-100, 8 ACGT + 8 Zipf), compacted (pos,id) per request, 40 GB budget" % (
                                   list(args.serve_rates), pool_bytes, pool_bytes)},
        "serve": rows, "clocks": sampler.summary(m0, m1),
        "extra": {"automata_table_bytes": table_bytes, "request_budget_bytes": budget - table_bytes,
                  "host_build_s": build_s, "generate_s": gen_s, "parity_requests_checked": checked},
    }
    for a in autos:
        a.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "zipf", "single"])
    ap.add_argument("--n", type=int, default=None, help="text bytes (default: the workload's size)")
    ap.add_argument("--kernel", default="tiled", choices=["tiled", "simple", "walk_slots", "thread_jump", "thread_jump_l1"])
    ap.add_argument("--out", default=None, choices=["dense", "count", "compact", "full"],
                    help="output kind (default: the workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default run: skip the byte-alphabet, batch and serve figures under extra")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of each extra figure")
    ap.add_argument("--no-chains", action="store_true", help="compile without chain records")
    ap.add_argument("--tune", action="append", default=[], metavar="FIELD=VALUE",
                    help="set a field of the automaton's tuning (block, stages, halo, per_thread, filter_bytes)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cpu-parallel", action="store_true", help="skip the all-cores oracle context figure")
    ap.add_argument("--compare-simple", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch from an ncu capture of the current kernel")
    ap.add_argument("--sweep", action="store_true",
                    help="input-size sweep and CPU/GPU crossover instead of the throughput line")
    ap.add_argument("--sweep-max", type=int, default=GIB)
    ap.add_argument("--sweep-keywords", action="store_true",
                    help="the CPU/GPU crossover against the keyword count (paper Fig. 8)")
    ap.add_argument("--sweep-keyword-counts", type=int, nargs="+", default=[5, 10, 100, 1000, 10000])
    ap.add_argument("--batch", action="store_true",
                    help="batched workload (4,096 texts, eight automata) instead of the throughput line")
    ap.add_argument("--batch-texts", type=int, default=4096)
    ap.add_argument("--autotune", action="store_true", help="batch: autotune each automaton first")
    ap.add_argument("--no-batch-lists", action="store_true",
                    help="batch: resolve the 8-bit-code sets' survivors in their warps (no survivor lists)")
    ap.add_argument("--serve", action="store_true",
                    help="served workload (Poisson arrivals, 16 automata) instead of the throughput line")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[1000, 3000, 10000, 30000, 100000])
    ap.add_argument("--serve-requests", type=int, nargs="+", default=[3000, 6000, 20000, 20000, 20000])
    ap.add_argument("--serve-pool", type=int, default=GIB)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.sweep:
        run_sweep(args)
        return
    if args.sweep_keywords:
        run_sweep_keywords(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.serve:
        if len(args.serve_requests) != len(args.serve_rates):
            raise SystemExit("--serve-requests needs one count per rate")
        run_serve(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_1412_7789_gb300 import build

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
