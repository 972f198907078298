#!/usr/bin/env python3
"""Benchmark of the GPU string sample sort (sorted order + LCP array).

Default workload (one GPU): the plain sort of 20 M synthetic URL-like strings
(~59 B mean, Zipf hosts, 1.19 GB of characters), inputs resident in HBM.  One
step = one complete sort through the C-ABI (ss_sort_ex), producing the
permutation and the LCP array.  Prints one JSON line.  On one GPU that line
also carries the metric's batched and served parts: "batched" (configuration
4: 4096 sets as one batch replayed from a CUDA graph against 4096 plain calls)
and "served" (configuration 5: 2000 Poisson requests through the serving loop
against a one-at-a-time plain loop, p50/p99 latency and throughput), each
with its parity check (--no-batched leaves them out).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--config c1|c2|c3|c4|c5|m2|s3|d3]

--config d3 sorts configuration 3 with alphabet compression (3-bit character
codes, 21 characters per key).
--config s3 times suffix array construction (prefix doubling on top of the
sort) of the 4 M-character DNA-like text of configuration 3, uncapped.
--config m2 times the K-way LCP merge instead: 16 sorted runs (a seeded
partition of the 20 M URL-like strings, each run sorted on the GPU before the
timed region) merged into one sorted order with its LCP array per step.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload.  Under torchrun (N > 1) every rank sorts its own copy of
the workload (independent replicas, weak scaling): the sort has no exchange
step, so ranks share nothing but the timing barrier.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

METRIC = "strings/s & D-bytes/s vs HBM roofline; batched/served vs plain p99 + throughput"
KIND = {"c1": "random", "c2": "url", "c3": "dna", "d3": "dna"}
CPU_SAMPLE = 2_000_000


# ---- distributed plumbing ------------------------------------------------------------------

def dist_init(backend: str = "nccl"):
    """One process per GPU (torchrun sets RANK / LOCAL_RANK / WORLD_SIZE /
    MASTER_*); the process group only carries the timing barrier and the
    max-over-ranks reduction (gloo on CPU in the tests)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if backend == "nccl":
        torch.cuda.set_device(local if ws > 1 else 0)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(local_ms: float, ws: int, units_per_rank: int, steps: int):
    """(slowest rank's ms, whole-job units/s): every rank processes the same
    number of units, the job takes as long as its slowest rank."""
    ms = max_over_ranks(local_ms, ws)
    return ms, ws * units_per_rank * steps / (ms / 1e3)


# ---- clocks during the timed region ---------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        """Keep only samples received inside the timed region [t0, t1]."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "window", (float("-inf"), float("inf")))
        for ts, ln in self.lines:
            if not (t0 <= ts <= t1 + 0.25):  # a sample arrives up to one period after it is taken
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---- workloads ----------------------------------------------------------------------------------

def workload(name: str, n: int | None = None):
    if name == "c1":
        return gen.config1(), "plain sort, 100k random strings (length 8-32, a-z)"
    if name == "c2" and n:  # reduced size, for profiler captures
        return gen.config2(n), f"plain sort, {n} URL-like strings (reduced configuration 2, for profiling)"
    if name == "c2":
        return gen.config2(), "plain sort, 20M URL-like strings (~59 B mean, Zipf(1.1) over 2000 hosts)"
    if name == "c3":
        return gen.config3(), "plain sort, all 4M suffixes of a DNA-like text, capped at 500 B"
    if name == "d3":
        return gen.config3(), ("plain sort, all 4M suffixes of a DNA-like text, capped at 500 B, with alphabet "
                               "compression (3-bit character codes, 21 characters per key)")
    raise ValueError(name)


def d_and_l(lcp: np.ndarray):
    """D and L from an LCP array: d_i = max(h_i, h_{i+1}) + 1 with h_0 = h_n = 0."""
    h = lcp.astype(np.int64)
    if h.size == 0:
        return 0, 0
    h[0] = 0
    nxt = np.append(h[1:], 0)
    return int(np.maximum(h, nxt).sum() + h.size), int(h[1:].sum())


# translation unit of each kernel whose DRAM traffic is recorded in
# profiles/traffic.json
KERNEL_UNITS = {"big_scatter": "ss_big.cu", "merge_round": "ss_merge.cu"}


def kernel_sources(kernel: str | None):
    """The files a kernel is compiled from: its translation unit and the
    headers it includes (transitively); all library sources when unknown."""
    d = os.path.join(ROOT, "paper_1808_00963_gb300", "csrc")
    unit = KERNEL_UNITS.get(kernel or "")
    if unit is None:
        return sorted(os.path.join(d, f) for f in os.listdir(d))
    seen, todo = [], [os.path.join(d, unit)]
    while todo:
        f = os.path.normpath(todo.pop())
        if f in seen or not os.path.exists(f):
            continue
        seen.append(f)
        with open(f) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith('#include "'):
                    todo.append(os.path.join(os.path.dirname(f), line.split('"')[1]))
    return sorted(seen)


def source_hash(kernel: str | None = None):
    """Hash of the sources a kernel is compiled from (a recorded traffic
    figure is used only while they are unchanged)."""
    hsh = hashlib.sha256()
    for f in kernel_sources(kernel):
        with open(f, "rb") as fh:
            hsh.update(os.path.basename(f).encode() + fh.read())
    return hsh.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s; MEASURED_PEAKS.json absent)"


def ncu_traffic(kernel: str, config: str):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if it
    was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(config, {}).get(kernel)
    if not e or e.get("source_hash") != source_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


MERGE_RUNS = 16
MERGE_SAMPLE = 2_000_000


def merge_assign(n: int, K: int = MERGE_RUNS):
    """The seeded partition of the strings into K runs."""
    return np.random.default_rng(5).integers(0, K, n)


def cpu_merge_runs(s, sample: int, K: int = MERGE_RUNS):
    """Sorted runs (with LCP arrays) of the first `sample` strings, made by the
    oracle: the inputs of the oracle's merge."""
    import oracle
    a = merge_assign(s.n, K)[:sample]
    offs = np.ascontiguousarray(s.offsets[:sample])
    runs = []
    for k in range(K):
        sub = np.nonzero(a == k)[0].astype(np.uint32)
        p, l = oracle.sort(s.chars, offs[sub], s.max_len)
        runs.append((sub[p], l))
    return offs, runs


def time_oracle_merge(s, sample: int, reps: int):
    import oracle
    offs, runs = cpu_merge_runs(s, sample)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.lcp_merge(s.chars, offs, runs, s.max_len)
        times.append(time.perf_counter() - t0)
    return times


# ---- reference arm: the CPU oracle ----------------------------------------------------------

def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    if args.config == "m2":
        return run_reference_merge(args)
    if args.config == "s3":
        return run_reference_sa(args)
    s, desc = workload(args.config)
    # each step sorts a bounded sample of the workload (the first strings,
    # generated i.i.d.) sized so that all warm-up and timed steps take about
    # 45 s of one host core at ~1e6 strings/s
    per_step = int(45e6 / max(1, args.steps + args.warmup))
    sample = max(min(20_000, s.n), min(per_step, CPU_SAMPLE, s.n))
    offs = np.ascontiguousarray(s.offsets[:sample])
    oracle.load()
    for _ in range(args.warmup):
        oracle.sort(s.chars, offs, s.max_len)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort(s.chars, offs, s.max_len)
    dt = time.perf_counter() - t0
    v = sample * args.steps / dt
    cores = 1
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "strings/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": desc, "n": s.n, "sample_strings": sample, "parallelism": "cpu, 1 thread"},
        "cpu_baseline": {"value": v, "unit": "strings/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} of the {s.n} strings (generated i.i.d.), same buffer"},
        "e2e": {"value": v, "unit": "strings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_merge(args):
    """The oracle's K-way LCP merge (Algorithm 4.5, one character per
    comparison) on the runs of a bounded sample of the merge workload."""
    s = gen.config2()
    per_step = int(30e6 / max(1, args.steps + args.warmup))
    sample = max(20_000, min(per_step, MERGE_SAMPLE, s.n))
    times = time_oracle_merge(s, sample, args.warmup + args.steps)[args.warmup:]
    dt = sum(times)
    v = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": "merged strings/s (K-way LCP merge)", "value": v, "unit": "strings/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"K-way LCP merge of {MERGE_RUNS} sorted runs of URL-like strings",
                   "sample_strings": sample, "parallelism": "cpu, 1 thread"},
        "cpu_baseline": {"value": v, "unit": "strings/s", "cores": 1, "kind": "oracle",
                         "sample": f"the {MERGE_RUNS} runs restricted to the first {sample} of the {s.n} strings"},
        "e2e": {"value": v, "unit": "strings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(s, config):
    import oracle
    sample = min(CPU_SAMPLE if config == "c2" else s.n, s.n)
    offs = np.ascontiguousarray(s.offsets[:sample])
    oracle.load()
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        oracle.sort(s.chars, offs, s.max_len)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return {"value": sample / t, "unit": "strings/s", "cores": 1, "kind": "oracle",
            "sample": (f"first {sample} of the {s.n} strings (generated i.i.d.), median of 3 runs, "
                       f"single thread of {os.cpu_count()} host cores")}


def profiled_pass(step, steps: int, stream):
    """Per-kernel device time for the roofline: CUDA events around every
    launch, on the launching stream, over a second pass of the same steps
    right after the timed region.  The events add host time between launches
    (not to the kernels), so this pass's step time is reported on its own and
    never as the value."""
    import torch

    import paper_1808_00963_gb300 as ss
    torch.cuda.synchronize()
    ss.reset_kernel_stats()
    ss.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    stats = ss.kernel_stats()
    ss.set_profiling(False)
    return stats, e0.elapsed_time(e1) / steps


# ---- our arm --------------------------------------------------------------------------------------

def run_ours(args, ws, rank, local):
    import torch

    import paper_1808_00963_gb300 as ss
    ss.load()
    s, desc = workload(args.config, args.n)
    dev = torch.device("cuda", torch.cuda.current_device())
    chars = torch.from_numpy(s.chars).to(dev)
    offsets = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    n = s.n
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    from paper_1808_00963_gb300 import tune
    tuned = {k: v for k, v in tune.options_for(KIND[args.config]).items() if v}
    wsb = ss.workspace_size(n, s.max_len, **tuned)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    opts = dict(workspace=work.data_ptr(), workspace_bytes=wsb, **tuned)
    stream = torch.cuda.current_stream()

    dna = args.config == "d3"

    def step():  # enqueues one sort (ss_sort_ex is asynchronous); the status is read after the timed steps
        ss.sort(chars, offsets, max_len=s.max_len, out=(perm, lcp), dna=dna, sync=dna, **opts)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    D, L = d_and_l(lcp.cpu().numpy().view(np.uint32))

    sampler = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = ss.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(t_start, time.perf_counter())
    ss.stream_status(stream)  # raises if a timed sort latched a device-side error
    launches = ss.launch_count() - launches0
    barrier(ws)
    clocks = sampler.stop()
    ms, value = weak_scaling_value(e0.elapsed_time(e1), ws, n, args.steps)
    stats, prof_ms = profiled_pass(step, args.steps, stream)
    ss.stream_status(stream)
    d_rate = ws * D * args.steps / (ms / 1e3)

    # roofline of the dominant kernel (largest share of device time)
    peak, peak_kind = measured_peaks()
    dom = max(stats.items(), key=lambda kv: kv[1][1]) if stats else None
    roof = None
    if dom:
        name, (nl, kms, kbytes) = dom
        achieved = (kbytes / nl) / (kms / nl / 1e3) / 1e9 if kms > 0 else 0.0
        path_bytes = D + 16 * n
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": ncu_traffic(name, args.config),
                "alg_bytes_per_launch": kbytes / nl, "launches": nl, "ms_per_launch": kms / nl,
                "path_alg_bytes_per_step": path_bytes,
                "path_frac": (path_bytes / (ms / args.steps / 1e3)) / 1e9 / peak,
                "kernel_share": {k: round(v[1] / sum(x[1] for x in stats.values()), 4) for k, v in stats.items()},
                "timing": "CUDA events around each launch in a profiled pass of the same steps after the timed region",
                "profiled_ms_per_step": prof_ms}

    # end to end through the host-buffer entry point (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hchars = torch.from_numpy(s.chars).pin_memory()
        hoffs = torch.from_numpy(s.offsets.view(np.int64)).pin_memory()
        hperm = torch.empty(n, dtype=torch.int32).pin_memory()
        hlcp = torch.empty(n, dtype=torch.int32).pin_memory()

        def e2e_step():
            if not dna:  # through the host-buffer entry point
                ss.sort_host(hchars, hoffs, s.max_len, perm=hperm, lcp=hlcp, **tuned)
                return
            dc = hchars.to(dev, non_blocking=True)
            do = hoffs.to(dev, non_blocking=True)
            ss.sort(dc, do, max_len=s.max_len, out=(perm, lcp), dna=True, **opts)
            hperm.copy_(perm, non_blocking=True)
            hlcp.copy_(lcp, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        et = max_over_ranks(time.perf_counter() - t0, ws)
        e2e = {"value": ws * n * args.steps / et, "unit": "strings/s",
               "h2d_bytes_per_step": int(s.N + 8 * n), "d2h_bytes_per_step": int(8 * n),
               "ms_per_step": et / args.steps * 1e3}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, args.config)

    # the metric's other two parts, on the same GPU: the batched form
    # (configuration 4) and the served form (configuration 5), each against
    # per-request plain calls
    batched = served = None
    if args.config == "c2" and ws == 1 and not args.no_batched:
        del work, perm, lcp
        torch.cuda.empty_cache()
        batched = batch_workload(args.sets, 3, min(args.steps, 20))
        torch.cuda.empty_cache()
        served = served_workload(args.requests)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "strings/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": desc, "n": n, "N": s.N, "D": D, "L": L, "max_len": s.max_len,
                       "l2": f"inputs larger than L2 (characters {s.N / 1e9:.2f} GB, offsets {8 * n / 1e6:.0f} MB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "per_step": "one sort: permutation + LCP array",
                       "options": tuned or "compiled defaults", "options_source": "autotuner table (tuned.json)"},
            "d_bytes_per_s": d_rate,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4), "alg_bytes": v[2]} for k, v in stats.items()},
        }
        if batched is not None:
            line["batched"] = batched
            line["served"] = served
        print(json.dumps(line), flush=True)


# ---- K-way LCP merge of sorted runs ------------------------------------------------------------

# Algorithmic bytes of the merge's rounds (the dominant kernel): per string and
# round, its 32-byte record read and written (index, offset, LCP, 16
# characters), the last round writing the index and LCP (8) instead.  The
# record gather before the rounds: index and LCP entry read (8), offset (8),
# 16 characters (16), record written (32).
MERGE_RECORD_BYTES = 32


def merge_round_bytes(n: int, runs: int) -> float:
    """Average algorithmic bytes per launch of the merge rounds."""
    rounds = max(1, (runs - 1).bit_length())
    return n * (2 * MERGE_RECORD_BYTES * (rounds - 1) + MERGE_RECORD_BYTES + 8) / rounds


def run_merge(args, ws, rank, local):
    import torch

    import paper_1808_00963_gb300 as ss
    ss.load()
    s = gen.config2(args.n) if args.n else gen.config2()
    K = MERGE_RUNS
    desc = (f"K-way LCP merge of {K} sorted runs: a seeded partition of {s.n} URL-like strings "
            "(~59 B mean, Zipf(1.1) over 2000 hosts), each run sorted on the GPU before timing")
    dev = torch.device("cuda", torch.cuda.current_device())
    chars = torch.from_numpy(s.chars).to(dev)
    offsets = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    assign = torch.from_numpy(merge_assign(s.n, K)).to(dev)
    runs = []
    for k in range(K):
        sub = torch.nonzero(assign == k).flatten()
        p, l = ss.sort(chars, offsets[sub].contiguous(), max_len=s.max_len)
        runs.append((sub[p.long()].int().contiguous(), l))
    del assign
    n = s.n
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    wsb = ss.merge_workspace_size(runs)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ss.merge(chars, offsets, runs, max_len=s.max_len, out=(perm, lcp), workspace=work.data_ptr(),
                 workspace_bytes=wsb)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = ss.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(t_start, time.perf_counter())
    launches = ss.launch_count() - launches0
    barrier(ws)
    clocks = sampler.stop()
    ms, value = weak_scaling_value(e0.elapsed_time(e1), ws, n, args.steps)
    stats, prof_ms = profiled_pass(step, args.steps, stream)

    peak, peak_kind = measured_peaks()
    roof = None
    if "merge_round" in stats:
        nl, kms, _ = stats["merge_round"]
        kbytes = merge_round_bytes(n, K)
        achieved = kbytes / (kms / nl / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "merge_round", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": ncu_traffic("merge_round", "m2"), "alg_bytes_per_launch": kbytes,
                "launches": nl, "ms_per_launch": kms / nl,
                "kernel_share": {k: round(v[1] / sum(x[1] for x in stats.values()), 4) for k, v in stats.items()},
                "timing": "CUDA events around each launch in a profiled pass of the same steps after the timed region",
                "profiled_ms_per_step": prof_ms}

    # end to end: runs, characters and offsets copied from pinned host memory,
    # the merged order and LCP array copied back, every step
    e2e = None
    if not args.no_e2e:
        h_chars = torch.from_numpy(s.chars).pin_memory()
        h_offs = torch.from_numpy(s.offsets.view(np.int64)).pin_memory()
        h_runs = [(p.cpu().pin_memory(), l.cpu().pin_memory()) for p, l in runs]
        h_perm = torch.empty(n, dtype=torch.int32).pin_memory()
        h_lcp = torch.empty(n, dtype=torch.int32).pin_memory()

        def e2e_step():
            d_chars = h_chars.to(dev, non_blocking=True)
            d_offs = h_offs.to(dev, non_blocking=True)
            d_runs = [(p.to(dev, non_blocking=True), l.to(dev, non_blocking=True)) for p, l in h_runs]
            ss.merge(d_chars, d_offs, d_runs, max_len=s.max_len, out=(perm, lcp), workspace=work.data_ptr(),
                     workspace_bytes=wsb)
            h_perm.copy_(perm, non_blocking=True)
            h_lcp.copy_(lcp, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        e2e_step()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        et = max_over_ranks(time.perf_counter() - t0, ws)
        e2e = {"value": ws * n * args.steps / et, "unit": "strings/s",
               "h2d_bytes_per_step": int(s.N + 8 * n + 8 * n), "d2h_bytes_per_step": int(8 * n),
               "ms_per_step": et / args.steps * 1e3}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample = min(MERGE_SAMPLE, n)
        t = statistics.median(time_oracle_merge(s, sample, 3))
        cpu = {"value": sample / t, "unit": "strings/s", "cores": 1, "kind": "oracle",
               "sample": (f"Algorithm 4.5 as written in the oracle (one character per comparison) on the "
                          f"{K} runs restricted to the first {sample} strings, median of 3, single thread")}
    if rank == 0:
        line = {
            "metric": "merged strings/s (K-way LCP merge)", "value": value, "unit": "strings/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": desc, "n": n, "runs": K, "N": s.N,
                       "l2": f"inputs larger than L2 (characters {s.N / 1e9:.2f} GB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "per_step": "one merge: permutation + LCP array",
                       "sample_step": "default"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in stats.items()},
        }
        print(json.dumps(line), flush=True)


# ---- suffix array by prefix doubling ------------------------------------------------------------

SA_SAMPLE = 2_000_000


def sa_text():
    s = gen.config3()
    return bytes(s.chars[:s.n]), s


def time_oracle_sa(text: bytes, reps: int):
    import oracle
    oracle.load()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.suffix_array(text)
        times.append(time.perf_counter() - t0)
    return times


def run_reference_sa(args):
    text, _ = sa_text()
    per_step = int(15e6 / max(1, args.steps + args.warmup))
    sample = max(100_000, min(per_step, SA_SAMPLE, len(text)))
    times = time_oracle_sa(text[:sample], args.warmup + args.steps)[args.warmup:]
    dt = sum(times)
    v = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": "suffixes/s (suffix array + LCP array)", "value": v, "unit": "suffixes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "suffix array of a DNA-like text", "sample_chars": sample,
                   "parallelism": "cpu, 1 thread"},
        "cpu_baseline": {"value": v, "unit": "suffixes/s", "cores": 1, "kind": "oracle",
                         "sample": f"suffix array of the first {sample} characters of the text"},
        "e2e": {"value": v, "unit": "suffixes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_sa(args, ws, rank, local):
    import torch

    import paper_1808_00963_gb300 as ss
    ss.load()
    text, s = sa_text()
    n = len(text)
    desc = (f"suffix array + LCP array of all {n} suffixes of a DNA-like text (order-3 Markov, 5 % duplicated "
            "1000-character blocks), uncapped, by prefix doubling on the string sort")
    dev = torch.device("cuda", torch.cuda.current_device())
    d_text = torch.from_numpy(np.frombuffer(text + b"\0", np.uint8).copy()).to(dev)
    sa = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ss.suffix_array(d_text, n, out=(sa, lcp))

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = ss.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(t_start, time.perf_counter())
    launches = ss.launch_count() - launches0
    barrier(ws)
    clocks = sampler.stop()
    ms, value = weak_scaling_value(e0.elapsed_time(e1), ws, n, args.steps)
    stats, prof_ms = profiled_pass(step, args.steps, stream)
    peak, peak_kind = measured_peaks()
    roof = None
    counted = {k: v for k, v in stats.items() if v[2] > 0}
    if counted:
        name, (nl, kms, kbytes) = max(counted.items(), key=lambda kv: kv[1][1])
        achieved = (kbytes / nl) / (kms / nl / 1e3) / 1e9 if kms > 0 else 0.0
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": None, "alg_bytes_per_launch": kbytes / nl, "launches": nl, "ms_per_launch": kms / nl,
                "kernel_share": {k: round(v[1] / sum(x[1] for x in stats.values()), 4) for k, v in stats.items()},
                "timing": "CUDA events around each launch in a profiled pass of the same steps after the timed region",
                "profiled_ms_per_step": prof_ms}
    e2e = None
    if not args.no_e2e:
        h_text = torch.from_numpy(np.frombuffer(text + b"\0", np.uint8).copy()).pin_memory()
        h_sa = torch.empty(n, dtype=torch.int32).pin_memory()
        h_lcp = torch.empty(n, dtype=torch.int32).pin_memory()

        def e2e_step():
            t = h_text.to(dev, non_blocking=True)
            ss.suffix_array(t, n, out=(sa, lcp))
            h_sa.copy_(sa, non_blocking=True)
            h_lcp.copy_(lcp, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        e2e_step()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        et = max_over_ranks(time.perf_counter() - t0, ws)
        e2e = {"value": ws * n * args.steps / et, "unit": "suffixes/s", "h2d_bytes_per_step": n + 1,
               "d2h_bytes_per_step": 8 * n, "ms_per_step": et / args.steps * 1e3}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample = min(SA_SAMPLE, n)
        t = statistics.median(time_oracle_sa(text[:sample], 3))
        cpu = {"value": sample / t, "unit": "suffixes/s", "cores": 1, "kind": "oracle",
               "sample": f"the oracle's sort of all suffixes of the first {sample} characters, median of 3, "
                         "single thread"}
    if rank == 0:
        line = {
            "metric": "suffixes/s (suffix array + LCP array)", "value": value, "unit": "suffixes/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": desc, "n": n, "l2": "text 4 MB; suffix array, names and LCPs 16 MB each",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "per_step": "one suffix array + LCP array", "initial_depth": "default (256)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in stats.items()},
        }
        print(json.dumps(line), flush=True)


# ---- batched workload (configuration 4) ---------------------------------------------------------

def batch_workload(num: int, warmup: int, steps: int):
    """Configuration 4: num independent string sets (log-uniform 100..200k
    strings, random / URL / DNA generators) sorted as one batch (one launch
    sequence, captured into a CUDA graph) against num plain calls on one
    stream.  The plain calls write their own buffers, which must equal the
    batch's.  Returns a dict for the JSON line."""
    import torch

    import paper_1808_00963_gb300 as ss
    ss.load()
    specs = gen.batch_specs(num, 4)
    sets = [gen.make_set(k, n, sd) for (k, n, sd) in specs]
    chars, offsets, cbase, first, mls = gen.concat(sets)
    total = int(offsets.shape[0])
    dev = torch.device("cuda", torch.cuda.current_device())
    chars_d = torch.from_numpy(chars).to(dev)
    offs_d = torch.from_numpy(offsets.view(np.int64)).to(dev)
    perm_d = torch.empty(total, dtype=torch.int32, device=dev)
    lcp_d = torch.empty(total, dtype=torch.int32, device=dev)
    descs = []
    for i, st in enumerate(sets):
        a, b = int(first[i]), int(first[i]) + st.n
        descs.append((chars_d[int(cbase[i]):], offs_d[a:b], int(mls[i]), perm_d[a:b], lcp_d[a:b]))
    from paper_1808_00963_gb300 import tune
    tuned = {k: v for k, v in tune.options_for(batched=True).items() if v}
    batch = ss.Batch(descs, **tuned)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(max(warmup, 3)):
            batch.run()
    batch.status(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.run()

    def timed(fn, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    launches0 = ss.launch_count()
    ms_graph = timed(graph.replay, steps)
    batch.status()
    with torch.cuda.stream(stream):
        ms_nograph = timed(lambda: batch.run(stream), steps)
    batch.status(stream)
    launches = ss.launch_count() - launches0
    # the batch's result (every set) before the plain loop runs
    batch_perm, batch_lcp = perm_d.clone(), lcp_d.clone()
    # plain: one ss_sort call per set, one after another, into its own buffers
    plain_perm = torch.full_like(perm_d, -1)
    plain_lcp = torch.full_like(lcp_d, -1)
    lat = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (ch, of, ml, _, _) in enumerate(descs):
        a = time.perf_counter()
        lo, hi = int(first[i]), int(first[i]) + sets[i].n
        ss.sort(ch, of, max_len=ml, out=(plain_perm[lo:hi], plain_lcp[lo:hi]))
        torch.cuda.current_stream().synchronize()
        lat.append((time.perf_counter() - a) * 1e3)
    plain_s = time.perf_counter() - t0
    lat = np.array(lat)
    # parity: the batch (graph replay) and the plain calls give identical arrays
    if not (torch.equal(batch_perm, plain_perm) and torch.equal(batch_lcp, plain_lcp)):
        raise SystemExit("batched and plain results differ")
    done = np.cumsum(lat)
    return {
        "workload": f"batched: {num} sets, log-uniform 100-200k strings, random/URL/DNA generators",
        "sets": num, "strings": total, "chars_bytes": int(chars.shape[0]),
        "options": tuned or "compiled defaults",
        "graph": {"ms": ms_graph, "strings_per_s": total / (ms_graph / 1e3),
                  "completion_ms_p50": ms_graph, "completion_ms_p99": ms_graph},
        "no_graph": {"ms": ms_nograph, "strings_per_s": total / (ms_nograph / 1e3)},
        "plain_loop": {"ms": plain_s * 1e3, "strings_per_s": total / plain_s,
                       "per_call_ms_p50": float(np.percentile(lat, 50)),
                       "per_call_ms_p99": float(np.percentile(lat, 99)),
                       "completion_ms_p50": float(np.percentile(done, 50)),
                       "completion_ms_p99": float(np.percentile(done, 99))},
        "speedup_vs_plain": plain_s * 1e3 / ms_graph,
        "p99_completion_speedup": float(np.percentile(done, 99)) / ms_graph,
        "parity": ("checked: every set's permutation and LCP array from the batch equal those of its own "
                   "ss_sort call"),
        "gpu_launches": launches,
    }


def run_batch(args, ws, rank, local):
    """Configuration 4 on its own line (value: batch strings/s, graph replay)."""
    r = batch_workload(args.sets, args.warmup, args.steps)
    line = {
        "metric": METRIC, "value": r["graph"]["strings_per_s"], "unit": "strings/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": r["graph"]["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": r["workload"], "sets": r["sets"], "strings": r["strings"],
                   "chars_bytes": r["chars_bytes"],
                   "per_step": "one batch (all sets sorted, perm + LCP), CUDA graph replay",
                   "options": r["options"], "options_source": "autotuner table (tuned.json)"},
        "batched_graph": r["graph"], "batched_no_graph": r["no_graph"], "plain_loop": r["plain_loop"],
        "speedup_vs_plain": r["speedup_vs_plain"], "p99_completion_speedup": r["p99_completion_speedup"],
        "parity": r["parity"], "gpu_launches": r["gpu_launches"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---- served workload (configuration 5) ----------------------------------------------------------

SERVED_POOL = 150


def served_trace(num_requests: int, pool_size: int = SERVED_POOL):
    """Configuration 5: a Poisson trace of num_requests sort requests (unit
    rate; log-uniform 1k..5M strings, mixed generators).  Request j replays
    set j mod pool_size of a pool generated from the trace's first pool_size
    entries, so that 2000 requests need no more host memory than 150."""
    spec = gen.trace(num_requests, 5, 1.0, smin=1000, smax=5_000_000)
    pool = [gen.make_set(kind, size, sd) for (_, kind, size, sd) in spec[:pool_size]]
    return spec, pool


def served_workload(num_requests: int, pool_size: int = SERVED_POOL, check: bool = True):
    """The served form against a one-at-a-time plain loop on the same trace
    (arrival rate 0.8 x the plain loop's measured capacity), plus both at
    saturation (every request available at once).  With check, every pool set
    is first sorted alone (ss_sort) and verified by the oracle's O(n + D)
    checker, and a last served pass at saturation compares every request's
    result with its set's.  Returns a dict for the JSON line."""
    import dataclasses

    import torch

    import paper_1808_00963_gb300 as ss
    from paper_1808_00963_gb300.serve import Server, make_request
    ss.load()
    spec, pool = served_trace(num_requests, pool_size)
    base = [make_request(i, 0.0, st.chars, st.offsets, st.max_len) for i, st in enumerate(pool)]
    reqs = []
    for j, (t, _, _, _) in enumerate(spec):
        r = dataclasses.replace(base[j % len(pool)], rid=j, arrival=t, meta={"pool": j % len(pool)})
        reqs.append(r)
    total = sum(r.n for r in reqs)

    expected = None
    if check:
        import oracle
        expected = []
        for st in pool:
            ch = torch.from_numpy(st.chars).cuda()
            of = torch.from_numpy(st.offsets.view(np.int64)).cuda()
            p, l = ss.sort(ch, of, max_len=st.max_len)
            hp, hl = p.cpu().numpy().view(np.uint32), l.cpu().numpy().view(np.uint32)
            r = oracle.check(st.chars, st.offsets, hp, hl, st.max_len)
            if r != -1:
                raise SystemExit(f"served pool set {st.name}: oracle check fails at {r}")
            expected.append((hp, hl))
        del ch, of, p, l

    def reset(arrivals):
        for r, a in zip(reqs, arrivals):
            r.arrival, r.start, r.done, r.batch_size = a, -1.0, -1.0, 0

    # warm-up and capacity of the plain loop (all requests available at once)
    reset([0.0] * len(reqs))
    Server(mode="plain").run(reqs)
    reset([0.0] * len(reqs))
    cap = Server(mode="plain").run(reqs)
    capacity = cap["strings_per_s"]
    reset([0.0] * len(reqs))
    cap_served = Server(mode="served", budget_bytes=30 << 30, streams=4).run(reqs)
    rate = 0.8 * capacity / (total / len(reqs))  # requests per second
    arrivals = [t / rate for (t, _, _, _) in spec]
    reset(arrivals)
    plain = Server(mode="plain").run(reqs)
    reset(arrivals)
    served = Server(mode="served", budget_bytes=30 << 30, streams=4).run(reqs)
    parity = "not checked"
    if check:
        checked = [0]

        def verify(r):
            hp, hl = expected[r.meta["pool"]]
            if not (np.array_equal(r.perm.numpy().view(np.uint32), hp)
                    and np.array_equal(r.lcp.numpy().view(np.uint32), hl)):
                raise RuntimeError(f"request {r.rid}: served result differs from its set sorted alone")
            checked[0] += 1

        reset([0.0] * len(reqs))
        v = Server(mode="served", budget_bytes=30 << 30, streams=4, on_done=verify).run(reqs)
        if v["errors"] or checked[0] != len(reqs):
            raise SystemExit(f"served parity check failed: {v['errors'][:3]}")
        parity = (f"checked: all {len(reqs)} served results equal their set sorted alone; the {len(pool)} pool "
                  "sets pass the oracle's O(n + D) checker")
    return {
        "workload": (f"served: Poisson stream of {len(reqs)} sort requests, log-uniform 1k-5M strings, mixed "
                     f"generators, 30 GB HBM budget (a pool of {len(pool)} generated sets replayed)"),
        "requests": len(reqs), "strings": total, "offered_load": 0.8,
        "plain_capacity_strings_per_s": capacity, "arrival_rate_per_s": rate,
        "served": served, "plain": plain,
        "saturated": {"plain_strings_per_s": capacity, "served_strings_per_s": cap_served["strings_per_s"],
                      "served_mean_batch": cap_served["mean_batch"],
                      "throughput_ratio": cap_served["strings_per_s"] / capacity},
        "p99_speedup": plain["latency_ms_p99"] / served["latency_ms_p99"],
        "throughput_ratio": served["strings_per_s"] / plain["strings_per_s"],
        "parity": parity,
    }


def run_served(args, ws, rank, local):
    """A Poisson stream of sort requests (log-uniform 1k..5M strings, mixed
    generators) replayed against the serving loop (admission by a 30 GB HBM
    budget, continuous batching on 4 streams) and against a one-at-a-time
    plain loop on the same trace.  Arrival rate: 0.8 x the plain loop's
    measured capacity."""
    r = served_workload(args.requests)
    served = r["served"]
    line = {
        "metric": METRIC, "value": served["strings_per_s"], "unit": "strings/s", "n_gpus": ws, "steps": 1,
        "warmup": 1, "ms_per_step": served["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": r["workload"], "requests": r["requests"], "strings": r["strings"],
                   "offered_load": 0.8, "plain_capacity_strings_per_s": r["plain_capacity_strings_per_s"],
                   "arrival_rate_per_s": r["arrival_rate_per_s"],
                   "per_step": "the whole trace; latency = completion (results on the host) - arrival"},
        **{k: r[k] for k in ("served", "plain", "saturated", "p99_speedup", "throughput_ratio", "parity")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "m2", "s3", "d3"])
    ap.add_argument("--requests", type=int, default=2000, help="number of requests (c5)")
    ap.add_argument("--sets", type=int, default=4096, help="number of sets (c4)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="leave out the batched (configuration 4) and served (configuration 5) parts of the "
                         "default line")
    ap.add_argument("--n", type=int, default=None, help="reduced string count (c2 and m2; profiler captures)")
    ap.add_argument("--no-graph-loop", action="store_true",
                    help="run the multi-block rounds launch by launch (for kernel profilers, which do not see "
                         "kernels inside graphs with conditional nodes)")
    args = ap.parse_args()
    if args.no_graph_loop and args.impl == "ours":
        import paper_1808_00963_gb300 as ss
        ss.set_graph_loop(False)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), rank)
        return
    ws, rank, local = dist_init()
    if args.config == "c4":
        run_batch(args, ws, rank, local)
    elif args.config == "c5":
        run_served(args, ws, rank, local)
    elif args.config == "m2":
        run_merge(args, ws, rank, local)
    elif args.config == "s3":
        run_sa(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
