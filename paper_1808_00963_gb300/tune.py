"""Autotuner for the sort's parameters.

The parameters do not change any result (the output is unique); they only
move time between the kernels:

  splitters_log2      v = 2^d - 1 splitters of the single-block steps
  big_splitters_log2  v of the multi-block steps
  small_cutoff        subsets up to this size are finished by the small sorts
  big_threshold       subsets above this size use multi-block steps
  tile_rounds         multi-block tile = 256 * rounds strings (0 = chosen per step)

For each workload class the tuner runs a coordinate descent (one parameter
at a time, two passes) timing complete sorts with CUDA events, starting from
the options the existing table holds for that class (so that a retune after
a kernel change moves only where it measures a gain), and writes
  tuned.json      best options per workload class (and for the batched form)
  csrc/ss_tuned.h the compiled-in defaults: the options with the best
                  geometric mean over the plain workload classes

Run on the GPU:  python -m paper_1808_00963_gb300.tune [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(_HERE, "tuned.json")
HEADER = os.path.join(_HERE, "csrc", "ss_tuned.h")

SPACE = {
    "splitters_log2": [7, 8, 9, 10],
    "big_splitters_log2": [8, 9],
    "small_cutoff": [128, 256, 512, 1024, 2048],
    "big_threshold": [8192, 16384, 32768, 65536],
    "tile_rounds": [0, 8, 16, 32],
}
START = {"splitters_log2": 8, "big_splitters_log2": 9, "small_cutoff": 1024, "big_threshold": 8192,
         "tile_rounds": 0}
# batches: big_threshold 2^30 leaves every set to the single-block steps
BATCH_SPACE = {"splitters_log2": [7, 8, 9, 10], "small_cutoff": [128, 256, 512, 1024, 2048],
               "big_threshold": [8192, 32768, 1 << 30]}


def _timer_plain(s, reps):
    import torch

    from . import load, sort, workspace_size
    load()
    chars = torch.from_numpy(s.chars).cuda()
    offs = torch.from_numpy(s.offsets.view(np.int64)).cuda()
    perm = torch.empty(s.n, dtype=torch.int32, device="cuda")
    lcp = torch.empty_like(perm)

    def run(opts):
        o = {k: v for k, v in opts.items() if v}
        wsb = workspace_size(s.n, s.max_len, **o)
        work = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        f = lambda: sort(chars, offs, max_len=s.max_len, out=(perm, lcp), workspace=work.data_ptr(),  # noqa: E731
                         workspace_bytes=wsb, **o)
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    return run


def _timer_batch(sets, reps):
    import torch

    from . import Batch, load
    load()
    descs = []
    for s in sets:
        ch = torch.from_numpy(s.chars).cuda()
        of = torch.from_numpy(s.offsets.view(np.int64)).cuda()
        descs.append((ch, of, s.max_len, torch.empty(s.n, dtype=torch.int32, device="cuda"),
                      torch.empty(s.n, dtype=torch.int32, device="cuda")))

    def run(opts):
        b = Batch(descs, own_workspace=True, **{k: v for k, v in opts.items() if v})
        b.run()
        b.status()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.run()
        e1.record()
        torch.cuda.synchronize()
        b.status()
        b.close()
        return e0.elapsed_time(e1) / reps

    return run


def coordinate_descent(run, space, start, passes=2, log=print, cache=None):
    best = dict(start)
    cache = {} if cache is None else cache

    def cost(o):
        key = tuple(sorted(o.items()))
        if key not in cache:
            cache[key] = run(o)
            log(f"    {o} -> {cache[key]:.3f} ms")
        return cache[key]

    best_ms = cost(best)
    for _ in range(passes):
        improved = False
        for name, values in space.items():
            for v in values:
                cand = dict(best, **{name: v})
                if cand.get("big_threshold", 1 << 30) < cand.get("small_cutoff", 0):
                    continue
                ms = cost(cand)
                if ms < best_ms * 0.995:
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    return best, best_ms, cache


def warm_start(table, path, space, default):
    """The options stored at table[path[0]][path[1]]...["options"] restricted
    to the keys and values of `space`, completed from `default`; `default`
    when the table has no such entry."""
    e = table
    for k in path:
        e = e.get(k, {}) if isinstance(e, dict) else {}
    o = e.get("options", {}) if isinstance(e, dict) else {}
    return {k: (o[k] if o.get(k) in vals else default[k]) for k, vals in space.items()}


def write_header(opts, path=HEADER):
    with open(path, "w") as f:
        f.write("// Generated by paper_1808_00963_gb300/tune.py on a GB300: compiled-in defaults of\n"
                "// the sort's tuning options (best geometric mean over the plain workload classes).\n"
                "#pragma once\n\n")
        f.write(f"#define SS_TUNED_SPLITTERS_LOG2 {opts['splitters_log2']}\n")
        f.write(f"#define SS_TUNED_BIG_SPLITTERS_LOG2 {opts['big_splitters_log2']}\n")
        f.write(f"#define SS_TUNED_SMALL_CUTOFF {opts['small_cutoff']}\n")
        f.write(f"#define SS_TUNED_BIG_THRESHOLD {opts['big_threshold']}\n")
        f.write(f"#define SS_TUNED_TILE_ROUNDS {opts['tile_rounds']}\n")


def options_for(kind: str | None = None, batched: bool = False) -> dict:
    """Tuned options for a workload class ('random', 'url', 'dna'), for the
    batched form, or the defaults; {} if no table exists."""
    try:
        with open(TABLE) as f:
            t = json.load(f)
    except OSError:
        return {}
    if batched:
        return dict(t.get("batched", {}).get("options", {}))
    if kind and kind in t.get("plain", {}):
        return dict(t["plain"][kind]["options"])
    return dict(t.get("default", {}).get("options", {}))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="smaller inputs and one pass")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--no-write", action="store_true")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(_HERE))
    import gen
    sets = {"url": gen.config2(4_000_000 if args.quick else 20_000_000),
            "dna": gen.config3(1_000_000 if args.quick else 4_000_000),
            "random": gen.config1()}
    passes = 1 if args.quick else 2
    try:
        with open(TABLE) as f:
            old = json.load(f)
    except (OSError, ValueError):
        old = {}
    table = {"plain": {}, "space": SPACE}
    all_costs = {}
    for name, s in sets.items():
        print(f"== {name}: n={s.n}", flush=True)
        run = _timer_plain(s, args.reps if name != "random" else 4 * args.reps)
        # START is timed for every class, so that the default below always
        # has a configuration every class measured
        best, ms, cache = coordinate_descent(run, SPACE, START, 0)
        best, ms, cache = coordinate_descent(run, SPACE, warm_start(old, ("plain", name), SPACE, START), passes,
                                             cache=cache)
        table["plain"][name] = {"options": best, "ms": ms, "n": s.n}
        all_costs[name] = cache
        print(f"   best {best} {ms:.3f} ms", flush=True)
    # default: best geometric mean over the configurations every class measured
    common = set.intersection(*[set(c) for c in all_costs.values()])
    geo = {k: math.exp(sum(math.log(all_costs[n][k]) for n in all_costs) / len(all_costs)) for k in common}
    dkey = min(geo, key=geo.get)
    table["default"] = {"options": dict(dkey), "geomean_ms": geo[dkey]}
    print(f"== default {dict(dkey)} geomean {geo[dkey]:.3f} ms", flush=True)
    # batched form (512 sets of the batched workload)
    bsets = gen.batch_sets(128 if args.quick else 512, 4)
    bstart = {"splitters_log2": 8, "small_cutoff": 1024, "big_threshold": 8192}
    best, ms, _ = coordinate_descent(_timer_batch(bsets, args.reps), BATCH_SPACE,
                                     warm_start(old, ("batched",), BATCH_SPACE, bstart), passes)
    table["batched"] = {"options": best, "ms": ms, "sets": len(bsets)}
    print(f"== batched {best} {ms:.3f} ms", flush=True)
    if not args.no_write:
        with open(TABLE, "w") as f:
            json.dump(table, f, indent=1)
        write_header(dict(dkey))
    print(json.dumps(table))


if __name__ == "__main__":
    main()
