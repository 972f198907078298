"""The autotuner's host logic (no GPU): coordinate descent finds the minimum
of a separable cost, the committed table is well-formed, and the generated
header carries the default options."""
import json
import os

from paper_1808_00963_gb300 import tune


def test_coordinate_descent_finds_separable_minimum():
    space = {"a": [1, 2, 3, 4], "b": [10, 20, 30]}
    target = {"a": 3, "b": 20}
    calls = []

    def run(o):
        calls.append(o)
        return 1.0 + (o["a"] - target["a"]) ** 2 + ((o["b"] - target["b"]) / 10) ** 2

    best, ms, cache = tune.coordinate_descent(run, space, {"a": 1, "b": 10}, passes=2, log=lambda *_: None)
    assert best == target and ms == 1.0
    assert len(calls) == len(cache)  # each configuration timed once


def test_committed_table_and_header():
    with open(tune.TABLE) as f:
        t = json.load(f)
    for kind in ("url", "dna", "random"):
        o = t["plain"][kind]["options"]
        assert set(o) == set(tune.SPACE)
        for k, v in o.items():
            assert v in tune.SPACE[k]
    assert tune.options_for("url") == t["plain"]["url"]["options"]
    assert tune.options_for(batched=True) == t["batched"]["options"]
    d = t["default"]["options"]
    hdr = open(tune.HEADER).read()
    assert f"#define SS_TUNED_SPLITTERS_LOG2 {d['splitters_log2']}" in hdr
    assert f"#define SS_TUNED_SMALL_CUTOFF {d['small_cutoff']}" in hdr
    assert f"#define SS_TUNED_BIG_THRESHOLD {d['big_threshold']}" in hdr


def test_write_header(tmp_path):
    p = os.path.join(tmp_path, "h.h")
    tune.write_header(tune.START, p)
    txt = open(p).read()
    assert "#define SS_TUNED_TILE_ROUNDS 0" in txt and "#pragma once" in txt


def test_warm_start_takes_stored_options_within_the_space():
    space = {"a": [1, 2, 3], "b": [10, 20]}
    table = {"plain": {"url": {"options": {"a": 3, "b": 99, "c": 5}}}}
    # a value outside the space and a missing key fall back to the default
    assert tune.warm_start(table, ("plain", "url"), space, {"a": 1, "b": 10}) == {"a": 3, "b": 10}
    assert tune.warm_start(table, ("plain", "dna"), space, {"a": 1, "b": 10}) == {"a": 1, "b": 10}
    assert tune.warm_start({}, ("batched",), space, {"a": 2, "b": 20}) == {"a": 2, "b": 20}


def test_descent_reuses_timings_across_starts():
    space = {"a": [1, 2, 3]}
    calls = []

    def run(o):
        calls.append(dict(o))
        return float(o["a"])

    _, _, cache = tune.coordinate_descent(run, space, {"a": 3}, 0, log=lambda *_: None)
    best, ms, cache = tune.coordinate_descent(run, space, {"a": 2}, 1, log=lambda *_: None, cache=cache)
    assert best == {"a": 1} and ms == 1.0
    assert len(calls) == 3  # a = 3 was timed once, then reused
