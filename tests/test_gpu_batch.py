"""Batched sorting (ss_batch_*): many independent string sets in one launch
sequence, also captured into a CUDA graph and replayed.  Every set's result
must equal the oracle's and the result of sorting that set alone (integer
outputs: identical)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def _device_sets(sets):
    import torch
    out = []
    for s in sets:
        ch = torch.from_numpy(np.ascontiguousarray(s.chars) if s.N else np.zeros(1, np.uint8)).cuda()
        of = torch.from_numpy(np.ascontiguousarray(s.offsets).view(np.int64)).cuda()
        p = torch.full((max(s.n, 1),), -1, dtype=torch.int32, device="cuda")
        l = torch.full((max(s.n, 1),), -1, dtype=torch.int32, device="cuda")
        out.append((ch, of, s.max_len, p, l))
    return out


def _mixed_sets(num, seed, smax=20000):
    specs = gen.batch_specs(num, seed, smin=2, smax=smax)
    sets = [gen.make_set(k, n, sd) for (k, n, sd) in specs]
    # degenerate members: empty set, single string, all-equal strings
    sets.append(gen.StringSet(np.zeros(1, np.uint8), np.zeros(0, np.uint64), 0))
    sets.append(gen.StringSet(np.frombuffer(b"x\0", np.uint8).copy(), np.zeros(1, np.uint64), 0))
    eq = oracle.from_strings([b"same-prefix-same-prefix"] * 300)
    sets.append(gen.StringSet(eq[0], eq[1], 0))
    return sets


def _check(sets, dev):
    for s, (_, _, _, p, l) in zip(sets, dev):
        if s.n == 0:
            continue
        gp = p[:s.n].cpu().numpy().view(np.uint32)
        gl = l[:s.n].cpu().numpy().view(np.uint32)
        wp, wl = oracle.sort(s.chars, s.offsets, s.max_len)
        assert np.array_equal(gp, wp), s.name
        assert np.array_equal(gl, wl), s.name


def test_batch_matches_oracle_and_single_calls():
    import torch

    import paper_1808_00963_gb300 as ss
    sets = _mixed_sets(120, 11)
    dev = _device_sets(sets)
    b = ss.Batch(dev)
    b.run()
    b.status()
    _check(sets, dev)
    # each set alone through ss_sort gives the same arrays
    for s, (ch, of, ml, p, l) in list(zip(sets, dev))[:40]:
        if s.n == 0:
            continue
        p1, l1 = ss.sort(ch, of, max_len=ml)
        assert torch.equal(p1, p[:s.n]) and torch.equal(l1, l[:s.n])
    b.close()


def test_batch_graph_replay():
    import torch

    import paper_1808_00963_gb300 as ss
    sets = _mixed_sets(60, 12)
    dev = _device_sets(sets)
    b = ss.Batch(dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.run()  # warm-up outside capture (sets kernel attributes)
    b.status(stream)
    for (_, _, _, p, l) in dev:
        p.fill_(-1)
        l.fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.run()
    for _ in range(2):
        for (_, _, _, p, l) in dev:
            p.fill_(-1)
            l.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        b.status()
        _check(sets, dev)
    b.close()


def test_batch_per_set_caps():
    import paper_1808_00963_gb300 as ss
    sets = []
    for k in range(10):
        s = gen.dna_suffix_set(3000 + 100 * k, 30 + k, nblocks=2, blocklen=300)
        s.max_len = [1, 7, 8, 9, 16, 50, 100, 500, 0, 3][k]
        sets.append(s)
    dev = _device_sets(sets)
    b = ss.Batch(dev)
    b.run()
    b.stream_status()
    _check(sets, dev)
    b.close()


def test_sort_batch_convenience():
    import ctypes

    import paper_1808_00963_gb300 as ss
    sets = _mixed_sets(20, 13, smax=5000)
    dev = _device_sets(sets)
    lib = ss.load()
    arr = (ss.SetDesc * len(dev))()
    for i, (ch, of, ml, p, l) in enumerate(dev):
        arr[i].chars, arr[i].offsets, arr[i].n = ch.data_ptr(), of.data_ptr(), int(of.numel())
        arr[i].max_len, arr[i].out_perm, arr[i].out_lcp = ml, p.data_ptr(), l.data_ptr()
    import torch
    rc = lib.ss_sort_batch(arr, len(dev), None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    _check(sets, dev)


def _config4_device(sets):
    """The sets of configuration 4 in one device buffer (as bench.py lays them
    out): descriptors of (chars from the set's base, offsets, cap, perm, lcp)."""
    import torch
    chars, offsets, cbase, first, mls = gen.concat(sets)
    chars_d = torch.from_numpy(chars).cuda()
    offs_d = torch.from_numpy(offsets.view(np.int64)).cuda()
    total = int(offsets.shape[0])
    perm_d = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    lcp_d = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    descs, spans = [], []
    for i, st in enumerate(sets):
        a, b = int(first[i]), int(first[i]) + st.n
        descs.append((chars_d[int(cbase[i]):], offs_d[a:b], int(mls[i]), perm_d[a:b], lcp_d[a:b]))
        spans.append((a, b))
    return descs, spans, perm_d, lcp_d


@pytest.mark.slow
def test_config4_full_batch_direct_and_graph_replay():
    """Configuration 4 at its stated size: 4096 sets of 100..200k strings
    (random, URL-like and DNA-suffix generators; 110 M strings), sorted as one
    batch directly and by CUDA-graph replay.  Every set is checked by the
    oracle's complete O(n + D) checker (permutation, order, ties by index,
    every LCP), the replay must reproduce the direct run exactly, and 100 sets
    (the 50 largest and 50 others) must equal single ss_sort calls."""
    import torch

    import paper_1808_00963_gb300 as ss
    from paper_1808_00963_gb300 import tune
    sets = gen.batch_sets(4096, 4)
    descs, spans, perm_d, lcp_d = _config4_device(sets)
    tuned = {k: v for k, v in tune.options_for(batched=True).items() if v}
    b = ss.Batch(descs, **tuned)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.run()
    b.status(stream)
    perm_h = perm_d.cpu().numpy().view(np.uint32)
    lcp_h = lcp_d.cpu().numpy().view(np.uint32)
    for s, (a, e) in zip(sets, spans):
        r = oracle.check(s.chars, s.offsets, perm_h[a:e], lcp_h[a:e], s.max_len)
        assert r == -1, f"{s.name}: oracle check fails at position {r}"
    first_p, first_l = perm_d.clone(), lcp_d.clone()
    perm_d.fill_(-1)
    lcp_d.fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.run()
    for _ in range(2):
        perm_d.fill_(-1)
        lcp_d.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        b.status()
        assert torch.equal(perm_d, first_p) and torch.equal(lcp_d, first_l)
    b.close()
    by_size = sorted(range(len(sets)), key=lambda i: -sets[i].n)
    pick = by_size[:50] + by_size[50::(len(sets) - 50) // 50][:50]
    for i in pick:
        ch, of, ml, _, _ = descs[i]
        a, e = spans[i]
        p1, l1 = ss.sort(ch, of, max_len=ml)
        assert torch.equal(p1, first_p[a:e]) and torch.equal(l1, first_l[a:e]), sets[i].name
