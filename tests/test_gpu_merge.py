"""The K-way LCP merge of sorted runs (Section 4.3.2, Algorithm 4.5, split into
pieces as in Section 4.3.3) against the oracle's definition of the merge (the
sorted union, ties by index, and its LCP array), element by element.

The runs are made on the CPU by the oracle (each run the oracle's sort of a
seeded subset of the strings); only the full-size case sorts its runs on the
GPU, and it is checked by the oracle's O(n + D) checker (the merged order of a
partition of all strings is the unique sorted order)."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def cpu_runs(s, assign, K):
    runs = []
    for k in range(K):
        sub = np.nonzero(assign == k)[0].astype(np.uint32)
        if sub.size:
            p, l = oracle.sort(s.chars, s.offsets[sub], s.max_len)
            runs.append((sub[p], l))
        else:
            runs.append((np.zeros(0, np.uint32), np.zeros(0, np.uint32)))
    return runs


def gpu_merge(s, runs, sample_step=0, with_lcp=True, stream=None, workspace=False):
    import torch

    import paper_1808_00963_gb300 as ss
    chars, offsets = to_device(s)
    druns = [(torch.from_numpy(p.view(np.int32)).cuda(), torch.from_numpy(l.view(np.int32)).cuda())
             for p, l in runs]
    kw = {}
    if workspace:
        wsb = ss.merge_workspace_size(druns, sample_step)
        buf = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda")
        kw = dict(workspace=buf.data_ptr(), workspace_bytes=wsb)
    perm, lcp = ss.merge(chars, offsets, druns, max_len=s.max_len, with_lcp=with_lcp, sample_step=sample_step,
                         stream=stream, **kw)
    torch.cuda.synchronize()
    return perm.cpu().numpy().view(np.uint32), (lcp.cpu().numpy().view(np.uint32) if lcp is not None else None)


def assert_merge_parity(s, runs, perm, lcp):
    want_p, want_l = oracle.merge(s.chars, s.offsets, [r[0] for r in runs], s.max_len)
    bad = np.nonzero(perm != want_p)[0]
    assert bad.size == 0, f"perm differs at {bad[:10]} (of {bad.size}); total={want_p.size}"
    if lcp is not None:
        bad = np.nonzero(lcp != want_l)[0]
        assert bad.size == 0, f"lcp differs at {bad[:10]}: got {lcp[bad[:5]]} want {want_l[bad[:5]]}"


WORKLOADS = {
    "random": lambda: gen.random_set(60000, 71, 0, 20, ord("a"), ord("d")),
    "url": lambda: gen.url_set(80000, 72),
    "dna": lambda: gen.dna_suffix_set(60000, 73, nblocks=12, blocklen=400),
    "equal_heavy": lambda: gen.random_set(50000, 74, 0, 3, ord("a"), ord("b")),
    "caps": lambda: gen.random_set(40000, 75, 0, 40, 1, 3),
}


@pytest.mark.parametrize("K", [1, 2, 5, 16, 64])
@pytest.mark.parametrize("case", sorted(WORKLOADS))
def test_merge_matches_oracle(case, K):
    s = WORKLOADS[case]()
    if case == "caps":
        s.max_len = 11
    rng = np.random.default_rng(1000 + K)
    assign = rng.integers(0, K, s.n)
    runs = cpu_runs(s, assign, K)
    for step in (16, 0):
        perm, lcp = gpu_merge(s, runs, sample_step=step)
        assert_merge_parity(s, runs, perm, lcp)


@pytest.mark.parametrize("layout", ["blocks", "round_robin", "one_giant", "sparse_runs", "all_equal",
                                    "shared_index", "tiny", "single"])
def test_merge_edge_cases(layout):
    """Runs that hold contiguous stretches of the sorted order (pieces made of
    one run), interleave it exactly, differ greatly in size, are mostly empty;
    equal strings spread over all runs (ties by index); an index present in
    two runs; one or two strings in all."""
    rng = np.random.default_rng(7)
    s = gen.url_set(30000, 81)
    K = 8
    if layout in ("blocks", "round_robin"):
        order, _ = oracle.sort(s.chars, s.offsets, s.max_len)
        rank = np.empty(s.n, np.int64)
        rank[order] = np.arange(s.n)
        assign = (rank * K // s.n) if layout == "blocks" else (rank % K)
    elif layout == "one_giant":
        assign = np.where(rng.random(s.n) < 0.995, 3, rng.integers(0, K, s.n))
    elif layout == "sparse_runs":
        K = 64
        assign = rng.choice([2, 17, 40, 63], s.n)
    elif layout == "all_equal":
        s = gen.random_set(20000, 82, 12, 12, ord("q"), ord("q"))
        assign = rng.integers(0, K, s.n)
    elif layout == "shared_index":
        assign = rng.integers(0, K, s.n)
    elif layout == "tiny":
        s = gen.url_set(2, 83)
        assign = np.array([5, 1])
    else:
        s = gen.url_set(1, 84)
        assign = np.array([0])
    runs = cpu_runs(s, assign, K)
    if layout == "shared_index":
        sub = np.sort(rng.choice(s.n, 3000, replace=False)).astype(np.uint32)
        p, l = oracle.sort(s.chars, s.offsets[sub], s.max_len)
        runs.append((sub[p], l))
    for step in (16, 0):
        perm, lcp = gpu_merge(s, runs, sample_step=step)
        assert_merge_parity(s, runs, perm, lcp)


def test_merge_without_lcp_and_with_caller_workspace():
    import torch
    s = gen.dna_suffix_set(50000, 91, nblocks=8, blocklen=300)
    s.max_len = 64
    runs = cpu_runs(s, np.random.default_rng(3).integers(0, 6, s.n), 6)
    st = torch.cuda.Stream()
    perm, lcp = gpu_merge(s, runs, sample_step=32, with_lcp=False, stream=st, workspace=True)
    assert lcp is None
    want_p, _ = oracle.merge(s.chars, s.offsets, [r[0] for r in runs], s.max_len)
    assert np.array_equal(perm, want_p)
    perm, lcp = gpu_merge(s, runs, sample_step=0, workspace=True)
    assert_merge_parity(s, runs, perm, lcp)


@pytest.mark.slow
def test_merge_full_size_urls():
    """20M URLs (the sort's URL workload) in 16 runs of a seeded partition,
    each run sorted on the GPU; the merged order must pass the oracle's
    checker (sorted, ties by index, exact LCPs, a permutation of all strings)."""
    import torch

    import paper_1808_00963_gb300 as ss
    s = gen.config2()
    chars, offsets = to_device(s)
    K = 16
    assign = torch.from_numpy(np.random.default_rng(5).integers(0, K, s.n)).cuda()
    runs = []
    for k in range(K):
        sub = torch.nonzero(assign == k).flatten()
        p, l = ss.sort(chars, offsets[sub].contiguous(), max_len=s.max_len)
        runs.append((sub[p.long()].int().contiguous(), l))
    perm, lcp = ss.merge(chars, offsets, runs, max_len=s.max_len)
    torch.cuda.synchronize()
    p = perm.cpu().numpy().view(np.uint32)
    l = lcp.cpu().numpy().view(np.uint32)
    assert oracle.check(s.chars, s.offsets, p, l, s.max_len) == -1


def test_merge_offsets_above_4gib():
    """Runs whose strings lie beyond byte 2^32 of the character buffer (the
    merge records carry full 64-bit offsets), mixed with strings below it and
    with every lower string repeated above."""
    base = gen.url_set(40_000, 23)
    hi = (1 << 32) + 777
    chars = np.zeros(hi + base.N + 64, np.uint8)
    chars[:base.N] = base.chars
    chars[hi:hi + base.N] = base.chars
    offsets = np.concatenate([base.offsets[:20_000], base.offsets + np.uint64(hi)])
    s = gen.StringSet(chars, offsets, 0)
    assign = np.random.default_rng(4).integers(0, 5, s.n)
    runs = cpu_runs(s, assign, 5)
    perm, lcp = gpu_merge(s, runs)
    assert_merge_parity(s, runs, perm, lcp)
    import torch
    torch.cuda.empty_cache()
