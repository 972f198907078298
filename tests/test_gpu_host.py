"""The host-buffer entry point with the copy overlapped with the sort: parts
sorted as their characters arrive, then LCP-merged (Section 4.3.1), against
the oracle element by element; sets whose strings are not packed in index
order take the whole-set sort instead, with the same result."""
import numpy as np
import pytest

import gen
from gpu_util import assert_parity

pytestmark = pytest.mark.gpu


def host_sort(s, with_lcp=True, **opts):
    import paper_1808_00963_gb300 as ss
    ss.reset_kernel_stats()
    ss.set_profiling(True)
    try:
        p, l = ss.sort_host(s.chars, s.offsets.view(np.int64), s.max_len, with_lcp=with_lcp, **opts)
        stats = ss.kernel_stats()
    finally:
        ss.set_profiling(False)
    return p, l, stats


def merged(stats):
    return "merge_round" in stats and "layout_check" in stats


def repack(s, order):
    """The strings of a packed set s re-laid back to back in the given index
    order (string i of the result is string order[i] of s)."""
    ends = np.append(s.offsets[1:], np.uint64(s.N)).astype(np.int64)
    starts = s.offsets.astype(np.int64)
    pieces = [s.chars[starts[i]:ends[i]] for i in order]
    lens = np.array([len(x) for x in pieces], np.int64)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64)
    return gen.StringSet(np.concatenate(pieces), offs, s.max_len)


@pytest.mark.parametrize("parts", [2, 4, 8, 16])
def test_parts_match_oracle(parts):
    s = gen.url_set(300_000, 31)
    p, l, st = host_sort(s, host_parts=parts)
    assert merged(st)
    assert_parity(s, p, l)


@pytest.mark.parametrize("kind", ["random", "url", "dups"])
def test_parts_kinds(kind):
    if kind == "random":
        s = gen.random_set(200_003, 5, 0, 12, ord("a"), ord("c"))  # empty strings and many equal ones
    elif kind == "url":
        s = gen.url_set(123_457, 6)
    else:  # every string repeated, copies in different parts
        base = gen.url_set(50_000, 7)
        rng = np.random.default_rng(1)
        s = repack(base, rng.integers(0, base.n, 150_000))
    p, l, st = host_sort(s, host_parts=4)
    assert merged(st)
    assert_parity(s, p, l)


def test_parts_capped():
    s = gen.url_set(200_000, 8)
    s.max_len = 23
    p, l, st = host_sort(s, host_parts=8)
    assert merged(st)
    assert_parity(s, p, l)


def test_parts_without_lcp():
    s = gen.url_set(100_000, 10)
    p, l, st = host_sort(s, with_lcp=False, host_parts=4)
    assert l is None
    want, _ = host_sort(s, host_parts=1)[:2]
    assert np.array_equal(p, want)


def test_parts_minimum_size():
    # 2 strings per part is the smallest split; fewer strings sort in one piece
    for n in (3, 4, 7, 8, 9, 33):
        s = gen.url_set(n, 12)
        p, l, _ = host_sort(s, host_parts=4)
        assert_parity(s, p, l)


@pytest.mark.parametrize("layout", ["suffixes", "shuffled", "shared", "gaps", "no_final_nul"])
def test_unpacked_layouts_fall_back(layout):
    """Layouts the parts cannot use: the whole-set sort runs again, and the
    result is still the oracle's."""
    rng = np.random.default_rng(2)
    if layout == "suffixes":
        s = gen.dna_suffix_set(60_000, 3)
    elif layout == "shuffled":  # packed, but not in index order
        s = gen.url_set(80_000, 4)
        s.offsets = s.offsets[rng.permutation(s.n)]
    elif layout == "shared":  # two indices on the same string
        s = gen.url_set(80_000, 4)
        s.offsets[1000] = s.offsets[999]
    elif layout == "gaps":  # a byte between two strings
        b = gen.url_set(80_000, 4)
        chars = np.insert(b.chars, int(b.offsets[40_000]), np.uint8(ord("x")))
        offs = b.offsets.copy()
        offs[40_000:] += 1
        s = gen.StringSet(chars, offs, 0)
    else:  # trailing bytes after the last terminator
        b = gen.url_set(80_000, 4)
        s = gen.StringSet(np.concatenate([b.chars, np.frombuffer(b"tail\0zz", np.uint8)]), b.offsets, 0)
    p, l, st = host_sort(s, host_parts=4)
    assert "layout_check" in st
    assert_parity(s, p, l)


def test_parts_two_million():
    """2^21 + 1 URL-like strings in 8 parts (parts of 262144 strings take the
    multi-block steps)."""
    s = gen.url_set((1 << 21) + 1, 13)
    p, l, st = host_sort(s, host_parts=8)
    assert merged(st)
    assert_parity(s, p, l)


def test_default_is_one_piece():
    s = gen.url_set(100_000, 15)
    p, l, st = host_sort(s)
    assert "merge_round" not in st and "layout_check" not in st
    assert_parity(s, p, l)


def test_device_offsets_rejected():
    import torch

    import paper_1808_00963_gb300 as ss
    s = gen.url_set(1000, 14)
    doff = torch.from_numpy(s.offsets.view(np.int64)).cuda()
    with pytest.raises(ss.SortError):
        ss.sort_host(s.chars, doff, host_parts=4)
