"""ss_sort_noalloc, the entry point for callers that may not allocate device
memory while they run (their memory is reserved up front or owned by another
allocator, or cudaMalloc / cudaFree would stall a latency-critical path).  Its
workspace is a fixed array in the library's device data, shared by all calls.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process.  Each case calls the entry point twice in a row through the
C-ABI (the second call finds the first call's leftovers in the shared array)
and compares both results with the ordinary entry point, ss_sort_ex: the
outputs are integers, so they must be identical."""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _dev(s):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(s.chars)).cuda(),
            torch.from_numpy(np.ascontiguousarray(s.offsets).view(np.int64)).cuda())


@pytest.mark.parametrize("case", ["url_5000", "dna_65536_cap500", "random_40", "words_3"])
def test_noalloc_matches_ss_sort_on_two_calls(case):
    import torch

    import paper_1808_00963_gb300 as ss
    ss.build()
    lib = ss.load()
    s = {"url_5000": lambda: gen.url_set(5000, 41),
         "dna_65536_cap500": lambda: gen.dna_suffix_set(65536, 42, nblocks=3, blocklen=1000),
         "random_40": lambda: gen.random_set(40, 43),
         "words_3": lambda: gen.StringSet(np.frombuffer(b"by\0a\0by\0", np.uint8).copy(),
                                          np.array([0, 3, 5], np.uint64))}[case]()
    chars, offsets = _dev(s)
    want_p, want_l = ss.sort(chars, offsets, max_len=s.max_len)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        p = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
        l = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
        rc = lib.ss_sort_noalloc(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), s.n,
                                 s.max_len, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(l.data_ptr()), stream)
        assert rc == 0, ss.STATUS.get(rc, rc)
        assert torch.equal(p, want_p)
        assert torch.equal(l, want_l)


def test_noalloc_rejects_more_than_its_limit():
    import paper_1808_00963_gb300 as ss
    ss.build()
    lib = ss.load()
    dummy = ctypes.c_void_p(256)
    assert lib.ss_sort_noalloc(dummy, dummy, ss.NOALLOC_MAX_STRINGS + 1, 0, dummy, dummy, None) == 4


def test_noalloc_subsets_requeued_many_times():
    """63 groups of 1040 identical 600-byte strings (65 520 strings): every
    group is an equality bucket above the small cutoff that goes back to the
    work queue 75 times, 4725 queue pushes in all.  The queue is a ring sized
    by the number of disjoint subsets it can hold, so this fits the fixed
    scratch; the result equals ss_sort_ex's, on two calls in a row."""
    import torch

    import paper_1808_00963_gb300 as ss
    ss.build()
    lib = ss.load()
    groups = []
    for g in range(63):
        body = bytes((ord("a") + (g * 7 + k) % 26) for k in range(592))
        groups.append(b"%08d" % (g * 7919 % 100000) + body)
    strs = [groups[i % 63] for i in range(63 * 1040)]
    chars_np = np.frombuffer(b"".join(x + b"\0" for x in strs), np.uint8).copy()
    offs_np = np.arange(len(strs), dtype=np.uint64) * 601
    s = gen.StringSet(chars_np, offs_np)
    chars, offsets = _dev(s)
    want_p, want_l = ss.sort(chars, offsets)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        p = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
        l = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
        rc = lib.ss_sort_noalloc(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), s.n,
                                 0, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(l.data_ptr()), stream)
        assert rc == 0, ss.STATUS.get(rc, rc)
        assert torch.equal(p, want_p)
        assert torch.equal(l, want_l)
