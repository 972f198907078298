"""ss_sort_ex is asynchronous (the multi-block rounds are planned on the
device and run as one graph launch with a conditional WHILE node): the call
returns while its stream is still busy, device-side errors are read later with
ss_stream_status, and sorts queued back to back on one stream, or running on
several streams at once, give the oracle's results."""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _check(s, perm, lcp):
    p = perm.cpu().numpy().view(np.uint32)
    l = lcp.cpu().numpy().view(np.uint32)
    assert oracle.check(s.chars, s.offsets, p, l, s.max_len) == -1, s.name


def test_sort_returns_before_its_stream_completes():
    import torch

    import paper_1808_00963_gb300 as ss
    lib = ss.load()
    s = gen.url_set(1_000_000, 81)
    chars, offsets = to_device(s)
    stream = torch.cuda.Stream()
    perm = torch.empty(s.n, dtype=torch.int32, device="cuda")
    lcp = torch.empty(s.n, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        ss.sort(chars, offsets, out=(perm, lcp), stream=stream)  # first call on the stream: builds its loop graph
        perm.fill_(-1)
        lcp.fill_(-1)
        torch.cuda._sleep(400_000_000)  # a kernel that keeps the stream busy for a while
        rc = lib.ss_sort_ex(ctypes.c_void_p(chars.data_ptr()), ctypes.c_void_p(offsets.data_ptr()), s.n,
                            ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(lcp.data_ptr()), None,
                            ctypes.c_void_p(stream.cuda_stream))
        ev = torch.cuda.Event()
        ev.record(stream)
        returned_early = not ev.query()
    assert rc == 0
    assert returned_early, "ss_sort_ex waited for its stream"
    ss.stream_status(stream)
    _check(s, perm, lcp)


def test_sorts_back_to_back_on_one_stream_and_on_several_streams():
    import torch

    import paper_1808_00963_gb300 as ss
    sets = [gen.url_set(400_000, 82), gen.random_set(300_000, 83), gen.dna_suffix_set(250_000, 84),
            gen.url_set(20_000, 85), gen.url_set(9000, 86), gen.random_set(150_000, 87)]
    dev = [to_device(s) for s in sets]
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = []
    for k in range(2):  # twice: the second pass reuses each stream's loop graph
        outs = []
        for i, (s, (ch, of)) in enumerate(zip(sets, dev)):
            st = streams[i % 3] if k else streams[0]
            p, l = ss.sort(ch, of, max_len=s.max_len, stream=st, sync=False)
            outs.append((p, l))
        for st in streams:
            ss.stream_status(st)
        for s, (p, l) in zip(sets, outs):
            _check(s, p, l)


def test_device_error_goes_to_the_stream_status():
    import torch

    import paper_1808_00963_gb300 as ss
    s = gen.url_set(6000, 88)
    chars, offsets = to_device(s)
    stream = torch.cuda.Stream()
    ss.sort(chars, offsets, stream=stream, sync=False, wait_limit_us=1)  # returns SS_OK: the error is on the device
    with pytest.raises(ss.SortError) as e:
        ss.stream_status(stream)
    assert e.value.code == 5
    ss.stream_status(stream)  # read and cleared
    p, l = ss.sort(chars, offsets, stream=stream)
    _check(s, p, l)
