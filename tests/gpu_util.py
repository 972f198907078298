"""Helpers for the GPU parity tests: move a generated string set to the device,
sort it through the C-ABI, compare with the CPU oracle."""
import numpy as np

import gen
import oracle
import paper_1808_00963_gb300 as ss

EXACT_LIMIT = 400_000  # above this, verify with the O(n + D) oracle checker


def to_device(s: gen.StringSet):
    import torch
    chars = torch.from_numpy(np.ascontiguousarray(s.chars)).cuda()
    offsets = torch.from_numpy(np.ascontiguousarray(s.offsets).view(np.int64)).cuda()
    return chars, offsets


def gpu_sort(s: gen.StringSet, with_lcp=True, **opts):
    import torch
    chars, offsets = to_device(s)
    perm, lcp = ss.sort(chars, offsets, max_len=s.max_len, with_lcp=with_lcp, **opts)
    torch.cuda.synchronize()
    p = perm.cpu().numpy().view(np.uint32)
    l = lcp.cpu().numpy().view(np.uint32) if lcp is not None else None
    return p, l


def assert_parity(s: gen.StringSet, perm, lcp, exact_limit=EXACT_LIMIT):
    if s.n <= exact_limit:
        want_p, want_l = oracle.sort(s.chars, s.offsets, s.max_len)
        bad = np.nonzero(perm != want_p)[0]
        assert bad.size == 0, f"perm differs at {bad[:10]} (of {bad.size}); n={s.n}"
        if lcp is not None:
            bad = np.nonzero(lcp != want_l)[0]
            assert bad.size == 0, f"lcp differs at {bad[:10]}: got {lcp[bad[:5]]} want {want_l[bad[:5]]}"
    else:
        r = oracle.check(s.chars, s.offsets, perm, lcp, s.max_len)
        assert r == -1, f"oracle check fails at position {r} (n={s.n})"


def from_strings(strs, max_len=0, name="fixture"):
    chars, offsets = oracle.from_strings(strs)
    return gen.StringSet(chars, offsets, max_len, name)
