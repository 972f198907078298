"""The device-side wait limit (ss_options.wait_limit_us) in a form that faults,
traps or hangs nothing: a sort whose root subset goes to the work queue starts
one persistent block on it while every other block waits for the subsets it
will push; with a 1-microsecond limit those waits run out, the blocks return,
and the call reports SS_ERR_TIMEOUT.  The next ordinary sort on the same
stream must then succeed with the oracle's result."""
import numpy as np
import pytest

import gen
from gpu_util import assert_parity, gpu_sort, to_device

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_the_next_sort_succeeds():
    import paper_1808_00963_gb300 as ss
    s = gen.url_set(6000, 77)  # above the small cutoff, below the multi-block threshold
    chars, offsets = to_device(s)
    with pytest.raises(ss.SortError) as e:
        ss.sort(chars, offsets, wait_limit_us=1)
        ss.stream_status()
    assert e.value.code == 5  # SS_ERR_TIMEOUT
    p, l = gpu_sort(s)
    assert_parity(s, p, l)
    r = gen.url_set(300_000, 78)
    p, l = gpu_sort(r)
    assert_parity(r, p, l)


def test_generous_wait_limit_changes_nothing():
    s = gen.url_set(50_000, 79)
    p, l = gpu_sort(s, wait_limit_us=2_000_000)
    assert_parity(s, p, l)


def test_expired_wait_leaves_in_range_outputs():
    """After a device-side error the sort writes the identity permutation and
    zero LCPs (outputs first filled with out-of-range values)."""
    import torch

    import paper_1808_00963_gb300 as ss
    s = gen.url_set(6000, 80)
    chars, offsets = to_device(s)
    perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(ss.SortError) as e:
        ss.sort(chars, offsets, out=(perm, lcp), wait_limit_us=1)
    assert e.value.code == 5
    assert np.array_equal(perm.cpu().numpy(), np.arange(s.n, dtype=np.int32))
    assert not lcp.cpu().numpy().any()
