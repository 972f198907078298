"""The C-ABI library: it builds for sm_103a, loads, exports every function
include/ss_sort.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import re

import pytest

import paper_1808_00963_gb300 as ss


@pytest.fixture(scope="module")
def lib():
    ss.build()
    return ss.load()


def declared_functions():
    text = open(ss.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ss_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(8):
        assert lib.ss_status_string(code)
    assert lib.ss_status_string(0) == b"ok"


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_host_side_argument_checks(lib):
    o = ss.make_options()
    dummy = ctypes.c_void_p(16)
    # n = 0 is a no-op, n >= 2^32 is too large, NULL inputs are invalid
    assert lib.ss_sort_ex(None, None, 0, None, None, ctypes.byref(o), None) == 0
    assert lib.ss_sort_ex(dummy, dummy, 1 << 32, dummy, None, ctypes.byref(o), None) == 4
    assert lib.ss_sort_ex(None, dummy, 5, dummy, None, ctypes.byref(o), None) == 1
    assert lib.ss_sort_ex(dummy, dummy, 5, None, None, ctypes.byref(o), None) == 1
    # option ranges
    for bad in (dict(splitters_log2=6), dict(splitters_log2=11), dict(small_cutoff=32),
                dict(small_cutoff=8192), dict(tile_rounds=64), dict(host_parts=3), dict(host_parts=32), dict(classifier=4),
                dict(small_cutoff=1024, big_threshold=512),
                dict(big_splitters_log2=7), dict(big_splitters_log2=10)):
        ob = ss.make_options(**bad)
        assert lib.ss_sort_ex(dummy, dummy, 5, dummy, None, ctypes.byref(ob), None) == 1, bad
        assert lib.ss_workspace_size(1000, ctypes.byref(ob)) == 0
    # misaligned caller workspace
    ob = ss.make_options(workspace=ctypes.c_void_p(4096 + 8), workspace_bytes=1 << 20)
    assert lib.ss_sort_ex(dummy, dummy, 5, dummy, None, ctypes.byref(ob), None) == 1
    if not _has_gpu():
        assert lib.ss_sort_ex(dummy, dummy, 5, dummy, None, ctypes.byref(o), None) == 7


def test_workspace_size(lib):
    o = ss.make_options()
    small = lib.ss_workspace_size(1000, ctypes.byref(o))
    big = lib.ss_workspace_size(10_000_000, ctypes.byref(o))
    assert 0 < small < big
    # records (2 x 12 B) + bucket array, plus task lists: tens of bytes per string
    assert 26 * 10_000_000 < big < 80 * 10_000_000
    sets = (ss.SetDesc * 2)()
    sets[0].n, sets[1].n = 500, 700
    sets[0].chars = sets[0].offsets = sets[0].out_perm = 64
    sets[1].chars = sets[1].offsets = sets[1].out_perm = 64
    assert lib.ss_batch_workspace_size(sets, 2, ctypes.byref(o)) > 0


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        ss.load(str(tmp_path / "nope.so"))


def test_merge_argument_checks(lib):
    dummy = ctypes.c_void_p(4096)
    runs = (ss.RunDesc * 65)()
    for r in runs:
        r.perm = r.lcp = 4096
        r.n = 100
    call = lambda k, step=0, chars=dummy, out=dummy: lib.ss_merge(  # noqa: E731
        chars, dummy, 0, runs, k, step, out, None, None, 0, None)
    assert call(0) == 1                      # no runs
    assert call(65) == 1                     # more than SS_MERGE_MAX_RUNS
    assert call(3, step=8) == 1              # sample step out of range
    assert call(3, step=1 << 17) == 1
    assert call(3, chars=None) == 1          # NULL chars with strings to merge
    assert call(3, out=None) == 1            # NULL output
    runs[1].reserved = 1
    assert call(3) == 1
    runs[1].reserved = 0
    runs[2].perm = None
    assert call(3) == 1                      # NULL run with n > 0
    runs[2].perm = 4096
    empty = (ss.RunDesc * 2)()
    assert lib.ss_merge(None, None, 0, empty, 2, 0, None, None, None, 0, None) == 0  # nothing to merge
    big = (ss.RunDesc * 2)()
    for r in big:
        r.perm = r.lcp = 4096
        r.n = 0x80000000
    assert lib.ss_merge(dummy, dummy, 0, big, 2, 0, dummy, None, None, 0, None) == 4
    # misaligned or short caller workspace
    assert lib.ss_merge(dummy, dummy, 0, runs, 3, 16, dummy, None, ctypes.c_void_p(4096 + 8), 1 << 20, None) == 1
    assert lib.ss_merge(dummy, dummy, 0, runs, 3, 16, dummy, None, ctypes.c_void_p(4096), 1, None) == 1
    if not _has_gpu():
        assert call(3) == 7


def test_merge_workspace_size(lib):
    runs = (ss.RunDesc * 3)()
    for r, n in zip(runs, (1000, 50, 3000)):
        r.perm = r.lcp = 4096
        r.n = n
    al = lambda x: (x + 255) // 256 * 256  # noqa: E731
    total = 4050
    # two 32-byte record buffers, the sample cuts of a round, the piece counter
    for step in (64, 4096):
        want = 2 * al(total * 32) + al((total // step + 3 + 1) * 4) + 256
        assert lib.ss_merge_workspace_size(runs, 3, step) == want
    assert lib.ss_merge_workspace_size(runs, 1, 0) == 256   # one run: a copy
    assert lib.ss_merge_workspace_size(runs, 0, 0) == 0


def test_suffix_array_argument_checks(lib):
    dummy = ctypes.c_void_p(4096)
    assert lib.ss_suffix_array(None, 0, None, None, 0, None) == 0          # empty text
    assert lib.ss_suffix_array(None, 10, dummy, None, 0, None) == 1        # NULL text
    assert lib.ss_suffix_array(dummy, 10, None, None, 0, None) == 1        # NULL output
    assert lib.ss_suffix_array(dummy, 1 << 32, dummy, None, 0, None) == 4  # too long
    assert lib.ss_suffix_array(dummy, 10, dummy, None, (1 << 20) + 1, None) == 1
    if not _has_gpu():
        assert lib.ss_suffix_array(dummy, 10, dummy, None, 0, None) == 7


def test_sort_dna_argument_checks(lib):
    o = ss.make_options()
    dummy = ctypes.c_void_p(4096)
    assert lib.ss_sort_dna(None, 0, None, 0, None, None, ctypes.byref(o), None) == 0          # n = 0
    assert lib.ss_sort_dna(dummy, 100, dummy, 1 << 32, dummy, None, ctypes.byref(o), None) == 4
    assert lib.ss_sort_dna(None, 100, dummy, 5, dummy, None, ctypes.byref(o), None) == 1      # NULL chars
    assert lib.ss_sort_dna(dummy, 0, dummy, 5, dummy, None, ctypes.byref(o), None) == 1       # no characters
    assert lib.ss_sort_dna(dummy, 100, dummy, 5, None, None, ctypes.byref(o), None) == 1      # NULL output
    bad = ss.make_options(small_cutoff=32)
    assert lib.ss_sort_dna(dummy, 100, dummy, 5, dummy, None, ctypes.byref(bad), None) == 1
    if not _has_gpu():
        assert lib.ss_sort_dna(dummy, 100, dummy, 5, dummy, None, ctypes.byref(o), None) == 7


def test_sort_host_argument_checks(lib):
    o = ss.make_options()
    dummy = ctypes.c_void_p(4096)
    assert lib.ss_sort_host(None, 0, None, 0, None, None, ctypes.byref(o), None) == 0            # n = 0
    assert lib.ss_sort_host(dummy, 100, dummy, 1 << 32, dummy, None, ctypes.byref(o), None) == 4
    assert lib.ss_sort_host(None, 100, dummy, 5, dummy, None, ctypes.byref(o), None) == 1        # NULL chars
    assert lib.ss_sort_host(dummy, 0, dummy, 5, dummy, None, ctypes.byref(o), None) == 1         # no characters
    assert lib.ss_sort_host(dummy, 100, None, 5, dummy, None, ctypes.byref(o), None) == 1        # NULL offsets
    assert lib.ss_sort_host(dummy, 100, dummy, 5, None, None, ctypes.byref(o), None) == 1        # NULL output
    for parts in (3, 5, 32):  # host_parts: a power of two up to 16
        bad = ss.make_options(host_parts=parts)
        assert lib.ss_sort_host(dummy, 100, dummy, 5, dummy, None, ctypes.byref(bad), None) == 1, parts
    if not _has_gpu():
        good = ss.make_options(host_parts=4)
        assert lib.ss_sort_host(dummy, 100, dummy, 5, dummy, None, ctypes.byref(good), None) == 7
