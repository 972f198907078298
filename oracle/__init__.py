"""CPU oracle for the string sort: TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline``
/ ``--impl reference`` legs may import this package.  The library's sorting
path never calls it and shares no code with it.

The arithmetic lives in ``ss_oracle.c`` (plain C, the definitions of Section
2.1, the compare loop of Algorithm 4.2, Lemma 2.1, the distinguishing
characters of Section 4.3.4, and the K-way merge of Section 4.3.2 both as its
definition and as Algorithm 4.5's LCP-aware tournament tree); this module
compiles it
with gcc and wraps it with ctypes.  Every function here has a parity pin in
``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ss_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libss_oracle.so")
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH, defines=()) -> str:
    """Compile the oracle C source into a shared library (gcc -O2)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(out))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *[f"-D{d}" for d in defines], src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    u64, u32, i64, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
    lib.oracle_sort.argtypes = [vp, vp, u64, u32, vp, vp]
    lib.oracle_sort.restype = ctypes.c_int
    lib.oracle_lcp_array.argtypes = [vp, vp, u64, u32, vp, vp]
    lib.oracle_lcp_array.restype = None
    lib.oracle_check.argtypes = [vp, vp, u64, u32, vp, vp]
    lib.oracle_check.restype = i64
    lib.oracle_dl.argtypes = [vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.oracle_dl.restype = None
    lib.oracle_cache.argtypes = [vp, vp, u64, u64, u32]
    lib.oracle_cache.restype = u64
    lib.oracle_bucket.argtypes = [u64, vp, u32]
    lib.oracle_bucket.restype = u32
    lib.oracle_tree.argtypes = [vp, u32, vp]
    lib.oracle_tree.restype = None
    lib.oracle_distinguishing.argtypes = [vp, vp, u64, u32, vp, vp, vp, vp]
    lib.oracle_distinguishing.restype = None
    lib.oracle_level_to_pre.argtypes = [u32, u32]
    lib.oracle_level_to_pre.restype = u32
    lib.oracle_pre_to_level.argtypes = [u32, u32]
    lib.oracle_pre_to_level.restype = u32
    lib.oracle_merge.argtypes = [vp, vp, u32, vp, u64, vp, vp]
    lib.oracle_merge.restype = ctypes.c_int
    lib.oracle_lcp_merge.argtypes = [vp, vp, u32, u32, vp, vp, vp, vp, vp, ctypes.POINTER(u64)]
    lib.oracle_lcp_merge.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load the oracle library (building it if needed).  ``path`` loads another
    build of the same source (used by the mutation tests)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _arrs(chars, offsets):
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    if chars.size == 0:
        chars = np.zeros(1, np.uint8)
    return chars, offsets


def sort(chars, offsets, max_len: int = 0, lib=None):
    """Sorted order (uint32[n], ties by index) and LCP array (uint32[n], lcp[0] = 0)."""
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    n = offsets.shape[0]
    perm = np.empty(n, np.uint32)
    lcp = np.empty(n, np.uint32)
    rc = lib.oracle_sort(chars.ctypes.data, offsets.ctypes.data, n, max_len, perm.ctypes.data,
                         lcp.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_sort failed")
    return perm, lcp


def lcp_array(chars, offsets, perm, max_len: int = 0, lib=None):
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    lcp = np.empty(perm.shape[0], np.uint32)
    lib.oracle_lcp_array(chars.ctypes.data, offsets.ctypes.data, perm.shape[0], max_len,
                         perm.ctypes.data, lcp.ctypes.data)
    return lcp


def check(chars, offsets, perm, lcp=None, max_len: int = 0, lib=None) -> int:
    """-1 if (perm, lcp) is the unique correct result, else the first bad position."""
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    if perm.shape[0] != offsets.shape[0]:
        return 0
    lp = None
    if lcp is not None:
        lcp = np.ascontiguousarray(lcp, dtype=np.uint32)
        lp = lcp.ctypes.data
    return int(lib.oracle_check(chars.ctypes.data, offsets.ctypes.data, perm.shape[0], max_len,
                                perm.ctypes.data, lp))


def dl(lcp, lib=None):
    """(D, L) of a sorted set from its LCP array (Lemma 2.1)."""
    lib = lib or load()
    lcp = np.ascontiguousarray(lcp, dtype=np.uint32)
    D, L = ctypes.c_uint64(0), ctypes.c_uint64(0)
    lib.oracle_dl(lcp.ctypes.data, lcp.shape[0], ctypes.byref(D), ctypes.byref(L))
    return int(D.value), int(L.value)


def cache(chars, offsets, i: int, h: int, max_len: int = 0, lib=None) -> int:
    """chars_h(s_i): 8 characters at depth h, first character most significant."""
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    return int(lib.oracle_cache(chars.ctypes.data, offsets.ctypes.data, i, h, max_len))


def bucket(c: int, x, lib=None) -> int:
    """Bucket index (0..2v) of key c for sorted splitters x (equality buckets odd)."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.uint64)
    return int(lib.oracle_bucket(c, x.ctypes.data if x.size else None, x.shape[0]))


def tree(x, lib=None):
    """Level-order splitter tree t[1..v] (t[0] unused) for sorted splitters x."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.uint64)
    t = np.zeros(x.shape[0] + 1, np.uint64)
    lib.oracle_tree(x.ctypes.data, x.shape[0], t.ctypes.data)
    return t


def distinguishing(chars, offsets, perm, lcp, max_len: int = 0, lib=None):
    """(c^, d): distinguishing character and distinguishing-prefix length of
    each sorted string (Section 4.3.4, Lemma 2.1)."""
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    lcp = np.ascontiguousarray(lcp, dtype=np.uint32)
    n = perm.shape[0]
    dchar = np.empty(n, np.uint8)
    dpre = np.empty(n, np.uint32)
    lib.oracle_distinguishing(chars.ctypes.data, offsets.ctypes.data, n, max_len, perm.ctypes.data,
                              lcp.ctypes.data, dchar.ctypes.data, dpre.ctypes.data)
    return dchar, dpre


def level_to_pre(l: int, w: int, lib=None) -> int:
    """Lemma 4.1 (i): one-based level-order index -> pre-order index."""
    return int((lib or load()).oracle_level_to_pre(l, w))


def pre_to_level(p: int, w: int, lib=None) -> int:
    """Lemma 4.1 (ii): one-based pre-order index -> level-order index."""
    return int((lib or load()).oracle_pre_to_level(p, w))


def merge(chars, offsets, runs, max_len: int = 0, lib=None):
    """Merged order and LCP array of K sorted runs (sequences of string
    indices): by definition the union of the runs in string order, ties by
    index (Section 4.3.2)."""
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    idx = np.ascontiguousarray(np.concatenate([np.asarray(r, np.uint32) for r in runs])
                               if len(runs) else np.zeros(0, np.uint32), dtype=np.uint32)
    n = idx.shape[0]
    perm = np.empty(n, np.uint32)
    lcp = np.empty(n, np.uint32)
    if lib.oracle_merge(chars.ctypes.data, offsets.ctypes.data, max_len, idx.ctypes.data, n,
                        perm.ctypes.data, lcp.ctypes.data) != 0:
        raise ValueError("oracle_merge failed")
    return perm, lcp


def lcp_merge(chars, offsets, runs, max_len: int = 0, lib=None):
    """The same merge by the LCP-aware tournament tree of Algorithm 4.5 with
    one character per comparison.  ``runs`` is a list of (perm, lcp) pairs
    (each run sorted, lcp its LCP array).  Returns (perm, lcp, character
    comparisons)."""
    lib = lib or load()
    chars, offsets = _arrs(chars, offsets)
    K = len(runs)
    sizes = [len(r[0]) for r in runs]
    if any(len(r[1]) != len(r[0]) for r in runs):
        raise ValueError("each run needs one LCP entry per string")
    start = np.zeros(K + 1, np.uint64)
    start[1:] = np.cumsum(sizes) if K else []
    cat = lambda xs: np.ascontiguousarray(np.concatenate([np.asarray(x, np.uint32) for x in xs])  # noqa: E731
                                          if sum(sizes) else np.zeros(1, np.uint32), dtype=np.uint32)
    idx = cat([r[0] for r in runs])
    rl = cat([r[1] for r in runs])
    n = int(sum(sizes))
    perm = np.empty(max(n, 1), np.uint32)
    lcp = np.empty(max(n, 1), np.uint32)
    cmps = ctypes.c_uint64(0)
    if lib.oracle_lcp_merge(chars.ctypes.data, offsets.ctypes.data, max_len, K, start.ctypes.data,
                            idx.ctypes.data, rl.ctypes.data, perm.ctypes.data, lcp.ctypes.data,
                            ctypes.byref(cmps)) != 0:
        raise ValueError("oracle_lcp_merge failed")
    return perm[:n], lcp[:n], int(cmps.value)


def h_names(chars, offsets, h: int, lib=None):
    """Section 8.2.1: the h-name of every string (the smallest rank of its
    group under the order limited to the first h characters), i.e. the
    inverse h-suffix array ISA^h when the strings are the suffixes of a text.
    By definition: the position, in the sort capped at h, of the first string
    whose capped prefix equals its own."""
    perm, lcp = sort(chars, offsets, h, lib=lib)
    n = perm.shape[0]
    names = np.empty(n, np.uint32)
    start = 0
    for j in range(n):
        if j == 0 or not _capped_equal(chars, offsets, perm[j - 1], perm[j], h):
            start = j
        names[perm[j]] = start
    return names


def _capped_equal(chars, offsets, a, b, h):
    """The first h characters of strings a and b agree, terminators included."""
    oa, ob = int(offsets[a]), int(offsets[b])
    for k in range(h):
        ca, cb = int(chars[oa + k]), int(chars[ob + k])
        if ca != cb:
            return False
        if ca == 0:
            return True
    return True


def suffix_array(text: bytes, lib=None):
    """Suffix array and LCP array of a text (its n non-empty suffixes), by
    definition: the sort of all suffixes."""
    chars = np.frombuffer(bytes(text) + b"\0", np.uint8).copy()
    offsets = np.arange(len(text), dtype=np.uint64)
    return sort(chars, offsets, 0, lib=lib)


def from_strings(strs, max_len: int = 0):
    """Helper for small fixtures: list of bytes -> (chars, offsets)."""
    buf = bytearray()
    offs = []
    for s in strs:
        offs.append(len(buf))
        buf += bytes(s) + b"\0"
    return np.frombuffer(bytes(buf) or b"\0", np.uint8).copy(), np.array(offs, np.uint64)
