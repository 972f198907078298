"""Seeded synthetic inputs for the string sort (shared by tests, bench and the
serving loop).

Strings are laid out as the sort's interface expects (Section 2.1): one uint8
buffer of NUL-terminated strings plus uint64 start offsets.  Generation is done
by the small C library ``ss_gen.c`` next to this file, which draws every random
number from a counter-based generator, so a given (config, seed) gives the same
bytes on x86 and on Arm, for any thread count.

Nothing here sorts or compares strings: this module is input plumbing only.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ss_gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libss_gen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ss_gen.c into _build/libss_gen.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, u32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        vp = ctypes.c_void_p
        lib.gen_random_size.argtypes = [u64, u64, u32, u32]
        lib.gen_random_size.restype = u64
        lib.gen_random_fill.argtypes = [u64, u64, u32, u32, u32, u32, vp, vp]
        lib.gen_random_fill.restype = None
        lib.gen_url_size.argtypes = [u64, u64, dbl]
        lib.gen_url_size.restype = u64
        lib.gen_url_fill.argtypes = [u64, u64, dbl, vp, vp]
        lib.gen_url_fill.restype = None
        lib.gen_dna_text.argtypes = [u64, u64, u32, u32, vp]
        lib.gen_dna_text.restype = ctypes.c_int
        lib.gen_rnd.argtypes = [u64, u64, u64]
        lib.gen_rnd.restype = u64
        lib.gen_unit.argtypes = [u64, u64, u64]
        lib.gen_unit.restype = dbl
        _lib = lib
    return _lib


@dataclass
class StringSet:
    """A string set in the sort's input layout.

    chars   : uint8[N]  NUL-terminated strings (may overlap, e.g. suffixes)
    offsets : uint64[n] start of string i in ``chars``
    max_len : 0 = strings end at their NUL; else string i also ends after
              max_len bytes (bytes beyond the cap count as the terminator)
    """
    chars: np.ndarray
    offsets: np.ndarray
    max_len: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0])

    @property
    def N(self) -> int:
        return int(self.chars.shape[0])


def random_set(n: int, seed: int, lmin: int = 8, lmax: int = 32,
               alo: int = ord("a"), ahi: int = ord("z")) -> StringSet:
    """n strings, length ~ U{lmin..lmax}, bytes ~ U{alo..ahi}, back to back."""
    lib = _load()
    assert 1 <= alo <= ahi <= 255 and 0 <= lmin <= lmax
    N = lib.gen_random_size(n, seed, lmin, lmax)
    chars = np.empty(max(N, 1), dtype=np.uint8)
    offsets = np.empty(n, dtype=np.uint64)
    lib.gen_random_fill(n, seed, lmin, lmax, alo, ahi, chars.ctypes.data, offsets.ctypes.data)
    return StringSet(chars[:N] if N else chars[:0], offsets, 0, f"random(n={n},seed={seed})",
                     {"kind": "random", "n": n, "seed": seed})


def url_set(n: int, seed: int, zipf_s: float = 1.1) -> StringSet:
    """n URL-like strings: http(s):// + Zipf(zipf_s) host from 2000 seeded
    host names + 1..6 path segments of 3..12 [a-z0-9]."""
    lib = _load()
    N = lib.gen_url_size(n, seed, zipf_s)
    chars = np.empty(max(N, 1), dtype=np.uint8)
    offsets = np.empty(n, dtype=np.uint64)
    lib.gen_url_fill(n, seed, zipf_s, chars.ctypes.data, offsets.ctypes.data)
    return StringSet(chars[:N] if N else chars[:0], offsets, 0, f"url(n={n},seed={seed})",
                     {"kind": "url", "n": n, "seed": seed})


def dna_suffix_set(text_len: int, seed: int, nblocks: int | None = None,
                   blocklen: int = 1000, max_len: int = 500) -> StringSet:
    """All text_len suffixes of a DNA-like text (order-3 Markov + nblocks
    duplicated blocklen-byte windows, 5 % of the text by default), each capped
    at max_len bytes."""
    lib = _load()
    if nblocks is None:
        nblocks = (text_len * 5 // 100) // blocklen
    text = np.empty(text_len + 1, dtype=np.uint8)
    rc = lib.gen_dna_text(text_len, seed, nblocks, blocklen, text.ctypes.data)
    if rc != 0:
        raise ValueError("dna text sizes do not fit")
    offsets = np.arange(text_len, dtype=np.uint64)
    return StringSet(text, offsets, max_len, f"dna(n={text_len},seed={seed})",
                     {"kind": "dna", "n": text_len, "seed": seed, "nblocks": nblocks})


# ---- the five workload configurations -----------------------------------------------

def config1() -> StringSet:
    """100 000 random strings, length 8-32, bytes a-z (seed 1)."""
    return random_set(100_000, 1)


def config2(n: int = 20_000_000) -> StringSet:
    """20 M URL-like strings (seed 2)."""
    return url_set(n, 2)


def config3(text_len: int = 4_000_000) -> StringSet:
    """All 4 M suffixes of a DNA-like text, capped at 500 bytes (seed 3)."""
    return dna_suffix_set(text_len, 3)


def batch_specs(num_sets: int = 4096, seed: int = 4, smin: int = 100, smax: int = 200_000):
    """Sizes and generator kinds of the batched workload: size log-uniform in
    [smin, smax], generator uniform over {random, url, dna}."""
    lib = _load()
    specs = []
    for j in range(num_sets):
        u = lib.gen_unit(seed, 100, j)
        size = int(round(math.exp(math.log(smin) + u * (math.log(smax) - math.log(smin)))))
        size = min(max(size, smin), smax)
        kind = ("random", "url", "dna")[lib.gen_rnd(seed, 101, j) % 3]
        sub_seed = int(lib.gen_rnd(seed, 102, j) >> 1)
        specs.append((kind, size, sub_seed))
    return specs


def make_set(kind: str, size: int, seed: int) -> StringSet:
    if kind == "random":
        return random_set(size, seed)
    if kind == "url":
        return url_set(size, seed)
    if kind == "dna":
        return dna_suffix_set(size, seed)
    raise ValueError(kind)


def batch_sets(num_sets: int = 4096, seed: int = 4, smin: int = 100, smax: int = 200_000):
    """The batched workload: num_sets independent string sets."""
    return [make_set(k, s, sd) for (k, s, sd) in batch_specs(num_sets, seed, smin, smax)]


def trace(num_requests: int, seed: int, rate_per_s: float, smin: int = 1000,
          smax: int = 5_000_000):
    """A Poisson request trace: list of (arrival_s, kind, size, seed) with
    exponential inter-arrival times (mean 1/rate_per_s), log-uniform sizes and
    a uniform mix of the three generators."""
    lib = _load()
    t = 0.0
    out = []
    for j in range(num_requests):
        t += -math.log(lib.gen_unit(seed, 200, j)) / rate_per_s
        u = lib.gen_unit(seed, 201, j)
        size = int(round(math.exp(math.log(smin) + u * (math.log(smax) - math.log(smin)))))
        size = min(max(size, smin), smax)
        kind = ("random", "url", "dna")[lib.gen_rnd(seed, 202, j) % 3]
        out.append((t, kind, size, int(lib.gen_rnd(seed, 203, j) >> 1)))
    return out


def concat(sets):
    """Concatenate string sets into one buffer (offsets rebased per set).
    Returns (chars, offsets, set_char_base, set_first, max_lens)."""
    bases, firsts, ml = [], [], []
    cb, fb = 0, 0
    for s in sets:
        bases.append(cb)
        firsts.append(fb)
        ml.append(s.max_len)
        cb += s.N
        fb += s.n
    chars = np.concatenate([s.chars for s in sets]) if sets else np.zeros(0, np.uint8)
    offsets = np.concatenate([s.offsets for s in sets]) if sets else np.zeros(0, np.uint64)
    return chars, offsets, np.array(bases, np.uint64), np.array(firsts, np.uint64), np.array(ml, np.uint32)
