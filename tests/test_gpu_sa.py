"""Suffix array construction by prefix doubling on top of the string sort
(Section 8.2) against the oracle's definition (the sort of all suffixes),
element by element, on the paper's printed examples and on texts whose
longest repeats force many doubling rounds."""
import numpy as np
import pytest

import gen
import oracle
from conftest import golden

pytestmark = pytest.mark.gpu


def gpu_sa(text: bytes, initial_depth=0, with_lcp=True):
    import torch

    import paper_1808_00963_gb300 as ss
    t = torch.from_numpy(np.frombuffer(text + b"\0", np.uint8).copy()).cuda()
    sa, lcp = ss.suffix_array(t, len(text), with_lcp=with_lcp, initial_depth=initial_depth)
    torch.cuda.synchronize()
    return sa.cpu().numpy().view(np.uint32), (lcp.cpu().numpy().view(np.uint32) if lcp is not None else None)


def fibonacci(n):
    a, b = b"a", b"ab"
    while len(b) < n:
        a, b = b, b + a
    return b[:n]


def texts():
    rng = np.random.default_rng(17)
    dna = gen.dna_suffix_set(150_000, 19, nblocks=20, blocklen=700)
    return {
        "random_abc": bytes(rng.integers(ord("a"), ord("d"), 200_000).astype(np.uint8)),
        "bytes_1_255": bytes(rng.integers(1, 256, 50_000).astype(np.uint8)),
        "dna_repeats": bytes(dna.chars[:dna.n]),
        "unary": b"a" * 3000,
        "periodic": b"abcab" * 900,
        "fibonacci": fibonacci(4000),
        "one_char": b"z",
        "two_chars": b"zz",
    }


TEXTS = texts()


@pytest.mark.parametrize("depth", [0, 1, 3, 8, 300])
@pytest.mark.parametrize("name", sorted(TEXTS))
def test_suffix_array_matches_oracle(name, depth):
    text = TEXTS[name]
    sa, lcp = gpu_sa(text, initial_depth=depth)
    want_sa, want_lcp = oracle.suffix_array(text)
    bad = np.nonzero(sa != want_sa)[0]
    assert bad.size == 0, f"sa differs at {bad[:10]} (of {bad.size}); n={len(text)}"
    bad = np.nonzero(lcp != want_lcp)[0]
    assert bad.size == 0, f"lcp differs at {bad[:10]}: got {lcp[bad[:5]]} want {want_lcp[bad[:5]]}"


@pytest.mark.parametrize("fixture", ["fig5_1.txt", "example_8_4.txt", "example_8_11.txt", "fig8_1.txt"])
def test_suffix_array_paper_examples(fixture):
    """The suffix arrays the paper prints (the empty suffix, which the paper
    lists first as '$', is not listed here)."""
    g = golden(fixture)
    text = g["text"].encode()
    perm = [int(x) for x in g["perm"].split()]
    want = [p for p in perm if p != len(text)]
    for depth in (0, 1, 2):
        sa, lcp = gpu_sa(text, initial_depth=depth)
        assert sa.tolist() == want
        if "lcp" in g:
            full = [int(x) for x in g["lcp"].split()]
            if perm[0] == len(text):  # drop the empty suffix's entry; the next entry becomes 0
                full = [0] + full[2:]
            assert lcp.tolist() == full


def test_suffix_array_without_lcp():
    text = TEXTS["dna_repeats"][:40_000]
    sa, lcp = gpu_sa(text, initial_depth=4, with_lcp=False)
    assert lcp is None
    assert np.array_equal(sa, oracle.suffix_array(text)[0])


@pytest.mark.slow
def test_suffix_array_full_size_dna():
    """All 4M suffixes of the DNA-like text of the suffix-sorting workload,
    uncapped: checked by the oracle's checker (a permutation, in order, exact
    LCPs)."""
    s = gen.config3()
    text = bytes(s.chars[:s.n])
    sa, lcp = gpu_sa(text)
    chars = np.frombuffer(text + b"\0", np.uint8).copy()
    assert oracle.check(chars, np.arange(len(text), dtype=np.uint64), sa, lcp, 0) == -1


REPEAT_TEXTS = {
    "period997": bytes(np.tile(np.random.default_rng(31).integers(97, 100, 997).astype(np.uint8), 20)),
    "unary": b"a" * 12_000,
    "fibonacci": fibonacci(15_000),
}
_REPEAT_WANT = {}


@pytest.mark.parametrize("depth", [0, 8, 1000])
@pytest.mark.parametrize("name", sorted(REPEAT_TEXTS))
def test_long_repeats_exact(name, depth):
    """Periodic texts whose LCPs run far beyond the first sort's depth (the
    LCPs above it come from the rounds' names), element by element."""
    text = REPEAT_TEXTS[name]
    if name not in _REPEAT_WANT:
        _REPEAT_WANT[name] = oracle.suffix_array(text)
    want_sa, want_lcp = _REPEAT_WANT[name]
    sa, lcp = gpu_sa(text, initial_depth=depth)
    assert np.array_equal(sa, want_sa)
    assert np.array_equal(lcp, want_lcp)


def test_unary_closed_form():
    """a^n: the suffixes in order of length, shortest first, and LCP[j] = j
    (the closed form, at a size whose LCP sum no direct comparison could
    afford: 2^21 characters, 21 doubling rounds)."""
    n = 1 << 21
    sa, lcp = gpu_sa(b"a" * n)
    assert np.array_equal(sa, np.arange(n - 1, -1, -1, dtype=np.uint32))
    assert np.array_equal(lcp, np.arange(n, dtype=np.uint32))


def test_periodic_large_sampled():
    """A 2M-character text of one 40000-character block repeated: adjacent
    suffix pairs checked one by one on a sample (order and exact LCP by
    direct comparison), plus the permutation property."""
    rng = np.random.default_rng(32)
    text = bytes(np.tile(rng.integers(97, 101, 40_000).astype(np.uint8), 50))
    n = len(text)
    sa, lcp = gpu_sa(text)
    assert np.array_equal(np.sort(sa), np.arange(n, dtype=np.uint32))
    tb = np.frombuffer(text, np.uint8)
    for j in rng.choice(np.arange(1, n), 300, replace=False):
        a, b, h = int(sa[j - 1]), int(sa[j]), int(lcp[j])
        m = min(n - a, n - b)
        assert h <= m and np.array_equal(tb[a:a + h], tb[b:b + h])
        if h < m:
            assert tb[a + h] < tb[b + h]
        else:
            assert n - a < n - b  # a proper prefix comes first
