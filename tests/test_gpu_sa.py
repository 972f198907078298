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
