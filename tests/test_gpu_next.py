"""Extensions of the sort, checked against the oracle: distinguishing
characters and prefixes from its outputs (Section 4.3.4, Lemma 2.1; D = sum of
the prefixes) and the classification variants of Section 4.2.3."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["random", "url", "dna", "binary_caps", "config1"])
def test_distinguishing_matches_oracle(case):
    import torch

    import paper_1808_00963_gb300 as ss
    s = {"random": lambda: gen.random_set(30000, 51, 0, 20, ord("a"), ord("c")),
         "url": lambda: gen.url_set(200000, 52),
         "dna": lambda: gen.dna_suffix_set(200000, 53),
         "binary_caps": lambda: gen.random_set(50000, 54, 0, 30, 1, 2),
         "config1": gen.config1}[case]()
    if case == "binary_caps":
        s.max_len = 9
    chars, offsets = to_device(s)
    perm, lcp = ss.sort(chars, offsets, max_len=s.max_len)
    dchar, dpre, D = ss.distinguishing(chars, offsets, perm, lcp, max_len=s.max_len)
    torch.cuda.synchronize()
    p = perm.cpu().numpy().view(np.uint32)
    l = lcp.cpu().numpy().view(np.uint32)
    want_c, want_d = oracle.distinguishing(s.chars, s.offsets, p, l, s.max_len)
    assert np.array_equal(dchar.cpu().numpy(), want_c)
    assert np.array_equal(dpre.cpu().numpy().view(np.uint32), want_d)
    assert int(D.item()) == oracle.dl(l)[0]


@pytest.mark.parametrize("classifier", [0, 1, 2, 3])
@pytest.mark.parametrize("case", ["binary", "dna", "url", "equal_heavy"])
def test_classifier_variants_same_output(classifier, case):
    """S5-UI, S5-UIC (Lemma 4.1 index map), S5-E (equality at every node) and
    S5-UI entered through a jump table give the oracle's output, on inputs
    whose samples hold many equal caches (duplicate splitters), through both
    the multi-block and single-block steps."""
    from gpu_util import assert_parity, gpu_sort
    s = {"binary": lambda: gen.random_set(80000, 61, 0, 24, ord("0"), ord("1")),
         "dna": lambda: gen.dna_suffix_set(120000, 62, nblocks=20, blocklen=500),
         "url": lambda: gen.url_set(150000, 63),
         "equal_heavy": lambda: gen.random_set(70000, 64, 0, 3, ord("a"), ord("b"))}[case]()
    p, l = gpu_sort(s, classifier=classifier, big_threshold=4096, small_cutoff=256)
    assert_parity(s, p, l)


def acgt_set(n, seed, lmin, lmax):
    """Random strings over A, C, G, T (a..d of the random generator mapped)."""
    s = gen.random_set(n, seed, lmin, lmax, ord("a"), ord("d"))
    table = np.arange(256, dtype=np.uint8)
    table[[ord("a"), ord("b"), ord("c"), ord("d")]] = [ord("A"), ord("C"), ord("G"), ord("T")]
    s.chars = table[s.chars]
    return s


def _dna_case(case):
    if case.startswith("suffixes_cap"):
        cap = int(case[len("suffixes_cap"):])
        s = gen.dna_suffix_set(120_000, 71, nblocks=15, blocklen=600)
        s.max_len = cap
        return s
    if case == "random_short":
        return acgt_set(60_000, 72, 0, 12)
    if case == "random_long":
        return acgt_set(40_000, 73, 30, 90)
    raise ValueError(case)


@pytest.mark.parametrize("opts", [{}, {"big_threshold": 4096, "small_cutoff": 256}, {"classifier": 2}])
@pytest.mark.parametrize("case", ["suffixes_cap500", "suffixes_cap21", "suffixes_cap22", "suffixes_cap1",
                                  "suffixes_cap0", "random_short", "random_long"])
def test_dna_alphabet_matches_oracle(case, opts):
    """Alphabet compression (3-bit codes, 21 characters per key) gives the
    oracle's output: suffix sets with caps on and off a key boundary, long
    repeats, empty and duplicate strings, the multi-block and single-block
    paths."""
    import torch

    import paper_1808_00963_gb300 as ss
    from gpu_util import assert_parity
    s = _dna_case(case)
    chars, offsets = to_device(s)
    perm, lcp = ss.sort(chars, offsets, max_len=s.max_len, dna=True, **opts)
    torch.cuda.synchronize()
    assert_parity(s, perm.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32))


def test_dna_alphabet_rejects_other_bytes():
    import torch

    import paper_1808_00963_gb300 as ss
    s = acgt_set(1000, 74, 1, 10)
    s.chars = s.chars.copy()
    s.chars[int(s.offsets[500])] = ord("N")
    chars, offsets = to_device(s)
    with pytest.raises(ss.SortError) as e:
        ss.sort(chars, offsets, dna=True)
    assert e.value.code == 1
    torch.cuda.synchronize()
