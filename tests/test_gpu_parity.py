"""Bit-exact parity of the CUDA sort (through the C-ABI) with the CPU oracle."""
import numpy as np
import pytest

import gen
import oracle
from conftest import golden
from gpu_util import assert_parity, from_strings, gpu_sort

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    import paper_1808_00963_gb300 as ss
    assert torch.cuda.is_available()
    ss.build()
    ss.load()


def _text_set(name):
    g = golden(name)
    text = g["text"].encode() + b"\0"
    chars = np.frombuffer(text, np.uint8).copy()
    offsets = np.array([int(x) for x in g["offsets"].split()], np.uint64)
    return gen.StringSet(chars, offsets, int(g["max_len"]), name), g


@pytest.mark.parametrize("name", ["fig5_1.txt", "example_8_4.txt", "example_8_11.txt", "fig6_5.txt"])
def test_paper_suffix_examples(name):
    s, g = _text_set(name)
    p, l = gpu_sort(s)
    assert p.tolist() == [int(x) for x in g["perm"].split()]
    if "lcp" in g:
        assert l.tolist() == [int(x) for x in g["lcp"].split()]


def test_word_list_ties():
    words = [w.encode() for w in golden("fig2_3.txt")["words"].split()]
    rng = np.random.default_rng(3)
    for _ in range(5):
        order = rng.permutation(len(words))
        s = from_strings([words[i] for i in order])
        p, l = gpu_sort(s)
        assert_parity(s, p, l)


def test_tiny_and_degenerate():
    for strs in ([b"x"], [b"", b""], [b"b", b"a"], [b"a", b"a"], [b""] * 50, [b"same"] * 40,
                 [b"ab", b"a", b"", b"abc", b"ab"], [bytes([255, 1]), bytes([1, 255]), bytes([128]), bytes([127])]):
        s = from_strings(strs)
        p, l = gpu_sort(s)
        assert_parity(s, p, l)


def test_empty_set():
    s = from_strings([])
    s.offsets = s.offsets[:0]
    p, l = gpu_sort(s)
    assert p.size == 0 and l.size == 0


@pytest.mark.parametrize("n", [33, 100, 3000])
def test_long_common_prefix(n):
    rng = np.random.default_rng(n)
    pre = bytes(rng.integers(97, 123, size=600).astype(np.uint8))
    strs = [pre + bytes(rng.integers(97, 99, size=int(rng.integers(0, 20))).astype(np.uint8)) for _ in range(n)]
    strs[::7] = [pre] * len(strs[::7])
    s = from_strings(strs)
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


@pytest.mark.parametrize("cap", [0, 100, 130])
def test_deep_runs_in_small_subsets(cap):
    """Many small subsets whose runs share 70 to 400 more characters, mixed
    with ones settled after one look-ahead: the warp pass that defers deep runs
    and the pass that finishes them, including runs that end inside, before or
    after a cap."""
    rng = np.random.default_rng(cap + 11)
    strs = []
    for g in range(3000):
        stem = bytes(rng.integers(97, 123, size=6).astype(np.uint8))
        deep = g % 3 != 0
        shared = bytes(rng.integers(97, 100, size=int(rng.integers(70, 400)) if deep else 3).astype(np.uint8))
        for _ in range(int(rng.integers(2, 9))):
            tail = bytes(rng.integers(97, 100, size=int(rng.integers(0, 4))).astype(np.uint8))
            strs.append(stem + shared + tail)
    order = rng.permutation(len(strs))
    s = from_strings([strs[i] for i in order], max_len=cap)
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


@pytest.mark.parametrize("cap", [1, 7, 8, 9, 16, 500])
def test_caps(cap):
    s = gen.random_set(5000, 11, 0, 40, ord("a"), ord("c"))
    s.max_len = cap
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


def test_high_bytes_unsigned():
    s = gen.random_set(20000, 12, 0, 12, 1, 255)
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


def test_last_string_at_buffer_end():
    strs = [b"zzzzzzzzzzzzz", b"zzzzzzzzzzzzy", b"a" * 15]
    s = from_strings(strs)
    assert s.chars[-1] == 0 and s.N == sum(len(x) + 1 for x in strs)
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


SIZES = [2, 3, 31, 32, 33, 63, 64, 65, 1023, 1024, 1025, 2047, 2048, 2049, 4097, 10000, 70000]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", ["random", "binary", "url", "dna"])
def test_sizes(kind, n):
    if kind == "random":
        s = gen.random_set(n, 100 + n)
    elif kind == "binary":
        s = gen.random_set(n, 200 + n, 0, 24, ord("0"), ord("1"))
    elif kind == "url":
        s = gen.url_set(n, 300 + n)
    else:
        s = gen.dna_suffix_set(max(n, 1), 400 + n, nblocks=(n // 20) // 100 if n >= 2000 else 0,
                               blocklen=100)
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


@pytest.mark.parametrize("kind", ["random", "url", "dna"])
@pytest.mark.parametrize("opts", [dict(big_threshold=2048), dict(big_threshold=4096, big_splitters_log2=8),
                                  dict(big_threshold=2048, big_splitters_log2=9, tile_rounds=8),
                                  dict(splitters_log2=8, small_cutoff=64),
                                  dict(splitters_log2=7, small_cutoff=128),
                                  dict(splitters_log2=7, big_threshold=32768),
                                  dict(splitters_log2=10, small_cutoff=4096),
                                  dict(small_cutoff=256, big_threshold=256)])
def test_paths(kind, opts):
    n = 60000
    s = {"random": lambda: gen.random_set(n, 7), "url": lambda: gen.url_set(n, 8),
         "dna": lambda: gen.dna_suffix_set(n, 9, nblocks=30, blocklen=100)}[kind]()
    p, l = gpu_sort(s, **opts)
    assert_parity(s, p, l)


def test_without_lcp():
    s = gen.url_set(30000, 5)
    p, l = gpu_sort(s, with_lcp=False)
    assert l is None
    want, _ = oracle.sort(s.chars, s.offsets)
    assert np.array_equal(p, want)


def test_deterministic():
    s = gen.url_set(200000, 6)
    a = gpu_sort(s)
    b = gpu_sort(s, seed=12345)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_config1_full():
    s = gen.config1()
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


def test_config3_reduced():
    s = gen.dna_suffix_set(300_000, 3)
    p, l = gpu_sort(s)
    assert_parity(s, p, l)


def test_url_1m_exact():
    s = gen.url_set(1_000_000, 2)
    p, l = gpu_sort(s)
    assert_parity(s, p, l, exact_limit=2_000_000)


def _tuned(kind):
    from paper_1808_00963_gb300 import tune
    return {k: v for k, v in tune.options_for(kind).items() if v}


@pytest.mark.slow
@pytest.mark.parametrize("options", ["defaults", "tuned"])
def test_config3_full(options):
    """All 4M suffixes, with the compiled defaults and with the options the
    autotuner table gives the bench for this workload class."""
    s = gen.config3()
    p, l = gpu_sort(s, **(_tuned("dna") if options == "tuned" else {}))
    assert_parity(s, p, l)


@pytest.mark.slow
@pytest.mark.parametrize("options", ["defaults", "tuned"])
def test_config2_full(options):
    s = gen.config2()
    p, l = gpu_sort(s, **(_tuned("url") if options == "tuned" else {}))
    assert_parity(s, p, l)
    # sampled exact ranks: the oracle's order restricted to a random sample of
    # strings is the order of those strings in the GPU permutation
    rng = np.random.default_rng(0)
    pos = np.sort(rng.choice(s.n, 2000, replace=False))
    sub = p[pos]
    sample = gen.StringSet(s.chars, s.offsets[np.sort(sub)], 0)
    sp, sl = oracle.sort(sample.chars, sample.offsets)
    assert np.array_equal(np.sort(sub)[sp], sub)


def _prefix_sets():
    rng = np.random.default_rng(44)

    def tails(n, lo, hi, alpha=b"abc"):
        a = np.frombuffer(alpha, np.uint8)
        return [bytes(a[rng.integers(0, len(a), int(rng.integers(lo, hi + 1)))]) for _ in range(n)]

    pre = bytes(rng.integers(97, 123, 45).astype(np.uint8))
    sets = {}
    sets["long_prefix"] = [pre + t for t in tails(50_000, 0, 10)]
    sets["short_prefix_dups"] = [pre[:12] + t for t in tails(30_000, 0, 2)]
    sets["outlier_first"] = [b"zzzzzzzzzz"] + [pre + t for t in tails(30_000, 1, 6)]
    groups = [bytes(rng.integers(97, 123, int(rng.integers(9, 60))).astype(np.uint8)) for _ in range(5)]
    sets["hosts"] = [groups[int(rng.integers(0, 5))] + b"/" + t for t in tails(60_000, 0, 12, b"abcdefgh")]
    sets["prefix_ends"] = [pre[:int(rng.integers(8, 45))] for _ in range(20_000)]  # prefixes of one string
    pre300 = bytes(rng.integers(97, 123, 300).astype(np.uint8))
    sets["prefix300"] = [pre300 + t for t in tails(20_000, 0, 6)]  # several jumps in a row
    sets["identical150"] = [pre300[:150]] * 12_000 + [pre300[:149]] * 50
    # groups of 1500..6000 strings (subsets of the work queue) sharing 20..200
    # more characters within the group
    grp = []
    for _ in range(16):
        head = bytes(rng.integers(97, 123, 6).astype(np.uint8))
        shared = bytes(rng.integers(97, 123, int(rng.integers(20, 200))).astype(np.uint8))
        grp += [head + shared + t for t in tails(int(rng.integers(1500, 6000)), 0, 5)]
    sets["queue_groups"] = grp
    return sets


PREFIX_SETS = _prefix_sets()


@pytest.mark.parametrize("cap", [0, 20, 40])
@pytest.mark.parametrize("opts", [dict(big_threshold=2048), dict(big_threshold=4096, classifier=2), dict(),
                                  dict(big_threshold=1 << 30)])
@pytest.mark.parametrize("name", sorted(PREFIX_SETS))
def test_subsets_with_long_common_prefixes(name, opts, cap):
    """Subsets whose strings share a long prefix, where a step jumps over the
    subset's common prefix (up to 64 characters at a time) instead of walking
    it 8 or 16 characters per step, against the oracle: multi-block subsets
    whose whole sample is one key, and (big_threshold 2^30: every subset in
    the work queue) subsets that fall whole into one equality bucket;
    prefixes of 12 to 300 characters, identical strings, strings ending
    inside the prefix, caps inside it, a first member that differs (no jump),
    several hosts, groups of queue-sized subsets."""
    s = from_strings(PREFIX_SETS[name], max_len=cap)
    p, l = gpu_sort(s, **opts)
    assert_parity(s, p, l)


def test_offsets_above_4gib():
    """Strings beyond byte 2^32 of the character buffer.  A record keeps only
    the low 32 bits of its string's offset, so a set with larger offsets takes
    them from the offset array; here mixed with strings below 2^32, and with
    every string of the lower part repeated above (ties across the boundary),
    uncapped and capped."""
    import torch

    import paper_1808_00963_gb300 as ss
    base = gen.url_set(60_000, 21)
    hi = (1 << 32) + 4096 + 3  # an unaligned start above 2^32
    chars = np.zeros(hi + base.N + 64, np.uint8)
    chars[:base.N] = base.chars
    chars[hi:hi + base.N] = base.chars
    offsets = np.concatenate([base.offsets[:30_000], base.offsets + np.uint64(hi)])
    dchars = torch.from_numpy(chars).cuda()
    doffs = torch.from_numpy(offsets.view(np.int64)).cuda()
    for cap in (0, 30):
        perm, lcp = ss.sort(dchars, doffs, max_len=cap)
        torch.cuda.synchronize()
        s = gen.StringSet(chars, offsets, cap)
        assert_parity(s, perm.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32))
    del dchars, doffs
    torch.cuda.empty_cache()


def test_sort_host_matches_device():
    import paper_1808_00963_gb300 as ss
    s = gen.url_set(100000, 9)
    p, l = ss.sort_host(s.chars, s.offsets.view(np.int64))
    assert_parity(s, p, l)
