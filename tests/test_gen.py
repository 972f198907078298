"""The seeded input generators: determinism and the configured shapes."""
import numpy as np

import gen


def _strs(s, limit=None):
    out = []
    for o in s.offsets[:limit]:
        o = int(o)
        e = o + int(np.argmax(s.chars[o:] == 0))
        out.append(bytes(s.chars[o:e]))
    return out


def test_deterministic():
    a, b = gen.url_set(5000, 7), gen.url_set(5000, 7)
    assert np.array_equal(a.chars, b.chars) and np.array_equal(a.offsets, b.offsets)
    c = gen.url_set(5000, 8)
    assert not np.array_equal(a.chars[:1000], c.chars[:1000])
    d1, d2 = gen.dna_suffix_set(30000, 3), gen.dna_suffix_set(30000, 3)
    assert np.array_equal(d1.chars, d2.chars)


def test_random_shape():
    s = gen.random_set(20000, 1)
    lens = [len(x) for x in _strs(s)]
    assert min(lens) >= 8 and max(lens) <= 32
    body = s.chars[s.chars != 0]
    assert body.min() >= ord("a") and body.max() <= ord("z")
    assert s.N == sum(lens) + s.n


def test_url_shape():
    s = gen.url_set(20000, 2)
    strs = _strs(s)
    assert all(x.startswith(b"http://") or x.startswith(b"https://") for x in strs)
    mean = s.N / s.n
    assert 55 <= mean <= 65
    # Zipf hosts: the most common host covers a large share
    hosts = {}
    for x in strs:
        h = x.split(b"/")[2]
        hosts[h] = hosts.get(h, 0) + 1
    assert max(hosts.values()) > 0.1 * len(strs)
    assert len(hosts) <= 2000


def test_dna_shape():
    s = gen.dna_suffix_set(100000, 3)
    assert s.n == 100000 and s.N == 100001 and s.max_len == 500
    assert s.chars[-1] == 0
    assert set(np.unique(s.chars[:-1]).tolist()) <= set(b"ACGT")
    assert s.meta["nblocks"] == 5


def test_batch_specs():
    specs = gen.batch_specs(4096, 4)
    sizes = np.array([sz for _, sz, _ in specs])
    assert sizes.min() >= 100 and sizes.max() <= 200000
    kinds = {k for k, _, _ in specs}
    assert kinds == {"random", "url", "dna"}
    assert 15000 < sizes.mean() < 40000
