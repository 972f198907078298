"""Parity pins for the CPU oracle.

Each pin checks the oracle against something other than itself: values the
paper prints for a worked example (tests/golden/), brute force over all n!
orders on tiny inputs, Python's own byte-string ordering (an independent
library sort), closed forms and invariants.  Every pin takes the oracle
library as an argument so that tests/test_oracle_mutants.py can run the same
pins against builds of the oracle with a planted mistake.
"""
from __future__ import annotations

import bisect
import itertools
import os

import numpy as np

import oracle
from conftest import golden


def _strings(chars, offsets, max_len=0):
    out = []
    for o in offsets:
        o = int(o)
        e = o
        while chars[e] != 0 and (max_len == 0 or e - o < max_len):
            e += 1
        out.append(bytes(chars[o:e]))
    return out


def _text_fixture(name):
    g = golden(name)
    text = g["text"].encode() + b"\0"
    chars = np.frombuffer(text, np.uint8).copy()
    offsets = np.array([int(x) for x in g["offsets"].split()], np.uint64)
    perm = [int(x) for x in g["perm"].split()]
    lcp = [int(x) for x in g["lcp"].split()] if "lcp" in g else None
    return chars, offsets, int(g["max_len"]), perm, lcp


def pin_paper_suffix_examples(lib):
    """Figure 5.1, Examples 8.4 and 8.11, Figure 6.5: printed suffix arrays
    (and LCP arrays where printed)."""
    for name in ("fig5_1.txt", "example_8_4.txt", "example_8_11.txt", "fig6_5.txt"):
        chars, offsets, max_len, perm, lcp = _text_fixture(name)
        p, l = oracle.sort(chars, offsets, max_len, lib=lib)
        assert p.tolist() == perm, name
        if lcp is not None:
            assert l.tolist() == lcp, name


def pin_word_list_ties(lib):
    """Figure 2.3: the word list is sorted; the three equal words keep their
    input order whatever order they are given in."""
    words = [w.encode() for w in golden("fig2_3.txt")["words"].split()]
    rng = np.random.default_rng(23)
    for _ in range(20):
        order = rng.permutation(len(words))
        shuffled = [words[i] for i in order]
        chars, offsets = oracle.from_strings(shuffled)
        p, l = oracle.sort(chars, offsets, lib=lib)
        assert [shuffled[i] for i in p] == words
        by = [int(i) for i in p if shuffled[i] == b"by"]
        assert by == sorted(by)
        assert l.tolist()[0] == 0


def pin_lemma_2_1(lib):
    """Lemma 2.1: the printed example (D = 8, L = 2) and n + L <= D <= 2L + n."""
    g = golden("lemma2_1.txt")
    words = [w.encode() for w in g["words"].split()]
    chars, offsets = oracle.from_strings(words)
    p, l = oracle.sort(chars, offsets, lib=lib)
    D, L = oracle.dl(l, lib=lib)
    assert (D, L) == (int(g["D"]), int(g["L"]))
    rng = np.random.default_rng(21)
    for t in range(30):
        n = int(rng.integers(1, 60))
        strs = [bytes(rng.integers(97, 100, size=int(rng.integers(0, 6))).astype(np.uint8)) for _ in range(n)]
        chars, offsets = oracle.from_strings(strs)
        p, l = oracle.sort(chars, offsets, lib=lib)
        D, L = oracle.dl(l, lib=lib)
        assert n + L <= D <= 2 * L + n
        # D counted directly from its definition in the lemma's proof:
        # d_i = 1 + the longer common prefix with either sorted neighbour.
        s = sorted(strs)
        direct = 0
        for i in range(n):
            best = 0
            for j in (i - 1, i + 1):
                if 0 <= j < n:
                    best = max(best, len(os.path.commonprefix([s[i], s[j]])))
            direct += best + 1
        assert D == direct


def _brute_force_order(strs):
    """The unique order that is non-decreasing with ties by index, found by
    trying every permutation (Python compares bytes lexicographically by
    unsigned value, a proper prefix first)."""
    n = len(strs)
    for perm in itertools.permutations(range(n)):
        if all((strs[perm[j - 1]], perm[j - 1]) < (strs[perm[j]], perm[j]) for j in range(1, n)):
            return list(perm)
    raise AssertionError("no order found")


def pin_brute_force(lib):
    """All n! orders, n <= 6, small alphabets incl. bytes >= 128, caps."""
    rng = np.random.default_rng(5)
    alphabets = [[ord("a"), ord("b")], [1, 200, 255], [ord("x")]]
    for t in range(150):
        n = int(rng.integers(1, 7))
        alpha = alphabets[t % 3]
        strs = [bytes(rng.choice(alpha, size=int(rng.integers(0, 5))).astype(np.uint8)) for _ in range(n)]
        if n > 2 and t % 4 == 0:
            strs[-1] = strs[0]
        max_len = [0, 0, 1, 2, 3][t % 5]
        view = [s[:max_len] if max_len else s for s in strs]
        chars, offsets = oracle.from_strings(strs)
        p, l = oracle.sort(chars, offsets, max_len, lib=lib)
        want = _brute_force_order(view)
        assert p.tolist() == want, (strs, max_len)
        lcps = [0] + [len(os.path.commonprefix([view[want[j - 1]], view[want[j]]])) for j in range(1, n)]
        assert l.tolist() == lcps


def pin_library_sort(lib):
    """Python's sorted() on bytes (ties by index) for larger random sets with
    duplicates, empty strings, high bytes and caps."""
    rng = np.random.default_rng(9)
    for t in range(12):
        n = int(rng.integers(100, 3000))
        lo, hi = [(97, 99), (1, 255), (65, 68)][t % 3]
        strs = [bytes(rng.integers(lo, hi + 1, size=int(rng.integers(0, 12))).astype(np.uint8)) for _ in range(n)]
        for k in range(0, n, 17):
            strs[k] = strs[(k * 7) % n]
        max_len = [0, 5, 1, 0][t % 4]
        view = [s[:max_len] if max_len else s for s in strs]
        chars, offsets = oracle.from_strings(strs)
        p, l = oracle.sort(chars, offsets, max_len, lib=lib)
        want = sorted(range(n), key=lambda i: (view[i], i))
        assert p.tolist() == want
        lcps = [0] + [len(os.path.commonprefix([view[want[j - 1]], view[want[j]]])) for j in range(1, n)]
        assert l.tolist() == lcps


def pin_checker(lib):
    """The O(n + D) checker accepts the true result and rejects planted errors."""
    rng = np.random.default_rng(11)
    strs = [bytes(rng.integers(97, 100, size=int(rng.integers(0, 6))).astype(np.uint8)) for _ in range(500)]
    chars, offsets = oracle.from_strings(strs)
    want = sorted(range(len(strs)), key=lambda i: (strs[i], i))
    perm = np.array(want, np.uint32)
    lcp = np.array([0] + [len(os.path.commonprefix([strs[want[j - 1]], strs[want[j]]]))
                          for j in range(1, len(want))], np.uint32)
    assert oracle.check(chars, offsets, perm, lcp, lib=lib) == -1
    bad = perm.copy()
    j = next(j for j in range(1, len(want)) if strs[want[j - 1]] != strs[want[j]])
    bad[j - 1], bad[j] = bad[j], bad[j - 1]
    assert oracle.check(chars, offsets, bad, lcp, lib=lib) != -1
    j = next(j for j in range(1, len(want)) if strs[want[j - 1]] == strs[want[j]])
    bad = perm.copy()
    bad[j - 1], bad[j] = bad[j], bad[j - 1]
    assert oracle.check(chars, offsets, bad, lcp, lib=lib) != -1  # tie order
    badl = lcp.copy()
    badl[len(badl) // 2] += 1
    assert oracle.check(chars, offsets, perm, badl, lib=lib) != -1
    dup = perm.copy()
    dup[3] = dup[4]
    assert oracle.check(chars, offsets, dup, lcp, lib=lib) != -1


def pin_cache(lib):
    """chars_h: the 8-byte window read as a big-endian integer (int.from_bytes)
    with everything at/after the terminator or cap as zero."""
    rng = np.random.default_rng(13)
    strs = [bytes(rng.integers(1, 256, size=int(rng.integers(0, 30))).astype(np.uint8)) for _ in range(200)]
    chars, offsets = oracle.from_strings(strs)
    for i, s in enumerate(strs):
        for cap in (0, 3, 8, 9):
            view = s[:cap] if cap else s
            for h in (0, 1, 5, 8, 13, 40):
                window = (view[h:h + 8] if h <= len(view) else b"").ljust(8, b"\0")
                assert oracle.cache(chars, offsets, i, h, cap, lib=lib) == int.from_bytes(window, "big")


def pin_bucket_and_tree(lib):
    """Section 4.2.3: the printed level-order layout for v = 7; a descent of
    that tree with i := 2i + [c > t_i] lands on bisect_left(x, c); and the
    bucket index satisfies the bucket definitions (x_{r-1} < c < x_r for 2r,
    c == x_r for 2r+1)."""
    g = golden("tree_v7.txt")
    v = int(g["v"])
    x = np.array([10 * (k + 1) for k in range(v)], np.uint64)
    t = oracle.tree(x, lib=lib)
    assert [int(z) for z in t[1:]] == [int(x[k]) for k in map(int, g["t_index"].split())]
    rng = np.random.default_rng(17)
    for d in (1, 2, 3, 5, 8):
        v = (1 << d) - 1
        for _ in range(20):
            x = np.sort(rng.integers(0, 50, size=v).astype(np.uint64))
            t = oracle.tree(x, lib=lib)
            xs = [int(z) for z in x]
            for c in rng.integers(0, 52, size=20):
                c = int(c)
                i = 1
                for _lvl in range(d):
                    i = 2 * i + (1 if c > int(t[i]) else 0)
                assert i - (v + 1) == bisect.bisect_left(xs, c)
                b = oracle.bucket(c, x, lib=lib)
                r = b // 2
                if b % 2:
                    assert xs[r] == c
                else:
                    assert (r == 0 or xs[r - 1] < c) and (r == v or c < xs[r])


def pin_distinguishing(lib):
    """Section 4.3.4 / Lemma 2.1: on Lemma 2.1's example the distinguishing
    prefixes are [2, 2, 2, 2] (sum D = 8) and the distinguishing characters
    [a, b, b, b]; on random sets (with caps) the characters equal the byte of
    each sorted string at its LCP with its predecessor (Python slicing), and
    the prefix lengths sum to D."""
    words = [w.encode() for w in golden("lemma2_1.txt")["words"].split()]
    chars, offsets = oracle.from_strings(words)
    p, l = oracle.sort(chars, offsets, lib=lib)
    dc, dp = oracle.distinguishing(chars, offsets, p, l, lib=lib)
    assert dp.tolist() == [2, 2, 2, 2] and bytes(dc.tolist()) == b"abbb"
    rng = np.random.default_rng(31)
    for t in range(20):
        n = int(rng.integers(1, 300))
        strs = [bytes(rng.integers(97, 100, size=int(rng.integers(0, 8))).astype(np.uint8)) for _ in range(n)]
        cap = [0, 3, 5][t % 3]
        view = [s[:cap] if cap else s for s in strs]
        chars, offsets = oracle.from_strings(strs)
        p, l = oracle.sort(chars, offsets, cap, lib=lib)
        dc, dp = oracle.distinguishing(chars, offsets, p, l, cap, lib=lib)
        srt = [view[i] for i in p]
        for j in range(n):
            h = 0 if j == 0 else len(os.path.commonprefix([srt[j - 1], srt[j]]))
            want = srt[j][h] if h < len(srt[j]) else 0
            assert dc[j] == want
        D, _ = oracle.dl(l, lib=lib)
        assert int(dp.astype(np.int64).sum()) == D


def pin_lemma_4_1(lib):
    """Lemma 4.1: the printed example (0101 level-order <-> 0110 pre-order),
    the two maps are inverse, and the pre-order index of every tree vertex is
    the one-based position of its splitter in sorted order (checked against
    the level-order tree t built from the sorted splitters)."""
    g = golden("lemma4_1.txt")
    w = int(g["w"])
    assert oracle.level_to_pre(int(g["level"], 2), w, lib=lib) == int(g["pre"], 2)
    assert oracle.pre_to_level(int(g["pre"], 2), w, lib=lib) == int(g["level"], 2)
    for w in range(1, 11):
        v = (1 << w) - 1
        x = np.arange(1, v + 1, dtype=np.uint64) * 3
        t = oracle.tree(x, lib=lib)
        for l in range(1, v + 1):
            p = oracle.level_to_pre(l, w, lib=lib)
            assert oracle.pre_to_level(p, w, lib=lib) == l
            assert int(t[l]) == int(x[p - 1])


def _py_runs(view, assign, K):
    """Runs sorted by Python's bytes order (ties by index) and their LCP arrays."""
    runs = []
    for k in range(K):
        r = sorted((i for i in range(len(view)) if assign[i] == k), key=lambda i: (view[i], i))
        lc = [0] * min(1, len(r)) + [len(os.path.commonprefix([view[r[j - 1]], view[r[j]]]))
                                     for j in range(1, len(r))]
        runs.append((np.array(r, np.uint32), np.array(lc, np.uint32)))
    return runs


def pin_merge(lib):
    """Section 4.3.2: merging K sorted runs gives Python's sorted() of their
    union (ties by index) with its LCP array, both as the definition and by
    Algorithm 4.5's LCP-aware tournament tree; the tree does at most
    dL + n log2 K + K character comparisons (Theorem 4.7) and needs none for
    a single run.  Runs of every count 1..17 (padded to powers of two), empty
    runs, equal strings in different runs, an index present in two runs, caps."""
    rng = np.random.default_rng(47)
    for t in range(60):
        n = int(rng.integers(0, 400))
        K = int(rng.integers(1, 18))
        lo, hi = [(97, 99), (1, 255), (120, 121)][t % 3]
        strs = [bytes(rng.integers(lo, hi + 1, size=int(rng.integers(0, 9))).astype(np.uint8)) for _ in range(n)]
        for k in range(0, n, 11):
            strs[k] = strs[(k * 5) % n]
        max_len = [0, 0, 3, 1][t % 4]
        view = [s[:max_len] if max_len else s for s in strs]
        assign = rng.integers(0, K, n) if t % 5 else np.minimum(rng.integers(0, 2 * K, n), K - 1)
        runs = _py_runs(view, assign, K)
        if t % 7 == 3 and n > 0:               # one index present in two runs
            extra = _py_runs(view, np.where(np.arange(n) == n // 2, 0, 1), 2)[0]
            runs.append(extra)
        members = sorted((int(i) for r in runs for i in r[0]), key=lambda i: (view[i], i))
        want_l = [0] + [len(os.path.commonprefix([view[members[j - 1]], view[members[j]]]))
                        for j in range(1, len(members))]
        chars, offsets = oracle.from_strings(strs)
        pm, lm = oracle.merge(chars, offsets, [r[0] for r in runs], max_len, lib=lib)
        assert pm.tolist() == members and lm.tolist() == want_l, (t, "definition")
        pk, lk, cmps = oracle.lcp_merge(chars, offsets, runs, max_len, lib=lib)
        assert pk.tolist() == members and lk.tolist() == want_l, (t, "Algorithm 4.5")
        kp = 1
        while kp < len(runs):
            kp *= 2
        dL = sum(want_l[1:]) - sum(int(r[1][1:].sum()) for r in runs)
        assert cmps <= dL + len(members) * (kp.bit_length() - 1) + kp, (t, cmps)
        if len(runs) == 1:
            assert cmps == 0


def pin_prefix_doubling_names(lib):
    """Figure 8.1: the printed inverse h-suffix arrays ISA^1, ISA^2, ISA^4 of
    tobeornottobe$ (smallest h-names), and the printed SA^8 as the suffix
    array."""
    g = golden("fig8_1.txt")
    text = g["text"].encode()
    chars = np.frombuffer(text + b"\0", np.uint8).copy()
    offsets = np.array([int(x) for x in g["offsets"].split()], np.uint64)
    for h in (1, 2, 4):
        want = [int(x) for x in g[f"isa{h}"].split()]
        assert oracle.h_names(chars, offsets, h, lib=lib).tolist() == want, h
    sa, _ = oracle.sort(chars, offsets, 0, lib=lib)
    assert sa.tolist() == [int(x) for x in g["perm"].split()]
    sa2, _ = oracle.suffix_array(text, lib=lib)
    assert sa2.tolist() == [int(x) for x in g["perm"].split()][1:]   # without the empty suffix


def pin_suffix_array_closed_forms(lib):
    """Texts whose suffix and LCP arrays have a closed form: a^n (suffixes by
    length, shortest first; LCP[j] = j) and (ab)^k (the a-suffixes by length,
    LCPs 0, 2, 4, ...; then the b-suffixes by length, LCPs 0, 1, 3, 5, ...)."""
    for n in (1, 2, 7, 40):
        sa, lcp = oracle.suffix_array(b"a" * n, lib=lib)
        assert sa.tolist() == list(range(n - 1, -1, -1)), n
        assert lcp.tolist() == list(range(n)), n
    for k in (1, 2, 5, 17):
        n = 2 * k
        sa, lcp = oracle.suffix_array(b"ab" * k, lib=lib)
        want_sa = list(range(n - 2, -1, -2)) + list(range(n - 1, 0, -2))
        want_lcp = [2 * m for m in range(k)] + [0] + [2 * m - 1 for m in range(1, k)]
        assert sa.tolist() == want_sa, k
        assert lcp.tolist() == want_lcp, k


ALL_PINS = [pin_paper_suffix_examples, pin_word_list_ties, pin_lemma_2_1, pin_brute_force,
            pin_library_sort, pin_checker, pin_cache, pin_bucket_and_tree, pin_distinguishing,
            pin_lemma_4_1, pin_merge, pin_prefix_doubling_names, pin_suffix_array_closed_forms]
