"""Plants plausible mistakes in copies of the CPU oracle (on the CPU) and checks
that the pins catch every one of them: a wrong sign, index, dropped term,
transposed byte order, broken tie rule, cap off by one."""
import os
import tempfile

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "ss_oracle.c")

MUTANTS = {
    "lemma41_swapped_parts": ("    for (uint32_t k = x + 1; k < w; ++k) pb[o++] = lb[k];\n    pb[o++] = lb[x];",
                              "    pb[o++] = lb[x];\n    for (uint32_t k = x + 1; k < w; ++k) pb[o++] = lb[k];"),
    "dprefix_min": ("dprefix[j] = (uint32_t)((h > next ? h : next) + 1);", "dprefix[j] = (uint32_t)((h < next ? h : next) + 1);"),
    "dchar_off_by_one": ("dchar[j] = (uint8_t)char_at(chars + offsets[perm[j]], h, max_len);",
                         "dchar[j] = (uint8_t)char_at(chars + offsets[perm[j]], h + 1, max_len);"),
    "signed_char_compare": ("return ca < cb ? -1 : 1;",
                            "return (signed char)ca < (signed char)cb ? -1 : 1;"),
    "ties_descending": ("return c < 0 || (c == 0 && i < k);", "return c < 0 || (c == 0 && i > k);"),
    "ties_unstable": ("return c < 0 || (c == 0 && i < k);", "return c <= 0;"),
    "lcp_plus_one": ("if (ca != cb || ca == 0) return j;", "if (ca != cb || ca == 0) return j + (j > 0);"),
    "cap_off_by_one": ("if (max_len != 0 && j >= max_len) return 0;",
                       "if (max_len != 0 && j > max_len) return 0;"),
    "d_drops_plus_one": ("d += (left > right ? left : right) + 1;", "d += (left > right ? left : right);"),
    "d_wrong_neighbour": ("uint64_t right = (i + 1 < n) ? lcp[i + 1] : 0;",
                          "uint64_t right = (i + 1 < n) ? lcp[i] : 0;"),
    "cache_little_endian": ("c = (c << 8) | b;", "c |= (uint64_t)b << (8 * k);"),
    "bucket_le": ("if (x[j] < c) ++r;", "if (x[j] <= c) ++r;"),
    "tree_mirrored": ("tree_fill(x, t, v, 2 * node, next);\n    t[node] = x[(*next)++];\n    tree_fill(x, t, v, 2 * node + 1, next);",
                      "tree_fill(x, t, v, 2 * node + 1, next);\n    t[node] = x[(*next)++];\n    tree_fill(x, t, v, 2 * node, next);"),
    "lcp_compare_cases_swapped": ("    if (x->h < y->h) { t = *x; *x = *y; *y = t; }\n}",
                                  "    if (x->h > y->h) { t = *x; *x = *y; *y = t; }\n}"),
    "lcp_compare_ties_by_larger_index": ("(ca == cb && x->idx <= y->idx)", "(ca == cb && x->idx >= y->idx)"),
    "lcp_compare_keeps_loser_h": ("        y->h = h;\n        return;", "        return;"),
    "kway_new_front_h_zero": ("            x.h = run_lcp[pos[r]];", "            x.h = 0;"),
    "kway_replay_skips_parent": ("for (uint32_t v = (kp + r) / 2; v >= 1; v /= 2)",
                                 "for (uint32_t v = (kp + r) / 4; v >= 1; v /= 2)"),
    "merge_takes_right_on_tie": ("if (goes_before(chars, offsets, max_len, perm[b], perm[a])) tmp[o++] = perm[b++];",
                                 "if (str_compare(chars + offsets[perm[b]], chars + offsets[perm[a]], max_len) <= 0) tmp[o++] = perm[b++];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    with tempfile.TemporaryDirectory() as d:
        msrc = os.path.join(d, "mutant.c")
        with open(msrc, "w") as f:
            f.write(src.replace(old, new))
        lib = oracle.load(oracle.build(force=True, src=msrc, out=os.path.join(d, "libmutant.so")))
        caught = []
        for pin in pins.ALL_PINS:
            try:
                pin(lib)
            except AssertionError:
                caught.append(pin.__name__)
        assert caught, f"no pin catches mutant {name}"
