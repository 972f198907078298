/*
 * CPU oracle for string sorting with LCP output.  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * library's sorting path never calls it.  It shares no code with the CUDA
 * sources.
 *
 * It is the plain definition, written to be checked by eye, with no blocking,
 * caching or fusion:
 *
 *   - Section 2.1: the input is n strings s_0..s_{n-1} over the alphabet
 *     {1..255}; each string ends at its first zero byte, and a shorter string
 *     that is a prefix of a longer one sorts first (the canonical
 *     lexicographic order).  Here string i starts at chars[offsets[i]] and,
 *     when max_len > 0, also ends after max_len bytes (a byte at position
 *     >= max_len is read as the terminator).
 *   - Ties (equal strings) are broken by the original index, ascending.  The
 *     paper leaves this open; this is the reading the sort implements.
 *   - Section 2.1: lcp(s, t) is the length of the longest common prefix; the
 *     LCP array of the sorted sequence is H = [h_0, h_1, ..., h_{n-1}] with
 *     h_i = lcp(s_{i-1}, s_i).  h_0 is undefined in the paper and is 0 here.
 *     As in the compare loop of Algorithm 4.2, matching stops at the
 *     terminator, so two equal strings have lcp = their length.
 *   - Lemma 2.1 (proof): the distinguishing prefix of the sorted string i is
 *     d_i = max(h_i, h_{i+1}) + 1 with h_0 = h_n = 0, D = sum d_i, and
 *     L = sum_{i>=1} h_i.
 *   - Section 4.3.2: the merge of sorted runs, as its definition (the sorted
 *     union) and as the LCP-aware tournament tree of Algorithm 4.5 (one
 *     character per comparison, counted for Theorem 4.7).
 *
 * Parity pins (see tests/): brute force over all n! orders on tiny inputs,
 * the suffix arrays printed in Figure 5.1, Examples 8.4 and 8.11 and
 * Figure 6.5, the word list of Figure 2.3, Lemma 2.1's example and bounds, and
 * an independent library sort on random inputs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Byte j of string s (a pointer to its first byte), with the cap applied. */
static inline unsigned char_at(const uint8_t* s, uint64_t j, uint32_t max_len) {
    if (max_len != 0 && j >= max_len) return 0;
    return s[j];
}

/* Lexicographic comparison of two strings: <0, 0, >0. */
static int str_compare(const uint8_t* a, const uint8_t* b, uint32_t max_len) {
    for (uint64_t j = 0;; ++j) {
        unsigned ca = char_at(a, j, max_len), cb = char_at(b, j, max_len);
        if (ca != cb) return ca < cb ? -1 : 1;
        if (ca == 0) return 0;
    }
}

/* lcp(a, b): matching positions before the first mismatch or terminator. */
static uint64_t str_lcp(const uint8_t* a, const uint8_t* b, uint32_t max_len) {
    uint64_t j = 0;
    for (;; ++j) {
        unsigned ca = char_at(a, j, max_len), cb = char_at(b, j, max_len);
        if (ca != cb || ca == 0) return j;
    }
}

/* "i goes before k": string order, ties by index. */
static int goes_before(const uint8_t* chars, const uint64_t* offsets, uint32_t max_len,
                       uint32_t i, uint32_t k) {
    int c = str_compare(chars + offsets[i], chars + offsets[k], max_len);
    return c < 0 || (c == 0 && i < k);
}

/* Top-down merge sort of perm[lo, hi) (plain, stable). */
static void merge_sort(const uint8_t* chars, const uint64_t* offsets, uint32_t max_len,
                       uint32_t* perm, uint32_t* tmp, uint64_t lo, uint64_t hi) {
    if (hi - lo < 2) return;
    uint64_t mid = lo + (hi - lo) / 2;
    merge_sort(chars, offsets, max_len, perm, tmp, lo, mid);
    merge_sort(chars, offsets, max_len, perm, tmp, mid, hi);
    uint64_t a = lo, b = mid, o = lo;
    while (a < mid && b < hi) {
        if (goes_before(chars, offsets, max_len, perm[b], perm[a])) tmp[o++] = perm[b++];
        else tmp[o++] = perm[a++];
    }
    while (a < mid) tmp[o++] = perm[a++];
    while (b < hi) tmp[o++] = perm[b++];
    memcpy(perm + lo, tmp + lo, (hi - lo) * sizeof(uint32_t));
}

/* Sort n strings; write the sorted order to perm[n] and, if lcp != NULL, the
 * LCP array to lcp[n].  Returns 0, or -1 on bad arguments / no memory. */
int oracle_sort(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t max_len,
                uint32_t* perm, uint32_t* lcp) {
    if (n > 0xFFFFFFFFull) return -1;
    if (n == 0) return 0;
    uint32_t* tmp = (uint32_t*)malloc(n * sizeof(uint32_t));
    if (!tmp) return -1;
    for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    merge_sort(chars, offsets, max_len, perm, tmp, 0, n);
    free(tmp);
    if (lcp) {
        lcp[0] = 0;
        for (uint64_t j = 1; j < n; ++j)
            lcp[j] = (uint32_t)str_lcp(chars + offsets[perm[j - 1]], chars + offsets[perm[j]], max_len);
    }
    return 0;
}

/* The naive LCP scan alone, for a given order. */
void oracle_lcp_array(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t max_len,
                      const uint32_t* perm, uint32_t* lcp) {
    if (n == 0) return;
    lcp[0] = 0;
    for (uint64_t j = 1; j < n; ++j)
        lcp[j] = (uint32_t)str_lcp(chars + offsets[perm[j - 1]], chars + offsets[perm[j]], max_len);
}

/* Checks a claimed result without sorting, in O(n + D) time:
 *   perm is a permutation of [0, n); adjacent strings are in order with ties
 *   ascending by index; lcp (if given) has lcp[0] = 0 and lcp[j] equal to the
 *   direct comparison of the two adjacent strings.
 * Such an order is unique, so passing this check is the same as matching the
 * oracle's output.  Returns -1 if all holds, else the first failing position
 * (n for a repeated or out-of-range index). */
int64_t oracle_check(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t max_len,
                     const uint32_t* perm, const uint32_t* lcp) {
    if (n == 0) return -1;
    uint8_t* seen = (uint8_t*)calloc(n, 1);
    if (!seen) return 0;
    for (uint64_t j = 0; j < n; ++j) {
        if (perm[j] >= n || seen[perm[j]]) { free(seen); return (int64_t)n; }
        seen[perm[j]] = 1;
    }
    free(seen);
    if (lcp && lcp[0] != 0) return 0;
    for (uint64_t j = 1; j < n; ++j) {
        const uint8_t* a = chars + offsets[perm[j - 1]];
        const uint8_t* b = chars + offsets[perm[j]];
        int c = str_compare(a, b, max_len);
        if (c > 0 || (c == 0 && perm[j - 1] > perm[j])) return (int64_t)j;
        if (lcp && lcp[j] != str_lcp(a, b, max_len)) return (int64_t)j;
    }
    return -1;
}

/* D and L of a sorted set from its LCP array (Lemma 2.1 and its proof). */
void oracle_dl(const uint32_t* lcp, uint64_t n, uint64_t* D, uint64_t* L) {
    uint64_t d = 0, l = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t left = (i == 0) ? 0 : lcp[i];
        uint64_t right = (i + 1 < n) ? lcp[i + 1] : 0;
        d += (left > right ? left : right) + 1;
        if (i >= 1) l += lcp[i];
    }
    *D = d;
    *L = l;
}

/* chars_h(s) of Algorithm 4.1: the w = 8 characters of string i at depth h,
 * packed so that the first character is the most significant byte, with every
 * position at or after the terminator (or the cap) read as 0.  Reads byte by
 * byte and never past the terminator. */
uint64_t oracle_cache(const uint8_t* chars, const uint64_t* offsets, uint64_t i, uint64_t h,
                      uint32_t max_len) {
    const uint8_t* s = chars + offsets[i];
    /* the string has a terminator at or after h only if no terminator lies before h */
    for (uint64_t j = 0; j < h; ++j)
        if (char_at(s, j, max_len) == 0) return 0;
    uint64_t c = 0;
    int ended = 0;
    for (int k = 0; k < 8; ++k) {
        unsigned b = ended ? 0 : char_at(s, h + (uint64_t)k, max_len);
        if (b == 0) ended = 1;
        c = (c << 8) | b;
    }
    return c;
}

/* The bucket of Algorithm 4.1 for a key c and v sorted splitters x_0..x_{v-1}:
 * r = the number of splitters smaller than c (bucket b_{2r}: x_{r-1} < c <
 * x_r), or the equality bucket 2r+1 when r < v and x_r = c.  Written as a
 * linear count, not as a tree descent. */
uint32_t oracle_bucket(uint64_t c, const uint64_t* x, uint32_t v) {
    uint32_t r = 0;
    for (uint32_t j = 0; j < v; ++j)
        if (x[j] < c) ++r;
    if (r < v && x[r] == c) return 2 * r + 1;
    return 2 * r;
}

/* The implicit splitter tree of Section 4.2.3: the perfect binary search tree
 * whose in-order sequence is x_0..x_{v-1} (v = 2^d - 1), stored in level order
 * as the one-based array t[1..v] (t[0] is left unused).  For v = 7 this is
 * t = [x_3, x_1, x_5, x_0, x_2, x_4, x_6].  Written as a recursive in-order
 * walk over the level-order indices. */
static void tree_fill(const uint64_t* x, uint64_t* t, uint32_t v, uint32_t node, uint32_t* next) {
    if (node > v) return;
    tree_fill(x, t, v, 2 * node, next);
    t[node] = x[(*next)++];
    tree_fill(x, t, v, 2 * node + 1, next);
}

void oracle_tree(const uint64_t* x, uint32_t v, uint64_t* t) {
    uint32_t next = 0;
    t[0] = 0;
    tree_fill(x, t, v, 1, &next);
}

/* For a sorted set (order perm, LCP array lcp): the distinguishing character
 * of sorted string j, c^_j = s_j[h_j] with h_j its LCP with its predecessor
 * (Section 4.3.4, caching variant of the LCP merge; h_0 = 0), 0 when the
 * string ends at h_j; and the length of its distinguishing prefix
 * d_j = max(h_j, h_{j+1}) + 1 with h_0 = h_n = 0 (proof of Lemma 2.1). */
void oracle_distinguishing(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t max_len,
                           const uint32_t* perm, const uint32_t* lcp, uint8_t* dchar, uint32_t* dprefix) {
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t h = (j == 0) ? 0 : lcp[j];
        uint64_t next = (j + 1 < n) ? lcp[j + 1] : 0;
        dchar[j] = (uint8_t)char_at(chars + offsets[perm[j]], h, max_len);
        dprefix[j] = (uint32_t)((h > next ? h : next) + 1);
    }
}

/* Lemma 4.1 (Section 4.2.3): index maps of a perfect binary tree with 2^w - 1
 * vertices between the one-based level-order index l = l_1 ... l_w and the
 * one-based pre-order (sorted-splitter) index p = p_1 ... p_w, as bit strings
 * (l_1, p_1 most significant).  (i) with l_x the first one bit of l:
 * p = l_{x+1} ... l_w  l_x  l_1 ... l_{x-1};  (ii) with p_y the last one bit of
 * p: l = p_{y+1} ... p_w  p_y  p_1 ... p_{y-1}.  Written on explicit bit
 * arrays. */
static void to_bits(uint32_t v, uint32_t w, int* b) {
    for (uint32_t k = 0; k < w; ++k) b[k] = (int)((v >> (w - 1 - k)) & 1u); /* b[0] = l_1 */
}
static uint32_t from_bits(const int* b, uint32_t w) {
    uint32_t v = 0;
    for (uint32_t k = 0; k < w; ++k) v = (v << 1) | (uint32_t)b[k];
    return v;
}

uint32_t oracle_level_to_pre(uint32_t l, uint32_t w) {
    int lb[32], pb[32];
    to_bits(l, w, lb);
    uint32_t x = 0;
    while (lb[x] == 0) ++x;          /* lb[x] is l_{x+1} in the lemma's one-based naming */
    uint32_t o = 0;
    for (uint32_t k = x + 1; k < w; ++k) pb[o++] = lb[k];
    pb[o++] = lb[x];
    for (uint32_t k = 0; k < x; ++k) pb[o++] = lb[k];
    return from_bits(pb, w);
}

uint32_t oracle_pre_to_level(uint32_t p, uint32_t w) {
    int pb[32], lb[32];
    to_bits(p, w, pb);
    uint32_t y = w - 1;
    while (pb[y] == 0) --y;          /* last one bit */
    uint32_t o = 0;
    for (uint32_t k = y + 1; k < w; ++k) lb[o++] = pb[k];
    lb[o++] = pb[y];
    for (uint32_t k = 0; k < y; ++k) lb[o++] = pb[k];
    return from_bits(lb, w);
}

/* ---- K-way merge of sorted runs (Section 4.3.2) --------------------------
 *
 * The merge of K runs (each a sorted sequence of string indices of the same
 * string set) has a plain definition: the union of the runs' indices in
 * string order, ties by index, with its LCP array.  oracle_merge writes
 * exactly that: the concatenated indices, merge-sorted with the comparison
 * above, and the naive LCP scan.  idx[total] holds the runs back to back (the
 * run boundaries do not matter to the definition). */
int oracle_merge(const uint8_t* chars, const uint64_t* offsets, uint32_t max_len, const uint32_t* idx,
                 uint64_t total, uint32_t* perm, uint32_t* lcp) {
    if (total > 0xFFFFFFFFull) return -1;
    if (total == 0) return 0;
    uint32_t* tmp = (uint32_t*)malloc(total * sizeof(uint32_t));
    if (!tmp) return -1;
    memcpy(perm, idx, total * sizeof(uint32_t));
    merge_sort(chars, offsets, max_len, perm, tmp, 0, total);
    free(tmp);
    oracle_lcp_array(chars, offsets, total, max_len, perm, lcp);
    return 0;
}

/* The same merge by the method of Section 4.3.2: a tournament (loser) tree
 * over the runs' front strings whose games are LCP-Compare (Algorithm 4.2),
 * kept LCP-aware as in Algorithm 4.5, comparing ONE character per step so
 * that the character comparisons can be counted against Theorem 4.7
 * (at most dL + n log2 K + K, K a power of two, dL = L(H_0) - sum_k L(H_k)).
 *
 * A player is (run, string index, h) where h is the LCP of its string with a
 * string p that precedes it; the two players of a game always share the same
 * p.  The tree has K leaves (runs padded with empty ones to a power of two);
 * internal node v (1..K-1, children 2v and 2v+1, leaf k at K + k) keeps the
 * loser of its last game with h = LCP(loser, that game's winner).  Runs that
 * are used up play a sentinel that loses every game. */
typedef struct {
    uint32_t run;                   /* K_pad: sentinel (used-up run) */
    uint32_t idx;
    uint64_t h;
} lm_player;

typedef struct {
    const uint8_t* chars;
    const uint64_t* offsets;
    uint32_t max_len;
    uint32_t sentinel;
    uint64_t cmps;                  /* character comparisons */
} lm_ctx;

/* LCP-Compare: plays *x against *y; afterwards *x is the winner (its h
 * unchanged: still its LCP with p) and *y the loser with h = LCP(loser,
 * winner).  Equal LCPs (case 1): compare characters from there on.  Unequal
 * LCPs (cases 2 and 3): the player with the larger LCP to p goes first, and
 * the LCP of the two is the smaller value, so no character is read. */
static void lcp_compare(lm_ctx* c, lm_player* x, lm_player* y) {
    lm_player t;
    if (y->run == c->sentinel) return;
    if (x->run == c->sentinel) { t = *x; *x = *y; *y = t; return; }
    if (x->h == y->h) {
        const uint8_t* sa = c->chars + c->offsets[x->idx];
        const uint8_t* sb = c->chars + c->offsets[y->idx];
        uint64_t h = x->h;
        unsigned ca, cb;
        for (;;) {
            ca = char_at(sa, h, c->max_len);
            cb = char_at(sb, h, c->max_len);
            c->cmps++;
            if (ca != cb || ca == 0) break;
            ++h;
        }
        int x_first = ca < cb || (ca == cb && x->idx <= y->idx);
        if (!x_first) { t = *x; *x = *y; *y = t; }
        y->h = h;
        return;
    }
    if (x->h < y->h) { t = *x; *x = *y; *y = t; }
}

/* run_idx / run_lcp hold the K runs back to back, run k at
 * [run_start[k], run_start[k+1]); run_lcp[j] = LCP with the previous string
 * of the same run (its first entry is not read).  Writes the merged order and
 * LCP array (total entries) and the number of character comparisons.
 * Returns 0, or -1 on bad arguments / no memory. */
int oracle_lcp_merge(const uint8_t* chars, const uint64_t* offsets, uint32_t max_len, uint32_t K,
                     const uint64_t* run_start, const uint32_t* run_idx, const uint32_t* run_lcp,
                     uint32_t* perm, uint32_t* lcp, uint64_t* char_cmps) {
    if (K == 0 || K > (1u << 20)) return -1;
    uint32_t kp = 1;
    while (kp < K) kp <<= 1;
    lm_ctx c = {chars, offsets, max_len, kp, 0};
    lm_player* node = (lm_player*)calloc(2 * (size_t)kp, sizeof(lm_player));
    uint64_t* pos = (uint64_t*)calloc(kp, sizeof(uint64_t));
    if (!node || !pos) { free(node); free(pos); return -1; }
    /* leaves: the first string of each run, h = 0 (p = the empty string) */
    for (uint32_t k = 0; k < kp; ++k) {
        lm_player* leaf = &node[kp + k];
        if (k < K && run_start[k] < run_start[k + 1]) {
            pos[k] = run_start[k];
            leaf->run = k;
            leaf->idx = run_idx[pos[k]];
            leaf->h = 0;
        } else {
            leaf->run = kp;
        }
    }
    /* first round: every game once, bottom-up; winners go up in w[] */
    lm_player* w = (lm_player*)calloc(2 * (size_t)kp, sizeof(lm_player));
    if (!w) { free(node); free(pos); return -1; }
    for (uint32_t k = 0; k < kp; ++k) w[kp + k] = node[kp + k];
    for (uint32_t v = kp - 1; v >= 1; --v) {
        lm_player x = w[2 * v], y = w[2 * v + 1];
        lcp_compare(&c, &x, &y);
        w[v] = x;
        node[v] = y;
    }
    lm_player win = kp > 1 ? w[1] : w[kp];
    free(w);
    uint64_t out = 0;
    while (win.run != kp) {
        perm[out] = win.idx;
        lcp[out] = out == 0 ? 0 : (uint32_t)win.h;
        ++out;
        /* the winner's run moves on; the new front string has h = its LCP
         * with the string just written, which is the common p of every loser
         * on the path to the root */
        uint32_t r = win.run;
        lm_player x;
        ++pos[r];
        if (pos[r] < run_start[r + 1]) {
            x.run = r;
            x.idx = run_idx[pos[r]];
            x.h = run_lcp[pos[r]];
        } else {
            x.run = kp;
            x.idx = 0;
            x.h = 0;
        }
        for (uint32_t v = (kp + r) / 2; v >= 1; v /= 2) lcp_compare(&c, &x, &node[v]);
        win = x;
    }
    free(node);
    free(pos);
    *char_cmps = c.cmps;
    return 0;
}
