/*
 * Seeded synthetic string-set generators.
 *
 * These produce the inputs that the CPU oracle and the CUDA sort are both run
 * on.  They hold no sorting arithmetic: they only lay strings out the way the
 * sort's interface expects them (one buffer of NUL-terminated bytes plus an
 * array of uint64 start offsets, Section 2.1 of the dissertation).
 *
 * Every random draw comes from a counter-based generator: a value is a pure
 * function of (seed, stream, counter), so the output is identical for any
 * thread count and on any host architecture.
 *
 * Shapes follow the paper's input classes (Table 2.2, Section 2.3.2):
 *   - random strings          (stand-in for "Random")
 *   - URL-like strings        (stand-in for "URLs" / "Sinha URLs")
 *   - DNA-like text suffixes  (stand-in for "Sinha DNA" and suffix sorting of
 *                              "Wikip")
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- counter-based generator ------------------------------------------- */

/* SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014). */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return mix64(mix64(mix64(seed) ^ stream) ^ (ctr * 0xD1B54A32D192ED03ull));
}

/* Uniform integer in [0, m) by multiply-shift (Lemire 2019). */
static inline uint64_t below(uint64_t r, uint64_t m) {
    return (uint64_t)(((unsigned __int128)r * m) >> 64);
}

/* Uniform double in (0, 1]. */
static inline double unit_open0(uint64_t r) {
    return ((double)(r >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* ---- random strings ------------------------------------------------------ */

static inline uint32_t random_len(uint64_t seed, uint64_t i, uint32_t lmin, uint32_t lmax) {
    return lmin + (uint32_t)below(rnd(seed, i, 0), (uint64_t)(lmax - lmin) + 1);
}

/* Total buffer size (bytes, NUL terminators included) of gen_random_fill. */
uint64_t gen_random_size(uint64_t n, uint64_t seed, uint32_t lmin, uint32_t lmax) {
    uint64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) total += random_len(seed, (uint64_t)i, lmin, lmax) + 1;
    return total;
}

/* n strings, length uniform in [lmin, lmax], bytes uniform in [alo, ahi]
 * (alo >= 1), stored back to back in generation order. */
void gen_random_fill(uint64_t n, uint64_t seed, uint32_t lmin, uint32_t lmax,
                     uint32_t alo, uint32_t ahi, uint8_t* chars, uint64_t* offsets) {
    uint64_t run = 0;
    for (uint64_t i = 0; i < n; ++i) {
        offsets[i] = run;
        run += random_len(seed, i, lmin, lmax) + 1;
    }
    const uint64_t span = (uint64_t)(ahi - alo) + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint32_t len = random_len(seed, (uint64_t)i, lmin, lmax);
        uint8_t* s = chars + offsets[i];
        for (uint32_t j = 0; j < len; ++j) s[j] = (uint8_t)(alo + below(rnd(seed, (uint64_t)i, 1 + j), span));
        s[len] = 0;
    }
}

/* ---- URL-like strings ---------------------------------------------------- */

#define URL_HOSTS 2000
#define URL_HOST_MAX 48
static const char* const kTld[7] = {".com", ".org", ".net", ".de", ".edu", ".io", ".info"};

typedef struct {
    uint8_t host[URL_HOSTS][URL_HOST_MAX];
    uint32_t hlen[URL_HOSTS];
    double cdf[URL_HOSTS]; /* Zipf(s) over host ranks 1..URL_HOSTS */
} url_tables;

static void url_build_tables(url_tables* t, uint64_t seed, double s) {
    const uint64_t stream0 = 1ull << 40;
    for (uint32_t h = 0; h < URL_HOSTS; ++h) {
        const uint64_t st = stream0 + h;
        uint32_t c = 0, k = 0;
        uint8_t* p = t->host[h];
        if (rnd(seed, st, c++) >> 63) { memcpy(p + k, "www.", 4); k += 4; }
        uint32_t lab = 8 + (uint32_t)below(rnd(seed, st, c++), 11);        /* [a-z]{8..18} */
        for (uint32_t j = 0; j < lab; ++j) p[k++] = (uint8_t)('a' + below(rnd(seed, st, c++), 26));
        if (rnd(seed, st, c++) >> 63) {                                    /* optional .[a-z]{3..8} */
            uint32_t sub = 3 + (uint32_t)below(rnd(seed, st, c++), 6);
            p[k++] = '.';
            for (uint32_t j = 0; j < sub; ++j) p[k++] = (uint8_t)('a' + below(rnd(seed, st, c++), 26));
        }
        const char* tld = kTld[below(rnd(seed, st, c++), 7)];
        size_t tl = strlen(tld);
        memcpy(p + k, tld, tl);
        k += (uint32_t)tl;
        t->hlen[h] = k;
    }
    double acc = 0;
    for (uint32_t r = 0; r < URL_HOSTS; ++r) { acc += pow((double)(r + 1), -s); t->cdf[r] = acc; }
    for (uint32_t r = 0; r < URL_HOSTS; ++r) t->cdf[r] /= acc;
}

static inline uint32_t url_host(const url_tables* t, uint64_t seed, uint64_t i) {
    double u = unit_open0(rnd(seed, i, 1));
    uint32_t lo = 0, hi = URL_HOSTS - 1; /* first rank with cdf >= u */
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (t->cdf[mid] >= u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static inline uint32_t url_len(const url_tables* t, uint64_t seed, uint64_t i) {
    uint32_t len = (rnd(seed, i, 0) >> 63) ? 8 : 7; /* https:// or http:// */
    len += t->hlen[url_host(t, seed, i)];
    uint32_t nseg = 1 + (uint32_t)below(rnd(seed, i, 2), 6);
    for (uint32_t j = 0; j < nseg; ++j) len += 1 + 3 + (uint32_t)below(rnd(seed, i, 3 + j), 10);
    return len;
}

uint64_t gen_url_size(uint64_t n, uint64_t seed, double zipf_s) {
    url_tables* t = (url_tables*)malloc(sizeof(url_tables));
    url_build_tables(t, seed, zipf_s);
    uint64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) total += url_len(t, seed, (uint64_t)i) + 1;
    free(t);
    return total;
}

/* n URL-like strings: "http://" or "https://" (p = 1/2), a host drawn
 * Zipf(zipf_s) from URL_HOSTS seeded host names, then 1..6 path segments
 * "/" + [a-z0-9]{3..12}. */
void gen_url_fill(uint64_t n, uint64_t seed, double zipf_s, uint8_t* chars, uint64_t* offsets) {
    url_tables* t = (url_tables*)malloc(sizeof(url_tables));
    url_build_tables(t, seed, zipf_s);
    uint64_t run = 0;
    for (uint64_t i = 0; i < n; ++i) { offsets[i] = run; run += url_len(t, seed, i) + 1; }
    static const char kPath[] = "abcdefghijklmnopqrstuvwxyz0123456789";
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < (int64_t)n; ++ii) {
        const uint64_t i = (uint64_t)ii;
        uint8_t* s = chars + offsets[i];
        uint32_t k = 0;
        if (rnd(seed, i, 0) >> 63) { memcpy(s, "https://", 8); k = 8; }
        else { memcpy(s, "http://", 7); k = 7; }
        uint32_t h = url_host(t, seed, i);
        memcpy(s + k, t->host[h], t->hlen[h]);
        k += t->hlen[h];
        uint32_t nseg = 1 + (uint32_t)below(rnd(seed, i, 2), 6);
        uint64_t c = 16;
        for (uint32_t j = 0; j < nseg; ++j) {
            uint32_t sl = 3 + (uint32_t)below(rnd(seed, i, 3 + j), 10);
            s[k++] = '/';
            for (uint32_t q = 0; q < sl; ++q) s[k++] = (uint8_t)kPath[below(rnd(seed, i, c++), 36)];
        }
        s[k] = 0;
    }
    free(t);
}

/* ---- DNA-like text --------------------------------------------------------- */

/* A text of exactly len bytes over {A,C,G,T} followed by a NUL at text[len]:
 * an order-3 Markov chain (64 contexts; each row of next-symbol probabilities
 * is a Dirichlet(1) draw) produces len - nblocks*blocklen symbols, and nblocks
 * copies of blocklen-symbol windows taken from earlier in the Markov text are
 * inserted at random positions.  Returns 0, or -1 if the sizes do not fit. */
int gen_dna_text(uint64_t len, uint64_t seed, uint32_t nblocks, uint32_t blocklen, uint8_t* text) {
    static const uint8_t kSym[4] = {'A', 'C', 'G', 'T'};
    const uint64_t dup = (uint64_t)nblocks * blocklen;
    if (dup > len || (nblocks && len - dup < (uint64_t)blocklen + 3)) return -1;
    const uint64_t m = len - dup;
    double prob[64][4];
    for (int c = 0; c < 64; ++c) {
        double e[4], sum = 0;
        for (int a = 0; a < 4; ++a) { e[a] = -log(unit_open0(rnd(seed, 7, (uint64_t)(c * 4 + a)))); sum += e[a]; }
        double acc = 0;
        for (int a = 0; a < 4; ++a) { acc += e[a] / sum; prob[c][a] = acc; }
        prob[c][3] = 1.0;
    }
    uint8_t* mk = (uint8_t*)malloc(m ? m : 1);
    uint32_t ctx = 0;
    for (uint64_t p = 0; p < m; ++p) {
        double u = unit_open0(rnd(seed, 8, p));
        uint32_t a;
        if (p < 3) a = (uint32_t)below(rnd(seed, 9, p), 4);
        else { a = 0; while (a < 3 && u > prob[ctx][a]) ++a; }
        mk[p] = kSym[a];
        ctx = ((ctx << 2) | a) & 63u;
    }
    /* insertion points (into the Markov text) and source windows */
    uint64_t* ins = (uint64_t*)malloc(sizeof(uint64_t) * (nblocks ? nblocks : 1));
    for (uint32_t b = 0; b < nblocks; ++b) ins[b] = blocklen + below(rnd(seed, 10, b), m - blocklen + 1);
    for (uint32_t b = 1; b < nblocks; ++b) { /* insertion sort: nblocks is small */
        uint64_t x = ins[b];
        int64_t j = (int64_t)b - 1;
        while (j >= 0 && ins[j] > x) { ins[j + 1] = ins[j]; --j; }
        ins[j + 1] = x;
    }
    uint64_t src = 0, out = 0;
    for (uint32_t b = 0; b < nblocks; ++b) {
        memcpy(text + out, mk + src, ins[b] - src);
        out += ins[b] - src;
        src = ins[b];
        uint64_t from = below(rnd(seed, 11, b), ins[b] - blocklen + 1);
        memcpy(text + out, mk + from, blocklen);
        out += blocklen;
    }
    memcpy(text + out, mk + src, m - src);
    out += m - src;
    text[out] = 0;
    free(ins);
    free(mk);
    return out == len ? 0 : -1;
}

/* ---- shared helpers for batch / trace generation ------------------------ */

uint64_t gen_rnd(uint64_t seed, uint64_t stream, uint64_t ctr) { return rnd(seed, stream, ctr); }

double gen_unit(uint64_t seed, uint64_t stream, uint64_t ctr) { return unit_open0(rnd(seed, stream, ctr)); }
