// Internal definitions shared by the CUDA translation units of ss_sort.
//
// Records: every string that is still being sorted is one 16-byte record
// (key, idx, off): key is the string's 8-byte character cache at its subset's
// current depth (chars_h of Algorithm 4.1, first character in the most
// significant byte), idx its index in its set, off the low 32 bits of its
// offset (the whole offset unless the set has offsets of 2^32 or more).  Records
// of one subset ("task") sit contiguously at [begin, begin + len) in one of
// two record buffers; a distribution step moves them to the same range of the
// other buffer (out-of-place redistribution with alternating roles,
// Section 4.2.8), so the range a record occupies after its last move is its
// final sorted position.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ss {

constexpr uint32_t kNoCap = 0xFFFFFFFFu;
constexpr uint32_t kMaxDepth = (1u << 30) - 16;  // deeper strings: SS_ERR_TOO_LARGE
constexpr uint32_t kLcpMark = 0x80000000u;        // out_lcp[j] = mark | depth: fix up later
constexpr uint32_t kLcpWide = 0x40000000u;        // ... the two strings differ within 2 keys (a wide step)

// Device status bits (latched with atomicOr; the host maps them to ss_status).
constexpr uint32_t kStQueueFull = 1u << 0;
constexpr uint32_t kStTimeout = 1u << 1;
constexpr uint32_t kStTooDeep = 1u << 2;

// One string set.
struct SetDesc {
  const uint8_t* chars;
  const uint64_t* offsets;
  uint32_t* perm;
  uint32_t* lcp;     // nullptr: no LCP output
  uint32_t n;
  uint32_t cap;      // kNoCap or max_len
  uint32_t base;     // first record position of this set
  uint32_t dna;      // 1: chars holds 3-bit character codes (see dna_key), not bytes
};

// One string being sorted (moved with one 16-byte load and store).
struct __align__(16) Rec {
  uint64_t key;
  uint32_t idx;
  uint32_t off;
};

__device__ __forceinline__ Rec load_rec(const Rec* p) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  return Rec{((uint64_t)v.y << 32) | v.x, v.z, v.w};
}

__device__ __forceinline__ void store_rec(Rec* p, uint64_t key, uint32_t idx, uint32_t off) {
  *reinterpret_cast<uint4*>(p) = make_uint4((uint32_t)key, (uint32_t)(key >> 32), idx, off);
}

// A subset of records with a common prefix of `depth` characters.
struct Task {
  uint32_t begin;
  uint32_t len;
  uint32_t depth;
  uint32_t meta;     // bit 31: record buffer (parity); bits 0..30: set id
};

__host__ __device__ inline uint32_t task_set(const Task& t) { return t.meta & 0x7FFFFFFFu; }
__host__ __device__ inline uint32_t task_par(const Task& t) { return t.meta >> 31; }
__host__ __device__ inline uint32_t make_meta(uint32_t set, uint32_t par) { return set | (par << 31); }

// Task of one multi-block step, augmented by the host plan.
struct GenTask {
  Task t;
  uint32_t tile_start;  // first global tile of this task
  uint32_t tiles;       // tiles of this task
  uint32_t rec_base;    // sum of len over earlier tasks of this step
  uint32_t cnt_base_lo; // first counter (low / high 32 bits)
  uint32_t cnt_base_hi;
  uint32_t pad[3];
};

// Append-only task list in device memory.
// Block-sort subsets of up to this many strings go to 64-thread blocks, larger
// ones to 256-thread blocks; each size class has its own task list.
constexpr uint32_t kSmallCtaNarrowMax = 256;

struct TaskList {
  Task* items;
  uint32_t* count;     // device counter
  uint32_t cap;
};

// Work queue of the persistent kernel: a ring of cap slots.  Push number k
// (and claim number k) uses slot k mod cap in lap k / cap; the slot's flag is
// 2 * lap while it waits for that lap's task, 2 * lap + 1 once the task is in,
// and the claim sets it to 2 * lap + 2 after reading it.  Flags start at 0.
// The tasks pushed and not yet claimed are disjoint subsets of more than
// small_cutoff records, so a ring of more than (records / (small_cutoff + 1))
// slots never holds a slot's next task before its last one has been claimed:
// the queue cannot overflow, however many times subsets are requeued.
struct WorkQueue {
  Task* items;
  uint32_t* ready;
  uint32_t* head;      // claims so far
  uint32_t* tail;      // pushes so far
  uint32_t* pending;   // tasks pushed and not yet finished
  uint32_t cap;
};

// Kernel classes for launch statistics and algorithmic-byte accounting.
enum KernelClass : uint32_t { kKInit = 0, kKBigSample, kKBigClassify, kKScan, kKBigEmit, kKBigScatter, kKQueue,
                              kKSmallWarp, kKSmallCta, kKLcpFix, kKClasses };

// Everything a kernel needs about the sort in flight.
struct SortCtx {
  const SetDesc* sets;
  uint32_t num_sets;
  uint32_t total;          // records over all sets
  Rec* rec[2];
  uint2* wid[2];           // (idx, off) of a record held in the wide form (multi-block subsets)
  uint32_t* wide;          // per set: 1 if some offset is 2^32 or more (then off is not enough)
  uint16_t* bucket_of;     // bucket index of each record (array o of Algorithm 4.1)
  uint32_t* status;
  unsigned long long* abytes;  // [kKClasses] algorithmic bytes moved, per kernel class
  TaskList big[2];         // multi-block tasks, ping-pong by step
  WorkQueue mq;            // tasks for the persistent single-block kernel
  TaskList small_warp;     // 2..32 records
  TaskList small_deep;     // runs the first warp pass deferred (long common prefixes)
  TaskList small_cta;      // 33..min(small_cutoff, kSmallCtaNarrowMax) records (64-thread block sorts)
  TaskList small_cta_wide; // kSmallCtaNarrowMax + 1..small_cutoff records (256-thread block sorts)
  uint32_t* small_claim;   // [2] next subset to claim, for the two block-sort launches
  uint32_t* marks;         // record positions whose LCP entry holds a mark (multi-block step boundaries)
  uint32_t* marks_count;
  uint32_t marks_cap;
  uint32_t small_cutoff;
  uint32_t big_threshold;  // tasks longer than this go to big[] (if big_enabled)
  uint32_t big_enabled;
  uint32_t seed;
  uint32_t classifier;     // classification variant (kClassifyUI / UIC / E)
  uint32_t big_cur;        // which big[] list the current step reads
  uint32_t dna;            // every set holds 3-bit character codes (SetDesc::dna)
  uint64_t wait_ns;        // bound on every device-side wait (then kStTimeout)
  uint32_t* fold_status;   // if set: the last kernel ORs *status into it (the stream's status word)
};

// ---------------------------------------------------------------------------
// Character cache: chars_h(s) of Algorithm 4.1 (w = 8).

// Index (0..7) of the lowest zero byte of a little-endian word, 8 if none.
// The borrow of (x - 0x01..01) can only flag bytes above a true zero byte, so
// the lowest flagged byte is exact.
__device__ __forceinline__ uint32_t first_zero_byte(uint64_t x) {
  uint64_t t = (x - 0x0101010101010101ull) & ~x & 0x8080808080808080ull;
  return t ? (uint32_t)(__ffsll((long long)t) - 1) >> 3 : 8u;
}

__device__ __forceinline__ uint64_t bswap64(uint64_t v) {
  uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
}

// The 8 characters of the string at chars + off from depth h on, first
// character in the most significant byte; positions at/after the terminator
// or at/after `cap` read as 0.  Precondition: the string has no terminator
// before position h (so the word holding position h holds a byte of the
// string or its terminator).  Loads only aligned 8-byte words holding at
// least one byte of the string or its terminator.
__device__ __forceinline__ uint64_t load_cache(const uint8_t* chars, uint64_t off, uint32_t h,
                                               uint32_t cap) {
  if (h >= cap) return 0;
  const uintptr_t a = (uintptr_t)(chars + off + h);
  const uint64_t* p = (const uint64_t*)(a & ~(uintptr_t)7);
  const uint32_t sh = (uint32_t)(a & 7);
  const uint32_t nb0 = 8 - sh;               // bytes of interest in the first word
  uint64_t v = __ldg(p) >> (8 * sh);
  const uint32_t room = cap - h;             // bytes before the cap (>= 1)
  uint32_t z;
  if (sh == 0) {
    z = first_zero_byte(v);
  } else {
    z = first_zero_byte(v | (~0ull << (8 * nb0)));
    if (z >= nb0 && room > nb0) {            // no terminator in the first word
      v |= __ldg(p + 1) << (8 * nb0);
      z = first_zero_byte(v);
    }
  }
  uint32_t keep = z < room ? z : room;       // bytes to keep (0..8)
  if (keep < 8) v &= (keep == 0) ? 0ull : (~0ull >> (64 - 8 * keep));
  return bswap64(v);
}

// load_cache with both words issued at once: when the window is unaligned and
// the second aligned word lies in the same 4 KiB block as byte h, it is loaded
// together with the first (one memory round trip instead of two; bytes past
// the terminator are discarded); across a block boundary it is loaded only if
// the first word holds no terminator, as in load_cache.  Same result and
// precondition as load_cache.
__device__ __forceinline__ uint64_t load_cache_2w(const uint8_t* chars, uint64_t off, uint32_t h,
                                                  uint32_t cap) {
  if (h >= cap) return 0;
  const uintptr_t a = (uintptr_t)(chars + off + h);
  const uint64_t* p = (const uint64_t*)(a & ~(uintptr_t)7);
  const uint32_t sh = (uint32_t)(a & 7);
  const bool same_block = (((uintptr_t)(p + 1)) & 4095u) != 0;
  const uint64_t w0 = __ldg(p);
  uint64_t w1 = (sh && same_block) ? __ldg(p + 1) : 0ull;
  uint64_t v = w0 >> (8 * sh);
  const uint32_t room = cap - h;
  uint32_t z;
  if (sh == 0) {
    z = first_zero_byte(v);
  } else {
    const uint32_t nb0 = 8 - sh;
    z = first_zero_byte(v | (~0ull << (8 * nb0)));
    if (z >= nb0 && room > nb0) {
      if (!same_block) w1 = __ldg(p + 1);
      v |= w1 << (8 * nb0);
      z = first_zero_byte(v);
    }
  }
  uint32_t keep = z < room ? z : room;
  if (keep < 8) v &= (keep == 0) ? 0ull : (~0ull >> (64 - 8 * keep));
  return bswap64(v);
}

constexpr int kLookWindows = 8;  // look-ahead: 8 windows = 64 characters per round

// Look-ahead read for the refinement of long common prefixes: the KW windows
// of 8 characters at depths h, h + 8, ..., h + 8(KW-1) (first character most
// significant, zero at/after the terminator or the cap).  Precondition: the
// string has no terminator before h, so the byte at h belongs to the string
// (or is its terminator).  All KW + 1 aligned words are issued at once, but
// only words inside the 4 KiB-aligned block that holds byte h are read: memory
// is mapped in blocks of at least 4 KiB, so these reads cannot fault, and bytes
// past the terminator are discarded.  Returns how many leading windows are
// fully determined (windows past the block, before a terminator was seen, are
// not).
//
// Two phases, so that a thread can have the reads of several strings in
// flight before it uses any of them: issue_windows loads the words,
// finish_windows turns them into the windows.
template <int KW>
struct WindowWords {
  uint64_t word[KW + 1];
};

// Loads the first `words` (<= KW + 1) of the words; a caller that uses only
// the first window may ask for 2 (the rest read as 0, and their windows are
// not to be used).
template <int KW>
__device__ __forceinline__ void issue_windows(const uint8_t* chars, uint64_t off, uint32_t h, uint32_t cap,
                                              WindowWords<KW>& ww, uint32_t words = KW + 1) {
  const uintptr_t a = (uintptr_t)(chars + off + h);
  const uintptr_t blk_end = (a & ~(uintptr_t)4095) + 4096;
  const uintptr_t p0 = a & ~(uintptr_t)7;
#pragma unroll
  for (int i = 0; i <= KW; ++i) {
    const uintptr_t q = p0 + 8 * (uintptr_t)i;
    ww.word[i] = ((uint32_t)i < words && h < cap && q < blk_end) ? __ldg(reinterpret_cast<const uint64_t*>(q)) : 0ull;
  }
}

// The same string and depth as the issue_windows call that filled ww.
template <int KW>
__device__ __forceinline__ uint32_t finish_windows(const WindowWords<KW>& ww, const uint8_t* chars, uint64_t off,
                                                   uint32_t h, uint32_t cap, uint64_t (&w)[KW]) {
#pragma unroll
  for (int j = 0; j < KW; ++j) w[j] = 0;
  if (h >= cap) return KW;
  const uintptr_t a = (uintptr_t)(chars + off + h);
  const uintptr_t blk_end = (a & ~(uintptr_t)4095) + 4096;
  const uint32_t sh = (uint32_t)(a & 7);
  const uint64_t known_total = (uint64_t)(blk_end - a);  // bytes from h that may be read (>= 1)
  const uint64_t room_total = (uint64_t)cap - h;         // bytes from h before the cap (>= 1)
  uint32_t nwin = KW;
  bool ended = false;
#pragma unroll
  for (int j = 0; j < KW; ++j) {
    if (ended || (uint32_t)j >= nwin) continue;
    uint64_t v = sh ? ((ww.word[j] >> (8 * sh)) | (ww.word[j + 1] << (64 - 8 * sh))) : ww.word[j];
    const uint64_t ws = 8ull * j;
    const uint32_t known = known_total > ws ? (known_total - ws >= 8 ? 8u : (uint32_t)(known_total - ws)) : 0u;
    const uint32_t room = room_total > ws ? (room_total - ws >= 8 ? 8u : (uint32_t)(room_total - ws)) : 0u;
    const uint32_t z = first_zero_byte(known < 8 ? (v | (~0ull << (8 * known))) : v);
    if (z < known || room <= known) {
      const uint32_t keep = z < room ? z : room;
      if (keep < 8) {
        v &= keep ? (~0ull >> (64 - 8 * keep)) : 0ull;
        ended = true;
      }
      w[j] = bswap64(v);
    } else {
      nwin = (uint32_t)j;  // bytes past the block decide this window
    }
  }
  return nwin;
}

template <int KW>
__device__ __forceinline__ uint32_t load_windows(const uint8_t* chars, uint64_t off, uint32_t h, uint32_t cap,
                                                 uint64_t (&w)[KW]) {
  WindowWords<KW> ww;
  issue_windows<KW>(chars, off, h, cap, ww);
  return finish_windows<KW>(ww, chars, off, h, cap, w);
}

// Offset of a record's string.
__device__ __forceinline__ uint64_t rec_offset(const SetDesc& sd, uint32_t wide, uint32_t idx, uint32_t off) {
  return wide ? sd.offsets[idx] : (uint64_t)off;
}

// Length of the common prefix of two caches, in characters (8 if equal).
__device__ __forceinline__ uint32_t lcp8(uint64_t a, uint64_t b) {
  uint64_t x = a ^ b;
  return x ? (uint32_t)__clzll((long long)x) >> 3 : 8u;
}

// True if the cache holds the terminator (after it every byte is 0, so the
// last byte is 0 iff a terminator lies inside the window).
__device__ __forceinline__ bool has_nul(uint64_t c) { return (c & 0xFFu) == 0; }

// Characters before the terminator inside a cache that holds one.
__device__ __forceinline__ uint32_t nnz_prefix(uint64_t c) {
  return c ? 8u - ((uint32_t)(__ffsll((long long)c) - 1) >> 3) : 0u;
}

// ---------------------------------------------------------------------------
// Alphabet compression for DNA (Section 4.4, "Alphabet compression"): each
// character is a 3-bit code (0 = end of string, 1..4 = A, C, G, T), packed
// most significant first into 64-bit words, so that a key holds 21
// characters (bits 63..1) instead of 8, still compares as an integer in
// string order, and still ends in a zero code when it holds the end.  Code 0
// keeps the terminator: with 2 bits per character a string that ends inside
// a word could not be told from one that continues with A.

constexpr uint32_t kDnaWidth = 21;                       // characters per key
constexpr uint64_t kDnaDigitLow = 0x2492492492492492ull;  // lowest bit of each code: bits 61, 58, ..., 1

// The 21 characters of the string at character offset `off` from depth h of
// a packed code buffer (padded with zero words past its end), with every code
// at or after the end (or the cap) zero.  Precondition as load_cache: the
// string does not end before h.
__device__ __forceinline__ uint64_t dna_key(const uint8_t* packed, uint64_t off, uint32_t h, uint32_t cap) {
  if (h >= cap) return 0;
  const uint64_t* p = reinterpret_cast<const uint64_t*>(packed);
  const uint64_t bit = 3 * (off + h);
  const uint64_t wi = bit >> 6;
  const uint32_t r = (uint32_t)(bit & 63);
  uint64_t x = __ldg(p + wi) << r;
  if (r) x |= __ldg(p + wi + 1) >> (64 - r);
  x &= ~1ull;
  const uint64_t y = x | (x >> 1) | (x >> 2);
  const uint64_t zeros = ~y & kDnaDigitLow;  // lowest bit of every zero code
  const uint32_t first_end = zeros ? (61u - (63u - (uint32_t)__clzll((long long)zeros))) / 3u : kDnaWidth;
  const uint32_t room = cap - h;
  const uint32_t keep = first_end < room ? first_end : room;
  if (keep < kDnaWidth) x &= keep ? (~0ull << (64 - 3 * keep)) : 0ull;
  return x;
}

// Key operations for both character encodings (dna = 0: bytes, 8 per key).
__device__ __forceinline__ uint32_t key_width(uint32_t dna) { return dna ? kDnaWidth : 8u; }

// Characters two keys at the same depth have in common (the whole key if equal).
__device__ __forceinline__ uint32_t key_lcp(uint64_t a, uint64_t b, uint32_t dna) {
  if (!dna) return lcp8(a, b);
  const uint64_t x = a ^ b;
  return x ? (uint32_t)__clzll((long long)x) / 3u : kDnaWidth;
}

// True if the key holds the end of its string.
__device__ __forceinline__ bool key_end(uint64_t c, uint32_t dna) {
  return dna ? (c & 0xEull) == 0 : (c & 0xFFull) == 0;
}

// Characters before the end inside a key that holds it.
__device__ __forceinline__ uint32_t key_nnz(uint64_t c, uint32_t dna) {
  if (!dna) return nnz_prefix(c);
  const uint64_t y = c | (c >> 1) | (c >> 2);
  const uint64_t zeros = ~y & kDnaDigitLow;
  return zeros ? (61u - (63u - (uint32_t)__clzll((long long)zeros))) / 3u : kDnaWidth;
}

__device__ __forceinline__ uint64_t load_key(const uint8_t* chars, uint64_t off, uint32_t h, uint32_t cap,
                                             uint32_t dna) {
  return dna ? dna_key(chars, off, h, cap) : load_cache(chars, off, h, cap);
}

// The KW keys at depths h, h + w, ..., h + (KW - 1) w (w = key_width) and how
// many of them are determined (all of them for the packed codes, whose buffer
// is padded; see load_windows for bytes).
template <int KW>
__device__ __forceinline__ uint32_t load_key_windows(const uint8_t* chars, uint64_t off, uint32_t h, uint32_t cap,
                                                     uint32_t dna, uint64_t (&w)[KW]) {
  if (!dna) return load_windows<KW>(chars, off, h, cap, w);
  bool ended = false;
#pragma unroll
  for (int j = 0; j < KW; ++j) {
    w[j] = ended ? 0ull : dna_key(chars, off, h + kDnaWidth * (uint32_t)j, cap);
    ended = ended || key_end(w[j], 1);
  }
  return KW;
}

// ---------------------------------------------------------------------------
// Wide keys of the multi-block steps: 16 characters (two bytes-caches) or 42
// packed DNA characters (two code words) per key, so that a step takes twice
// the characters of a narrow one (chars_h of Algorithm 4.1 with w = 16; the
// super-alphabet view of Section 4.4).  A key is compared as one 128-bit
// integer (first character most significant).  A record of a multi-block
// subset is held in the wide form: its key fills the 16-byte record slot
// (high word first), and (idx, off) sit at the same position of wid[].

typedef unsigned __int128 u128;

__device__ __forceinline__ uint64_t k_hi(u128 k) { return (uint64_t)(k >> 64); }
__device__ __forceinline__ uint64_t k_lo(u128 k) { return (uint64_t)k; }
__device__ __forceinline__ u128 make_k(uint64_t hi, uint64_t lo) { return ((u128)hi << 64) | lo; }

__device__ __forceinline__ u128 load_wkey(const Rec* p) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  return make_k(((uint64_t)v.y << 32) | v.x, ((uint64_t)v.w << 32) | v.z);
}

__device__ __forceinline__ void store_wkey(Rec* p, u128 k) {
  const uint64_t hi = k_hi(k), lo = k_lo(k);
  *reinterpret_cast<uint4*>(p) = make_uint4((uint32_t)hi, (uint32_t)(hi >> 32), (uint32_t)lo, (uint32_t)(lo >> 32));
}

// Key operations by key type (narrow: uint64_t, wide: u128) and encoding.
template <typename K>
struct KeyOps;

template <>
struct KeyOps<uint64_t> {
  static __device__ __forceinline__ uint32_t width(uint32_t dna) { return key_width(dna); }
  static __device__ __forceinline__ uint32_t lcp(uint64_t a, uint64_t b, uint32_t dna) { return key_lcp(a, b, dna); }
  static __device__ __forceinline__ bool end(uint64_t c, uint32_t dna) { return key_end(c, dna); }
  static __device__ __forceinline__ uint32_t nnz(uint64_t c, uint32_t dna) { return key_nnz(c, dna); }
  static __device__ __forceinline__ uint32_t top(uint64_t c, int bits) { return (uint32_t)(c >> (64 - bits)); }
  static __device__ __forceinline__ uint64_t shfl_xor(uint64_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
  static __device__ __forceinline__ uint64_t ones() { return ~0ull; }
};

template <>
struct KeyOps<u128> {
  static __device__ __forceinline__ uint32_t width(uint32_t dna) { return 2 * key_width(dna); }
  static __device__ __forceinline__ uint32_t lcp(u128 a, u128 b, uint32_t dna) {
    return k_hi(a) != k_hi(b) ? key_lcp(k_hi(a), k_hi(b), dna) : key_width(dna) + key_lcp(k_lo(a), k_lo(b), dna);
  }
  // the low word ends in the end code iff the string ends inside the key
  // (every position after the end is zero)
  static __device__ __forceinline__ bool end(u128 c, uint32_t dna) { return key_end(k_lo(c), dna); }
  static __device__ __forceinline__ uint32_t nnz(u128 c, uint32_t dna) {
    return key_end(k_hi(c), dna) ? key_nnz(k_hi(c), dna) : key_width(dna) + key_nnz(k_lo(c), dna);
  }
  static __device__ __forceinline__ uint32_t top(u128 c, int bits) { return (uint32_t)(k_hi(c) >> (64 - bits)); }
  static __device__ __forceinline__ u128 shfl_xor(u128 v, int m) {
    return make_k(__shfl_xor_sync(0xFFFFFFFFu, k_hi(v), m), __shfl_xor_sync(0xFFFFFFFFu, k_lo(v), m));
  }
  static __device__ __forceinline__ u128 ones() { return ~(u128)0; }
};

// The wide key of the string at `off` from depth h (precondition as
// load_cache).  Bytes: the 16 characters are fetched with the three aligned
// words that cover them in one round trip when they lie in the 4 KiB block of
// byte h (load_windows); otherwise word by word while the string continues.
__device__ __forceinline__ u128 load_key128(const uint8_t* chars, uint64_t off, uint32_t h, uint32_t cap,
                                            uint32_t dna) {
  if (dna) {
    const uint64_t hi = dna_key(chars, off, h, cap);
    const uint64_t lo = key_end(hi, 1) ? 0ull : dna_key(chars, off, h + kDnaWidth, cap);
    return make_k(hi, lo);
  }
  uint64_t w[2];
  const uint32_t nw = load_windows<2>(chars, off, h, cap, w);
  if (nw == 0) w[0] = load_cache(chars, off, h, cap);
  if (nw < 2) w[1] = has_nul(w[0]) ? 0ull : load_cache(chars, off, h + 8, cap);
  return make_k(w[0], w[1]);
}

// The narrow key (8 characters) d characters into a byte-encoded wide key,
// for d <= 8 (no memory access).
__device__ __forceinline__ uint64_t narrow_at(u128 k, uint32_t d) {
  if (d == 0) return k_hi(k);
  if (d >= 8) return k_lo(k);
  return (k_hi(k) << (8 * d)) | (k_lo(k) >> (64 - 8 * d));
}

// Counter-based hash for sample positions (SplitMix64 finaliser).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void latch_status(uint32_t* status, uint32_t bit) {
  atomicOr(status, bit);
}

// Append to a task list; on overflow the task is dropped and the status
// latched (the host then reports SS_ERR_QUEUE_FULL).
__device__ __forceinline__ void list_push(const TaskList& l, const Task& t, uint32_t* status) {
  uint32_t slot = atomicAdd(l.count, 1u);
  if (slot < l.cap) l.items[slot] = t;
  else latch_status(status, kStQueueFull);
}

// Waits (bounded by wait_ns) until *flag == want; false if the wait expired.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t want, uint64_t wait_ns) {
  volatile const uint32_t* f = flag;
  if (*f == want) return true;
  const uint64_t t0 = globaltimer_ns();
  uint32_t ns = 32;
  while (*f != want) {
    if (globaltimer_ns() - t0 > wait_ns) return false;
    __nanosleep(ns);
    ns = ns < 1024 ? ns * 2 : ns;
  }
  return true;
}

// Writes task t to slot k of the work queue's ring, once the slot's previous
// task has been claimed (see WorkQueue: that claim has always happened
// already; the wait only covers the moment between it and its read).  The
// caller has counted the task in q.pending and taken k from q.tail.
__device__ __forceinline__ void queue_put(const WorkQueue& q, uint32_t k, const Task& t, uint32_t* status,
                                          uint64_t wait_ns) {
  const uint32_t slot = k % q.cap, lap = k / q.cap;
  if (!wait_flag(q.ready + slot, 2 * lap, wait_ns)) {
    latch_status(status, kStTimeout);
    atomicSub(q.pending, 1u);
    return;
  }
  __threadfence();
  q.items[slot] = t;
  __threadfence();
  atomicExch(q.ready + slot, 2 * lap + 1);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Route new subsets (len >= 2, not finished) to the lists that handle their
// sizes.  The lanes of a warp that call it together take their slots in each
// list with one atomic per list: every block of the sort appends to the same
// few counters, and one atomic per lane would queue up at those addresses.
__device__ __forceinline__ void route_task(const SortCtx& c, const Task& t, uint32_t next_big) {
  constexpr uint32_t kToBig = 0, kToQueue = 1, kToCtaWide = 2, kToCta = 3, kToWarp = 4, kToNone = 5;
  const uint32_t len = t.len;
  uint32_t to = len > 32 ? (len > kSmallCtaNarrowMax ? kToCtaWide : kToCta) : kToWarp;
  to = len > c.small_cutoff ? kToQueue : to;
  to = (c.big_enabled && len > c.big_threshold) ? kToBig : to;
  to = t.depth > kMaxDepth ? kToNone : to;
  const uint32_t active = __activemask();
  uint32_t peers = 0;  // the calling lanes with the same destination
#pragma unroll
  for (uint32_t k = 0; k <= kToNone; ++k) {
    const uint32_t m = __ballot_sync(active, to == k);
    peers = to == k ? m : peers;
  }
  const uint32_t leader = __ffs(peers) - 1;
  uint32_t* const ctr = to == kToBig ? c.big[next_big].count
                        : to == kToQueue ? c.mq.tail
                        : to == kToCtaWide ? c.small_cta_wide.count
                        : to == kToCta ? c.small_cta.count : c.small_warp.count;
  uint32_t base = 0;
  if (to != kToNone && lane_id() == leader) {
    if (to == kToQueue) atomicAdd(c.mq.pending, (uint32_t)__popc(peers));  // counted before they can be claimed
    base = atomicAdd(ctr, (uint32_t)__popc(peers));
  }
  base = __shfl_sync(active, base, leader);
  const uint32_t k = base + __popc(peers & lanemask_lt());
  if (to == kToNone) {
    latch_status(c.status, kStTooDeep);
  } else if (to == kToQueue) {
    queue_put(c.mq, k, t, c.status, c.wait_ns);
  } else {
    const TaskList& l = to == kToBig ? c.big[next_big]
                        : to == kToCtaWide ? c.small_cta_wide
                        : to == kToCta ? c.small_cta : c.small_warp;
    if (k < l.cap) l.items[k] = t;
    else latch_status(c.status, kStQueueFull);
  }
}

// A slot of *counter for each calling lane of the warp with pred set: the
// lanes that call it together take consecutive slots with one atomic.
__device__ __forceinline__ uint32_t warp_slot(uint32_t* counter, bool pred) {
  const uint32_t active = __activemask();
  const uint32_t peers = __ballot_sync(active, pred);
  const uint32_t leader = peers ? __ffs(peers) - 1 : __ffs(active) - 1;
  uint32_t base = 0;
  if (peers && lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(peers));
  base = __shfl_sync(active, base, leader);
  return base + __popc(peers & lanemask_lt());
}

// Adds a thread's algorithmic byte count to its kernel class (one atomic per
// warp; every lane of the warp must call it).
__device__ __forceinline__ void account(const SortCtx& c, uint32_t cls, unsigned long long bytes) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xFFFFFFFFu, bytes, o);
  if ((threadIdx.x & 31u) == 0 && bytes) atomicAdd(c.abytes + cls, bytes);
}

}  // namespace ss
