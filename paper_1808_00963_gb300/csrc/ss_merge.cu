// K-way LCP-aware merge of sorted runs (Section 4.3.2) as ceil(log2 K) rounds
// of binary LCP merges (Algorithms 4.3 and 4.4), each split into independent
// pieces (Section 4.3.3).
//
// Records.  Every string of every run travels as a 32-byte record: its index,
// its offset, h = its LCP with the string before it in its run, and its
// characters [h, h + 16) as two big-endian words (the distinguishing
// characters of the caching variant of Section 4.3.4, 16 at a time).  A merge
// writes its output in the same form: the winner of each comparison already
// carries h = LCP with the string output before it and the characters from
// there on, so the output records of one round are the input of the next.
//
// Splitting.  Every S-th record of every run is a sample.  k_merge_cut counts,
// for each sample, the records of the partner run that go before it, with a
// binary search that skips the prefix every record between the two bounds
// shares with the sample.  The pieces of a pair of runs are the stretches of
// its output between consecutive samples; each warp takes 32 pieces at a
// time from a counter, one per lane.  With two runs a piece holds at most 2S
// records.
//
// Merging a piece.  Both front records carry h = LCP with the last string
// output (a piece starts after a sample, whose LCP with the other run's front
// is computed directly).  LCP-Compare (Algorithm 4.2): unequal h decide
// without reading characters (the larger h goes first, the loser keeps its
// h); equal h compare the cached characters, and read the strings only when
// all the cached characters both records still hold agree; the loser's h
// becomes its LCP with the winner.  The loser's cache then moves on to that
// depth by a shift (the characters between the old and the new h are the
// ones the two strings share), so a record holds from 1 to 16 valid cached
// characters; only a comparison that runs past them reads the strings, and
// the loser's cache is reloaded after it.  Ties of equal strings go by index,
// and an index present in both runs takes the first run's record first.
#include "../../include/ss_sort.h"
#include "ss_kernels.h"

namespace ss {

namespace {

constexpr uint32_t kMergeBlock = 128;
constexpr uint32_t kNoSample = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t cache_at(const uint8_t* chars, uint32_t cap, uint64_t off, uint32_t h) {
  return load_cache_2w(chars, off, h, cap);
}

// Compares string a (index ia, at offset oa) with string b (ib, ob); both
// share their first h characters (and neither ends before h).  Returns <0 / 0
// / >0 in the order (string, index) and sets *l = lcp(a, b).
__device__ __forceinline__ int cmp_from(const uint8_t* chars, uint32_t cap, uint32_t ia, uint64_t oa, uint32_t ib,
                                        uint64_t ob, uint32_t h, uint32_t* l) {
  while (true) {
    const uint64_t ca = cache_at(chars, cap, oa, h);
    const uint64_t cb = cache_at(chars, cap, ob, h);
    if (ca != cb) {
      *l = h + lcp8(ca, cb);
      return ca < cb ? -1 : 1;
    }
    if (has_nul(ca)) {
      *l = h + nnz_prefix(ca);
      return ia < ib ? -1 : (ia > ib ? 1 : 0);
    }
    h += 8;
  }
}

// A record in registers: the memory record plus how many of its 16 cached
// characters are not valid (the cache was shifted after a comparison).  In
// memory that count sits in the top byte of the offset (string offsets are
// below 2^56).
struct MRec {
  uint64_t w0, w1, off;
  uint32_t idx, h, miss;
};
constexpr uint64_t kOffMask = (1ull << 56) - 1;

__device__ __forceinline__ MRec load_mrec(const MergeRec* p) {
  const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
  const uint4 b = __ldg(reinterpret_cast<const uint4*>(p) + 1);
  MRec r;
  r.w0 = ((uint64_t)a.y << 32) | a.x;
  r.w1 = ((uint64_t)a.w << 32) | a.z;
  const uint64_t o = ((uint64_t)b.y << 32) | b.x;
  r.off = o & kOffMask;
  r.miss = (uint32_t)(o >> 56);
  r.idx = b.z;
  r.h = b.w;
  return r;
}

__device__ __forceinline__ void store_mrec(MergeRec* p, const MRec& r) {
  uint4* q = reinterpret_cast<uint4*>(p);
  const uint64_t o = r.off | ((uint64_t)r.miss << 56);
  q[0] = make_uint4((uint32_t)r.w0, (uint32_t)(r.w0 >> 32), (uint32_t)r.w1, (uint32_t)(r.w1 >> 32));
  q[1] = make_uint4((uint32_t)o, (uint32_t)(o >> 32), r.idx, r.h);
}

// Position (0..15) of the first zero byte of a 16-character cache (first
// character most significant), 16 if none.  Exact per byte: no borrow runs
// between bytes.
__device__ __forceinline__ uint32_t first_zero_char(uint64_t w0, uint64_t w1) {
  constexpr uint64_t k7F = 0x7F7F7F7F7F7F7F7Full;
  const uint64_t z0 = ~(((w0 & k7F) + k7F) | w0 | k7F);
  const uint64_t z1 = ~(((w1 & k7F) + k7F) | w1 | k7F);
  return z0 ? (uint32_t)__clzll((long long)z0) >> 3 : (z1 ? 8u + ((uint32_t)__clzll((long long)z1) >> 3) : 16u);
}

// The 16 characters of a string from depth h (no terminator before h): the
// three aligned words that cover them in one round trip when they lie in the
// 4 KiB block of byte h, otherwise word by word while the string continues.
__device__ __forceinline__ void finish_words(const WindowWords<2>& ww, const uint8_t* chars, uint32_t cap,
                                             uint64_t off, uint32_t h, uint64_t& w0, uint64_t& w1) {
  uint64_t w[2];
  const uint32_t nw = finish_windows<2>(ww, chars, off, h, cap, w);
  if (nw == 0) w[0] = cache_at(chars, cap, off, h);
  if (nw < 2) w[1] = has_nul(w[0]) ? 0ull : cache_at(chars, cap, off, h + 8);
  w0 = w[0];
  w1 = w[1];
}

__device__ __forceinline__ void load_words(const uint8_t* chars, uint32_t cap, uint64_t off, uint32_t h,
                                           uint64_t& w0, uint64_t& w1) {
  WindowWords<2> ww;
  issue_windows<2>(chars, off, h, cap, ww);
  finish_words(ww, chars, cap, off, h, w0, w1);
}

// Index of the last range whose start is <= i (starts non-decreasing).
__device__ __forceinline__ uint32_t find_range(const uint32_t* start, uint32_t count, uint32_t i) {
  uint32_t lo = 0, hi = count;  // start[lo] <= i < start[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (start[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// ---- round 0: records of the input runs --------------------------------------------------

// Records built per thread at once: the loads of all of them are issued
// level by level (entries, offsets, characters), one round trip each.
constexpr int kPrepBatch = 4;

__global__ void __launch_bounds__(256) k_merge_prep(MergePrepArgs a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < a.total; g0 += stride * kPrepBatch) {
    uint32_t idx[kPrepBatch], h[kPrepBatch];
    uint64_t off[kPrepBatch];
    WindowWords<2> ww[kPrepBatch];
#pragma unroll
    for (int u = 0; u < kPrepBatch; ++u) {
      const uint32_t g = g0 + u * stride;
      idx[u] = 0;
      h[u] = 0;
      if (g < a.total) {
        const uint32_t k = find_range(a.start, a.K, g);
        const uint32_t j = g - a.start[k];
        idx[u] = a.perm[k][j] + a.ibase[k];
        h[u] = j ? a.lcp[k][j] : 0u;
      }
    }
#pragma unroll
    for (int u = 0; u < kPrepBatch; ++u) off[u] = g0 + u * stride < a.total ? a.offsets[idx[u]] : 0ull;
#pragma unroll
    for (int u = 0; u < kPrepBatch; ++u)
      if (g0 + u * stride < a.total) issue_windows<2>(a.chars, off[u], h[u], a.cap, ww[u]);
#pragma unroll
    for (int u = 0; u < kPrepBatch; ++u) {
      const uint32_t g = g0 + u * stride;
      if (g >= a.total) continue;
      MRec r;
      r.idx = idx[u];
      r.h = h[u];
      r.off = off[u];
      r.miss = 0;
      finish_words(ww[u], a.chars, a.cap, off[u], h[u], r.w0, r.w1);
      store_mrec(a.dst + g, r);
    }
  }
}

// ---- splitting -------------------------------------------------------------------------

// For each sample: the records of the partner run that go before it (for a
// sample of the first run of a pair, the partner's records that are smaller;
// for one of the second run, those that are smaller or the same record).
__global__ void __launch_bounds__(256) k_merge_cut(MergeRoundArgs a) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nsamples; s += gridDim.x * blockDim.x) {
    const uint32_t c = find_range(a.sbase, a.ncur, s);
    const uint32_t pos = (s - a.sbase[c] + 1) * a.S - 1;
    const MRec x = load_mrec(a.src + a.start[c] + pos);
    const uint32_t q = c ^ 1u;
    uint32_t lo = 0, hi = 0;
    if (q < a.ncur) {
      const MergeRec* prt = a.src + a.start[q];
      hi = a.start[q + 1] - a.start[q];
      uint32_t llo = 0, lhi = 0;  // LCP of the sample with the records just below / at the bounds
      const bool strict = (c & 1u) == 0;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(prt + mid) + 1);
        const uint64_t off = (((uint64_t)b.y << 32) | b.x) & kOffMask;
        uint32_t l;
        const int cmp = cmp_from(a.chars, a.cap, b.z, off, x.idx, x.off, llo < lhi ? llo : lhi, &l);
        if (strict ? cmp < 0 : cmp <= 0) {
          lo = mid + 1;
          llo = l;
        } else {
          hi = mid;
          lhi = l;
        }
      }
    }
    a.cut[s] = lo;
  }
}

// End of a sample in its pair's output: records of the first and second run
// up to and including it.
__device__ __forceinline__ void sample_end(const MergeRoundArgs& a, uint32_t c, uint32_t t, uint32_t& ea,
                                           uint32_t& eb) {
  const uint32_t pos = (t + 1) * a.S;  // records of its own run up to and including it
  const uint32_t cut = a.cut[a.sbase[c] + t];
  if (c & 1u) {
    ea = cut;
    eb = pos;
  } else {
    ea = pos;
    eb = cut;
  }
}

// Last sample of run c whose end rank is below `rank` (its rank to r_out),
// or kNoSample.
__device__ __forceinline__ uint32_t last_sample_below(const MergeRoundArgs& a, uint32_t c, uint32_t rank,
                                                      uint32_t& r_out) {
  if (c >= a.ncur) return kNoSample;
  uint32_t lo = 0, hi = a.sbase[c + 1] - a.sbase[c];
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    uint32_t ea, eb;
    sample_end(a, c, mid, ea, eb);
    if (ea + eb < rank) lo = mid + 1; else hi = mid;
  }
  if (lo == 0) return kNoSample;
  uint32_t ea, eb;
  sample_end(a, c, lo - 1, ea, eb);
  r_out = ea + eb;
  return lo - 1;
}

// ---- merging ------------------------------------------------------------------------------

// Pieces are taken 32 at a time by a warp, one per lane, and the lanes merge
// them in lockstep: each iteration runs the same instructions on every lane
// (the choice between the fronts, the reload of the loser's words and the
// advance of the winner are selects and predicated loads), so lanes diverge
// only where a comparison has to read past the 16 cached characters; a lane
// whose piece is done idles until the longest piece of its warp is.
__global__ void __launch_bounds__(kMergeBlock) k_merge_round(MergeRoundArgs a) {
  const uint32_t npairs = (a.ncur + 1) / 2;
  const uint32_t npieces = a.nsamples + npairs;
  const uint32_t lane = lane_id();
  const bool last = a.dst == nullptr;
  while (true) {
    uint32_t q0 = 0;
    if (lane == 0) q0 = atomicAdd(a.counter, 32u);
    q0 = __shfl_sync(0xFFFFFFFFu, q0, 0);
    if (q0 >= npieces) return;
    const uint32_t q = q0 + lane;
    uint32_t out = 0, out_end = 0, ia = 0, jb = 0, ea = 0, eb = 0, base = 0;
    const MergeRec* A = a.src;
    const MergeRec* B = a.src;
    MRec fa{}, fb{};
    if (q < npieces) {
      // the pair and the end of this piece (records of each run up to it)
      uint32_t p;
      if (q < a.nsamples) {
        const uint32_t c = find_range(a.sbase, a.ncur, q);
        p = c >> 1;
        sample_end(a, c, q - a.sbase[c], ea, eb);
      } else {
        p = q - a.nsamples;
        ea = a.start[min(2 * p + 1, a.ncur)] - a.start[2 * p];
        eb = a.start[min(2 * p + 2, a.ncur)] - a.start[min(2 * p + 1, a.ncur)];
      }
      const uint32_t cA = 2 * p, cB = 2 * p + 1;
      base = a.start[cA];
      A = a.src + base;
      B = a.src + a.start[min(cB, a.ncur)];
      // the piece starts after the latest sample of the pair that ends before it
      uint32_t sa = 0, sb = 0, prev_run = 2;  // prev_run: 0 = A, 1 = B, 2 = none
      {
        uint32_t ra = 0, rb = 0;
        const uint32_t ta = last_sample_below(a, cA, ea + eb, ra);
        const uint32_t tb = last_sample_below(a, cB, ea + eb, rb);
        if (ta != kNoSample && (tb == kNoSample || ra > rb)) {
          sample_end(a, cA, ta, sa, sb);
          prev_run = 0;
        } else if (tb != kNoSample) {
          sample_end(a, cB, tb, sa, sb);
          prev_run = 1;
        }
      }
      out = sa + sb;
      out_end = ea + eb;
      ia = sa;
      jb = sb;
      if (out < out_end) {
        if (ia < ea) fa = load_mrec(A + ia);
        if (jb < eb) fb = load_mrec(B + jb);
        // LCP of the other run's front with the sample just before the piece
        if (prev_run == 0 && jb < eb) {
          const MRec P = load_mrec(A + sa - 1);
          cmp_from(a.chars, a.cap, P.idx, P.off, fb.idx, fb.off, 0, &fb.h);
          load_words(a.chars, a.cap, fb.off, fb.h, fb.w0, fb.w1);
          fb.miss = 0;
        } else if (prev_run == 1 && ia < ea) {
          const MRec P = load_mrec(B + sb - 1);
          cmp_from(a.chars, a.cap, P.idx, P.off, fa.idx, fa.off, 0, &fa.h);
          load_words(a.chars, a.cap, fa.off, fa.h, fa.w0, fa.w1);
          fa.miss = 0;
        }
      }
    }
    while (__any_sync(0xFFFFFFFFu, out < out_end)) {
      const bool act = out < out_end;
      const bool a_ok = act && ia < ea, b_ok = act && jb < eb;
      const bool both = a_ok && b_ok;
      const bool eqh = fa.h == fb.h;
      // equal LCPs with the last output: the m characters both caches still
      // hold decide unless they agree and neither string ends among them
      const uint32_t m = 16u - max(fa.miss, fb.miss);  // >= 1
      const u128 ka = make_k(fa.w0, fa.w1), kb = make_k(fb.w0, fb.w1);
      const u128 x = (ka ^ kb) & (m >= 16 ? ~(u128)0 : ~(~(u128)0 >> (8 * m)));
      const uint32_t za = first_zero_char(fa.w0, fa.w1);
      const uint64_t xh = k_hi(x), xl = k_lo(x);
      const uint32_t c = xh ? (uint32_t)__clzll((long long)xh) >> 3 : 8u + ((uint32_t)__clzll((long long)xl) >> 3);
      bool wtake = x != 0 ? ka < kb : fa.idx <= fb.idx;
      uint32_t lw = fa.h + (x != 0 ? c : za);
      const bool slow = both && eqh && x == 0 && za >= m;
      if (slow) wtake = cmp_from(a.chars, a.cap, fa.idx, fa.off, fb.idx, fb.off, fa.h + m, &lw) <= 0;
      // unequal LCPs decide without characters: the larger goes first, the
      // loser keeps its LCP
      const bool take_a = a_ok && (!b_ok || (eqh ? wtake : fa.h > fb.h));
      // after a comparison of equal LCPs the loser's LCP with the last output
      // becomes lw: its cache shifts by lw - h, or, after reading the strings,
      // is reloaded at lw
      const bool moved = both && eqh;
      const uint64_t loff = take_a ? fb.off : fa.off;
      WindowWords<2> ww;
      if (slow) issue_windows<2>(a.chars, loff, lw, a.cap, ww);
      // the winner is output; its run moves on
      const MRec w = take_a ? fa : fb;
      if (act) {
        if (last) {
          a.out_perm[base + out] = w.idx;
          if (a.out_lcp) a.out_lcp[base + out] = out == 0 ? 0u : w.h;
        } else {
          MRec o = w;
          if (out == 0) o.h = 0;
          store_mrec(a.dst + base + out, o);
        }
      }
      const uint32_t nia = ia + ((act && take_a) ? 1u : 0u);
      const uint32_t njb = jb + ((act && !take_a) ? 1u : 0u);
      const bool more = act && (take_a ? nia < ea : njb < eb);
      MRec nx{};
      if (more) nx = load_mrec(take_a ? A + nia : B + njb);
      // the loser's new cache
      MRec& lo = take_a ? fb : fa;
      uint64_t r0 = lo.w0, r1 = lo.w1;
      uint32_t rmiss = lo.miss;
      if (slow) {
        finish_words(ww, a.chars, a.cap, loff, lw, r0, r1);
        rmiss = 0;
      } else if (moved) {
        const uint32_t d = lw - lo.h;  // < m: the cache keeps at least one valid character
        const u128 sk = d ? (make_k(r0, r1) << (8 * d)) : make_k(r0, r1);
        r0 = k_hi(sk);
        r1 = k_lo(sk);
        rmiss += d;
      }
      if (act) {
        if (moved) {
          lo.h = lw;
          lo.w0 = r0;
          lo.w1 = r1;
          lo.miss = rmiss;
        }
        if (more) {
          if (take_a) fa = nx; else fb = nx;
        }
      }
      ia = nia;
      jb = njb;
      out += act ? 1u : 0u;
    }
  }
}

__global__ void k_merge_copy(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ lcp, uint32_t n,
                             uint32_t* __restrict__ out_perm, uint32_t* __restrict__ out_lcp) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    out_perm[j] = perm[j];
    if (out_lcp) out_lcp[j] = j ? lcp[j] : 0u;
  }
}

// Strings packed one after the other in index order: string i starts after
// string i - 1's terminator.  A set that passes can be sorted in parts while
// later parts are still being copied (each part's strings lie in its own
// stretch of chars).
__global__ void k_layout_check(const uint8_t* __restrict__ chars, uint64_t chars_len,
                               const uint64_t* __restrict__ offsets, uint32_t n, uint32_t* bad) {
  bool ok = true;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t o = offsets[i];
    const uint64_t e = i + 1 < n ? offsets[i + 1] : chars_len;
    ok = ok && o < e && e <= chars_len && chars[e - 1] == 0;
  }
  if (__syncthreads_or(!ok) && threadIdx.x == 0) *bad = 1u;
}

uint32_t grid_for(uint64_t items, uint32_t block, uint32_t sms, uint32_t per_sm) {
  const uint64_t g = (items + block - 1) / block;
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)sms * per_sm));
}

}  // namespace

cudaError_t launch_merge_prep(const MergePrepArgs& a, uint32_t sms, cudaStream_t st, const LaunchHook& hook) {
  hook.run("merge_prep", [&] { k_merge_prep<<<grid_for(a.total, 256, sms, 16), 256, 0, st>>>(a); });
  return cudaGetLastError();
}

cudaError_t launch_merge_round(const MergeRoundArgs& a, uint32_t sms, cudaStream_t st, const LaunchHook& hook) {
  if (a.nsamples) {
    hook.run("merge_cut", [&] { k_merge_cut<<<grid_for(a.nsamples, 256, sms, 16), 256, 0, st>>>(a); });
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const uint32_t pieces = a.nsamples + (a.ncur + 1) / 2;
  hook.run("merge_round",
           [&] { k_merge_round<<<grid_for(pieces, kMergeBlock, sms, 16), kMergeBlock, 0, st>>>(a); });
  return cudaGetLastError();
}

cudaError_t launch_merge_copy(const uint32_t* perm, const uint32_t* lcp, uint32_t n, uint32_t* out_perm,
                              uint32_t* out_lcp, uint32_t sms, cudaStream_t st, const LaunchHook& hook) {
  hook.run("merge_round",
           [&] { k_merge_copy<<<grid_for(n, 256, sms, 16), 256, 0, st>>>(perm, lcp, n, out_perm, out_lcp); });
  return cudaGetLastError();
}

cudaError_t launch_layout_check(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets, uint32_t n,
                                uint32_t* bad, uint32_t sms, cudaStream_t st, const LaunchHook& hook) {
  hook.run("layout_check",
           [&] { k_layout_check<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(chars, chars_len, offsets, n, bad); });
  return cudaGetLastError();
}

}  // namespace ss
