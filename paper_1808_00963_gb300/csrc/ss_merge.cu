// K-way LCP-aware merge of sorted runs (Section 4.3.2, Algorithm 4.5) and its
// parallel splitting into independent pieces (Section 4.3.3).
//
// Splitting.  Every S-th string of every run is a sample.  k_merge_cut gives
// each sample its cut vector: for every run j, the number of strings of run j
// that are <= the sample in the order (string, index), found by a binary
// search that skips the prefix every string between the two bounds shares
// with the sample; the sum is the sample's rank (its end position in the
// output).  The pieces are the stretches of the output between consecutive
// samples in rank order.  A sample's predecessor in that order is the largest
// -ranked of the runs' last samples below it, found by a binary search per
// run over that run's sample ranks (increasing, as the run is sorted), so no
// sample sort is needed.
//
// Merging.  One warp merges one piece; each lane holds the front strings of
// its runs with h = the LCP of the front with the last output string p (the
// common predecessor LCP-Compare, Algorithm 4.2, needs) and the 8 characters
// from depth h on (the distinguishing characters of the caching variant of
// Section 4.3.4, 8 at a time).  Each output is one tournament over all fronts,
// played as warp reductions instead of a replay of one root path of a loser
// tree: unequal LCPs decide without reading characters (the larger LCP goes
// first), equal LCPs compare the cached windows and read further windows only
// for fronts that are still tied.  As in Algorithm 4.5, the LCP of the winner
// is its h, and the string that replaces it enters with h = its LCP entry in
// its run; every other front's h becomes its LCP with the winner (unchanged
// below the maximum, from the compared windows at the maximum).  The first
// output of a piece gets its LCP by one direct comparison with the sample that
// ends the previous piece (the string just before it).
#include "../../include/ss_sort.h"
#include "ss_kernels.h"

namespace ss {

namespace {

constexpr uint32_t kNoRun = 0xFFFFFFFFu;
constexpr uint32_t kMergeBlock = 128;  // 4 warps

// Lanes of a warp are split into groups of G lanes (G = the padded run count,
// at least 4, at most 32); each group works on its own sample or piece, and
// each lane of a group holds run t * G + (lane % G) for t < NS.
template <int G>
struct Group {
  uint32_t lane, g, glane, mask;
  __device__ __forceinline__ Group() {
    lane = threadIdx.x & 31;
    g = lane / G;
    glane = lane % G;
    mask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1) << (g * G));
  }
  // index of this group among all groups of the grid
  __device__ __forceinline__ uint32_t id() const {
    return (blockIdx.x * (kMergeBlock / 32) + (threadIdx.x >> 5)) * (32 / G) + g;
  }
};

__device__ __forceinline__ uint64_t cache_at(const MergeParams& m, uint64_t off, uint32_t h) {
  return load_cache_2w(m.chars, off, h, m.cap);
}

// Compares string a (index ia, at offset oa) with string b (ib, ob); both
// share their first h characters (and neither ends before h).  Returns <0 / 0
// / >0 in the order (string, index) and sets *l = lcp(a, b).
__device__ __forceinline__ int cmp_from(const MergeParams& m, uint32_t ia, uint64_t oa, uint32_t ib, uint64_t ob,
                                        uint32_t h, uint32_t* l) {
  while (true) {
    const uint64_t ca = cache_at(m, oa, h);
    const uint64_t cb = cache_at(m, ob, h);
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

// The run that sample i belongs to (sample_base is non-decreasing in k).
__device__ __forceinline__ uint32_t sample_run(const MergeParams& m, uint32_t i) {
  uint32_t lo = 0, hi = m.K;  // last k with sample_base[k] <= i
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (m.run[mid].sample_base <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t sample_pos(const MergeParams& m, uint32_t k, uint32_t i) {
  return (i - m.run[k].sample_base + 1) * m.S - 1;
}

// Cut vectors and ranks; one lane group per sample, one lane per run.
template <int G, int NS>
__global__ void __launch_bounds__(kMergeBlock) k_merge_cut(MergeParams m) {
  const Group<G> gr;
  const uint32_t groups = gridDim.x * (kMergeBlock / 32) * (32 / G);
  for (uint32_t i = gr.id(); i < m.C; i += groups) {
    const uint32_t k = sample_run(m, i);
    const uint32_t p = sample_pos(m, k, i);
    const uint32_t sidx = m.run[k].perm[p];
    const uint64_t soff = m.offsets[sidx];
    uint32_t sum = 0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const uint32_t j = t * G + gr.glane;
      if (j >= m.K) continue;
      uint32_t cut;
      if (j == k) {
        cut = p + 1;
      } else {
        const uint32_t* perm = m.run[j].perm;
        uint32_t lo = 0, hi = m.run[j].n, llo = 0, lhi = 0;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          const uint32_t e = perm[mid];
          uint32_t l;
          const int c = cmp_from(m, e, m.offsets[e], sidx, soff, llo < lhi ? llo : lhi, &l);
          if (c <= 0) { lo = mid + 1; llo = l; } else { hi = mid; lhi = l; }
        }
        cut = lo;
      }
      m.cut[(size_t)i * m.K + j] = cut;
      sum += cut;
    }
    sum = __reduce_add_sync(gr.mask, sum);
    if (gr.glane == 0) m.rank[i] = sum;
  }
}

// Common prefix of two 8-character windows at the same depth, in characters:
// up to the first difference, or up to the terminator when they are equal and
// hold one (the strings end there), else all 8.
__device__ __forceinline__ uint32_t window_lcp(uint64_t a, uint64_t b) {
  return a != b ? lcp8(a, b) : (has_nul(a) ? nnz_prefix(a) : 8u);
}

// Group minimum of a 64-bit value (every lane of the group takes part; lanes
// without a candidate pass ~0).
__device__ __forceinline__ uint64_t group_min_u64(uint32_t mask, uint64_t v) {
  const uint32_t hi = __reduce_min_sync(mask, (uint32_t)(v >> 32));
  const uint32_t lo = __reduce_min_sync(mask, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0xFFFFFFFFu);
  return ((uint64_t)hi << 32) | lo;
}

// ---- 16-character windows loaded ahead of use --------------------------------------------
//
// A load is split into issuing the aligned words (Raw16) and reading them out
// (finish16) so that the memory round trip overlaps the tournaments that run
// in between.  The three words covering characters [h, h + 16) are issued at
// once only when they lie in the 4 KiB block that holds character h (the
// string or its terminator is in that block, so the reads cannot fault);
// otherwise the window is read later with the terminator-checked load.

struct Raw16 {
  uint64_t x0, x1, x2;
  uint64_t off;
  uint32_t h;
  uint32_t ok;   // 1: the words were issued
};

__device__ __forceinline__ void raw16_issue(const MergeParams& m, uint64_t off, uint32_t h, Raw16& r) {
  r.off = off;
  r.h = h;
  const uintptr_t a = (uintptr_t)(m.chars + off + h);
  const uintptr_t p = a & ~(uintptr_t)7;
  r.ok = (h < m.cap) && (p + 24 <= ((a | 4095u) + 1));
  if (r.ok) {
    const uint64_t* w = reinterpret_cast<const uint64_t*>(p);
    r.x0 = __ldg(w);
    r.x1 = __ldg(w + 1);
    r.x2 = __ldg(w + 2);
  } else {
    r.x0 = r.x1 = r.x2 = 0;
  }
}

// Raw little-endian bytes of a window, cut at the terminator or after `room`
// characters, as a big-endian key.
__device__ __forceinline__ uint64_t finish_window(uint64_t v, uint32_t room) {
  const uint32_t z = first_zero_byte(v);
  const uint32_t keep = z < room ? z : room;
  if (keep < 8) v &= keep == 0 ? 0ull : (~0ull >> (64 - 8 * keep));
  return bswap64(v);
}

// The window at depth h of a Raw16.
__device__ __forceinline__ uint64_t finish8(const MergeParams& m, const Raw16& r) {
  if (r.h >= m.cap) return 0;
  if (!r.ok) return cache_at(m, r.off, r.h);
  const uint32_t sh = (uint32_t)((uintptr_t)(m.chars + r.off + r.h) & 7) * 8;
  return finish_window(sh ? (r.x0 >> sh) | (r.x1 << (64 - sh)) : r.x0, m.cap - r.h);
}

// The windows at depths h and h + 8 of a Raw16.
__device__ __forceinline__ void finish16(const MergeParams& m, const Raw16& r, uint64_t& w0, uint64_t& w1) {
  if (r.h >= m.cap) {
    w0 = w1 = 0;
    return;
  }
  const uint32_t room = m.cap - r.h;
  if (r.ok) {
    const uint32_t sh = (uint32_t)((uintptr_t)(m.chars + r.off + r.h) & 7) * 8;
    const uint64_t v0 = sh ? (r.x0 >> sh) | (r.x1 << (64 - sh)) : r.x0;
    const uint64_t v1 = sh ? (r.x1 >> sh) | (r.x2 << (64 - sh)) : r.x1;
    w0 = finish_window(v0, room);
    w1 = (has_nul(w0) || room <= 8) ? 0ull : finish_window(v1, room - 8);
  } else {
    w0 = cache_at(m, r.off, r.h);
    w1 = (has_nul(w0) || room <= 8) ? 0ull : cache_at(m, r.off, r.h + 8);
  }
}

// One run of a piece as seen by its lane.  The front string is compared: its
// index, h = LCP with the last output, w0 = the 8 characters from depth h and
// the next 8 (w1, read out of the pending words `fr` when first needed).  The
// next string has its words in flight, the one after it its index, LCP entry
// and offset.
struct Slot {
  uint32_t pos, end;             // front at pos; valid while pos < end
  uint32_t fidx, fh;
  uint64_t fw0, fw1;
  Raw16 fr;                      // pending words for fw1 (fpend)
  bool fpend;
  uint32_t nidx;
  Raw16 nr;                      // next string: words at depth nr.h (its LCP entry)
  uint32_t n2idx, n2h;
  uint64_t n2off;
};

__device__ __forceinline__ void slot_fetch(const MergeParams& m, const MergeRun& r, uint32_t p, uint32_t end,
                                           uint32_t& idx, uint32_t& h, uint64_t& off) {
  if (p < end) {
    idx = r.perm[p];
    h = r.lcp[p];
    off = m.offsets[idx];
  } else {
    idx = 0;
    h = 0;
    off = 0;
  }
}

__device__ __forceinline__ void slot_init(const MergeParams& m, const MergeRun& r, Slot& s, uint32_t pos,
                                          uint32_t end) {
  s.pos = pos;
  s.end = end;
  uint32_t h;
  uint64_t off;
  slot_fetch(m, r, pos, end, s.fidx, h, off);  // the first string of a run in the piece: h = 0
  uint32_t nh;
  uint64_t noff;
  slot_fetch(m, r, pos + 1, end, s.nidx, nh, noff);
  slot_fetch(m, r, pos + 2, end, s.n2idx, s.n2h, s.n2off);
  s.fh = 0;
  s.fpend = false;
  s.fr.ok = 0;
  if (pos < end) {
    Raw16 r0;
    raw16_issue(m, off, 0, r0);
    finish16(m, r0, s.fw0, s.fw1);
    s.fr = r0;
  } else {
    s.fw0 = s.fw1 = 0;
    s.fr.off = 0;
    s.fr.h = 0;
  }
  if (pos + 1 < end) raw16_issue(m, noff, nh, s.nr);
  else s.nr.ok = 0, s.nr.off = 0, s.nr.h = 0;
}

__device__ __forceinline__ uint64_t slot_w1(const MergeParams& m, Slot& s) {
  if (s.fpend) {
    uint64_t w0;
    finish16(m, s.fr, w0, s.fw1);
    s.fpend = false;
  }
  return s.fw1;
}

__device__ __forceinline__ void slot_advance(const MergeParams& m, const MergeRun& r, Slot& s) {
  ++s.pos;
  s.fidx = s.nidx;
  s.fh = s.nr.h;
  s.fr = s.nr;
  s.fpend = false;
  if (s.pos < s.end) {
    s.fw0 = finish8(m, s.nr);
    s.fpend = !has_nul(s.fw0);  // w1 is read out of the same words when first needed
    if (!s.fpend) s.fw1 = 0;
  }
  s.nidx = s.n2idx;
  if (s.pos + 1 < s.end) raw16_issue(m, s.n2off, s.n2h, s.nr);
  slot_fetch(m, r, s.pos + 2, s.end, s.n2idx, s.n2h, s.n2off);
}

// The front lost with LCP lw > fh to the winner: move its windows to depth lw.
__device__ __forceinline__ void slot_deepen(const MergeParams& m, Slot& s, uint32_t lw) {
  const uint32_t d = lw - s.fh;
  const uint64_t off = s.fr.off;
  if (d < 8) {
    const uint64_t w1 = slot_w1(m, s);
    s.fw0 = (s.fw0 << (8 * d)) | (w1 >> (64 - 8 * d));
  } else if (d == 8) {
    s.fw0 = slot_w1(m, s);
  } else {
    s.fw0 = cache_at(m, off, lw);
  }
  s.fh = lw;
  if (has_nul(s.fw0)) {
    s.fw1 = 0;
    s.fpend = false;
    s.fr.h = lw;
  } else {
    raw16_issue(m, off, lw, s.fr);
    s.fpend = true;
  }
}

// One lane group merges one piece at a time, taking pieces from a counter.
// Every output is one LCP-aware tournament over the runs' front strings, all
// of which carry h = LCP with the last output p: the largest h goes first
// (cases 2 and 3 of LCP-Compare, no characters read); among the fronts with
// that h the 8 cached characters decide, then further 8-character windows of
// the fronts still tied, then the index (then the run, for an index present
// in two runs).  Afterwards every front's h becomes its LCP with the string
// just written: unchanged below the maximum, and from the compared windows for
// the fronts that had it.  The winner's run moves on; its next string enters
// with h = its LCP entry in the run.  Outputs are buffered one per lane and
// written G at a time.
template <int G, int NS>
__global__ void __launch_bounds__(kMergeBlock) k_merge_pieces(MergeParams m) {
  const Group<G> gr;
  const uint32_t gm = gr.mask;
  while (true) {
    uint32_t q = 0;
    if (gr.glane == 0) q = atomicAdd(m.next_piece, 1u);
    q = __shfl_sync(gm, q, gr.g * G);
    if (q > m.C) return;  // uniform within the group
    // predecessor sample: the largest rank below this piece's end sample
    const uint64_t rq = q < m.C ? (uint64_t)m.rank[q] : ~0ull;
    uint32_t best = 0, best_id = 0;  // rank + 1 of this lane's best candidate
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const uint32_t j = t * G + gr.glane;
      if (j >= m.K) continue;
      const uint32_t base = m.run[j].sample_base;
      uint32_t lo = 0, hi = m.run[j].n / m.S;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)m.rank[base + mid] < rq) lo = mid + 1; else hi = mid;
      }
      if (lo > 0 && m.rank[base + lo - 1] + 1 > best) {
        best = m.rank[base + lo - 1] + 1;
        best_id = base + lo - 1;
      }
    }
    const uint32_t pbest = __reduce_max_sync(gm, best);
    uint32_t pred = kNoRun;
    if (pbest > 0) {
      const uint32_t owner = __ffs(__ballot_sync(gm, best == pbest)) - 1;
      pred = __shfl_sync(gm, best_id, owner);
    }
    Slot sl[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const uint32_t j = t * G + gr.glane;
      uint32_t p0 = 0, e0 = 0;
      if (j < m.K) {
        p0 = pred == kNoRun ? 0u : m.cut[(size_t)pred * m.K + j];
        e0 = q < m.C ? m.cut[(size_t)q * m.K + j] : m.run[j].n;
      }
      slot_init(m, m.run[j < m.K ? j : 0], sl[t], p0, e0);
    }
    uint32_t out = pred == kNoRun ? 0u : pbest - 1;
    uint32_t pred_idx = 0;
    uint64_t pred_off = 0;
    if (pred != kNoRun) {
      const uint32_t k = sample_run(m, pred);
      pred_idx = m.run[k].perm[sample_pos(m, k, pred)];
      pred_off = m.offsets[pred_idx];
    }
    bool first = true;
    uint32_t cnt = 0, ob_idx = 0, ob_lcp = 0;
    while (true) {
      uint32_t hk = 0;
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (sl[t].pos < sl[t].end && sl[t].fh + 1 > hk) hk = sl[t].fh + 1;
      const uint32_t H1 = __reduce_max_sync(gm, hk);
      if (H1 == 0) break;
      const uint32_t H = H1 - 1;
      bool cand[NS];
      uint32_t ncand = 0, cslot = 0;
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        cand[t] = sl[t].pos < sl[t].end && sl[t].fh == H;
        const uint32_t b = __ballot_sync(gm, cand[t]);
        if (b) cslot = t * G + (__ffs(b) - 1) % G;
        ncand += __popc(b);
      }
      bool in[NS];
      uint32_t lw[NS];
      uint32_t wid, imin;
      if (ncand == 1) {
        // one front has the largest LCP with the last output: it goes first
        // (cases 2/3 of LCP-Compare), and no other front's LCP changes
        wid = cslot;
        uint32_t wi = 0;
#pragma unroll
        for (int t = 0; t < NS; ++t) {
          in[t] = cand[t];
          lw[t] = sl[t].fh;
          if (cand[t]) wi = sl[t].fidx;
        }
        imin = __shfl_sync(gm, wi, gr.g * G + wid % G);
      } else {
      uint64_t cm = ~0ull;
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (cand[t] && sl[t].fw0 < cm) cm = sl[t].fw0;
      const uint64_t cmin = group_min_u64(gm, cm);
      uint32_t nin = 0;
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        in[t] = cand[t] && sl[t].fw0 == cmin;
        lw[t] = cand[t] ? H + window_lcp(sl[t].fw0, cmin) : sl[t].fh;
        nin += in[t];
      }
      nin = __reduce_add_sync(gm, nin);
      if (nin > 1) {
        uint64_t key = cmin;
        uint32_t depth = H;
        while (!has_nul(key)) {  // tied fronts continue past this window: compare the next one
          depth += 8;
          uint64_t c2[NS];
          uint64_t mm = ~0ull;
#pragma unroll
          for (int t = 0; t < NS; ++t) {
            c2[t] = ~0ull;
            if (in[t]) c2[t] = depth == H + 8 ? slot_w1(m, sl[t]) : cache_at(m, sl[t].fr.off, depth);
            if (c2[t] < mm) mm = c2[t];
          }
          key = group_min_u64(gm, mm);
          uint32_t k2 = 0;
#pragma unroll
          for (int t = 0; t < NS; ++t) {
            if (in[t]) {
              lw[t] = depth + window_lcp(c2[t], key);
              if (c2[t] != key) in[t] = false;
            }
            k2 += in[t];
          }
          if (__reduce_add_sync(gm, k2) <= 1) break;
        }
      }
      // winner: smallest index among the fronts still tied, then the lowest slot
      uint32_t im = 0xFFFFFFFFu;
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (in[t] && sl[t].fidx < im) im = sl[t].fidx;
      imin = __reduce_min_sync(gm, im);
      uint32_t id = 0xFFFFFFFFu;
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (in[t] && sl[t].fidx == imin && t * G + gr.glane < id) id = t * G + gr.glane;
      wid = __reduce_min_sync(gm, id);
      }
      const uint32_t wlane = gr.g * G + wid % G;
      uint32_t olcp = H;
      if (first) {
        uint32_t l = 0;
        if (pred != kNoRun && wlane == gr.lane) {
          uint64_t woff = 0;
#pragma unroll
          for (int t = 0; t < NS; ++t)
            if ((uint32_t)t == wid / G) woff = sl[t].fr.off;
          cmp_from(m, pred_idx, pred_off, imin, woff, 0, &l);
        }
        olcp = __shfl_sync(gm, l, wlane);
        first = false;
      }
      if (gr.glane == cnt) {
        ob_idx = imin;
        ob_lcp = olcp;
      }
      if (++cnt == G) {
        m.out_perm[out + gr.glane] = ob_idx;
        if (m.out_lcp) m.out_lcp[out + gr.glane] = ob_lcp;
        out += G;
        cnt = 0;
      }
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        if ((uint32_t)t * G + gr.glane == wid) slot_advance(m, m.run[t * G + gr.glane], sl[t]);
        else if (cand[t] && lw[t] != sl[t].fh) slot_deepen(m, sl[t], lw[t]);
      }
    }
    if (gr.glane < cnt) {
      m.out_perm[out + gr.glane] = ob_idx;
      if (m.out_lcp) m.out_lcp[out + gr.glane] = ob_lcp;
    }
  }
}

template <int G, int NS>
cudaError_t launch_merge_g(const MergeParams& m, uint32_t sms, cudaStream_t st, const LaunchHook& hook) {
  constexpr uint32_t per_block = (kMergeBlock / 32) * (32 / G);
  if (m.C > 0) {
    const uint32_t cut_grid = std::max(1u, std::min(sms * 16, (m.C + per_block - 1) / per_block));
    hook.run("merge_cut", [&] { k_merge_cut<G, NS><<<cut_grid, kMergeBlock, 0, st>>>(m); });
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  static int resident = 0;  // blocks per SM (the same on every device this library runs on)
  if (resident == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_merge_pieces<G, NS>, kMergeBlock, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    resident = b;
  }
  const uint32_t grid = std::max(1u, std::min(sms * (uint32_t)resident, (m.C + 1 + per_block - 1) / per_block));
  hook.run("merge_pieces", [&] { k_merge_pieces<G, NS><<<grid, kMergeBlock, 0, st>>>(m); });
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_merge(const MergeParams& m, uint32_t logk, uint32_t sms, cudaStream_t st,
                         const LaunchHook& hook) {
  switch (logk) {
    case 0: case 1: case 2: return launch_merge_g<4, 1>(m, sms, st, hook);
    case 3: return launch_merge_g<8, 1>(m, sms, st, hook);
    case 4: return launch_merge_g<16, 1>(m, sms, st, hook);
    case 5: return launch_merge_g<32, 1>(m, sms, st, hook);
    case 6: return launch_merge_g<32, 2>(m, sms, st, hook);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ss
