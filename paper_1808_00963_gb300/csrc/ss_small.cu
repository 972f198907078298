// Small subsets, initial set-up and the final LCP fix-up.
//
// A subset of at most small_cutoff strings with a common prefix of `depth`
// characters is finished by one block (33..cutoff strings) or one warp (2..32)
// without further distribution steps: its records are sorted by
// (segment, cache, index) in shared memory or registers; runs of equal caches
// without a terminator are refined by reloading their caches 8 characters
// deeper and sorting again (the recursion of the equality buckets of
// Section 4.2.2, done in place).  This replaces the paper's sequential base
// cases (caching multikey quicksort and insertion sort, Section 4.2.8) with
// sorting networks that suit a warp or a block.  LCPs between neighbours are
// computed from the caches as they are separated (Section 4.2.3, "LCP via
// XOR").
#include "ss_kernels.h"
#include "ss_step.cuh"

namespace ss {

namespace {

__device__ __forceinline__ uint32_t find_set(const SortCtx& c, uint32_t r) {
  uint32_t lo = 0, hi = c.num_sets - 1;  // last set with base <= r
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (c.sets[mid].base <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Records of every set at depth 0, in index order (the stable starting point).
__global__ void __launch_bounds__(kBlock) k_init(SortCtx c) {
  const uint32_t stride = gridDim.x * blockDim.x;
  unsigned long long bytes = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < c.total; r += stride) {
    const uint32_t s = c.num_sets == 1 ? 0 : find_set(c, r);
    const SetDesc sd = c.sets[s];
    const uint32_t i = r - sd.base;
    const uint64_t off = sd.offsets[i];
    if ((off >> 32) && !c.wide[s]) atomicOr(c.wide + s, 1u);
    if (c.big_enabled && sd.n > c.big_threshold) {  // a multi-block root: wide records
      store_wkey(c.rec[0] + r, load_key128(sd.chars, off, 0, sd.cap, sd.dna));
      c.wid[0][r] = make_uint2(i, (uint32_t)off);
      bytes += 48;  // offset 8 + 16 characters read, wide record 24 written
    } else {
      store_rec(c.rec[0] + r, load_key(sd.chars, off, 0, sd.cap, sd.dna), i, (uint32_t)off);
      bytes += 32;  // offset 8 + 8 characters read, record 16 written
    }
  }
  account(c, kKInit, bytes);
}

// One root task per set.
__global__ void k_roots(SortCtx c) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= c.num_sets) return;
  const SetDesc sd = c.sets[s];
  if (sd.n == 0) return;
  if (sd.lcp) sd.lcp[0] = 0;
  if (sd.n == 1) { sd.perm[0] = 0; return; }
  route_task(c, Task{sd.base, sd.n, 0, make_meta(s, 0)}, c.big_cur);
}

// ---- warp-level refinement ----------------------------------------------------

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Order of the warp sort: (segment, key, source lane); tag = segment << 5 |
// source lane, segment 32 for idle lanes.  Evaluated without branches.
__device__ __forceinline__ bool wtag_less(uint64_t ka, uint32_t ta, uint64_t kb, uint32_t tb) {
  const uint32_t sa = ta >> 5, sb = tb >> 5;
  return (sa < sb) | ((sa == sb) & ((ka < kb) | ((ka == kb) & (ta < tb))));
}

// Bitonic sort of one (key, tag) per lane, ascending in lane order.
__device__ __forceinline__ void warp_sort(uint32_t& tag, uint64_t& key) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint32_t ot = __shfl_xor_sync(kFull, tag, j);
      const uint64_t ok = __shfl_xor_sync(kFull, key, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool take = (lower == up) ? wtag_less(ok, ot, key, tag) : wtag_less(key, tag, ok, ot);
      tag = take ? ot : tag;
      key = take ? ok : key;
    }
  }
}

// Finishes the subsets ("groups") held by a warp, one string per lane.  Lanes
// [g0, g0 + glen) hold one group: strings with a common prefix of their
// `depth` characters, in ascending index order, with key = their cache at that
// depth.  Lane-static (they do not move): active, g0, chars/cap of the group's
// set and lcp_g, the LCP output at the group's first position.  Sorting by
// (segment, cache, index) splits a group into runs of equal caches; a run of
// one string or of equal strings (cache holds the terminator) is finished;
// every other run jumps over the characters all its members share, found with
// a 64-character look-ahead, and is sorted again.  Writes lcp_g[j] for every
// position j > 0 of each group and returns the index at the lane's position.
// With max_jumps > 0, runs still open after that many look-aheads are handed
// to defer(position in group, run's first position, run length, cache, index,
// offset, depth) on each of their lanes and left unfinished: a few long
// common prefixes would otherwise keep whole warps busy while most of their
// lanes idle (their lcp_g entries after the run's first one stay unwritten).
template <typename Defer>
__device__ uint32_t warp_refine(bool active, uint32_t g0, uint32_t nact, uint64_t key, uint32_t idx,
                                uint64_t off, uint32_t depth, uint32_t cap, const uint8_t* chars, uint32_t dna,
                                uint32_t* lcp_g, uint32_t* status, unsigned long long& bytes, uint32_t max_jumps,
                                Defer&& defer) {
  const uint32_t lane = lane_id();
  uint32_t seg = active ? g0 : 0xFFFFFFFFu;
  uint32_t open = active ? 1u : 0u;
  uint32_t jumps = 0;
  if (!active) { key = ~0ull; idx = 0xFFFFFFFFu; off = 0; depth = 0; }
  const uint32_t upto = (lane == 31) ? kFull : ((2u << lane) - 1);
  while (true) {
    // sort only if some run is out of (cache, index) order: after a look-ahead
    // jump over characters all members share, the runs often still are
    {
      const uint32_t ps0 = __shfl_up_sync(kFull, seg, 1);
      const uint64_t pk0 = __shfl_up_sync(kFull, key, 1);
      const uint32_t pi0 = __shfl_up_sync(kFull, idx, 1);
      const bool disorder = active && lane > 0 && seg == ps0 && (key < pk0 || (key == pk0 && idx < pi0));
      if (__any_sync(kFull, disorder)) {
        // Segments occupy fixed lanes, and depth and open are the same for
        // every member of a segment, so only the key and the source lane
        // move; ties go by source lane, which within a segment is index
        // order.  Index and offset follow from the source lane.
        uint32_t tag = ((active ? seg : 32u) << 5) | lane;
        warp_sort(tag, key);
        const uint32_t src = tag & 31u;
        idx = __shfl_sync(kFull, idx, src);
        off = __shfl_sync(kFull, off, src);
      }
    }
    const uint32_t ps = __shfl_up_sync(kFull, seg, 1);
    const uint64_t pk = __shfl_up_sync(kFull, key, 1);
    const bool start = lane == 0 || seg != ps || key != pk;
    if (active && open && lane > g0 && seg == ps && key != pk && lcp_g) lcp_g[lane - g0] = depth + key_lcp(pk, key, dna);
    const uint32_t starts = __ballot_sync(kFull, active && start);
    const uint32_t my_start = 31 - __clz(starts & upto);
    const uint32_t above = starts & ~upto;
    const uint32_t next = above ? (uint32_t)(__ffs(above) - 1) : nact;
    if (active && open) {
      if (next - my_start == 1) {
        open = 0;
      } else if (key_end(key, dna)) {
        open = 0;
        if (lane != my_start && lcp_g) lcp_g[lane - g0] = depth + key_nnz(key, dna);
      }
    }
    if (active) seg = my_start;
    if (!__any_sync(kFull, active && open)) break;
    if (max_jumps && jumps == max_jumps) {
      if (active && open) defer(lane - g0, my_start - g0, next - my_start, key, idx, off, depth);
      break;
    }
    ++jumps;
    // look-ahead: the first window (8, 16, ... characters deeper) where the
    // members of the run differ or end; the run continues there
    uint64_t w[kLookWindows];
    uint32_t nwin = 0;
    const uint32_t kw = key_width(dna);
    if (active && open) nwin = load_key_windows<kLookWindows>(chars, off, depth + kw, cap, dna, w);
    const uint32_t segmask = (next >= 32 ? kFull : ((1u << next) - 1)) & ~((1u << my_start) - 1);
    uint32_t jstop = kLookWindows - 1;
    bool found = false;
#pragma unroll
    for (int j = 0; j < kLookWindows; ++j) {
      const uint64_t lw = __shfl_sync(kFull, w[j], my_start);
      const bool stop = active && open && ((uint32_t)j >= nwin || w[j] != lw || key_end(w[j], dna));
      const uint32_t b = __ballot_sync(kFull, stop) & segmask;
      if (!found && b) { jstop = (uint32_t)j; found = true; }
    }
    if (active && open) {
      const uint32_t nd = depth + kw * (jstop + 1);
      if (nd > kMaxDepth) {
        latch_status(status, kStTooDeep);
        open = 0;
      } else {
        uint64_t k = w[0];
#pragma unroll
        for (int j = 1; j < kLookWindows; ++j) if ((uint32_t)j == jstop) k = w[j];
        key = jstop < nwin ? k : load_key(chars, off, nd, cap, dna);
        depth = nd;
        bytes += 8ull * (jstop + 1);
      }
    }
  }
  return idx;
}

// Packs up to 16 items (lane k < nt holds item k's length, 1..32) into rounds
// of whole items that fit into 32 lanes, in order.  For each round calls
// round(active, g0, nact, k): the lane belongs to item k, whose first lane is
// g0; nact lanes are in use.
template <typename Round>
__device__ __forceinline__ void pack_rounds(uint32_t nt, uint32_t my_len, Round&& round) {
  const uint32_t lane = lane_id();
  const uint32_t upto = (lane == 31) ? kFull : ((2u << lane) - 1);
  uint32_t a = 0;
  while (a < nt) {
    const uint32_t mine = (lane < nt && lane >= a) ? my_len : 0u;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t fits = __ballot_sync(kFull, lane >= a && lane < nt && incl <= 32);
    const uint32_t b = 32 - __clz(fits);
    const uint32_t excl = incl - mine;
    const uint32_t startbits = __reduce_or_sync(kFull, (lane >= a && lane < b) ? (1u << excl) : 0u);
    const uint32_t nact = __shfl_sync(kFull, incl, b - 1);
    const uint32_t k = a + __popc(startbits & upto) - 1;
    const uint32_t g0 = 31 - __clz(startbits & upto);
    round(lane < nact, g0, nact, k);
    a = b;
  }
}

// Warps take runs of up to 16 consecutive small tasks and pack as many whole
// tasks as fit into 32 lanes per round.
constexpr uint32_t kPackChunk = 16;
// Passes over the warp tasks: look-aheads (64 characters each) a run may take
// in each pass before it is deferred to the next one (0: no limit).
constexpr uint32_t kWarpPassJumps[] = {1, 0};
constexpr uint32_t kWarpPasses = sizeof(kWarpPassJumps) / sizeof(kWarpPassJumps[0]);
static_assert(kWarpPassJumps[kWarpPasses - 1] == 0, "the last pass finishes every run");

// One pass over a list of warp tasks.  With max_jumps > 0, runs with long
// common prefixes are deferred to the list `out`: their records go back to
// the record buffer at their current positions, and each run becomes a task.
__global__ void __launch_bounds__(kBlock) k_small_warp(SortCtx c, TaskList list, TaskList out, uint32_t max_jumps) {
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t count = min(*list.count, list.cap);
  const uint32_t lane = lane_id();
  unsigned long long bytes = 0;
  // few tasks: one per warp (parallelism); many: up to 16 per warp (packing)
  const uint32_t chunk = min(kPackChunk, max(1u, (count + nwarps - 1) / nwarps));
  for (uint32_t c0 = warp * chunk; c0 < count; c0 += nwarps * chunk) {
    const uint32_t nt = min(chunk, count - c0);
    Task mt{0, 0, 0, 0};
    if (lane < nt) mt = list.items[c0 + lane];
    pack_rounds(nt, mt.len, [&](bool active, uint32_t g0, uint32_t nact, uint32_t k) {
      const uint32_t tb = __shfl_sync(kFull, mt.begin, k & 31);
      const uint32_t tdepth = __shfl_sync(kFull, mt.depth, k & 31);
      const uint32_t tmeta = __shfl_sync(kFull, mt.meta, k & 31);
      uint64_t key = 0, off = 0;
      uint32_t id = 0, cap = kNoCap, dna = 0;
      const uint8_t* chars = nullptr;
      uint32_t* lcp_g = nullptr;
      uint32_t* perm = nullptr;
      const uint32_t par = tmeta >> 31;
      if (active) {
        const SetDesc sd = c.sets[tmeta & 0x7FFFFFFFu];
        const uint32_t e = lane - g0;
        const Rec r = load_rec(c.rec[par] + tb + e);
        key = r.key;
        id = r.idx;
        off = rec_offset(sd, c.wide[tmeta & 0x7FFFFFFFu], r.idx, r.off);
        cap = sd.cap;
        chars = sd.chars;
        dna = sd.dna;
        lcp_g = sd.lcp ? sd.lcp + (tb - sd.base) : nullptr;
        perm = sd.perm + (tb - sd.base);
      }
      const uint32_t fin = warp_refine(
          active, g0, nact, key, id, off, tdepth, cap, chars, dna, lcp_g, c.status, bytes, max_jumps,
          [&](uint32_t e, uint32_t rs, uint32_t rl, uint64_t k, uint32_t ix, uint64_t o, uint32_t d) {
            store_rec(c.rec[par] + tb + e, k, ix, (uint32_t)o);
            bytes += 16;
            if (e == rs) list_push(out, Task{tb + rs, rl, d, tmeta}, c.status);
          });
      if (active) {
        perm[lane - g0] = fin;
        bytes += lcp_g ? 24 : 20;  // record 16 read; perm 4 (+ lcp 4) written
      }
    });
  }
  account(c, kKSmallWarp, bytes);
}

// ---- block-level refinement -------------------------------------------------------

// Element tags of the block sort: handed (1 bit) << 25 | segment (12 bits)
// << 13 | original position (12 bits) << 1 | open (1 bit).  Sorting by (segment, cache, tag)
// orders each segment by cache and, among equal caches, by original position
// (= ascending index).  Index and offset stay at the original position.
__device__ __forceinline__ uint32_t tag_seg(uint32_t t) { return (t >> 13) & 0xFFFu; }
constexpr uint32_t kHanded = 1u << 25;  // run passed on to the warp list
__device__ __forceinline__ uint32_t tag_pos(uint32_t t) { return (t >> 1) & 0xFFFu; }
__device__ __forceinline__ uint32_t make_tag(uint32_t seg, uint32_t pos, uint32_t open) {
  return (seg << 13) | (pos << 1) | open;
}

struct CtaSmem {  // carved from dynamic shared memory, pmax elements
  uint64_t* key;    // cache, in sorted position
  uint64_t* key2;   // second buffer of the merge sort
  uint32_t* tag2;
  uint64_t* off;    // string offset, by original position
  uint32_t* tag;    // in sorted position
  uint32_t* idx;    // index, by original position
  uint32_t* aux;    // segment sizes
  uint16_t* nseg;   // segment start of each position
};

// Order of the block sort: (segment, cache, tag), evaluated without branches.
// OneSeg: every element is in segment 0 and none is handed on (the first pass
// over a subset, which does nearly all of the block sorts' work), so the tags
// compare as original positions and the segment test drops out.
template <bool OneSeg>
__device__ __forceinline__ bool elem_less(uint64_t ka, uint32_t ta, uint64_t kb, uint32_t tb) {
  if (OneSeg) return (ka < kb) | ((ka == kb) & (ta < tb));
  const uint32_t sa = tag_seg(ta), sb = tag_seg(tb);
  return (sa < sb) | ((sa == sb) & ((ka < kb) | ((ka == kb) & (ta < tb))));
}

// Slots past the end of a subset: after every real element in elem_less order.
constexpr uint32_t kPadTag = 0xFFFFFFFFu;

// Bitonic sort of one (key, tag) per lane by elem_less, ascending in lane order.
// The stages of each merge level run as a loop: the smaller code was faster
// than the fully unrolled network in the block sort kernels.
template <bool OneSeg>
__device__ __forceinline__ void warp_sort_elems(uint64_t& key, uint32_t& tag) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll 1
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint32_t ot = __shfl_xor_sync(kFull, tag, j);
      const uint64_t ok = __shfl_xor_sync(kFull, key, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool take = (lower == up) ? elem_less<OneSeg>(ok, ot, key, tag) : elem_less<OneSeg>(key, tag, ok, ot);
      tag = take ? ot : tag;
      key = take ? ok : key;
    }
  }
}

// Stable block merge sort of (key, tag) at positions [0, n), n <= pmax.
// Each warp first sorts runs of 32 positions with a bitonic network in
// registers; then every merge pass doubles the run length, each thread
// producing ipt (<= 32) outputs of one merged pair of runs: it finds where its
// outputs start with a binary search along the merge path and merges
// sequentially.  Uses (key2, tag2) as the second buffer; the result ends in
// (m.key, m.tag).
template <uint32_t NT, bool OneSeg>
__device__ void block_sort(CtaSmem& m, uint32_t n) {
  uint32_t ipt = 1;
  while (ipt * NT < n) ipt <<= 1;
  for (uint32_t c0 = threadIdx.x & ~31u; c0 < n; c0 += NT) {
    const uint32_t p = c0 + lane_id();
    uint64_t k = p < n ? m.key[p] : ~0ull;
    uint32_t t = p < n ? m.tag[p] : kPadTag;
    warp_sort_elems<OneSeg>(k, t);
    if (p < n) {
      m.key[p] = k;
      m.tag[p] = t;
    }
  }
  __syncthreads();
  uint64_t* sk = m.key;
  uint32_t* st = m.tag;
  uint64_t* dk = m.key2;
  uint32_t* dt = m.tag2;
  for (uint32_t run = 32; run < n; run <<= 1) {
    const uint32_t out = threadIdx.x * ipt;
    if (out < n) {
      const uint32_t base = (out / (2 * run)) * (2 * run);
      const uint32_t la = min(run, n - base);
      const uint32_t lb = base + run < n ? min(run, n - base - run) : 0u;
      const uint64_t* ak = sk + base;
      const uint32_t* at = st + base;
      const uint64_t* bk = sk + base + run;
      const uint32_t* bt = st + base + run;
      const uint32_t d = out - base;
      uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
      while (lo < hi) {  // number of A elements among the first d outputs
        const uint32_t mid = (lo + hi) >> 1;
        if (!elem_less<OneSeg>(bk[d - mid - 1], bt[d - mid - 1], ak[mid], at[mid])) lo = mid + 1;
        else hi = mid;
      }
      uint32_t i = lo, j = d - lo;
      const uint32_t cnt = min(ipt, n - out);
      for (uint32_t q = 0; q < cnt; ++q) {
        const bool take_a = i < la && (j >= lb || !elem_less<OneSeg>(bk[j], bt[j], ak[i], at[i]));
        if (take_a) {
          dk[out + q] = ak[i];
          dt[out + q] = at[i];
          ++i;
        } else {
          dk[out + q] = bk[j];
          dt[out + q] = bt[j];
          ++j;
        }
      }
    }
    __syncthreads();
    uint64_t* tk = sk; sk = dk; dk = tk;
    uint32_t* tt = st; st = dt; dt = tt;
  }
  if (sk != m.key) {
    for (uint32_t j = threadIdx.x; j < n; j += NT) {
      m.key[j] = sk[j];
      m.tag[j] = st[j];
    }
    __syncthreads();
  }
}

// Inclusive max-scan of a[0..n) in place.
template <uint32_t NT>
__device__ void block_max_scan(uint16_t* a, uint32_t n) {
  constexpr uint32_t NW = NT / 32;
  __shared__ uint32_t wmax[NW];
  const uint32_t per = (n + NT - 1) / NT;
  const uint32_t b0 = threadIdx.x * per;
  uint32_t m = 0;
  for (uint32_t j = 0; j < per && b0 + j < n; ++j) m = max(m, (uint32_t)a[b0 + j]);
  uint32_t inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, inc, o);
    if (lane_id() >= (uint32_t)o) inc = max(inc, t);
  }
  const uint32_t w = threadIdx.x >> 5;
  if (lane_id() == 31) wmax[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane_id() < NW ? wmax[lane_id()] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, v, o);
      if (lane_id() >= (uint32_t)o) v = max(v, t);
    }
    if (lane_id() < NW) wmax[lane_id()] = v;
  }
  __syncthreads();
  uint32_t excl = __shfl_up_sync(kFull, inc, 1);
  if (lane_id() == 0) excl = 0;
  uint32_t run = max(excl, w ? wmax[w - 1] : 0u);
  for (uint32_t j = 0; j < per && b0 + j < n; ++j) {
    run = max(run, (uint32_t)a[b0 + j]);
    a[b0 + j] = (uint16_t)run;
  }
  __syncthreads();
}

// The narrow launch (narrow = 1) sorts the subsets of c.small_cta, the wide
// one those of c.small_cta_wide; while there are fewer than min_count subsets
// in all, the narrow launch leaves every subset to the wide one.  Each block
// claims one subset at a time from its launch's counter (subset sizes vary
// several-fold, so a fixed share per block left many SMs idle at the end).
template <uint32_t NT, bool DNA>
__global__ void __launch_bounds__(NT) k_small_cta(SortCtx c, uint32_t pmax, uint32_t min_count, uint32_t narrow) {
  constexpr uint32_t dna = DNA ? 1u : 0u;  // the character encoding, fixed per instance
  extern __shared__ __align__(16) uint8_t smem[];
  CtaSmem m;
  m.key = reinterpret_cast<uint64_t*>(smem);
  m.key2 = m.key + pmax;
  m.off = m.key2 + pmax;
  m.tag = reinterpret_cast<uint32_t*>(m.off + pmax);
  m.tag2 = m.tag + pmax;
  m.idx = m.tag2 + pmax;
  m.aux = m.idx + pmax;
  m.nseg = reinterpret_cast<uint16_t*>(m.aux + pmax);
  __shared__ uint32_t s_max_open, s_jstop, s_neq;
  __shared__ uint64_t s_lead[kLookWindows];
  unsigned long long bytes = 0;
  const uint32_t n_narrow = min(*c.small_cta.count, c.small_cta.cap);
  const uint32_t n_wide = min(*c.small_cta_wide.count, c.small_cta_wide.cap);
  const bool few = n_narrow + n_wide < min_count;
  if (narrow && few) return;
  // this launch's subsets: the first na of the narrow list, then the wide list
  const uint32_t na = (narrow || few) ? n_narrow : 0u;
  const uint32_t count = narrow ? n_narrow : na + n_wide;
  uint32_t* claim = c.small_claim + (narrow ? 0 : 1);
  __shared__ uint32_t s_ti;
  if (threadIdx.x == 0) s_ti = atomicAdd(claim, 1u);
  __syncthreads();
  for (uint32_t ti = s_ti; ti < count; ti = s_ti) {
    const Task t = ti < na ? c.small_cta.items[ti] : c.small_cta_wide.items[ti - na];
    __syncthreads();  // every thread has read s_ti
    if (threadIdx.x == 0) s_ti = atomicAdd(claim, 1u);  // the next subset, claimed while this one sorts
    if (t.len > pmax) {  // cannot happen: a list holds only sizes its launch's shared arrays take
      if (threadIdx.x == 0) latch_status(c.status, kStQueueFull);
      __syncthreads();
      continue;
    }
    const SetDesc sd = c.sets[task_set(t)];
    const uint32_t kw = key_width(dna);  // characters per key
    const uint32_t par = task_par(t);
    const uint32_t n = t.len;
    const uint32_t wide = c.wide[task_set(t)];
    for (uint32_t j = threadIdx.x; j < n; j += NT) {
      const Rec r = load_rec(c.rec[par] + t.begin + j);
      m.key[j] = r.key;
      m.idx[j] = r.idx;
      m.off[j] = rec_offset(sd, wide, r.idx, r.off);
      m.tag[j] = make_tag(0, j, 1);
    }
    uint32_t* lcp = sd.lcp ? sd.lcp + (t.begin - sd.base) : nullptr;
    uint32_t depth = t.depth;
    __syncthreads();

    // While every string of the subset has the same cache (and it holds no
    // terminator), jump over the common prefix: compare each string's next 64
    // characters with the first string's and continue at the first window
    // where some string differs or ends.
    while (true) {
      if (threadIdx.x == 0) s_neq = 0;
      __syncthreads();
      const uint64_t k0 = m.key[0];
      for (uint32_t j = threadIdx.x; j < n; j += NT)
        if (m.key[j] != k0) s_neq = 1;
      __syncthreads();
      if (s_neq || key_end(k0, dna) || depth + kw * kLookWindows > kMaxDepth) break;
      if (threadIdx.x == 0) {
        uint64_t w[kLookWindows];
        const uint32_t nwin = load_key_windows<kLookWindows>(sd.chars, m.off[0], depth + kw, sd.cap, dna, w);
        uint32_t js = kLookWindows - 1;
        for (int j = kLookWindows - 1; j >= 0; --j) {
          s_lead[j] = w[j];
          if ((uint32_t)j >= nwin || key_end(w[j], dna)) js = (uint32_t)j;
        }
        s_jstop = js;
      }
      __syncthreads();
      for (uint32_t j = threadIdx.x + 1; j < n; j += NT) {
        uint64_t w[kLookWindows];
        const uint32_t nwin = load_key_windows<kLookWindows>(sd.chars, m.off[j], depth + kw, sd.cap, dna, w);
        uint32_t js = kLookWindows;
#pragma unroll
        for (int q = kLookWindows - 1; q >= 0; --q)
          if ((uint32_t)q >= nwin || w[q] != s_lead[q]) js = (uint32_t)q;
        if (js < kLookWindows) atomicMin(&s_jstop, js);
      }
      __syncthreads();
      const uint32_t nd = depth + kw * (s_jstop + 1);
      for (uint32_t j = threadIdx.x; j < n; j += NT) {
        m.key[j] = load_key(sd.chars, m.off[j], nd, sd.cap, dna);
        bytes += 8ull * (s_jstop + 1);
      }
      depth = nd;
      __syncthreads();
    }

    bool first_pass = true;  // every tag is make_tag(0, position, 1)
    while (true) {
      if (first_pass) block_sort<NT, true>(m, n);
      else block_sort<NT, false>(m, n);
      first_pass = false;
      if (threadIdx.x == 0) s_max_open = 0;
      for (uint32_t j = threadIdx.x; j < n; j += NT) {
        const uint32_t tg = m.tag[j];
        const bool st = j == 0 || tag_seg(tg) != tag_seg(m.tag[j - 1]) || m.key[j] != m.key[j - 1];
        if (lcp && (tg & 1u) && j > 0 && tag_seg(tg) == tag_seg(m.tag[j - 1]) && m.key[j] != m.key[j - 1])
          lcp[j] = depth + key_lcp(m.key[j - 1], m.key[j], dna);
        m.nseg[j] = st ? (uint16_t)j : 0;
        m.aux[j] = 0;
      }
      __syncthreads();
      block_max_scan<NT>(m.nseg, n);
      for (uint32_t j = threadIdx.x; j < n; j += NT) atomicAdd(&m.aux[m.nseg[j]], 1u);
      __syncthreads();
      // Runs of one string or of equal strings are finished; runs of at most
      // 32 strings go back to the record buffer as new warp tasks (a warp
      // finishes them without holding this block); larger runs continue here.
      for (uint32_t j = threadIdx.x; j < n; j += NT) {
        const uint32_t s0 = m.nseg[j];
        uint32_t tg = m.tag[j];
        uint32_t open = tg & 1u, handed = tg & kHanded;
        if (open) {
          const uint32_t size = m.aux[s0];
          if (size == 1) {
            open = 0;
          } else if (key_end(m.key[j], dna)) {
            open = 0;
            if (lcp && j != s0) lcp[j] = depth + key_nnz(m.key[j], dna);
          } else if (size <= 32) {
            open = 0;
            handed = kHanded;
            store_rec(c.rec[par] + t.begin + j, m.key[j], m.idx[tag_pos(tg)], (uint32_t)m.off[tag_pos(tg)]);
            bytes += 16;
            if (j == s0) list_push(c.small_warp, Task{t.begin + j, size, depth, t.meta}, c.status);
          } else {
            atomicMax(&s_max_open, size);
          }
        }
        m.tag[j] = handed | make_tag(s0, tag_pos(tg), open);
      }
      __syncthreads();
      if (s_max_open == 0) break;
      if (depth + kw > kMaxDepth) {
        if (threadIdx.x == 0) latch_status(c.status, kStTooDeep);
        break;
      }
      depth += kw;
      for (uint32_t j = threadIdx.x; j < n; j += NT)
        if (m.tag[j] & 1u) {
          m.key[j] = load_key(sd.chars, m.off[tag_pos(m.tag[j])], depth, sd.cap, dna);
          bytes += 8;
        }
      __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < n; j += NT) {
      const uint32_t tg = m.tag[j];
      if (!(tg & kHanded)) sd.perm[t.begin - sd.base + j] = m.idx[tag_pos(tg)];
      bytes += sd.lcp ? 24 : 20;  // record 16 read; perm 4 (+ lcp 4) written
    }
    __syncthreads();
  }
  account(c, kKSmallCta, bytes);
}

// Resolves the boundary marks left by the multi-block steps (listed in
// c.marks): out_lcp[j] = mark | h means the strings at j-1 and j share exactly
// their first h characters plus the common prefix of their keys at depth h.
// (The single-block steps write their boundary LCPs themselves.)
__global__ void __launch_bounds__(kBlock) k_lcp_fix(SortCtx c) {
  const uint32_t stride = gridDim.x * blockDim.x;
  unsigned long long bytes = 0;
  // the last kernel of a sort: every other one has finished, so the sort's
  // status is final and goes into the stream's status word
  const uint32_t status = *c.status;
  if (c.fold_status && blockIdx.x == 0 && threadIdx.x == 0 && status) atomicOr(c.fold_status, status);
  if (status) {
    // a device-side error stopped the sort part way: positions it did not
    // reach hold whatever the output buffers held.  Give every set the
    // identity permutation and zero LCPs instead, so that no later kernel
    // (this one, or a caller's) follows an index that is out of range.
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < c.total; r += stride) {
      const SetDesc sd = c.sets[c.num_sets == 1 ? 0 : find_set(c, r)];
      sd.perm[r - sd.base] = r - sd.base;
      if (sd.lcp) sd.lcp[r - sd.base] = 0;
    }
    return;
  }
  const uint32_t nm = min(*c.marks_count, c.marks_cap);
  for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += stride) {
    const uint32_t r = c.marks[m];
    const uint32_t s = c.num_sets == 1 ? 0 : find_set(c, r);
    const SetDesc sd = c.sets[s];
    const uint32_t j = r - sd.base;
    const uint32_t v = sd.lcp[j];
    bytes += 8;  // list entry and LCP entry read
    if (j == 0 || !(v & kLcpMark)) continue;
    const uint32_t h = v & ~(kLcpMark | kLcpWide);
    const uint32_t pa = sd.perm[j - 1], pb = sd.perm[j];
    if (pa >= sd.n || pb >= sd.n) continue;  // cannot happen after a sort without errors
    if (v & kLcpWide) {  // a boundary of a multi-block step: the strings differ within its wide key
      const u128 a = load_key128(sd.chars, sd.offsets[pa], h, sd.cap, sd.dna);
      const u128 b = load_key128(sd.chars, sd.offsets[pb], h, sd.cap, sd.dna);
      sd.lcp[j] = h + KeyOps<u128>::lcp(a, b, sd.dna);
      bytes += 60;  // lcp 4 written; per string: perm 4 + offset 8 + 16 characters read
    } else {
      const uint64_t a = load_key(sd.chars, sd.offsets[pa], h, sd.cap, sd.dna);
      const uint64_t b = load_key(sd.chars, sd.offsets[pb], h, sd.cap, sd.dna);
      sd.lcp[j] = h + key_lcp(a, b, sd.dna);
      bytes += 44;  // lcp 4 written; per string: perm 4 + offset 8 + 8 characters read
    }
  }
  account(c, kKLcpFix, bytes);
}

// Distinguishing characters and prefix lengths of a sorted set (Section
// 4.3.4, proof of Lemma 2.1): c^_j = s_j[h_j] and d_j = max(h_j, h_{j+1}) + 1,
// h_0 = h_n = 0; optionally the sum of d_j (= D) into *sum_d.
__global__ void __launch_bounds__(kBlock) k_distinguishing(const uint8_t* __restrict__ chars,
                                                           const uint64_t* __restrict__ offsets, uint32_t n,
                                                           uint32_t cap, const uint32_t* __restrict__ perm,
                                                           const uint32_t* __restrict__ lcp, uint8_t* dchar,
                                                           uint32_t* dprefix, unsigned long long* sum_d) {
  unsigned long long acc = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t lim = (n + 31) / 32 * 32;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < lim; j += stride) {
    if (j < n) {
      const uint32_t h = j == 0 ? 0u : lcp[j];
      const uint32_t next = j + 1 < n ? lcp[j + 1] : 0u;
      const uint32_t d = max(h, next) + 1;
      if (dprefix) dprefix[j] = d;
      if (dchar) dchar[j] = h < cap ? chars[offsets[perm[j]] + h] : 0;
      acc += d;
    }
    if (sum_d) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
      if (lane_id() == 0 && acc) atomicAdd(sum_d, acc);
      acc = 0;
    }
  }
}

}  // namespace

// Packs a byte buffer over {A, C, G, T, terminator} into 3-bit codes (0 =
// terminator, 1..4 = A, C, G, T), most significant first, character p at
// bits [3p, 3p + 3) of the word stream; sets *bad if another byte occurs.
__global__ void k_pack_dna(const uint8_t* __restrict__ chars, uint64_t len, uint64_t* __restrict__ out,
                           uint64_t words, uint32_t* bad) {
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g0 = 64 * w;
    uint64_t v = 0;
    bool invalid = false;
    for (uint64_t p = g0 / 3; p <= (g0 + 63) / 3; ++p) {
      uint64_t code = 0;
      if (p < len) {
        const uint8_t ch = chars[p];
        code = ch == 'A' ? 1 : ch == 'C' ? 2 : ch == 'G' ? 3 : ch == 'T' ? 4 : 0;
        invalid = invalid || (ch != 0 && code == 0);
      }
      const int64_t s = (int64_t)(3 * p) - (int64_t)g0;  // first bit of the code, from the word's top
      v |= s <= 61 ? code << (61 - s) : code >> (s - 61);
    }
    out[w] = v;
    if (invalid) atomicOr(bad, 1u);
  }
}

size_t small_cta_smem(uint32_t pmax) { return (size_t)pmax * (8 + 8 + 8 + 4 + 4 + 4 + 4 + 2); }

cudaError_t launch_init(const SortCtx& c, cudaStream_t st, const LaunchHook& hook) {
  const uint32_t grid = max(1u, min((c.total + kBlock - 1) / kBlock, 152u * 16u));
  hook.run("init", [&] { k_init<<<grid, kBlock, 0, st>>>(c); });
  hook.run("init", [&] { k_roots<<<(c.num_sets + 127) / 128, 128, 0, st>>>(c); });
  return cudaGetLastError();
}

template <bool DNA>
static cudaError_t launch_small_t(const SortCtx& c, uint32_t pmax, uint32_t grid_warp, uint32_t grid_cta,
                                  cudaStream_t st, const LaunchHook& hook) {
  static uint32_t attr_pmax = 0;
  if (pmax > attr_pmax) {
    cudaError_t e = cudaFuncSetAttribute(k_small_cta<kBlock, DNA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)small_cta_smem(pmax));
    if (e != cudaSuccess) return e;
    attr_pmax = pmax;
  }
  // subsets of up to kSmallCtaNarrowMax strings: 64-thread blocks with small
  // shared arrays, many per SM (a subset's sort is latency-bound, so more of
  // them in flight beats more threads on each); larger ones: 256 threads
  // (when there are enough subsets to fill the GPU with them)
  const uint32_t min_count = 2 * grid_cta;
  if (pmax <= kSmallCtaNarrowMax) {
    hook.run("small_cta", [&] {
      k_small_cta<64, DNA><<<grid_cta * 4, 64, small_cta_smem(pmax), st>>>(c, pmax, 0u, 1u);
    });
  } else {
    hook.run("small_cta", [&] {
      k_small_cta<64, DNA><<<grid_cta * 4, 64, small_cta_smem(kSmallCtaNarrowMax), st>>>(
          c, kSmallCtaNarrowMax, min_count, 1u);
    });
    hook.run("small_cta", [&] {
      k_small_cta<kBlock, DNA><<<grid_cta, kBlock, small_cta_smem(pmax), st>>>(
          c, pmax, min_count, 0u);
    });
  }
  // the lists alternate: a pass reads one and defers into the other, emptied first
  for (uint32_t p = 0; p < kWarpPasses; ++p) {
    const TaskList in = (p & 1) ? c.small_deep : c.small_warp;
    const TaskList out = (p & 1) ? c.small_warp : c.small_deep;
    if (p > 0 && kWarpPassJumps[p] > 0) {
      const cudaError_t e = launch_upload(nullptr, out.count, 4, st, hook);
      if (e != cudaSuccess) return e;
    }
    hook.run("small_warp", [&] { k_small_warp<<<grid_warp, kBlock, 0, st>>>(c, in, out, kWarpPassJumps[p]); });
  }
  return cudaGetLastError();
}

cudaError_t launch_small(const SortCtx& c, uint32_t pmax, uint32_t grid_warp, uint32_t grid_cta,
                         cudaStream_t st, const LaunchHook& hook) {
  return c.dna ? launch_small_t<true>(c, pmax, grid_warp, grid_cta, st, hook)
               : launch_small_t<false>(c, pmax, grid_warp, grid_cta, st, hook);
}

cudaError_t launch_pack_dna(const uint8_t* chars, uint64_t len, uint64_t* out, uint64_t words, uint32_t* bad,
                            uint32_t grid, cudaStream_t st, const LaunchHook& hook) {
  hook.run("init", [&] { k_pack_dna<<<grid, kBlock, 0, st>>>(chars, len, out, words, bad); });
  return cudaGetLastError();
}

// Small host-to-device transfers and zero fills done by a kernel rather than
// by the copy engines, which a large copy queued on another stream can hold
// up for milliseconds: src is pinned host memory, which the device reads
// directly (null: write zeros).
__global__ void k_upload(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, uint32_t words) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
    dst[i] = src ? src[i] : 0u;
}

cudaError_t launch_upload(const void* host_src, void* dst, size_t bytes, cudaStream_t st, const LaunchHook& hook) {
  if (bytes == 0) return cudaSuccess;
  if ((bytes & 3) || (reinterpret_cast<uintptr_t>(dst) & 3) || (reinterpret_cast<uintptr_t>(host_src) & 3) ||
      bytes >= (4ull << 32))
    return cudaErrorInvalidValue;
  const uint32_t words = (uint32_t)(bytes / 4);
  const uint32_t grid = std::min<uint32_t>((words + kBlock - 1) / kBlock, 1024);
  hook.run("upload", [&] {
    k_upload<<<grid, kBlock, 0, st>>>(static_cast<const uint32_t*>(host_src), static_cast<uint32_t*>(dst), words);
  });
  return cudaGetLastError();
}

cudaError_t launch_distinguishing(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t cap,
                                  const uint32_t* perm, const uint32_t* lcp, uint8_t* dchar, uint32_t* dprefix,
                                  unsigned long long* sum_d, uint32_t grid, cudaStream_t st, const LaunchHook& hook) {
  hook.run("distinguishing", [&] {
    k_distinguishing<<<grid, kBlock, 0, st>>>(chars, offsets, n, cap, perm, lcp, dchar, dprefix, sum_d);
  });
  return cudaGetLastError();
}

cudaError_t launch_lcp_fix(const SortCtx& c, uint32_t grid, cudaStream_t st, const LaunchHook& hook) {
  hook.run("lcp_fix", [&] { k_lcp_fix<<<grid, kBlock, 0, st>>>(c); });
  return cudaGetLastError();
}

}  // namespace ss
