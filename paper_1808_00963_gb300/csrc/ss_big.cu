// Multi-block S^5 steps: the "fully parallel S^5" of Section 4.2.8 for
// subsets above the big-task threshold.  All big subsets of one round are
// processed together: one block samples each subset (SampleJob), every tile
// of every subset is classified and counted by its own block (CountJob), one
// device-wide prefix sum over the [subset][bucket][tile] counters gives every
// tile its destination in every bucket (the interleaved prefix sum of
// Theorem 4.4), one block per subset emits the new subsets, and every tile is
// redistributed by its own block (DistributeJob).
#include "ss_kernels.h"
#include "ss_step.cuh"

namespace ss {

namespace {

__device__ __forceinline__ uint32_t find_gen_task(const GenTask* gt, uint32_t G, uint32_t tile) {
  uint32_t lo = 0, hi = G - 1;  // last task with tile_start <= tile
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (gt[mid].tile_start <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The first tile of every subset of the round, for up to kTileStartsMax
// subsets, copied into shared memory when a kernel starts: a block then finds
// the subset of each tile it takes with a shared-memory search instead of a
// chain of dependent global loads.
constexpr uint32_t kTileStartsMax = 4096;

__device__ __forceinline__ void load_tile_starts(const GenTask* gt, uint32_t G, uint32_t* ts) {
  const uint32_t m = G < kTileStartsMax ? G : kTileStartsMax;
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) ts[i] = gt[i].tile_start;
  __syncthreads();
}

__device__ __forceinline__ uint32_t find_gen_task_ts(const GenTask* gt, const uint32_t* ts, uint32_t G,
                                                     uint32_t tile) {
  if (G > kTileStartsMax) return find_gen_task(gt, G, tile);
  uint32_t lo = 0, hi = G - 1;  // last task with tile_start <= tile
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (ts[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint64_t cnt_base(const GenTask& g) {
  return ((uint64_t)g.cnt_base_hi << 32) | g.cnt_base_lo;
}

// Prefix jump.  A step sees 16 characters, so a subset whose strings share a
// long prefix (many URLs of one site, repeated records) would be moved once
// for every 16 shared characters.  When the whole sample of a subset is one key
// without a terminator, the sampling block measures how far 64 of the
// sampled strings agree with one of them over the next kPjWindows windows;
// if they agree beyond 32 characters, the classification measures the same
// for every string, and if the whole subset then falls into that key's
// equality bucket,
// the bucket continues at depth + the smallest agreement instead of depth + 16.
// Any depth up to the subset's common prefix is correct: the jump only skips
// work, and the check on the sample keeps its cost away from subsets that
// share only the key.
constexpr int kPjWindows = 8;        // 64 characters
constexpr uint32_t kPjMinSample = 32;  // sampled agreement that turns the check on
constexpr uint32_t kPjSampleChecks = 64;  // sampled strings compared (of the sample's S)

// Splitters of one multi-block task, with the jump table of its tree (filled
// for the jump-table classifier only) and the prefix-jump state.
template <int LOGV>
struct BigSplitters {
  Splitters<LOGV, u128> sp;  // wide keys
  uint16_t jump[kJumpSize];
  uint64_t pj_ref;  // offset of the reference string (the first sampled one)
  uint32_t pj_on;   // check every string of the subset
  uint32_t pj_lcp;  // smallest agreement with the reference from the depth (atomicMin)
};

// The kPjWindows windows of a string from depth h (no terminator before h).
// load_windows reads only the 4 KiB block holding byte h; the windows it
// leaves open lie past that block, and since the string has not ended before
// them, they are read one at a time (load_cache reads the next block only
// while the string continues).  This happens for about 1 string in 64.
__device__ __forceinline__ void load_pj_windows(const uint8_t* chars, uint64_t off, uint32_t h, uint32_t cap,
                                                uint64_t (&w)[kPjWindows]) {
  const uint32_t nw = load_windows<kPjWindows>(chars, off, h, cap, w);
  for (uint32_t j = nw; j < (uint32_t)kPjWindows; ++j) {
    w[j] = load_cache(chars, off, h + 8 * j, cap);
    if (has_nul(w[j])) break;  // the later windows stay 0
  }
}

// How many characters from the depth a string shares with the reference.
__device__ __forceinline__ uint32_t window_lcp(const uint64_t (&w)[kPjWindows], const uint64_t* ref) {
#pragma unroll
  for (int j = 0; j < kPjWindows; ++j) {
    if (w[j] != ref[j]) return 8u * j + lcp8(w[j], ref[j]);
    if (has_nul(w[j])) return 8u * j + nnz_prefix(w[j]);
  }
  return 8u * kPjWindows;
}

// Smallest agreement with ref over the strings of items [0, items) taken by
// this block's threads (off_of(i) gives the string offset of item i), reduced
// over the block.
template <typename OffOf>
__device__ uint32_t block_min_agreement(const SetDesc& sd, uint32_t depth, uint32_t items, OffOf&& off_of,
                                        const uint64_t* ref, unsigned long long& bytes) {
  __shared__ uint32_t bmin;
  if (threadIdx.x == 0) bmin = 0xFFFFFFFFu;
  __syncthreads();
  uint32_t mn = 0xFFFFFFFFu;
  for (uint32_t i = threadIdx.x; i < items; i += blockDim.x) {
    uint64_t w[kPjWindows];
    load_pj_windows(sd.chars, off_of(i), depth, sd.cap, w);
    mn = min(mn, window_lcp(w, ref));
    bytes += 8 + 8 * kPjWindows;  // the record's index and offset, the windows
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
  if ((threadIdx.x & 31u) == 0 && mn != 0xFFFFFFFFu) atomicMin(&bmin, mn);
  __syncthreads();
  return bmin;
}

// ---- plan of a round ------------------------------------------------------------------

__device__ unsigned long long g_graph_launches;  // kernels launched by loop graphs (this device)

constexpr uint32_t kPlanThreads = 1024;

// Exclusive scan of one 64-bit value per thread of a kPlanThreads block;
// returns the block total.
__device__ uint64_t plan_scan(uint64_t v, uint64_t& excl) {
  __shared__ uint64_t wsum[kPlanThreads / 32];
  const uint32_t w = threadIdx.x >> 5, lane = lane_id();
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint64_t x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (uint32_t)o) x += t;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  excl = inc - v + (w ? wsum[w - 1] : 0ull);
  const uint64_t total = wsum[kPlanThreads / 32 - 1];
  __syncthreads();
  return total;
}

// Turns the big subsets left by the previous round (list ctl->cur) into the
// task table of this round: for every subset its tiles, its first tile, its
// first record among the round's records and its first counter (the host
// plan of a multi-block step, done on the device).  With use_cond it sets the
// loop graph's condition: 1 while there is a round to run.
__global__ void __launch_bounds__(kPlanThreads) k_big_plan(BigCtl* __restrict__ ctl,
                                                           cudaGraphConditionalHandle h, uint32_t use_cond) {
  __shared__ uint32_t s_G;
  const SortCtx& c = ctl->c;
  const uint32_t cur = ctl->cur;
  if (threadIdx.x == 0) {
    uint32_t g = min(*c.big[cur].count, ctl->cap_big);
    if (g && (*c.status != 0 || ctl->round >= kMaxBigRounds)) {
      if (ctl->round >= kMaxBigRounds) latch_status(c.status, kStTooDeep);
      g = 0;  // stop: this sort has latched an error, or the loop ran too long
    }
    s_G = g;
  }
  __syncthreads();
  uint32_t G = s_G;
  // strings in this round's subsets, for the tile size
  uint64_t mine = 0;
  for (uint32_t g = threadIdx.x; g < G; g += kPlanThreads) mine += c.big[cur].items[g].len;
  uint64_t ex;
  const uint64_t total = plan_scan(mine, ex);
  uint32_t R = ctl->R_fixed;
  if (!R) {
    const uint64_t per = total / ((uint64_t)ctl->sms * 2 * kBlock) + 1;
    R = (uint32_t)(per < 8 ? 8 : (per > kMaxRounds ? kMaxRounds : per));
  }
  const uint32_t T = kBlock * R;
  const uint64_t K = ctl->K;
  uint64_t tiles0 = 0, rec0 = 0, cnt0 = 0;
  for (uint32_t g0 = 0; g0 < G; g0 += kPlanThreads) {
    const uint32_t g = g0 + threadIdx.x;
    Task t{0, 0, 0, 0};
    if (g < G) t = c.big[cur].items[g];
    const uint32_t tl = (t.len + T - 1) / T;
    uint64_t e_tiles, e_rec, e_cnt;
    const uint64_t s_tiles = plan_scan(tl, e_tiles);
    const uint64_t s_rec = plan_scan(t.len, e_rec);
    const uint64_t s_cnt = plan_scan(K * tl, e_cnt);
    if (g < G) {
      GenTask x;
      x.t = t;
      x.tile_start = (uint32_t)(tiles0 + e_tiles);
      x.tiles = tl;
      x.rec_base = (uint32_t)(rec0 + e_rec);
      const uint64_t cb = cnt0 + e_cnt;
      x.cnt_base_lo = (uint32_t)cb;
      x.cnt_base_hi = (uint32_t)(cb >> 32);
      x.pad[0] = x.pad[1] = x.pad[2] = 0;
      ctl->gt[g] = x;
    }
    tiles0 += s_tiles;
    rec0 += s_rec;
    cnt0 += s_cnt;
  }
  if (threadIdx.x == 0) {
    if (cnt0 > ctl->ncounters_max) {  // cannot happen: the counters are sized for the largest round
      latch_status(c.status, kStQueueFull);
      G = 0;
    }
    ctl->G = G;
    ctl->tiles = G ? (uint32_t)tiles0 : 0u;
    ctl->R = R;
    ctl->ncounters = G ? cnt0 : 0ull;
    ctl->next_big = cur ^ 1u;
    for (int k = 0; k < 4; ++k) ctl->next_item[k] = 0;
    if (G) {
      *c.big[cur ^ 1u].count = 0;  // the list the round's new big subsets go to
      ctl->cur = cur ^ 1u;
      ctl->round += 1;
    }
    if (use_cond) {
      atomicAdd(&g_graph_launches, 1ull + (G ? kBigRoundKernels : 0ull));
      cudaGraphSetConditional(h, G ? 1u : 0u);
    }
  }
}

// ---- the kernels of one round -----------------------------------------------------------

// Records per lane moved together by the multi-block distribution (a wide
// record and its loads take twice the registers of a narrow one).
constexpr int kWideMoveBatch = 2;

// The items (subsets or tiles) of a round's kernel for this block, taken from
// the kernel's work counter one ahead: thread 0 claims the block's next item
// when the current one starts, so the atomic's round trip overlaps the work.
//   for (uint32_t i = items.first(); i < n; i = items.next()) { items.claim(); ... }
struct ItemStream {
  uint32_t* counter;
  uint32_t ahead;  // thread 0: the item claimed for after the current one
  __device__ __forceinline__ uint32_t share(uint32_t v) {
    __shared__ uint32_t s_item;
    __syncthreads();  // every thread is done with the previous item
    if (threadIdx.x == 0) s_item = v;
    __syncthreads();
    return s_item;
  }
  __device__ __forceinline__ uint32_t first() { return share(threadIdx.x == 0 ? atomicAdd(counter, 1u) : 0u); }
  __device__ __forceinline__ void claim() {
    if (threadIdx.x == 0) ahead = atomicAdd(counter, 1u);
  }
  __device__ __forceinline__ uint32_t next() { return share(ahead); }
};

template <int LOGV>
__global__ void __launch_bounds__(kBlock) k_big_sample(const BigCtl* __restrict__ ctl, uint32_t* __restrict__ work) {
  __shared__ __align__(16) Splitters<LOGV, u128> sp;
  __shared__ __align__(16) BuildScratch<LOGV, u128> bs;
  __shared__ uint64_t ref[kPjWindows];
  const uint32_t G = ctl->G;
  const SortCtx& c = ctl->c;
  BigSplitters<LOGV>* out = reinterpret_cast<BigSplitters<LOGV>*>(ctl->splitters);
  unsigned long long bytes = 0;
  ItemStream items{work, 0u};
  for (uint32_t gi = items.first(); gi < G; gi = items.next()) {
    items.claim();
    const GenTask g = ctl->gt[gi];
    const uint32_t par = task_par(g.t);
    const Rec* recs = c.rec[par] + g.t.begin;
    const uint2* wids = c.wid[par] + g.t.begin;
    const SetDesc sd = c.sets[task_set(g.t)];
    const uint64_t hseed = mix64(c.seed ^ ((uint64_t)g.t.begin << 20) ^ g.t.depth);
    build_splitters_k<LOGV, u128>([&](uint32_t pos) { return load_wkey(recs + pos); }, g.t.len, hseed, sp, bs,
                                  sd.dna);
    const uint4* src = reinterpret_cast<const uint4*>(&sp);
    uint4* dst = reinterpret_cast<uint4*>(&out[gi].sp);
    for (uint32_t i = threadIdx.x; i < sizeof(sp) / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) bytes += Geo<LOGV>::S * 16ull + sizeof(sp);
    // prefix jump: a one-key sample whose strings agree beyond kPjMinSample
    // characters turns on the check of the whole subset
    const u128 k0 = bs.sample[0];  // the sorted sample
    const bool one_key = !sd.dna && k0 == bs.sample[Geo<LOGV>::S - 1] && !KeyOps<u128>::end(k0, 0u);
    uint32_t on = 0;
    uint64_t ref_off = 0;
    if (one_key) {  // uniform over the block
      auto sample_pos = [&](uint32_t i) {
        return (uint32_t)(((mix64(hseed + i) >> 32) * (uint64_t)g.t.len) >> 32);
      };
      const uint32_t wide = c.wide[task_set(g.t)];
      auto off_of = [&](uint32_t i) {
        const uint2 w = wids[sample_pos(i)];
        return rec_offset(sd, wide, w.x, w.y);
      };
      ref_off = off_of(0);
      if (threadIdx.x == 0) {
        uint64_t w[kPjWindows];
        load_pj_windows(sd.chars, ref_off, g.t.depth, sd.cap, w);
        for (int j = 0; j < kPjWindows; ++j) ref[j] = w[j];
      }
      __syncthreads();
      const uint32_t agree = block_min_agreement(sd, g.t.depth, kPjSampleChecks, off_of, ref, bytes);
      on = agree > kPjMinSample && agree != 0xFFFFFFFFu ? 1u : 0u;
    }
    if (threadIdx.x == 0) {
      out[gi].pj_on = on;
      out[gi].pj_lcp = 0xFFFFFFFFu;
      out[gi].pj_ref = ref_off;
    }
    if (c.classifier == kClassifyUIJ) {
      for (uint32_t p = threadIdx.x; p < kJumpSize; p += blockDim.x)
        out[gi].jump[p] = (uint16_t)jump_entry<LOGV, u128>(p, sp.tree);
      if (threadIdx.x == 0) bytes += 2ull * kJumpSize;
    }
  }
  // sample reads + splitter (and jump table) writes
  account(c, kKBigSample, bytes);
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock, 4) k_big_classify(const BigCtl* __restrict__ ctl, uint32_t* __restrict__ work) {
  using Gm = Geo<LOGV>;
  __shared__ __align__(16) u128 tree[Gm::V + 1];
  __shared__ __align__(16) u128 x[Gm::V + 1];
  __shared__ uint32_t hist[Gm::KP];
  __shared__ __align__(16) uint16_t jump[kJumpSize];
  __shared__ uint64_t ref[kPjWindows];
  __shared__ uint32_t s_g;
  __shared__ uint32_t ts[kTileStartsMax];
  const uint32_t G = ctl->G, tiles = ctl->tiles, R = ctl->R;
  const SortCtx& c = ctl->c;
  const GenTask* __restrict__ gt = ctl->gt;
  BigSplitters<LOGV>* spl = reinterpret_cast<BigSplitters<LOGV>*>(ctl->splitters);
  const bool use_jump = c.classifier == kClassifyUIJ;
  load_tile_starts(gt, G, ts);
  unsigned long long bytes = 0;
  uint32_t loaded = 0xFFFFFFFFu;  // subset whose splitters are in shared memory
  ItemStream items{work, 0u};
  for (uint32_t tg = items.first(); tg < tiles; tg = items.next()) {
    items.claim();
    if (threadIdx.x == 0) s_g = find_gen_task_ts(gt, ts, G, tg);
    for (uint32_t b = threadIdx.x; b < Gm::KP; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t gi = s_g;
    const GenTask g = gt[gi];
    if (gi != loaded) {  // uniform over the block
      const Splitters<LOGV, u128>& sp = spl[gi].sp;
      for (uint32_t i = threadIdx.x; i <= Gm::V; i += blockDim.x) { tree[i] = sp.tree[i]; x[i] = sp.x[i]; }
      if (use_jump) {
        const uint4* js = reinterpret_cast<const uint4*>(spl[gi].jump);
        uint4* jd = reinterpret_cast<uint4*>(jump);
        for (uint32_t i = threadIdx.x; i < kJumpSize * 2 / 16; i += blockDim.x) jd[i] = js[i];
      }
      loaded = gi;
      __syncthreads();
    }
    const uint32_t tile = tg - g.tile_start;
    const uint32_t T = kBlock * R;
    const uint32_t t0 = tile * T;
    const uint32_t tl = min(T, g.t.len - t0);
    const uint32_t par = task_par(g.t);
    const Rec* recs = c.rec[par] + g.t.begin + t0;
    uint16_t* bo = c.bucket_of + g.t.begin + t0;
    const uint32_t mine = classify_count_k<LOGV, u128>([&](uint32_t p) { return load_wkey(recs + p); }, bo, tl,
                                                       tree, x, hist, c.classifier, use_jump ? jump : nullptr);
    __syncthreads();
    uint32_t* cnt = ctl->counters + cnt_base(g) + tile;
    for (uint32_t b = threadIdx.x; b < Gm::K; b += blockDim.x) cnt[(uint64_t)b * g.tiles] = hist[b];
    // per record: wide key 16 read + bucket index 2 written; per tile: K counters written
    bytes += 18ull * mine;
    if (threadIdx.x == 0) bytes += 4ull * Gm::K;
    if (spl[gi].pj_on) {  // prefix jump: every string's agreement with the reference
      const SetDesc sd = c.sets[task_set(g.t)];
      if (threadIdx.x == 0) {
        uint64_t w[kPjWindows];
        load_pj_windows(sd.chars, spl[gi].pj_ref, g.t.depth, sd.cap, w);
        for (int j = 0; j < kPjWindows; ++j) ref[j] = w[j];
      }
      __syncthreads();
      const uint2* wids = c.wid[par] + g.t.begin + t0;
      const uint32_t wide = c.wide[task_set(g.t)];
      const uint32_t bmin = block_min_agreement(
          sd, g.t.depth, tl, [&](uint32_t i) { const uint2 w = wids[i]; return rec_offset(sd, wide, w.x, w.y); },
          ref, bytes);
      if (threadIdx.x == 0 && bmin != 0xFFFFFFFFu) atomicMin(&spl[gi].pj_lcp, bmin);
    }
  }
  account(c, kKBigClassify, bytes);
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock) k_big_emit(const BigCtl* __restrict__ ctl, uint32_t* __restrict__ work) {
  using Gm = Geo<LOGV>;
  const uint32_t G = ctl->G;
  const SortCtx& c = ctl->c;
  const BigSplitters<LOGV>* spl = reinterpret_cast<const BigSplitters<LOGV>*>(ctl->splitters);
  const uint32_t next_big = ctl->next_big;
  unsigned long long bytes = 0;
  ItemStream items{work, 0u};
  for (uint32_t gi = items.first(); gi < G; gi = items.next()) {
    items.claim();
    const GenTask g = ctl->gt[gi];
    const Splitters<LOGV, u128>& sp = spl[gi].sp;
    const SetDesc sd = c.sets[task_set(g.t)];
    const uint32_t* sc = ctl->counters + cnt_base(g);
    for (uint32_t b = threadIdx.x; b < Gm::K; b += blockDim.x) {
      bytes += 16;  // two bucket offsets read, start and descriptor written
      const uint32_t s = sc[(uint64_t)b * g.tiles] - g.rec_base;
      const uint32_t e = (b + 1 < Gm::K) ? sc[(uint64_t)(b + 1) * g.tiles] - g.rec_base : g.t.len;
      const uint32_t size = e - s;
      ctl->gstart[(uint64_t)gi * Gm::KP + b] = s;
      uint32_t desc = kFin;
      if (size) {
        desc = bucket_desc<LOGV, u128>(b, size, g.t.depth, sp, sd.dna);
        // prefix jump: the whole subset is the key's equality bucket, and every
        // string agrees with the reference for pj_lcp characters from the depth
        if (spl[gi].pj_on && (b & 1u) && size == g.t.len && !(desc & kFin)) {
          const uint32_t J = spl[gi].pj_lcp;
          if (J > KeyOps<u128>::width(0) && J != 0xFFFFFFFFu) desc = g.t.depth + J;
        }
        emit_bucket(c, sd, g.t, s, size, desc, next_big, kLcpMark | kLcpWide);
        const bool mark = s > 0 && sd.lcp;  // the fix-up at the end visits the listed marks only
        const uint32_t k = warp_slot(c.marks_count, mark);
        if (mark) {
          if (k < c.marks_cap) c.marks[k] = g.t.begin + s;
          else latch_status(c.status, kStQueueFull);
        }
      }
      ctl->gdesc[(uint64_t)gi * Gm::KP + b] = desc;
    }
  }
  account(c, kKBigEmit, bytes);
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock, 3) k_big_scatter(const BigCtl* __restrict__ ctl, uint32_t* __restrict__ work) {
  using Gm = Geo<LOGV>;
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* cntw = reinterpret_cast<uint32_t*>(smem);
  uint32_t* base = cntw + kWarps * Gm::KP;
  uint32_t* desc = base + Gm::KP;
  uint32_t* bfirst = desc + Gm::KP;
  uint16_t* tb = reinterpret_cast<uint16_t*>(bfirst + Gm::KP);
  __shared__ uint32_t s_g;
  __shared__ uint32_t ts[kTileStartsMax];
  const uint32_t G = ctl->G, tiles = ctl->tiles, R = ctl->R;
  const SortCtx& c = ctl->c;
  const GenTask* __restrict__ gt = ctl->gt;
  load_tile_starts(gt, G, ts);
  unsigned long long bytes = 0;
  uint32_t loaded = 0xFFFFFFFFu;
  GenTask g{};
  SetDesc sd{};
  ItemStream items{work, 0u};
  for (uint32_t tg = items.first(); tg < tiles; tg = items.next()) {
    items.claim();
    if (threadIdx.x == 0) s_g = find_gen_task_ts(gt, ts, G, tg);
    __syncthreads();
    const uint32_t gi = s_g;
    // the subset's task, set and per-bucket descriptors and starts stay in
    // registers and shared memory while the block's tiles come from one subset
    const bool fresh = gi != loaded;  // uniform over the block
    if (fresh) {
      g = gt[gi];
      sd = c.sets[task_set(g.t)];
    }
    const uint32_t tile = tg - g.tile_start;
    const uint32_t T = kBlock * R;
    const uint32_t t0 = tile * T;
    const uint32_t tl = min(T, g.t.len - t0);
    const uint32_t par = task_par(g.t);
    const uint16_t* bo = c.bucket_of + g.t.begin + t0;
    for (uint32_t p = threadIdx.x; p < tl; p += kBlock) tb[p] = bo[p];
    const uint32_t* sc = ctl->counters + cnt_base(g) + tile;
    for (uint32_t b = threadIdx.x; b < Gm::K; b += kBlock) {
      base[b] = g.t.begin + sc[(uint64_t)b * g.tiles] - g.rec_base;
      if (fresh) {
        desc[b] = ctl->gdesc[(uint64_t)gi * Gm::KP + b];
        bfirst[b] = g.t.begin + ctl->gstart[(uint64_t)gi * Gm::KP + b];
      }
    }
    if (fresh && threadIdx.x == 0) bfirst[Gm::K] = g.t.begin + g.t.len;  // bucket sizes from neighbouring starts
    loaded = gi;
    __syncthreads();
    const uint32_t src0 = g.t.begin + t0;
    const uint32_t depth = g.t.depth;
    const uint32_t wide = c.wide[task_set(g.t)];
    if (threadIdx.x == 0) bytes += (fresh ? 12ull : 4ull) * Gm::K;  // per-bucket tile offsets (+ descriptors and starts)
    tile_scatter<LOGV, kWideMoveBatch>(
        tb, tl, R, base, cntw,
        [&](const uint32_t(&pp)[kWideMoveBatch], const uint32_t(&bb)[kWideMoveBatch],
            const uint32_t(&dd)[kWideMoveBatch]) {
          bytes += move_batch_wide<kWideMoveBatch>(c, sd, wide, par, src0, depth, desc,
                                                   [&](uint32_t b) { return bfirst[b]; }, pp, bb, dd);
        });
  }
  account(c, kKBigScatter, bytes);
}

// ---- exclusive prefix sum over uint32 (two phases) ------------------------------

constexpr uint32_t kScanItems = 16;
constexpr uint32_t kScanChunk = kBlock * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane_id() >= (uint32_t)o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& excl) {
  __shared__ uint32_t wsum[kWarps];
  const uint32_t w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  if (lane_id() == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane_id() < kWarps ? wsum[lane_id()] : 0;
    s = warp_incl_scan(s);
    if (lane_id() < kWarps) wsum[lane_id()] = s;
  }
  __syncthreads();
  excl = inc - v + (w ? wsum[w - 1] : 0);
  const uint32_t total = wsum[kWarps - 1];
  __syncthreads();
  return total;
}

// The kScanItems counters of thread t of chunk blk are a[blk * kScanChunk +
// t * kScanItems ...]; in a full chunk they are read as four 16-byte words
// (the counters start 256-byte aligned and a chunk spans 16 KiB).
__device__ __forceinline__ void load_scan_items(const uint32_t* __restrict__ a, uint64_t n, uint64_t k0,
                                                bool full, uint32_t (&v)[kScanItems]) {
  if (full) {
    const uint4* a4 = reinterpret_cast<const uint4*>(a + k0);
#pragma unroll
    for (uint32_t q = 0; q < kScanItems / 4; ++q) {
      const uint4 x = a4[q];
      v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (uint32_t j = 0; j < kScanItems; ++j) v[j] = k0 + j < n ? a[k0 + j] : 0u;
  }
}

// Phase 1: the total of every chunk of kScanChunk counters of the round
// (ctl->ncounters values).
__global__ void __launch_bounds__(kBlock) k_scan_reduce(const BigCtl* __restrict__ ctl) {
  const uint64_t n = ctl->ncounters;
  const uint32_t* __restrict__ a = ctl->counters;
  uint32_t* __restrict__ part = ctl->partials;
  const uint64_t nb = (n + kScanChunk - 1) / kScanChunk;
  unsigned long long bytes = 0;
  for (uint64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
    const uint64_t c0 = blk * kScanChunk;
    uint32_t v[kScanItems];
    load_scan_items(a, n, c0 + (uint64_t)threadIdx.x * kScanItems, c0 + kScanChunk <= n, v);
    uint32_t s = 0;
#pragma unroll
    for (uint32_t j = 0; j < kScanItems; ++j) s += v[j];
    uint32_t ex;
    const uint32_t total = block_excl_scan(s, ex);
    if (threadIdx.x == 0) {
      part[blk] = total;
      const uint64_t left = n - c0;
      bytes += 4ull * (left < kScanChunk ? left : kScanChunk);
    }
  }
  account(ctl->c, kKScan, bytes);
}

// Phase 2: every counter replaced by the sum of the counters before it.  A
// block finds the offset of its chunk by summing the chunk totals before it
// (carried from one of its chunks to its next), so no third kernel scans the
// totals.
__global__ void __launch_bounds__(kBlock) k_scan_down(const BigCtl* __restrict__ ctl) {
  const uint64_t n = ctl->ncounters;
  uint32_t* __restrict__ a = ctl->counters;
  const uint32_t* __restrict__ part = ctl->partials;
  const uint64_t nb = (n + kScanChunk - 1) / kScanChunk;
  unsigned long long bytes = 0;
  uint32_t pre = 0;   // sum of part[0, upto)
  uint64_t upto = 0;
  for (uint64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
    uint32_t ps = 0;
    for (uint64_t i = upto + threadIdx.x; i < blk; i += kBlock) ps += part[i];
    uint32_t unused;
    pre += block_excl_scan(ps, unused);
    upto = blk;
    const uint64_t c0 = blk * kScanChunk;
    const uint64_t k0 = c0 + (uint64_t)threadIdx.x * kScanItems;
    const bool full = c0 + kScanChunk <= n;
    uint32_t v[kScanItems];
    load_scan_items(a, n, k0, full, v);
    uint32_t s = 0;
#pragma unroll
    for (uint32_t j = 0; j < kScanItems; ++j) s += v[j];
    uint32_t ex;
    block_excl_scan(s, ex);
    uint32_t run = pre + ex;
#pragma unroll
    for (uint32_t j = 0; j < kScanItems; ++j) {
      const uint32_t x = v[j];
      v[j] = run;
      run += x;
    }
    if (full) {
      uint4* a4 = reinterpret_cast<uint4*>(a + k0);
#pragma unroll
      for (uint32_t q = 0; q < kScanItems / 4; ++q)
        a4[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
      for (uint32_t j = 0; j < kScanItems; ++j)
        if (k0 + j < n) a[k0 + j] = v[j];
    }
    const uint64_t left = n > k0 ? n - k0 : 0;
    bytes += 8ull * (left < kScanItems ? left : kScanItems);
  }
  account(ctl->c, kKScan, bytes);
}

}  // namespace

size_t big_splitters_bytes(int logv) {
  return logv == 8 ? sizeof(BigSplitters<8>) : sizeof(BigSplitters<9>);
}

size_t big_scatter_smem(int logv, uint32_t R) {
  const uint32_t KP = 2u << logv;
  return (size_t)(kWarps * KP + 3 * KP) * 4 + (size_t)kBlock * R * 2;
}

cudaError_t launch_big_plan(BigCtl* ctl, uint64_t cond_handle, bool use_cond, cudaStream_t st,
                            const LaunchHook& hook) {
  hook.run("big_sample", [&] {
    k_big_plan<<<1, kPlanThreads, 0, st>>>(ctl, (cudaGraphConditionalHandle)cond_handle, use_cond ? 1u : 0u);
  });
  return cudaGetLastError();
}

template <int LOGV>
static cudaError_t launch_big_round_t(BigCtl* ctl, uint32_t R_max, uint32_t sms, cudaStream_t st,
                                      const LaunchHook& hook) {
  const size_t smem = big_scatter_smem(LOGV, R_max);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_big_scatter<LOGV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)big_scatter_smem(LOGV, kMaxRounds));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  // fixed grids (the work of a round is only known on the device): blocks
  // loop over subsets, tiles or counter chunks and return when there are none
  hook.run("big_sample", [&] { k_big_sample<LOGV><<<sms * 8, kBlock, 0, st>>>(ctl, &ctl->next_item[0]); });
  hook.run("big_classify", [&] { k_big_classify<LOGV><<<sms * 8, kBlock, 0, st>>>(ctl, &ctl->next_item[1]); });
  hook.run("scan", [&] { k_scan_reduce<<<sms * 8, kBlock, 0, st>>>(ctl); });
  hook.run("scan", [&] { k_scan_down<<<sms * 8, kBlock, 0, st>>>(ctl); });
  hook.run("big_emit", [&] { k_big_emit<LOGV><<<sms * 8, kBlock, 0, st>>>(ctl, &ctl->next_item[2]); });
  hook.run("big_scatter", [&] { k_big_scatter<LOGV><<<sms * 3, kBlock, smem, st>>>(ctl, &ctl->next_item[3]); });
  return cudaGetLastError();
}

cudaError_t launch_big_round(int logv, BigCtl* ctl, uint32_t R_max, uint32_t sms, cudaStream_t st,
                             const LaunchHook& hook) {
  switch (logv) {
    case 8: return launch_big_round_t<8>(ctl, R_max, sms, st, hook);
    case 9: return launch_big_round_t<9>(ctl, R_max, sms, st, hook);
    default: return cudaErrorInvalidValue;  // 2^10 wide splitters exceed static shared memory
  }
}

uint64_t graph_launch_count() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_graph_launches, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}

}  // namespace ss
