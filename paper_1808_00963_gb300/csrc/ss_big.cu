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

__device__ __forceinline__ uint64_t cnt_base(const GenTask& g) {
  return ((uint64_t)g.cnt_base_hi << 32) | g.cnt_base_lo;
}

// Prefix jump.  A step sees 8 characters, so a subset whose strings share a
// long prefix (many URLs of one site, repeated records) would be moved once
// for every 8 shared characters.  When the whole sample of a subset is one key
// without a terminator, the sampling block measures how far 64 of the
// sampled strings agree with one of them over the next kPjWindows windows;
// if they agree beyond 32 characters, the classification measures the same
// for every string, and if the whole subset then falls into that key's
// equality bucket,
// the bucket continues at depth + the smallest agreement instead of depth + 8.
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
  Splitters<LOGV> sp;
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

// Smallest agreement with ref over the strings of records [0, n) taken by this
// block's threads (pos(i) gives the record of item i), reduced over the block.
template <typename Pos>
__device__ uint32_t block_min_agreement(const SortCtx& c, const Rec* recs, const SetDesc& sd, uint32_t wide,
                                        uint32_t depth, uint32_t items, Pos&& pos, const uint64_t* ref,
                                        unsigned long long& bytes) {
  __shared__ uint32_t bmin;
  if (threadIdx.x == 0) bmin = 0xFFFFFFFFu;
  __syncthreads();
  uint32_t mn = 0xFFFFFFFFu;
  for (uint32_t i = threadIdx.x; i < items; i += blockDim.x) {
    const Rec r = load_rec(recs + pos(i));
    uint64_t w[kPjWindows];
    load_pj_windows(sd.chars, rec_offset(sd, wide, r.idx, r.off), depth, sd.cap, w);
    mn = min(mn, window_lcp(w, ref));
    bytes += 8 + 8 * kPjWindows;  // the record's index and offset, the windows
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
  if ((threadIdx.x & 31u) == 0 && mn != 0xFFFFFFFFu) atomicMin(&bmin, mn);
  __syncthreads();
  return bmin;
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock) k_big_sample(SortCtx c, const GenTask* __restrict__ gt,
                                                       BigSplitters<LOGV>* __restrict__ out) {
  __shared__ __align__(16) Splitters<LOGV> sp;
  __shared__ __align__(16) BuildScratch<LOGV> bs;
  const GenTask g = gt[blockIdx.x];
  const Rec* recs = c.rec[task_par(g.t)] + g.t.begin;
  build_splitters<LOGV>(recs, g.t.len, mix64(c.seed ^ ((uint64_t)g.t.begin << 20) ^ g.t.depth), sp, bs,
                        c.sets[task_set(g.t)].dna);
  const uint64_t* src = reinterpret_cast<const uint64_t*>(&sp);
  uint64_t* dst = reinterpret_cast<uint64_t*>(&out[blockIdx.x].sp);
  for (uint32_t i = threadIdx.x; i < sizeof(Splitters<LOGV>) / 8; i += blockDim.x) dst[i] = src[i];
  unsigned long long bytes = threadIdx.x == 0 ? Geo<LOGV>::S * 8ull + sizeof(Splitters<LOGV>) : 0ull;
  // prefix jump: a one-key sample whose strings agree beyond kPjMinSample
  // characters turns on the check of the whole subset
  const SetDesc sd = c.sets[task_set(g.t)];
  const uint64_t k0 = bs.sample[0];  // the sorted sample
  const bool one_key = !sd.dna && k0 == bs.sample[Geo<LOGV>::S - 1] && !key_end(k0, 0u);
  uint32_t on = 0;
  uint64_t ref_off = 0;
  if (one_key) {  // uniform over the block
    const uint64_t hseed = mix64(c.seed ^ ((uint64_t)g.t.begin << 20) ^ g.t.depth);
    auto sample_pos = [&](uint32_t i) { return (uint32_t)(((mix64(hseed + i) >> 32) * (uint64_t)g.t.len) >> 32); };
    const uint32_t wide = c.wide[task_set(g.t)];
    __shared__ uint64_t ref[kPjWindows];
    const Rec r0 = load_rec(recs + sample_pos(0));
    ref_off = rec_offset(sd, wide, r0.idx, r0.off);
    if (threadIdx.x == 0) {
      uint64_t w[kPjWindows];
      load_pj_windows(sd.chars, ref_off, g.t.depth, sd.cap, w);
      for (int j = 0; j < kPjWindows; ++j) ref[j] = w[j];
    }
    __syncthreads();
    const uint32_t agree = block_min_agreement(c, recs, sd, wide, g.t.depth, kPjSampleChecks, sample_pos, ref, bytes);
    on = agree > kPjMinSample && agree != 0xFFFFFFFFu ? 1u : 0u;
  }
  if (threadIdx.x == 0) {
    out[blockIdx.x].pj_on = on;
    out[blockIdx.x].pj_lcp = 0xFFFFFFFFu;
    out[blockIdx.x].pj_ref = ref_off;
  }
  if (c.classifier == kClassifyUIJ) {
    for (uint32_t p = threadIdx.x; p < kJumpSize; p += blockDim.x)
      out[blockIdx.x].jump[p] = (uint16_t)jump_entry<LOGV>(p, sp.tree);
    if (threadIdx.x == 0) bytes += 2ull * kJumpSize;
  }
  // sample reads + splitter (and jump table) writes
  account(c, kKBigSample, bytes);
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock) k_big_classify(SortCtx c, const GenTask* __restrict__ gt,
                                                         uint32_t G, const BigSplitters<LOGV>* __restrict__ spl,
                                                         uint32_t* __restrict__ counters, uint32_t R) {
  using Gm = Geo<LOGV>;
  __shared__ __align__(16) uint64_t tree[Gm::V + 1];
  __shared__ __align__(16) uint64_t x[Gm::V + 1];
  __shared__ uint32_t hist[Gm::KP];
  __shared__ __align__(16) uint16_t jump[kJumpSize];
  __shared__ uint32_t s_g;
  if (threadIdx.x == 0) s_g = find_gen_task(gt, G, blockIdx.x);
  for (uint32_t b = threadIdx.x; b < Gm::KP; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const GenTask g = gt[s_g];
  const Splitters<LOGV>& sp = spl[s_g].sp;
  for (uint32_t i = threadIdx.x; i <= Gm::V; i += blockDim.x) { tree[i] = sp.tree[i]; x[i] = sp.x[i]; }
  const bool use_jump = c.classifier == kClassifyUIJ;
  if (use_jump) {
    const uint4* js = reinterpret_cast<const uint4*>(spl[s_g].jump);
    uint4* jd = reinterpret_cast<uint4*>(jump);
    for (uint32_t i = threadIdx.x; i < kJumpSize * 2 / 16; i += blockDim.x) jd[i] = js[i];
  }
  __syncthreads();
  const uint32_t tile = blockIdx.x - g.tile_start;
  const uint32_t T = kBlock * R;
  const uint32_t t0 = tile * T;
  const uint32_t tl = min(T, g.t.len - t0);
  const Rec* recs = c.rec[task_par(g.t)] + g.t.begin + t0;
  uint16_t* bo = c.bucket_of + g.t.begin + t0;
  const uint32_t mine = classify_count<LOGV>(recs, bo, tl, tree, x, hist, c.classifier, use_jump ? jump : nullptr);
  __syncthreads();
  uint32_t* cnt = counters + cnt_base(g) + tile;
  for (uint32_t b = threadIdx.x; b < Gm::K; b += blockDim.x) cnt[(uint64_t)b * g.tiles] = hist[b];
  // per record: cache 8 read + bucket index 2 written; per tile: K counters written
  unsigned long long bytes = 10ull * mine;
  if (threadIdx.x == 0) bytes += 4ull * Gm::K;
  if (spl[s_g].pj_on) {  // prefix jump: every string's agreement with the reference
    const SetDesc sd = c.sets[task_set(g.t)];
    __shared__ uint64_t ref[kPjWindows];
    if (threadIdx.x == 0) {
      uint64_t w[kPjWindows];
      load_pj_windows(sd.chars, spl[s_g].pj_ref, g.t.depth, sd.cap, w);
      for (int j = 0; j < kPjWindows; ++j) ref[j] = w[j];
    }
    __syncthreads();
    const uint32_t bmin = block_min_agreement(c, recs, sd, c.wide[task_set(g.t)], g.t.depth, tl,
                                              [](uint32_t i) { return i; }, ref, bytes);
    if (threadIdx.x == 0 && bmin != 0xFFFFFFFFu)
      atomicMin(&const_cast<BigSplitters<LOGV>*>(spl)[s_g].pj_lcp, bmin);
  }
  account(c, kKBigClassify, bytes);
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock) k_big_emit(SortCtx c, const GenTask* __restrict__ gt,
                                                     const BigSplitters<LOGV>* __restrict__ spl,
                                                     const uint32_t* __restrict__ scanned,
                                                     uint32_t* __restrict__ gstart, uint32_t* __restrict__ gdesc,
                                                     uint32_t next_big) {
  using Gm = Geo<LOGV>;
  const GenTask g = gt[blockIdx.x];
  const Splitters<LOGV>& sp = spl[blockIdx.x].sp;
  const SetDesc sd = c.sets[task_set(g.t)];
  const uint32_t* sc = scanned + cnt_base(g);
  unsigned long long bytes = 0;
  for (uint32_t b = threadIdx.x; b < Gm::K; b += blockDim.x) {
    bytes += 16;  // two bucket offsets read, start and descriptor written
    const uint32_t s = sc[(uint64_t)b * g.tiles] - g.rec_base;
    const uint32_t e = (b + 1 < Gm::K) ? sc[(uint64_t)(b + 1) * g.tiles] - g.rec_base : g.t.len;
    const uint32_t size = e - s;
    gstart[(uint64_t)blockIdx.x * Gm::KP + b] = s;
    uint32_t desc = kFin;
    if (size) {
      desc = bucket_desc<LOGV>(b, size, g.t.depth, sp, sd.dna);
      // prefix jump: the whole subset is the key's equality bucket, and every
      // string agrees with the reference for pj_lcp characters from the depth
      if (spl[blockIdx.x].pj_on && (b & 1u) && size == g.t.len && !(desc & kFin)) {
        const uint32_t J = spl[blockIdx.x].pj_lcp;
        if (J > 8u && J != 0xFFFFFFFFu) desc = g.t.depth + J;
      }
      emit_bucket(c, sd, g.t, s, size, desc, next_big);
    }
    gdesc[(uint64_t)blockIdx.x * Gm::KP + b] = desc;
  }
  account(c, kKBigEmit, bytes);
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock, 4) k_big_scatter(SortCtx c, const GenTask* __restrict__ gt, uint32_t G,
                                                        const uint32_t* __restrict__ scanned,
                                                        const uint32_t* __restrict__ gstart,
                                                        const uint32_t* __restrict__ gdesc, uint32_t R) {
  using Gm = Geo<LOGV>;
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* cntw = reinterpret_cast<uint32_t*>(smem);
  uint32_t* base = cntw + kWarps * Gm::KP;
  uint32_t* desc = base + Gm::KP;
  uint32_t* bfirst = desc + Gm::KP;
  uint16_t* tb = reinterpret_cast<uint16_t*>(bfirst + Gm::KP);
  __shared__ uint32_t s_g;
  if (threadIdx.x == 0) s_g = find_gen_task(gt, G, blockIdx.x);
  __syncthreads();
  const uint32_t gi = s_g;
  const GenTask g = gt[gi];
  const SetDesc sd = c.sets[task_set(g.t)];
  const uint32_t tile = blockIdx.x - g.tile_start;
  const uint32_t T = kBlock * R;
  const uint32_t t0 = tile * T;
  const uint32_t tl = min(T, g.t.len - t0);
  const uint32_t par = task_par(g.t);
  const uint16_t* bo = c.bucket_of + g.t.begin + t0;
  for (uint32_t p = threadIdx.x; p < tl; p += kBlock) tb[p] = bo[p];
  const uint32_t* sc = scanned + cnt_base(g) + tile;
  for (uint32_t b = threadIdx.x; b < Gm::K; b += kBlock) {
    base[b] = g.t.begin + sc[(uint64_t)b * g.tiles] - g.rec_base;
    desc[b] = gdesc[(uint64_t)gi * Gm::KP + b];
    bfirst[b] = g.t.begin + gstart[(uint64_t)gi * Gm::KP + b];
  }
  __syncthreads();
  const uint32_t src0 = g.t.begin + t0;
  const uint32_t depth = g.t.depth;
  const uint32_t wide = c.wide[task_set(g.t)];
  unsigned long long bytes = threadIdx.x == 0 ? 12ull * Gm::K : 0ull;  // per-bucket tile offsets
  tile_scatter<LOGV>(tb, tl, R, base, cntw, [&](const uint32_t(&pp)[kMoveBatch], const uint32_t(&bb)[kMoveBatch],
                                                const uint32_t(&dd)[kMoveBatch]) {
    bytes += move_batch(c, sd, wide, par, src0, depth, desc, [&](uint32_t b) { return bfirst[b]; }, pp, bb, dd);
  });
  account(c, kKBigScatter, bytes);
}

// ---- exclusive prefix sum over uint32 (three phases) ----------------------------

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

__global__ void __launch_bounds__(kBlock) k_scan_reduce(const uint32_t* __restrict__ a, uint64_t n,
                                                        uint32_t* __restrict__ part, SortCtx c) {
  const uint64_t b0 = (uint64_t)blockIdx.x * kScanChunk;
  uint32_t s = 0;
  for (uint32_t i = threadIdx.x; i < kScanChunk; i += kBlock) {
    const uint64_t k = b0 + i;
    if (k < n) s += a[k];
  }
  uint32_t ex;
  const uint32_t total = block_excl_scan(s, ex);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
  const uint64_t left = n > b0 ? n - b0 : 0;
  account(c, kKScan, threadIdx.x == 0 ? 4ull * (left < kScanChunk ? left : kScanChunk) : 0ull);
}

__global__ void __launch_bounds__(kBlock) k_scan_partials(uint32_t* __restrict__ part, uint32_t m) {
  uint32_t carry = 0;
  for (uint32_t i0 = 0; i0 < m; i0 += kBlock) {
    const uint32_t i = i0 + threadIdx.x;
    const uint32_t v = i < m ? part[i] : 0;
    uint32_t ex;
    const uint32_t total = block_excl_scan(v, ex);
    if (i < m) part[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kBlock) k_scan_down(uint32_t* __restrict__ a, uint64_t n,
                                                      const uint32_t* __restrict__ part, SortCtx c) {
  const uint64_t b0 = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (uint32_t j = 0; j < kScanItems; ++j) {
    const uint64_t k = b0 + j;
    v[j] = k < n ? a[k] : 0;
    s += v[j];
  }
  uint32_t ex;
  block_excl_scan(s, ex);
  uint32_t run = part[blockIdx.x] + ex;
#pragma unroll
  for (uint32_t j = 0; j < kScanItems; ++j) {
    const uint64_t k = b0 + j;
    if (k < n) a[k] = run;
    run += v[j];
  }
  const uint64_t left = n > b0 ? n - b0 : 0;
  account(c, kKScan, 8ull * (left < kScanItems ? left : kScanItems));
}

}  // namespace

size_t big_splitters_bytes(int logv) {
  switch (logv) {
    case 8: return sizeof(BigSplitters<8>);
    case 9: return sizeof(BigSplitters<9>);
    default: return sizeof(BigSplitters<10>);
  }
}

size_t big_scatter_smem(int logv, uint32_t R) {
  const uint32_t KP = 2u << logv;
  return (size_t)(kWarps * KP + 3 * KP) * 4 + (size_t)kBlock * R * 2;
}

template <int LOGV>
static cudaError_t launch_big_step_t(const BigStepArgs& a, cudaStream_t st, const LaunchHook& hook) {
  const size_t smem = big_scatter_smem(LOGV, a.R);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_big_scatter<LOGV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)big_scatter_smem(LOGV, kMaxRounds));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  auto* spl = reinterpret_cast<BigSplitters<LOGV>*>(a.splitters);
  hook.run("big_sample", [&] { k_big_sample<LOGV><<<a.G, kBlock, 0, st>>>(a.c, a.gt, spl); });
  hook.run("big_classify", [&] {
    k_big_classify<LOGV><<<a.tiles, kBlock, 0, st>>>(a.c, a.gt, a.G, spl, a.counters, a.R);
  });
  const uint32_t nb = (uint32_t)((a.ncounters + kScanChunk - 1) / kScanChunk);
  hook.run("scan", [&] { k_scan_reduce<<<nb, kBlock, 0, st>>>(a.counters, a.ncounters, a.partials, a.c); });
  hook.run("scan", [&] { k_scan_partials<<<1, kBlock, 0, st>>>(a.partials, nb); });
  hook.run("scan", [&] { k_scan_down<<<nb, kBlock, 0, st>>>(a.counters, a.ncounters, a.partials, a.c); });
  hook.run("big_emit", [&] {
    k_big_emit<LOGV><<<a.G, kBlock, 0, st>>>(a.c, a.gt, spl, a.counters, a.gstart, a.gdesc, a.next_big);
  });
  hook.run("big_scatter", [&] {
    k_big_scatter<LOGV><<<a.tiles, kBlock, smem, st>>>(a.c, a.gt, a.G, a.counters, a.gstart, a.gdesc, a.R);
  });
  return cudaGetLastError();
}

cudaError_t launch_big_step(int logv, const BigStepArgs& a, cudaStream_t st, const LaunchHook& hook) {
  switch (logv) {
    case 8: return launch_big_step_t<8>(a, st, hook);
    case 9: return launch_big_step_t<9>(a, st, hook);
    default: return launch_big_step_t<10>(a, st, hook);
  }
}

}  // namespace ss
