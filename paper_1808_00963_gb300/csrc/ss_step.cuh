// Building blocks of one Super Scalar String Sample Sort step (Algorithm 4.1),
// written for a 256-thread block.  Used by the multi-block step kernels and by
// the persistent single-block kernel.
#pragma once

#include "ss_internal.cuh"

namespace ss {

constexpr uint32_t kBlock = 256;
constexpr uint32_t kWarps = kBlock / 32;
constexpr uint32_t kMaxRounds = 32;                  // tile = 256 * rounds records
constexpr uint32_t kMaxTile = kBlock * kMaxRounds;
constexpr uint32_t kFin = 1u << 31;                  // bucket descriptor: finished
constexpr uint32_t kNulEq = 1u << 30;                // ... all members equal strings
constexpr uint32_t kLow30 = (1u << 30) - 1;

// v = 2^LOGV - 1 splitters x_0..x_{v-1}, k = 2v + 1 buckets (Section 4.2.2).
template <int LOGV>
struct Geo {
  static constexpr uint32_t V = (1u << LOGV) - 1;
  static constexpr uint32_t K = 2 * V + 1;
  static constexpr uint32_t KP = 2u << LOGV;        // K rounded up to a power of two
  static constexpr uint32_t S = 2u << LOGV;         // sample size alpha * (v + 1), alpha = 2
};

// Splitters of one step (K: uint64_t for narrow keys, u128 for wide ones).
template <int LOGV, typename K = uint64_t>
struct Splitters {
  K tree[Geo<LOGV>::V + 1];  // t[1..v], level order (t[0] unused)
  K x[Geo<LOGV>::V + 1];     // x_0..x_{v-1} sorted; x[v] unused
  uint8_t hp[Geo<LOGV>::V + 1];     // h'_0..h'_v: lcp of neighbouring splitters
};

// Scratch of the splitter construction (may alias other shared memory).
template <int LOGV, typename K = uint64_t>
struct BuildScratch {
  K sample[Geo<LOGV>::S];
  uint16_t lo[Geo<LOGV>::S];   // first sample position with a key >= sample[i]
  uint16_t hi[Geo<LOGV>::S];   // first sample position with a key >  sample[i]
};

// Ascending bitonic sort of the 32 * E keys a warp holds, E per lane in
// index order lane * E + e: partners closer than E sit in the same lane,
// farther ones are exchanged with shuffles.
template <int E, typename K>
__device__ __forceinline__ void warp_bitonic(K (&v)[E]) {
  constexpr uint32_t N = 32 * E;
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (uint32_t k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= E) {
        const uint32_t lj = j / E;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const K o = KeyOps<K>::shfl_xor(v[e], (int)lj);
          const bool up = ((lane * E + e) & k) == 0;
          const bool take_min = lower == up;
          v[e] = take_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & j) == 0) {
            const int f = e | (int)j;
            const bool up = ((lane * E + e) & k) == 0;
            if ((v[e] > v[f]) == up) {
              const K t = v[e];
              v[e] = v[f];
              v[f] = t;
            }
          }
        }
      }
    }
  }
}

// The sampling steps of Algorithm 4.1 for the len keys at `keys`: draw a sample of
// alpha * (v + 1) keys at pseudo-random positions, sort it, select the
// splitters with the recursive duplicate-skipping rule of Section 4.2.3
// ("Sampling"): the middle sample of a range becomes the splitter, the ranges
// left and right of the run of samples equal to it are split recursively.
// A node whose range is empty takes the sample just above its range (the
// nearest splitter on the right among its ancestors), or all-ones past the
// end, which keeps t a search tree.  Finally h'_i = lcp(x_{i-1}, x_i) with
// h'_0 = h'_v = 0, the splitter LCPs of Algorithm 4.1.
// The sample is sorted warp by warp in registers and merged by computing each
// key's rank (its position in its chunk plus, in every other chunk, the keys
// before it: <= for earlier chunks, < for later ones).  With the run of equal
// keys around every sample position known, each tree node finds its range by
// walking from the root along its level-order index, so the recursion needs
// no step-by-step synchronisation.  Ends with __syncthreads().
// key_at(pos) gives the key of the subset's record pos.
template <int LOGV, typename K, typename KeyAt>
__device__ void build_splitters_k(KeyAt&& key_at, uint32_t len, uint64_t hseed, Splitters<LOGV, K>& sp,
                                  BuildScratch<LOGV, K>& bs, uint32_t dna) {
  using G = Geo<LOGV>;
  constexpr uint32_t C = G::S / kWarps;  // keys per warp
  constexpr int E = (int)(C / 32);       // keys per lane
  static_assert(E >= 1 && C % 32 == 0, "sample does not split into whole warps");
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  K v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = w * C + lane * E + e;
    const uint64_t h = mix64(hseed + i);
    const uint32_t pos = (uint32_t)(((h >> 32) * (uint64_t)len) >> 32);
    v[e] = key_at(pos);
  }
  warp_bitonic<E, K>(v);
  K* s = bs.sample;
#pragma unroll
  for (int e = 0; e < E; ++e) s[w * C + lane * E + e] = v[e];
  __syncthreads();
  uint32_t rank[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    uint32_t r = lane * E + e;
#pragma unroll
    for (uint32_t ww = 0; ww < kWarps; ++ww) {
      if (ww == w) continue;
      const K* ch = s + ww * C;
      uint32_t a = 0, b = C;
      if (ww < w) {
        while (a < b) { const uint32_t m = (a + b) >> 1; if (ch[m] <= v[e]) a = m + 1; else b = m; }
      } else {
        while (a < b) { const uint32_t m = (a + b) >> 1; if (ch[m] < v[e]) a = m + 1; else b = m; }
      }
      r += a;
    }
    rank[e] = r;
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) s[rank[e]] = v[e];
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < G::S; i += blockDim.x) {
    const K val = s[i];
    uint32_t a = 0, b = i;
    while (a < b) { const uint32_t m = (a + b) >> 1; if (s[m] < val) a = m + 1; else b = m; }
    bs.lo[i] = (uint16_t)a;
    a = i + 1;
    b = G::S;
    while (a < b) { const uint32_t m = (a + b) >> 1; if (s[m] <= val) a = m + 1; else b = m; }
    bs.hi[i] = (uint16_t)a;
  }
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < G::V; q += blockDim.x) {
    const uint32_t i = q + 1;               // level-order index
    const int l = 31 - __clz(i);            // its level
    uint32_t a = 0, b = G::S;               // its range of the sorted sample
    for (int d = l - 1; d >= 0; --d) {
      if (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (((i >> d) & 1u) == 0) {
          const uint32_t le = bs.lo[m];
          b = le > a ? le : a;              // left of the run of keys equal to s[m]
        } else {
          const uint32_t rs = bs.hi[m];
          a = rs < b ? rs : b;              // right of that run
        }
      } else {
        a = b;
      }
    }
    const K val = a < b ? s[(a + b) >> 1] : (b < G::S ? s[b] : KeyOps<K>::ones());
    sp.tree[i] = val;
    sp.x[(2 * (i - (1u << l)) + 1) * (1u << (LOGV - 1 - l)) - 1] = val;
  }
  __syncthreads();
  for (uint32_t r = threadIdx.x; r <= G::V; r += blockDim.x)
    sp.hp[r] = (r == 0 || r == G::V) ? 0 : (uint8_t)KeyOps<K>::lcp(sp.x[r - 1], sp.x[r], dna);
  if (threadIdx.x == 0) sp.tree[0] = 0;
  __syncthreads();
}

// The sampling steps for a subset of narrow records.
template <int LOGV>
__device__ __forceinline__ void build_splitters(const Rec* __restrict__ recs, uint32_t len, uint64_t hseed,
                                                Splitters<LOGV>& sp, BuildScratch<LOGV>& bs, uint32_t dna) {
  build_splitters_k<LOGV, uint64_t>([&](uint32_t pos) { return recs[pos].key; }, len, hseed, sp, bs, dna);
}

// Lemma 4.1: one-based level-order index l <-> one-based pre-order index p
// (the position of the vertex's splitter in sorted order) of a perfect binary
// tree with w levels, by rotating the bits around the first (resp. last) one
// bit.
__device__ __forceinline__ uint32_t level_to_pre(uint32_t l, uint32_t w) {
  const uint32_t s = 31 - __clz(l);  // bits after the first one bit
  const uint32_t x = w - s;          // position of the first one bit, from the top
  return ((l & ((1u << s) - 1)) << x) | (1u << (x - 1));
}

__device__ __forceinline__ uint32_t pre_to_level(uint32_t p, uint32_t w) {
  const uint32_t t = (uint32_t)__ffs(p) - 1;  // bits after the last one bit
  const uint32_t y = w - t;                    // position of the last one bit, from the top
  return (1u << (y - 1)) | (p >> (t + 1));
}

// Classification variants of Section 4.2.3 (they give the same buckets up to
// the numbering of empty ones, hence the same output).
constexpr uint32_t kClassifyUI = 0;   // unrolled <=-descent, equality test on the sorted copy x
constexpr uint32_t kClassifyUIC = 1;  // same descent, equality test in t via Lemma 4.1 (no copy needed)
constexpr uint32_t kClassifyE = 2;    // equality test at every node of the descent
constexpr uint32_t kClassifyUIJ = 3;  // UI entered through a jump table over the key's top bits

// Jump tables (Section 4.4, "Jump tables"): for every value p of a key's top
// kJumpBits bits, the first node of the descent whose splitter does not
// decide by those bits alone (its top bits equal p), or the leaf reached
// (>= 2^LOGV) when every splitter on the way decides.  Keys with top bits p
// take the same path down to that node, so the descent can start there.
constexpr int kJumpBits = 12;
constexpr uint32_t kJumpSize = 1u << kJumpBits;

template <int LOGV, typename K>
__device__ __forceinline__ uint32_t jump_entry(uint32_t p, const K* tree) {
  uint32_t i = 1;
  while (i < (1u << LOGV)) {
    const uint32_t tp = KeyOps<K>::top(tree[i], kJumpBits);
    if (p == tp) break;
    i = 2 * i + (p > tp ? 1u : 0u);
  }
  return i;
}

// The UI classification entered at the jump table's node: the remaining
// levels are predicated off for keys already at a leaf.
template <int LOGV, typename K>
__device__ __forceinline__ uint32_t classify_jump(K c, const K* tree, const K* x, const uint16_t* jump) {
  uint32_t i = jump[KeyOps<K>::top(c, kJumpBits)];
#pragma unroll
  for (int l = 0; l < LOGV; ++l)
    if (i < (1u << LOGV)) i = 2 * i + (c > tree[i] ? 1u : 0u);
  const uint32_t r = i - (1u << LOGV);
  const bool eq = r < Geo<LOGV>::V && x[r] == c;
  return 2 * r + (eq ? 1u : 0u);
}

// The classification of one key in Algorithm 4.1: branch-free descent of the level-order tree,
// i := 2i + [c > t_i] (the reading of its descent step under which bucket b_{2r} holds
// x_{r-1} < c < x_r), then the single equality test with x_r.
template <int LOGV, typename K>
__device__ __forceinline__ uint32_t classify(K c, const K* tree, const K* x, uint32_t variant = kClassifyUI) {
  uint32_t i = 1;
  if (variant == kClassifyE) {
    uint32_t eq = 0;
#pragma unroll
    for (int l = 0; l < LOGV; ++l) {
      const K t = tree[i];
      if (!eq && c == t) eq = i;
      i = 2 * i + (c > t ? 1u : 0u);
    }
    if (eq) return 2 * (level_to_pre(eq, LOGV) - 1) + 1;
    return 2 * (i - (1u << LOGV));
  }
#pragma unroll
  for (int l = 0; l < LOGV; ++l) i = 2 * i + (c > tree[i] ? 1u : 0u);
  const uint32_t r = i - (1u << LOGV);
  bool eq = false;
  if (r < Geo<LOGV>::V) eq = (variant == kClassifyUIC) ? tree[pre_to_level(r + 1, LOGV)] == c : x[r] == c;
  return 2 * r + (eq ? 1u : 0u);
}

// Buckets of U keys.  For S5-UI the U descents advance one tree level at a
// time together, so that U independent shared-memory loads are in flight per
// level rather than one (20 M URL strings: the classification 0.64 -> 0.55 ms).
template <int LOGV, int U, typename K>
__device__ __forceinline__ void classify_batch(const K (&k)[U], uint32_t (&b)[U], const K* tree, const K* x,
                                               uint32_t variant, const uint16_t* jump) {
  if (variant == kClassifyUI) {
    uint32_t i[U];
#pragma unroll
    for (int u = 0; u < U; ++u) i[u] = 1;
#pragma unroll
    for (int l = 0; l < LOGV; ++l) {
#pragma unroll
      for (int u = 0; u < U; ++u) i[u] = 2 * i[u] + (k[u] > tree[i[u]] ? 1u : 0u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t r = i[u] - (1u << LOGV);
      b[u] = 2 * r + ((r < Geo<LOGV>::V && x[r] == k[u]) ? 1u : 0u);
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < U; ++u)
    b[u] = (variant == kClassifyUIJ && jump) ? classify_jump<LOGV, K>(k[u], tree, x, jump)
                                             : classify<LOGV, K>(k[u], tree, x, variant);
}

// Classifies n keys (the classification loop of Algorithm 4.1): writes the bucket of
// keys[p] to bo[p] and counts it in hist (one shared-memory atomic per key:
// cheaper than grouping a warp's equal buckets with __match_any_sync first).  Each thread loads 8 keys before descending the tree for them,
// so that the loads of a batch overlap.  Returns this thread's records.
template <int LOGV, typename K, typename KeyAt>
__device__ __forceinline__ uint32_t classify_count_k(KeyAt&& key_at, uint16_t* __restrict__ bo, uint32_t n,
                                                     const K* tree, const K* x, uint32_t* hist, uint32_t variant,
                                                     const uint16_t* jump, unsigned long long* bmin = nullptr,
                                                     unsigned long long* bmax = nullptr) {
  constexpr int U = sizeof(K) == 8 ? 8 : 4;  // keys per thread in flight (wide keys take 4 registers)
  uint32_t mine = 0;
  const uint32_t lim = (n + kBlock - 1) / kBlock * kBlock;
  for (uint32_t p0 = threadIdx.x; p0 < lim; p0 += U * kBlock) {
    K k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t p = p0 + u * kBlock;
      k[u] = p < n ? key_at(p) : (K)0;
    }
    uint32_t bb[U];
    classify_batch<LOGV, U, K>(k, bb, tree, x, variant, jump);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t p = p0 + u * kBlock;
      if (p >= lim) break;  // uniform across the block
      const bool valid = p < n;
      const uint32_t b = valid ? bb[u] : 0xFFFFu;
      if (valid) {
        bo[p] = (uint16_t)b;
        ++mine;
      }
      if (valid) atomicAdd(&hist[b], 1u);
      if constexpr (sizeof(K) == 8) {
        // smallest and largest key of each even bucket (an equality bucket's
        // keys all equal its splitter), for the LCPs at bucket boundaries
        if (bmin && valid && !(b & 1u)) {
          atomicMin(&bmin[b], (unsigned long long)k[u]);
          atomicMax(&bmax[b], (unsigned long long)k[u]);
        }
      }
    }
  }
  return mine;
}

template <int LOGV>
__device__ __forceinline__ uint32_t classify_count(const Rec* __restrict__ recs, uint16_t* __restrict__ bo,
                                                   uint32_t n, const uint64_t* tree, const uint64_t* x,
                                                   uint32_t* hist, uint32_t variant,
                                                   const uint16_t* jump = nullptr) {
  return classify_count_k<LOGV, uint64_t>([&](uint32_t p) { return recs[p].key; }, bo, n, tree, x, hist, variant,
                                          jump);
}

// What happens to bucket b of a step at depth h (Output of Algorithm 4.1 and
// Section 4.2.3): an even bucket b_{2r} continues at depth h + h'_r, an
// equality bucket at h + 8, unless its splitter holds the terminator (then all
// members are equal strings and the bucket is finished; their LCP is their
// length); a single string is finished.
template <int LOGV, typename K>
__device__ __forceinline__ uint32_t bucket_desc(uint32_t b, uint32_t size, uint32_t depth,
                                                const Splitters<LOGV, K>& sp, uint32_t dna) {
  const uint32_t r = b >> 1;
  if (b & 1) {
    const K xr = sp.x[r];
    if (KeyOps<K>::end(xr, dna)) return kFin | kNulEq | (depth + KeyOps<K>::nnz(xr, dna));
    if (size == 1) return kFin;
    return depth + KeyOps<K>::width(dna);
  }
  if (size == 1) return kFin;
  return depth + sp.hp[r];
}

// Records moved per batch of one warp in the distribution: the loads of a
// batch are issued together so that each warp keeps kMoveBatch rounds of
// memory accesses in flight.  4 (not 8) keeps the multi-block distribution at
// 64 registers, 4 blocks per SM: more warps in flight beat deeper batches.
constexpr int kMoveBatch = 4;
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

// The lanes of the warp whose record falls into the same bucket b as this
// lane's (valid lanes only; every lane of the warp calls it): the mask of
// valid lanes narrowed by one ballot per bit of the bucket index.  Cheaper to
// issue than __match_any_sync (measured on the distribution) and stable in
// lane order like it.
template <int LOGV>
__device__ __forceinline__ uint32_t bucket_peers(uint32_t b, bool valid) {
  uint32_t m = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
  for (int i = 0; i <= LOGV; ++i) {  // bucket indices have LOGV + 1 bits
    const bool bit = (b >> i) & 1u;
    const uint32_t v = __ballot_sync(0xFFFFFFFFu, bit);
    m &= bit ? v : ~v;
  }
  return m;
}

// Stable distribution of one tile of records (the redistribution of Algorithm 4.1 with the
// per-processor bucket arrays of Theorem 4.4, one per warp).
//   tb[0..tl)    bucket of each record of the tile (shared memory)
//   base[b]      in: destination of the tile's first record of bucket b;
//                out: base[b] + number of the tile's records in bucket b
//   cntw         shared scratch, kWarps * KP uint32
// Warp w owns records [w * 32R, (w + 1) * 32R) of the tile; inside a warp
// ranks come from the lanes with the same bucket (bucket_peers), so equal
// buckets keep input order.
// move(p[], b[], dest[]) is called with kMoveBatch rounds of one warp at a time
// (p = kInvalid for lanes without a record).  Ends with __syncthreads().
template <int LOGV, int MB = kMoveBatch, typename Move>
__device__ void tile_scatter(const uint16_t* tb, uint32_t tl, uint32_t R, uint32_t* base,
                             uint32_t* cntw, Move&& move) {
  using G = Geo<LOGV>;
  const uint32_t w = threadIdx.x >> 5, lane = lane_id();
  for (uint32_t i = threadIdx.x; i < kWarps * G::KP; i += blockDim.x) cntw[i] = 0;
  __syncthreads();
  uint32_t* mine = cntw + w * G::KP;
  const uint32_t p0 = w * 32 * R;
  for (uint32_t r = 0; r < R; ++r) {
    const uint32_t p = p0 + r * 32 + lane;
    if (p < tl) atomicAdd(&mine[tb[p]], 1u);  // counts only: no need to group equal buckets
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < G::K; b += blockDim.x) {
    uint32_t run = base[b];
#pragma unroll
    for (uint32_t ww = 0; ww < kWarps; ++ww) {
      const uint32_t c = cntw[ww * G::KP + b];
      cntw[ww * G::KP + b] = run;
      run += c;
    }
    base[b] = run;
  }
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  for (uint32_t r0 = 0; r0 < R; r0 += MB) {
    uint32_t pp[MB], bb[MB], dd[MB];
#pragma unroll
    for (int u = 0; u < MB; ++u) {
      const uint32_t r = r0 + u;
      const uint32_t p = p0 + r * 32 + lane;
      const bool valid = r < R && p < tl;
      const uint32_t b = valid ? tb[p] : 0u;
      const uint32_t peers = bucket_peers<LOGV>(b, valid);
      uint32_t dest = 0;
      if (valid) dest = mine[b] + __popc(peers & lt);
      __syncwarp();
      if (valid && lane == (uint32_t)(__ffs(peers) - 1)) mine[b] += __popc(peers);
      __syncwarp();
      pp[u] = valid ? p : kInvalid;
      bb[u] = b;
      dd[u] = dest;
    }
    move(pp, bb, dd);
  }
  __syncthreads();
}

// Moves a batch of records to their buckets (the body of the redistribution): a finished
// record writes its final index (and, inside a bucket of equal strings, its
// LCP); an open one is copied to the other buffer with its cache reloaded at
// the bucket's new depth (fused character gather).  All loads of the batch
// are issued before any of them is used.  bucket_first(b) is the position of
// the first record of bucket b.  Returns the algorithmic bytes: bucket index 2
// + record 16 read (the record carries the string's offset); finished: perm 4
// (+ lcp 4) written; open: record 16 written, plus 8 characters read when the
// cache is reloaded.
template <typename First>
__device__ __forceinline__ uint32_t move_batch(const SortCtx& c, const SetDesc& sd, uint32_t wide, uint32_t par,
                                               uint32_t src0, uint32_t depth, const uint32_t* desc,
                                               First&& bucket_first, const uint32_t (&pp)[kMoveBatch],
                                               const uint32_t (&bb)[kMoveBatch], const uint32_t (&dd)[kMoveBatch]) {
  uint32_t id[kMoveBatch], ds[kMoveBatch], o32[kMoveBatch];
  uint64_t key[kMoveBatch], off[kMoveBatch];
  uint32_t bytes = 0;
#pragma unroll
  for (int u = 0; u < kMoveBatch; ++u) {
    id[u] = 0;
    o32[u] = 0;
    ds[u] = kFin;
    key[u] = 0;
    if (pp[u] != kInvalid) {
      ds[u] = desc[bb[u]];
      const Rec r = load_rec(c.rec[par] + src0 + pp[u]);
      id[u] = r.idx;
      key[u] = r.key;
      o32[u] = r.off;
    }
  }
  // the characters of every byte-string reload are requested before any of
  // them is used (one memory round trip for the batch)
  WindowWords<1> ww[kMoveBatch];
#pragma unroll
  for (int u = 0; u < kMoveBatch; ++u) {
    off[u] = 0;
    if (pp[u] != kInvalid && !(ds[u] & kFin) && (ds[u] & kLow30) != depth) {
      off[u] = rec_offset(sd, wide, id[u], o32[u]);
      if (!sd.dna) issue_windows<1>(sd.chars, off[u], ds[u] & kLow30, sd.cap, ww[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < kMoveBatch; ++u) {
    if (pp[u] == kInvalid) continue;
    const uint32_t d = ds[u];
    const uint32_t dest = dd[u];
    if (d & kFin) {
      sd.perm[dest - sd.base] = id[u];
      bytes += 22;
      if (sd.lcp && (d & kNulEq) && dest != bucket_first(bb[u])) {
        sd.lcp[dest - sd.base] = d & kLow30;
        bytes += 4;
      }
      continue;
    }
    const uint32_t nd = d & kLow30;
    uint64_t k = key[u];
    bytes += 34;
    if (nd != depth) {
      if (sd.dna) {
        k = load_key(sd.chars, off[u], nd, sd.cap, 1u);
      } else {
        uint64_t w[1];
        // bytes past the 4 KiB block of the first character decide: word by word
        k = finish_windows<1>(ww[u], sd.chars, off[u], nd, sd.cap, w) ? w[0] : load_cache(sd.chars, off[u], nd, sd.cap);
      }
      bytes += 8;
    }
    store_rec(c.rec[par ^ 1] + dest, k, id[u], o32[u]);
  }
  return bytes;
}

// move_batch for records of a multi-block subset, held in the wide form (wide
// key in the record slot, (idx, off) in wid[]).  A record whose new bucket is
// itself a multi-block subset stays wide (key reloaded at the new depth unless
// the depth is unchanged); otherwise it becomes a narrow record, whose key is
// cut out of the wide one when the new depth is at most 8 characters deeper
// (bytes), or is the first or second half of it (DNA codes, 0 or 21 deeper),
// and gathered from the string otherwise.  bucket_first(b) is the position of
// bucket b's first record (bucket_first(b + 1) - bucket_first(b) its size).
// Returns the algorithmic bytes: bucket index 2 + wide record 24 read;
// finished: perm 4 (+ lcp 4) written; open: 24 (wide) or 16 (narrow) written,
// plus 16 (wide) or 8 (narrow) characters read when gathered.
template <int MB, typename First>
__device__ __forceinline__ uint32_t move_batch_wide(const SortCtx& c, const SetDesc& sd, uint32_t wide,
                                                    uint32_t par, uint32_t src0, uint32_t depth, const uint32_t* desc,
                                                    First&& bucket_first, const uint32_t (&pp)[MB],
                                                    const uint32_t (&bb)[MB], const uint32_t (&dd)[MB]) {
  constexpr uint32_t kSkip = 0, kFinal = 1, kKeep = 2, kGather = 3;  // what a record needs
  uint32_t ds[MB], how[MB];
  bool to_wide[MB];
  uint2 wi[MB];
  u128 key[MB];
  uint32_t bytes = 0;
#pragma unroll
  for (int u = 0; u < MB; ++u) {
    ds[u] = kFin;
    wi[u] = make_uint2(0, 0);
    key[u] = 0;
    if (pp[u] != kInvalid) {
      ds[u] = desc[bb[u]];
      key[u] = load_wkey(c.rec[par] + src0 + pp[u]);
      wi[u] = c.wid[par][src0 + pp[u]];
    }
  }
  // what each record needs; the characters of every byte-string gather are
  // requested before any of them is used (one memory round trip for the batch)
  WindowWords<2> ww[MB];
#pragma unroll
  for (int u = 0; u < MB; ++u) {
    how[u] = kSkip;
    to_wide[u] = false;
    if (pp[u] == kInvalid) continue;
    const uint32_t d = ds[u];
    if (d & kFin) {
      how[u] = kFinal;
      continue;
    }
    const uint32_t adv = (d & kLow30) - depth;
    const uint32_t size = bucket_first(bb[u] + 1) - bucket_first(bb[u]);
    to_wide[u] = c.big_enabled && size > c.big_threshold;
    const bool derive = to_wide[u] ? adv == 0 : (sd.dna ? (adv == 0 || adv == kDnaWidth) : adv <= 8);
    how[u] = derive ? kKeep : kGather;
    if (!derive && !sd.dna)  // a narrow key needs the first window only: two words, not three
      issue_windows<2>(sd.chars, rec_offset(sd, wide, wi[u].x, wi[u].y), d & kLow30, sd.cap, ww[u],
                       to_wide[u] ? 3u : 2u);
  }
#pragma unroll
  for (int u = 0; u < MB; ++u) {
    if (how[u] == kSkip) continue;
    const uint32_t dest = dd[u];
    if (how[u] == kFinal) {
      sd.perm[dest - sd.base] = wi[u].x;
      bytes += 30;
      if (sd.lcp && (ds[u] & kNulEq) && dest != bucket_first(bb[u])) {
        sd.lcp[dest - sd.base] = ds[u] & kLow30;
        bytes += 4;
      }
      continue;
    }
    const uint32_t nd = ds[u] & kLow30;
    const uint32_t adv = nd - depth;
    u128 k = key[u];
    if (how[u] == kGather) {
      if (sd.dna) {
        const uint64_t o = rec_offset(sd, wide, wi[u].x, wi[u].y);
        k = to_wide[u] ? load_key128(sd.chars, o, nd, sd.cap, 1u) : make_k(dna_key(sd.chars, o, nd, sd.cap), 0);
      } else {
        uint64_t w[2];
        const uint64_t o = rec_offset(sd, wide, wi[u].x, wi[u].y);
        const uint32_t nw = finish_windows<2>(ww[u], sd.chars, o, nd, sd.cap, w);
        // bytes past the 4 KiB block of the first character decide: word by word
        if (nw == 0) w[0] = load_cache(sd.chars, o, nd, sd.cap);
        if (to_wide[u] && nw < 2) w[1] = has_nul(w[0]) ? 0ull : load_cache(sd.chars, o, nd + 8, sd.cap);
        k = make_k(w[0], w[1]);
      }
      bytes += to_wide[u] ? 16 : 8;
    }
    if (to_wide[u]) {
      bytes += 50;
      store_wkey(c.rec[par ^ 1] + dest, k);
      c.wid[par ^ 1][dest] = wi[u];
    } else {
      bytes += 42;
      // a gathered narrow key is the first half; a kept one is cut out of the wide key
      const uint64_t nk = how[u] == kGather ? k_hi(k) : (sd.dna ? (adv ? k_lo(k) : k_hi(k)) : narrow_at(k, adv));
      store_rec(c.rec[par ^ 1] + dest, nk, wi[u].x, wi[u].y);
    }
  }
  return bytes;
}

// Emits the outcome of one non-empty bucket: its boundary LCP mark (resolved at
// the end, Section 4.2.8 "LCP Calculation": the LCP with the previous bucket is
// depth + lcp of the two strings' caches at this depth) and, if it is not
// finished, a new task.
__device__ __forceinline__ void emit_bucket(const SortCtx& c, const SetDesc& sd, const Task& t,
                                            uint32_t start, uint32_t size, uint32_t desc,
                                            uint32_t next_big, uint32_t mark = kLcpMark) {
  if (mark && start > 0 && sd.lcp) sd.lcp[t.begin + start - sd.base] = mark | t.depth;
  if (!(desc & kFin)) {
    Task ch{t.begin + start, size, desc & kLow30, make_meta(task_set(t), task_par(t) ^ 1)};
    route_task(c, ch, next_big);
  }
}

}  // namespace ss
