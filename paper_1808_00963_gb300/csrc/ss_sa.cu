// Suffix array construction by prefix doubling (Section 8.2, Observation 8.1,
// Algorithms 8.1 and 8.3) on top of the string sort.
//
// Round 0 sorts all suffixes by their first h0 characters with the string
// sort (a cap of h0) and names every suffix by the smallest rank of its
// h0-group (ISA^{h0}, names stored + 1 so that 0 stands for "past the end of
// the text").  Each following round takes only the suffixes of unfinished
// groups (those with more than one member; finished groups are discarded, as
// in Larsson and Sadakane's scheme), encodes the name pair (ISA^h[i],
// ISA^h[i + h]) of each as a 10-byte string of base-255 digits 1..255 (no zero
// byte, same order as the pair), sorts those strings with the string sort,
// writes them back into their groups' ranges of the suffix array and renames:
// a new 2h-group starts where the pair changes (LCP of the encoded strings
// below 10), its name is the suffix array position of its first member.  The
// kernels here are the per-round scans, compactions and conversions.
#include "ss_kernels.h"

namespace ss {

namespace {

constexpr uint32_t kScanBlock = 1024;
constexpr uint32_t kScanItems = 4;
constexpr uint32_t kScanTile = kScanBlock * kScanItems;
constexpr uint32_t kPairBytes = 10;   // two names of 5 base-255 digits
constexpr uint32_t kPairStride = 11;  // + terminator

struct OpSum {
  static __device__ __forceinline__ uint32_t id() { return 0u; }
  static __device__ __forceinline__ uint32_t f(uint32_t a, uint32_t b) { return a + b; }
};
struct OpMax {
  static __device__ __forceinline__ uint32_t id() { return 0u; }
  static __device__ __forceinline__ uint32_t f(uint32_t a, uint32_t b) { return a > b ? a : b; }
};

// Inclusive scan of one value per thread over the block (warp shuffles, then
// the warp totals); returns the block total through *total.
template <class Op>
__device__ __forceinline__ uint32_t block_inclusive(uint32_t v, uint32_t* warp_tot, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if (lane >= (uint32_t)d) v = Op::f(o, v);
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < kScanBlock / 32 ? warp_tot[lane] : Op::id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= (uint32_t)d) t = Op::f(o, t);
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  if (warp > 0) v = Op::f(warp_tot[warp - 1], v);
  *total = warp_tot[kScanBlock / 32 - 1];
  __syncthreads();
  return v;
}

// Phase 1: scan each tile in place (inclusive), tile totals to tot[b].
template <class Op>
__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(uint32_t* a, uint64_t n, uint32_t* tot) {
  __shared__ uint32_t wt[kScanBlock / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t x[kScanItems];
  uint32_t run = Op::id();
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    x[k] = base + k < n ? a[base + k] : Op::id();
    run = Op::f(run, x[k]);
    x[k] = run;
  }
  uint32_t total;
  const uint32_t incl = block_inclusive<Op>(run, wt, &total);
  const uint32_t excl_prev = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  // exclusive prefix of this thread = inclusive of the previous thread
  uint32_t before;
  {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane > 0) before = excl_prev;
    else before = warp > 0 ? wt[warp - 1] : Op::id();
  }
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k)
    if (base + k < n) a[base + k] = Op::f(before, x[k]);
  if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

// Phase 2: exclusive scan of the tile totals by one block, in chunks.
template <class Op>
__global__ void __launch_bounds__(kScanBlock) k_scan_totals(uint32_t* tot, uint32_t nt) {
  __shared__ uint32_t wt[kScanBlock / 32];
  uint32_t carry = Op::id();
  for (uint32_t c = 0; c < nt; c += kScanBlock) {
    const uint32_t i = c + threadIdx.x;
    const uint32_t v = i < nt ? tot[i] : Op::id();
    uint32_t total;
    const uint32_t incl = block_inclusive<Op>(v, wt, &total);
    // exclusive = carry (+) inclusive of the previous thread
    uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) prev = warp > 0 ? wt[warp - 1] : Op::id();
    __syncthreads();
    if (i < nt) tot[i] = Op::f(carry, prev);
    carry = Op::f(carry, total);
    __syncthreads();
  }
}

// Phase 3: combine each tile with the totals of the tiles before it.
template <class Op>
__global__ void __launch_bounds__(kScanBlock) k_scan_apply(uint32_t* a, uint64_t n, const uint32_t* tot) {
  const uint32_t pre = tot[blockIdx.x];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  for (uint32_t k = threadIdx.x; k < kScanTile; k += kScanBlock)
    if (base + k < n) a[base + k] = Op::f(pre, a[base + k]);
}

// ---- rounds ------------------------------------------------------------------------

__global__ void k_sa_iota(uint64_t* off, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    off[i] = i;
}

// After the first sort (LCPs capped at h0): gs[j] = j at the start of an
// h0-group, else 0 (for the max-scan that yields the group start).
__global__ void k_sa_heads0(const uint32_t* lcp0, uint32_t n, uint32_t h0, uint32_t* gs) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    gs[j] = (j == 0 || lcp0[j] < h0) ? j : 0u;
}

// Names after the first sort, and the positions of unfinished groups
// (flag[j] = 1 if the group of j has another member).
__global__ void k_sa_name0(const uint32_t* sa, const uint32_t* lcp0, const uint32_t* gs, uint32_t n, uint32_t h0,
                           uint32_t* isa, uint32_t* flag) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    isa[sa[j]] = gs[j] + 1;
    const bool head = j == 0 || lcp0[j] < h0;
    const bool next_same = j + 1 < n && lcp0[j + 1] >= h0;
    flag[j] = (!head || next_same) ? 1u : 0u;
  }
}

// Compaction from the inclusive sum of the 0/1 flags (j is flagged where the
// sum steps up): out[sum[j] - 1] = vals[j] (or j).
__global__ void k_sa_compact(const uint32_t* incl, const uint32_t* vals, uint32_t n, uint32_t* out) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t c = incl[j];
    if (c != (j ? incl[j - 1] : 0u)) out[c - 1] = vals ? vals[j] : j;
  }
}

__device__ __forceinline__ void put_digits(uint8_t* p, uint32_t v) {
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    p[k] = (uint8_t)(v % 255u + 1u);
    v /= 255u;
  }
}

// Name pairs of the unfinished members as 10-byte strings (+ terminator).
__global__ void k_sa_encode(const uint32_t* cpos, uint32_t M, const uint32_t* sa, const uint32_t* isa, uint32_t n,
                            uint32_t h, uint32_t* member, uint8_t* enc, uint64_t* eoff) {
  for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    const uint32_t i = sa[cpos[m]];
    member[m] = i;
    const uint32_t k1 = isa[i];
    const uint32_t k2 = (uint64_t)i + h < n ? isa[i + h] : 0u;
    uint8_t* p = enc + (uint64_t)m * kPairStride;
    put_digits(p, k1);
    put_digits(p + 5, k2);
    p[kPairBytes] = 0;
    eoff[m] = (uint64_t)m * kPairStride;
  }
}

// Write the sorted members back and mark the starts of the new groups.
__global__ void k_sa_apply(const uint32_t* cpos, uint32_t M, const uint32_t* member, const uint32_t* perm2,
                           const uint32_t* lcp2, uint32_t* sa, uint32_t* gs) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    sa[cpos[p]] = member[perm2[p]];
    gs[p] = (p == 0 || lcp2[p] < kPairBytes) ? cpos[p] : 0u;
  }
}

// New names of the members and the flags of the groups still unfinished.
__global__ void k_sa_rename(const uint32_t* member, const uint32_t* perm2, const uint32_t* lcp2, const uint32_t* gs,
                            uint32_t M, uint32_t* isa, uint32_t* flag) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    isa[member[perm2[p]]] = gs[p] + 1;
    const bool head = p == 0 || lcp2[p] < kPairBytes;
    const bool next_same = p + 1 < M && lcp2[p + 1] >= kPairBytes;
    flag[p] = (!head || next_same) ? 1u : 0u;
  }
}

// Final LCP array.  Entries below h0 come from the first sort (they sit at the
// starts of h0-groups, whose members were only permuted inside the group);
// k_sa_long_flags marks the others (flag 1 for j >= 1 with lcp >= h0) and
// k_sa_lcp gives each of them one warp.  Its first lane climbs down the name
// arrays of the rounds: suffixes a and b share their first h0 2^k characters
// from t on iff their names after round k at a + t and b + t agree, so taking
// each k from the last round down whenever they agree gives the largest
// multiple t of h0 with a and b equal in their first t characters (names do
// not agree past the end of the text).  The warp then compares the two
// suffixes from t on, 256 characters per step: lane k compares the
// 8-character windows at h + 8k, and the first lane that sees a difference
// (or the end of the shorter suffix) gives the LCP, fewer than h0 characters
// on.  The work per entry is O(rounds + h0 / 256) however long the LCP (a
// direct comparison from h0 took seconds on periodic texts).  A suffix at a
// has n - a characters, so no lane reads past the text.
__global__ void k_sa_long_flags(const uint32_t* lcp, uint32_t n, uint32_t h0, uint32_t* flag) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    flag[j] = (j > 0 && lcp[j] >= h0) ? 1u : 0u;
}

__global__ void k_sa_lcp(const uint8_t* text, const uint32_t* sa, uint32_t n, uint32_t h0, const uint32_t* pos,
                         uint32_t count, uint32_t* lcp, SaSnaps sn) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < count; w += warps) {
    const uint32_t j = pos[w];
    const uint64_t a = sa[j - 1], b = sa[j];
    const uint64_t la = n - a, lb = n - b;
    const uint64_t lmin = la < lb ? la : lb;
    unsigned long long t = h0;
    if (lane == 0 && sn.count) {
      t = 0;
      for (int k = (int)sn.count - 1; k >= 0; --k) {
        const uint32_t* nm = sn.p[k];
        if (a + t < n && b + t < n && nm[a + t] == nm[b + t]) t += (unsigned long long)h0 << k;
      }
    }
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    uint64_t h = t;
    uint64_t result = 0;
    while (true) {
      const uint64_t d = h + 8ull * lane;
      uint32_t stop = 8;  // characters that agree in this lane's window (8 = all)
      if (d >= lmin) {
        stop = 0;
      } else {
        const uint64_t ca = load_cache(text, a, (uint32_t)d, kNoCap);
        const uint64_t cb = load_cache(text, b, (uint32_t)d, kNoCap);
        if (ca != cb) stop = lcp8(ca, cb);
        else if (has_nul(ca)) stop = nnz_prefix(ca);
      }
      const uint32_t done = __ballot_sync(0xFFFFFFFFu, stop < 8);
      if (done) {
        const uint32_t first = __ffs(done) - 1;
        const uint32_t s_first = __shfl_sync(0xFFFFFFFFu, stop, first);
        result = h + 8ull * first + s_first;
        break;
      }
      h += 256;
    }
    if (lane == 0) lcp[j] = (uint32_t)result;
  }
}

template <class Op>
cudaError_t scan_impl(uint32_t* a, uint64_t n, uint32_t* tot, cudaStream_t st, const LaunchHook& hook) {
  if (n == 0) return cudaSuccess;
  const uint32_t nt = (uint32_t)((n + kScanTile - 1) / kScanTile);
  hook.run("sa_scan", [&] { k_scan_tiles<Op><<<nt, kScanBlock, 0, st>>>(a, n, tot); });
  if (nt > 1) {
    hook.run("sa_scan", [&] { k_scan_totals<Op><<<1, kScanBlock, 0, st>>>(tot, nt); });
    hook.run("sa_scan", [&] { k_scan_apply<Op><<<nt, kScanBlock, 0, st>>>(a, n, tot); });
  }
  return cudaGetLastError();
}

}  // namespace

size_t sa_scan_totals(uint64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t sa_scan_max(uint32_t* a, uint64_t n, uint32_t* tot, cudaStream_t st, const LaunchHook& hook) {
  return scan_impl<OpMax>(a, n, tot, st, hook);
}

cudaError_t sa_scan_sum(uint32_t* a, uint64_t n, uint32_t* tot, cudaStream_t st, const LaunchHook& hook) {
  return scan_impl<OpSum>(a, n, tot, st, hook);
}

cudaError_t sa_launch(SaKernel k, const SaArgs& x, uint32_t grid, cudaStream_t st, const LaunchHook& hook) {
  switch (k) {
    case SaKernel::kIota:
      hook.run("sa_iota", [&] { k_sa_iota<<<grid, 256, 0, st>>>(x.off, x.n); });
      break;
    case SaKernel::kHeads0:
      hook.run("sa_name", [&] { k_sa_heads0<<<grid, 256, 0, st>>>(x.lcp, (uint32_t)x.n, x.h, x.gs); });
      break;
    case SaKernel::kName0:
      hook.run("sa_name", [&] { k_sa_name0<<<grid, 256, 0, st>>>(x.sa, x.lcp, x.gs, (uint32_t)x.n, x.h, x.isa, x.flag); });
      break;
    case SaKernel::kCompact:
      hook.run("sa_compact", [&] { k_sa_compact<<<grid, 256, 0, st>>>(x.flag, x.vals, (uint32_t)x.n, x.out); });
      break;
    case SaKernel::kEncode:
      hook.run("sa_encode", [&] {
        k_sa_encode<<<grid, 256, 0, st>>>(x.cpos, x.M, x.sa, x.isa, (uint32_t)x.n, x.h, x.member, x.enc, x.eoff);
      });
      break;
    case SaKernel::kApply:
      hook.run("sa_apply", [&] { k_sa_apply<<<grid, 256, 0, st>>>(x.cpos, x.M, x.member, x.perm2, x.lcp2, x.sa, x.gs); });
      break;
    case SaKernel::kRename:
      hook.run("sa_name", [&] { k_sa_rename<<<grid, 256, 0, st>>>(x.member, x.perm2, x.lcp2, x.gs, x.M, x.isa, x.flag); });
      break;
    case SaKernel::kLongFlags:
      hook.run("sa_lcp", [&] { k_sa_long_flags<<<grid, 256, 0, st>>>(x.lcp_out, (uint32_t)x.n, x.h, x.flag); });
      break;
    case SaKernel::kLcp:
      hook.run("sa_lcp", [&] {
        k_sa_lcp<<<grid, 256, 0, st>>>(x.text, x.sa, (uint32_t)x.n, x.h, x.cpos, x.M, x.lcp_out, x.snaps);
      });
      break;
  }
  return cudaGetLastError();
}

}  // namespace ss
