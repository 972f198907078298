// Persistent work-queue kernel: the GPU counterpart of the job queue of
// Section 4.2.8.  Each block repeatedly claims a subset from a device queue
// and runs one complete S^5 step on it (Algorithm 4.1: sample, splitter tree,
// classification, counting, prefix sum, stable redistribution).  Buckets that
// are still unsorted and larger than the small-sort cutoff are pushed back
// onto the same queue (an equality bucket whose splitter has no terminator is
// requeued at depth + 8); smaller ones go to the small-sort lists.
//
// Termination: `pending` counts tasks pushed and not yet finished; a block
// that finds its claimed slot empty exits once pending is 0.  Every wait is
// bounded (SortCtx::wait_ns of wall-clock time), after which the status word
// is latched and the block exits.
#include "ss_kernels.h"
#include "ss_step.cuh"

namespace ss {

namespace {

template <int LOGV>
struct QueueSmem {
  Splitters<LOGV> sp;
  uint32_t hist[Geo<LOGV>::KP];    // bucket sizes, then running destinations
  uint32_t bstart[Geo<LOGV>::KP];  // bucket starts relative to the task (KP >= K + 1)
  uint32_t desc[Geo<LOGV>::KP];
  union U {
    BuildScratch<LOGV> bs;
    struct {
      unsigned long long bmin[Geo<LOGV>::KP];  // smallest / largest key of each even bucket
      unsigned long long bmax[Geo<LOGV>::KP];
      uint32_t prev[Geo<LOGV>::KP];            // last non-empty bucket before each bucket, + 1 (0: none)
    } mm;
    struct {
      uint32_t cntw[kWarps * Geo<LOGV>::KP];
      uint16_t tb[kMaxTile];
    } sc;
  } u;
  Task task;
  uint32_t got;
};

// Claims the next task: waits (bounded) until it has been pushed, or until all
// work is done (no task pending: nothing can be pushed any more).
__device__ bool claim_task(const WorkQueue& q, Task* out, uint32_t* status, uint64_t wait_ns) {
  const uint32_t k = atomicAdd(q.head, 1u);
  const uint32_t slot = k % q.cap, lap = k / q.cap;
  const uint64_t t0 = globaltimer_ns();
  uint32_t ns = 64;
  volatile uint32_t* ready = q.ready;
  volatile uint32_t* pending = q.pending;
  while (true) {
    if (ready[slot] == 2 * lap + 1) {
      __threadfence();
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(q.items + slot));
      *out = Task{v.x, v.y, v.z, v.w};
      __threadfence();  // the task is read before the slot is handed to the next lap
      atomicExch(q.ready + slot, 2 * lap + 2);
      return true;
    }
    if (*pending == 0) return false;
    if (globaltimer_ns() - t0 > wait_ns) {
      latch_status(status, kStTimeout);
      return false;
    }
    __nanosleep(ns);
    ns = ns < 2048 ? ns * 2 : ns;
  }
}

// Exclusive scan of n (a multiple of the block size) counters in shared memory.
__device__ void block_excl_scan_smem(const uint32_t* in, uint32_t* out, uint32_t n) {
  __shared__ uint32_t wsum[kWarps];
  const uint32_t per = n / kBlock;
  const uint32_t b0 = threadIdx.x * per;
  uint32_t s = 0;
  for (uint32_t j = 0; j < per; ++j) s += in[b0 + j];
  uint32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane_id() >= (uint32_t)o) inc += t;
  }
  const uint32_t w = threadIdx.x >> 5;
  if (lane_id() == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane_id() < kWarps ? wsum[lane_id()] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane_id() >= (uint32_t)o) v += t;
    }
    if (lane_id() < kWarps) wsum[lane_id()] = v;
  }
  __syncthreads();
  uint32_t run = inc - s + (w ? wsum[w - 1] : 0);
  for (uint32_t j = 0; j < per; ++j) {
    const uint32_t v = in[b0 + j];
    out[b0 + j] = run;
    run += v;
  }
  __syncthreads();
}

// Inclusive max-scan of n (a multiple of the block size) values in shared memory.
__device__ void block_max_scan_smem(uint32_t* a, uint32_t n) {
  __shared__ uint32_t wmax[kWarps];
  const uint32_t per = n / kBlock;
  const uint32_t b0 = threadIdx.x * per;
  uint32_t m = 0;
  for (uint32_t j = 0; j < per; ++j) m = max(m, a[b0 + j]);
  uint32_t inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane_id() >= (uint32_t)o) inc = max(inc, t);
  }
  const uint32_t w = threadIdx.x >> 5;
  if (lane_id() == 31) wmax[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane_id() < kWarps ? wmax[lane_id()] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane_id() >= (uint32_t)o) v = max(v, t);
    }
    if (lane_id() < kWarps) wmax[lane_id()] = v;
  }
  __syncthreads();
  uint32_t run = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
  if (lane_id() == 0) run = 0;
  run = max(run, w ? wmax[w - 1] : 0u);
  for (uint32_t j = 0; j < per; ++j) {
    run = max(run, a[b0 + j]);
    a[b0 + j] = run;
  }
  __syncthreads();
}

// One S^5 step on task t by this block.
// Returns this thread's share of the step's algorithmic bytes: the sample,
// cache 8 read + bucket index 2 written per record while classifying, and the
// bytes of each record's move.
template <int LOGV>
__device__ unsigned long long queue_step(const SortCtx& c, const Task& t, QueueSmem<LOGV>& s, uint32_t R) {
  using Gm = Geo<LOGV>;
  const SetDesc sd = c.sets[task_set(t)];
  const uint32_t par = task_par(t);
  const Rec* recs = c.rec[par] + t.begin;
  const uint32_t wide = c.wide[task_set(t)];
  build_splitters<LOGV>(recs, t.len, mix64(c.seed ^ ((uint64_t)t.begin << 20) ^ t.depth), s.sp, s.u.bs, sd.dna);
  unsigned long long bytes = threadIdx.x == 0 ? Gm::S * 8ull : 0ull;

  // classification (Algorithm 4.1): classify into the array o and count; with
  // an LCP output also the smallest and largest key of each even bucket
  const bool with_lcp = sd.lcp != nullptr;
  for (uint32_t b = threadIdx.x; b < Gm::KP; b += kBlock) {
    s.hist[b] = 0;
    s.u.mm.bmin[b] = ~0ull;
    s.u.mm.bmax[b] = 0ull;
  }
  __syncthreads();
  uint16_t* bo = c.bucket_of + t.begin;
  bytes += 10ull * classify_count_k<LOGV, uint64_t>([&](uint32_t p) { return recs[p].key; }, bo, t.len, s.sp.tree,
                                                    s.sp.x, s.hist, c.classifier, nullptr,
                                                    with_lcp ? s.u.mm.bmin : nullptr,
                                                    with_lcp ? s.u.mm.bmax : nullptr);
  __syncthreads();

  // prefix sum over the bucket sizes; bucket outcomes
  block_excl_scan_smem(s.hist, s.bstart, Gm::KP);  // bstart[K] = len (hist[K] is 0)
  if (with_lcp) {
    // LCP at each bucket boundary (Section 4.2.3 "LCP via XOR", Section 4.2.8
    // "LCP Calculation"): the last string of the previous non-empty bucket
    // and the first string of this one are the largest key of the one and
    // the smallest of the other, which differ within the step's 8 characters
    for (uint32_t b = threadIdx.x; b < Gm::KP; b += kBlock) s.u.mm.prev[b] = (b < Gm::K && s.hist[b]) ? b + 1 : 0u;
    __syncthreads();
    block_max_scan_smem(s.u.mm.prev, Gm::KP);  // prev[b] - 1: last non-empty bucket <= b
    for (uint32_t b = threadIdx.x + 1; b < Gm::K; b += kBlock) {
      const uint32_t q = s.u.mm.prev[b - 1];
      if (!s.hist[b] || q == 0) continue;
      const uint32_t pb = q - 1;
      const uint64_t hi = (pb & 1u) ? s.sp.x[pb >> 1] : s.u.mm.bmax[pb];
      const uint64_t lo = (b & 1u) ? s.sp.x[b >> 1] : s.u.mm.bmin[b];
      sd.lcp[t.begin + s.bstart[b] - sd.base] = t.depth + key_lcp(hi, lo, sd.dna);
    }
    __syncthreads();  // hist is overwritten below
  }
  for (uint32_t b = threadIdx.x; b < Gm::K; b += kBlock) {
    const uint32_t size = s.hist[b];
    s.desc[b] = size ? bucket_desc<LOGV>(b, size, t.depth, s.sp, sd.dna) : kFin;
    s.hist[b] = t.begin + s.bstart[b];
  }
  __syncthreads();

  // redistribution: stable and out of place, tile by tile; a subset that fits
  // one tile is spread over all warps (each warp owns 32 * R consecutive
  // records of a tile)
  R = min(R, (t.len + kBlock - 1) / kBlock);
  const uint32_t T = kBlock * R;
  for (uint32_t t0 = 0; t0 < t.len; t0 += T) {
    const uint32_t tl = min(T, t.len - t0);
    for (uint32_t p = threadIdx.x; p < tl; p += kBlock) s.u.sc.tb[p] = bo[t0 + p];
    __syncthreads();
    const uint32_t src0 = t.begin + t0;
    tile_scatter<LOGV>(s.u.sc.tb, tl, R, s.hist, s.u.sc.cntw,
                       [&](const uint32_t(&pp)[kMoveBatch], const uint32_t(&bb)[kMoveBatch],
                           const uint32_t(&dd)[kMoveBatch]) {
                         bytes += move_batch(c, sd, wide, par, src0, t.depth, s.desc,
                                             [&](uint32_t b) { return t.begin + s.bstart[b]; }, pp, bb, dd);
                       });
  }
  __threadfence();
  __syncthreads();

  // new subsets become visible only after their records have been moved
  for (uint32_t b = threadIdx.x; b < Gm::K; b += kBlock) {
    const uint32_t start = s.bstart[b];
    const uint32_t size = s.bstart[b + 1] - start;
    if (size) emit_bucket(c, sd, t, start, size, s.desc[b], 0, 0u);  // boundary LCPs are written already
  }
  return bytes;
}

template <int LOGV>
__global__ void __launch_bounds__(kBlock, 3) k_queue(SortCtx c, uint32_t R) {
  extern __shared__ __align__(16) uint8_t smem[];
  QueueSmem<LOGV>& s = *reinterpret_cast<QueueSmem<LOGV>*>(smem);
  unsigned long long bytes = 0;
  while (true) {
    if (threadIdx.x == 0) s.got = claim_task(c.mq, &s.task, c.status, c.wait_ns) ? 1u : 0u;
    __syncthreads();
    if (!s.got) break;
    const Task t = s.task;
    bytes += queue_step<LOGV>(c, t, s, R);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicSub(c.mq.pending, 1u);
    }
  }
  account(c, kKQueue, bytes);
}

template <int LOGV>
cudaError_t set_queue_attr() {
  static cudaError_t e = cudaFuncSetAttribute(k_queue<LOGV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)sizeof(QueueSmem<LOGV>));
  return e;
}

}  // namespace

size_t queue_smem(int logv) {
  switch (logv) {
    case 7: return sizeof(QueueSmem<7>);
    case 8: return sizeof(QueueSmem<8>);
    case 9: return sizeof(QueueSmem<9>);
    default: return sizeof(QueueSmem<10>);
  }
}

cudaError_t queue_occupancy(int logv, int* blocks_per_sm) {
  switch (logv) {
    case 7:
      if (cudaError_t e = set_queue_attr<7>()) return e;
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_queue<7>, kBlock, sizeof(QueueSmem<7>));
    case 8:
      if (cudaError_t e = set_queue_attr<8>()) return e;
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_queue<8>, kBlock, sizeof(QueueSmem<8>));
    case 9:
      if (cudaError_t e = set_queue_attr<9>()) return e;
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_queue<9>, kBlock, sizeof(QueueSmem<9>));
    default:
      if (cudaError_t e = set_queue_attr<10>()) return e;
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_queue<10>, kBlock,
                                                           sizeof(QueueSmem<10>));
  }
}

cudaError_t launch_queue(int logv, const SortCtx& c, uint32_t grid, uint32_t R, cudaStream_t st,
                         const LaunchHook& hook) {
  switch (logv) {
    case 7:
      if (cudaError_t e = set_queue_attr<7>()) return e;
      hook.run("queue", [&] { k_queue<7><<<grid, kBlock, sizeof(QueueSmem<7>), st>>>(c, R); });
      break;
    case 8:
      if (cudaError_t e = set_queue_attr<8>()) return e;
      hook.run("queue", [&] { k_queue<8><<<grid, kBlock, sizeof(QueueSmem<8>), st>>>(c, R); });
      break;
    case 9:
      if (cudaError_t e = set_queue_attr<9>()) return e;
      hook.run("queue", [&] { k_queue<9><<<grid, kBlock, sizeof(QueueSmem<9>), st>>>(c, R); });
      break;
    default:
      if (cudaError_t e = set_queue_attr<10>()) return e;
      hook.run("queue", [&] { k_queue<10><<<grid, kBlock, sizeof(QueueSmem<10>), st>>>(c, R); });
      break;
  }
  return cudaGetLastError();
}

}  // namespace ss
