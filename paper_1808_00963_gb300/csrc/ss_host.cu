// Host orchestrator and C-ABI of ss_sort (declared in include/ss_sort.h).
//
// One sort (Section 4.2.8, adapted to one GPU):
//   1. every string gets a record (cache at depth 0, index) and each set a
//      root subset;
//   2. while some subset is larger than the big-task threshold, all such
//      subsets run one multi-block S^5 step together (the host reads how many
//      there are after each step, which is the only host synchronisation);
//   3. one persistent work-queue launch runs single-block S^5 steps until
//      every remaining subset is at most small_cutoff strings;
//   4. warps and blocks finish the small subsets;
//   5. the LCP entries at distribution-step boundaries are resolved.
// Batches skip step 2 (their launch sequence is fixed, so it can be captured
// into a CUDA graph).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ss_sort.h"
#include "ss_kernels.h"
#include "ss_step.cuh"
#include "ss_tuned.h"

namespace ss {

// ---- launch accounting and profiling -------------------------------------------------

static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_profiling{0};
static std::atomic<int> g_graph_loop{1};  // 0: the host runs the multi-block rounds (see ss_set_graph_loop)
static std::mutex g_stats_mu;
static std::map<std::string, std::pair<uint64_t, double>> g_stats;
static std::map<std::string, unsigned long long> g_bytes;
static const char* const kClassNames[kKClasses] = {"init",      "big_sample", "big_classify", "scan",
                                                   "big_emit",  "big_scatter", "queue",       "small_warp",
                                                   "small_cta", "lcp_fix"};

struct PendingEvent {
  const char* name;
  cudaEvent_t a, b;
  int dev;
};
static thread_local std::vector<PendingEvent> t_pending;
// Events are reused (creating two per launch costs more host time than the
// launch itself); an event belongs to the device it was created on.
static thread_local std::map<int, std::vector<cudaEvent_t>> t_event_pool;

static cudaEvent_t pooled_event(int dev) {
  auto& pool = t_event_pool[dev];
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static thread_local bool t_no_count = false;  // set while our own loop graphs are captured

void LaunchHook::run(const char* name, const std::function<void()>& launch) const {
  if (!t_no_count) g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!g_profiling.load() || cudaStreamIsCapturing(stream, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    launch();
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  PendingEvent p{name, pooled_event(dev), pooled_event(dev), dev};
  cudaEventRecord(p.a, stream);
  launch();
  cudaEventRecord(p.b, stream);
  t_pending.push_back(p);
}

// Accumulates the timings of this thread's finished launches.
static void collect_profile() {
  if (t_pending.empty()) return;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  for (auto& p : t_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& e = g_stats[p.name];
      e.first += 1;
      e.second += ms;
    }
    t_event_pool[p.dev].push_back(p.a);
    t_event_pool[p.dev].push_back(p.b);
  }
  t_pending.clear();
}

// ---- device information --------------------------------------------------------------

struct DevInfo {
  bool ok = false;
  int sms = 0;
  int queue_blocks[11] = {0};
};

static std::mutex g_dev_mu;
static std::map<int, DevInfo> g_dev;

static ss_status device_info(DevInfo& out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev.find(dev);
  if (it == g_dev.end()) {
    DevInfo d;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return SS_ERR_NO_DEVICE;
    d.ok = (p.major == 10 && p.minor == 3);
    d.sms = p.multiProcessorCount;
    if (d.ok) {
      for (int l = 7; l <= 10; ++l) {
        int b = 0;
        if (queue_occupancy(l, &b) != cudaSuccess || b < 1) return SS_ERR_CUDA;
        d.queue_blocks[l] = b;
      }
      // keep freed stream-ordered allocations in the pool between calls
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
    }
    it = g_dev.emplace(dev, d).first;
  }
  if (!it->second.ok) return SS_ERR_NO_DEVICE;
  out = it->second;
  return SS_OK;
}

// ---- options and workspace layout -----------------------------------------------------

// Defaults come from the autotuner's table (ss_tuned.h).
// Bound on every device-side wait of a sort (queue slots, flags).
constexpr uint64_t kDefaultWaitNs = 30ull * 1000 * 1000 * 1000;

struct Opts {
  uint32_t cap = kNoCap;
  int logv = SS_TUNED_SPLITTERS_LOG2;           // single-block steps
  int logv_big = SS_TUNED_BIG_SPLITTERS_LOG2;   // multi-block steps
  uint32_t R = SS_TUNED_TILE_ROUNDS;            // 0 = choose per step
  uint32_t cutoff = SS_TUNED_SMALL_CUTOFF;
  uint32_t big_thr = SS_TUNED_BIG_THRESHOLD;
  uint32_t seed = 0x5EED;
  uint32_t classifier = 0;
  uint32_t host_parts = 0;  // ss_sort_host: 0 = automatic
  uint64_t wait_ns = kDefaultWaitNs;
};

constexpr uint32_t kMaxHostParts = 16;

static ss_status resolve_opts(const ss_options* o, Opts& r) {
  r = Opts();
  if (!o) return SS_OK;
  if (o->host_parts > kMaxHostParts || (o->host_parts & (o->host_parts - 1))) return SS_ERR_INVALID;
  r.host_parts = o->host_parts;
  if (o->max_len) r.cap = o->max_len;
  if (o->splitters_log2) {
    if (o->splitters_log2 < 7 || o->splitters_log2 > 10) return SS_ERR_INVALID;
    r.logv = (int)o->splitters_log2;
  }
  if (o->big_splitters_log2) {  // wide keys: 2^10 splitters would not fit a block's static shared memory
    if (o->big_splitters_log2 < 8 || o->big_splitters_log2 > 9) return SS_ERR_INVALID;
    r.logv_big = (int)o->big_splitters_log2;
  }
  if (o->tile_rounds) {
    if (o->tile_rounds < 8 || o->tile_rounds > kMaxRounds) return SS_ERR_INVALID;
    r.R = o->tile_rounds;
  }
  if (o->small_cutoff) {
    if (o->small_cutoff < 64 || o->small_cutoff > 4096) return SS_ERR_INVALID;
    r.cutoff = o->small_cutoff;
  }
  if (o->big_threshold) r.big_thr = o->big_threshold;
  if (r.big_thr < r.cutoff) return SS_ERR_INVALID;
  if (o->seed) r.seed = o->seed;
  if (o->classifier > 3) return SS_ERR_INVALID;
  r.classifier = o->classifier;
  if (o->workspace && ((uintptr_t)o->workspace & 255)) return SS_ERR_INVALID;
  if (o->wait_limit_us) r.wait_ns = (uint64_t)o->wait_limit_us * 1000;
  return SS_OK;
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static uint32_t pmax_of(uint32_t cutoff) {
  uint32_t p = 64;
  while (p < cutoff) p <<= 1;
  return p;
}

constexpr uint32_t kCtrlWords = 64;                          // status and list counters
constexpr size_t kCtrlBytes = kCtrlWords * 4 + kKClasses * 8;  // + algorithmic byte counters
enum Ctrl : uint32_t { kCStatus = 0, kCBig0 = 1, kCBig1 = 2, kCHead = 3, kCTail = 4, kCPending = 5,
                       kCSmallW = 6, kCSmallC = 7, kCSmallD = 8, kCMarks = 9, kCSmallCW = 10,
                       kCClaim = 11 /* and 12 */ };

struct Layout {
  size_t ctrl, sets, wide, rec0, rec1, wid0, wid1, bucket_of, big0, big1, gen, spl, counters, partials, gstart,
      gdesc, bigctl, marks, mq_items, mq_ready, sw_items, sc_items, scw_items, total;
  uint32_t cap_big, cap_mq, cap_sw, cap_sc, cap_scw;
  uint64_t ncounters_max;
};

static Layout make_layout(uint64_t M, uint32_t num_sets, const Opts& o, bool big) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
  L.cap_big = big ? (uint32_t)(M / ((uint64_t)o.big_thr + 1) + 2) : 0;
  // the work queue's ring: more slots than disjoint subsets of > cutoff
  // records can exist, so it never overflows (see WorkQueue)
  L.cap_mq = (uint32_t)std::max<uint64_t>(4096, M / ((uint64_t)o.cutoff + 1) + 1024);
  // warp tasks: subsets and runs the block sort passes on, disjoint and of at
  // least 2 strings (<= M/2), then as many deferred runs (<= M/2)
  L.cap_sw = (uint32_t)(M / 2 + 1);
  L.cap_sc = (uint32_t)(M / 33 + 2);
  L.cap_scw = (uint32_t)(M / (kSmallCtaNarrowMax + 1) + 2);
  const uint64_t KP = 2ull << o.logv_big;
  const uint64_t tiles_max = big ? M / (kBlock * 8) + L.cap_big : 0;
  L.ncounters_max = big ? KP * (tiles_max + L.cap_big) : 0;
  L.ctrl = take(kCtrlBytes);
  L.sets = take((size_t)num_sets * sizeof(SetDesc));
  L.wide = take((size_t)num_sets * 4);
  L.rec0 = take(M * sizeof(Rec));
  L.rec1 = take(M * sizeof(Rec));
  L.wid0 = take(big ? M * sizeof(uint2) : 0);  // (idx, off) of the wide records of multi-block subsets
  L.wid1 = take(big ? M * sizeof(uint2) : 0);
  L.bucket_of = take(M * 2);
  L.big0 = take((size_t)L.cap_big * sizeof(Task));
  L.big1 = take((size_t)L.cap_big * sizeof(Task));
  L.gen = take((size_t)L.cap_big * sizeof(GenTask));
  L.spl = take((size_t)L.cap_big * big_splitters_bytes(o.logv_big));
  L.counters = take(L.ncounters_max * 4);
  L.partials = take((L.ncounters_max / 4096 + 2) * 4);
  L.gstart = take((size_t)L.cap_big * KP * 4);
  L.gdesc = take((size_t)L.cap_big * KP * 4);
  L.bigctl = take(big ? sizeof(BigCtl) : 0);  // a batch's loop control block (plain sorts use the stream's)
  L.marks = take(big ? M * 4 : 0);             // LCP marks of multi-block steps (distinct positions: < M)
  L.mq_items = take((size_t)L.cap_mq * sizeof(Task));
  L.mq_ready = take((size_t)L.cap_mq * 4);
  L.sw_items = take(2 * (size_t)L.cap_sw * sizeof(Task));
  L.sc_items = take((size_t)L.cap_sc * sizeof(Task));
  L.scw_items = take((size_t)L.cap_scw * sizeof(Task));
  L.total = off;
  return L;
}

static SortCtx make_ctx(uint8_t* ws, const Layout& L, uint32_t num_sets, uint32_t total, const Opts& o, bool big) {
  SortCtx c{};
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(ws + L.ctrl);
  c.sets = reinterpret_cast<const SetDesc*>(ws + L.sets);
  c.num_sets = num_sets;
  c.total = total;
  c.wide = reinterpret_cast<uint32_t*>(ws + L.wide);
  c.rec[0] = reinterpret_cast<Rec*>(ws + L.rec0);
  c.rec[1] = reinterpret_cast<Rec*>(ws + L.rec1);
  c.wid[0] = reinterpret_cast<uint2*>(ws + L.wid0);
  c.wid[1] = reinterpret_cast<uint2*>(ws + L.wid1);
  c.bucket_of = reinterpret_cast<uint16_t*>(ws + L.bucket_of);
  c.status = ctrl + kCStatus;
  c.abytes = reinterpret_cast<unsigned long long*>(ctrl + kCtrlWords);
  c.big[0] = TaskList{reinterpret_cast<Task*>(ws + L.big0), ctrl + kCBig0, L.cap_big};
  c.big[1] = TaskList{reinterpret_cast<Task*>(ws + L.big1), ctrl + kCBig1, L.cap_big};
  c.mq = WorkQueue{reinterpret_cast<Task*>(ws + L.mq_items), reinterpret_cast<uint32_t*>(ws + L.mq_ready),
                   ctrl + kCHead, ctrl + kCTail, ctrl + kCPending, L.cap_mq};
  c.small_warp = TaskList{reinterpret_cast<Task*>(ws + L.sw_items), ctrl + kCSmallW, L.cap_sw};
  c.small_deep = TaskList{reinterpret_cast<Task*>(ws + L.sw_items) + L.cap_sw, ctrl + kCSmallD, L.cap_sw};
  c.small_cta = TaskList{reinterpret_cast<Task*>(ws + L.sc_items), ctrl + kCSmallC, L.cap_sc};
  c.small_cta_wide = TaskList{reinterpret_cast<Task*>(ws + L.scw_items), ctrl + kCSmallCW, L.cap_scw};
  c.small_claim = ctrl + kCClaim;
  c.marks = reinterpret_cast<uint32_t*>(ws + L.marks);
  c.marks_count = ctrl + kCMarks;
  c.marks_cap = big ? total : 0u;
  c.small_cutoff = o.cutoff;
  c.big_threshold = o.big_thr;
  c.big_enabled = big ? 1u : 0u;
  c.seed = o.seed;
  c.classifier = o.classifier;
  c.big_cur = 0;
  c.wait_ns = o.wait_ns;
  return c;
}

static ss_status map_status(uint32_t st) {
  if (st & kStTooDeep) return SS_ERR_TOO_LARGE;
  if (st & kStQueueFull) return SS_ERR_QUEUE_FULL;
  if (st & kStTimeout) return SS_ERR_TIMEOUT;
  return SS_OK;
}

#define SS_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      if (e_ == cudaErrorMemoryAllocation) return SS_ERR_OOM; \
      return SS_ERR_CUDA;                                 \
    }                                                     \
  } while (0)

// Pinned host staging, one per thread, grown as needed.
struct Pinned {
  void* p = nullptr;
  size_t n = 0;
  ~Pinned() { if (p) cudaFreeHost(p); }
  ss_status reserve(size_t bytes) {
    if (bytes <= n) return SS_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) return SS_ERR_OOM;
    n = bytes;
    return SS_OK;
  }
};
static thread_local Pinned t_down, t_up;

// Small uploads and zero fills of the sort: on the copy engines, except while
// a large copy on another stream holds them (the overlapped host path), when
// a kernel that reads the pinned staging memory does them instead.  (A kernel
// reading host memory costs 6-55 us per launch on the GB300 machine, more than
// the copy engine when it is free.)
static thread_local bool t_kernel_copies = false;

static cudaError_t zero_fill(void* dst, size_t bytes, cudaStream_t st, const LaunchHook& hook) {
  if (t_kernel_copies) return launch_upload(nullptr, dst, bytes, st, hook);
  return cudaMemsetAsync(dst, 0, bytes, st);
}

// Writes a set descriptor into the workspace: a kernel parameter, so the host
// neither stages it nor waits for a copy before enqueuing the sort.
__global__ void k_set_desc(SetDesc* dst, SetDesc v) { *dst = v; }

// Writes the control block of the multi-block loop (same reason).
__global__ void k_set_ctl(BigCtl* dst, BigCtl v) { *dst = v; }

// A batch's set descriptors, up to kDescChunk per launch (kernel parameters).
constexpr uint32_t kDescChunk = 128;
struct SetDescChunk {
  SetDesc d[kDescChunk];
};
__global__ void k_set_descs(SetDesc* dst, uint32_t count, SetDescChunk v) {
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) dst[i] = v.d[i];
}

// ---- the multi-block loop as a CUDA graph -------------------------------------------------
//
// One round of multi-block steps is a plan kernel plus the round's kernels, all
// reading the control block in device memory.  The rounds run in a graph with
// a conditional WHILE node: the plan before the loop and the plan at the end
// of each round set the condition to 1 while big subsets remain, so the host
// enqueues the whole loop with one graph launch and never waits for it.  The
// graph depends only on the control block's address and the step geometry;
// it is built once per stream (whose control block every sort and batch run
// on that stream uses) and reused.  A run inside a caller's stream capture
// adds the same loop, over the batch's own control block, to the caller's
// graph instead.

struct LoopKey {
  int dev;
  const void* ctl;
  int logv;
  uint32_t R_max;
  bool operator<(const LoopKey& o) const {
    return std::tie(dev, ctl, logv, R_max) < std::tie(o.dev, o.ctl, o.logv, o.R_max);
  }
};
struct LoopGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
};
static std::mutex g_loop_mu;
static std::map<LoopKey, LoopGraph> g_loops;

// Streams of this thread (per device) that the loop is captured on when a
// graph is built.
struct CaptureStreams {
  cudaStream_t main = nullptr, body = nullptr;
};
static thread_local std::map<int, CaptureStreams> t_capture;

static cudaError_t capture_streams(CaptureStreams*& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  CaptureStreams& c = t_capture[dev];
  if (!c.main && (e = cudaStreamCreateWithFlags(&c.main, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if (!c.body && (e = cudaStreamCreateWithFlags(&c.body, cudaStreamNonBlocking)) != cudaSuccess) return e;
  out = &c;
  return cudaSuccess;
}

// Adds the loop to the graph being captured on `st`: the first plan, then a
// WHILE node whose body is one round and the next plan.  Work captured on st
// afterwards depends on the loop.
static cudaError_t add_loop(cudaStream_t st, BigCtl* ctl, int logv, uint32_t R_max, uint32_t sms) {
  CaptureStreams* cs = nullptr;
  cudaError_t e = capture_streams(cs);
  if (e != cudaSuccess) return e;
  const LaunchHook hook{st};
  cudaStreamCaptureStatus status;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if ((e = cudaStreamGetCaptureInfo(st, &status, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess) return e;
  if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
  if ((e = launch_big_plan(ctl, (uint64_t)h, true, st, hook)) != cudaSuccess) return e;
  if ((e = cudaStreamGetCaptureInfo(st, &status, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &p)) != cudaSuccess) return e;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(cs->body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
      cudaSuccess)
    return e;
  const LaunchHook bhook{cs->body};
  cudaError_t e1 = launch_big_round(logv, ctl, R_max, sms, cs->body, bhook);
  cudaError_t e2 = launch_big_plan(ctl, (uint64_t)h, true, cs->body, bhook);
  cudaGraph_t done = nullptr;
  e = cudaStreamEndCapture(cs->body, &done);
  if (e1 != cudaSuccess) return e1;
  if (e2 != cudaSuccess) return e2;
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The instantiated loop graph for a control block (built on first use).
static cudaError_t loop_exec(BigCtl* ctl, int logv, uint32_t R_max, uint32_t sms, cudaGraphExec_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_loop_mu);
  LoopGraph& lg = g_loops[LoopKey{dev, ctl, logv, R_max}];
  if (!lg.exec) {
    CaptureStreams* cs = nullptr;
    if ((e = capture_streams(cs)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(cs->main, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    t_no_count = true;  // these kernels run once per graph launch; the plan kernels count them
    cudaError_t e1 = add_loop(cs->main, ctl, logv, R_max, sms);
    t_no_count = false;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs->main, &g);
    if (e1 != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return e1 != cudaSuccess ? e1 : e;
    }
    if ((e = cudaGraphInstantiate(&lg.exec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      lg.exec = nullptr;
      return e;
    }
    lg.g = g;
  }
  *out = lg.exec;
  return cudaSuccess;
}

// ---- per-stream state of asynchronous sorts ---------------------------------------------

// Device memory of one (device, stream): the status word the stream's sorts
// fold their device status into, and the multi-block loop's control block.
struct StreamSlot {
  uint32_t status;
  uint32_t pad[63];
  BigCtl ctl;
};

static std::mutex g_slot_mu;
static std::map<std::pair<int, void*>, StreamSlot*> g_slots;

static ss_status stream_slot(cudaStream_t st, bool create, StreamSlot** out) {
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  auto key = std::make_pair(dev, static_cast<void*>(st));
  auto it = g_slots.find(key);
  if (it != g_slots.end()) {
    *out = it->second;
    return SS_OK;
  }
  if (!create) return SS_OK;
  StreamSlot* p = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&p), sizeof(StreamSlot)) != cudaSuccess) return SS_ERR_OOM;
  if (cudaMemsetAsync(p, 0, sizeof(StreamSlot), st) != cudaSuccess) {  // ordered before the stream's first use
    cudaFree(p);
    return SS_ERR_CUDA;
  }
  g_slots[key] = p;
  *out = p;
  return SS_OK;
}

// Enqueues everything after the set descriptors are in place.  ctl: where the
// multi-block loop's control block lives (needed when big).
static ss_status run_sort(uint8_t* ws, const Layout& L, SortCtx c, const Opts& o, const DevInfo& dev,
                          bool big, cudaStream_t st, BigCtl* ctl = nullptr) {
  const LaunchHook hook{st};
  SS_CUDA(zero_fill(ws + L.ctrl, kCtrlBytes, st, hook));
  SS_CUDA(zero_fill(ws + L.mq_ready, (size_t)L.cap_mq * 4, st, hook));
  SS_CUDA(zero_fill(ws + L.wide, (size_t)c.num_sets * 4, st, hook));
  SS_CUDA(launch_init(c, st, hook));
  if (big) {
    if (!ctl) return SS_ERR_INVALID;
    BigCtl v{};
    v.c = c;
    v.gt = reinterpret_cast<GenTask*>(ws + L.gen);
    v.splitters = ws + L.spl;
    v.counters = reinterpret_cast<uint32_t*>(ws + L.counters);
    v.partials = reinterpret_cast<uint32_t*>(ws + L.partials);
    v.gstart = reinterpret_cast<uint32_t*>(ws + L.gstart);
    v.gdesc = reinterpret_cast<uint32_t*>(ws + L.gdesc);
    v.ncounters_max = L.ncounters_max;
    v.cap_big = L.cap_big;
    v.R_fixed = o.R;
    v.sms = (uint32_t)dev.sms;
    v.K = (2u << o.logv_big) - 1;
    v.cur = 0;
    v.round = 0;
    hook.run("init", [&] { k_set_ctl<<<1, 1, 0, st>>>(ctl, v); });
    SS_CUDA(cudaGetLastError());
    const uint32_t R_max = o.R ? o.R : kMaxRounds;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SS_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusActive) {
      // the caller is capturing a graph: the loop becomes part of it
      SS_CUDA(add_loop(st, ctl, o.logv_big, R_max, (uint32_t)dev.sms));
    } else if (g_profiling.load() || !g_graph_loop.load()) {
      // launch by launch (timed, or for a profiler): the host runs the rounds, reading each plan
      if (t_down.reserve(64) != SS_OK) return SS_ERR_OOM;
      uint32_t* hG = static_cast<uint32_t*>(t_down.p);
      while (true) {
        SS_CUDA(launch_big_plan(ctl, 0, false, st, hook));
        SS_CUDA(cudaMemcpyAsync(hG, &ctl->G, 4, cudaMemcpyDeviceToHost, st));
        SS_CUDA(cudaStreamSynchronize(st));
        collect_profile();
        if (*hG == 0) break;
        SS_CUDA(launch_big_round(o.logv_big, ctl, R_max, (uint32_t)dev.sms, st, hook));
      }
    } else {
      cudaGraphExec_t exec = nullptr;
      SS_CUDA(loop_exec(ctl, o.logv_big, R_max, (uint32_t)dev.sms, &exec));
      SS_CUDA(cudaGraphLaunch(exec, st));
    }
  }
  const uint32_t qgrid = (uint32_t)(dev.sms * dev.queue_blocks[o.logv]);
  SS_CUDA(launch_queue(o.logv, c, qgrid, kMaxRounds, st, hook));
  SS_CUDA(launch_small(c, pmax_of(o.cutoff), (uint32_t)dev.sms * 8, (uint32_t)dev.sms * 4, st, hook));
  const uint32_t fgrid = std::max(1u, std::min<uint32_t>((c.total + kBlock - 1) / kBlock, (uint32_t)dev.sms * 16));
  SS_CUDA(launch_lcp_fix(c, fgrid, st, hook));
  return SS_OK;
}

static ss_status read_status(uint8_t* ws, const Layout& L, cudaStream_t st) {
  if (t_down.reserve(kCtrlBytes) != SS_OK) return SS_ERR_OOM;
  uint32_t* h = static_cast<uint32_t*>(t_down.p);
  SS_CUDA(cudaMemcpyAsync(h, ws + L.ctrl, kCtrlBytes, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  collect_profile();
  if (g_profiling.load()) {
    const unsigned long long* ab = reinterpret_cast<const unsigned long long*>(h + kCtrlWords);
    std::lock_guard<std::mutex> lk(g_stats_mu);
    for (uint32_t k = 0; k < kKClasses; ++k)
      if (ab[k]) g_bytes[kClassNames[k]] += ab[k];
  }
  return map_status(h[kCStatus]);
}

static ss_status sort_device(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t* perm,
                             uint32_t* lcp, const ss_options* opt, cudaStream_t st, uint32_t dna = 0) {
  Opts o;
  ss_status s = resolve_opts(opt, o);
  if (s != SS_OK) return s;
  if (n >= 0xFFFFFFFFull) return SS_ERR_TOO_LARGE;
  if (n == 0) return SS_OK;
  if (!chars || !offsets || !perm) return SS_ERR_INVALID;
  DevInfo dev;
  if ((s = device_info(dev)) != SS_OK) return s;
  const bool big = n > o.big_thr;
  const Layout L = make_layout(n, 1, o, big);
  uint8_t* ws = nullptr;
  bool owned = false;
  if (opt && opt->workspace) {
    if (opt->workspace_bytes < L.total) return SS_ERR_INVALID;
    ws = static_cast<uint8_t*>(opt->workspace);
  } else {
    if (cudaMallocAsync(reinterpret_cast<void**>(&ws), L.total, st) != cudaSuccess) return SS_ERR_OOM;
    owned = true;
  }
  StreamSlot* slot = nullptr;
  if ((s = stream_slot(st, true, &slot)) != SS_OK) {
    if (owned) cudaFreeAsync(ws, st);
    return s;
  }
  SetDesc sd{chars, offsets, perm, lcp, (uint32_t)n, o.cap, 0, dna};
  ss_status r = SS_OK;
  LaunchHook{st}.run("init", [&] { k_set_desc<<<1, 1, 0, st>>>(reinterpret_cast<SetDesc*>(ws + L.sets), sd); });
  if (cudaGetLastError() != cudaSuccess) r = SS_ERR_CUDA;
  SortCtx ctx = make_ctx(ws, L, 1, (uint32_t)n, o, big);
  ctx.dna = dna;
  ctx.fold_status = &slot->status;  // the device status goes to the stream's status word
  if (r == SS_OK) r = run_sort(ws, L, ctx, o, dev, big, st, &slot->ctl);
  if (g_profiling.load()) read_status(ws, L, st);  // waits: per-kernel times and bytes
  if (owned) cudaFreeAsync(ws, st);
  return r;
}

// Waits for the stream and returns the device status its sorts have left in
// its status word since it was last read (clearing it).
static ss_status take_stream_status(cudaStream_t st) {
  StreamSlot* slot = nullptr;
  stream_slot(st, false, &slot);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SS_ERR_CUDA;
  collect_profile();
  if (!slot) return SS_OK;
  if (t_down.reserve(64) != SS_OK) return SS_ERR_OOM;
  uint32_t* h = static_cast<uint32_t*>(t_down.p);
  SS_CUDA(cudaMemcpyAsync(h, &slot->status, 4, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  const uint32_t v = *h;
  if (v) {
    SS_CUDA(cudaMemsetAsync(&slot->status, 0, 4, st));
    SS_CUDA(cudaStreamSynchronize(st));
  }
  return map_status(v);
}

}  // namespace ss

// ---- batches ------------------------------------------------------------------------------

struct ss_batch {
  ss::Opts o;
  ss::Layout L;
  ss::DevInfo dev;
  uint8_t* ws = nullptr;
  bool owned = false;
  bool big = false;  // some set is larger than the multi-block threshold
  uint32_t num_sets = 0;
  uint32_t total = 0;
  std::vector<ss::SetDesc> sd;  // the set descriptors, written into the workspace by each run
};

using namespace ss;

// Last asynchronous run enqueued on each stream (for ss_stream_status).
static std::mutex g_stream_mu;
static std::map<void*, ss_batch*> g_stream_last;

extern "C" {

const char* ss_status_string(ss_status s) {
  switch (s) {
    case SS_OK: return "ok";
    case SS_ERR_INVALID: return "invalid argument";
    case SS_ERR_OOM: return "out of memory";
    case SS_ERR_CUDA: return "CUDA runtime error";
    case SS_ERR_TOO_LARGE: return "input too large (n >= 2^32 or a string of 2^30 bytes or more)";
    case SS_ERR_TIMEOUT: return "a bounded device-side wait expired";
    case SS_ERR_QUEUE_FULL: return "a device task list overflowed";
    case SS_ERR_NO_DEVICE: return "no sm_103 CUDA device";
  }
  return "unknown status";
}

uint64_t ss_launch_count(void) {
  // host launches, plus the kernels the loop graphs launched (counted on the
  // device by their plan kernels; reading that count waits for the device)
  uint64_t graph = 0;
  int dev = 0;
  {
    std::lock_guard<std::mutex> lk(g_loop_mu);
    if (!g_loops.empty() && cudaGetDevice(&dev) == cudaSuccess) graph = graph_launch_count();
  }
  return g_launches.load() + graph;
}

void ss_set_profiling(int enabled) { g_profiling.store(enabled ? 1 : 0); }

void ss_set_graph_loop(int enabled) { g_graph_loop.store(enabled ? 1 : 0); }

void ss_reset_kernel_stats(void) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  g_stats.clear();
  g_bytes.clear();
}

uint32_t ss_kernel_stats(const char** names, uint64_t* launches, double* total_ms, uint64_t* alg_bytes,
                         uint32_t cap) {
  collect_profile();  // launches of asynchronous calls (merge, distinguishing) made by this thread
  std::lock_guard<std::mutex> lk(g_stats_mu);
  uint32_t i = 0;
  for (auto& kv : g_stats) {
    if (i < cap) {
      if (names) names[i] = kv.first.c_str();
      if (launches) launches[i] = kv.second.first;
      if (total_ms) total_ms[i] = kv.second.second;
      if (alg_bytes) {
        auto it = g_bytes.find(kv.first);
        alg_bytes[i] = it == g_bytes.end() ? 0 : it->second;
      }
    }
    ++i;
  }
  return i;
}

ss_status ss_distinguishing(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t max_len,
                            const uint32_t* perm, const uint32_t* lcp, uint8_t* out_char, uint32_t* out_dprefix,
                            uint64_t* out_D, void* stream) {
  if (n >= 0xFFFFFFFFull) return SS_ERR_TOO_LARGE;
  if (n == 0) return SS_OK;
  if (!perm || !lcp || (out_char && (!chars || !offsets))) return SS_ERR_INVALID;
  DevInfo dev;
  ss_status s = device_info(dev);
  if (s != SS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t grid = std::max(1u, std::min<uint32_t>((uint32_t)((n + kBlock - 1) / kBlock), (uint32_t)dev.sms * 16));
  const LaunchHook hook{st};
  if (launch_distinguishing(chars, offsets, (uint32_t)n, max_len ? max_len : kNoCap, perm, lcp, out_char,
                            out_dprefix, reinterpret_cast<unsigned long long*>(out_D), grid, st, hook) != cudaSuccess)
    return SS_ERR_CUDA;
  return SS_OK;
}

// ---- K-way LCP merge ------------------------------------------------------------------

static uint32_t merge_step(uint32_t sample_step) { return sample_step ? sample_step : 64; }

static ss_status merge_geometry(const ss_run* runs, uint32_t num_runs, uint32_t sample_step, uint64_t* total,
                                uint32_t* S) {
  if (num_runs == 0 || num_runs > SS_MERGE_MAX_RUNS || !runs) return SS_ERR_INVALID;
  if (sample_step != 0 && (sample_step < 16 || sample_step > 65536)) return SS_ERR_INVALID;
  uint64_t t = 0;
  for (uint32_t k = 0; k < num_runs; ++k) {
    if (runs[k].reserved != 0) return SS_ERR_INVALID;
    if (runs[k].n > 0 && (!runs[k].perm || !runs[k].lcp)) return SS_ERR_INVALID;
    t += runs[k].n;
  }
  if (t >= 0xFFFFFFFFull) return SS_ERR_TOO_LARGE;
  *total = t;
  *S = merge_step(sample_step);
  return SS_OK;
}

// two record buffers (32 bytes per string), the sample cuts of a round, the
// piece counter
static size_t merge_ws_bytes(uint64_t total, uint32_t num_runs, uint32_t S) {
  if (num_runs <= 1) return 256;
  return 2 * align256(total * sizeof(MergeRec)) + align256((total / S + num_runs + 1) * 4) + 256;
}

size_t ss_merge_workspace_size(const ss_run* runs, uint32_t num_runs, uint32_t sample_step) {
  uint64_t total;
  uint32_t S;
  if (merge_geometry(runs, num_runs, sample_step, &total, &S) != SS_OK) return 0;
  return merge_ws_bytes(total, num_runs, S);
}

ss_status ss_merge(const uint8_t* chars, const uint64_t* offsets, uint32_t max_len, const ss_run* runs,
                   uint32_t num_runs, uint32_t sample_step, uint32_t* out_perm, uint32_t* out_lcp,
                   void* workspace, size_t workspace_bytes, void* stream) {
  uint64_t total;
  uint32_t S;
  ss_status s = merge_geometry(runs, num_runs, sample_step, &total, &S);
  if (s != SS_OK) return s;
  if (total == 0) return SS_OK;
  if (!chars || !offsets || !out_perm) return SS_ERR_INVALID;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return SS_ERR_INVALID;
  const size_t need = merge_ws_bytes(total, num_runs, S);
  if (workspace && workspace_bytes < need) return SS_ERR_INVALID;
  DevInfo dev;
  s = device_info(dev);
  if (s != SS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const LaunchHook hook{st};
  const uint32_t sms = (uint32_t)dev.sms;
  const uint32_t K = num_runs;
  std::vector<uint32_t> start(K + 1, 0);
  for (uint32_t k = 0; k < K; ++k) start[k + 1] = start[k] + runs[k].n;
  if (K == 1) {
    return launch_merge_copy(runs[0].perm, runs[0].lcp, (uint32_t)total, out_perm, out_lcp, sms, st, hook) ==
                   cudaSuccess
               ? SS_OK
               : SS_ERR_CUDA;
  }
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const bool own = !ws;
  if (own && cudaMallocAsync(reinterpret_cast<void**>(&ws), need, st) != cudaSuccess) return SS_ERR_OOM;
  const size_t recb = align256(total * sizeof(MergeRec));
  MergeRec* rec[2] = {reinterpret_cast<MergeRec*>(ws), reinterpret_cast<MergeRec*>(ws + recb)};
  uint32_t* cut = reinterpret_cast<uint32_t*>(ws + 2 * recb);
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws + 2 * recb + align256((total / S + K + 1) * 4));
  const uint32_t cap = max_len ? std::min<uint32_t>(max_len, 1u << 30) : (1u << 30);
  MergePrepArgs pa{};
  pa.chars = chars;
  pa.offsets = offsets;
  pa.cap = cap;
  pa.K = K;
  pa.total = (uint32_t)total;
  pa.dst = rec[0];
  for (uint32_t k = 0; k <= K; ++k) pa.start[k] = start[k];
  for (uint32_t k = 0; k < K; ++k) {
    pa.perm[k] = runs[k].perm;
    pa.lcp[k] = runs[k].lcp;
  }
  bool ok = launch_merge_prep(pa, sms, st, hook) == cudaSuccess;
  uint32_t rounds = 0;
  while ((1u << rounds) < K) ++rounds;
  int cur = 0;
  for (uint32_t r = 0; ok && r < rounds; ++r) {
    const uint32_t w = 1u << r;
    MergeRoundArgs ra{};
    ra.chars = chars;
    ra.offsets = offsets;
    ra.cap = cap;
    ra.ncur = (K + w - 1) / w;
    ra.S = S;
    ra.src = rec[cur];
    ra.dst = r + 1 == rounds ? nullptr : rec[cur ^ 1];
    ra.cut = cut;
    ra.out_perm = out_perm;
    ra.out_lcp = out_lcp;
    ra.counter = counter;
    uint32_t ns = 0;
    for (uint32_t c = 0; c <= ra.ncur; ++c) {
      ra.start[c] = start[std::min(c * w, K)];
      ra.sbase[c] = ns;
      if (c < ra.ncur) ns += (start[std::min((c + 1) * w, K)] - start[c * w]) / S;
    }
    ra.nsamples = ns;
    ok = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st) == cudaSuccess &&
         launch_merge_round(ra, sms, st, hook) == cudaSuccess;
    cur ^= 1;
  }
  if (own && cudaFreeAsync(ws, st) != cudaSuccess) ok = false;
  return ok ? SS_OK : SS_ERR_CUDA;
}

// ---- suffix array by prefix doubling --------------------------------------------------

// The suffix array's own sorts (the capped sort of all suffixes and the rounds'
// pair sorts) hand subsets of up to 128 strings to the block sorts and keep
// subsets of up to 32768 on single-block steps: the subsets of a text's
// suffixes after the first characters are many and small, and on a GB300 these
// two settings took the 4M-character DNA-like text from 2.44 to 2.16 ms
// (1024 / 8192, the plain sort's defaults; 256 / 32768 gave 2.18 ms).
constexpr uint32_t kSaSmallCutoff = 128;
constexpr uint32_t kSaBigThreshold = 32768;

ss_status ss_suffix_array(const uint8_t* text, uint64_t n, uint32_t* out_sa, uint32_t* out_lcp,
                          uint32_t initial_depth, void* stream) {
  if (n >= 0xFFFFFFFEull) return SS_ERR_TOO_LARGE;
  if (n == 0) return SS_OK;
  if (!text || !out_sa) return SS_ERR_INVALID;
  if (initial_depth > (1u << 20)) return SS_ERR_INVALID;
  const uint32_t h0 = initial_depth ? initial_depth : 256;
  DevInfo dev;
  ss_status s = device_info(dev);
  if (s != SS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // workspace: offsets, capped LCPs (unless out_lcp holds them), names, group
  // starts, flags, two compacted position lists, scan totals, and per round
  // the members, their encoded name pairs, offsets and sorted order / LCPs
  const size_t a4 = align256(n * 4), a8 = align256(n * 8);
  const size_t tot_b = align256(sa_scan_totals(n) * 4);
  const size_t need = a8 + (out_lcp ? 0 : a4) + 7 * a4 + tot_b + align256(n * 11 + 16) + a8;
  uint8_t* ws = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&ws), need, st) != cudaSuccess) return SS_ERR_OOM;
  uint8_t* p = ws;
  auto take = [&](size_t b) { uint8_t* q = p; p += b; return q; };
  uint64_t* off = reinterpret_cast<uint64_t*>(take(a8));
  uint32_t* lcp0 = out_lcp ? out_lcp : reinterpret_cast<uint32_t*>(take(a4));
  uint32_t* isa = reinterpret_cast<uint32_t*>(take(a4));
  uint32_t* gs = reinterpret_cast<uint32_t*>(take(a4));
  uint32_t* flag = reinterpret_cast<uint32_t*>(take(a4));
  uint32_t* cpos[2] = {reinterpret_cast<uint32_t*>(take(a4)), reinterpret_cast<uint32_t*>(take(a4))};
  uint32_t* member = reinterpret_cast<uint32_t*>(take(a4));
  uint32_t* perm2 = reinterpret_cast<uint32_t*>(take(a4));
  uint32_t* tot = reinterpret_cast<uint32_t*>(take(tot_b));
  uint8_t* enc = take(align256(n * 11 + 16));
  uint64_t* eoff = reinterpret_cast<uint64_t*>(take(a8));
  uint32_t* lcp2 = reinterpret_cast<uint32_t*>(off);  // the offsets of round 0 are dead by then
  const LaunchHook hook{st};
  auto grid_for = [&](uint64_t m) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((m + 255) / 256, (uint64_t)dev.sms * 32));
  };
  auto read_u32 = [&](const uint32_t* d, uint32_t* h) {
    return cudaMemcpyAsync(h, d, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
  };
  SaArgs x;
  x.text = text;
  x.n = n;
  x.off = off;
  x.sa = out_sa;
  x.lcp = lcp0;
  x.isa = isa;
  x.gs = gs;
  x.flag = flag;
  x.h = h0;
  // with an LCP output: the names after every round, for the LCPs above h0
  std::vector<uint32_t*> snaps;
  auto snapshot = [&]() {
    if (!out_lcp) return true;
    if (snaps.size() >= kSaMaxSnaps) return false;  // cannot happen: at most 33 rounds for n < 2^32
    uint32_t* q = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&q), n * 4, st) != cudaSuccess) return false;
    snaps.push_back(q);
    return cudaMemcpyAsync(q, isa, n * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  };
  bool ok = sa_launch(SaKernel::kIota, x, grid_for(n), st, hook) == cudaSuccess;
  // round 0: the string sort by the first h0 characters
  if (ok) {
    ss_options o{};
    o.max_len = h0;
    o.small_cutoff = kSaSmallCutoff;
    o.big_threshold = kSaBigThreshold;
    s = sort_device(text, off, n, out_sa, lcp0, &o, st);
    ok = s == SS_OK;
  }
  uint32_t M = 0;
  if (ok) {
    ok = sa_launch(SaKernel::kHeads0, x, grid_for(n), st, hook) == cudaSuccess &&
         sa_scan_max(gs, n, tot, st, hook) == cudaSuccess &&
         sa_launch(SaKernel::kName0, x, grid_for(n), st, hook) == cudaSuccess &&
         sa_scan_sum(flag, n, tot, st, hook) == cudaSuccess && read_u32(flag + n - 1, &M) && snapshot();
    SaArgs c = x;
    c.vals = nullptr;
    c.out = cpos[0];
    if (ok && M) ok = sa_launch(SaKernel::kCompact, c, grid_for(n), st, hook) == cudaSuccess;
  }
  // doubling rounds over the unfinished groups (Observation 8.1)
  uint64_t h = h0;
  int cur = 0;
  while (ok && s == SS_OK && M > 0) {
    SaArgs r = x;
    r.M = M;
    r.h = (uint32_t)std::min<uint64_t>(h, 0xFFFFFFFFull);
    r.cpos = cpos[cur];
    r.member = member;
    r.enc = enc;
    r.eoff = eoff;
    r.perm2 = perm2;
    r.lcp2 = lcp2;
    ok = sa_launch(SaKernel::kEncode, r, grid_for(M), st, hook) == cudaSuccess;
    if (ok) {
      ss_options o2{};
      o2.small_cutoff = kSaSmallCutoff;
      o2.big_threshold = kSaBigThreshold;
      s = sort_device(enc, eoff, M, perm2, lcp2, &o2, st);
      ok = s == SS_OK;
    }
    uint32_t M2 = 0;
    if (ok)
      ok = sa_launch(SaKernel::kApply, r, grid_for(M), st, hook) == cudaSuccess &&
           sa_scan_max(gs, M, tot, st, hook) == cudaSuccess &&
           sa_launch(SaKernel::kRename, r, grid_for(M), st, hook) == cudaSuccess &&
           sa_scan_sum(flag, M, tot, st, hook) == cudaSuccess && read_u32(flag + M - 1, &M2) && snapshot();
    if (ok && M2) {
      SaArgs c = r;
      c.n = M;
      c.vals = cpos[cur];
      c.out = cpos[cur ^ 1];
      ok = sa_launch(SaKernel::kCompact, c, grid_for(M), st, hook) == cudaSuccess;
    }
    if (ok && M2 && h >= n) ok = false;  // cannot happen: every group is a singleton by depth n
    M = M2;
    cur ^= 1;
    h *= 2;
  }
  if (ok && s == SS_OK && out_lcp) {
    // LCPs of at least h0: list those positions, then one warp each
    SaArgs l = x;
    l.lcp_out = out_lcp;
    l.snaps.count = (uint32_t)snaps.size();
    for (size_t k = 0; k < snaps.size(); ++k) l.snaps.p[k] = snaps[k];
    uint32_t L = 0;
    ok = sa_launch(SaKernel::kLongFlags, l, grid_for(n), st, hook) == cudaSuccess &&
         sa_scan_sum(flag, n, tot, st, hook) == cudaSuccess && read_u32(flag + n - 1, &L);
    if (ok && L) {
      SaArgs c = x;
      c.vals = nullptr;
      c.out = cpos[0];
      l.cpos = cpos[0];
      l.M = L;
      ok = sa_launch(SaKernel::kCompact, c, grid_for(n), st, hook) == cudaSuccess &&
           sa_launch(SaKernel::kLcp, l, grid_for(32ull * L), st, hook) == cudaSuccess;
    }
  }
  for (uint32_t* q : snaps) cudaFreeAsync(q, st);
  cudaFreeAsync(ws, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && ok) ok = false;
  collect_profile();
  if (s != SS_OK) return s;
  const ss_status ds = take_stream_status(st);  // device status of the rounds' sorts
  if (ds != SS_OK) return ds;
  return ok ? SS_OK : SS_ERR_CUDA;
}

size_t ss_workspace_size(uint64_t n, const ss_options* opt) {
  Opts o;
  if (resolve_opts(opt, o) != SS_OK || n >= 0xFFFFFFFFull) return 0;
  return make_layout(n, 1, o, n > o.big_thr).total;
}

ss_status ss_sort_ex(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t* out_perm,
                     uint32_t* out_lcp, const ss_options* opt, void* stream) {
  return sort_device(chars, offsets, n, out_perm, out_lcp, opt, static_cast<cudaStream_t>(stream));
}

ss_status ss_sort(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t* out_perm,
                  uint32_t* out_lcp, void* stream) {
  return ss_sort_ex(chars, offsets, n, out_perm, out_lcp, nullptr, stream);
}

ss_status ss_sort_dna(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets, uint64_t n,
                      uint32_t* out_perm, uint32_t* out_lcp, const ss_options* opt, void* stream) {
  if (n >= 0xFFFFFFFFull) return SS_ERR_TOO_LARGE;
  if (n == 0) return SS_OK;
  if (!chars || !offsets || !out_perm || chars_len == 0) return SS_ERR_INVALID;
  if (chars_len >= (1ull << 60)) return SS_ERR_TOO_LARGE;
  Opts o;
  ss_status s = resolve_opts(opt, o);
  if (s != SS_OK) return s;
  DevInfo dev;
  if ((s = device_info(dev)) != SS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // packed codes, four zero words of padding (a key reads the word after its
  // own), then the invalid-byte flag
  const uint64_t words = (3 * chars_len + 63) / 64 + 4;
  const size_t flag_at = align256(words * 8);
  uint8_t* d = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), flag_at + 256, st) != cudaSuccess) return SS_ERR_OOM;
  uint32_t* bad = reinterpret_cast<uint32_t*>(d + flag_at);
  const LaunchHook hook{st};
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((words + kBlock - 1) / kBlock,
                                                                           (uint64_t)dev.sms * 16));
  ss_status r = SS_OK;
  if (cudaMemsetAsync(bad, 0, 4, st) != cudaSuccess ||
      launch_pack_dna(chars, chars_len, reinterpret_cast<uint64_t*>(d), words, bad, grid, st, hook) != cudaSuccess)
    r = SS_ERR_CUDA;
  if (r == SS_OK) r = sort_device(d, offsets, n, out_perm, out_lcp, opt, st, 1);
  uint32_t hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    if (r == SS_OK) r = SS_ERR_CUDA;
  cudaFreeAsync(d, st);
  if (r == SS_OK && hbad) r = SS_ERR_INVALID;
  const ss_status ds = take_stream_status(st);
  if (r == SS_OK) r = ds;
  return r;
}

// ---- host buffers ------------------------------------------------------------------

// With the default (0) the whole set is copied, then sorted: on the GB300's
// host link (about 210 GB/s) sorting the parts and merging them costs more
// than the overlap saves (20 M URL-like strings: 13.5 ms in one piece, 14.5 /
// 16.0 / 20.4 ms in 2 / 4 / 8 parts).
constexpr uint32_t kPipeAutoParts = 1;
// Merges of the parts use a sample step between these two, the largest that
// still gives about 1024 pieces per SM (a piece is merged by one lane).
constexpr uint32_t kPipeMinStep = 16, kPipeMaxStep = 64;
static_assert(sizeof(SetDesc) % 4 == 0 && sizeof(GenTask) % 4 == 0, "uploads move whole words");

// A copy stream and its events, per thread and device.
struct CopyLane {
  cudaStream_t cs = nullptr;
  cudaEvent_t start = nullptr, offs = nullptr, chunk[kMaxHostParts] = {};
  bool ready = false;
  ~CopyLane() {
    for (cudaEvent_t e : chunk)
      if (e) cudaEventDestroy(e);
    if (offs) cudaEventDestroy(offs);
    if (start) cudaEventDestroy(start);
    if (cs) cudaStreamDestroy(cs);
  }
};
static thread_local std::map<int, CopyLane> t_lanes;

static ss_status copy_lane(CopyLane*& out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_NO_DEVICE;
  CopyLane& l = t_lanes[dev];
  if (!l.ready) {
    bool ok = cudaStreamCreateWithFlags(&l.cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&l.start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&l.offs, cudaEventDisableTiming) == cudaSuccess;
    for (uint32_t p = 0; ok && p < kMaxHostParts; ++p)
      ok = cudaEventCreateWithFlags(&l.chunk[p], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return SS_ERR_CUDA;
    l.ready = true;
  }
  out = &l;
  return SS_OK;
}

// One binary LCP merge of two adjacent sorted ranges [lo, mid) and [mid, hi)
// of a record buffer (into the same range of dst, or of the outputs if dst is
// null).
static bool merge_pair(const uint8_t* chars, const uint64_t* offsets, uint32_t cap, const MergeRec* src,
                       MergeRec* dst, uint32_t lo, uint32_t mid, uint32_t hi, uint32_t* perm, uint32_t* lcp,
                       uint32_t* cut, uint32_t* counter, uint32_t sms, cudaStream_t st, const LaunchHook& hook) {
  uint32_t S = kPipeMaxStep;
  while (S > kPipeMinStep && (hi - lo) / S < sms * 1024u) S >>= 1;
  MergeRoundArgs ra{};
  ra.chars = chars;
  ra.offsets = offsets;
  ra.cap = cap;
  ra.ncur = 2;
  ra.S = S;
  ra.src = src + lo;
  ra.dst = dst ? dst + lo : nullptr;
  ra.cut = cut;
  ra.out_perm = perm + lo;
  ra.out_lcp = lcp + lo;
  ra.counter = counter;
  ra.start[0] = 0;
  ra.start[1] = mid - lo;
  ra.start[2] = hi - lo;
  ra.sbase[0] = 0;
  ra.sbase[1] = (mid - lo) / S;
  ra.sbase[2] = ra.sbase[1] + (hi - mid) / S;
  ra.nsamples = ra.sbase[2];
  return launch_upload(nullptr, counter, sizeof(uint32_t), st, hook) == cudaSuccess &&
         launch_merge_round(ra, sms, st, hook) == cudaSuccess;
}

// The copy overlapped with the sort (the scheme of Section 4.3.1 for NUMA
// machines, with the host link in the role of the slow interconnect): the
// strings are cut into P parts by index; part p's characters are copied on a
// second stream while part p - 1 is sorted; each sorted part becomes a run of
// 32-byte merge records, and adjacent runs are LCP-merged as soon as both
// exist (a binary tree, the last level writing the outputs).  This needs
// every part's strings inside its own stretch of chars (strings packed in
// index order), which k_layout_check verifies on the device once everything
// has arrived; a set that fails is sorted again as a whole (the parts'
// results are discarded).  Returns SS_OK with *done = false when the layout
// check failed.
static ss_status sort_host_parts(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets, uint64_t n,
                                 uint32_t P, uint8_t* dchars, uint64_t* doff, uint32_t* dperm, uint32_t* dlcp,
                                 uint8_t* scratch, const Opts& o, const ss_options* opt, const DevInfo& dev,
                                 cudaStream_t st, bool* done) {
  *done = false;
  CopyLane* lane = nullptr;
  ss_status s = copy_lane(lane);
  if (s != SS_OK) return s;
  // whatever happens below, no copy is still writing the buffers on return,
  // and the sort's small uploads are back on the copy engines
  struct Drain {
    cudaStream_t cs;
    ~Drain() {
      cudaStreamSynchronize(cs);
      t_kernel_copies = false;
    }
  } drain{lane->cs};
  t_kernel_copies = true;
  const LaunchHook hook{st};
  const uint32_t sms = (uint32_t)dev.sms;
  const size_t recb = align256(n * sizeof(MergeRec));
  MergeRec* rec[2] = {reinterpret_cast<MergeRec*>(scratch), reinterpret_cast<MergeRec*>(scratch + recb)};
  uint32_t* cut = reinterpret_cast<uint32_t*>(scratch + 2 * recb);
  uint32_t* ctl = reinterpret_cast<uint32_t*>(scratch + 2 * recb + align256((n / kPipeMinStep + 4) * 4));
  uint32_t* counter = ctl;
  uint32_t* bad = ctl + 1;
  // part p = strings [a[p], a[p + 1]); its characters [b[p], b[p + 1])
  uint64_t a[kMaxHostParts + 1], b[kMaxHostParts + 1];
  for (uint32_t p = 0; p <= P; ++p) a[p] = n * p / P;
  b[0] = 0;
  for (uint32_t p = 1; p < P; ++p) b[p] = std::max(b[p - 1], std::min<uint64_t>(offsets[a[p]], chars_len));
  b[P] = chars_len;
  SS_CUDA(launch_upload(nullptr, ctl, 8, st, hook));
  SS_CUDA(cudaEventRecord(lane->start, st));
  SS_CUDA(cudaStreamWaitEvent(lane->cs, lane->start, 0));
  SS_CUDA(cudaMemcpyAsync(doff, offsets, n * 8, cudaMemcpyHostToDevice, lane->cs));
  SS_CUDA(cudaEventRecord(lane->offs, lane->cs));
  for (uint32_t p = 0; p < P; ++p) {
    if (b[p + 1] > b[p])
      SS_CUDA(cudaMemcpyAsync(dchars + b[p], chars + b[p], b[p + 1] - b[p], cudaMemcpyHostToDevice, lane->cs));
    SS_CUDA(cudaEventRecord(lane->chunk[p], lane->cs));
  }
  SS_CUDA(cudaStreamWaitEvent(st, lane->offs, 0));
  const uint32_t cap = std::min<uint32_t>(o.cap, 1u << 30);
  for (uint32_t p = 0; p < P; ++p) {
    SS_CUDA(cudaStreamWaitEvent(st, lane->chunk[p], 0));
    const uint32_t lo = (uint32_t)a[p], np = (uint32_t)(a[p + 1] - a[p]);
    s = sort_device(dchars, doff + lo, np, dperm + lo, dlcp + lo, opt, st);
    if (s != SS_OK) return s;
    MergePrepArgs pa{};
    pa.chars = dchars;
    pa.offsets = doff;
    pa.cap = cap;
    pa.K = 1;
    pa.total = np;
    pa.dst = rec[0] + lo;
    pa.start[0] = 0;
    pa.start[1] = np;
    pa.perm[0] = dperm + lo;
    pa.lcp[0] = dlcp + lo;
    pa.ibase[0] = lo;
    SS_CUDA(launch_merge_prep(pa, sms, st, hook));
    // merge every complete pair of runs up the tree
    for (uint32_t w = 2, lvl = 1; w <= P && (p + 1) % w == 0; w <<= 1, ++lvl) {
      const uint32_t q0 = p + 1 - w;
      MergeRec* dst = w == P ? nullptr : rec[lvl & 1];
      if (!merge_pair(dchars, doff, cap, rec[(lvl - 1) & 1], dst, (uint32_t)a[q0], (uint32_t)a[q0 + w / 2],
                      (uint32_t)a[p + 1], dperm, dlcp, cut, counter, sms, st, hook))
        return SS_ERR_CUDA;
    }
  }
  SS_CUDA(launch_layout_check(dchars, chars_len, doff, (uint32_t)n, bad, sms, st, hook));
  if (t_down.reserve(256) != SS_OK) return SS_ERR_OOM;
  uint32_t* hbad = static_cast<uint32_t*>(t_down.p);
  SS_CUDA(cudaMemcpyAsync(hbad, bad, 4, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  *done = *hbad == 0;
  return SS_OK;
}

ss_status ss_sort_host(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets, uint64_t n,
                       uint32_t* out_perm, uint32_t* out_lcp, const ss_options* opt, void* stream) {
  if (n >= 0xFFFFFFFFull) return SS_ERR_TOO_LARGE;
  if (n == 0) return SS_OK;
  if (!chars || !offsets || !out_perm || chars_len == 0) return SS_ERR_INVALID;
  Opts o;
  ss_status s = resolve_opts(opt, o);
  if (s != SS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevInfo dev;
  s = device_info(dev);
  if (s != SS_OK) return s;
  uint32_t P = o.host_parts;
  if (P == 0) P = kPipeAutoParts;
  if (n < 2ull * P) P = 1;
  if (P > 1) {  // the part boundaries are read from the offsets on the host
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, offsets) != cudaSuccess) {
      cudaGetLastError();
      return SS_ERR_INVALID;
    }
    if (at.type == cudaMemoryTypeDevice) return SS_ERR_INVALID;
  }
  const size_t cb = align256(chars_len + 16), ob = align256(n * 8), pb = align256(n * 4);
  const size_t scratch = P > 1 ? 2 * align256(n * sizeof(MergeRec)) + align256((n / kPipeMinStep + 4) * 4) + 256
                               : 0;
  const size_t need = cb + ob + 2 * pb + scratch;
  uint8_t* d = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), need, st) != cudaSuccess) return SS_ERR_OOM;
  uint8_t* dchars = d;
  uint64_t* doff = reinterpret_cast<uint64_t*>(d + cb);
  uint32_t* dperm = reinterpret_cast<uint32_t*>(d + cb + ob);
  uint32_t* dlcp = reinterpret_cast<uint32_t*>(d + cb + ob + pb);
  ss_status r = SS_OK;
  // zeros after the last byte: a read past it finds a terminator
  if (cudaMemsetAsync(dchars + chars_len, 0, cb - chars_len, st) != cudaSuccess) r = SS_ERR_CUDA;
  bool done = false;
  if (r == SS_OK && P > 1)
    r = sort_host_parts(chars, chars_len, offsets, n, P, dchars, doff, dperm, dlcp, d + cb + ob + 2 * pb, o, opt,
                        dev, st, &done);
  if (r == SS_OK && !done) {
    if (P == 1 && (cudaMemcpyAsync(dchars, chars, chars_len, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                   cudaMemcpyAsync(doff, offsets, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess))
      r = SS_ERR_CUDA;
    if (r == SS_OK) r = sort_device(dchars, doff, n, dperm, out_lcp ? dlcp : nullptr, opt, st);
  }
  if (r == SS_OK) {
    if (cudaMemcpyAsync(out_perm, dperm, n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) r = SS_ERR_CUDA;
    if (out_lcp && cudaMemcpyAsync(out_lcp, dlcp, n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      r = SS_ERR_CUDA;
  }
  cudaFreeAsync(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && r == SS_OK) r = SS_ERR_CUDA;
  const ss_status ds = take_stream_status(st);
  if (r == SS_OK) r = ds;
  return r;
}

// Total strings of a batch, and whether some set takes multi-block steps.
static ss_status batch_geometry(const ss_set* sets, uint32_t num_sets, const Opts& o, uint64_t* total, bool* big) {
  if (num_sets && !sets) return SS_ERR_INVALID;
  uint64_t t = 0;
  bool b = false;
  for (uint32_t i = 0; i < num_sets; ++i) {
    const ss_set& s = sets[i];
    if (s.n && (!s.chars || !s.offsets || !s.out_perm)) return SS_ERR_INVALID;
    t += s.n;
    b = b || s.n > o.big_thr;
  }
  if (t >= 0xFFFFFFFFull) return SS_ERR_TOO_LARGE;
  *total = t;
  *big = b;
  return SS_OK;
}

size_t ss_batch_workspace_size(const ss_set* sets, uint32_t num_sets, const ss_options* opt) {
  Opts o;
  uint64_t total = 0;
  bool big = false;
  if (resolve_opts(opt, o) != SS_OK || batch_geometry(sets, num_sets, o, &total, &big) != SS_OK) return 0;
  return make_layout(total, num_sets, o, big).total;
}

ss_status ss_batch_create(const ss_set* sets, uint32_t num_sets, const ss_options* opt, ss_batch** out) {
  if (!out) return SS_ERR_INVALID;
  *out = nullptr;
  ss_batch b;
  ss_status s = resolve_opts(opt, b.o);
  if (s != SS_OK) return s;
  uint64_t total = 0;
  if ((s = batch_geometry(sets, num_sets, b.o, &total, &b.big)) != SS_OK) return s;
  if ((s = device_info(b.dev)) != SS_OK) return s;
  b.L = make_layout(total, num_sets, b.o, b.big);
  if (opt && opt->workspace) {
    if (opt->workspace_bytes < b.L.total) return SS_ERR_INVALID;
    b.ws = static_cast<uint8_t*>(opt->workspace);
  } else {
    if (cudaMalloc(reinterpret_cast<void**>(&b.ws), b.L.total) != cudaSuccess) return SS_ERR_OOM;
    b.owned = true;
  }
  // The descriptors go into the workspace with each run, on its stream: a
  // caller's workspace is stream-ordered memory that earlier work on that
  // stream may still be using when the batch is created.
  b.sd.resize(num_sets);
  uint32_t base = 0;
  for (uint32_t i = 0; i < num_sets; ++i) {
    const ss_set& x = sets[i];
    b.sd[i] = SetDesc{x.chars, x.offsets, x.out_perm, x.out_lcp, x.n, x.max_len ? x.max_len : kNoCap, base, 0};
    base += x.n;
  }
  b.num_sets = num_sets;
  b.total = (uint32_t)total;
  *out = new ss_batch(b);
  return SS_OK;
}

ss_status ss_batch_run(ss_batch* b, void* stream) {
  if (!b) return SS_ERR_INVALID;
  if (b->num_sets == 0) return SS_OK;
  {
    std::lock_guard<std::mutex> lk(g_stream_mu);
    g_stream_last[stream] = b;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the set descriptors, as kernel parameters (no staging copy to wait for,
  // and capturable)
  SetDesc* dsets = reinterpret_cast<SetDesc*>(b->ws + b->L.sets);
  for (uint32_t i0 = 0; i0 < b->num_sets; i0 += kDescChunk) {
    SetDescChunk ch;
    const uint32_t cnt = std::min(kDescChunk, b->num_sets - i0);
    std::copy(b->sd.begin() + i0, b->sd.begin() + i0 + cnt, ch.d);
    LaunchHook{st}.run("init", [&] { k_set_descs<<<1, kBlock, 0, st>>>(dsets + i0, cnt, ch); });
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
  }
  SortCtx c = make_ctx(b->ws, b->L, b->num_sets, b->total, b->o, b->big);
  // the multi-block loop's control block: inside a caller's capture the
  // batch's own (its address goes into the caller's graph); otherwise the
  // stream's, whose loop graph is built once per stream
  BigCtl* ctl = nullptr;
  if (b->big) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return SS_ERR_CUDA;
    if (cs == cudaStreamCaptureStatusActive) {
      ctl = reinterpret_cast<BigCtl*>(b->ws + b->L.bigctl);
    } else {
      StreamSlot* slot = nullptr;
      ss_status s = stream_slot(st, true, &slot);
      if (s != SS_OK) return s;
      ctl = &slot->ctl;
    }
  }
  return run_sort(b->ws, b->L, c, b->o, b->dev, b->big, st, ctl);
}

ss_status ss_batch_status(ss_batch* b, void* stream) {
  if (!b) return SS_ERR_INVALID;
  if (b->num_sets == 0) return SS_OK;
  return read_status(b->ws, b->L, static_cast<cudaStream_t>(stream));
}

ss_status ss_batch_destroy(ss_batch* b) {
  if (!b) return SS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(g_stream_mu);
    for (auto it = g_stream_last.begin(); it != g_stream_last.end();)
      it = (it->second == b) ? g_stream_last.erase(it) : std::next(it);
  }
  if (b->owned) cudaFree(b->ws);
  delete b;
  return SS_OK;
}

ss_status ss_stream_status(void* stream) {
  ss_batch* b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_stream_mu);
    auto it = g_stream_last.find(stream);
    if (it != g_stream_last.end()) b = it->second;
  }
  // the sorts' status word of the stream, then the last batch run on it
  const ss_status s = take_stream_status(static_cast<cudaStream_t>(stream));
  if (s != SS_OK || !b) return s;
  return ss_batch_status(b, stream);
}

ss_status ss_sort_batch(const ss_set* sets, uint32_t num_sets, const ss_options* opt, void* stream) {
  ss_batch* b = nullptr;
  ss_status s = ss_batch_create(sets, num_sets, opt, &b);
  if (s != SS_OK) return s;
  s = ss_batch_run(b, stream);
  ss_status s2 = ss_batch_status(b, stream);
  ss_batch_destroy(b);
  return s != SS_OK ? s : s2;
}

}  // extern "C"

// ---- sorting without any allocation ------------------------------------------------------
//
// For callers that cannot allocate device memory while they run: for example a
// service that reserves all of its GPU memory at start-up and forbids later
// allocation, code whose device memory belongs to another allocator, or a
// latency-critical path where cudaMalloc / cudaFree (which may synchronise the
// device) are not allowed.  The workspace of these sorts is a fixed array in
// the library's device data, so the call itself allocates nothing.

namespace ss {

// Scratch of ss_sort_noalloc.  Every GPU that loads this library holds it
// until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[SS_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static uint8_t* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};


// Device address of the scratch on the current device, looked up once per
// device.  Host code only ever passes this address to kernels: the name
// g_noalloc_scratch in host code is a host-side stand-in, not device memory.
static ss_status noalloc_scratch(uint8_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_NO_DEVICE;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SS_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SS_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SS_OK;
}

}  // namespace ss

extern "C" ss_status ss_sort_noalloc(const uint8_t* chars, const uint64_t* offsets, uint64_t n,
                                     uint32_t max_len, uint32_t* out_perm, uint32_t* out_lcp, void* stream) {
  using namespace ss;
  if (n > SS_NOALLOC_MAX_STRINGS) return SS_ERR_TOO_LARGE;
  if (n == 0) return SS_OK;
  if (!chars || !offsets || !out_perm) return SS_ERR_INVALID;
  if (g_profiling.load()) return SS_ERR_INVALID;  // profiling would create CUDA events
  Opts o;
  if (max_len) o.cap = max_len;
  const Layout L = make_layout(n, 1, o, false);
  if (L.total > SS_NOALLOC_SCRATCH_BYTES) return SS_ERR_TOO_LARGE;
  DevInfo dev;
  ss_status s = device_info(dev);
  if (s != SS_OK) return s;
  uint8_t* ws = nullptr;
  if ((s = noalloc_scratch(&ws)) != SS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SetDesc sd{chars, offsets, out_perm, out_lcp, (uint32_t)n, o.cap, 0, 0};
  const LaunchHook hook{st};
  hook.run("init", [&] { k_set_desc<<<1, 1, 0, st>>>(reinterpret_cast<SetDesc*>(ws + L.sets), sd); });
  if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
  // run_sort clears the control words and the queue flags, the only scratch
  // that must start at zero; everything else is written before it is read.
  s = run_sort(ws, L, make_ctx(ws, L, 1, (uint32_t)n, o, false), o, dev, false, st);
  if (s != SS_OK) return s;
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, ws + L.ctrl, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SS_ERR_CUDA;
  return map_status(status);
}
