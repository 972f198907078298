// Host-side launch interface between the orchestrator (ss_host.cu) and the
// kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>

#include <cuda_runtime.h>

#include "ss_internal.cuh"

namespace ss {

// Wraps every kernel launch: counts it and, when profiling is on, brackets it
// with CUDA events on the launching stream.
struct LaunchHook {
  cudaStream_t stream;
  void run(const char* name, const std::function<void()>& launch) const;
};

// Control block of the multi-block steps in device memory.  The host fills
// the first part once per sort; k_big_plan writes the plan of each round from
// the list of big subsets the previous round left, and every kernel of the
// round reads it there, so rounds follow one another with no host in the loop
// (Section 4.2.8: the fully parallel levels need no sequential coordinator).
struct BigCtl {
  SortCtx c;
  GenTask* gt;            // cap_big tasks of the current round
  void* splitters;        // cap_big * big_splitters_bytes(logv)
  uint32_t* counters;     // [task][bucket][tile] counters of the round
  uint32_t* partials;     // ncounters_max / 4096 + 2
  uint32_t* gstart;       // cap_big * KP bucket starts
  uint32_t* gdesc;        // cap_big * KP bucket descriptors
  uint64_t ncounters_max;
  uint32_t cap_big;
  uint32_t R_fixed;       // tile rounds; 0: chosen per round from the strings in big subsets
  uint32_t sms;
  uint32_t K;             // buckets per step, 2^(logv + 1) - 1
  // the plan of the current round (k_big_plan)
  uint32_t cur;           // big list the next plan reads
  uint32_t next_big;      // big list the current round's new big subsets go to
  uint32_t round;
  uint32_t G;             // big subsets of the round (0: the loop ends)
  uint32_t tiles;         // tiles over them
  uint32_t R;             // tile = 256 * R records
  uint64_t ncounters;
  // work counters of the round's kernels (zeroed by the plan): blocks take
  // the next subset or tile from them, so that uneven tiles balance out
  uint32_t next_item[4];  // sample, classify, emit, scatter
};

// Most rounds of multi-block steps one sort may take (each advances every big
// subset by at least one character; a subset sharing more than about 2^20
// characters is reported as SS_ERR_TOO_LARGE).
constexpr uint32_t kMaxBigRounds = 1u << 20;

// Kernel launches of one multi-block round after its plan: sample, classify,
// the two prefix-sum kernels, emit and scatter.
constexpr uint32_t kBigRoundKernels = 6;

size_t big_splitters_bytes(int logv);
size_t big_scatter_smem(int logv, uint32_t R);
// The plan of the next round; with use_cond it also sets the loop graph's
// condition (1 while big subsets remain).
cudaError_t launch_big_plan(BigCtl* ctl, uint64_t cond_handle, bool use_cond, cudaStream_t st,
                            const LaunchHook& hook);
// The kernels of one round (they do nothing when the plan found no subset).
cudaError_t launch_big_round(int logv, BigCtl* ctl, uint32_t R_max, uint32_t sms, cudaStream_t st,
                             const LaunchHook& hook);
// Kernels the loop graphs of this device have launched so far (their plan
// kernels count them on the device; reading the count waits for the device).
uint64_t graph_launch_count();

// Persistent work-queue kernel (single-block S^5 steps).
size_t queue_smem(int logv);
cudaError_t queue_occupancy(int logv, int* blocks_per_sm);
cudaError_t launch_queue(int logv, const SortCtx& c, uint32_t grid, uint32_t R, cudaStream_t st,
                         const LaunchHook& hook);

// Small subsets, set-up and LCP fix-up.
size_t small_cta_smem(uint32_t pmax);
cudaError_t launch_init(const SortCtx& c, cudaStream_t st, const LaunchHook& hook);
cudaError_t launch_small(const SortCtx& c, uint32_t pmax, uint32_t grid_warp, uint32_t grid_cta,
                         cudaStream_t st, const LaunchHook& hook);
cudaError_t launch_lcp_fix(const SortCtx& c, uint32_t grid, cudaStream_t st, const LaunchHook& hook);
// Packs bytes over {A, C, G, T, 0} into 3-bit codes (dna_key's layout).
// Copies bytes (a multiple of 4, 4-byte aligned) from pinned host memory
// with a kernel, or zero-fills dst when host_src is null.
cudaError_t launch_upload(const void* host_src, void* dst, size_t bytes, cudaStream_t st, const LaunchHook& hook);
cudaError_t launch_pack_dna(const uint8_t* chars, uint64_t len, uint64_t* out, uint64_t words, uint32_t* bad,
                            uint32_t grid, cudaStream_t st, const LaunchHook& hook);
cudaError_t launch_distinguishing(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t cap,
                                  const uint32_t* perm, const uint32_t* lcp, uint8_t* dchar, uint32_t* dprefix,
                                  unsigned long long* sum_d, uint32_t grid, cudaStream_t st, const LaunchHook& hook);

// K-way LCP merge of sorted runs (ss_merge.cu): ceil(log2 K) rounds of
// pairwise LCP merges over 32-byte records.
constexpr uint32_t kMergeMaxRuns = 64;

struct MergeRec {
  uint64_t w0, w1;   // the string's characters [h, h + 16), first one most significant
  uint64_t off;      // string offset
  uint32_t idx;      // string index
  uint32_t h;        // LCP with the preceding string of its run
};

// Records of all runs, run k at [start[k], start[k + 1]).
struct MergePrepArgs {
  const uint8_t* chars;
  const uint64_t* offsets;
  uint32_t cap;
  uint32_t K;
  uint32_t total;
  MergeRec* dst;
  uint32_t start[kMergeMaxRuns + 1];
  const uint32_t* perm[kMergeMaxRuns];
  const uint32_t* lcp[kMergeMaxRuns];
  uint32_t ibase[kMergeMaxRuns];  // added to run k's entries (runs sorted with local indices)
};

// One round: current run c at [start[c], start[c + 1]); runs 2p and 2p + 1
// are merged into the same range; every S-th record of a run is a sample,
// the samples of run c being [sbase[c], sbase[c + 1]).
struct MergeRoundArgs {
  const uint8_t* chars;
  const uint64_t* offsets;
  uint32_t cap;
  uint32_t ncur;
  uint32_t S;
  uint32_t nsamples;
  const MergeRec* src;
  MergeRec* dst;            // null in the last round
  uint32_t* cut;            // per sample: records of the partner run before it
  uint32_t* out_perm;       // last round
  uint32_t* out_lcp;        // last round, may be null
  uint32_t* counter;        // piece counter, zero at launch
  uint32_t start[kMergeMaxRuns + 1];
  uint32_t sbase[kMergeMaxRuns + 1];
};

cudaError_t launch_merge_prep(const MergePrepArgs& a, uint32_t sms, cudaStream_t st, const LaunchHook& hook);
cudaError_t launch_merge_round(const MergeRoundArgs& a, uint32_t sms, cudaStream_t st, const LaunchHook& hook);
cudaError_t launch_merge_copy(const uint32_t* perm, const uint32_t* lcp, uint32_t n, uint32_t* out_perm,
                              uint32_t* out_lcp, uint32_t sms, cudaStream_t st, const LaunchHook& hook);
// Sets *bad unless every string i lies in [offsets[i], offsets[i + 1]) with
// its terminator at offsets[i + 1] - 1 (the last one ending at chars_len - 1).
cudaError_t launch_layout_check(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets, uint32_t n,
                                uint32_t* bad, uint32_t sms, cudaStream_t st, const LaunchHook& hook);

// Suffix array by prefix doubling (ss_sa.cu).
enum class SaKernel { kIota, kHeads0, kName0, kCompact, kEncode, kApply, kRename, kLongFlags, kLcp };

// Name arrays of the suffixes after each round (ISA^{h0 2^k}, k = 0..count-1),
// kept for the LCPs above h0.
constexpr uint32_t kSaMaxSnaps = 40;
struct SaSnaps {
  const uint32_t* p[kSaMaxSnaps];
  uint32_t count;
};

struct SaArgs {
  const uint8_t* text = nullptr;
  uint64_t n = 0;             // strings the kernel runs over (suffixes, or members M)
  uint32_t h = 0;             // current depth (h0 for kHeads0 / kName0 / kLcp)
  uint32_t M = 0;
  uint64_t* off = nullptr;
  uint32_t* sa = nullptr;
  const uint32_t* lcp = nullptr;  // capped LCPs of the first sort
  uint32_t* lcp_out = nullptr;    // final LCP array (holds the capped LCPs on entry)
  uint32_t* isa = nullptr;
  uint32_t* gs = nullptr;
  uint32_t* flag = nullptr;       // flags, then their inclusive sum
  const uint32_t* vals = nullptr;
  uint32_t* out = nullptr;
  const uint32_t* cpos = nullptr;
  uint32_t* member = nullptr;
  uint8_t* enc = nullptr;
  uint64_t* eoff = nullptr;
  const uint32_t* perm2 = nullptr;
  const uint32_t* lcp2 = nullptr;
  SaSnaps snaps{};
};

size_t sa_scan_totals(uint64_t n);  // entries of the scan's tile-total buffer
cudaError_t sa_scan_max(uint32_t* a, uint64_t n, uint32_t* tot, cudaStream_t st, const LaunchHook& hook);
cudaError_t sa_scan_sum(uint32_t* a, uint64_t n, uint32_t* tot, cudaStream_t st, const LaunchHook& hook);
cudaError_t sa_launch(SaKernel k, const SaArgs& x, uint32_t grid, cudaStream_t st, const LaunchHook& hook);

}  // namespace ss
