// hist_api.cpp -- the C ABI declared in include/hist.h.
//
// A histogram object plays the role of the paper's GPU histogram class
// (Sec. 3.2): it owns the device allocations (bins, statistics, axis
// tables, launch scratch), fills bulk by bulk on the caller's stream, and
// copies the result back once on request.  Fills accumulate (Sec. 3.3: the
// statistics of the previous bulk are combined with the current ones, never
// overwritten).  All argument checks run on the host before any launch.

#include <cuda_runtime.h>

#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hist.h"
#include "axis_compile.h"
#include "hist_internal.h"

using namespace hgb;

namespace {

constexpr int kDefaultFxElo = 1015;             // |w| in [2^-8, 2^8) summed exactly
constexpr size_t kSmemTableBudget = 64 * 1024;  // threshold keys staged per block
constexpr size_t kSmemBucketBudget = 32 * 1024; // bucket counts staged per block
constexpr int64_t kDirectFlushMaxEvents = 1 << 22; // fills up to this size flush their bins in the fill kernel
constexpr int64_t kDefaultHostBulk = 1 << 22;    // events per staged bulk of hist_fill_host
constexpr int64_t kHostGraphBulk = 1 << 20;      // bulks up to this size replay as one graph
constexpr int64_t kHostGraphBulks = 4096;        // ... when there are at most this many
constexpr int kBucketMax = 1 << 22;             // buckets of one axis at most
constexpr int kBucketMaxRun = 16;               // most thresholds in one bucket for LOC_BUCKET
constexpr size_t kExactBytes = (size_t)kExactStats * (kExactLimbs + kEscapeLimbs + 3) * 8;
#ifndef HGB_SMEM_BINS_BUDGET
#define HGB_SMEM_BINS_BUDGET (96 * 1024)
#endif
constexpr size_t kSmemBinsBudget = HGB_SMEM_BINS_BUDGET;  // per-block bins (96 KB keeps >= 2 blocks per SM)

}  // namespace

struct hist {
  int device = 0;
  int sm_count = 0;
  int ndim = 0;
  int nstats = 0;
  uint32_t flags = 0;
  int acc_mode = ACC_UNIT;
  int32_t kind[kMaxDim] = {0, 0, 0};
  int32_t nbins[kMaxDim] = {0, 0, 0};
  int64_t nbins_total = 0;
  // axis tables
  long long* d_T = nullptr;  // concatenated thresholds, nbins + 3 keys per axis
  int32_t t_off[kMaxDim] = {0, 0, 0};
  int32_t table_keys = 0;
  int32_t smem_keys = 0;     // how many keys are staged into shared memory
  int32_t loc_mode[kMaxDim] = {0, 0, 0};
  float scale[kMaxDim] = {0, 0, 0}, offset[kMaxDim] = {0, 0, 0}, eps[kMaxDim] = {1, 1, 1};
  std::vector<int64_t> T_host[kMaxDim];  // host copy of the thresholds
  // bucket maps of the LOC_BUCKET axes
  int* d_BK = nullptr;       // concatenated bucket counts
  int32_t bk_off[kMaxDim] = {-1, -1, -1};
  int32_t smem_bk = 0;       // how many bucket counts are staged into shared memory
  BucketDev bk[kMaxDim] = {};
  int2* lm_knots[kMaxDim] = {nullptr, nullptr, nullptr};
  LearnedDev lm[kMaxDim] = {};
  int config_version = 0;    // bumped when a locator is installed (batches rebuild descriptors)
  bool smem_unit = true;     // unit-weight fills keep per-block bins in shared memory
  bool smem_weighted = true; // weighted fills likewise (16 bytes per bin)
  int fx_elo = kDefaultFxElo;
  // persistent accumulators
  unsigned long long* g_lo = nullptr;
  long long* g_hi = nullptr;
  unsigned long long* g_count = nullptr;
  unsigned long long* g_unit = nullptr;
  double* g_f64 = nullptr;
  double* g_sumw2 = nullptr;  // HIST_SUMW2: binary64 per-bin sum of w^2 of weighted fills
  unsigned long long* g_passed = nullptr;  // entries of filtered fills (counted on the device)
  unsigned* d_ticket = nullptr;            // the direct-flush fills' finished-block counter (0 between fills)
  // HIST_STATS_EXACT: limbs, escape limbs and special-term counts of the 4 statistics
  long long* d_exact = nullptr;
  int32_t exact_grid[kExactStats] = {};
  int64_t exact_launches = 0;
  double* g_stats = nullptr;
  int64_t n_entries = 0;
  bool counts_complete = true;  // false once a weighted fill ran without HIST_TRACK_COUNTS
  int64_t fx_global_since_norm = 0;
  // launch scratch
  void* part_bins = nullptr;
  size_t part_bins_bytes = 0;
  double* part_stats = nullptr;
  int part_stats_blocks = 0;
  double* part_sumw2 = nullptr;
  size_t part_sumw2_bytes = 0;
  // ordering of fills issued on different streams
  cudaEvent_t done = nullptr;
  bool have_done = false;
  // host-bulk pipeline (hist_fill_host): two device staging slots
  double* d_stage[2] = {nullptr, nullptr};
  int64_t stage_events = 0;  // events per slot
  cudaStream_t copy_stream[2] = {nullptr, nullptr};  // one per slot: two copies in flight
  cudaEvent_t copied[2] = {nullptr, nullptr};
  cudaEvent_t consumed[2] = {nullptr, nullptr};
  bool slot_used[2] = {false, false};
  cudaEvent_t fork_ev = nullptr;
  bool capturing = false;   // inside a graph capture: no waits on events recorded outside it
  // graph of a whole pipelined fill, replayed while its arguments repeat
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t host_exec = nullptr;
  const double* g_values = nullptr;
  const double* g_weights = nullptr;
  int64_t g_n = -1, g_bulk = -1;
  // optional timing of the fill kernel alone (pairs of events around it)
  bool timing = false;
  std::vector<cudaEvent_t> t_ev;
  size_t t_used = 0;  // pairs recorded since the last hist_kernel_time
};

namespace {

// Ints of an axis' bucket table.
int bucket_ints(const BucketDev& b) { return b.single ? 4 * b.nbk : b.nbk + 1; }

template <class T>
int dalloc(T** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return HIST_ERR_OOM;
  }
  return e == cudaSuccess ? HIST_OK : HIST_ERR_CUDA;
}

void free_state(hist* h) {
  for (int i = 0; i < 2; ++i)
    if (h->copy_stream[i]) cudaStreamSynchronize(h->copy_stream[i]);
  for (int i = 0; i < 2; ++i) {
    if (h->consumed[i]) cudaEventSynchronize(h->consumed[i]);
    if (h->copied[i]) cudaEventDestroy(h->copied[i]);
    if (h->consumed[i]) cudaEventDestroy(h->consumed[i]);
    cudaFree(h->d_stage[i]);
  }
  for (int i = 0; i < 2; ++i)
    if (h->copy_stream[i]) cudaStreamDestroy(h->copy_stream[i]);
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->host_exec) cudaGraphExecDestroy(h->host_exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->done) cudaEventDestroy(h->done);
  for (cudaEvent_t e : h->t_ev) cudaEventDestroy(e);
  cudaFree(h->d_T);
  cudaFree(h->d_BK);
  cudaFree(h->g_lo);
  cudaFree(h->g_hi);
  cudaFree(h->g_count);
  cudaFree(h->g_unit);
  cudaFree(h->g_f64);
  cudaFree(h->g_stats);
  cudaFree(h->g_sumw2);
  cudaFree(h->g_passed);
  cudaFree(h->d_ticket);
  cudaFree(h->d_exact);
  cudaFree(h->part_sumw2);
  cudaFree(h->part_bins);
  cudaFree(h->part_stats);
  for (int d = 0; d < kMaxDim; ++d) cudaFree(h->lm_knots[d]);
}

int acc_mode_of(uint32_t flags, bool unit) {
  if (unit) return ACC_UNIT;
  switch (flags & HIST_PREC_MASK) {
    case HIST_PREC_F64ATOMIC:
      return ACC_F64;
    case HIST_PREC_FP32C:
      return ACC_F32C;
    default:
      return ACC_FX;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Build the launch parameters of one fill (or locate) call.
FillParams make_params(const hist* h, const double* values, const double* weights, int64_t n, int acc) {
  FillParams p;
  std::memset(&p, 0, sizeof(p));
  for (int d = 0; d < h->ndim; ++d) {
    AxisDev& a = p.ax[d];
    a.T = h->d_T + h->t_off[d];
    a.nbins = h->nbins[d];
    a.mode = h->loc_mode[d];
    a.smem_off = (h->t_off[d] + h->nbins[d] + 3 <= h->smem_keys) ? h->t_off[d] : -1;
    a.scale = h->scale[d];
    a.offset = h->offset[d];
    a.eps = h->eps[d];
    a.lm = h->lm[d];
    a.bk = h->bk[d];
    if (h->bk_off[d] >= 0) a.bk.smem_off = (h->bk_off[d] + bucket_ints(h->bk[d]) <= h->smem_bk) ? h->bk_off[d] : -1;
    p.col[d] = values + (size_t)d * (size_t)n;
  }
  p.w = weights;
  p.T_concat = h->d_T;
  p.n = n;
  p.nbins_total = h->nbins_total;
  p.ndim = h->ndim;
  p.nstats = h->nstats;
  p.stat_overflows = (h->flags & HIST_STAT_OVERFLOWS) ? 1 : 0;
  p.track_counts = (h->flags & HIST_TRACK_COUNTS) ? 1 : 0;
  p.fx_elo = h->fx_elo;
  p.table_keys = h->smem_keys;
  p.BK_concat = h->d_BK;
  p.table_bk = h->smem_bk;
  bool al = weights == nullptr || aligned16(weights);
  for (int d = 0; d < h->ndim; ++d) al = al && aligned16(p.col[d]);
  p.aligned = al ? 1 : 0;
  p.smem_bins = (acc == ACC_UNIT ? h->smem_unit : h->smem_weighted) ? 1 : 0;
  p.sumw2 = (acc != ACC_UNIT && (h->flags & HIST_SUMW2)) ? 1 : 0;
  p.g_sumw2 = h->g_sumw2;
  // small fills with exact fixed-point or unit-count shared bins flush
  // themselves (integer atomics from every block, statistics summed by the
  // last block): no partial bins and no reduce launch, which took most of a
  // 32768-event fill (the paper's bulks: 1.9 -> 2.7 Gevents/s from host
  // memory).  Large fills keep the reduce: there the two cost the same within
  // 1 % of the call, and the fill kernel stays free of the flush.
  p.direct_flush = (n <= kDirectFlushMaxEvents && fill_direct_ok(p, acc)) ? 1 : 0;
  p.ticket = h->d_ticket;
  p.g_stats = h->g_stats;
  p.part_bins = h->part_bins;
  p.part_stats = h->part_stats;
  p.part_sumw2 = h->part_sumw2;
  p.g_lo = h->g_lo;
  p.g_hi = h->g_hi;
  p.g_count = h->g_count;
  p.g_unit = h->g_unit;
  p.g_f64 = h->g_f64;
  return p;
}

// A captured host-pipeline graph holds the scratch pointers: drop it when
// they move (it is captured again on its next use).
void drop_host_graph(hist* h) {
  if (h->host_exec) {
    if (h->have_done) cudaEventSynchronize(h->done);
    cudaGraphExecDestroy(h->host_exec);
    h->host_exec = nullptr;
  }
}

int ensure_scratch(hist* h, int grid, int acc, bool smem_bins) {
  const size_t need = smem_bins ? (size_t)grid * (size_t)h->nbins_total * part_bin_bytes(acc, 0) : 16;
  const bool grows = need > h->part_bins_bytes || grid > h->part_stats_blocks ||
                     ((smem_bins && (h->flags & HIST_SUMW2)) &&
                      (size_t)grid * (size_t)h->nbins_total * 8 > h->part_sumw2_bytes);
  if (grows && h->capturing) return HIST_ERR_CUDA;  // pipeline_prepare sized them before the capture
  if (grows) drop_host_graph(h);
  if (need > h->part_bins_bytes) {
    cudaFree(h->part_bins);
    h->part_bins = nullptr;
    h->part_bins_bytes = 0;
    int rc = dalloc(&h->part_bins, need);
    if (rc != HIST_OK) return rc;
    h->part_bins_bytes = need;
  }
  const size_t need2 = (smem_bins && (h->flags & HIST_SUMW2)) ? (size_t)grid * (size_t)h->nbins_total * 8 : 0;
  if (need2 > h->part_sumw2_bytes) {
    cudaFree(h->part_sumw2);
    h->part_sumw2 = nullptr;
    h->part_sumw2_bytes = 0;
    int rc = dalloc(&h->part_sumw2, need2);
    if (rc != HIST_OK) return rc;
    h->part_sumw2_bytes = need2;
  }
  if (grid > h->part_stats_blocks) {
    cudaFree(h->part_stats);
    h->part_stats = nullptr;
    h->part_stats_blocks = 0;
    int rc = dalloc(&h->part_stats, (size_t)grid * kMaxStats * sizeof(double));
    if (rc != HIST_OK) return rc;
    h->part_stats_blocks = grid;
  }
  return HIST_OK;
}

// Order this call after the previous fill when it used another stream.
int order_after_previous(hist* h, cudaStream_t s) {
  if (h->have_done && !h->capturing) {
    if (cudaStreamWaitEvent(s, h->done, 0) != cudaSuccess) return HIST_ERR_CUDA;
  }
  return HIST_OK;
}

int fill_impl(hist* h, const double* values, const double* weights, int64_t n, cudaStream_t stream,
              const ExprDev* ex = nullptr) {
  const int acc = (weights == nullptr) ? ACC_UNIT : acc_mode_of(h->flags, false);
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  int rc = order_after_previous(h, stream);
  if (rc != HIST_OK) return rc;
  FillParams p = make_params(h, values, weights, n, acc);
  if (ex != nullptr) {
    p.direct_flush = 0;  // (the Filter/Define kernels keep the reduce)
    p.ex = *ex;
    p.ex.g_passed = h->g_passed;
  }
  LaunchShape shape;
  if (plan_fill(p, acc, h->sm_count, &shape) != 0) return HIST_ERR_CUDA;
  rc = ensure_scratch(h, shape.grid, acc, p.smem_bins != 0);
  if (rc != HIST_OK) return rc;
  p.part_bins = h->part_bins;
  p.part_stats = h->part_stats;
  p.part_sumw2 = h->part_sumw2;  // (re)allocated by ensure_scratch for this grid
  if (p.sumw2 && p.smem_bins && (acc == ACC_FX || acc == ACC_F32C) && p.part_sumw2 == nullptr) return HIST_ERR_CUDA;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (h->timing && !h->capturing) {
    while (h->t_ev.size() < 2 * (h->t_used + 1)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return HIST_ERR_CUDA;
      h->t_ev.push_back(e);
    }
    t0 = h->t_ev[2 * h->t_used];
    t1 = h->t_ev[2 * h->t_used + 1];
    if (cudaEventRecord(t0, stream) != cudaSuccess) return HIST_ERR_CUDA;
  }
  if (launch_fill(p, acc, shape, stream) != 0) return HIST_ERR_CUDA;
  if (h->timing && !h->capturing) {
    if (cudaEventRecord(t1, stream) != cudaSuccess) return HIST_ERR_CUDA;
    ++h->t_used;
  }
  ReduceParams r;
  std::memset(&r, 0, sizeof(r));
  r.part_bins = p.smem_bins ? h->part_bins : nullptr;
  r.part_stats = h->part_stats;
  r.nblocks = p.direct_flush ? 0 : shape.grid;
  r.nstats = h->nstats;
  r.nbins_total = h->nbins_total;
  r.mode = acc;
  r.track_counts = p.track_counts;
  r.g_lo = h->g_lo;
  r.g_hi = h->g_hi;
  r.g_count = h->g_count;
  r.g_unit = h->g_unit;
  r.g_f64 = h->g_f64;
  r.g_stats = h->g_stats;
  const bool sw2_shared = p.sumw2 && p.smem_bins && (acc == ACC_FX || acc == ACC_F32C);
  r.part_sumw2 = sw2_shared ? h->part_sumw2 : nullptr;
  r.g_sumw2 = h->g_sumw2;
  if (!p.direct_flush && launch_reduce(r, stream) != 0) return HIST_ERR_CUDA;
  if (h->d_exact != nullptr) {
    if (ex != nullptr) return HIST_ERR_UNSUPPORTED;
    ExactParams e;
    std::memset(&e, 0, sizeof(e));
    for (int d = 0; d < h->ndim; ++d) {
      e.col[d] = values + (size_t)d * (size_t)n;
      e.lo_key[d] = h->T_host[d][1];
      e.hi_key[d] = h->T_host[d][h->nbins[d] + 1];
    }
    e.w = weights;
    e.n = n;
    e.ndim = h->ndim;
    e.stat_overflows = (h->flags & HIST_STAT_OVERFLOWS) ? 1 : 0;
    for (int k = 0; k < kExactStats; ++k) e.grid[k] = h->exact_grid[k];
    e.limbs = h->d_exact;
    e.escape = h->d_exact + kExactStats * kExactLimbs;
    e.special = reinterpret_cast<unsigned long long*>(h->d_exact + kExactStats * (kExactLimbs + kEscapeLimbs));
    // statistics 1 .. nstats-1, up to kExactGroup per pass over the bulk
    for (e.s0 = 0; e.s0 < h->nstats - 1; e.s0 += kExactGroup) {
      e.ns = std::min(kExactGroup, h->nstats - 1 - e.s0);
      if (launch_stats_exact(e, weights == nullptr, h->sm_count, stream) != 0) return HIST_ERR_CUDA;
    }
    if (++h->exact_launches % 1024 == 0 && launch_exact_normalise(h->d_exact, stream) != 0) return HIST_ERR_CUDA;
  }
  if (acc == ACC_FX && (!p.smem_bins || p.direct_flush)) {
    // each event (global bins) or each block (direct flush) grows g_lo by
    // less than 2^32
    h->fx_global_since_norm += p.smem_bins ? (int64_t)shape.grid : n;
    if (h->fx_global_since_norm > (int64_t)1 << 31) {
      if (launch_normalize_fx(h->g_lo, h->g_hi, h->nbins_total, stream) != 0) return HIST_ERR_CUDA;
      h->fx_global_since_norm = 0;
    }
  }
  // (inside a capture the graph's launch records completion instead)
  if (!h->capturing && cudaEventRecord(h->done, stream) != cudaSuccess) return HIST_ERR_CUDA;
  h->have_done = true;
  if (ex == nullptr) h->n_entries += n;  // filtered fills count their passing events on the device
  if (acc != ACC_UNIT && !(h->flags & HIST_TRACK_COUNTS)) h->counts_complete = false;
  return HIST_OK;
}

// Staging slots, streams and events of the host pipeline, and the fill
// scratch for its bulk sizes (nothing is allocated while it is enqueued,
// which may be inside a graph capture).
int pipeline_prepare(hist* h, int64_t n, int64_t bulk, bool weighted) {
  if (h->copy_stream[0] == nullptr) {
    for (int i = 0; i < 2; ++i)
      if (cudaStreamCreateWithFlags(&h->copy_stream[i], cudaStreamNonBlocking) != cudaSuccess) return HIST_ERR_CUDA;
    if (cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess) return HIST_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreateWithFlags(&h->copied[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->consumed[i], cudaEventDisableTiming) != cudaSuccess)
        return HIST_ERR_CUDA;
  }
  if (bulk > h->stage_events) {  // grow the slots (after their last use)
    if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
      if (cudaStreamSynchronize(h->copy_stream[i]) != cudaSuccess) return HIST_ERR_CUDA;
    for (int i = 0; i < 2; ++i) {
      cudaFree(h->d_stage[i]);
      h->d_stage[i] = nullptr;
      h->slot_used[i] = false;
    }
    h->stage_events = 0;
    if (h->host_exec) {
      cudaGraphExecDestroy(h->host_exec);
      h->host_exec = nullptr;
    }
    for (int i = 0; i < 2; ++i) {
      const int rc = dalloc(&h->d_stage[i], (size_t)bulk * (size_t)(h->ndim + 1) * sizeof(double));
      if (rc != HIST_OK) return rc;
    }
    h->stage_events = bulk;
  }
  const int acc = weighted ? h->acc_mode : ACC_UNIT;
  for (int64_t m : {bulk, n % bulk}) {
    if (m == 0) continue;
    FillParams p = make_params(h, h->d_stage[0], weighted ? h->d_stage[0] : nullptr, m, acc);
    LaunchShape shape;
    if (plan_fill(p, acc, h->sm_count, &shape) != 0) return HIST_ERR_CUDA;
    const int rc = ensure_scratch(h, shape.grid, acc, p.smem_bins != 0);
    if (rc != HIST_OK) return rc;
  }
  return HIST_OK;
}

// Bulk i: copied into slot i % 2 on the copy stream once the fill that last
// read the slot is done, then filled from it on stream s.
int pipeline_enqueue(hist* h, const double* values, const double* weights, int64_t n, int64_t bulk,
                     cudaStream_t s) {
  if (cudaEventRecord(h->fork_ev, s) != cudaSuccess) return HIST_ERR_CUDA;  // after s's earlier work
  for (int i = 0; i < 2; ++i)
    if (cudaStreamWaitEvent(h->copy_stream[i], h->fork_ev, 0) != cudaSuccess) return HIST_ERR_CUDA;
  for (int64_t off = 0, i = 0; off < n; off += bulk, ++i) {
    const int slot = (int)(i & 1);
    const int64_t m = std::min<int64_t>(bulk, n - off);
    double* dst = h->d_stage[slot];
    cudaStream_t cs = h->copy_stream[slot];
    if (i >= 2 && cudaStreamWaitEvent(cs, h->consumed[slot], 0) != cudaSuccess) return HIST_ERR_CUDA;
    for (int d = 0; d < h->ndim; ++d)
      if (cudaMemcpyAsync(dst + (size_t)d * m, values + (size_t)d * n + off, (size_t)m * sizeof(double),
                          cudaMemcpyHostToDevice, cs) != cudaSuccess)
        return HIST_ERR_CUDA;
    if (weights != nullptr &&
        cudaMemcpyAsync(dst + (size_t)h->ndim * m, weights + off, (size_t)m * sizeof(double), cudaMemcpyHostToDevice,
                        cs) != cudaSuccess)
      return HIST_ERR_CUDA;
    if (cudaEventRecord(h->copied[slot], cs) != cudaSuccess) return HIST_ERR_CUDA;
    if (cudaStreamWaitEvent(s, h->copied[slot], 0) != cudaSuccess) return HIST_ERR_CUDA;
    const int rc = fill_impl(h, dst, weights != nullptr ? dst + (size_t)h->ndim * m : nullptr, m, s);
    if (rc != HIST_OK) return rc;
    if (cudaEventRecord(h->consumed[slot], s) != cudaSuccess) return HIST_ERR_CUDA;
    h->slot_used[slot] = true;
  }
  // join both copy streams back into s (a capture must end joined)
  for (int i = 0; i < 2; ++i)
    if (cudaEventRecord(h->copied[i], h->copy_stream[i]) != cudaSuccess ||
        cudaStreamWaitEvent(s, h->copied[i], 0) != cudaSuccess)
      return HIST_ERR_CUDA;
  return HIST_OK;
}

}  // namespace

extern "C" {

const char* hist_version(void) { return "gb300-hist 0.1 (sm_103a)"; }

int hist_locator_mode(const hist_t* h, int axis) {
  if (h == nullptr || axis < 0 || axis >= h->ndim) return HIST_ERR_ARG;
  return h->loc_mode[axis];
}

int hist_set_kernel_timing(hist_t* h, int on) {
  if (h == nullptr) return HIST_ERR_ARG;
  h->timing = on != 0;
  h->t_used = 0;
  return HIST_OK;
}

int hist_kernel_time(hist_t* h, double* ms, int64_t* launches) {
  if (h == nullptr || ms == nullptr || launches == nullptr) return HIST_ERR_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  double total = 0.0;
  for (size_t i = 0; i < h->t_used; ++i) {
    if (cudaEventSynchronize(h->t_ev[2 * i + 1]) != cudaSuccess) return HIST_ERR_CUDA;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, h->t_ev[2 * i], h->t_ev[2 * i + 1]) != cudaSuccess) return HIST_ERR_CUDA;
    total += t;
  }
  *ms = total;
  *launches = (int64_t)h->t_used;
  h->t_used = 0;
  return HIST_OK;
}

const char* hist_strerror(int code) {
  switch (code) {
    case HIST_OK:
      return "ok";
    case HIST_ERR_ARG:
      return "invalid argument";
    case HIST_ERR_AXIS:
      return "invalid axis";
    case HIST_ERR_CUDA:
      return "CUDA runtime error";
    case HIST_ERR_OOM:
      return "out of memory";
    case HIST_ERR_ALIGN:
      return "misaligned pointer";
    case HIST_ERR_TIMEOUT:
      return "device wait timed out";
    case HIST_ERR_LOCATOR:
      return "learned locator unavailable";
    case HIST_ERR_STATE:
      return "invalid state for this call";
    case HIST_ERR_UNSUPPORTED:
      return "unsupported combination";
    case HIST_ERR_TOO_LARGE:
      return "size exceeds the fixed maximum of this entry point";
    default:
      return "unknown status";
  }
}

int hist_book(const hist_axis_t* axes, int ndim, uint32_t flags, hist_t** out) {
  if (out == nullptr || axes == nullptr || ndim < 1 || ndim > kMaxDim) return HIST_ERR_ARG;
  *out = nullptr;
  const uint32_t known =
      HIST_TRACK_COUNTS | HIST_STAT_OVERFLOWS | HIST_SUMW2 | HIST_STATS_EXACT | HIST_PREC_MASK | HIST_LOCATOR_MASK;
  if (flags & ~known) return HIST_ERR_ARG;
  if ((flags & HIST_PREC_MASK) == (3u << 4)) return HIST_ERR_ARG;
  if ((flags & HIST_LOCATOR_MASK) > HIST_LOCATOR_BSEARCH) return HIST_ERR_ARG;
  int64_t total = 1;
  for (int d = 0; d < ndim; ++d) {
    const hist_axis_t& a = axes[d];
    if (validate_axis(a.kind, a.nbins, a.xmin, a.xmax, a.edges) != 0) return HIST_ERR_AXIS;
    total *= (int64_t)a.nbins + 2;
    if (total >= ((int64_t)1 << 31)) return HIST_ERR_AXIS;
  }
  hist* h = new (std::nothrow) hist();
  if (h == nullptr) return HIST_ERR_OOM;
  int rc = HIST_OK;
  do {
    if (cudaGetDevice(&h->device) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    h->ndim = ndim;
    h->nstats = ndim == 1 ? 5 : (ndim == 2 ? 8 : 12);
    h->flags = flags;
    h->nbins_total = total;
    std::vector<int64_t> T;
    std::vector<int32_t> BK;
    for (int d = 0; d < ndim; ++d) {
      const hist_axis_t& a = axes[d];
      h->kind[d] = a.kind;
      h->nbins[d] = a.nbins;
      h->t_off[d] = (int32_t)T.size();
      T.resize(T.size() + (size_t)a.nbins + 3);
      int64_t* Td = T.data() + h->t_off[d];
      if (a.kind == HIST_AXIS_FIXED) {
        build_fixed_thresholds(a.nbins, a.xmin, a.xmax, Td);
        h->loc_mode[d] =
            affine_estimate(a.nbins, a.xmin, a.xmax, &h->scale[d], &h->offset[d], &h->eps[d]) ? LOC_AFFINE
                                                                                              : LOC_BSEARCH;
      } else {
        build_variable_thresholds(a.nbins, a.edges, Td);
        h->loc_mode[d] = LOC_BSEARCH;
        if ((flags & HIST_LOCATOR_MASK) != HIST_LOCATOR_BSEARCH) {
          // a bucket map when one keeps every bucket's thresholds few
          // small axes: 4 buckets per bin and, when no bucket holds two
          // thresholds, the 16-byte pair table (staged in shared memory);
          // large axes: 2 buckets per bin and the 4-byte counts, so that the
          // tables of a batch of large axes stay within L2
          int nbk = 64;
          const bool small = 16LL * 4 * (a.nbins + 1) <= (long long)kSmemBucketBudget;
          while (nbk < (small ? 4 : 2) * (a.nbins + 1) && nbk < kBucketMax) nbk *= 2;
          BucketMap m;
          std::vector<int32_t> cnt;
          const int most = build_bucket_map(a.nbins, Td, nbk, &m, &cnt);
          if (most >= 0 && most <= kBucketMaxRun) {
            h->loc_mode[d] = LOC_BUCKET;
            while (BK.size() % 4) BK.push_back(0);  // 16-byte aligned tables
            h->bk_off[d] = (int32_t)BK.size();
            if (most <= 1 && 16LL * nbk <= (long long)kSmemBucketBudget) {
              // (threshold, cnt) pairs: the bucket's one threshold, or INT64_MAX
              for (int b = 0; b < nbk; ++b) {
                const int64_t thr = cnt[(size_t)b + 1] > cnt[(size_t)b] ? Td[cnt[(size_t)b] + 1]
                                                                       : std::numeric_limits<int64_t>::max();
                const int64_t kk = cnt[(size_t)b];
                int32_t w[4];
                std::memcpy(w, &thr, 8);
                std::memcpy(w + 2, &kk, 8);
                BK.insert(BK.end(), w, w + 4);
              }
            } else {
              BK.insert(BK.end(), cnt.begin(), cnt.end());
            }
            BucketDev& bd = h->bk[d];
            bd.single = (most <= 1 && 16LL * nbk <= (long long)kSmemBucketBudget) ? 1 : 0;
            bd.lo_key = Td[1];
            bd.hi_key = Td[a.nbins + 1];
            bd.nbk = m.nbk;
            bd.key_map = m.key_map;
            bd.scale = m.scale;
            bd.offset = m.offset;
            bd.shift = m.shift;
            bd.kbase = m.kbase;
            bd.top = m.top;
            bd.smem_off = -1;
          }
        }
      }
      h->T_host[d].assign(Td, Td + a.nbins + 3);
    }
    h->table_keys = (int32_t)T.size();
    // stage a prefix of the axes' tables into shared memory
    h->smem_keys = 0;
    for (int d = 0; d < ndim; ++d) {
      const int32_t end = h->t_off[d] + h->nbins[d] + 3;
      if ((size_t)end * 8 <= kSmemTableBudget) h->smem_keys = end;
    }
    // and a prefix of the bucket counts
    h->smem_bk = 0;
    for (int d = 0; d < ndim; ++d)
      if (h->bk_off[d] >= 0 && (size_t)(h->bk_off[d] + bucket_ints(h->bk[d])) * 4 <= kSmemBucketBudget)
        h->smem_bk = h->bk_off[d] + bucket_ints(h->bk[d]);
    if (!BK.empty()) {
      if ((rc = dalloc(&h->d_BK, BK.size() * sizeof(int32_t))) != HIST_OK) break;
      if (cudaMemcpy(h->d_BK, BK.data(), BK.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = HIST_ERR_CUDA;
        break;
      }
      for (int d = 0; d < ndim; ++d)
        if (h->bk_off[d] >= 0) h->bk[d].cnt = h->d_BK + h->bk_off[d];
    }
    rc = dalloc(&h->d_T, T.size() * sizeof(int64_t));
    if (rc != HIST_OK) break;
    if (cudaMemcpy(h->d_T, T.data(), T.size() * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    // weighted fills use the precision mode; unit fills always count
    h->acc_mode = acc_mode_of(flags, false);
    h->smem_unit = (size_t)total * smem_bin_bytes(ACC_UNIT, 0) <= kSmemBinsBudget;
    h->smem_weighted = (size_t)total * smem_bin_bytes(h->acc_mode, (flags & HIST_TRACK_COUNTS) ? 1 : 0,
                                                       (flags & HIST_SUMW2) ? 1 : 0) <=
                       kSmemBinsBudget;
    const size_t nb = (size_t)total;
    if ((rc = dalloc(&h->g_lo, nb * 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->g_hi, nb * 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->g_count, nb * 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->g_unit, nb * 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->g_f64, nb * 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->g_stats, kMaxStats * sizeof(double))) != HIST_OK) break;
    if ((flags & HIST_SUMW2) && (rc = dalloc(&h->g_sumw2, nb * 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->g_passed, 8)) != HIST_OK) break;
    if ((rc = dalloc(&h->d_ticket, 4)) != HIST_OK) break;
    if (cudaMemset(h->d_ticket, 0, 4) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    if (flags & HIST_STATS_EXACT) {
      if ((rc = dalloc(&h->d_exact, kExactBytes)) != HIST_OK) break;
      // grids: the statistic's largest expected term 2^T (|w| < 2^16, each
      // coordinate |c_d| < 2^X_d over its in-range values) sets its
      // 127-binade fast window
      int X[kMaxDim] = {64, 64, 64};
      for (int d = 0; d < ndim; ++d) {
        const double lo = axes[d].kind == HIST_AXIS_FIXED ? axes[d].xmin : axes[d].edges[0];
        const double hi = axes[d].kind == HIST_AXIS_FIXED ? axes[d].xmax : axes[d].edges[axes[d].nbins];
        if (!(flags & HIST_STAT_OVERFLOWS)) {
          int e = 0;
          std::frexp(std::max(std::fabs(lo), std::fabs(hi)), &e);
          X[d] = e;  // |c_d| < 2^e
        }
      }
      const int Wb = 16;
      // w, w^2, wx, wx^2, wy, wy^2, wxy, wz, wz^2, wxz, wyz
      const int T[kExactStats] = {Wb,        2 * Wb,           Wb + X[0],        Wb + 2 * X[0],
                                  Wb + X[1], Wb + 2 * X[1],    Wb + X[0] + X[1], Wb + X[2],
                                  Wb + 2 * X[2], Wb + X[0] + X[2], Wb + X[1] + X[2]};
      for (int k = 0; k < kExactStats; ++k) h->exact_grid[k] = std::max(T[k] - 52 - kExactFastTop, -1074);
    }
    if (cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
  } while (false);
  if (rc == HIST_OK) rc = hist_reset(h);
  if (rc != HIST_OK) {
    free_state(h);
    delete h;
    return rc;
  }
  *out = h;
  return HIST_OK;
}

int hist_reset(hist_t* h) {
  if (h == nullptr) return HIST_ERR_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
  const size_t nb = (size_t)h->nbins_total;
  if (cudaMemset(h->g_lo, 0, nb * 8) != cudaSuccess || cudaMemset(h->g_hi, 0, nb * 8) != cudaSuccess ||
      cudaMemset(h->g_count, 0, nb * 8) != cudaSuccess || cudaMemset(h->g_unit, 0, nb * 8) != cudaSuccess ||
      cudaMemset(h->g_f64, 0, nb * 8) != cudaSuccess ||
      cudaMemset(h->g_stats, 0, kMaxStats * sizeof(double)) != cudaSuccess ||
      (h->g_sumw2 != nullptr && cudaMemset(h->g_sumw2, 0, nb * 8) != cudaSuccess) ||
      cudaMemset(h->g_passed, 0, 8) != cudaSuccess ||
      (h->d_exact != nullptr && cudaMemset(h->d_exact, 0, kExactBytes) != cudaSuccess))
    return HIST_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return HIST_ERR_CUDA;
  h->n_entries = 0;
  h->fx_global_since_norm = 0;
  h->counts_complete = true;
  return HIST_OK;
}

void hist_free(hist_t* h) {
  if (h == nullptr) return;
  cudaSetDevice(h->device);
  if (h->have_done) cudaEventSynchronize(h->done);
  free_state(h);
  delete h;
}

int hist_axis_thresholds(const hist_axis_t* axis, int64_t* out) {
  if (axis == nullptr || out == nullptr) return HIST_ERR_ARG;
  if (validate_axis(axis->kind, axis->nbins, axis->xmin, axis->xmax, axis->edges) != 0) return HIST_ERR_AXIS;
  if (axis->kind == HIST_AXIS_FIXED)
    build_fixed_thresholds(axis->nbins, axis->xmin, axis->xmax, out);
  else
    build_variable_thresholds(axis->nbins, axis->edges, out);
  return HIST_OK;
}

int hist_axis_affine(const hist_axis_t* axis, float* scale, float* offset, float* eps) {
  if (axis == nullptr || scale == nullptr || offset == nullptr || eps == nullptr) return HIST_ERR_ARG;
  if (validate_axis(axis->kind, axis->nbins, axis->xmin, axis->xmax, axis->edges) != 0 ||
      axis->kind != HIST_AXIS_FIXED)
    return HIST_ERR_AXIS;
  return affine_estimate(axis->nbins, axis->xmin, axis->xmax, scale, offset, eps) ? HIST_OK : HIST_ERR_UNSUPPORTED;
}

int64_t hist_nbins_total(const hist_t* h) { return h ? h->nbins_total : -1; }
int hist_nstats(const hist_t* h) { return h ? h->nstats : -1; }
int hist_ndim(const hist_t* h) { return h ? h->ndim : -1; }

int hist_fill_bulk(hist_t* h, const double* values, const double* weights, int64_t n, hist_stream_t stream) {
  if (h == nullptr || n < 0) return HIST_ERR_ARG;
  if (n == 0) return HIST_OK;
  if (values == nullptr) return HIST_ERR_ARG;
  if (!aligned8(values) || (weights != nullptr && !aligned8(weights))) return HIST_ERR_ALIGN;
  return fill_impl(h, values, weights, n, reinterpret_cast<cudaStream_t>(stream));
}

int hist_fill_host(hist_t* h, const double* values, const double* weights, int64_t n, int64_t bulk,
                   hist_stream_t stream) {
  if (h == nullptr || n < 0 || bulk < 0) return HIST_ERR_ARG;
  if (n == 0) return HIST_OK;
  if (values == nullptr) return HIST_ERR_ARG;
  if (bulk == 0) bulk = kDefaultHostBulk;
  if (bulk > n) bulk = n;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = pipeline_prepare(h, n, bulk, weights != nullptr);
  if (rc != HIST_OK) return rc;
  const int acc = weights == nullptr ? ACC_UNIT : h->acc_mode;
  const bool smem = acc == ACC_UNIT ? h->smem_unit : h->smem_weighted;
  // small bulks are launch-bound: replay the whole pipelined fill as one
  // CUDA graph (exact integer bins in shared memory only: the global
  // fixed-point path needs host-side overflow bookkeeping per fill)
  const bool graph = bulk <= kHostGraphBulk && smem && (n + bulk - 1) / bulk <= kHostGraphBulks &&
                     h->d_exact == nullptr;  // exact statistics keep host-side launch counts
  if (!graph) return pipeline_enqueue(h, values, weights, n, bulk, s);
  if (h->host_exec == nullptr || h->g_values != values || h->g_weights != weights || h->g_n != n ||
      h->g_bulk != bulk) {
    if (h->host_exec) {
      cudaGraphExecDestroy(h->host_exec);
      h->host_exec = nullptr;
    }
    if (h->cap_stream == nullptr && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return HIST_ERR_CUDA;
    const int64_t entries = h->n_entries;
    const bool complete = h->counts_complete, had_done = h->have_done;
    if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
    h->capturing = true;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      h->capturing = false;
      return HIST_ERR_CUDA;
    }
    rc = pipeline_enqueue(h, values, weights, n, bulk, h->cap_stream);
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
    h->capturing = false;
    h->n_entries = entries;
    h->counts_complete = complete;
    h->have_done = had_done;
    if (rc != HIST_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != HIST_OK ? rc : HIST_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->host_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->host_exec = nullptr;
      return HIST_ERR_CUDA;
    }
    h->g_values = values;
    h->g_weights = weights;
    h->g_n = n;
    h->g_bulk = bulk;
  }
  if ((rc = order_after_previous(h, s)) != HIST_OK) return rc;
  if (cudaGraphLaunch(h->host_exec, s) != cudaSuccess) return HIST_ERR_CUDA;
  if (cudaEventRecord(h->done, s) != cudaSuccess) return HIST_ERR_CUDA;
  h->have_done = true;
  h->n_entries += n;
  if (acc != ACC_UNIT && !(h->flags & HIST_TRACK_COUNTS)) h->counts_complete = false;
  for (int i = 0; i < 2; ++i) h->slot_used[i] = false;  // the graph orders its own slot reuse
  return HIST_OK;
}

int hist_locate(hist_t* h, const double* values, int64_t n, int64_t* out, hist_stream_t stream) {
  if (h == nullptr || n < 0) return HIST_ERR_ARG;
  if (n == 0) return HIST_OK;
  if (values == nullptr || out == nullptr) return HIST_ERR_ARG;
  if (!aligned8(values) || !aligned8(out)) return HIST_ERR_ALIGN;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  FillParams p = make_params(h, values, nullptr, n, ACC_UNIT);
  if (launch_locate(p, reinterpret_cast<long long*>(out), reinterpret_cast<void*>(stream)) != 0)
    return HIST_ERR_CUDA;
  return HIST_OK;
}

namespace {

// Is linear bin g inside the range on every axis?
bool bin_in_range(const hist* h, int64_t g) {
  for (int d = 0; d < h->ndim; ++d) {
    const int64_t n2 = (int64_t)h->nbins[d] + 2;
    const int64_t k = g % n2;
    g /= n2;
    if (k < 1 || k > h->nbins[d]) return false;
  }
  return true;
}

}  // namespace

int hist_result(hist_t* h, double* bins, double* stats) {
  if (h == nullptr) return HIST_ERR_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
  const size_t nb = (size_t)h->nbins_total;
  std::vector<unsigned long long> lo(nb), unit(nb);
  std::vector<long long> hi(nb);
  std::vector<double> f64(nb);
  if (cudaMemcpy(lo.data(), h->g_lo, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hi.data(), h->g_hi, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(unit.data(), h->g_unit, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(f64.data(), h->g_f64, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return HIST_ERR_CUDA;
  // Bin content = (fixed-point words + unit entries, as one exact integer in
  // units of 2^(fx_elo - 1065)) rounded once to binary64, plus the binary64
  // words (slow-path weights, binary64 mode).
  const int shift = 1065 - h->fx_elo;
  const double lsb = std::ldexp(1.0, -shift);
  const bool all = (h->flags & HIST_STAT_OVERFLOWS) != 0;
  __int128 sel_fx = 0;           // exact sum over the statistics' bins
  double sel_f64 = 0.0, sel_c = 0.0;  // compensated sum of their binary64 words
  unsigned long long sel_unit = 0;
  for (size_t g = 0; g < nb; ++g) {
    const __int128 fx = ((__int128)hi[g] << 32) + (__int128)lo[g] + ((__int128)unit[g] << shift);
    if (bins != nullptr) bins[g] = (double)fx * lsb + f64[g];
    if (all || bin_in_range(h, (int64_t)g)) {
      sel_fx += fx;
      sel_unit += unit[g];
      const double t = sel_f64 + f64[g];
      if (std::isfinite(t))
        sel_c += (std::fabs(sel_f64) >= std::fabs(f64[g])) ? (sel_f64 - t) + f64[g] : (f64[g] - t) + sel_f64;
      sel_f64 = t;
    }
  }
  if (stats != nullptr) {
    double s[kMaxStats];
    if (cudaMemcpy(s, h->g_stats, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return HIST_ERR_CUDA;
    unsigned long long passed = 0;
    if (cudaMemcpy(&passed, h->g_passed, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return HIST_ERR_CUDA;
    s[0] = (double)(h->n_entries + (int64_t)passed);
    // sum w over the statistics' entries = sum of those bins' contents
    s[1] = (double)sel_fx * lsb + (sel_f64 + sel_c);
    // unit-weight entries add 1 each to sum w^2
    s[2] += (double)sel_unit;
    if (h->d_exact != nullptr) {  // the exact sums of the rounded terms, rounded once
      std::vector<long long> ex(kExactBytes / 8);
      if (cudaMemcpy(ex.data(), h->d_exact, kExactBytes, cudaMemcpyDeviceToHost) != cudaSuccess) return HIST_ERR_CUDA;
      const long long* limbs = ex.data();
      const long long* esc = limbs + kExactStats * kExactLimbs;
      const unsigned long long* sp =
          reinterpret_cast<const unsigned long long*>(esc + kExactStats * kEscapeLimbs);
      for (int k = 0; k < h->nstats - 1; ++k)
        s[1 + k] = exact_round(limbs + k * kExactLimbs, h->exact_grid[k], esc + k * kEscapeLimbs, sp + 3 * k);
    }
    for (int k = 0; k < h->nstats; ++k) stats[k] = s[k];
  }
  return HIST_OK;
}

int hist_counts(hist_t* h, uint64_t* counts) {
  if (h == nullptr || counts == nullptr) return HIST_ERR_ARG;
  if (!h->counts_complete) return HIST_ERR_STATE;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
  const size_t nb = (size_t)h->nbins_total;
  std::vector<unsigned long long> unit(nb);
  if (cudaMemcpy(counts, h->g_count, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(unit.data(), h->g_unit, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return HIST_ERR_CUDA;
  for (size_t g = 0; g < nb; ++g) counts[g] += unit[g];
  return HIST_OK;
}

int hist_fill_columns(hist_t* h, const double* const* cols, int ncols, const hist_define_t* defines,
                      const hist_filter_t* filters, int nfilters, const double* weights, int64_t n,
                      hist_stream_t stream) {
  if (h == nullptr || n < 0 || ncols < 1 || ncols > kExprMaxSrc || cols == nullptr || defines == nullptr ||
      nfilters < 0 || nfilters > kExprMaxFilters || (nfilters > 0 && filters == nullptr))
    return HIST_ERR_ARG;
  if (h->ndim > 2 || (h->flags & (HIST_SUMW2 | HIST_STATS_EXACT))) return HIST_ERR_UNSUPPORTED;
  ExprDev ex;
  std::memset(&ex, 0, sizeof(ex));
  ex.nsrc = ncols;
  for (int c = 0; c < ncols; ++c) {
    if (n > 0 && cols[c] == nullptr) return HIST_ERR_ARG;
    if (!aligned8(cols[c])) return HIST_ERR_ALIGN;
    ex.src[c] = cols[c];
  }
  if (weights != nullptr && !aligned8(weights)) return HIST_ERR_ALIGN;
  for (int d = 0; d < h->ndim; ++d) {
    const hist_define_t& df = defines[d];
    if (df.op < HIST_DEF_COL || df.op > HIST_DEF_SUB || df.a < 0 || df.a >= ncols ||
        (df.op != HIST_DEF_COL && (df.b < 0 || df.b >= ncols)))
      return HIST_ERR_ARG;
    ex.def_op[d] = df.op;
    ex.def_a[d] = df.a;
    ex.def_b[d] = df.op == HIST_DEF_COL ? df.a : df.b;
  }
  ex.nfilt = nfilters;
  for (int k = 0; k < nfilters; ++k) {
    if (filters[k].col < 0 || filters[k].col >= ncols || filters[k].op < HIST_FLT_NE || filters[k].op > HIST_FLT_GE)
      return HIST_ERR_ARG;
    ex.filt_col[k] = filters[k].col;
    ex.filt_op[k] = filters[k].op;
    ex.filt_val[k] = filters[k].value;
  }
  if (n == 0) return HIST_OK;
  return fill_impl(h, cols[0], weights, n, reinterpret_cast<cudaStream_t>(stream), &ex);
}

int hist_sumw2(hist_t* h, double* sumw2) {
  if (h == nullptr || sumw2 == nullptr) return HIST_ERR_ARG;
  if (!(h->flags & HIST_SUMW2)) return HIST_ERR_STATE;
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
  const size_t nb = (size_t)h->nbins_total;
  std::vector<unsigned long long> unit(nb);
  if (cudaMemcpy(sumw2, h->g_sumw2, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(unit.data(), h->g_unit, nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return HIST_ERR_CUDA;
  for (size_t g = 0; g < nb; ++g) sumw2[g] += (double)unit[g];  // unit weights: w^2 = 1 per entry
  return HIST_OK;
}

}  // extern "C"

namespace {

// FP32 value of a binary64 truncated to 24 significant bits (as the device's
// est_float: saturating to +-0 and +-2^127 outside the FP32 range).
float host_trunc24(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned e = (hi >> 20) & 0x7FFu;
  unsigned f = ((unsigned)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu;
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7F000000u : f;
  f |= hi & 0x80000000u;
  float r;
  std::memcpy(&r, &f, 4);
  return r;
}

// Largest k with T[k] <= key (host binary search over the thresholds).
int host_bin_of_key(const std::vector<int64_t>& T, int64_t key) {
  int lo = 0, hi = (int)T.size() - 2;  // answer in [0, nbins+1]
  while (lo < hi) {
    const int mid = lo + (hi - lo + 1) / 2;
    if (T[mid] <= key)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <class T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() { cudaFree(p); }
  int alloc(size_t count) { return dalloc(&p, count * sizeof(T)); }
};

int lm_certify(const LearnedDev& m, const long long* dT, int nbins, int* d_err, int* window) {
  if (cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) return HIST_ERR_CUDA;
  if (launch_lm_certify(m, dT, nbins, d_err, nullptr) != 0) return HIST_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HIST_ERR_CUDA;
  *window = err;  // the largest error over every non-NaN coordinate (see learned.cu)
  return HIST_OK;
}

}  // namespace

extern "C" int hist_locator_loss_grad(int nseg, float u0, float u_scale, const int32_t* base, const float* theta,
                                      const double* x, const float* target, int64_t n, double* loss, float* grad) {
  if (nseg < 1 || base == nullptr || theta == nullptr || x == nullptr || target == nullptr || n < 1 ||
      loss == nullptr || grad == nullptr)
    return HIST_ERR_ARG;
  DevBuf<int> d_base;
  DevBuf<float> d_theta, d_target, d_grad;
  DevBuf<unsigned long long> d_x;
  DevBuf<double> d_loss;
  int rc;
  if ((rc = d_base.alloc(nseg + 1)) || (rc = d_theta.alloc(nseg + 1)) || (rc = d_grad.alloc(nseg + 1)) ||
      (rc = d_target.alloc(n)) || (rc = d_x.alloc(n)) || (rc = d_loss.alloc(1)))
    return rc;
  if (cudaMemcpy(d_base.p, base, sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_theta.p, theta, sizeof(float) * (nseg + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_x.p, x, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_target.p, target, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d_grad.p, 0, sizeof(float) * (nseg + 1)) != cudaSuccess ||
      cudaMemset(d_loss.p, 0, sizeof(double)) != cudaSuccess)
    return HIST_ERR_CUDA;
  if (launch_lm_fwd_bwd(u0, u_scale, nseg, d_base.p, d_theta.p, d_x.p, d_target.p, n, d_grad.p, d_loss.p, nullptr) != 0)
    return HIST_ERR_CUDA;
  if (cudaMemcpy(grad, d_grad.p, sizeof(float) * (nseg + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(loss, d_loss.p, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HIST_ERR_CUDA;
  return HIST_OK;
}

extern "C" int hist_train_locator(hist_t* h, int axis, const hist_locator_opts_t* opts, hist_locator_report_t* report) {
  if (h == nullptr || axis < 0 || axis >= h->ndim || h->kind[axis] != HIST_AXIS_VARIABLE) return HIST_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  if (cudaSetDevice(h->device) != cudaSuccess) return HIST_ERR_CUDA;
  if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
  const int nb = h->nbins[axis];
  const std::vector<int64_t>& T = h->T_host[axis];
  auto edge = [&](int j) { return host_double_of_key(T[j + 1]); };  // e_j, j = 0..nb
  int S = opts && opts->segments > 0 ? opts->segments : 16;
  if (!(opts && opts->segments > 0))
    while (S < (1 << 20) && S * 8 < nb) S <<= 1;
  if (S < 1 || S > (1 << 22)) return HIST_ERR_ARG;
  const int steps = opts && opts->steps > 0 ? opts->steps : 400;
  const float lr = opts && opts->lr > 0.0f ? opts->lr : 0.05f;
  const float u0 = host_trunc24(edge(0));
  const float un = host_trunc24(edge(nb));
  if (!(un > u0)) return HIST_ERR_LOCATOR;
  const float u_scale = (float)((double)S / ((double)un - (double)u0));
  if (!std::isfinite(u_scale) || !(u_scale > 0.0f)) return HIST_ERR_LOCATOR;
  // knots: exact bin at the knot position, residual = the fractional index
  // there (the untrained model interpolates the in-bin position linearly)
  std::vector<int> base(S + 1);
  std::vector<float> theta(S + 1);
  for (int j = 0; j <= S; ++j) {
    const double xj = (double)u0 + (double)j / (double)u_scale;
    const int k = host_bin_of_key(T, host_key(xj));
    base[j] = k;
    double frac = 0.0;
    if (k >= 1 && k <= nb) frac = (xj - edge(k - 1)) / (edge(k) - edge(k - 1)) - 0.5;
    else if (k == 0) frac = 0.5;
    else frac = -0.5;
    theta[j] = (float)frac;
  }
  // training pairs from the exact binning
  const long long ns = 2LL * nb;
  std::vector<unsigned long long> xs(ns);
  std::vector<float> ys(ns);
  for (int j = 1; j <= nb; ++j) {
    const double a = edge(j - 1), b = edge(j);
    const double mid = a + 0.5 * (b - a);
    std::memcpy(&xs[2 * (j - 1)], &a, 8);
    std::memcpy(&xs[2 * (j - 1) + 1], &mid, 8);
    ys[2 * (j - 1)] = (float)j - 0.5f;
    ys[2 * (j - 1) + 1] = (float)j;
  }
  DevBuf<int> d_base, d_err;
  DevBuf<float> d_theta, d_m1, d_m2, d_grad, d_y;
  DevBuf<unsigned long long> d_x;
  DevBuf<double> d_loss;
  int2* d_knots = nullptr;
  int rc;
  if ((rc = d_base.alloc(S + 1)) || (rc = d_theta.alloc(S + 1)) || (rc = d_m1.alloc(S + 1)) ||
      (rc = d_m2.alloc(S + 1)) || (rc = d_grad.alloc(S + 1)) || (rc = d_y.alloc(ns)) || (rc = d_x.alloc(ns)) ||
      (rc = d_loss.alloc(1)) || (rc = d_err.alloc(1)) || (rc = dalloc(&d_knots, sizeof(int2) * (S + 1))))
    return rc;
  auto fail = [&](int code) {
    cudaFree(d_knots);
    return code;
  };
  if (cudaMemcpy(d_base.p, base.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_theta.p, theta.data(), sizeof(float) * (S + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_x.p, xs.data(), 8 * ns, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_y.p, ys.data(), 4 * ns, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d_m1.p, 0, sizeof(float) * (S + 1)) != cudaSuccess ||
      cudaMemset(d_m2.p, 0, sizeof(float) * (S + 1)) != cudaSuccess)
    return fail(HIST_ERR_CUDA);
  const long long* dT = h->d_T + h->t_off[axis];
  LearnedDev m;
  m.knots = d_knots;
  m.u0 = u0;
  m.u_scale = u_scale;
  m.nseg = S;
  m.window = 0;
  auto loss_pass = [&](double* out) -> int {
    if (cudaMemset(d_grad.p, 0, sizeof(float) * (S + 1)) != cudaSuccess ||
        cudaMemset(d_loss.p, 0, sizeof(double)) != cudaSuccess)
      return HIST_ERR_CUDA;
    if (launch_lm_fwd_bwd(u0, u_scale, S, d_base.p, d_theta.p, d_x.p, d_y.p, ns, d_grad.p, d_loss.p, nullptr) != 0)
      return HIST_ERR_CUDA;
    if (out && cudaMemcpy(out, d_loss.p, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return HIST_ERR_CUDA;
    return HIST_OK;
  };
  double loss0 = 0.0, loss1 = 0.0;
  int w0 = 0, w1 = 0;
  if ((rc = loss_pass(&loss0)) != HIST_OK) return fail(rc);
  if (launch_lm_pack(d_base.p, d_theta.p, d_knots, S + 1, nullptr) != 0) return fail(HIST_ERR_CUDA);
  if ((rc = lm_certify(m, dT, nb, d_err.p, &w0)) != HIST_OK) return fail(rc);
  for (int it = 1; it <= steps; ++it) {
    if ((rc = loss_pass(nullptr)) != HIST_OK) return fail(rc);
    if (launch_lm_adam(d_theta.p, d_m1.p, d_m2.p, d_grad.p, S + 1, lr, 0.9f, 0.999f, 1e-12f, it, nullptr) != 0)
      return fail(HIST_ERR_CUDA);
  }
  if ((rc = loss_pass(&loss1)) != HIST_OK) return fail(rc);
  if (launch_lm_pack(d_base.p, d_theta.p, d_knots, S + 1, nullptr) != 0) return fail(HIST_ERR_CUDA);
  if ((rc = lm_certify(m, dT, nb, d_err.p, &w1)) != HIST_OK) return fail(rc);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(HIST_ERR_CUDA);
  if (report) {
    report->segments = S;
    report->steps = steps;
    report->window_untrained = w0;
    report->window = w1;
    report->loss_untrained = loss0;
    report->loss = loss1;
    report->train_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (opts && opts->apply) {
    cudaFree(h->lm_knots[axis]);
    h->lm_knots[axis] = d_knots;
    m.window = w1;
    h->lm[axis] = m;
    h->loc_mode[axis] = LOC_LEARNED;
    ++h->config_version;
    return HIST_OK;
  }
  return fail(HIST_OK);
}

// ============================================================== batches ====

// The partitioned strategy's plan for one column: its members (contiguous
// in batch order), its ranges and their staged tables on the device.
struct PartPlan {
  int col = 0, h0 = 0, nh = 0;  // the column and its members [h0, h0 + nh)
  int nranges = 0, max_keys = 0, max_bins = 0, max_nbk = 0, row = 8, count_grid = 0, fill_per_sm = 0;
  size_t smem = 0;              // the fill kernel's dynamic shared memory
  long long* d_splits = nullptr;
  PartRangeDev* d_ranges = nullptr;
  PartSliceDev* d_slices = nullptr;
  long long* d_keys = nullptr;
  unsigned short* d_cum = nullptr;
  unsigned short* d_bcnt = nullptr;
  unsigned short* d_sbcnt = nullptr;  // the split keys' bucket counts
  PartRangeDev split_map{};           // ... and their bucket map
  int items = 0, block_base = 0;  // the fill's grid and first statistics partial (set per event count)
  void release() {
    cudaFree(d_splits);
    cudaFree(d_ranges);
    cudaFree(d_slices);
    cudaFree(d_keys);
    cudaFree(d_cum);
    cudaFree(d_bcnt);
    cudaFree(d_sbcnt);
    d_bcnt = nullptr;
    d_sbcnt = nullptr;
    d_splits = nullptr;
    d_ranges = nullptr;
    d_slices = nullptr;
    d_keys = nullptr;
    d_cum = nullptr;
  }
};

struct hist_batch {
  std::vector<hist*> hs;     // member histograms, sorted by column
  std::vector<int> col;      // column of each (sorted order)
  int ncols = 0;             // columns referenced (max column + 1)
  int device = 0, sm_count = 0;
  uint32_t flags = 0;
  bool f32c = false;         // every member booked HIST_PREC_FP32C: the FP32 compensated wide kernel
  int col_begin[kBatchMaxCols + 1] = {};
  BatchStatsSpec st = {};     // statistics groups and the cores of the columns
  int group_col[kBatchMaxGroups] = {};
  std::vector<int> group;    // statistics group of each member
  // staged threshold tables
  long long* d_T = nullptr;
  int table_keys = 0;
  std::vector<int> t_off;    // offset of each member's table in d_T, -1 = not staged
  // descriptors
  BatchHistDev* d_desc = nullptr;
  BatchHistDev* d_desc_tune = nullptr;
  int* d_group = nullptr;
  int* d_col = nullptr;
  double** d_stats = nullptr;
  double** d_stats_tune = nullptr;
  std::vector<int> built_versions;
  // tuning scratch accumulators (one block of memory per member)
  std::vector<void*> scratch;
  double* d_part_stats = nullptr;
  int part_blocks = 0;
  // configuration
  int smem_budget = 96 * 1024;
  int grid = 0;
  size_t smem = 0;
  std::vector<int> sbin_off;
  int sbin_words = 0;
  cudaEvent_t done = nullptr;  // completion of the batch's last fill or tuning run
  bool have_done = false;
  // strategy: 0 wide (batch.cu), 1 sliced (batch_slices.cu)
  int strategy = 0;
  // sliced plan
  std::vector<SliceDev> slices;
  std::vector<SliceFragDev> frags;        // pointers filled at upload
  std::vector<int> frag_member;           // member of each fragment
  std::vector<int64_t> slice_keys;
  int max_frags = 0, max_keys = 0, max_words = 0;
  size_t own_bytes = 0;                   // largest slice's own keys, bins and fragments
  int shared_frags = 0, shared_keys = 0, shared_words = 0;
  int shared_col_begin[kBatchMaxCols + 1] = {};
  int slice_replicas = 1, slice_window = 0;
  int pace_tiles = -1;                    // pacing window in tiles: -1 default, 0 off
  int wide_minb = 2, wide_kev = 4;        // wide: blocks per SM compiled for, events per thread
  bool placed_unit = false;               // wide: shared bins placed at one word per bin (unit fills only)
  double slice_cap = 0.0;
  SliceDev* d_slices = nullptr;
  SliceFragDev* d_frags = nullptr;
  SliceFragDev* d_frags_tune = nullptr;
  long long* d_slice_keys = nullptr;
  int* d_done = nullptr;
  long long done_cap = 0;
  size_t slices_cap = 0, frags_cap = 0, keys_cap = 0;
  // partitioned plan (strategy 2; batch_partition.cu): one per column
  std::vector<PartPlan> plans;
  double* d_px = nullptr;            // the partitioned column and weights (capacity part_n_cap events)
  double* d_pw = nullptr;
  long long part_n_cap = 0, part_w_cap = 0;
  unsigned* d_counts = nullptr;
  unsigned long long* d_offsets = nullptr;
  unsigned long long* d_rscan = nullptr;  // [2][kPartMaxRanges] range totals and starts, then item bases
  size_t counts_cap = 0;
  PartItem* d_items = nullptr;
  int* d_nitems = nullptr;
  int items_cap = 0;
  // graph cache
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const double*> g_cols;
  const double* g_w = nullptr;
  int64_t g_n = -1;
};

namespace {

constexpr int kBatchTableKeys = 2048;  // threshold keys staged per block (24 KB with high words)

void batch_release(hist_batch* b) {
  if (b->have_done) cudaEventSynchronize(b->done);
  if (b->done) cudaEventDestroy(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->d_T);
  cudaFree(b->d_desc);
  cudaFree(b->d_desc_tune);
  cudaFree(b->d_group);
  cudaFree(b->d_col);
  cudaFree(b->d_stats);
  cudaFree(b->d_stats_tune);
  cudaFree(b->d_part_stats);
  cudaFree(b->d_slices);
  cudaFree(b->d_frags);
  cudaFree(b->d_frags_tune);
  cudaFree(b->d_slice_keys);
  cudaFree(b->d_done);
  for (PartPlan& q : b->plans) q.release();
  cudaFree(b->d_px);
  cudaFree(b->d_pw);
  cudaFree(b->d_counts);
  cudaFree(b->d_offsets);
  cudaFree(b->d_rscan);
  cudaFree(b->d_items);
  cudaFree(b->d_nitems);
  for (void* q : b->scratch) cudaFree(q);
}

// Which members keep block-private bins in shared memory under a budget:
// the smallest first (two words per bin, enough for unit and weighted fills).
void batch_place(hist_batch* b, int budget) {
  const int nh = (int)b->hs.size();
  std::vector<int> order(nh);
  for (int i = 0; i < nh; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->hs[x]->nbins[0] < b->hs[y]->nbins[0]; });
  b->sbin_off.assign(nh, -1);
  int words = 0;
  for (int i : order) {  // one word per bin suffices for unit weights, two for fixed-point sums
    const int need = (b->placed_unit ? 1 : 2) * (b->hs[i]->nbins[0] + 2);
    if ((long long)(words + need) * 4 > budget) break;
    b->sbin_off[i] = words;
    words += need;
  }
  b->sbin_words = words;
  b->smem_budget = budget;
}

size_t batch_smem_bytes(const hist_batch* b) {
  return (((size_t)b->table_keys * 12 + 15) & ~(size_t)15) + (((size_t)b->sbin_words * 4 + 15) & ~(size_t)15) +
         sizeof(BatchHistDev) * b->hs.size();
}

// Upload descriptors for the current placement and locators; `tune` points
// the accumulators at the scratch copies instead of the histograms'.
int batch_upload(hist_batch* b) {
  if (b->have_done && cudaEventSynchronize(b->done) != cudaSuccess) return HIST_ERR_CUDA;
  const int nh = (int)b->hs.size();
  std::vector<BatchHistDev> real(nh), tune(nh);
  std::vector<double*> st(nh), st_tune(nh);
  for (int i = 0; i < nh; ++i) {
    hist* h = b->hs[i];
    BatchHistDev d;
    std::memset(&d, 0, sizeof(d));
    d.ax.T = h->d_T + h->t_off[0];
    d.ax.nbins = h->nbins[0];
    d.ax.mode = h->loc_mode[0];
    d.ax.smem_off = b->t_off[i];
    d.ax.scale = h->scale[0];
    d.ax.offset = h->offset[0];
    d.ax.eps = h->eps[0];
    d.ax.lm = h->lm[0];
    d.ax.bk = h->bk[0];
    d.ax.bk.smem_off = -1;
    d.col = b->col[i];
    d.group = b->group[i];
    d.sbin_off = b->sbin_off[i];
    d.g_lo = h->g_lo;
    d.g_hi = h->g_hi;
    d.g_unit = h->g_unit;
    d.g_f64 = h->g_f64;
    real[i] = d;
    unsigned char* sc = static_cast<unsigned char*>(b->scratch[i]);
    const size_t nbb = (size_t)(h->nbins[0] + 2) * 8;
    d.g_lo = reinterpret_cast<unsigned long long*>(sc);
    d.g_hi = reinterpret_cast<long long*>(sc + nbb);
    d.g_unit = reinterpret_cast<unsigned long long*>(sc + 2 * nbb);
    d.g_f64 = reinterpret_cast<double*>(sc + 3 * nbb);
    tune[i] = d;
    st[i] = h->g_stats;
    st_tune[i] = reinterpret_cast<double*>(sc + 4 * nbb);
  }
  if (cudaMemcpy(b->d_desc, real.data(), sizeof(BatchHistDev) * nh, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_desc_tune, tune.data(), sizeof(BatchHistDev) * nh, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_stats, st.data(), sizeof(double*) * nh, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_stats_tune, st_tune.data(), sizeof(double*) * nh, cudaMemcpyHostToDevice) != cudaSuccess)
    return HIST_ERR_CUDA;
  b->built_versions.resize(nh);
  for (int i = 0; i < nh; ++i) b->built_versions[i] = b->hs[i]->config_version;
  if (b->exec) {  // descriptors are baked into a captured graph only by pointer; contents changed is fine
  }
  return HIST_OK;
}

// ---- sliced strategy: planning (see batch_slices.cu) ----
constexpr double kSliceTestCost = 0.15;  // key range test of a split fragment, in units of one locate + add
constexpr double kSliceEventCost = 0.5;  // loading and converting one event, per slice
constexpr double kSliceStatCost = 0.3;   // one statistics group
constexpr long long kSliceMinFragBins = 64;
constexpr int kSliceBlock = 512, kSliceTile = 2048;
constexpr int kSliceDefaultBudget = 96 * 1024;
constexpr double kSliceDefaultCap = 3.0;
constexpr int kSliceDefaultWindow = 512;  // tiles of 2048 events: 32 MB of four columns

SliceFragDev slice_frag(const hist* h, long long a, long long m) {
  SliceFragDev d;
  std::memset(&d, 0, sizeof(d));
  d.ax.T = h->d_T + h->t_off[0];
  d.ax.nbins = h->nbins[0];
  d.ax.mode = h->loc_mode[0];
  d.ax.smem_off = -1;
  d.ax.scale = h->scale[0];
  d.ax.offset = h->offset[0];
  d.ax.eps = h->eps[0];
  d.ax.lm = h->lm[0];
  d.ax.bk = h->bk[0];
  d.ax.bk.smem_off = -1;
  d.a = (int)a;
  d.b = (int)(a + m);
  d.Ta = h->T_host[0][a];
  d.Tb = h->T_host[0][a + m];
  d.whole = (a == 0 && m == h->nbins[0] + 2) ? 1 : 0;
  return d;
}

// Stage the fragment's keys (non-affine axes) and reserve its bins.
bool slice_own_locator(const hist* h) { return h->loc_mode[0] != LOC_BSEARCH; }

void slice_place(const hist* h, SliceFragDev& d, std::vector<int64_t>& keys, int* nkeys, int* nwords) {
  d.bin_off = *nwords;
  *nwords += 2 * (d.b - d.a);
  if (slice_own_locator(h)) {  // the histogram's own locator; no staged keys
    d.key_off = -1;
    d.top = 0;
    return;
  }
  d.key_off = *nkeys;
  const int nint = d.b - d.a - 1;
  for (int k = d.a + 1; k < d.b; ++k) keys.push_back(h->T_host[0][k]);
  *nkeys += nint;
  int top = nint > 0 ? 1 : 0;
  while (nint > 0 && top * 2 <= nint) top *= 2;
  d.top = top;
}

// The plan: the smallest members (up to `shared_cap` bytes) are held whole
// by every block; the others are cut into slices of at most `budget` bytes
// (with the shared part) and about `cap` units of per-event work, a whole
// histogram costing one unit and a fragment its range test plus its share
// of the bins.
void slice_plan(hist_batch* b, int budget, double cap) {
  b->slices.clear();
  b->frags.clear();
  b->frag_member.clear();
  b->slice_keys.clear();
  const long long desc = (long long)sizeof(SliceFragDev);
  const int nh = (int)b->hs.size();
  auto bytes_of = [&](int i) {
    const hist* h = b->hs[i];
    return (long long)(h->nbins[0] + 2) * (slice_own_locator(h) ? 8 : 16) + desc;
  };
  // shared members: smallest first, up to half the budget
  std::vector<int> order(nh);
  for (int i = 0; i < nh; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->hs[x]->nbins[0] < b->hs[y]->nbins[0]; });
  std::vector<char> shared(nh, 0);
  long long used = 0;
  for (int i : order) {
    if (used + bytes_of(i) > budget / 2) break;
    shared[i] = 1;
    used += bytes_of(i);
  }
  int nkeys = 0, nwords = 0;
  for (int c = 0; c <= kBatchMaxCols; ++c) b->shared_col_begin[c] = 0;
  for (int c = 0; c < kBatchMaxCols; ++c) {
    b->shared_col_begin[c] = (int)b->frags.size();
    for (int i = b->col_begin[c]; i < b->col_begin[c + 1]; ++i) {
      if (!shared[i]) continue;
      SliceFragDev d = slice_frag(b->hs[i], 0, b->hs[i]->nbins[0] + 2);
      slice_place(b->hs[i], d, b->slice_keys, &nkeys, &nwords);
      b->frags.push_back(d);
      b->frag_member.push_back(i);
    }
  }
  b->shared_col_begin[kBatchMaxCols] = (int)b->frags.size();
  b->shared_frags = (int)b->frags.size();
  b->shared_keys = nkeys;
  b->shared_words = nwords;
  const long long room_all = (long long)budget - used;
  // slices of the other members, column by column, smallest first
  for (int c = 0; c < b->ncols; ++c) {
    std::vector<int> mem;
    for (int i = b->col_begin[c]; i < b->col_begin[c + 1]; ++i)
      if (!shared[i]) mem.push_back(i);
    std::stable_sort(mem.begin(), mem.end(), [&](int x, int y) { return b->hs[x]->nbins[0] < b->hs[y]->nbins[0]; });
    SliceDev cur;
    std::memset(&cur, 0, sizeof(cur));
    bool open = false;
    double cost = 0.0;
    long long bytes = 0;
    auto open_slice = [&]() {
      std::memset(&cur, 0, sizeof(cur));
      cur.col = c;
      cur.frag_begin = cur.frag_end = (int)b->frags.size();
      cur.key_base = (int)b->slice_keys.size();
      cost = kSliceEventCost;
      bytes = 0;
      open = true;
    };
    auto close_slice = [&]() {
      if (open && cur.frag_end > cur.frag_begin) b->slices.push_back(cur);
      open = false;
    };
    for (int i : mem) {
      const hist* h = b->hs[i];
      const long long nbt = h->nbins[0] + 2;
      const long long per_bin = slice_own_locator(h) ? 8 : 16;
      long long a = 0;
      while (a < nbt) {
        if (!open) open_slice();
        const bool fresh = cur.frag_end == cur.frag_begin;
        const long long rest = nbt - a;
        const long long by_bytes = std::max(0LL, (room_all - bytes - desc) / per_bin);
        const double room = cap - cost;
        long long m;
        if (a == 0 && rest <= by_bytes && room >= 1.0)
          m = rest;
        else
          m = std::min(std::min(rest, by_bytes), (long long)std::max(0.0, (room - kSliceTestCost) * (double)nbt));
        if (fresh)
          m = std::max(m, std::min(rest, std::max(1LL, by_bytes)));
        else if (m < std::min(rest, kSliceMinFragBins)) {
          close_slice();
          continue;
        }
        SliceFragDev d = slice_frag(h, a, m);
        int nk = cur.nkeys, nw = cur.nwords;
        slice_place(h, d, b->slice_keys, &nk, &nw);
        cur.nkeys = nk;
        cur.nwords = nw;
        b->frags.push_back(d);
        b->frag_member.push_back(i);
        cur.frag_end = (int)b->frags.size();
        cost += d.whole ? 1.0 : kSliceTestCost + (double)m / (double)nbt;
        bytes += per_bin * m + desc;
        a += m;
      }
    }
    close_slice();
  }
  if (b->slices.empty()) {  // everything is shared: one slice without fragments of its own
    SliceDev d;
    std::memset(&d, 0, sizeof(d));
    d.col = b->col[0];
    d.frag_begin = d.frag_end = (int)b->frags.size();
    d.key_base = (int)b->slice_keys.size();
    b->slices.push_back(d);
  }
  b->max_frags = b->max_keys = b->max_words = 0;
  b->own_bytes = 0;
  for (const SliceDev& sd : b->slices) {
    b->max_frags = std::max(b->max_frags, sd.frag_end - sd.frag_begin);
    b->max_keys = std::max(b->max_keys, sd.nkeys);
    b->max_words = std::max(b->max_words, sd.nwords);
    b->own_bytes = std::max(b->own_bytes, slice_smem_bytes(sd.nkeys, sd.nwords, sd.frag_end - sd.frag_begin));
  }
  b->slice_cap = cap;
}

// Upload the slice plan with the accumulators of the members (and of their
// tuning scratch).
int slice_upload(hist_batch* b) {
  if (b->have_done && cudaEventSynchronize(b->done) != cudaSuccess) return HIST_ERR_CUDA;
  const size_t nf = b->frags.size();
  std::vector<SliceFragDev> real(b->frags), tune(b->frags);
  for (size_t f = 0; f < nf; ++f) {
    const int i = b->frag_member[f];
    hist* h = b->hs[i];
    real[f].g_lo = h->g_lo;
    real[f].g_hi = h->g_hi;
    real[f].g_unit = h->g_unit;
    real[f].g_f64 = h->g_f64;
    real[f].ax.T = h->d_T + h->t_off[0];
    real[f].ax.lm = h->lm[0];
    tune[f].ax = real[f].ax;
    unsigned char* sc = static_cast<unsigned char*>(b->scratch[i]);
    const size_t nbb = (size_t)(h->nbins[0] + 2) * 8;
    tune[f].g_lo = reinterpret_cast<unsigned long long*>(sc);
    tune[f].g_hi = reinterpret_cast<long long*>(sc + nbb);
    tune[f].g_unit = reinterpret_cast<unsigned long long*>(sc + 2 * nbb);
    tune[f].g_f64 = reinterpret_cast<double*>(sc + 3 * nbb);
  }
  // grow the device copies only when the plan outgrows them (a captured
  // graph holds these pointers and is dropped when they move)
  if (b->slices.size() > b->slices_cap || nf > b->frags_cap || b->slice_keys.size() > b->keys_cap) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaFree(b->d_slices);
    cudaFree(b->d_frags);
    cudaFree(b->d_frags_tune);
    cudaFree(b->d_slice_keys);
    b->d_slices = nullptr;
    b->d_frags = b->d_frags_tune = nullptr;
    b->d_slice_keys = nullptr;
    b->slices_cap = b->frags_cap = b->keys_cap = 0;
    const size_t ns = std::max(b->slices.size(), (size_t)64), nfc = std::max(nf, (size_t)128);
    const size_t nk = std::max(b->slice_keys.size(), (size_t)1);
    int rc;
    if ((rc = dalloc(&b->d_slices, sizeof(SliceDev) * ns)) != HIST_OK) return rc;
    if ((rc = dalloc(&b->d_frags, sizeof(SliceFragDev) * nfc)) != HIST_OK) return rc;
    if ((rc = dalloc(&b->d_frags_tune, sizeof(SliceFragDev) * nfc)) != HIST_OK) return rc;
    if ((rc = dalloc(&b->d_slice_keys, nk * 8)) != HIST_OK) return rc;
    b->slices_cap = ns;
    b->frags_cap = nfc;
    b->keys_cap = nk;
  }
  if (cudaMemcpy(b->d_slices, b->slices.data(), sizeof(SliceDev) * b->slices.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_frags, real.data(), sizeof(SliceFragDev) * nf, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_frags_tune, tune.data(), sizeof(SliceFragDev) * nf, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!b->slice_keys.empty() && cudaMemcpy(b->d_slice_keys, b->slice_keys.data(), b->slice_keys.size() * 8,
                                            cudaMemcpyHostToDevice) != cudaSuccess))
    return HIST_ERR_CUDA;
  return HIST_OK;
}

int batch_part_stats(hist_batch* b) {
  if (b->grid <= b->part_blocks) return HIST_OK;
  cudaFree(b->d_part_stats);
  b->d_part_stats = nullptr;
  b->part_blocks = 0;
  int rc = dalloc(&b->d_part_stats, (size_t)b->grid * kStatSlots * 3 * sizeof(double));
  if (rc != HIST_OK) return rc;
  b->part_blocks = b->grid;
  return HIST_OK;
}

int slice_configure(hist_batch* b, int budget, double cap) {
  if (b->f32c) return HIST_ERR_UNSUPPORTED;  // the sliced kernel keeps exact fixed-point bins only
  int maxopt = 0;
  if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess)
    return HIST_ERR_CUDA;
  const int limit = maxopt - 10 * 1024;  // the kernel's static arrays
  if (budget > limit - 256) budget = limit - 256;
  slice_plan(b, budget, cap);
  if (b->slices.empty()) return HIST_ERR_UNSUPPORTED;
  b->smem = slice_smem_bytes(b->shared_keys, b->shared_words, b->shared_frags) + b->own_bytes;
  if (b->smem > (size_t)limit) return HIST_ERR_UNSUPPORTED;
  int per_sm = 0;
  if (slice_max_blocks_per_sm(kSliceBlock, b->smem, &per_sm) != 0 || per_sm < 1) return HIST_ERR_CUDA;
  const int resident = per_sm * b->sm_count;
  const int ns = (int)b->slices.size();
  b->slice_replicas = std::max(1, resident / ns);
  b->grid = ns * b->slice_replicas;
  b->slice_window = b->pace_tiles < 0 ? std::max(4 * b->slice_replicas, kSliceDefaultWindow)
                                      : (b->pace_tiles == 0 ? 0 : std::max(4 * b->slice_replicas, b->pace_tiles));
  b->smem_budget = budget;
  b->strategy = 1;
  int rc = batch_part_stats(b);
  if (rc != HIST_OK) return rc;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return slice_upload(b);
}

int batch_configure(hist_batch* b, int budget) {
  // the bins' budget is what remains of the per-block shared memory after
  // the staged tables and the descriptors (and the kernel's static arrays)
  int maxopt = 0;
  if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess)
    return HIST_ERR_CUDA;
  const size_t fixed = (((size_t)b->table_keys * 12 + 15) & ~(size_t)15) + sizeof(BatchHistDev) * b->hs.size() + 16 +
                       8 * 1024;
  if ((size_t)maxopt <= fixed) return HIST_ERR_UNSUPPORTED;
  if ((size_t)budget > (size_t)maxopt - fixed) budget = (int)((size_t)maxopt - fixed);
  batch_place(b, budget);
  b->smem = batch_smem_bytes(b);
  int per_sm = 0;
  if (batch_max_blocks_per_sm(256, b->smem, b->wide_minb, b->wide_kev, &per_sm) != 0 || per_sm < 1)
    return HIST_ERR_CUDA;
  b->grid = per_sm * b->sm_count;
  b->strategy = 0;
  int rc = batch_part_stats(b);
  if (rc != HIST_OK) return rc;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return batch_upload(b);
}

// ---- partitioned strategy: planning (see batch_partition.cu) ----
constexpr int kPartChunkMax = 1 << 19;  // events per fill work item at most
constexpr int kPartCopySlots = 32;      // bin slots a slice may take with its copies (one bank each)
constexpr int kPartChunkMin = 1 << 14;  // ... and at least (below: the staging dominates)
constexpr int kPartWaves = 6;           // work items aimed at per resident fill block

// Bin of a key on a member's thresholds (the largest k with T[k] <= key).
int host_bin(const std::vector<int64_t>& T, long long key) {
  return (int)(std::upper_bound(T.begin(), T.end(), (int64_t)key) - T.begin()) - 1;
}

// The bucket map of M sorted distinct keys (the axes' bucket map, built on
// the pseudo-axis [-inf, keys..., +inf] with a power of two >= M buckets):
// its fields in R, its counts appended to bcnt (R.bk_base their first).
int part_bucket_map(const std::vector<long long>& keys, PartRangeDev* R, std::vector<uint16_t>* bcnt) {
  const int M = (int)keys.size();
  R->lo_key = M > 0 ? keys.front() : std::numeric_limits<long long>::max();
  R->hi_key = M > 0 ? keys.back() : std::numeric_limits<long long>::max();
  R->kbase = 0;
  R->scale = R->offset = 0.0f;
  R->bk_base = (int32_t)bcnt->size();
  R->nbk = R->key_map = R->shift = R->top = R->pad = 0;
  if (M < 2) return 0;
  int nbk = 4;
  while (nbk < M) nbk *= 2;
  std::vector<int64_t> T(1, std::numeric_limits<int64_t>::min());
  T.insert(T.end(), keys.begin(), keys.end());
  T.push_back(std::numeric_limits<int64_t>::max());
  BucketMap map;
  std::vector<int32_t> bc;
  if (build_bucket_map(M - 1, T.data(), nbk, &map, &bc) < 0) return -1;
  R->kbase = map.kbase;
  R->scale = map.scale;
  R->offset = map.offset;
  R->nbk = map.nbk;
  R->key_map = map.key_map;
  R->shift = map.shift;
  R->top = map.top;
  for (int q = 0; q <= nbk; ++q) bcnt->push_back((uint16_t)bc[(size_t)q]);
  return nbk;
}

// Plan one column's members [h0, h0 + nh): cut the column's key space into
// ranges that fit `budget` bytes of shared memory.  Every member's thresholds
// are sorted together; a range takes thresholds until the next would pass
// its capacity C, and the next range starts at that threshold (a range's
// first threshold is a slice boundary, not one of its interior thresholds).
// A range costs, per interior threshold, one bin slot of 8 bytes (12 in an
// FP32C batch: three FP32 words), one merged key
// of 8 bytes, one count row of 2 row bytes and at most two bucket counts of
// 2 bytes, plus per member 16 bytes of descriptor, one more bin and up to
// copy_slots - 1 bin copies (a slice keeps 2^rsh <= 32 copies of each bin,
// as many as fit copy_slots slots, so that a warp's adds spread over the
// banks; copy_slots is kPartCopySlots, halved while the copies would take
// more than half the budget).  Each
// range gets the axes' bucket map (build_bucket_map) over its merged
// thresholds, with a power of two >= M buckets.  On success the plan's
// tables are on the device.
int part_plan_column(const hist_batch* b, int col, int h0, int nh, int budget, int limit, PartPlan* out) {
  if (nh < 1 || nh > kPartMaxMembers) return HIST_ERR_UNSUPPORTED;
  const int row = 8 * ((nh + 7) / 8);
  // bin copies may take up to half the budget
  const int slot_bytes = b->f32c ? 12 : 8;  // FP32C: three FP32 words per slot
  int copy_slots = kPartCopySlots;
  while (copy_slots > 1 && (16LL + (long long)slot_bytes * (copy_slots + 1)) * nh > budget / 2) copy_slots /= 2;
  const long long C = ((long long)budget - (16LL + (long long)slot_bytes * (copy_slots + 1)) * nh - 2LL * row - 48) /
                      (12 + slot_bytes + 2 * row);
  if (C < 16) return HIST_ERR_UNSUPPORTED;
  std::vector<long long> all;
  for (int h = h0; h < h0 + nh; ++h) {
    const hist* m = b->hs[(size_t)h];
    for (int k = 1; k <= m->nbins[0] + 1; ++k) all.push_back(m->T_host[0][k]);
  }
  std::sort(all.begin(), all.end());
  std::vector<long long> splits;
  long long acc = 0;
  for (size_t i = 0; i < all.size();) {
    size_t j = i;
    while (j < all.size() && all[j] == all[i]) ++j;
    const long long m = (long long)(j - i);
    if (acc > 0 && acc + m > C) {
      splits.push_back(all[i]);  // starts a range: its thresholds bound the slices there
      acc = 0;
    } else {
      acc += m;
    }
    i = j;
  }
  const int nranges = (int)splits.size() + 1;
  if (nranges > kPartMaxRanges) return HIST_ERR_UNSUPPORTED;
  std::vector<PartRangeDev> ranges(nranges);
  std::vector<PartSliceDev> slices((size_t)nranges * nh);
  std::vector<long long> keys;
  std::vector<uint16_t> cum, bcnt;
  int max_keys = 0, max_bins = 0, max_nbk = 0;
  std::vector<long long> merged;
  std::vector<int> a(nh), e(nh);
  for (int r = 0; r < nranges; ++r) {
    const long long lo = r == 0 ? std::numeric_limits<long long>::min() : splits[(size_t)r - 1];
    const long long hi_m1 = r + 1 < nranges ? splits[(size_t)r] - 1 : std::numeric_limits<long long>::max() - 1;
    PartRangeDev& R = ranges[(size_t)r];
    // the members' slices and their interior thresholds, merged and distinct
    merged.clear();
    int nb = 0;
    for (int h = 0; h < nh; ++h) {
      const std::vector<int64_t>& T = b->hs[(size_t)(h0 + h)]->T_host[0];
      a[h] = host_bin(T, lo);
      e[h] = host_bin(T, hi_m1);
      PartSliceDev& S = slices[(size_t)r * nh + h];
      S.a = a[h];
      S.len = e[h] - a[h] + 1;
      S.boff = nb;
      S.rsh = 0;
      while (S.rsh < 5 && (S.len << (S.rsh + 1)) <= copy_slots) ++S.rsh;
      nb += S.len << S.rsh;
      for (int k = a[h] + 1; k <= e[h]; ++k) merged.push_back(T[(size_t)k]);
    }
    std::sort(merged.begin(), merged.end());
    merged.erase(std::unique(merged.begin(), merged.end()), merged.end());
    const int M = (int)merged.size();
    R.key_base = (int32_t)keys.size();
    R.nkeys = M;
    R.nbins = nb;
    R.cum_base = (int32_t)cum.size();
    keys.insert(keys.end(), merged.begin(), merged.end());
    // row p: each member's count of its interior thresholds <= merged[p - 1]
    const size_t row0 = cum.size();
    cum.resize(row0 + (size_t)(M + 1) * row, 0);
    for (int h = 0; h < nh; ++h) {
      const std::vector<int64_t>& T = b->hs[(size_t)(h0 + h)]->T_host[0];
      const int rsh = slices[(size_t)r * nh + h].rsh;
      int k = a[h] + 1, c = 0;
      for (int q = 1; q <= M; ++q) {
        while (k <= e[h] && T[(size_t)k] <= merged[(size_t)q - 1]) {
          ++k;
          ++c;
        }
        cum[row0 + (size_t)q * row + h] = (uint16_t)(c << rsh);
      }
    }
    // the bucket map of the merged thresholds
    const int nbk = part_bucket_map(merged, &R, &bcnt);
    if (nbk < 0) return HIST_ERR_UNSUPPORTED;
    max_nbk = std::max(max_nbk, nbk);
    max_keys = std::max(max_keys, M);
    max_bins = std::max(max_bins, nb);
  }
  if (keys.size() > (size_t)std::numeric_limits<int32_t>::max() ||
      cum.size() > (size_t)std::numeric_limits<int32_t>::max() ||
      bcnt.size() > (size_t)std::numeric_limits<int32_t>::max())
    return HIST_ERR_UNSUPPORTED;
  const size_t fill_smem = part_fill_smem(max_keys, max_bins, nh, row, max_nbk, slot_bytes);
  if (fill_smem > (size_t)limit) return HIST_ERR_UNSUPPORTED;
  PartPlan q;
  q.col = col;
  q.h0 = h0;
  q.nh = nh;
  q.nranges = nranges;
  q.max_keys = max_keys;
  q.max_bins = max_bins;
  q.max_nbk = max_nbk;
  q.row = row;
  q.smem = fill_smem;
  // the split keys' bucket map (the count and scatter passes' locate)
  std::vector<uint16_t> sbcnt;
  if (part_bucket_map(splits, &q.split_map, &sbcnt) < 0) return HIST_ERR_UNSUPPORTED;
  q.split_map.nkeys = (int32_t)splits.size();
  if (part_grids(b->sm_count, nranges, q.split_map.nbk, fill_smem, &q.count_grid, &q.fill_per_sm) != 0)
    return HIST_ERR_CUDA;
  int rc;
  if ((rc = dalloc(&q.d_splits, std::max<size_t>(splits.size(), 1) * 8)) != HIST_OK ||
      (rc = dalloc(&q.d_ranges, sizeof(PartRangeDev) * ranges.size())) != HIST_OK ||
      (rc = dalloc(&q.d_slices, sizeof(PartSliceDev) * slices.size())) != HIST_OK ||
      (rc = dalloc(&q.d_keys, std::max<size_t>(keys.size(), 1) * 8)) != HIST_OK ||
      (rc = dalloc(&q.d_cum, cum.size() * 2)) != HIST_OK ||
      (rc = dalloc(&q.d_bcnt, std::max<size_t>(bcnt.size(), 8) * 2)) != HIST_OK ||
      (rc = dalloc(&q.d_sbcnt, std::max<size_t>(sbcnt.size(), 8) * 2)) != HIST_OK) {
    q.release();
    return rc;
  }
  if ((!splits.empty() &&
       cudaMemcpy(q.d_splits, splits.data(), splits.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(q.d_ranges, ranges.data(), sizeof(PartRangeDev) * ranges.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(q.d_slices, slices.data(), sizeof(PartSliceDev) * slices.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (!keys.empty() && cudaMemcpy(q.d_keys, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(q.d_cum, cum.data(), cum.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!bcnt.empty() && cudaMemcpy(q.d_bcnt, bcnt.data(), bcnt.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) ||
      (!sbcnt.empty() &&
       cudaMemcpy(q.d_sbcnt, sbcnt.data(), sbcnt.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)) {
    q.release();
    return HIST_ERR_CUDA;
  }
  *out = q;
  return HIST_OK;
}

// The partitioned strategy: one plan per column (every column at most
// kPartMaxMembers members); exact or FP32 compensated bins.
int part_configure(hist_batch* b, int budget) {
  int maxopt = 0;
  if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess)
    return HIST_ERR_CUDA;
  const int limit = maxopt - 10 * 1024;  // the fill kernel's static arrays
  if (budget > limit) budget = limit;
  for (int c = 0; c < b->ncols; ++c)
    if (b->col_begin[c + 1] - b->col_begin[c] > kPartMaxMembers) return HIST_ERR_UNSUPPORTED;
  std::vector<PartPlan> plans;
  int rc = HIST_OK;
  for (int c = 0; c < b->ncols && rc == HIST_OK; ++c) {
    const int h0 = b->col_begin[c], nh = b->col_begin[c + 1] - h0;
    if (nh == 0) continue;
    PartPlan q;
    rc = part_plan_column(b, c, h0, nh, budget, limit, &q);
    if (rc == HIST_OK) plans.push_back(q);
  }
  if (rc != HIST_OK) {
    for (PartPlan& q : plans) q.release();
    return rc;
  }
  for (PartPlan& q : b->plans) q.release();
  b->plans.swap(plans);
  // the counts of the count and scatter passes, one per (range, block),
  // shared by the plans (their fills run one after the other)
  size_t nc = 0, smem = 0;
  for (const PartPlan& q : b->plans) {
    nc = std::max(nc, (size_t)q.nranges * q.count_grid);
    smem = std::max(smem, q.smem);
  }
  if (nc > b->counts_cap) {
    cudaFree(b->d_counts);
    cudaFree(b->d_offsets);
    b->d_counts = nullptr;
    b->d_offsets = nullptr;
    b->counts_cap = 0;
    if ((rc = dalloc(&b->d_counts, nc * 4)) != HIST_OK || (rc = dalloc(&b->d_offsets, nc * 8)) != HIST_OK) return rc;
    b->counts_cap = nc;
  }
  if (b->d_nitems == nullptr && (rc = dalloc(&b->d_nitems, 16)) != HIST_OK) return rc;
  if (b->d_rscan == nullptr && (rc = dalloc(&b->d_rscan, (size_t)kPartMaxRanges * 20)) != HIST_OK) return rc;
  b->smem = smem;
  b->smem_budget = budget;
  b->strategy = 2;
  b->grid = 0;  // the fills' grids depend on the events: batch_reserve
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return HIST_OK;
}

// Events per work item for a fill of n events: about kPartWaves items per
// resident fill block (so the last wave is short), within the bounds above.
int part_chunk(const PartPlan& q, int sm_count, int64_t n) {
  const long long target = (long long)kPartWaves * std::max(1, q.fill_per_sm) * sm_count;
  long long c = (n + target - 1) / target;
  c = std::max<long long>(kPartChunkMin, std::min<long long>(kPartChunkMax, c));
  return (int)c;
}

// Work items of a fill of n events, at most (each range's events in runs of
// at most one chunk).
int part_items(const PartPlan& q, int sm_count, int64_t n) {
  const int chunk = part_chunk(q, sm_count, n);
  return q.nranges + (int)((n + chunk - 1) / chunk) + 1;
}

int batch_check_args(const hist_batch* b, const double* const* cols, int ncols, const double* weights, int64_t n) {
  if (cols == nullptr || n < 0 || ncols < b->ncols) return HIST_ERR_ARG;
  for (int c = 0; c < b->ncols; ++c) {
    if (n > 0 && cols[c] == nullptr) return HIST_ERR_ARG;
    if (((uintptr_t)cols[c]) & 7u) return HIST_ERR_ALIGN;
  }
  if (((uintptr_t)weights) & 7u) return HIST_ERR_ALIGN;
  return HIST_OK;
}

BatchParams batch_params(const hist_batch* b, const double* const* cols, const double* weights, int64_t n,
                         bool tune) {
  BatchParams p;
  std::memset(&p, 0, sizeof(p));
  for (int c = 0; c < b->ncols; ++c) p.col[c] = cols[c];
  p.w = weights;
  p.hists = tune ? b->d_desc_tune : b->d_desc;
  p.T_concat = b->d_T;
  p.part_stats = b->d_part_stats;
  p.n = n;
  p.ncols = b->ncols;
  p.nh = (int)b->hs.size();
  p.fx_elo = kDefaultFxElo;
  p.table_keys = b->table_keys;
  p.sbin_words = b->sbin_words;
  p.aligned = 1;
  for (int c = 0; c <= kBatchMaxCols; ++c) p.col_begin[c] = b->col_begin[c];
  p.st = b->st;
  return p;
}

// Scratch of a fill of n events (before any capture): the sliced strategy's
// pacing counters; the partitioned strategy's copy of the column (and of the
// weights, for weighted fills), work items and statistics partials.
int batch_reserve(hist_batch* b, int64_t n, bool weighted) {
  if (b->strategy == 2) {
    int rc;
    const long long cap = std::max<long long>(n, 1);
    if (cap > b->part_n_cap) {
      cudaFree(b->d_px);
      b->d_px = nullptr;
      b->part_n_cap = 0;
      if ((rc = dalloc(&b->d_px, (size_t)cap * 8)) != HIST_OK) return rc;
      b->part_n_cap = cap;
    }
    if (weighted && cap > b->part_w_cap) {
      cudaFree(b->d_pw);
      b->d_pw = nullptr;
      b->part_w_cap = 0;
      if ((rc = dalloc(&b->d_pw, (size_t)cap * 8)) != HIST_OK) return rc;
      b->part_w_cap = cap;
    }
    // each column's fill: its work items and its blocks' statistics
    // partials (after the previous columns')
    int total = 0, most = 0;
    bool changed = false;
    for (PartPlan& q : b->plans) {
      const int items = part_items(q, b->sm_count, n);
      changed = changed || items != q.items || total != q.block_base;
      q.items = items;
      q.block_base = total;
      total += items;
      most = std::max(most, items);
    }
    if (most > b->items_cap) {
      cudaFree(b->d_items);
      b->d_items = nullptr;
      b->items_cap = 0;
      if ((rc = dalloc(&b->d_items, sizeof(PartItem) * (size_t)most)) != HIST_OK) return rc;
      b->items_cap = most;
    }
    if ((changed || total != b->grid) && b->exec) {  // a captured fill launched other grids
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    b->grid = total;
    return batch_part_stats(b);
  }
  if (b->strategy != 1) return HIST_OK;
  const long long nt = (n + kSliceTile - 1) / kSliceTile;
  if (nt <= b->done_cap) return HIST_OK;
  cudaFree(b->d_done);
  b->d_done = nullptr;
  b->done_cap = 0;
  const int rc = dalloc(&b->d_done, (size_t)nt * sizeof(int));
  if (rc != HIST_OK) return rc;
  b->done_cap = nt;
  return HIST_OK;
}

int batch_launch(const hist_batch* b, const double* const* cols, const double* weights, int64_t n, bool tune,
                 cudaStream_t s) {
  if (b->strategy == 2) {
    if ((weights != nullptr && b->part_w_cap < n) || b->part_n_cap < n) return HIST_ERR_CUDA;
    // one column after the other: they share the partitioned copy, the
    // counts and the work items
    for (const PartPlan& q : b->plans) {
      PartParams p;
      std::memset(&p, 0, sizeof(p));
      p.col = cols[q.col];
      p.w = weights;
      p.px = b->d_px;
      p.pw = weights != nullptr ? b->d_pw : nullptr;
      p.splits = q.d_splits;
      p.ranges = q.d_ranges;
      p.slices = q.d_slices;
      p.keys = q.d_keys;
      p.cum = q.d_cum;
      p.bcnt = q.d_bcnt;
      p.sbcnt = q.d_sbcnt;
      p.split_map = q.split_map;
      p.row_u16 = q.row;
      p.hists = (tune ? b->d_desc_tune : b->d_desc) + q.h0;
      p.counts = b->d_counts;
      p.offsets = b->d_offsets;
      p.rtotal = b->d_rscan;
      p.rstart = b->d_rscan + kPartMaxRanges;
      p.ibase = reinterpret_cast<int*>(b->d_rscan + 2 * kPartMaxRanges);
      p.items = b->d_items;
      p.nitems = b->d_nitems;
      p.part_stats = b->d_part_stats + (size_t)q.block_base * kStatSlots * 3;
      p.n = n;
      p.nranges = q.nranges;
      p.nh = q.nh;
      p.grid_count = q.count_grid;
      p.fx_elo = kDefaultFxElo;
      p.chunk = part_chunk(q, b->sm_count, n);
      p.max_items = q.items;
      p.max_keys = q.max_keys;
      p.max_bins = q.max_bins;
      p.max_nbk = q.max_nbk;
      p.stat_col = q.col;
      p.st = b->st;
      if (q.items != part_items(q, b->sm_count, n) || q.items > b->items_cap ||
          (size_t)q.nranges * q.count_grid > b->counts_cap || q.block_base + q.items > b->part_blocks)
        return HIST_ERR_CUDA;  // batch_reserve sized the scratch for these events
      if (launch_part_fill(p, weights == nullptr, b->f32c, q.items, q.smem, s) != 0) return HIST_ERR_CUDA;
    }
  } else if (b->strategy == 1) {
    SliceParams p;
    std::memset(&p, 0, sizeof(p));
    for (int c = 0; c < b->ncols; ++c) p.col[c] = cols[c];
    p.w = weights;
    p.slices = b->d_slices;
    p.frags = tune ? b->d_frags_tune : b->d_frags;
    p.keys = b->d_slice_keys;
    p.part_stats = b->d_part_stats;
    p.n = n;
    p.ntiles = (n + kSliceTile - 1) / kSliceTile;
    p.nslices = (int)b->slices.size();
    p.replicas = b->slice_replicas;
    p.tile = kSliceTile;
    p.window = b->slice_window;
    p.done = (p.window > 0 && p.ntiles <= b->done_cap) ? b->d_done : nullptr;
    if (p.done == nullptr) p.window = 0;
    p.ncols = b->ncols;
    p.shared_frags = b->shared_frags;
    for (int c = 0; c <= kBatchMaxCols; ++c) p.shared_col_begin[c] = b->shared_col_begin[c];
    p.shared_keys = b->shared_keys;
    p.shared_words = b->shared_words;
    p.max_frags = b->max_frags;
    p.max_keys = b->max_keys;
    p.max_words = b->max_words;
    p.fx_elo = kDefaultFxElo;
    p.st = b->st;
    if (p.done != nullptr && cudaMemsetAsync(p.done, 0, (size_t)p.ntiles * sizeof(int), s) != cudaSuccess)
      return HIST_ERR_CUDA;
    if (launch_slice_fill(p, kSliceBlock, b->grid, b->smem, s) != 0) return HIST_ERR_CUDA;
  } else {
    const BatchParams p = batch_params(b, cols, weights, n, tune);
    if (launch_batch_fill(p, 256, b->grid, b->smem, b->wide_minb, b->wide_kev, b->f32c, s) != 0) return HIST_ERR_CUDA;
  }
  BatchReduceParams r;
  std::memset(&r, 0, sizeof(r));
  r.part_stats = b->d_part_stats;
  r.nblocks = b->grid;
  r.nh = (int)b->hs.size();
  r.hist_col = b->d_col;
  r.hist_group = b->d_group;
  r.hist_stats = tune ? b->d_stats_tune : b->d_stats;
  if (launch_batch_reduce(r, s) != 0) return HIST_ERR_CUDA;
  return HIST_OK;
}

}  // namespace

extern "C" int hist_batch_create(hist_t* const* hists, int nh, const int32_t* col_of_hist, uint32_t flags,
                                 hist_batch_t** out) {
  if (out == nullptr || hists == nullptr || col_of_hist == nullptr || nh < 1 || nh > 128) return HIST_ERR_ARG;
  if (flags & ~(HIST_BATCH_GRAPH | HIST_BATCH_WIDE | HIST_BATCH_SLICED)) return HIST_ERR_ARG;
  if ((flags & HIST_BATCH_WIDE) && (flags & HIST_BATCH_SLICED)) return HIST_ERR_ARG;
  *out = nullptr;
  const uint32_t stat_flag = hists[0] ? (hists[0]->flags & HIST_STAT_OVERFLOWS) : 0;
  int n_f32c = 0;
  for (int i = 0; i < nh; ++i) {
    if (hists[i] == nullptr || col_of_hist[i] < 0 || col_of_hist[i] >= kBatchMaxCols) return HIST_ERR_ARG;
    n_f32c += hists[i]->acc_mode == ACC_F32C ? 1 : 0;
    if (hists[i]->ndim != 1) return HIST_ERR_UNSUPPORTED;
    if (hists[i]->flags & (HIST_SUMW2 | HIST_STATS_EXACT)) return HIST_ERR_UNSUPPORTED;
    if (hists[i]->device != hists[0]->device) return HIST_ERR_ARG;
    if ((hists[i]->flags & HIST_STAT_OVERFLOWS) != stat_flag) return HIST_ERR_UNSUPPORTED;
    for (int j = 0; j < i; ++j)
      if (hists[j] == hists[i]) return HIST_ERR_ARG;
  }
  // one precision per batch: every member FP32 compensated, or none
  if (n_f32c != 0 && n_f32c != nh) return HIST_ERR_UNSUPPORTED;
  if (n_f32c == nh && (flags & HIST_BATCH_SLICED)) return HIST_ERR_UNSUPPORTED;
  hist_batch* b = new (std::nothrow) hist_batch();
  if (b == nullptr) return HIST_ERR_OOM;
  int rc = HIST_OK;
  do {
    b->flags = flags;
    b->f32c = n_f32c == nh;
    b->device = hists[0]->device;
    b->sm_count = hists[0]->sm_count;
    if (cudaSetDevice(b->device) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    std::vector<int> order(nh);
    for (int i = 0; i < nh; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return col_of_hist[x] < col_of_hist[y]; });
    for (int i : order) {
      b->hs.push_back(hists[i]);
      b->col.push_back(col_of_hist[i]);
    }
    b->ncols = b->col.back() + 1;
    for (int c = 0; c <= kBatchMaxCols; ++c) {
      int k = 0;
      while (k < nh && b->col[k] < c) ++k;
      b->col_begin[c] = k;
    }
    // statistics groups: distinct (column, range) pairs, in column order;
    // with HIST_STAT_OVERFLOWS every event counts, so one group per column
    b->group.assign(nh, 0);
    int ngroups = 0;
    for (int c = 0; c <= kBatchMaxCols; ++c) b->st.group_begin[c] = 0;
    for (int i = 0; i < nh && rc == HIST_OK; ++i) {
      const hist* h = b->hs[i];
      long long lo = h->T_host[0][1], hi = h->T_host[0][h->nbins[0] + 1];
      if (stat_flag) {
        lo = std::numeric_limits<long long>::min();
        hi = std::numeric_limits<long long>::max();
      }
      const int c = b->col[i];
      int found = -1;
      for (int g = 0; g < ngroups; ++g)
        if (b->group_col[g] == c && b->st.group_lo[g] == lo && b->st.group_hi[g] == hi) found = g;
      if (found < 0) {
        if (ngroups >= kBatchMaxGroups) {
          rc = HIST_ERR_UNSUPPORTED;
          break;
        }
        found = ngroups++;
        b->group_col[found] = c;
        b->st.group_lo[found] = lo;
        b->st.group_hi[found] = hi;
      }
      b->group[i] = found;
    }
    if (rc != HIST_OK) break;
    // members are sorted by column, so their groups are too
    for (int c = 0; c < kBatchMaxCols; ++c) {
      int g0 = 0;
      while (g0 < ngroups && b->group_col[g0] < c) ++g0;
      int g1 = g0;
      while (g1 < ngroups && b->group_col[g1] == c) ++g1;
      b->st.group_begin[c] = g0;
      b->st.group_begin[c + 1] = g1;
      long long lo = std::numeric_limits<long long>::max(), hi = std::numeric_limits<long long>::min();
      if (g1 > g0) {
        lo = std::numeric_limits<long long>::min();
        hi = std::numeric_limits<long long>::max();
        for (int g = g0; g < g1; ++g) {
          lo = std::max(lo, b->st.group_lo[g]);
          hi = std::min(hi, b->st.group_hi[g]);
        }
      }
      b->st.core_lo[c] = lo;
      b->st.core_hi[c] = hi;
    }
    if (rc != HIST_OK) break;
    // stage the smallest search tables
    b->t_off.assign(nh, -1);
    std::vector<int> by_size(nh);
    for (int i = 0; i < nh; ++i) by_size[i] = i;
    std::stable_sort(by_size.begin(), by_size.end(), [&](int x, int y) { return b->hs[x]->nbins[0] < b->hs[y]->nbins[0]; });
    std::vector<int64_t> T;
    for (int i : by_size) {
      const std::vector<int64_t>& Th = b->hs[i]->T_host[0];
      if (T.size() + Th.size() > (size_t)kBatchTableKeys) continue;
      b->t_off[i] = (int)T.size();
      T.insert(T.end(), Th.begin(), Th.end());
    }
    b->table_keys = (int)T.size();
    if ((rc = dalloc(&b->d_T, std::max<size_t>(T.size(), 1) * 8)) != HIST_OK) break;
    if (!T.empty() && cudaMemcpy(b->d_T, T.data(), T.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    if ((rc = dalloc(&b->d_desc, sizeof(BatchHistDev) * nh)) != HIST_OK) break;
    if ((rc = dalloc(&b->d_desc_tune, sizeof(BatchHistDev) * nh)) != HIST_OK) break;
    if ((rc = dalloc(&b->d_group, sizeof(int) * nh)) != HIST_OK) break;
    if ((rc = dalloc(&b->d_stats, sizeof(double*) * nh)) != HIST_OK) break;
    if ((rc = dalloc(&b->d_stats_tune, sizeof(double*) * nh)) != HIST_OK) break;
    if ((rc = dalloc(&b->d_col, sizeof(int) * nh)) != HIST_OK) break;
    if (cudaMemcpy(b->d_group, b->group.data(), sizeof(int) * nh, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_col, b->col.data(), sizeof(int) * nh, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    for (int i = 0; i < nh && rc == HIST_OK; ++i) {
      void* q = nullptr;
      rc = dalloc(&q, (size_t)(b->hs[i]->nbins[0] + 2) * 32 + kMaxStats * sizeof(double));
      if (rc == HIST_OK) b->scratch.push_back(q);
    }
    if (rc != HIST_OK) break;
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    if ((rc = batch_configure(b, 96 * 1024)) != HIST_OK) break;
    bool all_shared = true;
    for (int o : b->sbin_off) all_shared &= o >= 0;
    if (!b->f32c && ((flags & HIST_BATCH_SLICED) || (!all_shared && !(flags & HIST_BATCH_WIDE))))
      rc = slice_configure(b, kSliceDefaultBudget, kSliceDefaultCap);
  } while (false);
  if (rc != HIST_OK) {
    batch_release(b);
    delete b;
    return rc;
  }
  *out = b;
  return HIST_OK;
}

extern "C" void hist_batch_free(hist_batch_t* b) {
  if (b == nullptr) return;
  cudaSetDevice(b->device);
  batch_release(b);  // waits for the batch's own last work; never touches the member histograms
  delete b;
}

extern "C" int hist_batch_fill(hist_batch_t* b, const double* const* cols, int ncols, const double* weights,
                               int64_t n, hist_stream_t stream) {
  if (b == nullptr) return HIST_ERR_ARG;
  int rc = batch_check_args(b, cols, ncols, weights, n);
  if (rc != HIST_OK || n == 0) return rc;
  if (cudaSetDevice(b->device) != cudaSuccess) return HIST_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (b->hs[i]->config_version != b->built_versions[i]) {
      if ((rc = batch_upload(b)) != HIST_OK) return rc;
      if (b->strategy == 1 && (rc = slice_upload(b)) != HIST_OK) return rc;
      break;
    }
  if (weights != nullptr && b->placed_unit && b->strategy == 0) {  // bins placed for unit fills only
    b->placed_unit = false;
    if ((rc = batch_configure(b, b->smem_budget)) != HIST_OK) return rc;
  }
  for (hist* h : b->hs)
    if ((rc = order_after_previous(h, s)) != HIST_OK) return rc;
  if ((rc = batch_reserve(b, n, weights != nullptr)) != HIST_OK) return rc;
  if (b->flags & HIST_BATCH_GRAPH) {
    std::vector<const double*> cv(cols, cols + b->ncols);
    if (b->exec == nullptr || cv != b->g_cols || weights != b->g_w || n != b->g_n) {
      if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HIST_ERR_CUDA;
      rc = batch_launch(b, cols, weights, n, false, b->cap_stream);
      if (cudaStreamEndCapture(b->cap_stream, &graph) != cudaSuccess || rc != HIST_OK) {
        if (graph) cudaGraphDestroy(graph);
        return HIST_ERR_CUDA;
      }
      const cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        b->exec = nullptr;
        return HIST_ERR_CUDA;
      }
      b->g_cols = cv;
      b->g_w = weights;
      b->g_n = n;
    }
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return HIST_ERR_CUDA;
  } else {
    if ((rc = batch_launch(b, cols, weights, n, false, s)) != HIST_OK) return rc;
  }
  if (cudaEventRecord(b->done, s) != cudaSuccess) return HIST_ERR_CUDA;
  b->have_done = true;
  for (hist* h : b->hs) {
    if (cudaEventRecord(h->done, s) != cudaSuccess) return HIST_ERR_CUDA;
    h->have_done = true;
    h->n_entries += n;
    if (weights != nullptr && !(h->flags & HIST_TRACK_COUNTS)) h->counts_complete = false;
    if (weights != nullptr) {
      // direct global adds grow g_lo by < 2^32 per event: fold before 2^31 events
      h->fx_global_since_norm += std::max<int64_t>(n, b->grid);
      if (h->fx_global_since_norm > (int64_t)1 << 31) {
        if (launch_normalize_fx(h->g_lo, h->g_hi, h->nbins_total, s) != 0) return HIST_ERR_CUDA;
        h->fx_global_since_norm = 0;
      }
    }
  }
  if (weights != nullptr)
    for (hist* h : b->hs)
      if (h->flags & HIST_TRACK_COUNTS) h->counts_complete = false;  // batches do not count weighted entries
  return HIST_OK;
}

namespace {
void batch_report(const hist_batch* b, hist_batch_tuning_t* r) {
  std::memset(r, 0, sizeof(*r));
  r->candidates = 1;
  r->smem_bytes = b->smem_budget;
  int per_sm = 0;
  if (b->strategy == 0) {
    batch_max_blocks_per_sm(256, b->smem, b->wide_minb, b->wide_kev, &per_sm);
  } else if (b->strategy == 1) {
    slice_max_blocks_per_sm(kSliceBlock, b->smem, &per_sm);
  } else {
    per_sm = 1 << 30;
    for (const PartPlan& q : b->plans) per_sm = std::min(per_sm, q.fill_per_sm);
  }
  r->blocks_per_sm = per_sm;
  int nsm = 0;
  if (b->strategy == 0)
    for (int o : b->sbin_off) nsm += (o >= 0);
  else
    nsm = (int)b->hs.size();
  r->smem_hists = nsm;
  r->strategy = b->strategy;
  int nranges = 0;
  for (const PartPlan& q : b->plans) nranges += q.nranges;
  r->slices = b->strategy == 1 ? (int)b->slices.size() : (b->strategy == 2 ? nranges : 0);
  r->replicas = b->strategy == 1 ? b->slice_replicas : 0;
  r->cost_cap_tenths = b->strategy == 1 ? (int)(10.0 * b->slice_cap + 0.5) : 0;
  if (b->strategy == 0) {
    r->events_per_thread = b->wide_kev;
  } else if (b->strategy == 1) {
    r->events_per_thread = 4;
  } else {
    // the partitioned fill's kernel for the tuned sample's weights
    r->events_per_thread = 2;
    for (const PartPlan& q : b->plans)
      r->events_per_thread = std::max(r->events_per_thread, part_fill_events(b->placed_unit, b->f32c, q.row, q.smem));
  }
}
}  // namespace

extern "C" int hist_batch_tune(hist_batch_t* b, const double* const* cols, int ncols, const double* weights,
                               int64_t n, hist_batch_tuning_t* report) {
  if (b == nullptr || n <= 0) return HIST_ERR_ARG;
  int rc = batch_check_args(b, cols, ncols, weights, n);
  if (rc != HIST_OK) return rc;
  if (cudaSetDevice(b->device) != cudaSuccess) return HIST_ERR_CUDA;
  for (hist* h : b->hs)
    if (h->have_done && cudaEventSynchronize(h->done) != cudaSuccess) return HIST_ERR_CUDA;
  b->placed_unit = weights == nullptr;  // unit samples place one word per bin (a weighted fill re-places)
  // candidates: the wide strategy at five budgets times two occupancies
  // times two events per thread, the sliced one at two budgets times two
  // work caps (exact batches: an FP32C batch refuses it), the partitioned
  // one at three budgets (unless the batch was created with a fixed strategy)
  struct Cand {
    int strategy, budget;
    double cap;
    int minb, kev;
  };
  std::vector<Cand> cands;
  if (!(b->flags & HIST_BATCH_SLICED))
    for (int kb : {16, 48, 96, 144, 200})
      for (int minb : {2, 4})
        for (int kev : {4, 2}) cands.push_back({0, kb * 1024, 0.0, minb, kev});
  if (!(b->flags & HIST_BATCH_WIDE))
    for (int kb : {96, 200})
      for (double cap : {3.0, 12.0}) cands.push_back({1, kb * 1024, cap, 2, 4});
  if (!(b->flags & (HIST_BATCH_WIDE | HIST_BATCH_SLICED)))
    for (int kb : {48, 100, 200}) cands.push_back({2, kb * 1024, 0.0, 2, 4});
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HIST_ERR_CUDA;
  double best = 1e300, worst = 0.0;
  Cand best_c = cands.front();
  int tried = 0;
  std::vector<long long> seen;
  for (const Cand& c : cands) {
    b->wide_minb = c.minb;
    b->wide_kev = c.kev;
    rc = c.strategy == 0 ? batch_configure(b, c.budget)
                         : (c.strategy == 1 ? slice_configure(b, c.budget, c.cap) : part_configure(b, c.budget));
    if (rc == HIST_ERR_UNSUPPORTED) {
      rc = HIST_OK;
      continue;
    }
    if (rc != HIST_OK) break;
    if (c.strategy == 0) {  // budgets clamp to the same placement: time each variant once
      const long long sig = ((long long)b->smem_budget << 8) | (c.minb << 4) | c.kev;
      if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
      seen.push_back(sig);
    }
    if ((rc = batch_reserve(b, n, weights != nullptr)) != HIST_OK) break;
    if ((rc = batch_launch(b, cols, weights, n, true, nullptr)) != HIST_OK) break;  // warm-up
    cudaEventRecord(e0, nullptr);
    for (int r = 0; r < 3 && rc == HIST_OK; ++r) rc = batch_launch(b, cols, weights, n, true, nullptr);
    cudaEventRecord(e1, nullptr);
    if (rc != HIST_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = HIST_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.0f;
    ++tried;
    if (ms < best) {
      best = ms;
      best_c = c;
      best_c.budget = b->smem_budget;
    }
    worst = std::max(worst, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaDeviceSynchronize() != cudaSuccess) return HIST_ERR_CUDA;
  if (rc != HIST_OK) return rc;
  b->wide_minb = best_c.minb;
  b->wide_kev = best_c.kev;
  rc = best_c.strategy == 0
           ? batch_configure(b, best_c.budget)
           : (best_c.strategy == 1 ? slice_configure(b, best_c.budget, best_c.cap) : part_configure(b, best_c.budget));
  if (rc != HIST_OK) return rc;
  if (report) {
    batch_report(b, report);
    report->candidates = tried;
    report->best_ms = best;
    report->worst_ms = worst;
  }
  return HIST_OK;
}

extern "C" int hist_batch_configure(hist_batch_t* b, int32_t strategy, int32_t smem_bytes, int32_t cost_cap_tenths,
                                    int32_t pace_tiles, int32_t blocks_per_sm, int32_t events_per_thread,
                                    hist_batch_tuning_t* info) {
  if (b == nullptr || strategy < 0 || strategy > 2 || smem_bytes < 1024 ||
      (strategy == 1 && cost_cap_tenths < 10) || pace_tiles < -1 || (blocks_per_sm != 2 && blocks_per_sm != 4) ||
      (events_per_thread != 2 && events_per_thread != 4))
    return HIST_ERR_ARG;
  b->pace_tiles = pace_tiles;
  b->wide_minb = blocks_per_sm;
  b->wide_kev = events_per_thread;
  if (cudaSetDevice(b->device) != cudaSuccess) return HIST_ERR_CUDA;
  if (b->have_done && cudaEventSynchronize(b->done) != cudaSuccess) return HIST_ERR_CUDA;
  const int rc = strategy == 0   ? batch_configure(b, smem_bytes)
                 : strategy == 1 ? slice_configure(b, smem_bytes, 0.1 * cost_cap_tenths)
                                 : part_configure(b, smem_bytes);
  if (rc != HIST_OK) return rc;
  if (info) batch_report(b, info);
  return HIST_OK;
}
