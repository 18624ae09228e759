// batch_stats.cuh -- statistics sums of the batched fills (both strategies).
//
// Per histogram the statistics are sum w^2, sum wx, sum wx^2 over its
// in-range entries (sum w and the entry count come from the bins on the
// host), each term rounded as defined: w*w, w*x, (w*x)*x.  They depend only
// on the column and the range, so the batch groups members by (column,
// range); an event inside its column's core (the range every group of the
// column contains) adds to the column's core sums once, and only events
// outside the core walk the column's groups (tail sums, per thread in local
// memory: rare by construction).  Accumulation is binary64 per thread; each
// block sums its threads in one fixed order.
#pragma once

#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {

template <bool UNIT>
__device__ __forceinline__ void stat_core_add(double (&s)[3], unsigned long long xb, unsigned long long wb) {
  const double x = __longlong_as_double((long long)xb);
  const double w = __longlong_as_double((long long)wb);
  const double wx = UNIT ? x : __dmul_rn(w, x);
  if (!UNIT) s[0] = __fma_rn(w, w, s[0]);
  s[1] = __dadd_rn(s[1], wx);
  s[2] = __fma_rn(wx, x, s[2]);
}

// An event outside the core of column c: add it to the tail sums of every
// group of the column whose range holds it.
template <bool UNIT>
__device__ __noinline__ void stat_tail(const BatchStatsSpec& st, int c, long long key, unsigned long long xb,
                                       unsigned long long wb, double* tail) {
  const double x = __longlong_as_double((long long)xb);
  const double w = __longlong_as_double((long long)wb);
  const double wx = UNIT ? x : __dmul_rn(w, x);
  for (int g = st.group_begin[c]; g < st.group_begin[c + 1]; ++g) {
    if (key < st.group_lo[g] || key >= st.group_hi[g]) continue;
    if (!UNIT) tail[3 * g] = __fma_rn(w, w, tail[3 * g]);
    tail[3 * g + 1] = __dadd_rn(tail[3 * g + 1], wx);
    tail[3 * g + 2] = __fma_rn(wx, x, tail[3 * g + 2]);
  }
}

template <bool UNIT>
__device__ __forceinline__ void stat_event(const BatchStatsSpec& st, int c, long long key, unsigned long long xb,
                                           unsigned long long wb, double (&core)[3], double* tail) {
  if (key >= st.core_lo[c] && key < st.core_hi[c])
    stat_core_add<UNIT>(core, xb, wb);
  else
    stat_tail<UNIT>(st, c, key, xb, wb, tail);
}

// Block sums of every slot (cores of the columns, then tails of the groups),
// threads in one fixed order; `sred` holds [warps][kStatSlots * 3].
__device__ __forceinline__ void block_stats_store(const double (&core)[kBatchMaxCols][3], const double* tail,
                                                  double* sred, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int kVals = kStatSlots * 3;
#pragma unroll
  for (int c = 0; c < kBatchMaxCols; ++c)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double v = core[c][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
      if (lane == 0) sred[warp * kVals + c * 3 + q] = v;
    }
  for (int t = 0; t < kBatchMaxGroups * 3; ++t) {
    double v = tail[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sred[warp * kVals + kBatchMaxCols * 3 + t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kVals; t += blockDim.x) {
    double v = 0.0;
    for (int wi = 0; wi < nwarps; ++wi) v = __dadd_rn(v, sred[wi * kVals + t]);
    out[t] = v;
  }
}

}  // namespace
}  // namespace hgb
