// fill_device.cuh -- device pieces of the fill kernels (fill_kernels.cu): the
// per-thread statistics accumulator (FP32 double-word partials on two
// lanes, binary64 flushes), the binary64 statistics terms of rare events,
// the out-of-line bin updates (binary64 slow path, signed fixed-point add
// with carries, per-bin sum of w^2) and the block-wide statistics reduce.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {

constexpr int kFlushIters = 32;  // pairs of events (64 events) between binary64 flushes

// ---------------------------------------------------------------- statistics

// Statistics slots (stats[k]): 1 sum w, 2 sum w^2, 3 sum wx, 4 sum wx^2,
// 5 sum wy, 6 sum wy^2, 7 sum wxy, 8 sum wz, 9 sum wz^2, 10 sum wxz,
// 11 sum wyz.  Slot 0 (entries) and slot 1 (and slot 2 for unit weights)
// come from the host: the entry count and the in-range bin contents.
template <int NDIM>
struct NStats {
  static constexpr int NS = NDIM == 1 ? 5 : (NDIM == 2 ? 8 : 12);
};

template <int NDIM, bool UNIT>
struct StatAcc {
  static constexpr int NS = NStats<NDIM>::NS;
  FF2 s[NS];     // double-word partial sums of slots 3.. on two lanes (the two events of a pair)
  double d[NS];  // binary64 sums, refreshed every flush
  double w2;     // sum w^2, one binary64 FMA per event (weighted fills)

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      s[k].hi = make_float2(0.0f, 0.0f);
      s[k].lo = make_float2(0.0f, 0.0f);
      d[k] = 0.0;
    }
    w2 = 0.0;
  }

  // Coordinates and weight of two events, already split and packed (a lane
  // whose event takes no part is all zeros: it adds exact zeros).
  __device__ __forceinline__ void add_ff2(const FF2* c, FF2 W) {
    if (UNIT) {
      ff2_acc(s[3], c[0]);
      ff2_acc(s[4], ff2_mul(c[0], c[0]));
      if (NDIM >= 2) {
        ff2_acc(s[5], c[1]);
        ff2_acc(s[6], ff2_mul(c[1], c[1]));
        ff2_acc(s[7], ff2_mul(c[0], c[1]));
      }
      if (NDIM >= 3) {
        ff2_acc(s[8], c[2]);
        ff2_acc(s[9], ff2_mul(c[2], c[2]));
        ff2_acc(s[10], ff2_mul(c[0], c[2]));
        ff2_acc(s[11], ff2_mul(c[1], c[2]));
      }
    } else {
      const FF2 WX = ff2_mul(W, c[0]);
      ff2_acc(s[3], WX);
      ff2_acc(s[4], ff2_mul(WX, c[0]));
      if (NDIM >= 2) {
        const FF2 WY = ff2_mul(W, c[1]);
        ff2_acc(s[5], WY);
        ff2_acc(s[6], ff2_mul(WY, c[1]));
        ff2_acc(s[7], ff2_mul(WX, c[1]));
        if (NDIM >= 3) {
          const FF2 WZ = ff2_mul(W, c[2]);
          ff2_acc(s[8], WZ);
          ff2_acc(s[9], ff2_mul(WZ, c[2]));
          ff2_acc(s[10], ff2_mul(WX, c[2]));
          ff2_acc(s[11], ff2_mul(WY, c[2]));
        }
      }
    }
  }

  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int k = 3; k < NS; ++k) {
      const FF a = {s[k].hi.x, s[k].lo.x}, b = {s[k].hi.y, s[k].lo.y};
      d[k] = __dadd_rn(d[k], __dadd_rn(ff_to_double(a), ff_to_double(b)));
      s[k].hi = make_float2(0.0f, 0.0f);
      s[k].lo = make_float2(0.0f, 0.0f);
    }
  }
};

// binary64 statistics terms of one event, rounded as in the definition
// (w*x*x = (w*x)*x), added into d[2..NS) (d[2] only for weighted fills: the
// host adds sum w^2 of unit-weight entries).  Kept out of line: it runs only
// for coordinates or weights outside the double-word range and for the
// binary64-atomic mode.
template <int NDIM, bool UNIT>
__device__ __noinline__ void stat_f64(double* d, const unsigned long long* cb, unsigned long long wb) {
  double c[NDIM];
#pragma unroll
  for (int k = 0; k < NDIM; ++k) c[k] = __longlong_as_double((long long)cb[k]);
  const double w = __longlong_as_double((long long)wb);
  const double wx = __dmul_rn(w, c[0]);
  if (!UNIT) d[2] = __dadd_rn(d[2], __dmul_rn(w, w));  // unit weights: the host adds sum w^2
  d[3] = __dadd_rn(d[3], wx);
  d[4] = __dadd_rn(d[4], __dmul_rn(wx, c[0]));
  if (NDIM >= 2) {
    const double wy = __dmul_rn(w, c[1]);
    d[5] = __dadd_rn(d[5], wy);
    d[6] = __dadd_rn(d[6], __dmul_rn(wy, c[1]));
    d[7] = __dadd_rn(d[7], __dmul_rn(wx, c[1]));
    if (NDIM >= 3) {
      const double wz = __dmul_rn(w, c[2]);
      d[8] = __dadd_rn(d[8], wz);
      d[9] = __dadd_rn(d[9], __dmul_rn(wz, c[2]));
      d[10] = __dadd_rn(d[10], __dmul_rn(wx, c[2]));
      d[11] = __dadd_rn(d[11], __dmul_rn(wy, c[2]));
    }
  }
}

// Slow-path bin update: binary64 atomic into the global slow words.
__device__ __noinline__ void slow_bin(double* g_f64, long long g, unsigned long long wb) {
  atomicAdd(&g_f64[g], __longlong_as_double((long long)wb));
}

__device__ __noinline__ void sumw2_global(double* g_sumw2, long long g, unsigned long long wb) {
  const double w = __longlong_as_double((long long)wb);
  atomicAdd(&g_sumw2[g], __dmul_rn(w, w));
}

// w^2 into FP32 compensated shared words (hi, lo) of bin g: the square as an
// FP32 double-word from the weight's hi + lo split (within 2^-45 w^2 of
// fl(w*w)), hi added by an atomic that returns the old value so its
// rounding error is recovered exactly (TwoSum) and added with the low part;
// weights outside the double-word range take the binary64 global atomic.
__device__ __noinline__ void sumw2_shared(unsigned* words, double* g_sumw2, long long g, unsigned long long wb) {
  if (!in_ff(exp_field(wb))) {
    sumw2_global(g_sumw2, g, wb);
    return;
  }
  const FF W = ff_split(wb, hi24(wb));
  const float ph = __fmul_rn(W.hi, W.hi);
  const float pe = __fmaf_rn(W.hi, W.hi, -ph);
  const float pl = __fmaf_rn(__fadd_rn(W.hi, W.hi), W.lo, pe);
  float* a = reinterpret_cast<float*>(&words[2 * g]);
  const float old = atomicAdd(a, ph);
  const float sum = __fadd_rn(old, ph);
  const float bv = __fsub_rn(sum, old);
  const float err = __fadd_rn(__fsub_rn(old, __fsub_rn(sum, bv)), __fsub_rn(ph, bv));
  atomicAdd(a + 1, __fadd_rn(err, pl));
}

// Signed fixed-point value V into a shared bin's low 64 bits (words a[0],
// a[1]): a 96-bit add with carries.  Each atomic returns the old word, so the
// carry it produced is known exactly whatever the interleaving; the rare
// top-word change (a carry out of bit 63, or the sign of a negative addend
// not absorbed by a carry) goes to the global high word, which holds the sum
// in units of 2^32.  Out of line: the hot loop keeps the positive case only.
__device__ __noinline__ void fx_add_shared(unsigned* a, long long* ghi, long long V) {
  const unsigned v0 = (unsigned)V;
  const unsigned o0 = atomicAdd(a, v0);
  const unsigned c0 = (o0 + v0 < o0) ? 1u : 0u;
  const unsigned a1 = (unsigned)((unsigned long long)V >> 32) + c0;
  const unsigned c1a = (a1 < c0) ? 1u : 0u;
  const unsigned o1 = atomicAdd(a + 1, a1);
  const unsigned c1 = c1a | ((o1 + a1 < o1) ? 1u : 0u);
  const int top = (int)(V >> 63) + (int)c1;
  if (top != 0) atomicAdd(reinterpret_cast<unsigned long long*>(ghi), (unsigned long long)((long long)top << 32));
}

__device__ __noinline__ void f64_bin(double* bins, long long slot, unsigned long long wb) {
  atomicAdd(&bins[slot], __longlong_as_double((long long)wb));
}

// Block-wide sum of per-thread binary64 statistics (warp shuffles, then the
// warps in order); thread k < kMaxStats writes slot k of the block partial.
template <int NS>
__device__ __forceinline__ void block_reduce_stats(const double* d, double* out, double* sred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 2; k < NS; ++k) {
    double v = d[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sred[warp * kMaxStats + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxStats) {
    const int k = threadIdx.x;
    double v = 0.0;
    if (k >= 2 && k < NS)
      for (int wi = 0; wi < nwarps; ++wi) v = __dadd_rn(v, sred[wi * kMaxStats + k]);
    out[k] = v;
  }
}

}  // namespace
}  // namespace hgb
