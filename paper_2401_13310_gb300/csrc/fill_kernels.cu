// fill_kernels.cu -- device side of bulk histogram filling for sm_103a.
//
// One fill launch runs the three steps of Sec. 3.1 of the paper for every
// event of a bulk: find the bin on each axis, add the weight to the bin,
// update the statistics sums (Sec. 3.2: sum w, w^2, wx, wx^2 in 1D).  The
// paper's kernel fills a per-block histogram in shared memory with block
// atomics and merges it into the global histogram with grid atomics
// (Sec. 3.2, two-stage filling), and reduces the statistics in separate
// kernels (one per statistic).  Here:
//
//  * find-bin never uses binary64 arithmetic (on GB300 the binary64 pipe
//    issues under two operations per clock per SM, about 1/60 of the FP32
//    rate).  Every axis is a table of exact threshold keys (hist_internal.h).
//    Fixed axes first evaluate the formula in FP32 from the coordinate's bits;
//    the host proves a bound eps on the distance between that value and the
//    binary64 one, so whenever the FP32 value is farther than eps from an
//    integer its floor IS the binary64 bin.  The rare rest (and variable axes)
//    compare ordered int64 keys against the thresholds.
//  * weighted bins are summed exactly in fixed point: |w| in the window
//    [2^(e-1023), 2^(e-1007)) (e = fx_elo) becomes a 64-bit integer multiple
//    of 2^(e-1065) (truncation error <= 2^-42 |w|), added to a 96-bit
//    per-block accumulator held as three u32 words in shared memory by 32-bit
//    atomics that propagate their carries (u32 shared atomics sustain about 7
//    per clock per SM, against 0.7-1 for binary64 ones and 1.5 for 64-bit
//    ones).  The sum is exact, so the order of the atomics does not matter.
//    Other weights take a slow path (binary64 atomic in global memory).
//  * sum w is not accumulated per event: it equals the sum of the in-range
//    bin contents, which the host forms exactly from the fixed-point bins.
//    The other statistics terms are formed and summed per thread in FP32
//    double-word arithmetic (error-free products with FMA, TwoSum
//    accumulation), flushed to binary64 every 64 events, reduced across the
//    block with warp shuffles and written as one partial per block; the
//    reduce kernel adds the partials in block order (deterministic).
//  * each thread handles four events per iteration (two coalesced pairs), so
//    loads and the carry-chained atomics of independent events overlap.
//  * per-block bin partials go to scratch; the reduce kernel sums them in
//    slices and merges the exact integer sums with 64-bit atomics.
//
// Nothing here is compiled with FMA contraction (-fmad=false); every
// error-free transformation uses explicit round-to-nearest intrinsics, and
// rarely-taken binary64 paths live in non-inlined functions so that they are
// real branches, not predicated code issued for every event.

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "fill_device.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {
#ifndef HGB_MIN_BLOCKS
#define HGB_MIN_BLOCKS 1
#endif
#ifndef HGB_MIN_BLOCKS_1D
#define HGB_MIN_BLOCKS_1D 4  // 1D kernels fit in 64 registers: four 256-thread blocks per SM
#endif
// ---------------------------------------------------------------- loads


// ---------------------------------------------------------------- fill kernel

// Per-thread state of one fill launch and the three steps for one event.
template <int NDIM, int ACC, bool SMEM, int LOC, bool SW2 = false>
struct Filler {
  static constexpr bool UNIT = (ACC == ACC_UNIT);
  static constexpr int NS = NStats<NDIM>::NS;
  const FillParams& p;
  const long long* Tax[NDIM];
  const int* BKx[NDIM];  // bucket counts (LOC_BUCKET), shared or global
  const int* Thi[NDIM];  // high words of the shared-memory thresholds (nullptr: global table)
  unsigned* sbins;
  double* sbins_f64;
  int stride1, stride2;
  StatAcc<NDIM, UNIT> st;
  double* slow;  // binary64 statistics of slow-path events (local memory)

  __device__ __forceinline__ Filler(const FillParams& pp) : p(pp) {}

  // w^2 of the event into its bin's sum of squares (out of line: the hot
  // loop of fills without HIST_SUMW2 keeps only the test)
  __device__ __forceinline__ void sumw2_add(long long g, unsigned long long wb) {
    constexpr bool kShared = SMEM && (ACC == ACC_FX || ACC == ACC_F32C);
    if (kShared)
      sumw2_shared(sbins + (p.track_counts ? 3 : 2) * (int)p.nbins_total, p.g_sumw2, g, wb);
    else
      sumw2_global(p.g_sumw2, g, wb);
  }

  // Whether an event enters the statistics, and through the double-word path.
  struct StatIn {
    bool take, fast;
  };

  // Steps 1 and 2 of one event (and its w^2 for HIST_SUMW2).
  __device__ __forceinline__ StatIn bin_step(const unsigned long long* cb, unsigned long long wb) {
    // ---- step 1: the bin on every axis, linearised x fastest
    float xf[NDIM];
    unsigned ef[NDIM];
    long long g = 0;
    bool inr = true;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      ef[d] = exp_field(cb[d]);
      xf[d] = hi24(cb[d]);
      // (the FP32 estimate is trusted inside the double-word range, a subset
      // of the exact-truncation range that the statistics test anyway)
      const int k = locate_mode<LOC>(p.ax[d], Tax[d], Thi[d], BKx[d], cb[d], xf[d], in_ff(ef[d]));
      inr = inr && ((unsigned)(k - 1) < (unsigned)p.ax[d].nbins);
      g += (long long)k * (d == 0 ? 1 : (d == 1 ? stride1 : stride2));
    }
    // ---- step 2: the bin content
    bool w_ok = true;
    if (UNIT) {
      if (SMEM)
        atomicAdd(&sbins[g], 1u);
      else
        atomicAdd(&p.g_unit[g], 1ull);
    } else if (ACC == ACC_FX && SMEM) {
      // the weight's fixed-point value U = trunc(|w| 2^(1065 - elo)) as two
      // u32 words, from 32-bit funnel shifts of its significand (the same
      // value as fx_of): M << 10 >> (20 - rel), 5 <= 20 - rel <= 20
      const unsigned whi = (unsigned)(wb >> 32), wlo = (unsigned)wb;
      const unsigned rel = ((whi >> 20) & 0x7FFu) - (unsigned)p.fx_elo;
      w_ok = rel < 16u;
      if (!w_ok) {
        slow_bin(p.g_f64, g, wb);
      } else {
        const unsigned mh = (whi & 0x000FFFFFu) | 0x00100000u;
        const unsigned sh = 20u - rel;
        const unsigned h10 = __funnelshift_l(wlo, mh, 10);
        const unsigned u0 = __funnelshift_r(wlo << 10, h10, sh);
        const unsigned u1 = h10 >> sh;  // < 2^26
        unsigned* a = &sbins[2 * g];
        if ((int)whi < 0) {
          fx_add_shared(a, &p.g_hi[g], -(long long)(((unsigned long long)u1 << 32) | u0));
        } else {
          // 64-bit add with carries (a positive addend: the only top-word
          // change is a carry out of bit 63, added to the global high word)
          const unsigned o0 = atomicAdd(a, u0);
          const unsigned a1 = u1 + ((o0 + u0 < o0) ? 1u : 0u);
          const unsigned o1 = atomicAdd(a + 1, a1);
          if (o1 + a1 < o1) atomicAdd(reinterpret_cast<unsigned long long*>(&p.g_hi[g]), 1ull << 32);
        }
      }
      if (p.track_counts) atomicAdd(&sbins[2 * (int)p.nbins_total + g], 1u);
    } else if (ACC == ACC_FX) {  // bins in global memory
      long long V;
      w_ok = fx_of(wb, p.fx_elo, &V);
      if (!w_ok) {
        slow_bin(p.g_f64, g, wb);
      } else if (V != 0) {
        // two fire-and-forget 64-bit reductions (the low 32 bits, the rest
        // in units of 2^32): one atomic that returns the old value for an
        // exact carry was measured slower here (1e6 bins, hot central bins:
        // 2.36 against 1.84 ms per 1e8 2D events), its latency on the
        // critical path
        atomicAdd(&p.g_lo[g], (unsigned long long)(unsigned)V);
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.g_hi[g]), (unsigned long long)(V >> 32));
      }
      if (p.track_counts) atomicAdd(&p.g_count[g], 1ull);
    } else if (ACC == ACC_F32C) {
      // FP32 compensated partials: the weight as hi + lo (FP32 double-word);
      // hi goes to the block's FP32 bin by an atomic that returns the old
      // value, so the rounding error of that addition is recovered exactly
      // (TwoSum) and added, with lo, to the bin's FP32 compensation word
      w_ok = in_ff(exp_field(wb));
      if (!w_ok || !SMEM) {
        slow_bin(p.g_f64, g, wb);  // outside the double-word range, or bins in global memory
      } else {
        const FF W = ff_split(wb, hi24(wb));
        float* a = reinterpret_cast<float*>(&sbins[2 * g]);
        const float old = atomicAdd(a, W.hi);
        const float sum = __fadd_rn(old, W.hi);
        const float bv = __fsub_rn(sum, old);
        const float err = __fadd_rn(__fsub_rn(old, __fsub_rn(sum, bv)), __fsub_rn(W.hi, bv));
        atomicAdd(a + 1, __fadd_rn(err, W.lo));
      }
      if (p.track_counts) {
        if (SMEM)
          atomicAdd(&sbins[2 * (int)p.nbins_total + g], 1u);
        else
          atomicAdd(&p.g_count[g], 1ull);
      }
    } else {  // ACC_F64: the paper's binary64 atomics
      if (SMEM) {
        f64_bin(sbins_f64, 2 * g, wb);
        if (p.track_counts) f64_bin(sbins_f64, 2 * g + 1, 0x3FF0000000000000ull);
      } else {
        f64_bin(p.g_f64, g, wb);
        if (p.track_counts) atomicAdd(&p.g_count[g], 1ull);
      }
    }
    // ---- per-bin sum of w^2 (ROOT's Sumw2)
    if (SW2) sumw2_add(g, wb);
    StatIn si;
    si.take = inr || p.stat_overflows;
    bool fast = (ACC != ACC_F64) && w_ok;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) fast = fast && in_ff(ef[d]);
    si.fast = fast;
    return si;
  }

  // ---- step 3: statistics of two events; the double-word sums run on two
  // lanes of the packed FP32x2 instructions, one lane per event
  __device__ __forceinline__ void stats2(const unsigned long long* ca, unsigned long long wa, StatIn ia,
                                         const unsigned long long* cb, unsigned long long wb, StatIn ib) {
    if (ia.take && !ia.fast) stat_f64<NDIM, UNIT>(slow, ca, wa);
    if (ib.take && !ib.fast) stat_f64<NDIM, UNIT>(slow, cb, wb);
    const bool fa = ia.take && ia.fast, fb = ib.take && ib.fast;
    if constexpr (NDIM == 1) {
      // 1D: the integer work, not the FP32 pipe, bounds the kernel; each
      // event runs the scalar double-word forms on its own lane
      if (fa) stat1(ca[0], wa, 0);
      if (fb) stat1(cb[0], wb, 1);
      return;
    }
    if (!(fa || fb)) return;
    FF2 c2[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const FF xa = ff_split(ca[d], hi24(ca[d])), xb = ff_split(cb[d], hi24(cb[d]));
      c2[d].hi = make_float2(fa ? xa.hi : 0.0f, fb ? xb.hi : 0.0f);
      c2[d].lo = make_float2(fa ? xa.lo : 0.0f, fb ? xb.lo : 0.0f);
    }
    FF2 W2;
    if (UNIT) {
      W2.hi = make_float2(fa ? 1.0f : 0.0f, fb ? 1.0f : 0.0f);
      W2.lo = make_float2(0.0f, 0.0f);
    } else {
      // in-window weights lie in the double-word range
      const FF a = ff_split(wa, hi24(wa)), b = ff_split(wb, hi24(wb));
      W2.hi = make_float2(fa ? a.hi : 0.0f, fb ? b.hi : 0.0f);
      W2.lo = make_float2(fa ? a.lo : 0.0f, fb ? b.lo : 0.0f);
      // the binary64 pipe is otherwise idle: w^2 costs one issue slot there
      const double da = fa ? __longlong_as_double((long long)wa) : 0.0;
      const double db = fb ? __longlong_as_double((long long)wb) : 0.0;
      st.w2 = __fma_rn(da, da, st.w2);
      st.w2 = __fma_rn(db, db, st.w2);
    }
    st.add_ff2(c2, W2);
  }

  // One 1D event into lane `lane` of the double-word sums (scalar forms).
  __device__ __forceinline__ void stat1(unsigned long long xb, unsigned long long wb, int lane) {
    const FF X = ff_split(xb, hi24(xb));
    FF W;
    if (UNIT) {
      W.hi = 1.0f;
      W.lo = 0.0f;
    } else {
      W = ff_split(wb, hi24(wb));
      const double w = __longlong_as_double((long long)wb);
      st.w2 = __fma_rn(w, w, st.w2);
    }
    FF s3 = lane ? FF{st.s[3].hi.y, st.s[3].lo.y} : FF{st.s[3].hi.x, st.s[3].lo.x};
    FF s4 = lane ? FF{st.s[4].hi.y, st.s[4].lo.y} : FF{st.s[4].hi.x, st.s[4].lo.x};
    const FF WX = UNIT ? X : ff_mul(W, X);
    ff_acc(s3, WX);
    ff_acc(s4, ff_mul(WX, X));
    if (lane) {
      st.s[3].hi.y = s3.hi; st.s[3].lo.y = s3.lo;
      st.s[4].hi.y = s4.hi; st.s[4].lo.y = s4.lo;
    } else {
      st.s[3].hi.x = s3.hi; st.s[3].lo.x = s3.lo;
      st.s[4].hi.x = s4.hi; st.s[4].lo.x = s4.lo;
    }
  }

  __device__ __forceinline__ void event(const unsigned long long* cb, unsigned long long wb) {
    const StatIn i = bin_step(cb, wb);
    stats2(cb, wb, i, cb, wb, StatIn{false, false});
  }

  __device__ __forceinline__ void event_pair(const unsigned long long* c0, unsigned long long w0,
                                             const unsigned long long* c1, unsigned long long w1) {
    if constexpr (NDIM == 1) {  // one event after the other, as scalar code schedules best
      event(c0, w0);
      event(c1, w1);
      return;
    }
    const StatIn i0 = bin_step(c0, w0);
    const StatIn i1 = bin_step(c1, w1);
    stats2(c0, w0, i0, c1, w1, i1);
  }
};

// Two consecutive binary64 values as raw bits (no double-typed value ever
// flows through the hot loop, so nothing is scheduled on the binary64 pipe
// by accident).
template <bool VEC>
__device__ __forceinline__ void load_pair(const double* __restrict__ p, long long i, unsigned long long& a,
                                          unsigned long long& b) {
  const unsigned long long* q = reinterpret_cast<const unsigned long long*>(p);
  if (VEC) {
    const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(q + i));
    a = v.x;
    b = v.y;
  } else {
    a = __ldcs(q + i);
    b = __ldcs(q + i + 1);
  }
}

// All full pairs of events, grid-strided: thread t takes pairs t, t + T,
// t + 2T, ... (T threads), counted with 32-bit indices from its own column
// pointers.  Two register buffers alternate: the next pair's loads are
// issued before the current pair is processed, so each thread keeps two
// pairs of loads in flight across the long per-event work, and nothing is
// copied between buffers.
//
// 2D and 3D fills keep one buffer that the next pair's loads are copied
// into: their per-event work is large, and with two copies of it in the
// loop body the 3D fill of 1e8 uniform triples into 100^3 bins took 2.57 ms
// against 1.77 ms.
template <int NDIM, int ACC, bool SMEM, int LOC, bool SW2, bool VEC>
__device__ __forceinline__ void fill_pairs_nd(Filler<NDIM, ACC, SMEM, LOC, SW2>& f, long long npairs) {
  const FillParams& p = f.p;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  int iters = 0;
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned long long c0[NDIM], c1[NDIM], w0 = 0x3FF0000000000000ull, w1 = 0x3FF0000000000000ull;
  if (q < npairs) {
#pragma unroll
    for (int d = 0; d < NDIM; ++d) load_pair<VEC>(p.col[d], 2 * q, c0[d], c1[d]);
    if (ACC != ACC_UNIT) load_pair<VEC>(p.w, 2 * q, w0, w1);
  }
  for (; q < npairs; q += nthreads) {
    unsigned long long n0[NDIM], n1[NDIM], nw0 = 0x3FF0000000000000ull, nw1 = 0x3FF0000000000000ull;
    const long long qn = q + nthreads;
    if (qn < npairs) {
#pragma unroll
      for (int d = 0; d < NDIM; ++d) load_pair<VEC>(p.col[d], 2 * qn, n0[d], n1[d]);
      if (ACC != ACC_UNIT) load_pair<VEC>(p.w, 2 * qn, nw0, nw1);
    }
    f.event_pair(c0, w0, c1, w1);
    if (++iters == kFlushIters) {
      f.st.flush();
      iters = 0;
    }
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      c0[d] = n0[d];
      c1[d] = n1[d];
    }
    w0 = nw0;
    w1 = nw1;
  }
}

template <int NDIM, int ACC, bool SMEM, int LOC, bool SW2, bool VEC>
__device__ __forceinline__ void fill_pairs(Filler<NDIM, ACC, SMEM, LOC, SW2>& f, long long npairs) {
  if constexpr (NDIM > 1) {
    fill_pairs_nd<NDIM, ACC, SMEM, LOC, SW2, VEC>(f, npairs);
    return;
  }
  const FillParams& p = f.p;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long q0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q0 >= npairs) return;
  const int cnt = (int)((npairs - q0 + nthreads - 1) / nthreads);  // pairs of this thread
  const double* xc[NDIM];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) xc[d] = p.col[d] + 2 * q0;
  const double* wc = ACC != ACC_UNIT ? p.w + 2 * q0 : nullptr;
  const long long step = 2 * nthreads;
  auto load = [&](int it, unsigned long long* e0, unsigned long long* e1, unsigned long long& w0,
                  unsigned long long& w1) {
    const long long off = (long long)it * step;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) load_pair<VEC>(xc[d], off, e0[d], e1[d]);
    if (ACC != ACC_UNIT) load_pair<VEC>(wc, off, w0, w1);
  };
  if constexpr (ACC == ACC_UNIT && LOC == LOC_AFFINE) {
    // Unit weights on a fixed axis (the paper's own benchmark shape): the
    // per-event work is short and the loads' latency shows (long-scoreboard
    // stalls as frequent as issue-slot contention with two pairs in flight),
    // so four register buffers rotate and each thread keeps three pairs'
    // loads in flight while it processes the fourth.
    constexpr unsigned long long kOne = 0x3FF0000000000000ull;
    unsigned long long a0[NDIM], a1[NDIM], b0[NDIM], b1[NDIM], e0[NDIM], e1[NDIM], g0[NDIM], g1[NDIM], u0, u1;
    load(0, a0, a1, u0, u1);
    if (1 < cnt) load(1, b0, b1, u0, u1);
    if (2 < cnt) load(2, e0, e1, u0, u1);
    int it = 0, iters = 0;
    while (true) {
      if (it + 3 < cnt) load(it + 3, g0, g1, u0, u1);
      f.event_pair(a0, kOne, a1, kOne);
      if (++it >= cnt) break;
      if (it + 3 < cnt) load(it + 3, a0, a1, u0, u1);
      f.event_pair(b0, kOne, b1, kOne);
      if (++it >= cnt) break;
      if (it + 3 < cnt) load(it + 3, b0, b1, u0, u1);
      f.event_pair(e0, kOne, e1, kOne);
      if (++it >= cnt) break;
      if (it + 3 < cnt) load(it + 3, e0, e1, u0, u1);
      f.event_pair(g0, kOne, g1, kOne);
      if (++it >= cnt) break;
      if (++iters == kFlushIters / 4) {  // four pairs per turn of the loop
        f.st.flush();
        iters = 0;
      }
    }
    return;
  }
  unsigned long long a0[NDIM], a1[NDIM], aw0 = 0x3FF0000000000000ull, aw1 = 0x3FF0000000000000ull;
  unsigned long long b0[NDIM], b1[NDIM], bw0 = 0x3FF0000000000000ull, bw1 = 0x3FF0000000000000ull;
  load(0, a0, a1, aw0, aw1);
  int it = 0, iters = 0;
  while (true) {
    if (it + 1 < cnt) load(it + 1, b0, b1, bw0, bw1);
    f.event_pair(a0, aw0, a1, aw1);
    if (++it >= cnt) break;
    if (it + 1 < cnt) load(it + 1, a0, a1, aw0, aw1);
    f.event_pair(b0, bw0, b1, bw1);
    if (++it >= cnt) break;
    if (++iters == kFlushIters / 2) {  // two pairs per turn of the loop
      f.st.flush();
      iters = 0;
    }
  }
}

// Fused Filter/Define: every event of the source columns, grid-strided;
// the filters (each a binary64 comparison with a constant) decide whether
// it is filled at all, and the defines give its coordinates, each
// operation rounded once as written (x*x + y*y is fl(fl(x*x) + fl(y*y))).
// Passing events are counted (the entry count).
__device__ __forceinline__ bool expr_pass(const ExprDev& ex, const double* v) {
  bool ok = true;
  for (int k = 0; k < ex.nfilt; ++k) {
    const double a = v[ex.filt_col[k]], c = ex.filt_val[k];
    bool t;
    switch (ex.filt_op[k]) {
      case FLT_NE: t = a != c; break;
      case FLT_EQ: t = a == c; break;
      case FLT_LT: t = a < c; break;
      case FLT_LE: t = a <= c; break;
      case FLT_GT: t = a > c; break;
      default: t = a >= c; break;
    }
    ok = ok && t;
  }
  return ok;
}

__device__ __forceinline__ double expr_define(int op, double a, double b) {
  switch (op) {
    case DEF_SUMSQ: return __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
    case DEF_HYPOT: return __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
    case DEF_MUL: return __dmul_rn(a, b);
    case DEF_ADD: return __dadd_rn(a, b);
    case DEF_SUB: return __dsub_rn(a, b);
    default: return a;
  }
}

template <int NDIM, int ACC, bool SMEM, int LOC, bool SW2>
__device__ __forceinline__ void fill_expr(Filler<NDIM, ACC, SMEM, LOC, SW2>& f) {
  const FillParams& p = f.p;
  const ExprDev& ex = p.ex;
  const long long n = p.n;
  unsigned long long passed = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v[kExprMaxSrc];
#pragma unroll
    for (int c = 0; c < kExprMaxSrc; ++c) v[c] = c < ex.nsrc ? __ldcs(ex.src[c] + i) : 0.0;
    if (!expr_pass(ex, v)) continue;
    ++passed;
    unsigned long long cb[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d)
      cb[d] = (unsigned long long)__double_as_longlong(expr_define(ex.def_op[d], v[ex.def_a[d]], v[ex.def_b[d]]));
    const unsigned long long wb =
        ACC == ACC_UNIT ? 0x3FF0000000000000ull : __ldcs(reinterpret_cast<const unsigned long long*>(p.w) + i);
    f.event(cb, wb);
    if ((passed & 63) == 0) f.st.flush();  // at most 64 events between flushes, as in fill_pairs
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) passed += __shfl_down_sync(0xffffffffu, passed, o);
  if ((threadIdx.x & 31) == 0 && passed) atomicAdd(ex.g_passed, passed);
}

// DIRECT: the block adds its bins to the persistent accumulators itself and
// the last block sums the statistics partials (small 1D fills: no partial
// bins and no reduce launch); compiled apart so that the other fills keep
// none of its code.
template <int NDIM, int ACC, bool SMEM, int LOC, bool SW2, bool EXPR, bool DIRECT = false>
__global__ void __launch_bounds__(256, NDIM == 1 ? HGB_MIN_BLOCKS_1D : HGB_MIN_BLOCKS) k_fill(const FillParams p) {
  static_assert(!DIRECT || (NDIM == 1 && SMEM && (ACC == ACC_UNIT || ACC == ACC_FX) && !SW2 && !EXPR),
                "direct flush: 1D exact or unit-count shared bins");
  constexpr bool UNIT = (ACC == ACC_UNIT);
  constexpr int NS = NStats<NDIM>::NS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nkeys = p.table_keys;
  long long* skeys = reinterpret_cast<long long*>(smem_raw);
  int* shi = reinterpret_cast<int*>(smem_raw + (size_t)nkeys * 8);
  int* sbk = reinterpret_cast<int*>(smem_raw + (((size_t)nkeys * 12 + 15) & ~(size_t)15));
  unsigned char* after_keys =
      smem_raw + (((size_t)nkeys * 12 + 15) & ~(size_t)15) + (((size_t)p.table_bk * 4 + 15) & ~(size_t)15);
  __shared__ double sred[8 * kMaxStats];

  Filler<NDIM, ACC, SMEM, LOC, SW2> f(p);
  f.sbins = reinterpret_cast<unsigned*>(after_keys);
  f.sbins_f64 = reinterpret_cast<double*>(after_keys);
  for (int i = threadIdx.x; i < nkeys; i += blockDim.x) {
    const long long t = p.T_concat[i];
    skeys[i] = t;
    shi[i] = (int)(t >> 32);
  }
  for (int i = threadIdx.x; i < p.table_bk; i += blockDim.x) sbk[i] = p.BK_concat[i];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    const bool staged = p.ax[d].smem_off >= 0;
    f.Tax[d] = staged ? skeys + p.ax[d].smem_off : p.ax[d].T;
    f.Thi[d] = staged ? shi + p.ax[d].smem_off : nullptr;
    f.BKx[d] = p.ax[d].bk.smem_off >= 0 ? sbk + p.ax[d].bk.smem_off : p.ax[d].bk.cnt;
  }
  const int nb = (int)p.nbins_total;
  if (SMEM) {
    const int words = (UNIT ? 1
                            : ((ACC == ACC_FX || ACC == ACC_F32C) ? (p.track_counts ? 3 : 2) + (p.sumw2 ? 2 : 0)
                                                                  : 4)) *
                      nb;
    for (int i = threadIdx.x; i < words; i += blockDim.x) f.sbins[i] = 0u;
  }
  f.stride1 = p.ax[0].nbins + 2;
  f.stride2 = NDIM >= 2 ? f.stride1 * (p.ax[1].nbins + 2) : 0;
  f.st.init();
  double slow[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) slow[k] = 0.0;
  f.slow = slow;
  __syncthreads();

  // every full pair of events, then the odd last event
  const long long n = p.n;
  if (EXPR)
    fill_expr(f);
  else if (p.aligned)
    fill_pairs<NDIM, ACC, SMEM, LOC, SW2, true>(f, n >> 1);
  else
    fill_pairs<NDIM, ACC, SMEM, LOC, SW2, false>(f, n >> 1);
  if (!EXPR && (n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
    unsigned long long c[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) c[d] = __ldcs(reinterpret_cast<const unsigned long long*>(p.col[d]) + (n - 1));
    const unsigned long long w =
        UNIT ? 0x3FF0000000000000ull : __ldcs(reinterpret_cast<const unsigned long long*>(p.w) + (n - 1));
    f.event(c, w);
  }
  f.st.flush();
  f.st.d[2] = f.st.w2;
#pragma unroll
  for (int k = 2; k < NS; ++k) f.st.d[k] = __dadd_rn(f.st.d[k], slow[k]);

  __syncthreads();
  if constexpr (DIRECT) {
    // the block's exact words straight into the persistent accumulators
    // (integer sums: the order of the blocks does not matter)
    if (UNIT) {
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const unsigned c = f.sbins[i];
        if (c) atomicAdd(&p.g_unit[i], (unsigned long long)c);
      }
    } else {
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const unsigned lo = f.sbins[2 * i], hi = f.sbins[2 * i + 1];
        if (lo) atomicAdd(&p.g_lo[i], (unsigned long long)lo);
        if (hi) atomicAdd(reinterpret_cast<unsigned long long*>(&p.g_hi[i]), (unsigned long long)hi);
        if (p.track_counts) {
          const unsigned c = f.sbins[2 * nb + i];
          if (c) atomicAdd(&p.g_count[i], (unsigned long long)c);
        }
      }
    }
  } else if (SMEM) {
    if (UNIT) {
      unsigned* out = reinterpret_cast<unsigned*>(p.part_bins) + (size_t)blockIdx.x * nb;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) out[i] = f.sbins[i];
    } else {
      uint4* out = reinterpret_cast<uint4*>(p.part_bins) + (size_t)blockIdx.x * nb;
      if (ACC == ACC_FX) {
        // {low word, next word, top word (kept in global), entries}
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
          out[i] = make_uint4(f.sbins[2 * i], f.sbins[2 * i + 1], 0u, p.track_counts ? f.sbins[2 * nb + i] : 0u);
      } else if (ACC == ACC_F32C) {
        // {hi + lo in binary64, entries}: the reduction sums blocks in binary64
        double2* out2 = reinterpret_cast<double2*>(p.part_bins) + (size_t)blockIdx.x * nb;
        const float* sf = reinterpret_cast<const float*>(f.sbins);
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
          out2[i] = make_double2(__dadd_rn((double)sf[2 * i], (double)sf[2 * i + 1]),
                                 p.track_counts ? (double)f.sbins[2 * nb + i] : 0.0);
      } else {
        const uint4* sb4 = reinterpret_cast<const uint4*>(f.sbins);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) out[i] = sb4[i];
      }
    }
  }
  if (SW2 && SMEM && (ACC == ACC_FX || ACC == ACC_F32C)) {
    const float* sf = reinterpret_cast<const float*>(f.sbins) + (p.track_counts ? 3 : 2) * nb;
    double* out = p.part_sumw2 + (size_t)blockIdx.x * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      out[i] = __dadd_rn((double)sf[2 * i], (double)sf[2 * i + 1]);
  }
  block_reduce_stats<NS>(f.st.d, p.part_stats + (size_t)blockIdx.x * kMaxStats, sred);
  if constexpr (DIRECT) {
    // the last block to finish adds the statistics partials, in block
    // order with a fixed shuffle tree (k_reduce's order), and resets the
    // ticket for the next fill
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
      __threadfence();
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int k = 2 + warp; k < p.nstats; k += blockDim.x >> 5) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s = __dadd_rn(s, __ldcg(p.part_stats + (size_t)b * kMaxStats + k));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
        if (lane == 0) p.g_stats[k] = __dadd_rn(p.g_stats[k], s);
      }
      if (threadIdx.x == 0) *p.ticket = 0u;
    }
  }
}

// Reduce: grid (bin tiles) x (slices of partials).  Thread (tile, slice, t)
// sums bin g over partials [slice*r.slice, ...) and merges the result into
// the persistent accumulators -- with integer atomics for the exact modes
// (order-independent), with binary64 atomics for the binary64 mode.  CTA
// (0, 0) also adds the statistics partials, in block order, with a fixed
// shuffle tree (deterministic).
__global__ void __launch_bounds__(256) k_reduce(const ReduceParams r) {
  const long long nb = r.nbins_total;
  if (r.part_bins != nullptr) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int b0 = blockIdx.y * r.slice;
    const int b1 = min(r.nblocks, b0 + r.slice);
    if (g < nb && b0 < b1) {
      if (r.mode == ACC_UNIT) {
        const unsigned* pb = reinterpret_cast<const unsigned*>(r.part_bins);
        unsigned long long c = 0;
        for (int b = b0; b < b1; ++b) c += pb[(size_t)b * nb + g];
        if (c) atomicAdd(&r.g_unit[g], c);
      } else if (r.mode == ACC_FX) {
        const uint4* pb = reinterpret_cast<const uint4*>(r.part_bins);
        __int128 acc = 0;
        unsigned long long c = 0;
        for (int b = b0; b < b1; ++b) {
          const uint4 v = pb[(size_t)b * nb + g];
          acc += (__int128)(((unsigned long long)v.y << 32) | v.x) + ((__int128)(int)v.z << 64);
          c += v.w;
        }
        const unsigned long long lo = (unsigned long long)(acc & (__int128)0xFFFFFFFFull);
        const long long hi = (long long)(acc >> 32);
        if (lo) atomicAdd(&r.g_lo[g], lo);
        if (hi) atomicAdd(reinterpret_cast<unsigned long long*>(&r.g_hi[g]), (unsigned long long)hi);
        if (r.track_counts && c) atomicAdd(&r.g_count[g], c);
      } else {
        const double2* pb = reinterpret_cast<const double2*>(r.part_bins);
        double s = 0.0, c = 0.0;
        for (int b = b0; b < b1; ++b) {
          const double2 v = pb[(size_t)b * nb + g];
          s = __dadd_rn(s, v.x);
          c = __dadd_rn(c, v.y);
        }
        atomicAdd(&r.g_f64[g], s);
        if (r.track_counts && c != 0.0) atomicAdd(&r.g_count[g], (unsigned long long)c);
      }
      if (r.part_sumw2 != nullptr) {
        double s2 = 0.0;
        for (int b = b0; b < b1; ++b) s2 = __dadd_rn(s2, r.part_sumw2[(size_t)b * nb + g]);
        if (s2 != 0.0) atomicAdd(&r.g_sumw2[g], s2);
      }
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 2 + warp; k < r.nstats; k += blockDim.x >> 5) {
      double s = 0.0;
      for (int b = lane; b < r.nblocks; b += 32) s = __dadd_rn(s, r.part_stats[(size_t)b * kMaxStats + k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
      if (lane == 0) r.g_stats[k] = __dadd_rn(r.g_stats[k], s);
    }
  }
}

// Fold the low-word sums into the high words so neither can overflow.
__global__ void k_normalize_fx(unsigned long long* g_lo, long long* g_hi, long long nb) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < nb;
       g += (long long)gridDim.x * blockDim.x) {
    const unsigned long long lo = g_lo[g];
    g_hi[g] += (long long)(lo >> 32);
    g_lo[g] = lo & 0xFFFFFFFFull;
  }
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_locate(const FillParams p, long long* __restrict__ out) {
  const long long n = p.n;
  const int stride1 = p.ax[0].nbins + 2;
  const int stride2 = NDIM >= 2 ? stride1 * (p.ax[1].nbins + 2) : 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    long long g = 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const unsigned long long b = dbits(__ldcs(p.col[d] + i));
      const int k = locate_axis(p.ax[d], p.ax[d].T, nullptr, p.ax[d].bk.cnt, b, hi24(b), in_f32(exp_field(b)));
      g += (long long)k * (d == 0 ? 1 : (d == 1 ? stride1 : stride2));
    }
    out[i] = g;
  }
}

template <int NDIM, int ACC, bool SMEM>
const void* fill_fn(int loc, bool sw2, bool expr, bool direct) {
  if constexpr (NDIM <= 2) {
    // Filter/Define fills (1D and 2D; run-time locate)
    if (expr) return sw2 ? nullptr : reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, -1, false, true>);
  } else {
    if (expr) return nullptr;
  }
  if constexpr (ACC != ACC_UNIT) {
    // the per-bin sum of w^2 has its own kernels (run-time locate): the
    // other fills keep none of its code
    if (sw2) return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, -1, true, false>);
  }
  if constexpr (NDIM > 1) {
    return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, -1, false, false>);
  } else {
    if constexpr (SMEM && (ACC == ACC_UNIT || ACC == ACC_FX)) {
      if (direct) {
        if (loc == LOC_AFFINE) return reinterpret_cast<const void*>(&k_fill<1, ACC, true, LOC_AFFINE, false, false, true>);
        if (loc == LOC_LEARNED)
          return reinterpret_cast<const void*>(&k_fill<1, ACC, true, LOC_LEARNED, false, false, true>);
        if (loc == LOC_BUCKET) return reinterpret_cast<const void*>(&k_fill<1, ACC, true, LOC_BUCKET, false, false, true>);
        if (loc == LOC_BSEARCH)
          return reinterpret_cast<const void*>(&k_fill<1, ACC, true, LOC_BSEARCH, false, false, true>);
        return nullptr;
      }
    }
    if (loc == LOC_AFFINE) return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, LOC_AFFINE, false, false>);
    if (loc == LOC_LEARNED) return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, LOC_LEARNED, false, false>);
    if (loc == LOC_BUCKET) return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, LOC_BUCKET, false, false>);
    if constexpr (ACC != ACC_UNIT) {
      if (loc == kLocBucketHiSingle)
        return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, kLocBucketHiSingle, false, false>);
    }
    return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM, LOC_BSEARCH, false, false>);
  }
}

// 1D kernels are specialised per locate mode; ND kernels choose per axis at run time.
const void* pick_fill(int ndim, int acc, bool smem, int loc, bool sw2, bool expr, bool direct) {
#define HGB_PICK(N, A)                                                                   \
  if (ndim == N && acc == A)                                                             \
    return smem ? fill_fn<N, A, true>(loc, sw2, expr, direct) : fill_fn<N, A, false>(loc, sw2, expr, direct);
  HGB_PICK(1, ACC_UNIT)
  HGB_PICK(1, ACC_FX)
  HGB_PICK(1, ACC_F64)
  HGB_PICK(1, ACC_F32C)
  HGB_PICK(2, ACC_UNIT)
  HGB_PICK(2, ACC_FX)
  HGB_PICK(2, ACC_F64)
  HGB_PICK(2, ACC_F32C)
  HGB_PICK(3, ACC_UNIT)
  HGB_PICK(3, ACC_FX)
  HGB_PICK(3, ACC_F64)
  HGB_PICK(3, ACC_F32C)
#undef HGB_PICK
  return nullptr;
}

}  // namespace

size_t part_bin_bytes(int acc_mode, int /*track_counts*/) { return acc_mode == ACC_UNIT ? 4 : 16; }

size_t smem_bin_bytes(int acc_mode, int track_counts, int sumw2) {
  if (acc_mode == ACC_UNIT) return 4;
  if (acc_mode == ACC_FX || acc_mode == ACC_F32C) return (track_counts ? 12 : 8) + (sumw2 ? 8 : 0);
  return 16;
}

// The first axis's locate as a kernel-template value (the specialised bucket
// kernel serves weighted fills only).
int fill_loc(const FillParams& p, int acc_mode) {
  const AxisDev& a = p.ax[0];
  if (acc_mode != ACC_UNIT && a.mode == LOC_BUCKET && a.bk.key_map && a.bk.shift >= 32 && a.bk.single)
    return kLocBucketHiSingle;
  return a.mode;
}

// The kernel of a fill.
const void* fill_kernel(const FillParams& p, int acc_mode) {
  return pick_fill(p.ndim, acc_mode, p.smem_bins != 0, fill_loc(p, acc_mode), p.sumw2 != 0, p.ex.nsrc > 0,
                   p.direct_flush != 0);
}

// Whether a fill has a direct-flush kernel: 1D, exact fixed-point or
// unit-count shared bins, no sum of w^2, no Filter/Define; the specialised
// bucket-pair kernel keeps the reduce.
bool fill_direct_ok(const FillParams& p, int acc_mode) {
  return p.ndim == 1 && p.smem_bins && !p.sumw2 && p.ex.nsrc == 0 && (acc_mode == ACC_UNIT || acc_mode == ACC_FX) &&
         fill_loc(p, acc_mode) != kLocBucketHiSingle;
}

int plan_fill(const FillParams& p, int acc_mode, int sm_count, LaunchShape* shape) {
  const void* fn = fill_kernel(p, acc_mode);
  if (fn == nullptr) return -1;
  const int block = 256;
  size_t smem = (((size_t)p.table_keys * 12 + 15) & ~(size_t)15) + (((size_t)p.table_bk * 4 + 15) & ~(size_t)15);
  if (p.smem_bins) smem += (size_t)p.nbins_total * smem_bin_bytes(acc_mode, p.track_counts, p.sumw2);
  {  // always: it also loads the kernel before the occupancy query
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess) return -2;
  if (per_sm < 1) return -3;
  const long long want = (p.n + 2LL * block - 1) / (2LL * block);
  long long grid = (long long)per_sm * sm_count;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  shape->grid = (int)grid;
  shape->block = block;
  shape->smem = smem;
  return 0;
}

int launch_fill(const FillParams& p, int acc_mode, const LaunchShape& s, void* stream) {
  const void* fn = fill_kernel(p, acc_mode);
  if (fn == nullptr) return -1;
  void* args[] = {const_cast<FillParams*>(&p)};
  const cudaError_t e = cudaLaunchKernel(fn, dim3(s.grid), dim3(s.block), args, s.smem, (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : -2;
}

int launch_reduce(const ReduceParams& r0, void* stream) {
  ReduceParams r = r0;
  long long tiles = (r.nbins_total + 255) / 256;
  int slices = 1;
  if (r.part_bins != nullptr) {
    // 8 partials per thread: the reduce of a 608-block fill of 1000 bins
    // then runs 4 x 76 blocks (the summing thread's loads are the latency;
    // 32 partials per thread took 4 us more per fill call)
    r.slice = 8;
    slices = (r.nblocks + r.slice - 1) / r.slice;
    if (slices > 65535) slices = 65535;
    r.slice = (r.nblocks + slices - 1) / slices;
  } else {
    tiles = 1;
    r.slice = r.nblocks;
  }
  if (tiles > 65535LL * 16) return -1;
  dim3 grid((unsigned)tiles, (unsigned)slices);
  k_reduce<<<grid, 256, 0, (cudaStream_t)stream>>>(r);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_normalize_fx(unsigned long long* g_lo, long long* g_hi, long long nbins, void* stream) {
  long long blocks = (nbins + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_normalize_fx<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(g_lo, g_hi, nbins);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_locate(const FillParams& p, long long* out, void* stream) {
  long long blocks = (p.n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  if (blocks < 1) blocks = 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (p.ndim == 1)
    k_locate<1><<<(int)blocks, 256, 0, s>>>(p, out);
  else if (p.ndim == 2)
    k_locate<2><<<(int)blocks, 256, 0, s>>>(p, out);
  else
    k_locate<3><<<(int)blocks, 256, 0, s>>>(p, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
