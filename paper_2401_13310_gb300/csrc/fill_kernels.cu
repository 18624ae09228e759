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
//  * find-bin is integer-only: every axis is a table of exact threshold keys
//    (see hist_internal.h).  Fixed axes take an FP32 estimate built from the
//    coordinate's bits with integer operations and correct it by one compare
//    each way; variable axes binary-search the keys.  No binary64 arithmetic
//    runs per event (on GB300 the binary64 pipe issues fewer than two
//    operations per clock per SM, about 1/60 of the FP32 rate).
//  * weighted bins are summed exactly in fixed point: |w| in the window
//    [2^(e-1023), 2^(e-1007)) (e = fx_elo) becomes a 64-bit integer multiple
//    of 2^(e-1065) (truncation error <= 2^-42 |w|), added to a 96-bit
//    per-block accumulator held as three u32 words in shared memory with
//    32-bit atomics that propagate carries (u32 shared atomics sustain about
//    7 per clock per SM, against 0.7-1 for binary64 ones and 1.5 for 64-bit
//    ones).  The sum is exact and independent of the order of the atomics.
//    Other weights take a slow path (binary64 atomic in global memory).
//  * the statistics terms are formed and summed per thread in FP32
//    double-word arithmetic (error-free products with FMA, TwoSum
//    accumulation), flushed to binary64 every 64 events, reduced across the
//    block with warp shuffles and written as one partial per block; a second
//    kernel adds the partials in block order (deterministic).
//  * per-block bin partials are written to scratch and summed by the same
//    second kernel, which replaces the grid-wide atomic merge.
//
// Nothing here is compiled with FMA contraction (-fmad=false); every
// error-free transformation uses explicit round-to-nearest intrinsics.

#include <cuda_runtime.h>

#include <cstdint>

#include "hist_internal.h"

namespace hgb {
namespace {

constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kExpInf = 0x7FF0000000000000ull;
constexpr unsigned long long kMant = 0x000FFFFFFFFFFFFFull;
constexpr unsigned long long kHidden = 0x0010000000000000ull;
constexpr int kFlushIters = 32;  // two events per iteration: flush every 64 events

__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// Ordered key of a binary64: compares like the double; -0 and +0 both map to
// 0; every NaN maps to kNanKey, above +inf (the overflow bin).
__device__ __forceinline__ long long key_of(unsigned long long b) {
  unsigned long long mag = b & kMag;
  long long k = (long long)mag;
  k = ((long long)b < 0) ? -k : k;
  return (mag > kExpInf) ? kNanKey : k;
}

// FP32 value of a binary64 with the mantissa truncated to 23 bits, built with
// integer operations (a binary64 -> FP32 conversion would use the binary64
// pipe).  |x| < 2^-126 gives +-0, |x| >= 2^128 (and inf/NaN) gives +-2^127.
__device__ __forceinline__ float est_float(unsigned long long b) {
  unsigned hi = (unsigned)(b >> 32);
  unsigned sgn = hi & 0x80000000u;
  unsigned e = (hi >> 20) & 0x7FFu;
  unsigned f = ((unsigned)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu;
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7F000000u : f;
  return __uint_as_float(f | sgn);
}

// Largest k in [0, nkeys) with T[k] <= key (T[0] = INT64_MIN).
__device__ __forceinline__ int bsearch_keys(const long long* T, int nkeys, long long key) {
  int base = 0, len = nkeys;
  while (len > 1) {
    int half = len >> 1;
    base = (T[base + half] <= key) ? base + half : base;
    len -= half;
  }
  return base;
}

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((unsigned)h << 16); }

// Bin of one coordinate on one axis (Sec. 3.1 step 1), exact.
__device__ __forceinline__ int locate_axis(const AxisDev& a, const long long* T, unsigned long long b) {
  const long long key = key_of(b);
  if (a.mode == LOC_AFFINE) {
    float v = fmaf(est_float(b), a.scale, a.offset);
    v = fminf(fmaxf(v, 0.0f), (float)(a.nbins + 1));
    int k = (int)(__float_as_uint(__fadd_rd(v, 12582912.0f)) - 0x4B400000u);
    if (key < T[k]) {
      --k;
      if (key < T[k]) k = bsearch_keys(T, a.nbins + 2, key);
    } else if (key >= T[k + 1]) {
      ++k;
      if (key >= T[k + 1]) k = bsearch_keys(T, a.nbins + 2, key);
    }
    return k;
  }
  if (a.mode == LOC_LEARNED) {
    // Piecewise-linear index model: k^ = base[s] + th0[s] + th1[s] * t,
    // t = fractional position in segment s; then an exact search inside the
    // certified window; the full binary search judges any miss.
    const LearnedDev& m = a.lm;
    float u = (est_float(b) - m.u0) * m.u_scale;
    u = fminf(fmaxf(u, 0.0f), (float)m.nseg - 0.5f);
    int s = (int)u;
    float t = u - (float)s;
    float kh = (float)m.base[s] + bf16_to_f32(m.th0[s]) + bf16_to_f32(m.th1[s]) * t;
    int k0 = (int)floorf(kh + 0.5f);
    int lo = k0 - m.window, hi = k0 + m.window;
    lo = lo < 0 ? 0 : lo;
    hi = hi > a.nbins + 1 ? a.nbins + 1 : hi;
    if (lo <= hi && T[lo] <= key && key < T[hi + 1]) {
      return lo + bsearch_keys(T + lo, hi - lo + 1, key);
    }
    return bsearch_keys(T, a.nbins + 2, key);
  }
  return bsearch_keys(T, a.nbins + 2, key);
}

// ---------------------------------------------------------------- FP32 double-word

struct FF {
  float hi, lo;
};

// Split a binary64 with |x| in [2^-40, 2^40) or x = +-0 into hi + lo: hi
// holds the leading 24 significant bits, lo the remaining 29 rounded to 24
// (|x - hi - lo| <= 2^-48 |x|).  Integer operations and one u32 -> f32
// conversion only.
__device__ __forceinline__ FF ff_from_bits(unsigned long long b) {
  unsigned hi32 = (unsigned)(b >> 32);
  unsigned sgn = hi32 & 0x80000000u;
  unsigned e = (hi32 >> 20) & 0x7FFu;
  unsigned fh = (((unsigned)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu) | sgn;
  float lo = __fmul_rn(__uint2float_rn((unsigned)b & 0x1FFFFFFFu), __uint_as_float((e - 948u) << 23));
  unsigned fl = __float_as_uint(lo) | sgn;
  const bool zero = (b & kMag) == 0;
  FF r;
  r.hi = zero ? 0.0f : __uint_as_float(fh);
  r.lo = zero ? 0.0f : __uint_as_float(fl);
  return r;
}

// True when |x| is in [2^-40, 2^40) or x = +-0: the double-word path is exact
// enough and no product of statistics terms over- or underflows FP32.
__device__ __forceinline__ bool ff_ok(unsigned long long b) {
  unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  return (e - 983u) < 80u || (b & kMag) == 0;
}

// a * b as an unevaluated sum p + e (the a.lo * b.lo term, <= 2^-48 |ab|, is dropped).
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}

// s += t with TwoSum on the high parts (Knuth): the rounding error of
// s.hi + t.hi is recovered exactly and folded into s.lo.
__device__ __forceinline__ void ff_acc(FF& s, FF t) {
  float sum = __fadd_rn(s.hi, t.hi);
  float bp = __fsub_rn(sum, s.hi);
  float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(sum, bp)), __fsub_rn(t.hi, bp));
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, err));
  s.hi = sum;
}

__device__ __forceinline__ double ff_to_double(FF s) { return __dadd_rn((double)s.hi, (double)s.lo); }

// ---------------------------------------------------------------- fixed point

// Weight -> signed fixed-point integer V = trunc(|w| * 2^(1065 - elo)) * sign.
// Returns false (slow path) unless w = +-0 or its biased exponent is in
// [elo, elo + 16).  |V| < 2^58.
__device__ __forceinline__ bool fx_of(unsigned long long wb, int elo, long long* V) {
  const unsigned long long mag = wb & kMag;
  if (mag == 0) {
    *V = 0;
    return true;
  }
  const unsigned e = (unsigned)(wb >> 52) & 0x7FFu;
  if (e - (unsigned)elo >= 16u) return false;
  const unsigned long long M = (wb & kMant) | kHidden;
  const int s = (int)e - elo - 10;
  const unsigned long long U = (s >= 0) ? (M << s) : (M >> (-s));
  *V = ((long long)wb < 0) ? -(long long)U : (long long)U;
  return true;
}

// a[2]:a[1]:a[0] += V (96-bit two's complement) with 32-bit shared atomics.
// Each atomic returns the old word, so the carry it produced is known
// exactly; the final words equal the exact sum modulo 2^96 for any
// interleaving of concurrent adds.
__device__ __forceinline__ void smem_add96(unsigned* a, long long V) {
  const unsigned v0 = (unsigned)V;
  const unsigned v1 = (unsigned)((unsigned long long)V >> 32);
  const unsigned v2 = (unsigned)(V >> 63);
  const unsigned o0 = atomicAdd(&a[0], v0);
  const unsigned c0 = (o0 + v0 < o0) ? 1u : 0u;
  const unsigned a1 = v1 + c0;
  unsigned c1 = (a1 < c0) ? 1u : 0u;
  const unsigned o1 = atomicAdd(&a[1], a1);
  c1 |= (o1 + a1 < o1) ? 1u : 0u;
  const unsigned a2 = v2 + c1;
  if (a2 != 0u) atomicAdd(&a[2], a2);
}

// ---------------------------------------------------------------- statistics

// Per-thread statistics accumulator.  Slot numbering (stats[k]):
// 1 sum w, 2 sum w^2, 3 sum wx, 4 sum wx^2, 5 sum wy, 6 sum wy^2, 7 sum wxy,
// 8 sum wz, 9 sum wz^2, 10 sum wxz, 11 sum wyz.  Slot 0 (the entry count) is
// added on the host.
template <int NDIM, bool UNIT>
struct StatAcc {
  static constexpr int NS = NDIM == 1 ? 5 : (NDIM == 2 ? 8 : 12);
  FF s[NS];
  double d[NS];
  unsigned cnt;  // unit weights: in-range entries (sum w = sum w^2)

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      s[k].hi = 0.0f;
      s[k].lo = 0.0f;
      d[k] = 0.0;
    }
    cnt = 0;
  }

  // Double-word path: coordinates (and weight) already split.
  __device__ __forceinline__ void add_ff(const FF* c, FF W) {
    if (UNIT) {
      ++cnt;
      ff_acc(s[3], c[0]);
      ff_acc(s[4], ff_mul(c[0], c[0]));
      if (NDIM >= 2) {
        ff_acc(s[5], c[1]);
        ff_acc(s[6], ff_mul(c[1], c[1]));
        ff_acc(s[7], ff_mul(c[0], c[1]));
      }
      if (NDIM >= 3) {
        ff_acc(s[8], c[2]);
        ff_acc(s[9], ff_mul(c[2], c[2]));
        ff_acc(s[10], ff_mul(c[0], c[2]));
        ff_acc(s[11], ff_mul(c[1], c[2]));
      }
    } else {
      ff_acc(s[1], W);
      ff_acc(s[2], ff_mul(W, W));
      const FF WX = ff_mul(W, c[0]);
      ff_acc(s[3], WX);
      ff_acc(s[4], ff_mul(WX, c[0]));
      if (NDIM >= 2) {
        const FF WY = ff_mul(W, c[1]);
        ff_acc(s[5], WY);
        ff_acc(s[6], ff_mul(WY, c[1]));
        ff_acc(s[7], ff_mul(WX, c[1]));
        if (NDIM >= 3) {
          const FF WZ = ff_mul(W, c[2]);
          ff_acc(s[8], WZ);
          ff_acc(s[9], ff_mul(WZ, c[2]));
          ff_acc(s[10], ff_mul(WX, c[2]));
          ff_acc(s[11], ff_mul(WY, c[2]));
        }
      }
    }
  }

  // binary64 path (rare: coordinates or weight outside the double-word range,
  // non-finite values with HIST_STAT_OVERFLOWS).  Terms rounded as in the
  // definition: w*x*x = (w*x)*x.
  __device__ __forceinline__ void add_f64(const double* c, double w) {
    const double wx = __dmul_rn(w, c[0]);
    d[1] = __dadd_rn(d[1], w);
    d[2] = __dadd_rn(d[2], __dmul_rn(w, w));
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

  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      d[k] = __dadd_rn(d[k], ff_to_double(s[k]));
      s[k].hi = 0.0f;
      s[k].lo = 0.0f;
    }
    if (UNIT) {
      d[1] = __dadd_rn(d[1], (double)cnt);
      d[2] = __dadd_rn(d[2], (double)cnt);
      cnt = 0;
    }
  }
};

// Block-wide sum of the per-thread binary64 statistics (warp shuffles, then
// one pass over the warps in order); thread 0 writes the block's partial.
template <int NS>
__device__ __forceinline__ void block_reduce_stats(double* d, double* out, double* sred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 1; k < NS; ++k) {
    double v = d[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sred[warp * kMaxStats + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxStats) {
    const int k = threadIdx.x;
    double v = 0.0;
    if (k >= 1 && k < NS)
      for (int wi = 0; wi < nwarps; ++wi) v = __dadd_rn(v, sred[wi * kMaxStats + k]);
    out[k] = v;
  }
}

// ---------------------------------------------------------------- loads

__device__ __forceinline__ void load2(const double* __restrict__ p, long long i, bool vec, double& a,
                                      double& b) {
  if (vec) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p + i));
    a = v.x;
    b = v.y;
  } else {
    a = __ldcs(p + i);
    b = __ldcs(p + i + 1);
  }
}

// ---------------------------------------------------------------- fill kernel

struct SmemLayout {
  long long* keys;
  unsigned* bins;
};

// One event: locate on every axis, accumulate into the bins, update the
// statistics.  SMEM selects per-block shared bins vs global atomics.
template <int NDIM, int ACC, bool SMEM>
__device__ __forceinline__ void do_event(const FillParams& p, const long long* const* Tax, unsigned* sbins,
                                         double* sbins_f64, const double* c, double w,
                                         StatAcc<NDIM, ACC == ACC_UNIT>& st, int stride1, int stride2) {
  unsigned long long cb[NDIM];
  int k[NDIM];
  bool in_range = true;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    cb[d] = dbits(c[d]);
    k[d] = locate_axis(p.ax[d], Tax[d], cb[d]);
    in_range = in_range && (k[d] >= 1) && (k[d] <= p.ax[d].nbins);
  }
  long long g = k[0];
  if (NDIM >= 2) g += (long long)k[1] * stride1;
  if (NDIM >= 3) g += (long long)k[2] * stride2;

  const unsigned long long wb = dbits(w);
  // ---- step 2: the bin
  if (ACC == ACC_UNIT) {
    if (SMEM)
      atomicAdd(&sbins[g], 1u);
    else
      atomicAdd(&p.g_unit[g], 1ull);
  } else if (ACC == ACC_FX) {
    long long V;
    if (fx_of(wb, p.fx_elo, &V)) {
      if (SMEM) {
        if (V != 0) smem_add96(&sbins[4 * g], V);
        if (p.track_counts) atomicAdd(&sbins[4 * g + 3], 1u);
      } else {
        if (V != 0) {
          atomicAdd(&p.g_lo[g], (unsigned long long)(unsigned)V);
          atomicAdd(reinterpret_cast<unsigned long long*>(&p.g_hi[g]), (unsigned long long)(V >> 32));
        }
        if (p.track_counts) atomicAdd(&p.g_count[g], 1ull);
      }
    } else {
      atomicAdd(&p.g_f64[g], w);
      if (p.track_counts) {
        if (SMEM)
          atomicAdd(&sbins[4 * g + 3], 1u);
        else
          atomicAdd(&p.g_count[g], 1ull);
      }
    }
  } else if (ACC == ACC_F64) {
    if (SMEM) {
      atomicAdd(&sbins_f64[2 * g], w);
      if (p.track_counts) atomicAdd(&sbins_f64[2 * g + 1], 1.0);
    } else {
      atomicAdd(&p.g_f64[g], w);
      if (p.track_counts) atomicAdd(&p.g_count[g], 1ull);
    }
  }
  // ---- step 3: statistics
  if (!(in_range || p.stat_overflows)) return;
  if (ACC == ACC_F64) {
    st.add_f64(c, w);
    return;
  }
  bool fast = true;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) fast = fast && ff_ok(cb[d]);
  if (ACC == ACC_FX) fast = fast && ff_ok(wb);
  if (fast) {
    FF cf[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) cf[d] = ff_from_bits(cb[d]);
    FF W;
    if (ACC == ACC_UNIT) {
      W.hi = 1.0f;
      W.lo = 0.0f;
    } else {
      W = ff_from_bits(wb);
    }
    st.add_ff(cf, W);
  } else {
    st.add_f64(c, ACC == ACC_UNIT ? 1.0 : w);
  }
}

template <int NDIM, int ACC, bool SMEM>
__global__ void __launch_bounds__(256) k_fill(const FillParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nkeys = p.table_keys;
  long long* skeys = reinterpret_cast<long long*>(smem_raw);
  unsigned char* after_keys = smem_raw + (((size_t)nkeys * 8 + 15) & ~(size_t)15);
  unsigned* sbins = reinterpret_cast<unsigned*>(after_keys);
  double* sbins_f64 = reinterpret_cast<double*>(after_keys);
  __shared__ double sred[8 * kMaxStats];

  // stage threshold keys
  for (int i = threadIdx.x; i < nkeys; i += blockDim.x) skeys[i] = p.T_concat[i];
  const long long* Tax[NDIM];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) Tax[d] = (p.ax[d].smem_off >= 0) ? skeys + p.ax[d].smem_off : p.ax[d].T;

  const int nb = (int)p.nbins_total;
  if (SMEM) {
    const int words = (ACC == ACC_UNIT) ? nb : (ACC == ACC_FX ? 4 * nb : 4 * nb);
    for (int i = threadIdx.x; i < words; i += blockDim.x) sbins[i] = 0u;
  }
  __syncthreads();

  const int stride1 = p.ax[0].nbins + 2;
  const int stride2 = NDIM >= 2 ? stride1 * (p.ax[1].nbins + 2) : 0;

  StatAcc<NDIM, ACC == ACC_UNIT> st;
  st.init();

  const long long n = p.n;
  const long long tstride = 2LL * gridDim.x * blockDim.x;
  const bool vec = p.aligned != 0;
  int iters = 0;
  for (long long i = 2LL * (blockIdx.x * (long long)blockDim.x + threadIdx.x); i < n; i += tstride) {
    double c0[NDIM], c1[NDIM], w0 = 1.0, w1 = 1.0;
    const bool pair = (i + 1 < n);
    if (pair) {
#pragma unroll
      for (int d = 0; d < NDIM; ++d) load2(p.col[d], i, vec, c0[d], c1[d]);
      if (ACC != ACC_UNIT) load2(p.w, i, vec, w0, w1);
    } else {
#pragma unroll
      for (int d = 0; d < NDIM; ++d) c0[d] = __ldcs(p.col[d] + i);
      if (ACC != ACC_UNIT) w0 = __ldcs(p.w + i);
    }
    do_event<NDIM, ACC, SMEM>(p, Tax, sbins, sbins_f64, c0, w0, st, stride1, stride2);
    if (pair) do_event<NDIM, ACC, SMEM>(p, Tax, sbins, sbins_f64, c1, w1, st, stride1, stride2);
    if (++iters == kFlushIters) {
      if (ACC != ACC_F64) st.flush();
      iters = 0;
    }
  }
  if (ACC != ACC_F64) st.flush();

  __syncthreads();
  // per-block partial bins -> scratch
  if (SMEM) {
    if (ACC == ACC_UNIT) {
      unsigned* out = reinterpret_cast<unsigned*>(p.part_bins) + (size_t)blockIdx.x * nb;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) out[i] = sbins[i];
    } else if (ACC == ACC_FX) {
      uint4* out = reinterpret_cast<uint4*>(p.part_bins) + (size_t)blockIdx.x * nb;
      const uint4* sb4 = reinterpret_cast<const uint4*>(sbins);
      for (int i = threadIdx.x; i < nb; i += blockDim.x) out[i] = sb4[i];
    } else {
      double2* out = reinterpret_cast<double2*>(p.part_bins) + (size_t)blockIdx.x * nb;
      const double2* sb2 = reinterpret_cast<const double2*>(sbins_f64);
      for (int i = threadIdx.x; i < nb; i += blockDim.x) out[i] = sb2[i];
    }
  }
  block_reduce_stats<StatAcc<NDIM, ACC == ACC_UNIT>::NS>(st.d, p.part_stats + (size_t)blockIdx.x * kMaxStats,
                                                         sred);
}

// Sum of the per-block partials, in block order, into the persistent
// accumulators; block 0 also sums the statistics partials.
__global__ void __launch_bounds__(256) k_reduce(const ReduceParams r) {
  const long long nb = r.nbins_total;
  if (r.part_bins != nullptr) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < nb;
         g += (long long)gridDim.x * blockDim.x) {
      if (r.mode == ACC_UNIT) {
        const unsigned* pb = reinterpret_cast<const unsigned*>(r.part_bins);
        unsigned long long c = 0;
        for (int b = 0; b < r.nblocks; ++b) c += pb[(size_t)b * nb + g];
        r.g_unit[g] += c;
      } else if (r.mode == ACC_FX) {
        const uint4* pb = reinterpret_cast<const uint4*>(r.part_bins);
        __int128 acc = 0;
        unsigned long long c = 0;
        for (int b = 0; b < r.nblocks; ++b) {
          const uint4 v = pb[(size_t)b * nb + g];
          // sign-extend the 96-bit word triple
          const __int128 lo64 = (__int128)(((unsigned long long)v.y << 32) | v.x);
          const __int128 hi32 = (__int128)(int)v.z;
          acc += lo64 + (hi32 << 64);
          c += v.w;
        }
        r.g_lo[g] += (unsigned long long)(acc & (__int128)0xFFFFFFFFull);
        r.g_hi[g] += (long long)(acc >> 32);
        if (r.track_counts) r.g_count[g] += c;
      } else {
        const double2* pb = reinterpret_cast<const double2*>(r.part_bins);
        double s = 0.0, c = 0.0;
        for (int b = 0; b < r.nblocks; ++b) {
          const double2 v = pb[(size_t)b * nb + g];
          s = __dadd_rn(s, v.x);
          c = __dadd_rn(c, v.y);
        }
        r.g_f64[g] = __dadd_rn(r.g_f64[g], s);
        if (r.track_counts) r.g_count[g] += (unsigned long long)c;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < r.nstats && threadIdx.x >= 1) {
    const int k = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < r.nblocks; ++b) s = __dadd_rn(s, r.part_stats[(size_t)b * kMaxStats + k]);
    r.g_stats[k] = __dadd_rn(r.g_stats[k], s);
  }
}

// Fold the low-word sums into the high words so neither can overflow.
__global__ void k_normalize_fx(unsigned long long* g_lo, long long* g_hi, long long nb) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < nb; g += (long long)gridDim.x * blockDim.x) {
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
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long g = 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const int k = locate_axis(p.ax[d], p.ax[d].T, dbits(__ldcs(p.col[d] + i)));
      g += (long long)k * (d == 0 ? 1 : (d == 1 ? stride1 : stride2));
    }
    out[i] = g;
  }
}

template <int NDIM, int ACC, bool SMEM>
const void* fill_fn() {
  return reinterpret_cast<const void*>(&k_fill<NDIM, ACC, SMEM>);
}

const void* pick_fill(int ndim, int acc, bool smem) {
#define HGB_PICK(N, A)                                                       \
  if (ndim == N && acc == A) return smem ? fill_fn<N, A, true>() : fill_fn<N, A, false>();
  HGB_PICK(1, ACC_UNIT)
  HGB_PICK(1, ACC_FX)
  HGB_PICK(1, ACC_F64)
  HGB_PICK(2, ACC_UNIT)
  HGB_PICK(2, ACC_FX)
  HGB_PICK(2, ACC_F64)
  HGB_PICK(3, ACC_UNIT)
  HGB_PICK(3, ACC_FX)
  HGB_PICK(3, ACC_F64)
#undef HGB_PICK
  return nullptr;
}

}  // namespace

size_t part_bin_bytes(int acc_mode, int /*track_counts*/) {
  if (acc_mode == ACC_UNIT) return 4;
  return 16;
}

int plan_fill(const FillParams& p, int acc_mode, int sm_count, LaunchShape* shape) {
  const void* fn = pick_fill(p.ndim, acc_mode, p.smem_bins != 0);
  if (fn == nullptr) return -1;
  const int block = 256;
  size_t smem = (((size_t)p.table_keys * 8 + 15) & ~(size_t)15);
  if (p.smem_bins) smem += (size_t)p.nbins_total * part_bin_bytes(acc_mode, p.track_counts);
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess) return -2;
  if (per_sm < 1) return -3;
  long long want = (p.n + 2LL * block - 1) / (2LL * block);
  long long grid = (long long)per_sm * sm_count;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  shape->grid = (int)grid;
  shape->block = block;
  shape->smem = smem;
  return 0;
}

int launch_fill(const FillParams& p, int acc_mode, const LaunchShape& s, void* stream) {
  const void* fn = pick_fill(p.ndim, acc_mode, p.smem_bins != 0);
  if (fn == nullptr) return -1;
  void* args[] = {const_cast<FillParams*>(&p)};
  cudaError_t e = cudaLaunchKernel(fn, dim3(s.grid), dim3(s.block), args, s.smem, (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : -2;
}

int launch_reduce(const ReduceParams& r, void* stream) {
  long long blocks = (r.nbins_total + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  if (r.part_bins == nullptr) blocks = 1;
  k_reduce<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(r);
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
