// device_common.cuh -- device helpers shared by the fill kernels: ordered
// keys of binary64 values, FP32 views of binary64 bits, the exact find-bin
// paths (fixed-axis FP32 fast path with proven bound, threshold searches,
// learned model with certified window), FP32 double-word arithmetic and the
// exact fixed-point weight accumulation.  See fill_kernels.cu for the
// reasoning behind each piece.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hist_internal.h"
#include "learned_eval.cuh"

namespace hgb {
namespace {

constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kExpInf = 0x7FF0000000000000ull;
constexpr unsigned long long kMant = 0x000FFFFFFFFFFFFFull;
constexpr unsigned long long kHidden = 0x0010000000000000ull;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23

__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}


// Ordered key of a binary64: compares like the double; -0 and +0 both map to
// 0; every NaN maps to kNanKey, above +inf (the overflow bin).
__device__ __forceinline__ long long key_of(unsigned long long b) {
  const unsigned long long mag = b & kMag;
  long long k = (long long)mag;
  k = ((long long)b < 0) ? -k : k;
  return (mag > kExpInf) ? kNanKey : k;
}

// FP32 value of a binary64 with the significand truncated to 24 bits, built
// with integer operations (a binary64 -> FP32 conversion would use the
// binary64 pipe).  |x| < 2^-126 gives +-0, |x| >= 2^128 (and inf/NaN) +-2^127.
__device__ __forceinline__ float est_float(unsigned long long b) {
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sgn = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;
  unsigned f = ((unsigned)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu;
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7F000000u : f;
  return __uint_as_float(f | sgn);
}

// The same value without the saturation: only meaningful when in_f32(b).
__device__ __forceinline__ float hi24(unsigned long long b) {
  const unsigned hi = (unsigned)(b >> 32);
  return __uint_as_float((((unsigned)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u));
}

// Biased exponent field of a binary64, in place (bits 20..30 of the high word).
__device__ __forceinline__ unsigned exp_field(unsigned long long b) { return (unsigned)(b >> 32) & 0x7FF00000u; }

// |x| in [2^-126, 2^128): hi24 is exact truncation (zeros, subnormals,
// huge values, inf and NaN are all outside).
__device__ __forceinline__ bool in_f32(unsigned ef) { return ef - 0x38100000u < 0x0FE00000u; }

// |x| in [2^-40, 2^40): the double-word statistics path is accurate and no
// product of statistics terms over- or underflows FP32.
__device__ __forceinline__ bool in_ff(unsigned ef) { return ef - (983u << 20) < (80u << 20); }

// Largest k in [0, nkeys) with T[k] <= key (T[0] = INT64_MIN).
__device__ __forceinline__ int bsearch_keys(const long long* T, int nkeys, long long key) {
  int base = 0, len = nkeys;
  while (len > 1) {
    const int half = len >> 1;
    base = (T[base + half] <= key) ? base + half : base;
    len -= half;
  }
  return base;
}

// Largest k in [0, nkeys) with T[k] <= key, searching the 32-bit high words
// Thi[k] = T[k] >> 32 (half the bytes and compares of a 64-bit search), then
// stepping back over the few thresholds that share key's high word: any j
// with Thi[j] < key >> 32 has T[j] < key, so only equal high words need the
// full compare.
__device__ __forceinline__ int bsearch_hi(const long long* T, const int* Thi, int nkeys, long long key) {
  const int kh = (int)(key >> 32);
  int base = 0, len = nkeys;
  while (len > 1) {
    const int half = len >> 1;
    base = (Thi[base + half] <= kh) ? base + half : base;
    len -= half;
  }
  while (T[base] > key) --base;  // T[0] = INT64_MIN ends the walk
  return base;
}

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((unsigned)h << 16); }

// Exact bin from the thresholds, starting at a guess k0 in [0, nbins+1]:
// one step each way, then a full binary search if still not bracketed.
__device__ __noinline__ int locate_exact(const long long* T, int nbins, int k, unsigned long long b) {
  const long long key = key_of(b);
  if (key < T[k]) {
    --k;
    if (key < T[k]) k = bsearch_keys(T, nbins + 2, key);
  } else if (key >= T[k + 1]) {
    ++k;
    if (key >= T[k + 1]) k = bsearch_keys(T, nbins + 2, key);
  }
  return k;
}

// LOC_BUCKET: range tests on the key, the coordinate's bucket, then the
// bucket's own thresholds (at most a few) by binary lifting.  Exact: the map
// is monotone and the host placed every threshold with the same arithmetic.
__device__ __forceinline__ int locate_bucket(const AxisDev& a, const long long* T, const int* cnt,
                                             unsigned long long b, long long key) {
  int bk;
  if (a.bk.key_map && a.bk.shift > 0) {
    // the key map is monotone over every key (NaN's included) and T[1]
    // lies in bucket 0: clamped out-of-range keys land in the end buckets,
    // whose counts and thresholds give 0 and nbins + 1 -- no range tests
    if (a.bk.shift >= 32) {
      // key >> shift and kbase are 32-bit values: the same map on the key's
      // high word (the difference, after the lower clamp, is taken unsigned)
      const int hk = (int)(key >> 32) >> (a.bk.shift - 32);
      const int kb = (int)a.bk.kbase;
      bk = (int)min((unsigned)max(hk, kb) - (unsigned)kb, (unsigned)(a.bk.nbk - 1));
    } else {
      long long q = (key >> a.bk.shift) - a.bk.kbase;
      q = q < 0 ? 0 : (q > a.bk.nbk - 1 ? a.bk.nbk - 1 : q);
      bk = (int)q;
    }
  } else {
    if (key < a.bk.lo_key) return 0;
    if (key >= a.bk.hi_key) return a.nbins + 1;
    if (a.bk.key_map) {
      bk = (int)((key >> a.bk.shift) - a.bk.kbase);
    } else {
      const float t = fminf(fmaxf(__fmaf_rn(est_float(b), a.bk.scale, a.bk.offset), -1.0f), (float)a.bk.nbk);
      bk = __float2int_rd(t);
    }
    bk = min(max(bk, 0), a.bk.nbk - 1);
  }
  if (a.bk.single) {
    const longlong2 e = reinterpret_cast<const longlong2*>(cnt)[bk];
    return (int)e.y + (key >= e.x ? 1 : 0);
  }
  const int k = cnt[bk];
  const int n_in = cnt[bk + 1] - k;
  int pos = 0;
  for (int step = a.bk.top; step > 0; step >>= 1) {
    const int q = pos + step;
    if (q <= n_in && T[k + q] <= key) pos = q;
  }
  return k + pos;
}

// Bucket of a key under the key map of an axis (key_map set, shift > 0), as
// in locate_bucket.
__device__ __forceinline__ int key_bucket(const AxisDev& a, long long key) {
  if (a.bk.shift >= 32) {
    const int hk = (int)(key >> 32) >> (a.bk.shift - 32);
    const int kb = (int)a.bk.kbase;
    return (int)min((unsigned)max(hk, kb) - (unsigned)kb, (unsigned)(a.bk.nbk - 1));
  }
  long long q = (key >> a.bk.shift) - a.bk.kbase;
  q = q < 0 ? 0 : (q > a.bk.nbk - 1 ? a.bk.nbk - 1 : q);
  return (int)q;
}

// LOC_BUCKET for N coordinates at once, step by step, so that the table
// loads of the N events (in L2 when the tables are large) are in flight
// together rather than one event's chain after another's.  Same bins as
// locate_bucket.
template <int N>
__device__ __forceinline__ void locate_bucket_n(const AxisDev& a, const long long* T, const int* cnt,
                                                const unsigned long long* b, const long long* key, int* k) {
  if (!(a.bk.key_map && a.bk.shift > 0)) {
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = locate_bucket(a, T, cnt, b[i], key[i]);
    return;
  }
  int bk[N];
#pragma unroll
  for (int i = 0; i < N; ++i) bk[i] = key_bucket(a, key[i]);
  if (a.bk.single) {
    longlong2 e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) e[i] = reinterpret_cast<const longlong2*>(cnt)[bk[i]];
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = (int)e[i].y + (key[i] >= e[i].x ? 1 : 0);
    return;
  }
  int c0[N], n_in[N], pos[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    c0[i] = cnt[bk[i]];
    n_in[i] = cnt[bk[i] + 1] - c0[i];
    pos[i] = 0;
  }
  for (int step = a.bk.top; step > 0; step >>= 1) {
    long long t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = T[c0[i] + min(pos[i] + step, n_in[i])];  // (always a threshold of the bucket's range)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (pos[i] + step <= n_in[i] && t[i] <= key[i]) pos[i] += step;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) k[i] = c0[i] + pos[i];
}

// LOC_LEARNED: the trained index model's bin k0 when its two thresholds
// bracket the key (most events), else an exact search of the certified
// window around it; -1 when even the window misses (the caller then runs
// the full binary search).
__device__ __forceinline__ int locate_learned(const AxisDev& a, const long long* T, unsigned long long b,
                                              long long key) {
  const float kh = lm_eval(a.lm, est_float(b));
  const int k0 = min(max((int)floorf(__fadd_rn(kh, 0.5f)), 0), a.nbins + 1);
  if (T[k0] <= key && key < T[k0 + 1]) return k0;
  const int lo = max(k0 - a.lm.window, 0);
  const int hi = min(k0 + a.lm.window, a.nbins + 1);
  if (T[lo] <= key && key < T[hi + 1]) return lo + bsearch_keys(T + lo, hi - lo + 1, key);
  return -1;
}

// Bin of one coordinate on one axis (Sec. 3.1 step 1), exact.
// xf: the coordinate as FP32 (hi24), valid when in_f32 of its exponent field.
__device__ __forceinline__ int locate_axis(const AxisDev& a, const long long* T, const int* Thi, const int* cnt,
                                           unsigned long long b, float xf, bool f32ok) {
  if (a.mode == LOC_AFFINE) {
    // v estimates 1 + q; t = floor(v) + 1.5*2^23 exactly while |v| < 2^22.
    // Outside that range either v is an integer (fr = 0, not sure) or the
    // clamp below puts k in the right flow bin.
    const float v = __fmaf_rn(xf, a.scale, a.offset);
    const float t = __fadd_rd(v, kMagic);
    int k = (int)(__float_as_uint(t) - 0x4B400000u);  // (unsigned: no signed overflow for t < 0)
    const float fr = __fsub_rn(v, __fsub_rn(t, kMagic));
    const bool sure = f32ok && (fabsf(__fsub_rn(fr, 0.5f)) < 0.5f - a.eps);
    k = min(max(k, 0), a.nbins + 1);
    if (sure) return k;
    return locate_exact(T, a.nbins, k, b);
  }
  const long long key = key_of(b);
  if (a.mode == LOC_BUCKET) return locate_bucket(a, T, cnt, b, key);
  if (a.mode == LOC_LEARNED) {
    const int k = locate_learned(a, T, b, key);
    if (k >= 0) return k;
  }
  if (Thi != nullptr) return bsearch_hi(T, Thi, a.nbins + 2, key);
  return bsearch_keys(T, a.nbins + 2, key);
}

// Kernel-template value of the locate for LOC_BUCKET axes whose key map
// works on the key's high word (shift >= 32) with at most one threshold per
// bucket (a (threshold, count) pair table): the weighted 1D fills' most
// common variable-axis case, specialised so it runs without the map-type
// tests.
constexpr int kLocBucketHiSingle = 4;

// Find-bin with the axis mode fixed at compile time (LOC >= 0: the 1D
// kernels are specialised per mode so each keeps only its own path), or
// chosen at run time (LOC < 0).
template <int LOC>
__device__ __forceinline__ int locate_mode(const AxisDev& a, const long long* T, const int* Thi, const int* cnt,
                                           unsigned long long b, float xf, bool f32ok) {
  if (LOC < 0) return locate_axis(a, T, Thi, cnt, b, xf, f32ok);
  if (LOC == kLocBucketHiSingle) {  // locate_bucket's high-word map, then the pair
    const long long key = key_of(b);
    const int hk = (int)(key >> 32) >> (a.bk.shift - 32);
    const int kb = (int)a.bk.kbase;
    const int bk = (int)min((unsigned)max(hk, kb) - (unsigned)kb, (unsigned)(a.bk.nbk - 1));
    const longlong2 e = reinterpret_cast<const longlong2*>(cnt)[bk];
    return (int)e.y + (key >= e.x ? 1 : 0);
  }
  if (LOC == LOC_AFFINE) {  // as in locate_axis
    const float v = __fmaf_rn(xf, a.scale, a.offset);
    const float t = __fadd_rd(v, kMagic);
    int k = (int)(__float_as_uint(t) - 0x4B400000u);  // (unsigned: no signed overflow for t < 0)
    const float fr = __fsub_rn(v, __fsub_rn(t, kMagic));
    const bool sure = f32ok && (fabsf(__fsub_rn(fr, 0.5f)) < 0.5f - a.eps);
    k = min(max(k, 0), a.nbins + 1);
    if (sure) return k;
    return locate_exact(T, a.nbins, k, b);
  }
  const long long key = key_of(b);
  if (LOC == LOC_BUCKET) return locate_bucket(a, T, cnt, b, key);
  if (LOC == LOC_LEARNED) {
    const int k = locate_learned(a, T, b, key);
    if (k >= 0) return k;
  }
  if (Thi != nullptr) return bsearch_hi(T, Thi, a.nbins + 2, key);
  return bsearch_keys(T, a.nbins + 2, key);
}

// ---------------------------------------------------------------- FP32 double-word

struct FF {
  float hi, lo;
};

// hi + lo with hi = the leading 24 significant bits of x (hi24) and lo the
// remaining 29 bits rounded to 24 (|x - hi - lo| <= 2^-48 |x|), for |x| in
// [2^-40, 2^40).  Integer operations and one u32 -> f32 conversion only.
__device__ __forceinline__ FF ff_split(unsigned long long b, float hi) {
  const unsigned hi32 = (unsigned)(b >> 32);
  const float scale = __uint_as_float(((hi32 >> 20) - 948u) << 23);  // 2^(e-1075), sign bit shifted out
  const float lo = __fmul_rn(__uint2float_rn((unsigned)b & 0x1FFFFFFFu), scale);
  FF r;
  r.hi = hi;
  r.lo = __uint_as_float(__float_as_uint(lo) | (hi32 & 0x80000000u));
  return r;
}

// a * b as an unevaluated sum p + e (a.lo * b.lo, <= 2^-48 |ab|, is dropped).
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}

// s += t with TwoSum on the high parts (Knuth): the rounding error of
// s.hi + t.hi is recovered exactly and folded into s.lo.
__device__ __forceinline__ void ff_acc(FF& s, FF t) {
  const float sum = __fadd_rn(s.hi, t.hi);
  const float bp = __fsub_rn(sum, s.hi);
  const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(sum, bp)), __fsub_rn(t.hi, bp));
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, err));
  s.hi = sum;
}

// The same double-word arithmetic on two independent lanes at once, with
// Blackwell's packed FP32x2 instructions (two events per instruction; per
// lane the numerics are exactly those of the scalar forms above: a - b is
// computed as fma(b, -1, a), one rounding).
struct FF2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

__device__ __forceinline__ FF2 ff2_mul(FF2 a, FF2 b) {
  const float2 p = __fmul2_rn(a.hi, b.hi);
  float2 e = __ffma2_rn(a.hi, b.hi, __fmul2_rn(p, make_float2(-1.0f, -1.0f)));
  e = __ffma2_rn(a.hi, b.lo, e);
  e = __ffma2_rn(a.lo, b.hi, e);
  return {p, e};
}

__device__ __forceinline__ void ff2_acc(FF2& s, FF2 t) {
  const float2 sum = __fadd2_rn(s.hi, t.hi);
  const float2 bp = f2_sub(sum, s.hi);
  const float2 err = __fadd2_rn(f2_sub(s.hi, f2_sub(sum, bp)), f2_sub(t.hi, bp));
  s.lo = __fadd2_rn(s.lo, __fadd2_rn(t.lo, err));
  s.hi = sum;
}

// Exact FP32 -> binary64 widening with integer operations (the conversion
// instruction runs on the binary64 pipe at half its add rate).  Normal
// values and zeros only; the double-word parts here are never subnormal.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long mag =
      ((unsigned long long)(((u >> 23) & 0xFFu) + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)(((u & 0x7FFFFFFFu) == 0u) ? sgn : (sgn | mag)));
}

__device__ __forceinline__ double ff_to_double(FF s) {
  return __dadd_rn(f32_to_f64_bits(s.hi), f32_to_f64_bits(s.lo));
}

// ---------------------------------------------------------------- fixed point

// Weight -> signed fixed-point integer V = trunc(|w| * 2^(1065 - elo)) * sign.
// Returns false (slow path: zeros, tiny, huge, inf, NaN) unless the biased
// exponent is in [elo, elo + 16).  With the significand M (hidden bit
// included) pre-shifted left by 10, V = (M << 10) >> (20 - (e - elo)) --
// always a right shift by 5..20, so no bit of an in-window weight above
// 2^-42 |w| is lost.  |V| < 2^58.
__device__ __forceinline__ bool fx_of(unsigned long long wb, int elo, long long* V) {
  const unsigned rel = ((unsigned)(wb >> 52) & 0x7FFu) - (unsigned)elo;
  const unsigned long long M10 = ((wb << 10) & (kMant << 10)) | (kHidden << 10);
  const unsigned long long U = M10 >> ((20u - rel) & 63u);
  *V = ((long long)wb < 0) ? -(long long)U : (long long)U;
  return rel < 16u;
}

}  // namespace
}  // namespace hgb
