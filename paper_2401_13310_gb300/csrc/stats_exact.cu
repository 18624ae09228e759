// stats_exact.cu -- order-independent, exactly summed statistics.
//
// With HIST_STATS_EXACT every statistic is the exact sum of its rounded
// terms -- the terms of Sec. 3.1's statistics as the oracle rounds them:
// w, fl(w*w), fl(w*x), fl(fl(w*x)*x) in 1D; ROOT's TH2/TH3 sets add
// fl(w*y), fl(fl(w*y)*y), fl(fl(w*x)*y) in 2D and fl(w*z), fl(fl(w*z)*z),
// fl(fl(w*x)*z), fl(fl(w*y)*z) in 3D -- rounded once to binary64 on the
// host: the same bits whatever the launch shape, the order of the atomics
// or the way the events were split into fills.
//
// Each term t = +-m 2^(E-1075) (m the 53-bit significand) is an integer
// multiple of 2^g_s, g_s the statistic's grid, when E - 1075 >= g_s; it is
// added into six radix-2^32 limbs held in int64 registers (the register
// limbs absorb carries; each thread normalises them before the block and
// grid sums, which are integer additions and hence exact and associative).
// A term outside the grid's window (tiny, huge, subnormal) takes an escape
// path into a 72-limb accumulator spanning every finite double; NaN and
// infinite terms are counted instead.  One pass sums up to four statistics
// (their limbs fill the registers), so 2D and 3D fills take two and three
// passes over the bulk.

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {

constexpr int kThreads = 256;

struct Limbs {
  long long v[kExactLimbs];
};

// Adds t into the statistic's limbs (fast window) or the escape limbs.
__device__ __forceinline__ void exact_add(Limbs& L, double t, int g, const ExactParams& p, int stat,
                                          unsigned long long (&special)[3]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0x7FF) {  // NaN, +inf, -inf
    const int k = (b & kMant) ? 0 : (((long long)b < 0) ? 2 : 1);
    special[k] += 1;
    return;
  }
  if ((b & kMag) == 0) return;  // +-0
  const bool neg = (long long)b < 0;
  const unsigned long long m = (b & kMant) | (E ? kHidden : 0ull);
  const int e = (E ? E : 1) - 1075;  // t = +-m 2^e
  const int pos = e - g;
  if (E != 0 && pos >= 0 && pos <= kExactFastTop) {
    const int l = pos >> 5, sh = pos & 31;
    const unsigned long long lo = m << sh;
    const unsigned long long hi = sh ? (m >> (64 - sh)) : 0ull;
    long long a0 = (long long)(lo & 0xFFFFFFFFull), a1 = (long long)(lo >> 32), a2 = (long long)hi;
    if (neg) {
      a0 = -a0;
      a1 = -a1;
      a2 = -a2;
    }
    // the terms of one statistic share their magnitude, so l is nearly
    // always the same across a warp: a branch per limb offset is cheap
    switch (l) {
      case 0: L.v[0] += a0; L.v[1] += a1; L.v[2] += a2; break;
      case 1: L.v[1] += a0; L.v[2] += a1; L.v[3] += a2; break;
      case 2: L.v[2] += a0; L.v[3] += a1; L.v[4] += a2; break;
      default: L.v[3] += a0; L.v[4] += a1; L.v[5] += a2; break;
    }
    return;
  }
  // escape: an exact add at the term's own position among the 2^-1100 limbs
  const int pe = e + kEscapeBias;
  const int l = pe >> 5, sh = pe & 31;
  const unsigned long long lo = m << sh;
  const unsigned long long hi = sh ? (m >> (64 - sh)) : 0ull;
  long long a[3] = {(long long)(lo & 0xFFFFFFFFull), (long long)(lo >> 32), (long long)hi};
  long long* esc = p.escape + (size_t)stat * kEscapeLimbs;
  for (int k = 0; k < 3; ++k)
    if (a[k]) atomicAdd(reinterpret_cast<unsigned long long*>(&esc[l + k]), (unsigned long long)(neg ? -a[k] : a[k]));
}

// Carries of each limb into the next (the top limb keeps the sign).
__device__ __forceinline__ void normalise(Limbs& L) {
#pragma unroll
  for (int j = 0; j + 1 < kExactLimbs; ++j) {
    const long long c = L.v[j] >> 32;
    L.v[j] -= c << 32;
    L.v[j + 1] += c;
  }
}

// Term s (0-based statistic index) of one in-range event, rounded as defined.
template <int NDIM>
__device__ __forceinline__ double exact_term(int s, double w, const double* c) {
  switch (s) {
    case 0: return w;
    case 1: return __dmul_rn(w, w);
    case 2: return __dmul_rn(w, c[0]);
    case 3: return __dmul_rn(__dmul_rn(w, c[0]), c[0]);
    case 4: return NDIM >= 2 ? __dmul_rn(w, c[1 % NDIM]) : 0.0;
    case 5: return NDIM >= 2 ? __dmul_rn(__dmul_rn(w, c[1 % NDIM]), c[1 % NDIM]) : 0.0;
    case 6: return NDIM >= 2 ? __dmul_rn(__dmul_rn(w, c[0]), c[1 % NDIM]) : 0.0;
    case 7: return NDIM >= 3 ? __dmul_rn(w, c[2 % NDIM]) : 0.0;
    case 8: return NDIM >= 3 ? __dmul_rn(__dmul_rn(w, c[2 % NDIM]), c[2 % NDIM]) : 0.0;
    case 9: return NDIM >= 3 ? __dmul_rn(__dmul_rn(w, c[0]), c[2 % NDIM]) : 0.0;
    default: return NDIM >= 3 ? __dmul_rn(__dmul_rn(w, c[1 % NDIM]), c[2 % NDIM]) : 0.0;
  }
}

template <bool UNIT, int NDIM>
__global__ void __launch_bounds__(kThreads, 2) k_stats_exact(const __grid_constant__ ExactParams p) {
  __shared__ long long sred[kThreads / 32][kExactGroup][kExactLimbs];
  Limbs acc[kExactGroup];
#pragma unroll
  for (int j = 0; j < kExactGroup; ++j)
#pragma unroll
    for (int l = 0; l < kExactLimbs; ++l) acc[j].v[l] = 0;
  unsigned long long special[kExactGroup][3] = {};
  const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.w);
  auto one = [&](long long i) {
    double c[NDIM];
    bool inr = true;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const unsigned long long xb = __ldcs(reinterpret_cast<const unsigned long long*>(p.col[d]) + i);
      const long long key = key_of(xb);
      inr = inr && key >= p.lo_key[d] && key < p.hi_key[d];
      c[d] = __longlong_as_double((long long)xb);
    }
    if (!p.stat_overflows && !inr) return;
    const double w = UNIT ? 1.0 : __longlong_as_double((long long)__ldcs(wq + i));
#pragma unroll
    for (int j = 0; j < kExactGroup; ++j) {
      if (j >= p.ns) break;
      const int st = p.s0 + j;
      exact_add(acc[j], exact_term<NDIM>(st, w, c), p.grid[st], p, st, special[j]);
    }
  };
  // two events per thread and turn, the second's loads overlapping the first
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.n; i += 2 * stride) {
    one(i);
    if (i + stride < p.n) one(i + stride);
  }
  // normalise, then sum over the warp, the block and the grid (exact integers)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kExactGroup; ++j) {
    normalise(acc[j]);
#pragma unroll
    for (int l = 0; l < kExactLimbs; ++l) {
      long long v = acc[j].v[l];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sred[warp][j][l] = v;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned long long cnt = special[j][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
      if (lane == 0 && cnt && j < p.ns) atomicAdd(&p.special[(p.s0 + j) * 3 + k], cnt);
    }
  }
  __syncthreads();
  if (threadIdx.x < kExactGroup * kExactLimbs) {
    const int j = threadIdx.x / kExactLimbs, l = threadIdx.x % kExactLimbs;
    long long v = 0;
    for (int wi = 0; wi < kThreads / 32; ++wi) v += sred[wi][j][l];
    if (v && j < p.ns)
      atomicAdd(reinterpret_cast<unsigned long long*>(&p.limbs[(p.s0 + j) * kExactLimbs + l]), (unsigned long long)v);
  }
}

// Carry the global limbs so that many launches cannot overflow them.
__global__ void k_exact_normalise(long long* limbs) {
  const int s = threadIdx.x;
  if (s >= kExactStats) return;
  long long* v = limbs + s * kExactLimbs;
  for (int j = 0; j + 1 < kExactLimbs; ++j) {
    const long long c = v[j] >> 32;
    v[j] -= c << 32;
    v[j + 1] += c;
  }
}

}  // namespace

int launch_exact_normalise(long long* limbs, void* stream) {
  k_exact_normalise<<<1, 32, 0, (cudaStream_t)stream>>>(limbs);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_stats_exact(const ExactParams& p, bool unit, int sm_count, void* stream) {
  if (p.n <= 0) return 0;
  if (p.ndim < 1 || p.ndim > kMaxDim || p.ns < 1 || p.ns > kExactGroup || p.s0 < 0 || p.s0 + p.ns > kExactStats)
    return -1;
  long long grid = (p.n + kThreads - 1) / kThreads;
  if (grid > 2LL * sm_count * 4) grid = 2LL * sm_count * 4;
  const cudaStream_t s = (cudaStream_t)stream;
#define HGB_EXACT(U, D) \
  if (unit == U && p.ndim == D) k_stats_exact<U, D><<<(int)grid, kThreads, 0, s>>>(p);
  HGB_EXACT(true, 1)
  HGB_EXACT(false, 1)
  HGB_EXACT(true, 2)
  HGB_EXACT(false, 2)
  HGB_EXACT(true, 3)
  HGB_EXACT(false, 3)
#undef HGB_EXACT
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
