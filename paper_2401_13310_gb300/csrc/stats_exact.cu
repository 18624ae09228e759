// stats_exact.cu -- order-independent, exactly summed 1D statistics.
//
// With HIST_STATS_EXACT every statistic of a 1D histogram is the exact sum
// of its rounded terms (w, fl(w*w), fl(w*x), fl(fl(w*x)*x), the terms of
// Sec. 3.1's statistics as the oracle rounds them), rounded once to
// binary64 on the host -- the same bits whatever the launch shape, the
// order of the atomics or the way the events were split into fills.
//
// Each term t = +-m 2^(E-1075) (m the 53-bit significand) is an integer
// multiple of 2^g_s, g_s the statistic's grid, when E - 1075 >= g_s; it is
// added into six radix-2^32 limbs held in int64 registers (the register
// limbs absorb carries; each thread normalises them before the block and
// grid sums, which are integer additions and hence exact and associative).
// A term outside the grid's window (tiny, huge, subnormal) takes an escape
// path into a 70-limb accumulator spanning every finite double; NaN and
// infinite terms are counted instead.

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

template <bool UNIT>
__global__ void __launch_bounds__(kThreads, 2) k_stats_exact(const __grid_constant__ ExactParams p) {
  __shared__ long long sred[kThreads / 32][kExactStats][kExactLimbs];
  Limbs acc[kExactStats];
#pragma unroll
  for (int s = 0; s < kExactStats; ++s)
#pragma unroll
    for (int j = 0; j < kExactLimbs; ++j) acc[s].v[j] = 0;
  unsigned long long special[kExactStats][3] = {};
  const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.x);
  const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.w);
  auto one = [&](unsigned long long xb, unsigned long long wb) {
    const long long key = key_of(xb);
    if (!p.stat_overflows && !(key >= p.lo_key && key < p.hi_key)) return;
    const double x = __longlong_as_double((long long)xb);
    const double w = UNIT ? 1.0 : __longlong_as_double((long long)wb);
    const double wx = UNIT ? x : __dmul_rn(w, x);
    exact_add(acc[0], w, p.grid[0], p, 0, special[0]);
    exact_add(acc[1], UNIT ? 1.0 : __dmul_rn(w, w), p.grid[1], p, 1, special[1]);
    exact_add(acc[2], wx, p.grid[2], p, 2, special[2]);
    exact_add(acc[3], __dmul_rn(wx, x), p.grid[3], p, 3, special[3]);
  };
  // pairs of events, the next pair's loads in flight while this one is added
  const long long npairs = p.n >> 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned long long x0 = 0, x1 = 0, w0 = 0, w1 = 0;
  auto load = [&](long long k, unsigned long long& a, unsigned long long& b, unsigned long long& c,
                  unsigned long long& d) {
    a = __ldcs(xq + 2 * k);
    b = __ldcs(xq + 2 * k + 1);
    if (!UNIT) {
      c = __ldcs(wq + 2 * k);
      d = __ldcs(wq + 2 * k + 1);
    }
  };
  if (q < npairs) load(q, x0, x1, w0, w1);
  for (; q < npairs; q += stride) {
    unsigned long long nx0 = 0, nx1 = 0, nw0 = 0, nw1 = 0;
    if (q + stride < npairs) load(q + stride, nx0, nx1, nw0, nw1);
    one(x0, w0);
    one(x1, w1);
    x0 = nx0;
    x1 = nx1;
    w0 = nw0;
    w1 = nw1;
  }
  if ((p.n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
    one(__ldcs(xq + p.n - 1), UNIT ? 0ull : __ldcs(wq + p.n - 1));
  // normalise, then sum over the warp, the block and the grid (exact integers)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < kExactStats; ++s) {
    normalise(acc[s]);
#pragma unroll
    for (int j = 0; j < kExactLimbs; ++j) {
      long long v = acc[s].v[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sred[warp][s][j] = v;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned long long c = special[s][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
      if (lane == 0 && c) atomicAdd(&p.special[s * 3 + k], c);
    }
  }
  __syncthreads();
  if (threadIdx.x < kExactStats * kExactLimbs) {
    const int s = threadIdx.x / kExactLimbs, j = threadIdx.x % kExactLimbs;
    long long v = 0;
    for (int wi = 0; wi < kThreads / 32; ++wi) v += sred[wi][s][j];
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&p.limbs[s * kExactLimbs + j]), (unsigned long long)v);
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
  long long grid = (p.n + kThreads - 1) / kThreads;
  if (grid > 2LL * sm_count * 4) grid = 2LL * sm_count * 4;
  if (unit)
    k_stats_exact<true><<<(int)grid, kThreads, 0, (cudaStream_t)stream>>>(p);
  else
    k_stats_exact<false><<<(int)grid, kThreads, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
