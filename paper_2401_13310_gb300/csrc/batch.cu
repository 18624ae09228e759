// batch.cu -- many 1D histograms filled from one event stream in one launch.
//
// The paper's closing remarks point at computing several histograms from the
// same data, and at its kernels being small and launch-bound.  Here one
// persistent launch reads every column and the weight once per event and
// fills all histograms of the batch:
//  * histograms are sorted by column; the per-column work (the FP32 view of
//    the coordinate, its range flags) and the per-event weight work (the
//    exact fixed-point value) happen once per event, not once per histogram;
//  * each thread holds KEV events in registers and walks the histograms
//    outermost, so a histogram's descriptor is read once per KEV events
//    (KEV and the blocks per SM the launch is compiled for are tuned);
//  * small histograms keep block-private bins in shared memory: the low 64
//    bits of the exact fixed-point sum as two u32 words updated by
//    carry-propagating atomics, the rare carry out of bit 63 going straight
//    to the histogram's global high word; at the end each block adds its
//    words into the global accumulators with 64-bit integer atomics (exact,
//    so the order does not matter);
//  * large histograms add every event to the global accumulators with two
//    64-bit integer atomics (exact);
//  * a batch of histograms booked with HIST_PREC_FP32C runs the FP32
//    compensated form instead: each weight split into FP32 hi + lo once per
//    event; a small histogram's shared bin is an FP32 (hi, lo) pair, hi
//    added by an atomic whose returned old value gives the rounding error
//    exactly (TwoSum), which goes with lo to the lo word; blocks add their
//    pairs into the binary64 bins in binary64 at the end; large histograms
//    take binary64 atomics (one per event);
//  * statistics are shared by the histograms with the same column and range
//    and accumulated once per event for the column's common core (see
//    batch_stats.cuh), binary64 per thread: the binary64 pipe is otherwise
//    idle in this kernel; a second kernel adds each histogram's sums.

#include <cuda_runtime.h>

#include <cstdint>

#include "batch_stats.cuh"
#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {


// FP32 compensated form: W = hi + lo of the weight (wok: in the double-word
// range; other weights take a binary64 atomic).
template <bool SMEM>
__device__ __forceinline__ void batch_add_f32c(const BatchHistDev& d, unsigned* sbins, int k, FF W, bool wok,
                                               unsigned long long wb) {
  if (!SMEM || !wok) {
    atomicAdd(&d.g_f64[k], __longlong_as_double((long long)wb));
    return;
  }
  float* a = reinterpret_cast<float*>(&sbins[d.sbin_off + 2 * k]);
  const float old = atomicAdd(a, W.hi);
  const float sum = __fadd_rn(old, W.hi);
  const float bv = __fsub_rn(sum, old);
  const float err = __fadd_rn(__fsub_rn(old, __fsub_rn(sum, bv)), __fsub_rn(W.hi, bv));
  atomicAdd(a + 1, __fadd_rn(err, W.lo));
}

template <bool UNIT, bool SMEM>
__device__ __forceinline__ void batch_add(const BatchHistDev& d, unsigned* sbins, int k, long long V, bool wok,
                                          unsigned long long wb) {
  if (UNIT) {
    if (SMEM)
      atomicAdd(&sbins[d.sbin_off + k], 1u);
    else
      atomicAdd(&d.g_unit[k], 1ull);
    return;
  }
  if (!wok) {
    atomicAdd(&d.g_f64[k], __longlong_as_double((long long)wb));
    return;
  }
  if (V == 0) return;
  if (SMEM) {
    // low 64 bits in shared memory (two words, carry-chained); a carry out
    // of bit 63 (or the sign extension of a negative addend) goes to the
    // global high word, scaled by 2^32 in its carry-save representation
    unsigned* a = &sbins[d.sbin_off + 2 * k];
    const unsigned v0 = (unsigned)V;
    const unsigned o0 = atomicAdd(a, v0);
    const unsigned c0 = (o0 + v0 < o0) ? 1u : 0u;
    const unsigned a1 = (unsigned)((unsigned long long)V >> 32) + c0;
    const unsigned c1a = (a1 < c0) ? 1u : 0u;
    const unsigned o1 = atomicAdd(a + 1, a1);
    const unsigned c1 = c1a | ((o1 + a1 < o1) ? 1u : 0u);
    const int top = (int)(V >> 63) + (int)c1;  // -1, 0 or 1 units of 2^64
    if (top != 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.g_hi[k]), (unsigned long long)((long long)top << 32));
  } else {
    atomicAdd(&d.g_lo[k], (unsigned long long)(unsigned)V);
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.g_hi[k]), (unsigned long long)(V >> 32));
  }
}

// One event's bin update for one histogram, in the batch's precision.
template <bool UNIT, bool F32C>
__device__ __forceinline__ void batch_update(const BatchHistDev& d, unsigned* sbins, bool in_smem, int k, long long V,
                                             FF W, bool wok, unsigned long long wb) {
  if (F32C && !UNIT) {
    if (in_smem)
      batch_add_f32c<true>(d, sbins, k, W, wok, wb);
    else
      batch_add_f32c<false>(d, sbins, k, W, wok, wb);
  } else {
    if (in_smem)
      batch_add<UNIT, true>(d, sbins, k, V, wok, wb);
    else
      batch_add<UNIT, false>(d, sbins, k, V, wok, wb);
  }
}

template <bool UNIT, bool F32C, int MINB, int KEV>
__global__ void __launch_bounds__(256, MINB) k_batch_fill(const __grid_constant__ BatchParams p) {
  constexpr int kEv = KEV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nkeys = p.table_keys;
  long long* skeys = reinterpret_cast<long long*>(smem_raw);
  int* shi = reinterpret_cast<int*>(smem_raw + (size_t)nkeys * 8);
  const size_t off_bins = ((size_t)nkeys * 12 + 15) & ~(size_t)15;
  unsigned* sbins = reinterpret_cast<unsigned*>(smem_raw + off_bins);
  const size_t off_desc = off_bins + (((size_t)p.sbin_words * 4 + 15) & ~(size_t)15);
  BatchHistDev* sdesc = reinterpret_cast<BatchHistDev*>(smem_raw + off_desc);
  __shared__ double sred[8 * kStatSlots * 3];

  for (int i = threadIdx.x; i < nkeys; i += blockDim.x) {
    const long long t = p.T_concat[i];
    skeys[i] = t;
    shi[i] = (int)(t >> 32);
  }
  for (int i = threadIdx.x; i < p.sbin_words; i += blockDim.x) sbins[i] = 0u;
  {
    const int words = (int)(sizeof(BatchHistDev) / 4) * p.nh;
    const unsigned* src = reinterpret_cast<const unsigned*>(p.hists);
    unsigned* dst = reinterpret_cast<unsigned*>(sdesc);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();

  double core[kBatchMaxCols][3];
#pragma unroll
  for (int c = 0; c < kBatchMaxCols; ++c) core[c][0] = core[c][1] = core[c][2] = 0.0;
  double tail[kBatchMaxGroups * 3];
  for (int t = 0; t < kBatchMaxGroups * 3; ++t) tail[t] = 0.0;

  const long long n = p.n;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.w);
  for (long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x; base < n; base += kEv * nthreads) {
    // kEv events per thread, each load coalesced across the warp
    bool valid[kEv];
    unsigned long long wb[kEv];
    long long V[kEv];
    FF W[kEv];
    bool wok[kEv];
#pragma unroll
    for (int e = 0; e < kEv; ++e) {
      const long long i = base + e * nthreads;
      valid[e] = i < n;
      wb[e] = (UNIT || !valid[e]) ? 0x3FF0000000000000ull : __ldcs(wq + i);
      V[e] = 0;
      W[e].hi = W[e].lo = 0.0f;
      if (UNIT) {
        wok[e] = true;
      } else if (F32C) {
        wok[e] = in_ff(exp_field(wb[e]));
        if (wok[e]) W[e] = ff_split(wb[e], hi24(wb[e]));
      } else {
        wok[e] = fx_of(wb[e], p.fx_elo, &V[e]);
      }
    }
#pragma unroll
    for (int c = 0; c < kBatchMaxCols; ++c) {
      if (c >= p.ncols) break;
      const unsigned long long* cq = reinterpret_cast<const unsigned long long*>(p.col[c]);
      unsigned long long xb[kEv];
      float xf[kEv];
      bool f32ok[kEv];
#pragma unroll
      for (int e = 0; e < kEv; ++e) {
        const long long i = base + e * nthreads;
        xb[e] = valid[e] ? __ldcs(cq + i) : 0ull;
        xf[e] = hi24(xb[e]);
        f32ok[e] = in_f32(exp_field(xb[e]));
      }
      // every histogram of this column
      for (int h = p.col_begin[c]; h < p.col_begin[c + 1]; ++h) {
        const BatchHistDev& d = sdesc[h];  // read in place: its fields load as they are used
        const bool staged = d.ax.smem_off >= 0;
        const long long* T = staged ? skeys + d.ax.smem_off : d.ax.T;
        const int* Thi = staged ? shi + d.ax.smem_off : nullptr;
        const bool in_smem = d.sbin_off >= 0;
        if (d.ax.mode == LOC_BUCKET) {
          // the kEv bins first: their table loads overlap (an invalid
          // event's zero coordinate still maps to a bin; it is not added)
          long long key[kEv];
          int k[kEv];
#pragma unroll
          for (int e = 0; e < kEv; ++e) key[e] = key_of(xb[e]);
          locate_bucket_n<kEv>(d.ax, T, d.ax.bk.cnt, xb, key, k);
#pragma unroll
          for (int e = 0; e < kEv; ++e) {
            if (!valid[e]) continue;
            batch_update<UNIT, F32C>(d, sbins, in_smem, k[e], V[e], W[e], wok[e], wb[e]);
          }
        } else {
#pragma unroll
          for (int e = 0; e < kEv; ++e) {
            if (!valid[e]) continue;
            const int k = locate_axis(d.ax, T, Thi, d.ax.bk.cnt, xb[e], xf[e], f32ok[e]);
            batch_update<UNIT, F32C>(d, sbins, in_smem, k, V[e], W[e], wok[e], wb[e]);
          }
        }
      }
      // statistics of this column
      if (p.st.group_begin[c] < p.st.group_begin[c + 1]) {
#pragma unroll
        for (int e = 0; e < kEv; ++e)
          if (valid[e]) stat_event<UNIT>(p.st, c, key_of(xb[e]), xb[e], wb[e], core[c], tail);
      }
    }
  }
  __syncthreads();

  // block-private bins -> the histograms' exact global accumulators
  for (int h = 0; h < p.nh; ++h) {
    const BatchHistDev& d = sdesc[h];
    if (d.sbin_off < 0) continue;
    const int nb = d.ax.nbins + 2;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      if (UNIT) {
        const unsigned c = sbins[d.sbin_off + k];
        if (c) atomicAdd(&d.g_unit[k], (unsigned long long)c);
      } else if (F32C) {
        const float* f = reinterpret_cast<const float*>(&sbins[d.sbin_off + 2 * k]);
        const double v = __dadd_rn((double)f[0], (double)f[1]);
        if (v != 0.0) atomicAdd(&d.g_f64[k], v);
      } else {
        const unsigned a0 = sbins[d.sbin_off + 2 * k], a1 = sbins[d.sbin_off + 2 * k + 1];
        if (a0) atomicAdd(&d.g_lo[k], (unsigned long long)a0);
        if (a1) atomicAdd(reinterpret_cast<unsigned long long*>(&d.g_hi[k]), (unsigned long long)a1);
      }
    }
  }
  // per-block statistics partials, one fixed reduction order
  __syncthreads();
  block_stats_store(core, tail, sred, p.part_stats + (size_t)blockIdx.x * kStatSlots * 3);
}

// Warp (h, q) adds statistic 2 + q of histogram h: its column's core sum
// plus its group's tail sum over the block partials.  Lane l takes blocks
// l, l + 32, l + 64, ... in order, then a fixed shuffle tree adds the lanes:
// the same partials give the same sum on every run.  (The partitioned
// strategy writes one partial per work item, thousands per fill; a single
// thread walking them in turn took 1.8 ms per fill of the 64-histogram
// batch.)
__global__ void k_batch_reduce(const BatchReduceParams r) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int h = warp / 3, q = warp % 3;
  if (h >= r.nh) return;  // (uniform across the warp)
  const int c = r.hist_col[h], g = r.hist_group[h];
  double s = 0.0;
  for (int b = lane; b < r.nblocks; b += 32) {
    const double* part = r.part_stats + (size_t)b * kStatSlots * 3;
    s = __dadd_rn(s, __dadd_rn(part[c * 3 + q], part[(kBatchMaxCols + g) * 3 + q]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
  if (lane == 0) r.hist_stats[h][2 + q] = __dadd_rn(r.hist_stats[h][2 + q], s);
}

}  // namespace

// The compiled variants: blocks per SM the registers allow (2 or 4) times
// events per thread (2 or 4).
// events per thread (2 or 4), and the precision of weighted batches
// (exact fixed point or FP32 compensated).
const void* batch_fn(bool unit, bool f32c, int minb, int kev) {
#define HGB_BATCH(U, F, M, K) \
  if (unit == U && f32c == F && minb == M && kev == K) return reinterpret_cast<const void*>(&k_batch_fill<U, F, M, K>);
  HGB_BATCH(false, false, 2, 4)
  HGB_BATCH(false, false, 2, 2)
  HGB_BATCH(false, false, 4, 4)
  HGB_BATCH(false, false, 4, 2)
  HGB_BATCH(false, true, 2, 4)
  HGB_BATCH(false, true, 2, 2)
  HGB_BATCH(false, true, 4, 4)
  HGB_BATCH(false, true, 4, 2)
  HGB_BATCH(true, false, 2, 4)
  HGB_BATCH(true, false, 2, 2)
  HGB_BATCH(true, false, 4, 4)
  HGB_BATCH(true, false, 4, 2)
#undef HGB_BATCH
  return nullptr;
}

int batch_max_blocks_per_sm(int block, size_t smem, int minb, int kev, int* per_sm) {
  int least = 1 << 30;
  for (int v = 0; v < 3; ++v) {  // weighted fixed point, weighted FP32 compensated, unit
    const void* fn = batch_fn(v == 2, v == 1, minb, kev);
    if (fn == nullptr) return -1;
    // always: it also loads the kernel before the occupancy query
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
    int a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, block, smem) != cudaSuccess) return -2;
    least = a < least ? a : least;
  }
  *per_sm = least;
  return 0;
}

int launch_batch_fill(const BatchParams& p, int block, int grid, size_t smem, int minb, int kev, bool f32c,
                      void* stream) {
  const void* fn = batch_fn(p.w == nullptr, f32c && p.w != nullptr, minb, kev);
  if (fn == nullptr) return -1;
  {  // always: it also loads the kernel before the occupancy query
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  }
  void* args[] = {const_cast<BatchParams*>(&p)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, (cudaStream_t)stream) == cudaSuccess ? 0 : -2;
}

int launch_batch_reduce(const BatchReduceParams& r, void* stream) {
  const int threads = r.nh * 3 * 32;  // a warp per statistic
  k_batch_reduce<<<(threads + 127) / 128, 128, 0, (cudaStream_t)stream>>>(r);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
