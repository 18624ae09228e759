// batch_partition.cu -- the partitioned strategy of the batched fill, for
// batches whose histograms all read one column (many binnings of the same
// quantity, such as the eight mixture-quantile axes of the learned-locator
// workload).
//
// A member with 1e4 .. 1e6 bins cannot keep block-private bins, so the wide
// strategy adds its events with global atomics and looks its bin up in
// tables that live in L2 -- per event and member several L2 requests, which
// set the pace.  Here the events are first partitioned by coordinate:
//
//  * the host cuts the column's key space into ranges [S_r, S_r+1) such that
//    every member's bins over one range (its slice: bins a .. a + len - 1)
//    fit one block's shared memory together with the range's merged
//    thresholds -- the distinct thresholds of all members strictly inside
//    the range, sorted -- and, for every position p among them, each
//    member's count of its own thresholds among the first p (16-bit, one
//    row of at most 16 members per position);
//  * count: each block counts its grid-strided events per range (a binary
//    search over the split keys in shared memory, two events at a time);
//  * scan: the counts become per-(range, block) offsets and a list of work
//    items (a range and a run of at most `chunk` of its events): a warp per
//    range with coalesced reads, and one block scanning the range totals;
//  * scatter: each block writes its events (and weights) to their range's
//    segment of a partitioned copy of the column, at the offsets found (the
//    same grid-strided assignment as the count);
//  * fill: each work item's block stages its range -- merged thresholds,
//    count rows, zeroed bins -- in shared memory, reads its run of events
//    coalesced, two per thread at a time; one binary search over the merged
//    thresholds gives the position p of an event, one 16- or 32-byte load
//    its row, and member h's bin is a_h + row[h]: one add to the shared bins
//    per member (u32 counters, or the exact fixed-point words with carries
//    of the other strategies).  At the end the block adds its bins into the
//    members' global accumulators (integer atomics: exact, so the order and
//    the split into items do not matter).
//
// Every step but the fill is a stream over the column; the fill touches L2
// only for its staging and flush.  Statistics are those of the other
// strategies (batch_stats.cuh), accumulated in the fill.

#include <cuda_runtime.h>

#include <cstdint>

#include "batch_stats.cuh"
#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {

// Number of the n sorted keys K[0..n) that are <= key (two keys at once:
// their search steps interleave).
__device__ __forceinline__ void count_le2(const long long* K, int n, long long k0, long long k1, int& j0, int& j1) {
  int a = 0, b = 0, len = n + 1;  // answers in [0, n]
  while (len > 1) {
    const int half = len >> 1;
    const long long t0 = K[a + half - 1], t1 = K[b + half - 1];
    a = (t0 <= k0) ? a + half : a;
    b = (t1 <= k1) ? b + half : b;
    len -= half;
  }
  j0 = a;
  j1 = b;
}

__global__ void __launch_bounds__(kPartBlock) k_part_count(const __grid_constant__ PartParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* splits = reinterpret_cast<long long*>(smem_raw);
  unsigned* cnt = reinterpret_cast<unsigned*>(smem_raw + (size_t)p.nranges * 8);
  for (int i = threadIdx.x; i < p.nranges - 1; i += blockDim.x) splits[i] = p.splits[i];
  for (int i = threadIdx.x; i < p.nranges; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.col);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.n; i += 2 * stride) {
    const bool two = i + stride < p.n;
    const long long k0 = key_of(__ldcs(xq + i));
    const long long k1 = two ? key_of(__ldcs(xq + i + stride)) : k0;
    int r0, r1;
    count_le2(splits, p.nranges - 1, k0, k1, r0, r1);
    atomicAdd(&cnt[r0], 1u);
    if (two) atomicAdd(&cnt[r1], 1u);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < p.nranges; r += blockDim.x) p.counts[(size_t)r * gridDim.x + blockIdx.x] = cnt[r];
}

// The scan, in three small launches: per-range totals (a warp per range,
// coalesced reads of its blocks' counts); their exclusive scan and the work
// items' bases (one block: at most kPartMaxRanges ranges); the per-(range,
// block) offsets (a warp scan per range) and the work items.
__global__ void __launch_bounds__(256) k_part_totals(const __grid_constant__ PartParams p) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= p.nranges) return;
  const int G = p.grid_count;
  unsigned long long s = 0;
  for (int b = lane; b < G; b += 32) s += p.counts[(size_t)r * G + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) p.rtotal[r] = s;
}

__global__ void __launch_bounds__(1024) k_part_rscan(const __grid_constant__ PartParams p) {
  __shared__ unsigned long long sv[1024];
  __shared__ int si[1024];
  // each thread scans a run of ranges; the runs' sums are scanned in turn
  const int per = (p.nranges + blockDim.x - 1) / blockDim.x;
  const int r0 = threadIdx.x * per, r1 = min(p.nranges, r0 + per);
  unsigned long long s = 0;
  int it = 0;
  for (int r = r0; r < r1; ++r) {
    const unsigned long long len = p.rtotal[r];
    s += len;
    it += (int)((len + (unsigned long long)p.chunk - 1) / (unsigned long long)p.chunk);
  }
  sv[threadIdx.x] = s;
  si[threadIdx.x] = it;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // inclusive Hillis-Steele scans
    const unsigned long long a = threadIdx.x >= (unsigned)o ? sv[threadIdx.x - o] : 0ull;
    const int b = threadIdx.x >= (unsigned)o ? si[threadIdx.x - o] : 0;
    __syncthreads();
    sv[threadIdx.x] += a;
    si[threadIdx.x] += b;
    __syncthreads();
  }
  unsigned long long run = sv[threadIdx.x] - s;
  int ib = si[threadIdx.x] - it;
  for (int r = r0; r < r1; ++r) {
    const unsigned long long len = p.rtotal[r];
    p.rstart[r] = run;
    p.ibase[r] = ib;
    run += len;
    ib += (int)((len + (unsigned long long)p.chunk - 1) / (unsigned long long)p.chunk);
  }
  if (threadIdx.x == blockDim.x - 1) *p.nitems = min(si[threadIdx.x], p.max_items);
}

__global__ void __launch_bounds__(256) k_part_offsets(const __grid_constant__ PartParams p) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= p.nranges) return;
  const int G = p.grid_count;
  unsigned long long run = p.rstart[r];
  for (int b0 = 0; b0 < G; b0 += 32) {
    const int b = b0 + lane;
    const unsigned long long v = b < G ? p.counts[(size_t)r * G + b] : 0ull;
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (b < G) p.offsets[(size_t)r * G + b] = run + inc - v;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  const long long e0 = (long long)p.rstart[r];
  const long long e1 = e0 + (long long)p.rtotal[r];
  const int nch = (int)((e1 - e0 + p.chunk - 1) / p.chunk);
  for (int k = lane; k < nch; k += 32) {
    const int it = p.ibase[r] + k;
    if (it >= p.max_items) break;
    PartItem item;
    item.e0 = e0 + (long long)k * p.chunk;
    item.e1 = min(e1, item.e0 + (long long)p.chunk);
    item.r = r;
    item.pad = 0;
    p.items[it] = item;
  }
}

__global__ void __launch_bounds__(kPartBlock) k_part_scatter(const __grid_constant__ PartParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* splits = reinterpret_cast<long long*>(smem_raw);
  unsigned long long* base = reinterpret_cast<unsigned long long*>(smem_raw + (size_t)p.nranges * 8);
  unsigned* cursor = reinterpret_cast<unsigned*>(smem_raw + (size_t)p.nranges * 16);
  for (int i = threadIdx.x; i < p.nranges - 1; i += blockDim.x) splits[i] = p.splits[i];
  for (int r = threadIdx.x; r < p.nranges; r += blockDim.x) {
    base[r] = p.offsets[(size_t)r * gridDim.x + blockIdx.x];
    cursor[r] = 0u;
  }
  __syncthreads();
  const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.col);
  const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.w);
  unsigned long long* px = reinterpret_cast<unsigned long long*>(p.px);
  unsigned long long* pw = reinterpret_cast<unsigned long long*>(p.pw);
  const long long stride = (long long)gridDim.x * blockDim.x;
  // the same events per block as the count pass, in the same pairs
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.n; i += 2 * stride) {
    const bool two = i + stride < p.n;
    const unsigned long long x0 = __ldcs(xq + i);
    const unsigned long long x1 = two ? __ldcs(xq + i + stride) : x0;
    int r0, r1;
    count_le2(splits, p.nranges - 1, key_of(x0), key_of(x1), r0, r1);
    const unsigned long long q0 = base[r0] + atomicAdd(&cursor[r0], 1u);
    px[q0] = x0;
    if (wq != nullptr) pw[q0] = __ldcs(wq + i);
    if (two) {
      const unsigned long long q1 = base[r1] + atomicAdd(&cursor[r1], 1u);
      px[q1] = x1;
      if (wq != nullptr) pw[q1] = __ldcs(wq + i + stride);
    }
  }
}

// Signed fixed-point value V into a shared bin's two u32 words with carries;
// the rare change of the top (a carry out of bit 63, or a negative addend's
// sign) goes to the global high word in units of 2^32.
__device__ __forceinline__ void part_fx_add(unsigned* a, long long* ghi, long long V) {
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

template <bool UNIT, int ROW>
struct PartFill {
  const PartParams& p;
  const unsigned short* cum;
  const PartSliceDev* sl;
  unsigned* bins;
  int boff[ROW];  // each member's first bin slot (registers)

  // An event (weight wb) at merged position pos into every member's bin.
  __device__ __forceinline__ void add(int pos, unsigned long long wb) const {
    uint4 q[ROW / 8];
    const uint4* rp = reinterpret_cast<const uint4*>(cum + (size_t)pos * ROW);
#pragma unroll
    for (int k = 0; k < ROW / 8; ++k) q[k] = rp[k];
    long long V = 0;
    const bool wok = UNIT ? true : fx_of(wb, p.fx_elo, &V);
#pragma unroll
    for (int h = 0; h < ROW; ++h) {
      if (h >= p.nh) break;
      const unsigned w32 = reinterpret_cast<const unsigned*>(&q[h >> 3])[(h & 7) >> 1];
      const int j = (int)((h & 1) ? (w32 >> 16) : (w32 & 0xFFFFu));
      if (UNIT) {
        atomicAdd(&bins[boff[h] + j], 1u);
      } else if (!wok) {
        atomicAdd(&p.hists[h].g_f64[sl[h].a + j], __longlong_as_double((long long)wb));
      } else if (V != 0) {
        part_fx_add(&bins[2 * (boff[h] + j)], &p.hists[h].g_hi[sl[h].a + j], V);
      }
    }
  }
};

template <bool UNIT, int ROW>
__global__ void __launch_bounds__(kPartBlock) k_part_fill(const __grid_constant__ PartParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [count rows (16-byte aligned)][merged keys][slices][bins]
  unsigned short* cum = reinterpret_cast<unsigned short*>(smem_raw);
  const size_t cum_bytes = ((size_t)(p.max_keys + 1) * ROW * 2 + 15) & ~(size_t)15;
  long long* keys = reinterpret_cast<long long*>(smem_raw + cum_bytes);
  PartSliceDev* sl = reinterpret_cast<PartSliceDev*>(smem_raw + cum_bytes + (size_t)p.max_keys * 8);
  unsigned* bins = reinterpret_cast<unsigned*>(smem_raw + cum_bytes + (size_t)p.max_keys * 8 +
                                               sizeof(PartSliceDev) * p.nh);
  __shared__ double sred[(kPartBlock / 32) * kStatSlots * 3];
  __shared__ PartItem item;
  __shared__ PartRangeDev range;

  double core[kBatchMaxCols][3];
#pragma unroll
  for (int c = 0; c < kBatchMaxCols; ++c) core[c][0] = core[c][1] = core[c][2] = 0.0;
  double tail[kBatchMaxGroups * 3];
  for (int t = 0; t < kBatchMaxGroups * 3; ++t) tail[t] = 0.0;

  const bool active = blockIdx.x < *p.nitems;
  if (active) {
    if (threadIdx.x == 0) {
      item = p.items[blockIdx.x];
      range = p.ranges[item.r];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < range.nkeys; j += blockDim.x) keys[j] = p.keys[range.key_base + j];
    {
      const uint4* src = reinterpret_cast<const uint4*>(p.cum + (size_t)range.cum_base);
      uint4* dst = reinterpret_cast<uint4*>(cum);
      const int n16 = (range.nkeys + 1) * ROW / 8;
      for (int j = threadIdx.x; j < n16; j += blockDim.x) dst[j] = src[j];
    }
    for (int h = threadIdx.x; h < p.nh; h += blockDim.x) sl[h] = p.slices[(size_t)item.r * p.nh + h];
    const int nwords = (UNIT ? 1 : 2) * range.nbins;
    for (int j = threadIdx.x; j < nwords; j += blockDim.x) bins[j] = 0u;
    __syncthreads();

    PartFill<UNIT, ROW> f{p, cum, sl, bins, {}};
#pragma unroll
    for (int h = 0; h < ROW; ++h) f.boff[h] = h < p.nh ? sl[h].boff : 0;
    const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.px);
    const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.pw);
    const long long e1 = item.e1;
    for (long long e = item.e0 + threadIdx.x; e < e1; e += 2 * (long long)blockDim.x) {
      const long long e2 = e + blockDim.x;
      const bool two = e2 < e1;
      const unsigned long long x0 = __ldcs(xq + e);
      const unsigned long long x1 = two ? __ldcs(xq + e2) : x0;
      const unsigned long long w0 = UNIT ? 0x3FF0000000000000ull : __ldcs(wq + e);
      const unsigned long long w1 = UNIT ? 0x3FF0000000000000ull : (two ? __ldcs(wq + e2) : w0);
      const long long k0 = key_of(x0), k1 = key_of(x1);
      int j0, j1;
      count_le2(keys, range.nkeys, k0, k1, j0, j1);
      f.add(j0, w0);
      stat_event<UNIT>(p.st, 0, k0, x0, w0, core[0], tail);
      if (two) {
        f.add(j1, w1);
        stat_event<UNIT>(p.st, 0, k1, x1, w1, core[0], tail);
      }
    }
    __syncthreads();
    // the range's bins into the members' exact global accumulators
    for (int h = 0; h < p.nh; ++h) {
      const PartSliceDev s = sl[h];
      const BatchHistDev& d = p.hists[h];
      for (int j = threadIdx.x; j < s.len; j += blockDim.x) {
        if (UNIT) {
          const unsigned c = bins[s.boff + j];
          if (c) atomicAdd(&d.g_unit[s.a + j], (unsigned long long)c);
        } else {
          const unsigned a0 = bins[2 * (s.boff + j)], a1 = bins[2 * (s.boff + j) + 1];
          if (a0) atomicAdd(&d.g_lo[s.a + j], (unsigned long long)a0);
          if (a1) atomicAdd(reinterpret_cast<unsigned long long*>(&d.g_hi[s.a + j]), (unsigned long long)a1);
        }
      }
    }
  }
  // every block writes its statistics partial (zeros for idle blocks)
  __syncthreads();
  block_stats_store(core, tail, sred, p.part_stats + (size_t)blockIdx.x * kStatSlots * 3);
}

const void* part_fill_fn(bool unit, int row) {
  if (unit) return row == 8 ? reinterpret_cast<const void*>(&k_part_fill<true, 8>)
                            : reinterpret_cast<const void*>(&k_part_fill<true, 16>);
  return row == 8 ? reinterpret_cast<const void*>(&k_part_fill<false, 8>)
                  : reinterpret_cast<const void*>(&k_part_fill<false, 16>);
}

}  // namespace

size_t part_count_smem(int nranges) { return (size_t)nranges * 16 + (size_t)nranges * 4; }

size_t part_fill_smem(int max_keys, int max_bins, int nh, int row_u16) {
  return (((size_t)(max_keys + 1) * row_u16 * 2 + 15) & ~(size_t)15) + (size_t)max_keys * 8 +
         sizeof(PartSliceDev) * (size_t)nh + (size_t)max_bins * 8;
}

int part_grids(int sm_count, int nranges, size_t fill_smem, int* count_grid, int* fill_per_sm) {
  const size_t cs = part_count_smem(nranges);
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_count), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cs) != cudaSuccess ||
      cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_scatter),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs) != cudaSuccess)
    return -2;
  int per_sm = 0, least = 1 << 30;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(&k_part_scatter),
                                                    kPartBlock, cs) != cudaSuccess)
    return -2;
  for (int v = 0; v < 4; ++v) {
    const void* fn = part_fill_fn(v & 1, (v & 2) ? 16 : 8);
    int a = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, kPartBlock, fill_smem) != cudaSuccess)
      return -2;
    least = a < least ? a : least;
  }
  if (per_sm < 1 || least < 1) return -3;
  // (at most 4 blocks per SM: fewer (range, block) segments, each longer,
  // so the scatter's writes fill whole cache lines)
  *count_grid = (per_sm < 4 ? per_sm : 4) * sm_count;
  *fill_per_sm = least;
  return 0;
}

int launch_part_fill(const PartParams& p, bool unit, int fill_grid, size_t fill_smem, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cs = part_count_smem(p.nranges);
  // (the attributes are per kernel: another batch may have set others)
  const void* fill = part_fill_fn(unit, p.row_u16);
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_count), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cs) != cudaSuccess ||
      cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_scatter),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs) != cudaSuccess ||
      cudaFuncSetAttribute(fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem) != cudaSuccess)
    return -2;
  const int wblocks = (p.nranges + 7) / 8;  // a warp per range, 8 per block
  k_part_count<<<p.grid_count, kPartBlock, cs, s>>>(p);
  k_part_totals<<<wblocks, 256, 0, s>>>(p);
  k_part_rscan<<<1, 1024, 0, s>>>(p);
  k_part_offsets<<<wblocks, 256, 0, s>>>(p);
  k_part_scatter<<<p.grid_count, kPartBlock, cs, s>>>(p);
  void* args[] = {const_cast<PartParams*>(&p)};
  if (cudaLaunchKernel(fill, dim3(fill_grid), dim3(kPartBlock), args, fill_smem, s) != cudaSuccess) return -2;
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
