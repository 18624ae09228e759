// batch_partition.cu -- the partitioned strategy of the batched fill: many
// binnings of the same quantity (the eight mixture-quantile axes of the
// learned-locator workload, or the ~21 histograms of each of pT, phi and eta
// in the 64-histogram workload).  Each column's members are filled by one
// run of the kernels below; a batch over several columns runs them once per
// column, one after the other.
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
//    row of at most 32 members per position, padded to a multiple of 8);
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
//    thresholds gives the position p of an event, one to four 16-byte loads
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

#include <climits>
#include <cstdint>

#include "batch_stats.cuh"
#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {

// Merged position (how many of the range's M merged thresholds are <= the
// key) of two keys at once: the bounds first, then the range's bucket map
// and a search of the bucket's thresholds, the two keys' steps interleaved.
struct PartLocator {
  const long long* keys;       // the range's merged thresholds (shared)
  const unsigned short* bcnt;  // its bucket counts (shared)
  long long lo, hi, kbase;
  float scale, offset;
  int m, nbk, key_map, shift, top;

  __device__ __forceinline__ int bucket(long long key, unsigned long long xb) const {
    int b;
    if (key_map) {
      const long long q = (key >> shift) - kbase;
      b = (int)(q < 0 ? 0 : (q > nbk - 1 ? nbk - 1 : q));
    } else {
      const float t = fminf(fmaxf(__fmaf_rn(est_float(xb), scale, offset), -1.0f), (float)nbk);
      b = min(max(__float2int_rd(t), 0), nbk - 1);
    }
    return b;
  }

  __device__ __forceinline__ void locate2(long long k0, unsigned long long x0, long long k1, unsigned long long x1,
                                          int& j0, int& j1) const {
    const bool in0 = k0 >= lo && k0 < hi, in1 = k1 >= lo && k1 < hi;
    const int b0 = in0 ? bucket(k0, x0) : 0, b1 = in1 ? bucket(k1, x1) : 0;
    const int c0 = in0 ? (int)bcnt[b0] : 0, c1 = in1 ? (int)bcnt[b1] : 0;
    const int n0 = in0 ? (int)bcnt[b0 + 1] - c0 : 0, n1 = in1 ? (int)bcnt[b1 + 1] - c1 : 0;
    int p0 = 0, p1 = 0;
    for (int step = top; step > 0; step >>= 1) {
      const int q0 = p0 + step, q1 = p1 + step;
      const long long t0 = q0 <= n0 ? keys[c0 + q0 - 1] : LLONG_MAX;
      const long long t1 = q1 <= n1 ? keys[c1 + q1 - 1] : LLONG_MAX;
      p0 = t0 <= k0 ? q0 : p0;
      p1 = t1 <= k1 ? q1 : p1;
    }
    j0 = k0 < lo ? 0 : (k0 >= hi ? m : c0 + p0);
    j1 = k1 < lo ? 0 : (k1 >= hi ? m : c1 + p1);
  }
};

// The split keys' locator over their shared copy: the range of a key is its
// position among the nranges - 1 splits.
__device__ __forceinline__ PartLocator split_locator(const PartParams& p, const long long* splits,
                                                     const unsigned short* sbc) {
  const PartRangeDev& m = p.split_map;
  return PartLocator{splits, sbc, m.lo_key, m.hi_key, m.kbase, m.scale, m.offset, m.nkeys, m.nbk, m.key_map,
                     m.shift, m.top};
}

// Stage the split keys and their bucket counts: [splits][bucket counts].
__device__ __forceinline__ void stage_splits(const PartParams& p, unsigned char* smem, long long*& splits,
                                             unsigned short*& sbc, size_t& used) {
  splits = reinterpret_cast<long long*>(smem);
  const size_t sb = (((size_t)(p.nranges - 1) * 8) + 15) & ~(size_t)15;
  sbc = reinterpret_cast<unsigned short*>(smem + sb);
  used = sb + ((((size_t)p.split_map.nbk + 1) * 2 + 15) & ~(size_t)15);
  for (int i = threadIdx.x; i < p.nranges - 1; i += blockDim.x) splits[i] = p.splits[i];
  for (int i = threadIdx.x; i <= p.split_map.nbk && p.split_map.nbk > 0; i += blockDim.x) sbc[i] = p.sbcnt[i];
}

// Count: block b takes tiles b, b + G, b + 2G, ... of kPartTile consecutive
// events (thread t events t, t + 256, ... of a tile) and counts them per
// range; the scatter takes the same events in the same blocks.
__global__ void __launch_bounds__(kPartBlock) k_part_count(const __grid_constant__ PartParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* splits;
  unsigned short* sbc;
  size_t used;
  stage_splits(p, smem_raw, splits, sbc, used);
  unsigned* cnt = reinterpret_cast<unsigned*>(smem_raw + used);
  for (int i = threadIdx.x; i < p.nranges; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  const PartLocator L = split_locator(p, splits, sbc);
  const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.col);
  constexpr int kPer = kPartTile / kPartBlock;
  const long long gstep = (long long)gridDim.x * kPartTile;
  // the tile's loads all in flight together, and the next tile's issued
  // before this one is located
  unsigned long long x[kPer];
  long long base = (long long)blockIdx.x * kPartTile;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const long long i = base + threadIdx.x + (long long)k * kPartBlock;
    x[k] = i < p.n ? __ldcs(xq + i) : 0ull;
  }
  for (; base < p.n; base += gstep) {
    unsigned long long nx[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const long long i = base + gstep + threadIdx.x + (long long)k * kPartBlock;
      nx[k] = i < p.n ? __ldcs(xq + i) : 0ull;
    }
#pragma unroll
    for (int k = 0; k < kPer; k += 2) {
      const long long i0 = base + threadIdx.x + (long long)k * kPartBlock, i1 = i0 + kPartBlock;
      int r0, r1;
      L.locate2(key_of(x[k]), x[k], key_of(x[k + 1]), x[k + 1], r0, r1);
      if (i0 < p.n) atomicAdd(&cnt[r0], 1u);
      if (i1 < p.n) atomicAdd(&cnt[r1], 1u);
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) x[k] = nx[k];
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

// Exclusive scan of v[0 .. n) into out (n <= kPartMaxRanges; every thread
// of the block calls it): each thread scans a run of consecutive entries,
// the runs' sums are scanned by warp shuffles and the warps' totals.
__device__ __forceinline__ void block_exclusive_scan(const unsigned* v, unsigned* out, int n, unsigned* wsum) {
  const int per = (n + kPartBlock - 1) / kPartBlock;
  const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
  unsigned own = 0;
  for (int i = i0; i < i1; ++i) own += v[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  unsigned run = inc - own;
  for (int w = 0; w < warp; ++w) run += wsum[w];
  for (int i = i0; i < i1; ++i) {
    out[i] = run;
    run += v[i];
  }
}

// Scatter, a tile at a time (the count's tiles): the tile's events are
// ranked within their ranges by shared atomics, placed in range order in
// shared memory, and written out so that consecutive threads write the
// consecutive events of one range -- each range's run of the tile is one
// contiguous piece of its segment.
template <bool WEIGHTED>
__global__ void __launch_bounds__(kPartBlock) k_part_scatter(const __grid_constant__ PartParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* splits;
  unsigned short* sbc;
  size_t used;
  stage_splits(p, smem_raw, splits, sbc, used);
  const int nr = p.nranges;
  // [.. splits][next (u64)][tcnt (u32)][tstart (u32)][buf_x][buf_w][buf_r (u16)]
  unsigned long long* next = reinterpret_cast<unsigned long long*>(smem_raw + used);
  unsigned* tcnt = reinterpret_cast<unsigned*>(smem_raw + used + (size_t)nr * 8);
  unsigned* tstart = tcnt + nr;
  const size_t bx = (used + (size_t)nr * 16 + 15) & ~(size_t)15;
  unsigned long long* buf_x = reinterpret_cast<unsigned long long*>(smem_raw + bx);
  unsigned long long* buf_w = buf_x + kPartTile;
  unsigned short* buf_r = reinterpret_cast<unsigned short*>(buf_x + (WEIGHTED ? 2 : 1) * kPartTile);
  __shared__ unsigned wsum[kPartBlock / 32];
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    next[r] = p.offsets[(size_t)r * gridDim.x + blockIdx.x];
    tcnt[r] = 0u;
  }
  __syncthreads();
  const PartLocator L = split_locator(p, splits, sbc);
  const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.col);
  const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.w);
  unsigned long long* px = reinterpret_cast<unsigned long long*>(p.px);
  unsigned long long* pw = reinterpret_cast<unsigned long long*>(p.pw);
  constexpr int kPer = kPartTile / kPartBlock;
  const long long gstep = (long long)gridDim.x * kPartTile;
  // the tile's coordinates all in flight together, and the next tile's
  // issued before this one is placed
  unsigned long long x[kPer];
  long long base = (long long)blockIdx.x * kPartTile;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const long long i = base + threadIdx.x + (long long)k * kPartBlock;
    x[k] = i < p.n ? __ldcs(xq + i) : 0ull;
  }
  for (; base < p.n; base += gstep) {
    unsigned long long w[kPer], nx[kPer];
    int r[kPer];
    unsigned rank[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const long long i = base + threadIdx.x + (long long)k * kPartBlock;
      if (WEIGHTED) w[k] = i < p.n ? __ldcs(wq + i) : 0ull;
      const long long in = i + gstep;
      nx[k] = in < p.n ? __ldcs(xq + in) : 0ull;
    }
#pragma unroll
    for (int k = 0; k < kPer; k += 2) {
      const long long i0 = base + threadIdx.x + (long long)k * kPartBlock, i1 = i0 + kPartBlock;
      L.locate2(key_of(x[k]), x[k], key_of(x[k + 1]), x[k + 1], r[k], r[k + 1]);
      rank[k] = i0 < p.n ? atomicAdd(&tcnt[r[k]], 1u) : 0u;
      rank[k + 1] = i1 < p.n ? atomicAdd(&tcnt[r[k + 1]], 1u) : 0u;
    }
    __syncthreads();
    block_exclusive_scan(tcnt, tstart, nr, wsum);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (base + threadIdx.x + (long long)k * kPartBlock < p.n) {
        const unsigned q = tstart[r[k]] + rank[k];
        buf_x[q] = x[k];
        if (WEIGHTED) buf_w[q] = w[k];
        buf_r[q] = (unsigned short)r[k];
      }
    }
    __syncthreads();
    const int tile_n = (int)min((long long)kPartTile, p.n - base);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int q = threadIdx.x + k * kPartBlock;
      if (q < tile_n) {
        const int rr = buf_r[q];
        const unsigned long long pos = next[rr] + (unsigned)(q - (int)tstart[rr]);
        px[pos] = buf_x[q];
        if (WEIGHTED) pw[pos] = buf_w[q];
      }
    }
    __syncthreads();
    for (int rr = threadIdx.x; rr < nr; rr += blockDim.x) {
      next[rr] += tcnt[rr];
      tcnt[rr] = 0u;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) x[k] = nx[k];
    __syncthreads();
  }
}

// Signed fixed-point value V into a shared bin's two u32 words with carries
// (two 32-bit atomics that return the old value: one 64-bit shared atomic
// measured 1.5x slower on the 64-histogram workload); the rare change of
// the top (a carry out of bit 63, or a negative addend's sign) goes to the
// global high word in units of 2^32.
// The low words of a range's bins are one array and the high words another
// (lanes adding to consecutive slots touch consecutive banks).
__device__ __forceinline__ void part_fx_add(unsigned* lo, unsigned* hi, long long* ghi, long long V) {
  const unsigned v0 = (unsigned)V;
  const unsigned o0 = atomicAdd(lo, v0);
  const unsigned c0 = (o0 + v0 < o0) ? 1u : 0u;
  const unsigned a1 = (unsigned)((unsigned long long)V >> 32) + c0;
  const unsigned c1a = (a1 < c0) ? 1u : 0u;
  const unsigned o1 = atomicAdd(hi, a1);
  const unsigned c1 = c1a | ((o1 + a1 < o1) ? 1u : 0u);
  const int top = (int)(V >> 63) + (int)c1;
  if (top != 0) atomicAdd(reinterpret_cast<unsigned long long*>(ghi), (unsigned long long)((long long)top << 32));
}

// A member whose slice of a range has few bins would see most lanes of a
// warp add to the same bin (the range's events all fall in those few bins),
// and same-address shared atomics serialise.  Such a slice keeps 2^rsh
// copies of every bin (as many as fit 32 slots, one bank each: 64 slots
// measured 20 % slower on the 8-axis workload, two slots then sharing a
// bank), lane l adding to copy l mod 2^rsh; the count rows hold c << rsh
// for bin c, and each thread's
// first slot is offset by its copy, so the add stays one add per member.
// F32C: FP32 compensated bins (HIST_PREC_FP32C batches) -- the weight as
// FP32 hi + lo; hi is added to the slot's sum word by an atomic whose
// returned old value gives the addition's rounding error exactly (TwoSum);
// that error plus lo (their sum's own rounding error recovered by TwoSum) is
// added the same way to a compensation word, whose rounding errors go to a
// third word.  Three planes: sums, compensations, second compensations.
// A range's events can all fall in one bin of a coarse member, so a bin copy
// may collect ~2^14 entries in one work item: with one compensation word
// its own rounding (~m 2^-48 of the bin) would exceed 1e-11; the third word
// leaves ~m^2 2^-72.
// The rounding error of fl(a + b), exactly (Knuth's TwoSum).
__device__ __forceinline__ float two_sum_err(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

template <bool UNIT, bool F32C, int ROW>
struct PartFill {
  const PartParams& p;
  const unsigned short* cum;
  const PartSliceDev* sl;
  unsigned* bins;  // [nslots] counters; [nslots] low then high words; or three FP32 planes
  int nslots;
  int boff[ROW];  // each member's first bin slot for this thread's copy (registers)

  // An event (weight wb) at merged position pos into every member's bin.
  __device__ __forceinline__ void add(int pos, unsigned long long wb) const {
    uint4 q[ROW / 8];
    const uint4* rp = reinterpret_cast<const uint4*>(cum + (size_t)pos * ROW);
#pragma unroll
    for (int k = 0; k < ROW / 8; ++k) q[k] = rp[k];
    long long V = 0;
    FF W{0.0f, 0.0f};
    bool wok = true;
    if (F32C) {
      wok = in_ff(exp_field(wb));
      if (wok) W = ff_split(wb, hi24(wb));
    } else if (!UNIT) {
      wok = fx_of(wb, p.fx_elo, &V);
    }
#pragma unroll
    for (int h = 0; h < ROW; ++h) {
      if (h >= p.nh) break;
      const unsigned w32 = reinterpret_cast<const unsigned*>(&q[h >> 3])[(h & 7) >> 1];
      const int j = (int)((h & 1) ? (w32 >> 16) : (w32 & 0xFFFFu));
      if (UNIT) {
        atomicAdd(&bins[boff[h] + j], 1u);
      } else if (F32C && wok) {
        float* f = reinterpret_cast<float*>(bins) + boff[h] + j;
        const float e0 = two_sum_err(atomicAdd(f, W.hi), W.hi);
        const float t = __fadd_rn(e0, W.lo);
        const float d = two_sum_err(e0, W.lo);
        const float e1 = two_sum_err(atomicAdd(f + nslots, t), t);
        atomicAdd(f + 2 * nslots, __fadd_rn(e1, d));
      } else if (!wok) {
        atomicAdd(&p.hists[h].g_f64[sl[h].a + (j >> sl[h].rsh)], __longlong_as_double((long long)wb));
      } else if (!F32C && V != 0) {
        part_fx_add(&bins[boff[h] + j], &bins[nslots + boff[h] + j], &p.hists[h].g_hi[sl[h].a + (j >> sl[h].rsh)],
                    V);
      }
    }
  }
};

// Threads per fill block (256; 512-thread blocks measured 4 % slower on the
// 8-axis workload).  The two-events kernel's registers are sized for three
// blocks per SM with weights (80 registers, so that the small ranges of a
// 48 KB budget run three blocks per SM -- the fill waits mostly on
// shared-memory latency, so resident warps set its pace) and four with unit
// weights (64 registers).
template <bool UNIT>
__host__ __device__ constexpr int part_fill_block() {
  return 256;
}

// EV: events a thread takes at a time, 2 or 4.  Four (unit weights or exact
// fixed point, two blocks per SM, up to 128 registers) serve the ranges
// whose tables already hold the fill to two blocks per SM: the dependent
// shared-memory lookups of four events are in flight together.
template <bool UNIT, bool F32C, int ROW, int EV = 2>
__global__ void __launch_bounds__(part_fill_block<UNIT>(), EV == 4 ? 2 : (UNIT ? 4 : 3))
    k_part_fill(const __grid_constant__ PartParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [count rows][bucket counts][merged keys][slices][bins], each part
  // 16-byte aligned
  unsigned short* cum = reinterpret_cast<unsigned short*>(smem_raw);
  const size_t cum_bytes = ((size_t)(p.max_keys + 1) * ROW * 2 + 15) & ~(size_t)15;
  unsigned short* bcnt = reinterpret_cast<unsigned short*>(smem_raw + cum_bytes);
  const size_t bcnt_bytes = ((size_t)(p.max_nbk + 1) * 2 + 15) & ~(size_t)15;
  long long* keys = reinterpret_cast<long long*>(smem_raw + cum_bytes + bcnt_bytes);
  PartSliceDev* sl = reinterpret_cast<PartSliceDev*>(smem_raw + cum_bytes + bcnt_bytes + (size_t)p.max_keys * 8);
  unsigned* bins = reinterpret_cast<unsigned*>(smem_raw + cum_bytes + bcnt_bytes + (size_t)p.max_keys * 8 +
                                               sizeof(PartSliceDev) * p.nh);
  __shared__ double sred[(part_fill_block<UNIT>() / 32) * kStatSlots * 3];
  __shared__ PartItem item;
  __shared__ PartRangeDev range;

  double core1[3] = {0.0, 0.0, 0.0};  // the column's core sums
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
    for (int j = threadIdx.x; j <= range.nbk && range.nbk > 0; j += blockDim.x) bcnt[j] = p.bcnt[range.bk_base + j];
    for (int h = threadIdx.x; h < p.nh; h += blockDim.x) sl[h] = p.slices[(size_t)item.r * p.nh + h];
    const int nwords = (UNIT ? 1 : (F32C ? 3 : 2)) * range.nbins;
    for (int j = threadIdx.x; j < nwords; j += blockDim.x) bins[j] = 0u;
    __syncthreads();

    const PartLocator loc{keys,         bcnt,         range.lo_key, range.hi_key, range.kbase,
                          range.scale,  range.offset, range.nkeys,  range.nbk,    range.key_map,
                          range.shift,  range.top};
    PartFill<UNIT, F32C, ROW> f{p, cum, sl, bins, range.nbins, {}};
#pragma unroll
    for (int h = 0; h < ROW; ++h)
      f.boff[h] = h < p.nh ? sl[h].boff + (int)(threadIdx.x & ((1u << sl[h].rsh) - 1u)) : 0;
    const unsigned long long* xq = reinterpret_cast<const unsigned long long*>(p.px);
    const unsigned long long* wq = reinterpret_cast<const unsigned long long*>(p.pw);
    const long long e1 = item.e1;
    constexpr unsigned long long kOne = 0x3FF0000000000000ull;
    if constexpr (EV == 4) {
      // events e, e + B, e + 2B, e + 3B (B threads), the next four loaded
      // before the current ones are processed
      const long long B = blockDim.x;
      long long e = item.e0 + threadIdx.x;
      unsigned long long x[4] = {0, 0, 0, 0}, w[4] = {kOne, kOne, kOne, kOne};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (e + i * B < e1) {
          x[i] = __ldcs(xq + e + i * B);
          if (!UNIT) w[i] = __ldcs(wq + e + i * B);
        }
      for (; e < e1; e += 4 * B) {
        const long long en = e + 4 * B;
        unsigned long long nx[4] = {0, 0, 0, 0}, nw[4] = {kOne, kOne, kOne, kOne};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (en + i * B < e1) {
            nx[i] = __ldcs(xq + en + i * B);
            if (!UNIT) nw[i] = __ldcs(wq + en + i * B);
          }
        long long k[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) k[i] = key_of(x[i]);
        int j[4];
        loc.locate2(k[0], x[0], k[1], x[1], j[0], j[1]);
        loc.locate2(k[2], x[2], k[3], x[3], j[2], j[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (e + i * B < e1) {
            f.add(j[i], w[i]);
            stat_event<UNIT>(p.st, p.stat_col, k[i], x[i], w[i], core1, tail);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          x[i] = nx[i];
          w[i] = nw[i];
        }
      }
    } else {
    const long long step = 2 * (long long)blockDim.x;
    // two events per thread at a time (e and e + blockDim.x); the next two
    // are loaded before the current ones are processed
    long long e = item.e0 + threadIdx.x;
    unsigned long long x0 = 0, x1 = 0, w0 = kOne, w1 = kOne;
    if (e < e1) {
      const bool two = e + blockDim.x < e1;
      x0 = __ldcs(xq + e);
      x1 = two ? __ldcs(xq + e + blockDim.x) : x0;
      if (!UNIT) {
        w0 = __ldcs(wq + e);
        w1 = two ? __ldcs(wq + e + blockDim.x) : w0;
      }
    }
    for (; e < e1; e += step) {
      const bool two = e + blockDim.x < e1;
      const long long en = e + step;
      unsigned long long nx0 = 0, nx1 = 0, nw0 = kOne, nw1 = kOne;
      if (en < e1) {
        const bool ntwo = en + blockDim.x < e1;
        nx0 = __ldcs(xq + en);
        nx1 = ntwo ? __ldcs(xq + en + blockDim.x) : nx0;
        if (!UNIT) {
          nw0 = __ldcs(wq + en);
          nw1 = ntwo ? __ldcs(wq + en + blockDim.x) : nw0;
        }
      }
      const long long k0 = key_of(x0), k1 = key_of(x1);
      int j0, j1;
      loc.locate2(k0, x0, k1, x1, j0, j1);
      f.add(j0, w0);
      stat_event<UNIT>(p.st, p.stat_col, k0, x0, w0, core1, tail);
      if (two) {
        f.add(j1, w1);
        stat_event<UNIT>(p.st, p.stat_col, k1, x1, w1, core1, tail);
      }
      x0 = nx0;
      x1 = nx1;
      w0 = nw0;
      w1 = nw1;
    }
    }
    __syncthreads();
    // the range's bins into the members' exact global accumulators
    // (a bin's copies summed first: 64-bit sums of at most 32 words)
    for (int h = 0; h < p.nh; ++h) {
      const PartSliceDev s = sl[h];
      const int nc = 1 << s.rsh;
      const BatchHistDev& d = p.hists[h];
      for (int j = threadIdx.x; j < s.len; j += blockDim.x) {
        const int b0 = s.boff + (j << s.rsh);
        if (UNIT) {
          unsigned long long c = 0;
          for (int r = 0; r < nc; ++r) c += bins[b0 + r];
          if (c) atomicAdd(&d.g_unit[s.a + j], c);
        } else if (F32C) {
          const float* f = reinterpret_cast<const float*>(bins);
          const int nb = range.nbins;
          double v = 0.0;
          for (int r = 0; r < nc; ++r)
            v = __dadd_rn(v, __dadd_rn((double)f[b0 + r], __dadd_rn((double)f[nb + b0 + r], (double)f[2 * nb + b0 + r])));
          if (v != 0.0) atomicAdd(&d.g_f64[s.a + j], v);
        } else {
          unsigned long long a0 = 0, a1 = 0;
          for (int r = 0; r < nc; ++r) {
            a0 += bins[b0 + r];
            a1 += bins[range.nbins + b0 + r];
          }
          if (a0) atomicAdd(&d.g_lo[s.a + j], a0);
          if (a1) atomicAdd(reinterpret_cast<unsigned long long*>(&d.g_hi[s.a + j]), a1);
        }
      }
    }
  }
  // every block writes its statistics partial (zeros for idle blocks and
  // for the other columns' slots)
  double core[kBatchMaxCols][3];
#pragma unroll
  for (int c = 0; c < kBatchMaxCols; ++c)
#pragma unroll
    for (int q = 0; q < 3; ++q) core[c][q] = c == p.stat_col ? core1[q] : 0.0;
  __syncthreads();
  block_stats_store(core, tail, sred, p.part_stats + (size_t)blockIdx.x * kStatSlots * 3);
}

template <bool UNIT, bool F32C, int EV = 2>
const void* part_fill_row(int row) {
  switch (row) {
    case 8: return reinterpret_cast<const void*>(&k_part_fill<UNIT, F32C, 8, EV>);
    case 16: return reinterpret_cast<const void*>(&k_part_fill<UNIT, F32C, 16, EV>);
    case 24: return reinterpret_cast<const void*>(&k_part_fill<UNIT, F32C, 24, EV>);
    default: return reinterpret_cast<const void*>(&k_part_fill<UNIT, F32C, 32, EV>);
  }
}

// row: u16 per count row, 8, 16, 24 or 32; f32c: FP32 compensated bins
// (weighted fills of an FP32C batch; a unit-weight fill counts exactly).
// A fill (unit weights or exact fixed point) whose shared tables allow at
// most two blocks per SM takes the four-events-at-a-time kernel.
const void* part_fill_fn(bool unit, bool f32c, int row, size_t fill_smem, int* events = nullptr) {
  if (events != nullptr) *events = 2;
  if (f32c && !unit) return part_fill_row<false, true>(row);
  const void* two = unit ? part_fill_row<true, false>(row) : part_fill_row<false, false>(row);
  int per_sm = 0;
  if (cudaFuncSetAttribute(two, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, two, part_fill_block<true>(), fill_smem) == cudaSuccess &&
      per_sm >= 1 && per_sm <= 2) {
    if (events != nullptr) *events = 4;
    return unit ? part_fill_row<true, false, 4>(row) : part_fill_row<false, false, 4>(row);
  }
  cudaGetLastError();
  return two;
}

int part_fill_threads(bool unit) { return unit ? part_fill_block<true>() : part_fill_block<false>(); }

}  // namespace

size_t part_count_smem(int nranges, int split_nbk) {
  return ((((size_t)(nranges - 1) * 8) + 15) & ~(size_t)15) + ((((size_t)split_nbk + 1) * 2 + 15) & ~(size_t)15) +
         (size_t)nranges * 4;
}

size_t part_scatter_smem(int nranges, int split_nbk, bool weighted) {
  const size_t used =
      ((((size_t)(nranges - 1) * 8) + 15) & ~(size_t)15) + ((((size_t)split_nbk + 1) * 2 + 15) & ~(size_t)15);
  const size_t bx = (used + (size_t)nranges * 16 + 15) & ~(size_t)15;
  return bx + (size_t)kPartTile * ((weighted ? 16 : 8) + 2);
}

size_t part_fill_smem(int max_keys, int max_bins, int nh, int row_u16, int max_nbk, int slot_bytes) {
  return (((size_t)(max_keys + 1) * row_u16 * 2 + 15) & ~(size_t)15) + (((size_t)(max_nbk + 1) * 2 + 15) & ~(size_t)15) +
         (size_t)max_keys * 8 + sizeof(PartSliceDev) * (size_t)nh + (size_t)max_bins * slot_bytes;
}

int part_fill_events(bool unit, bool f32c, int row, size_t fill_smem) {
  int events = 2;
  part_fill_fn(unit, f32c, row, fill_smem, &events);
  return events;
}

int part_grids(int sm_count, int nranges, int split_nbk, size_t fill_smem, int* count_grid, int* fill_per_sm) {
  const size_t cs = part_count_smem(nranges, split_nbk);
  const size_t ss = part_scatter_smem(nranges, split_nbk, true);
  const size_t su = part_scatter_smem(nranges, split_nbk, false);
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_count), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cs) != cudaSuccess ||
      cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_scatter<true>),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss) != cudaSuccess ||
      cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_scatter<false>),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)su) != cudaSuccess)
    return -2;
  int per_sm = 0, least = 1 << 30;
  // (the count and the scatter share a grid: the weighted scatter's occupancy)
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(&k_part_scatter<true>),
                                                    kPartBlock, ss) != cudaSuccess)
    return -2;
  for (int v = 0; v < 12; ++v) {
    const bool unit = v % 3 == 0, f32c = v % 3 == 2;
    const void* fn = part_fill_fn(unit, f32c, 8 * (1 + v / 3), fill_smem);
    int a = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, part_fill_threads(unit), fill_smem) != cudaSuccess)
      return -2;
    least = a < least ? a : least;
  }
  if (per_sm < 1 || least < 1) return -3;
  // one resident wave of the scatter (each block its tiles in turn)
  *count_grid = per_sm * sm_count;
  *fill_per_sm = least;
  return 0;
}

int launch_part_fill(const PartParams& p, bool unit, bool f32c, int fill_grid, size_t fill_smem, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cs = part_count_smem(p.nranges, p.split_map.nbk);
  const size_t ss = part_scatter_smem(p.nranges, p.split_map.nbk, !unit);
  const void* scatter = unit ? reinterpret_cast<const void*>(&k_part_scatter<false>)
                             : reinterpret_cast<const void*>(&k_part_scatter<true>);
  // (the attributes are per kernel: another batch may have set others)
  const void* fill = part_fill_fn(unit, f32c, p.row_u16, fill_smem);
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_part_count), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cs) != cudaSuccess ||
      cudaFuncSetAttribute(scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss) != cudaSuccess ||
      cudaFuncSetAttribute(fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem) != cudaSuccess)
    return -2;
  const int wblocks = (p.nranges + 7) / 8;  // a warp per range, 8 per block
  k_part_count<<<p.grid_count, kPartBlock, cs, s>>>(p);
  k_part_totals<<<wblocks, 256, 0, s>>>(p);
  k_part_rscan<<<1, 1024, 0, s>>>(p);
  k_part_offsets<<<wblocks, 256, 0, s>>>(p);
  void* args[] = {const_cast<PartParams*>(&p)};
  if (cudaLaunchKernel(scatter, dim3(p.grid_count), dim3(kPartBlock), args, ss, s) != cudaSuccess) return -2;
  if (cudaLaunchKernel(fill, dim3(fill_grid), dim3(part_fill_threads(unit)), args, fill_smem, s) != cudaSuccess)
    return -2;
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
