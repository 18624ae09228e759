// batch_slices.cu -- the sliced strategy of the batched fill.
//
// When a batch holds more bins than one block's shared memory, the wide
// strategy (batch.cu) sends the large histograms to global atomics, whose
// throughput on random bins is a small fraction of shared-memory atomics.
// The sliced strategy keeps every bin in shared memory instead: the host
// cuts the batch's bins into slices of at most one block's budget (a slice
// is a run of fragments, each a bin range [a, b) of one histogram, all on
// one column), balancing the work per slice, and block (s, r) fills slice s
// from the event tiles r, r + R, r + 2R, ...  Every slice reads every event,
// so a tile is read from HBM once and then from L2 by the other slices; the
// blocks pace themselves so that no slice runs more than a window of tiles
// ahead of the slowest (a bounded wait that only serves L2 locality: the
// results never depend on it).
//
// Per event and fragment: one key range test (T[a] <= key < T[b]), then the
// bin -- the fixed axis' affine estimate with its exact correction, or a
// binary search over the fragment's own thresholds staged in shared memory
// -- and the exact fixed-point (or unit) add into the block's bins.  The
// small histograms are held whole by every block and filled, with the
// statistics, by one block per tile, in turn.

#include <cuda_runtime.h>

#include <cstdint>

#include "batch_stats.cuh"
#include "device_common.cuh"
#include "hist_internal.h"

namespace hgb {
namespace {

constexpr int kSliceThreads = 512;

// Bytes of keys, bin words and fragment descriptors, each part 16-byte aligned.
__host__ __device__ __forceinline__ size_t slice_bytes(int keys, int words, int frags) {
  return (((size_t)keys * 8 + 15) & ~(size_t)15) + (((size_t)words * 4 + 15) & ~(size_t)15) +
         sizeof(SliceFragDev) * (size_t)frags;
}
constexpr int kSliceEv = 4;             // events per thread per tile
constexpr int kPaceSleepNs = 256;
constexpr int kPaceBudget = 16384;      // spin iterations a block may spend pacing in one launch (~4 ms)
constexpr int kPaceEvery = 16;          // a block checks its pace every 16 of its tiles

__device__ __forceinline__ int count_le(const long long* K, int n, int top, long long key) {
  int pos = 0;
  for (int step = top; step > 0; step >>= 1) {
    const int q = pos + step;
    if (q <= n && K[q - 1] <= key) pos = q;
  }
  return pos;
}

template <bool UNIT>
__device__ __forceinline__ void slice_add(const SliceFragDev& d, unsigned* sb, int k, long long V, bool wok,
                                          unsigned long long wb) {
  unsigned* a = sb + d.bin_off + 2 * (k - d.a);
  if (UNIT) {
    atomicAdd(a, 1u);
    return;
  }
  if (!wok) {
    atomicAdd(&d.g_f64[k], __longlong_as_double((long long)wb));
    return;
  }
  if (V == 0) return;
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
}

// Wait (bounded) until every slice has finished tile t; only for L2 locality.
__device__ __forceinline__ void pace(const int* done, int nslices, int* budget) {
  if (threadIdx.x == 0 && *budget > 0) {
    const volatile int* f = done;
    int spins = 0;
    while (*f < nslices && spins < *budget) {
      __nanosleep(kPaceSleepNs);
      ++spins;
    }
    *budget -= spins;
  }
  __syncthreads();
}

// Per-thread view of kSliceEv events of one column in a tile.
struct EvCol {
  unsigned long long xb[kSliceEv];
  long long key[kSliceEv];
};

__device__ __forceinline__ void load_col(EvCol& ev, const unsigned long long* cq, long long i0, long long n) {
#pragma unroll
  for (int e = 0; e < kSliceEv; ++e) {
    const long long i = i0 + (long long)e * kSliceThreads;
    ev.xb[e] = i < n ? __ldcg(cq + i) : 0ull;
  }
}

__device__ __forceinline__ void load_w(unsigned long long (&wb)[kSliceEv], const unsigned long long* wq, long long i0,
                                       long long n) {
#pragma unroll
  for (int e = 0; e < kSliceEv; ++e) {
    const long long i = i0 + (long long)e * kSliceThreads;
    wb[e] = (wq != nullptr && i < n) ? __ldcg(wq + i) : 0x3FF0000000000000ull;
  }
}

// Fragments [f0, f1) of the block's shared-memory table for these events.
template <bool UNIT>
__device__ __forceinline__ void fill_frags(const SliceFragDev* sfr, int f0, int f1, const long long* skeys,
                                           unsigned* sbins, const EvCol& ev, const bool (&valid)[kSliceEv],
                                           const long long (&V)[kSliceEv], const bool (&wok)[kSliceEv],
                                           const unsigned long long (&wb)[kSliceEv]) {
  for (int f = f0; f < f1; ++f) {
    const SliceFragDev& d = sfr[f];
    const int koff = d.key_off;
    if (koff < 0) {
      // the histogram's own locator (affine estimate, bucket map, learned
      // model) over its global tables, for every event alike -- no
      // divergence -- then the fragment test on the bin
      const AxisDev ax = d.ax;
      const int a = d.a, b = d.b;
#pragma unroll
      for (int e = 0; e < kSliceEv; ++e) {
        if (!valid[e]) continue;
        const unsigned long long xb = ev.xb[e];
        const int k = locate_axis(ax, ax.T, nullptr, ax.bk.cnt, xb, hi24(xb), in_f32(exp_field(xb)));
        if (k >= a && k < b) slice_add<UNIT>(d, sbins, k, V[e], wok[e], wb[e]);
      }
    } else {
      // binary search over the fragment's own thresholds in shared memory
      const long long Ta = d.Ta, Tb = d.Tb;
      const bool whole = d.whole != 0;
#pragma unroll
      for (int e = 0; e < kSliceEv; ++e) {
        if (!valid[e]) continue;
        const long long key = ev.key[e];
        if (!whole && (key < Ta || key >= Tb)) continue;
        const int k = d.a + count_le(skeys + koff, d.b - d.a - 1, d.top, key);
        slice_add<UNIT>(d, sbins, k, V[e], wok[e], wb[e]);
      }
    }
  }
}

template <bool UNIT>
__global__ void __launch_bounds__(kSliceThreads, 1) k_slice_fill(const __grid_constant__ SliceParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = (int)(blockIdx.x % (unsigned)p.nslices);
  const int r = (int)(blockIdx.x / (unsigned)p.nslices);
  const SliceDev sl = p.slices[s];
  // [shared keys][shared bins][shared frags] then the slice's own [keys][bins][frags]
  long long* skeys = reinterpret_cast<long long*>(smem_raw);
  unsigned* sbins = reinterpret_cast<unsigned*>(smem_raw + slice_bytes(p.shared_keys, 0, 0));
  SliceFragDev* sfr = reinterpret_cast<SliceFragDev*>(smem_raw + slice_bytes(p.shared_keys, p.shared_words, 0));
  unsigned char* own = smem_raw + slice_bytes(p.shared_keys, p.shared_words, p.shared_frags);
  long long* okeys = reinterpret_cast<long long*>(own);
  unsigned* obins = reinterpret_cast<unsigned*>(own + slice_bytes(sl.nkeys, 0, 0));
  SliceFragDev* ofr = reinterpret_cast<SliceFragDev*>(own + slice_bytes(sl.nkeys, sl.nwords, 0));
  __shared__ double sred[(kSliceThreads / 32) * kStatSlots * 3];
  __shared__ int pace_budget;

  const int nsh = p.shared_frags;
  const int nown = sl.frag_end - sl.frag_begin;
  for (int i = threadIdx.x; i < p.shared_keys; i += blockDim.x) skeys[i] = p.keys[i];
  for (int i = threadIdx.x; i < sl.nkeys; i += blockDim.x) okeys[i] = p.keys[sl.key_base + i];
  for (int i = threadIdx.x; i < p.shared_words; i += blockDim.x) sbins[i] = 0u;
  for (int i = threadIdx.x; i < sl.nwords; i += blockDim.x) obins[i] = 0u;
  {
    constexpr int W = (int)(sizeof(SliceFragDev) / 4);
    const unsigned* src = reinterpret_cast<const unsigned*>(p.frags);
    const unsigned* srco = reinterpret_cast<const unsigned*>(p.frags + sl.frag_begin);
    unsigned* dst = reinterpret_cast<unsigned*>(sfr);
    unsigned* dsto = reinterpret_cast<unsigned*>(ofr);
    for (int i = threadIdx.x; i < W * nsh; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < W * nown; i += blockDim.x) dsto[i] = srco[i];
  }
  if (threadIdx.x == 0) pace_budget = kPaceBudget;
  __syncthreads();

  double core[kBatchMaxCols][3];
#pragma unroll
  for (int c = 0; c < kBatchMaxCols; ++c) core[c][0] = core[c][1] = core[c][2] = 0.0;
  double tail[kBatchMaxGroups * 3];
  for (int t = 0; t < kBatchMaxGroups * 3; ++t) tail[t] = 0.0;

  const unsigned long long* cq = reinterpret_cast<const unsigned long long*>(p.col[sl.col]);
  const unsigned long long* wq = UNIT ? nullptr : reinterpret_cast<const unsigned long long*>(p.w);
  const long long n = p.n;
  const int R = p.replicas, S = p.nslices;

  // software pipeline: the next tile's column and weights are in flight
  // while this one is filled
  EvCol ev, nev;
  unsigned long long wb[kSliceEv], nwb[kSliceEv];
  long long t = r;
  if (t < p.ntiles) {
    load_col(nev, cq, t * (long long)p.tile + threadIdx.x, n);
    load_w(nwb, wq, t * (long long)p.tile + threadIdx.x, n);
  }
  // j = (t - r) / R counts this block's tiles; its turn for the shared work
  // comes when j = s (mod S)
  int turn = s == 0 ? 0 : S - s, jp = 0;
  for (; t < p.ntiles; t += R, turn = (turn + 1 == S) ? 0 : turn + 1, jp = (jp + 1) & (kPaceEvery - 1)) {
    if (p.done != nullptr && jp == 0 && t >= p.window) pace(p.done + (t - p.window), S, &pace_budget);
    const long long i0 = t * (long long)p.tile + threadIdx.x;
#pragma unroll
    for (int e = 0; e < kSliceEv; ++e) {
      ev.xb[e] = nev.xb[e];
      wb[e] = nwb[e];
    }
    if (t + R < p.ntiles) {
      load_col(nev, cq, (t + R) * (long long)p.tile + threadIdx.x, n);
      load_w(nwb, wq, (t + R) * (long long)p.tile + threadIdx.x, n);
    }
    bool valid[kSliceEv], wok[kSliceEv];
    long long V[kSliceEv];
#pragma unroll
    for (int e = 0; e < kSliceEv; ++e) {
      valid[e] = i0 + (long long)e * kSliceThreads < n;
      wok[e] = UNIT ? true : fx_of(wb[e], p.fx_elo, &V[e]);
      if (UNIT) V[e] = 0;
      ev.key[e] = key_of(ev.xb[e]);
    }
    fill_frags<UNIT>(ofr, 0, nown, okeys, obins, ev, valid, V, wok, wb);

    if (turn == 0) {
      // this block's turn for the shared histograms and the statistics
#pragma unroll
      for (int c = 0; c < kBatchMaxCols; ++c) {
        if (c >= p.ncols) break;
        const bool has_h = p.shared_col_begin[c] < p.shared_col_begin[c + 1];
        const bool has_s = p.st.group_begin[c] < p.st.group_begin[c + 1];
        if (!has_h && !has_s) continue;
        EvCol evc;
        if (c == sl.col) {
          evc = ev;
        } else {
          load_col(evc, reinterpret_cast<const unsigned long long*>(p.col[c]), i0, n);
#pragma unroll
          for (int e = 0; e < kSliceEv; ++e) evc.key[e] = key_of(evc.xb[e]);
        }
        if (has_h) fill_frags<UNIT>(sfr, p.shared_col_begin[c], p.shared_col_begin[c + 1], skeys, sbins, evc, valid, V, wok, wb);
        if (has_s) {
#pragma unroll
          for (int e = 0; e < kSliceEv; ++e)
            if (valid[e]) stat_event<UNIT>(p.st, c, evc.key[e], evc.xb[e], wb[e], core[c], tail);
        }
      }
    }
    // progress of this block (thread 0's share stands for the block's: pacing
    // only needs an estimate)
    if (p.done != nullptr && threadIdx.x == 0) atomicAdd(p.done + t, 1);
  }
  __syncthreads();

  // block-private bins (shared histograms and the slice) -> the histograms'
  // exact global accumulators
  for (int f = 0; f < nsh + nown; ++f) {
    const SliceFragDev& d = f < nsh ? sfr[f] : ofr[f - nsh];
    const unsigned* fb = (f < nsh ? sbins : obins) + d.bin_off;
    const int nb = d.b - d.a;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      const unsigned a0 = fb[2 * j];
      if (UNIT) {
        if (a0) atomicAdd(&d.g_unit[d.a + j], (unsigned long long)a0);
      } else {
        const unsigned a1 = fb[2 * j + 1];
        if (a0) atomicAdd(&d.g_lo[d.a + j], (unsigned long long)a0);
        if (a1) atomicAdd(reinterpret_cast<unsigned long long*>(&d.g_hi[d.a + j]), (unsigned long long)a1);
      }
    }
  }
  block_stats_store(core, tail, sred, p.part_stats + (size_t)blockIdx.x * kStatSlots * 3);
}

}  // namespace

size_t slice_smem_bytes(int keys, int words, int frags) { return slice_bytes(keys, words, frags); }

int slice_max_blocks_per_sm(int block, size_t smem, int* per_sm) {
  const void* fn = reinterpret_cast<const void*>(&k_slice_fill<false>);
  const void* fu = reinterpret_cast<const void*>(&k_slice_fill<true>);
  if (block != kSliceThreads) return -1;
  {  // always: it also loads the kernel before the occupancy query
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
    if (cudaFuncSetAttribute(fu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  }
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, block, smem) != cudaSuccess) return -2;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fu, block, smem) != cudaSuccess) return -2;
  *per_sm = a < b ? a : b;
  return 0;
}

int launch_slice_fill(const SliceParams& p, int block, int grid, size_t smem, void* stream) {
  if (block != kSliceThreads || p.tile != kSliceThreads * kSliceEv) return -1;
  const void* fn = (p.w == nullptr) ? reinterpret_cast<const void*>(&k_slice_fill<true>)
                                    : reinterpret_cast<const void*>(&k_slice_fill<false>);
  {  // always: it also loads the kernel before the occupancy query
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  }
  void* args[] = {const_cast<SliceParams*>(&p)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, (cudaStream_t)stream) == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
