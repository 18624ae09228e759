// noalloc.cu -- a 1D bulk fill that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory manager (which owns every device allocation and may
// forbid or intercept raw CUDA allocations), allocation-free real-time or
// embedded loops, and callers that must not trigger the implicit
// synchronisation an allocation can cause.  hist_fill_bulk_noalloc serves
// them.  The caller passes the inputs and the outputs; every piece of
// scratch the fill needs (the axis thresholds, the per-block partial bins
// and statistics, the exact accumulators) lives in one file-scope
// __device__ array of fixed size, kNoallocScratchBytes.  Every GPU that loads
// the library holds that array until the process exits.
//
// The array's name means a device address only in device code.  Host code
// obtains that address per device with cudaGetSymbolAddress, once, with the
// device current: the first call of the entry point on each device does
// this set-up, so that first call should come before any stream capture;
// every later call only enqueues kernels and may be captured into a graph.
//
// All calls share the array and it keeps the last call's contents: each
// call clears the parts that must start at zero.  Calls whose work overlaps
// on the GPU (different streams, or different host threads, without
// ordering between them) race on the array and give wrong results; order
// them on one stream or with events.
//
// The axis thresholds travel to the device by value, as a kernel parameter
// of the set-up kernel (at most 1025 keys, 8.2 KB), so no host-to-device
// copy from pageable memory is needed: the call only enqueues kernels.
// The fill runs at most kNoallocMaxGrid blocks (the per-block partials
// region of the scratch is sized for that many); on a GPU whose regular
// fill would launch more, this fill launches fewer, larger-strided blocks
// (same results, possibly lower throughput).

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/hist.h"
#include "axis_compile.h"
#include "hist_internal.h"

namespace hgb {
namespace {

constexpr int kNoallocMaxBins = 1024;  // nbins + 2 flow bins
constexpr int kNoallocMaxGrid = 304;   // fill blocks (two per SM on GB300)
constexpr int kNoallocMaxDevices = 64;

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t kOffT = 0;                                                   // int64 [nbins+3]
constexpr size_t kOffLo = 16384;                                              // u64 [bins]
constexpr size_t kOffHi = kOffLo + 8 * kNoallocMaxBins;                       // i64 [bins]
constexpr size_t kOffCount = kOffHi + 8 * kNoallocMaxBins;                    // u64 [bins]
constexpr size_t kOffUnit = kOffCount + 8 * kNoallocMaxBins;                  // u64 [bins]
constexpr size_t kOffF64 = kOffUnit + 8 * kNoallocMaxBins;                    // double [bins]
constexpr size_t kOffStats = kOffF64 + 8 * kNoallocMaxBins;                   // double [kMaxStats]
constexpr size_t kOffPartStats = kOffStats + 256;                             // double [grid][kMaxStats]
constexpr size_t kOffPartBins = kOffPartStats + 8 * kMaxStats * kNoallocMaxGrid;  // uint4 [grid][bins]
constexpr size_t kNoallocScratchBytes = kOffPartBins + 16 * (size_t)kNoallocMaxBins * kNoallocMaxGrid;
static_assert(kOffLo >= 8 * (kNoallocMaxBins + 1), "threshold region too small");
static_assert(kOffPartStats % 256 == 0 && kOffPartBins % 256 == 0, "misaligned scratch region");
static_assert(kOffPartBins - kOffPartStats >= 8 * (size_t)kMaxStats * kNoallocMaxGrid,
              "statistics partials region smaller than kNoallocMaxGrid blocks");
static_assert((kOffPartStats - kOffLo) % 8 == 0, "accumulator region not a whole number of words");

// The thresholds of one axis, passed by value to the set-up kernel.
struct NoallocTable {
  int64_t T[kNoallocMaxBins + 1];  // nbins + 3 keys
  int nkeys;
};
static_assert(sizeof(NoallocTable) <= 32000, "kernel parameter beyond the 32 KB limit");

// The scratch itself (about 5 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device).  Returns nullptr on failure.
unsigned char* scratch_on_current_device(int device) {
  if (device < 0 || device >= kNoallocMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_ptr[device] == nullptr) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return nullptr;
    g_scratch_ptr[device] = static_cast<unsigned char*>(ptr);
  }
  return g_scratch_ptr[device];
}

// Set-up of one call: the thresholds into the scratch, the accumulators
// (fixed-point words, counts, binary64 words, statistics) to zero.
__global__ void __launch_bounds__(256) k_noalloc_setup(const __grid_constant__ NoallocTable t,
                                                      unsigned char* __restrict__ s) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  long long* T = reinterpret_cast<long long*>(s + kOffT);
  for (int i = tid; i < t.nkeys; i += nthr) T[i] = t.T[i];
  unsigned long long* z = reinterpret_cast<unsigned long long*>(s + kOffLo);
  constexpr int kWords = (int)((kOffPartStats - kOffLo) / 8);
  for (int i = tid; i < kWords; i += nthr) z[i] = 0ull;
}

// Neumaier's compensated addition (s, c) += v, as hist_result sums the
// binary64 words.
__device__ __forceinline__ void comp_add(double& s, double& c, double v) {
  const double t = __dadd_rn(s, v);
  if (isfinite(t))
    c = __dadd_rn(c, fabs(s) >= fabs(v) ? __dadd_rn(__dsub_rn(s, t), v) : __dadd_rn(__dsub_rn(v, t), s));
  s = t;
}

// Turn the exact accumulators into binary64 bin contents and statistics,
// as hist_result does on the host: content = (fixed-point words + unit
// entries) rounded once, plus the binary64 slow-path words; sum w is the
// exact sum over the statistics' bins.
__global__ void __launch_bounds__(256) k_noalloc_finish(const unsigned char* __restrict__ s, int nbins_total,
                                                       int nbins, int fx_elo, int stat_all, long long n_entries,
                                                       double* __restrict__ bins_out, double* __restrict__ stats_out) {
  const unsigned long long* lo = reinterpret_cast<const unsigned long long*>(s + kOffLo);
  const long long* hi = reinterpret_cast<const long long*>(s + kOffHi);
  const unsigned long long* unit = reinterpret_cast<const unsigned long long*>(s + kOffUnit);
  const double* f64 = reinterpret_cast<const double*>(s + kOffF64);
  const double* st = reinterpret_cast<const double*>(s + kOffStats);
  __shared__ __int128 s_fx[256];
  __shared__ double s_f64[256], s_c[256];
  __shared__ unsigned long long s_unit[256];
  const int shift = 1065 - fx_elo;
  const double lsb = ldexp(1.0, -shift);
  __int128 sel_fx = 0;
  double sel_f64 = 0.0, sel_c = 0.0;
  unsigned long long sel_unit = 0;
  for (int g = threadIdx.x; g < nbins_total; g += blockDim.x) {
    const __int128 fx = ((__int128)hi[g] << 32) + (__int128)lo[g] + ((__int128)unit[g] << shift);
    bins_out[g] = __dadd_rn(__dmul_rn((double)fx, lsb), f64[g]);
    if (stat_all || (g >= 1 && g <= nbins)) {
      sel_fx += fx;
      comp_add(sel_f64, sel_c, f64[g]);
      sel_unit += unit[g];
    }
  }
  s_fx[threadIdx.x] = sel_fx;
  s_f64[threadIdx.x] = sel_f64;
  s_c[threadIdx.x] = sel_c;
  s_unit[threadIdx.x] = sel_unit;
  __syncthreads();
  if (threadIdx.x == 0) {
    __int128 a = 0;
    double b = 0.0, c = 0.0;
    unsigned long long u = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      a += s_fx[t];
      comp_add(b, c, s_f64[t]);
      comp_add(b, c, s_c[t]);
      u += s_unit[t];
    }
    stats_out[0] = (double)n_entries;
    stats_out[1] = __dadd_rn(__dmul_rn((double)a, lsb), __dadd_rn(b, c));
    stats_out[2] = __dadd_rn(st[2], (double)u);
    stats_out[3] = st[3];
    stats_out[4] = st[4];
  }
}

}  // namespace
}  // namespace hgb

using namespace hgb;

extern "C" int hist_fill_bulk_noalloc(const hist_axis_t* axis, const double* values, const double* weights,
                                      int64_t n, uint32_t flags, double* bins_out, double* stats_out,
                                      hist_stream_t stream) {
  if (axis == nullptr || bins_out == nullptr || stats_out == nullptr || n < 0) return HIST_ERR_ARG;
  if (flags & ~HIST_STAT_OVERFLOWS) return HIST_ERR_ARG;
  if (n > 0 && values == nullptr) return HIST_ERR_ARG;
  if (validate_axis(axis->kind, axis->nbins, axis->xmin, axis->xmax, axis->edges) != 0) return HIST_ERR_AXIS;
  if (axis->nbins + 2 > kNoallocMaxBins) return HIST_ERR_TOO_LARGE;
  const uintptr_t m = (uintptr_t)values | (uintptr_t)weights | (uintptr_t)bins_out | (uintptr_t)stats_out;
  if (m & 7u) return HIST_ERR_ALIGN;
  int device = 0, sm_count = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return HIST_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HIST_ERR_CUDA;
  unsigned char* s = scratch_on_current_device(device);
  if (s == nullptr) return HIST_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // thresholds built on the host, handed to the set-up kernel by value
  // (with the zeroing of the accumulators, which start at zero every call)
  const int nb = axis->nbins;
  NoallocTable tab;
  tab.nkeys = nb + 3;
  float scale = 0.0f, offset = 0.0f, eps = 1.0f;
  int32_t mode = LOC_BSEARCH;
  if (axis->kind == HIST_AXIS_FIXED) {
    build_fixed_thresholds(nb, axis->xmin, axis->xmax, tab.T);
    if (affine_estimate(nb, axis->xmin, axis->xmax, &scale, &offset, &eps)) mode = LOC_AFFINE;
  } else {
    build_variable_thresholds(nb, axis->edges, tab.T);
  }
  k_noalloc_setup<<<8, 256, 0, st>>>(tab, s);
  if (cudaGetLastError() != cudaSuccess) return HIST_ERR_CUDA;

  if (n > 0) {
    const int acc = (weights == nullptr) ? ACC_UNIT : ACC_FX;
    FillParams p;
    std::memset(&p, 0, sizeof(p));
    AxisDev& a = p.ax[0];
    a.T = reinterpret_cast<const long long*>(s + kOffT);
    a.nbins = nb;
    a.mode = mode;
    a.smem_off = 0;
    a.scale = scale;
    a.offset = offset;
    a.eps = eps;
    p.col[0] = values;
    p.w = weights;
    p.T_concat = reinterpret_cast<const long long*>(s + kOffT);
    p.n = n;
    p.nbins_total = nb + 2;
    p.ndim = 1;
    p.nstats = 5;
    p.stat_overflows = (flags & HIST_STAT_OVERFLOWS) ? 1 : 0;
    p.track_counts = 0;
    p.fx_elo = 1015;
    p.table_keys = nb + 3;
    p.aligned = (((uintptr_t)values | (uintptr_t)weights) & 15u) == 0 ? 1 : 0;
    p.smem_bins = 1;
    p.part_bins = s + kOffPartBins;
    p.part_stats = reinterpret_cast<double*>(s + kOffPartStats);
    p.g_lo = reinterpret_cast<unsigned long long*>(s + kOffLo);
    p.g_hi = reinterpret_cast<long long*>(s + kOffHi);
    p.g_count = reinterpret_cast<unsigned long long*>(s + kOffCount);
    p.g_unit = reinterpret_cast<unsigned long long*>(s + kOffUnit);
    p.g_f64 = reinterpret_cast<double*>(s + kOffF64);
    LaunchShape shape;
    if (plan_fill(p, acc, sm_count, &shape) != 0) return HIST_ERR_CUDA;
    if (shape.grid > kNoallocMaxGrid) shape.grid = kNoallocMaxGrid;
    if (launch_fill(p, acc, shape, st) != 0) return HIST_ERR_CUDA;
    ReduceParams r;
    std::memset(&r, 0, sizeof(r));
    r.part_bins = p.part_bins;
    r.part_stats = p.part_stats;
    r.nblocks = shape.grid;
    r.nstats = 5;
    r.nbins_total = nb + 2;
    r.mode = acc;
    r.track_counts = 0;
    r.g_lo = p.g_lo;
    r.g_hi = p.g_hi;
    r.g_count = p.g_count;
    r.g_unit = p.g_unit;
    r.g_f64 = p.g_f64;
    r.g_stats = reinterpret_cast<double*>(s + kOffStats);
    if (launch_reduce(r, st) != 0) return HIST_ERR_CUDA;
  }
  k_noalloc_finish<<<1, 256, 0, st>>>(s, nb + 2, nb, 1015, (flags & HIST_STAT_OVERFLOWS) ? 1 : 0, (long long)n,
                                       bins_out, stats_out);
  if (cudaGetLastError() != cudaSuccess) return HIST_ERR_CUDA;
  return HIST_OK;
}
