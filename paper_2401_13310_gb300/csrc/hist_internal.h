// hist_internal.h -- types shared by the library's host and device code.
//
// Every axis, fixed or variable, is reduced at booking time to a table of
// threshold keys T[0..nbins+2]: T[0] = INT64_MIN, T[nbins+2] = INT64_MAX and,
// for k = 1..nbins+1, T[k] is the smallest key whose coordinate falls in bin
// k or above.  The bin of x is then the largest k with T[k] <= key(x), where
// key() maps a binary64 to an int64 that orders like the double (-0 and +0
// share key 0; NaN maps just below INT64_MAX, i.e. to the overflow bin).
// For a variable axis T[k] = key(edge[k-1]) (Sec. 3.1 binary search over
// the edges, lower-inclusive bins).  For a fixed axis the host finds T[k] by
// bisection over keys with the binary64 formula of Sec. 3.1, which is
// monotone in x, so the device reproduces the formula exactly with integer
// comparisons and never needs binary64 arithmetic.
#pragma once

#include <cstdint>

namespace hgb {

constexpr int kMaxDim = 3;
constexpr int kMaxStats = 12;
constexpr long long kNanKey = 0x7FFFFFFFFFFFFFFELL;

// How the device finds the bin on one axis.
enum LocMode : int32_t {
  LOC_AFFINE = 0,   // FP32 affine estimate from the coordinate, then <= 1 step correction
  LOC_BSEARCH = 1,  // branchless binary search over the thresholds
  LOC_LEARNED = 2,  // trained piecewise-linear index model + windowed search
  LOC_BUCKET = 3,   // monotone bucket map of the coordinate + the bucket's few thresholds
};

// LOC_BUCKET: a monotone map m of the in-range key onto nbk buckets
// (linear in the coordinate: floor(xf * scale + offset), xf the coordinate
// truncated to FP32; or a shift of the key itself: (key >> shift) - kbase,
// which is logarithmic in the coordinate), and cnt[b] = the number of
// thresholds T[1..nbins+1] whose own key maps below bucket b.  Every
// threshold below bucket b is <= any key in it and every one above is
// greater, so the bin of an in-range key in bucket b is cnt[b] plus the
// number of the bucket's own thresholds T[cnt[b]+1 .. cnt[b+1]] that are <=
// the key.
// When no bucket holds more than one threshold the table is stored as
// (threshold, cnt) pairs instead, one 16-byte load per locate: the bin is
// cnt[b] + (key >= the bucket's threshold), INT64_MAX standing for none.
struct BucketDev {
  const int* cnt;          // [nbk + 1] counts, or [nbk] (threshold, cnt) int64 pairs when `single`
                           // (global; the fill kernels may stage it)
  long long lo_key;        // T[1]: keys below are underflow
  long long hi_key;        // T[nbins + 1]: keys from here on are overflow
  long long kbase;         // key map: bucket = (key >> shift) - kbase
  int32_t nbk;             // number of buckets
  int32_t key_map;         // 1: key map, 0: linear map
  float scale, offset;     // linear map
  int32_t shift;           // key map
  int32_t top;             // largest power of two <= the most thresholds in one bucket (0: none)
  int32_t smem_off;        // offset of the table in the shared copy (ints), -1: global
  int32_t single;          // 1: the pair table
};

// How weights reach the bins.
enum AccMode : int32_t {
  ACC_UNIT = 0,  // unit weights: u32 counters
  ACC_FX = 1,    // exact fixed-point sums (u32 limb atomics with carries)
  ACC_F64 = 2,   // binary64 atomics
  ACC_F32C = 3,  // FP32 compensated (hi, lo) partials
};

struct LearnedDev {
  const int2* knots;  // [nseg + 1] {exact bin at the segment boundary, bf16 residual in the low 16 bits}
  float u0, u_scale;  // u = (xf - u0) * u_scale in [0, nseg)
  int32_t nseg;
  int32_t window;     // certified half-width of the exact search window
};

struct AxisDev {
  const long long* T;  // device thresholds (nbins + 3 keys)
  int32_t nbins;
  int32_t mode;        // LocMode
  int32_t smem_off;    // offset of this axis' keys in the shared copy, -1 = read T from global
  float scale, offset; // LOC_AFFINE: v = xf * scale + offset estimates 1 + q of the formula
  float eps;           // proven bound on |v - (1 + q)|; floor(v) is exact when frac(v) is farther than eps from an integer
  LearnedDev lm;
  BucketDev bk;
};

// Fused Filter/Define (the paper's RDataFrame example, Sec. 2): events of
// the source columns that pass every filter are filled with coordinates
// computed per axis in binary64, each operation rounded once, left to right.
constexpr int kExprMaxSrc = 4;
constexpr int kExprMaxFilters = 2;
enum DefineOp : int32_t { DEF_COL = 0, DEF_SUMSQ = 1, DEF_HYPOT = 2, DEF_MUL = 3, DEF_ADD = 4, DEF_SUB = 5 };
enum FilterOp : int32_t { FLT_NE = 0, FLT_EQ = 1, FLT_LT = 2, FLT_LE = 3, FLT_GT = 4, FLT_GE = 5 };
struct ExprDev {
  const double* src[kExprMaxSrc];
  int32_t nsrc, nfilt;
  int32_t def_op[kMaxDim], def_a[kMaxDim], def_b[kMaxDim];
  int32_t filt_col[kExprMaxFilters], filt_op[kExprMaxFilters];
  double filt_val[kExprMaxFilters];
  unsigned long long* g_passed;  // events that passed the filters (entry count)
};

// Exactly summed statistics (HIST_STATS_EXACT): see stats_exact.cu.
constexpr int kExactStats = 11;    // statistics slots 1..11: sum w, w^2, wx, wx^2 (1D), + wy, wy^2, wxy (2D),
                                   // + wz, wz^2, wxz, wyz (3D)
constexpr int kExactGroup = 4;     // statistics summed in one pass (their limbs live in registers)
constexpr int kExactLimbs = 6;     // radix-2^32 limbs per statistic
constexpr int kExactFastTop = 32 * (kExactLimbs - 2) - 1;  // largest bit offset of a term's lowest bit
constexpr int kEscapeLimbs = 72;   // limbs of the escape accumulator (every finite double)
constexpr int kEscapeBias = 1100;  // its lowest limb is 2^-1100
struct ExactParams {
  const double* col[kMaxDim];   // coordinates, one column per axis
  const double* w;              // nullptr: unit weights
  long long n;
  int32_t ndim;
  int32_t stat_overflows;
  long long lo_key[kMaxDim], hi_key[kMaxDim];  // the in-range keys [T[1], T[nbins+1]) per axis
  int32_t s0, ns;               // this pass sums statistics s0 .. s0 + ns - 1 (0 = sum w), ns <= kExactGroup
  int32_t grid[kExactStats];    // each statistic's grid exponent
  long long* limbs;             // [kExactStats][kExactLimbs]
  long long* escape;            // [kExactStats][kEscapeLimbs]
  unsigned long long* special;  // [kExactStats][3]: NaN, +inf, -inf terms
};
int launch_stats_exact(const ExactParams& p, bool unit, int sm_count, void* stream);
int launch_exact_normalise(long long* limbs, void* stream);

// The exact value of sum_j limbs[j] 2^(32 j + grid) + sum_k esc[k] 2^(32 k - kEscapeBias),
// rounded once to binary64 (nearest, ties to even), with the special-term counts.
double exact_round(const long long* limbs, int grid, const long long* esc, const unsigned long long* special);

struct FillParams {
  AxisDev ax[kMaxDim];
  ExprDev ex;                   // used by the expression kernels only
  const double* col[kMaxDim];
  const double* w;              // nullptr = unit weights
  const long long* T_concat;    // all axes' keys back to back (shared-memory staging source)
  const int* BK_concat;         // all bucket-mapped axes' bucket counts back to back
  int32_t table_bk;             // bucket counts staged into shared memory
  long long n;
  long long nbins_total;
  int32_t ndim;
  int32_t nstats;
  int32_t stat_overflows;
  int32_t track_counts;
  int32_t fx_elo;               // biased binary64 exponent of the fixed-point window's low end
  int32_t table_keys;           // keys staged into shared memory (sum over staged axes)
  int32_t aligned;              // columns and weights all 16-byte aligned
  int32_t smem_bins;            // 1 = per-block shared-memory bins, 0 = global atomics
  int32_t sumw2;                // 1 = also the per-bin sum of squared weights (weighted fills)
  // direct flush (exact fixed-point or unit-count shared bins, no sum of
  // w^2): each block adds its bins to the persistent accumulators with
  // integer atomics, and the last block to finish (ticket: a counter that
  // starts at 0 and that block resets) adds the statistics partials in block
  // order into g_stats -- no partial bins and no reduce launch
  int32_t direct_flush;
  unsigned* ticket;
  double* g_stats;
  // per-launch partial results (scratch)
  void* part_bins;              // [grid][nbins_total] words per bin depend on the mode
  double* part_stats;           // [grid][kMaxStats]
  // persistent accumulators owned by the histogram
  unsigned long long* g_lo;     // fixed point: sum of the low 32 bits of every addend
  long long* g_hi;              // fixed point: sum of (addend >> 32)
  unsigned long long* g_count;  // entries of weighted fills (HIST_TRACK_COUNTS)
  unsigned long long* g_unit;   // entries of unit-weight fills (each adds weight 1)
  double* g_f64;                // binary64 bins (F64 mode, F32C mode, FX slow path)
  double* g_sumw2;              // binary64 per-bin sum of w^2 (sumw2)
  double* part_sumw2;           // [grid][nbins_total] block partials of sum w^2 (sumw2, shared bins)
};

struct ReduceParams {
  const void* part_bins;
  const double* part_stats;
  int32_t nblocks;      // number of per-block partials
  int32_t slice;        // partials summed by one reducing thread
  int32_t nstats;
  long long nbins_total;
  int32_t mode;          // AccMode
  int32_t track_counts;
  unsigned long long* g_lo;
  long long* g_hi;
  unsigned long long* g_count;
  unsigned long long* g_unit;
  double* g_f64;
  double* g_stats;
  const double* part_sumw2;     // [nblocks][nbins_total] or nullptr
  double* g_sumw2;
};

// ---- batched fill: many 1D histograms from one event stream -------------
constexpr int kBatchMaxCols = 4;     // columns per batch
constexpr int kBatchMaxGroups = 16;  // statistics groups: distinct (column, range) pairs
constexpr int kStatSlots = kBatchMaxCols + kBatchMaxGroups;  // partial sums: a core per column, a tail per group

// Statistics of a batch.  The statistics of a 1D histogram depend only on
// its column and its in-range test, so members with the same column and
// range share a group.  The groups of a column overlap on a common core
// [core_lo, core_hi) (keys; empty when lo >= hi): an event in the core adds
// to the column's core sums once, for all its groups; only the rare event
// outside it walks the column's groups and adds to the tail sums of those
// whose range holds it.  A group's sums are its column's core plus its tail.
struct BatchStatsSpec {
  long long core_lo[kBatchMaxCols], core_hi[kBatchMaxCols];
  long long group_lo[kBatchMaxGroups], group_hi[kBatchMaxGroups];
  int32_t group_begin[kBatchMaxCols + 1];  // groups sorted by column: [group_begin[c], group_begin[c+1])
  int32_t pad;
};

struct BatchHistDev {
  AxisDev ax;                   // T: global thresholds; smem_off: staged keys (-1: global)
  int32_t col;                  // column read by this histogram
  int32_t group;                // statistics group (same column and range)
  int32_t sbin_off;             // word offset of its per-block bins in shared memory, -1: global atomics
  int32_t pad;                  // (the batch's precision is a kernel-template choice: see batch.cu)
  unsigned long long* g_lo;     // the histogram's accumulators (or tuning scratch)
  long long* g_hi;
  unsigned long long* g_unit;
  double* g_f64;
};

struct BatchParams {
  const double* col[kBatchMaxCols];
  const double* w;              // nullptr: unit weights
  const BatchHistDev* hists;    // device [nh]
  const long long* T_concat;    // staged keys of all staged axes, back to back
  double* part_stats;           // [grid][kStatSlots][3]: sum w^2, sum wx, sum wx^2
  long long n;
  int32_t ncols, nh, fx_elo;
  int32_t table_keys;           // staged keys (8-byte keys + 4-byte high words each)
  int32_t sbin_words;           // shared-memory words of all block-private bins
  int32_t aligned;
  int32_t col_begin[kBatchMaxCols + 1];  // histograms sorted by column: [col_begin[c], col_begin[c+1])
  BatchStatsSpec st;
};

struct BatchReduceParams {
  const double* part_stats;
  int32_t nblocks, nh;
  const int* hist_col;          // device [nh]
  const int* hist_group;        // device [nh]
  double* const* hist_stats;    // device [nh] pointers to each histogram's statistics
};

// Sliced strategy: the large histograms' bins are cut into slices that
// each fit one block's shared memory; a slice is a run of fragments (a
// histogram's bin range [a, b)), all on one column.  Block (slice s,
// replica r) fills slice s from the event tiles t = r, r + R, r + 2R, ...
// so the R replicas of every slice sweep the stream together and each tile
// is read from HBM once and from L2 by every slice.  The small histograms
// are held whole by every block (the "shared" fragments) and filled, with
// the statistics, by one block per tile (the slice (t / R) mod S), which
// spreads that work and its hot bins over every block.
struct SliceFragDev {
  AxisDev ax;                   // T: global thresholds (fixed axes' rare exact step)
  long long Ta, Tb;             // the fragment holds the keys [Ta, Tb) = [T[a], T[b])
  int32_t a, b;                 // bins [a, b) of the histogram (flows included)
  int32_t key_off;              // shared offset of T[a+1 .. b-1] (non-affine axes); -1: affine locate
  int32_t top;                  // largest power of two <= b - a - 1 (0 if none)
  int32_t bin_off;              // shared word offset of bin a (two words per bin)
  int32_t whole;                // 1: a = 0 and b = nbins + 2 (no range test)
  unsigned long long* g_lo;     // the histogram's accumulators (bin 0 based) or tuning scratch
  long long* g_hi;
  unsigned long long* g_unit;
  double* g_f64;
};

struct SliceDev {
  int32_t col;                  // column of every fragment
  int32_t frag_begin, frag_end; // its fragments [frag_begin, frag_end) of the plan
  int32_t key_base, nkeys;      // its keys in the concatenated key array
  int32_t nwords;               // shared words of its bins
};

struct SliceParams {
  const double* col[kBatchMaxCols];
  const double* w;              // nullptr: unit weights
  const SliceDev* slices;       // device [nslices]
  const SliceFragDev* frags;    // device: shared fragments first, then the slices'
  const long long* keys;        // concatenated keys: the shared fragments' first
  double* part_stats;           // [grid][kStatSlots][3]
  int* done;                    // [ntiles] slices finished per tile (pacing only), or nullptr
  long long n;
  long long ntiles;
  int32_t nslices, replicas, ncols;
  int32_t tile;                 // events per tile
  int32_t window;               // a block starts tile t once tile t - window is done everywhere (0: off)
  int32_t shared_frags;         // fragments [0, shared_frags) are the small histograms, by column:
  int32_t shared_col_begin[kBatchMaxCols + 1];  // [shared_col_begin[c], shared_col_begin[c+1])
  int32_t shared_keys, shared_words;            // their keys (at 0) and bin words (at 0)
  int32_t max_frags, max_keys, max_words;       // largest slice (shared-memory sizing)
  int32_t fx_elo;
  BatchStatsSpec st;
};

// Partitioned strategy (batch_partition.cu): every member reads one column;
// its key space is cut into ranges [S_r, S_r+1) whose slices (each member's
// bins over the range) fit one block's shared memory together with the
// range's merged thresholds: the distinct thresholds of all members strictly
// inside the range, sorted, and for each position p among them (p of them
// <= a key) every member's count of its own thresholds among the first p --
// so one binary search gives every member's bin.  The events are partitioned
// by range, then each work item (a range and a run of its events) fills the
// slices in shared memory.
constexpr int kPartBlock = 256;
constexpr int kPartMaxMembers = 32;   // members per column of a partitioned batch (16-bit counts, rows <= 64 bytes)
constexpr int kPartMaxRanges = 2048;
constexpr int kPartTile = 2048;       // events per tile of the count and scatter passes (8 per thread)
struct PartRangeDev {
  int32_t key_base;             // its merged thresholds in the concatenated key array
  int32_t nkeys;                // how many (M); positions p = 0 .. M
  int32_t nbins;                // bin slots of all its slices
  int32_t cum_base;             // its count rows (M + 1 of row_u16 each) in the concatenated count array
  // bucket map of the merged thresholds (the axes' bucket map, on them):
  // keys below lo_key have position 0, keys from hi_key on position M; a
  // key in between lies in bucket b, whose thresholds are merged positions
  // bcnt[b] .. bcnt[b + 1] - 1
  int64_t lo_key, hi_key;       // first and last merged threshold (M >= 1; M = 0: both INT64_MAX)
  int64_t kbase;                // key map: bucket = (key >> shift) - kbase
  float scale, offset;          // linear map of the truncated coordinate
  int32_t bk_base;              // its bucket counts ([nbk + 1] u16) in the concatenated bucket array
  int32_t nbk;                  // buckets (0: M <= 1, the bounds decide)
  int32_t key_map, shift;
  int32_t top;                  // largest power of two <= the most thresholds in one bucket (0: none)
  int32_t pad;
};
struct PartSliceDev {           // one member over one range
  int32_t a;                    // first bin
  int32_t len;                  // bins a .. a + len - 1
  int32_t boff;                 // its first bin slot in the range's shared bins
  int32_t rsh;                  // log2 of its copies per bin: bin a + c has slots boff + (c << rsh) + (lane & (2^rsh - 1))
};
struct PartItem {
  long long e0, e1;             // events [e0, e1) of the partitioned column
  int32_t r;                    // their range
  int32_t pad;
};
struct PartParams {
  const double* col;            // the column
  const double* w;              // weights or nullptr
  double* px;                   // [n] the column partitioned by range
  double* pw;                   // [n] the weights alike (weighted fills)
  const long long* splits;      // [nranges - 1] split keys S_1 .. S_{nranges-1}
  const PartRangeDev* ranges;   // [nranges]
  const PartSliceDev* slices;   // [nranges][nh]
  const long long* keys;        // every range's merged thresholds, back to back
  const unsigned short* cum;    // every range's count rows, back to back
  const unsigned short* bcnt;   // every range's bucket counts, back to back
  const unsigned short* sbcnt;  // the split keys' bucket counts ([split_map.nbk + 1])
  PartRangeDev split_map;       // the bucket map of the split keys (nkeys = nranges - 1)
  const BatchHistDev* hists;    // [nh] the members' accumulators (or tuning scratch)
  unsigned* counts;             // [nranges][grid_count] events per (range, block)
  unsigned long long* offsets;  // [nranges][grid_count] their exclusive prefix sums
  unsigned long long* rtotal;   // [nranges] events per range
  unsigned long long* rstart;   // [nranges] first event of each range in the partitioned column
  int* ibase;                   // [nranges] first work item of each range
  PartItem* items;              // [max_items] the fill's work items
  int* nitems;                  // how many
  double* part_stats;           // [fill grid][kStatSlots][3]
  long long n;
  int32_t nranges, nh, grid_count, fx_elo;
  int32_t chunk;                // events per work item at most
  int32_t max_items;
  int32_t max_keys, max_bins;   // the largest range's thresholds and bin slots
  int32_t max_nbk;              // the most buckets of a range
  int32_t row_u16;              // u16 per count row: nh rounded up to 8, 16, 24 or 32
  int32_t stat_col;             // the column's index among the batch's columns (its statistics slots)
  BatchStatsSpec st;
};
size_t part_count_smem(int nranges, int split_nbk);
size_t part_scatter_smem(int nranges, int split_nbk, bool weighted);
size_t part_fill_smem(int max_keys, int max_bins, int nh, int row_u16, int max_nbk, int slot_bytes);
int part_grids(int sm_count, int nranges, int split_nbk, size_t fill_smem, int* count_grid, int* fill_per_sm);
// events each thread of the partitioned fill holds at a time (2 or 4) for
// this precision, count row and shared-memory size
int part_fill_events(bool unit, bool f32c, int row, size_t fill_smem);
int launch_part_fill(const PartParams& p, bool unit, bool f32c, int fill_grid, size_t fill_smem, void* stream);

int launch_slice_fill(const SliceParams& p, int block, int grid, size_t smem, void* stream);
int slice_max_blocks_per_sm(int block, size_t smem, int* per_sm);
size_t slice_smem_bytes(int keys, int words, int frags);

int launch_batch_fill(const BatchParams& p, int block, int grid, size_t smem, int minb, int kev, bool f32c,
                      void* stream);
int batch_max_blocks_per_sm(int block, size_t smem, int minb, int kev, int* per_sm);
int launch_batch_reduce(const BatchReduceParams& r, void* stream);

// Launchers (fill_kernels.cu).
struct LaunchShape {
  int grid;
  int block;
  size_t smem;
};

int plan_fill(const FillParams& p, int acc_mode, int sm_count, LaunchShape* shape);
// Whether a fill has a kernel that flushes its bins itself (p.direct_flush).
bool fill_direct_ok(const FillParams& p, int acc_mode);
int launch_fill(const FillParams& p, int acc_mode, const LaunchShape& shape, void* stream);
int launch_reduce(const ReduceParams& r, void* stream);
int launch_locate(const FillParams& p, long long* out, void* stream);
int launch_normalize_fx(unsigned long long* g_lo, long long* g_hi, long long nbins, void* stream);

// Learned locator (learned.cu).  All pointers are device pointers.
int launch_lm_fwd_bwd(float u0, float u_scale, int nseg, const int* base, const float* theta,
                      const unsigned long long* x, const float* target, long long n, float* grad, double* loss,
                      void* stream);
int launch_lm_adam(float* theta, float* m1, float* m2, const float* grad, int count, float lr, float b1, float b2,
                   float eps, int step, void* stream);
int launch_lm_pack(const int* base, const float* theta, int2* knots, int count, void* stream);
int launch_lm_certify(const LearnedDev& m, const long long* T, int nbins, int* max_err, void* stream);
size_t part_bin_bytes(int acc_mode, int track_counts);
size_t smem_bin_bytes(int acc_mode, int track_counts, int sumw2 = 0);  // per bin, block-private shared memory

}  // namespace hgb
