/*
 * hist.h -- C ABI of the GB300 bulk histogram-filling library (libhist.so).
 *
 * The operation (Chen, Dessole, Varbanescu 2024, Sec. 3.1 "Histogramming
 * Action"): for every event of a bulk, (1) find the bin of its coordinate on
 * each axis -- fixed-width bins by the formula
 * 1 + floor(nbins * (x - min) / (max - min)), variable-width bins by a binary
 * search over the edges, coordinates outside the range in the underflow bin 0
 * or the overflow bin nbins + 1, higher dimensions repeating the search per
 * axis -- (2) add one, or the event weight, to that bin, and (3) update the
 * statistics sums (Sec. 3.2: in 1D sum w, sum w^2, sum w*x, sum w*x^2).
 * As in the paper's GPU histogram class (Sec. 3.2), the library owns the
 * device allocations, fills bulk by bulk and copies the result back once.
 *
 * Semantics (the same readings as the CPU oracle that the tests compare
 * against):
 *   - bins are lower-inclusive [e_j, e_{j+1});
 *   - the fixed formula is evaluated left to right in binary64 without fused
 *     multiply-add, and a coordinate x < max is never overflow;
 *   - NaN coordinates go to the overflow bin; +-inf to overflow / underflow;
 *   - ND bins are linearised x fastest: g = b0 + (n0+2) * (b1 + (n1+2) * b2);
 *   - statistics cover events whose every axis bin is in range (all events
 *     with HIST_STAT_OVERFLOWS); slot 0 counts every event;
 *   - fills accumulate: a fill adds to the previous fills, never overwrites.
 *
 * Conventions: every function returns a status (HIST_OK = 0 or a negative
 * HIST_ERR_*); nothing is thrown across the ABI; all argument checks happen
 * on the host before any launch.  Device pointers are CUDA device (or
 * managed) addresses on the histogram's device; host pointers are ordinary
 * host memory.  A stream argument is a cudaStream_t (NULL = the legacy
 * default stream).
 */
#ifndef HIST_H
#define HIST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *hist_stream_t; /* the same type as cudaStream_t */

/* Status codes. */
enum {
  HIST_OK = 0,
  HIST_ERR_ARG = -1,      /* bad argument (null pointer, n < 0, bad flags, ...) */
  HIST_ERR_AXIS = -2,     /* invalid axis: nbins < 1, min >= max, non-finite or
                             non-increasing edges */
  HIST_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  HIST_ERR_OOM = -4,      /* device or host allocation failed */
  HIST_ERR_ALIGN = -5,    /* pointer not 8-byte aligned */
  HIST_ERR_TIMEOUT = -6,  /* a bounded device wait gave up */
  HIST_ERR_LOCATOR = -7,  /* learned locator not trained / unusable */
  HIST_ERR_STATE = -8,    /* call not valid in the object's current state */
  HIST_ERR_UNSUPPORTED = -9,
  HIST_ERR_TOO_LARGE = -10 /* size beyond a fixed maximum (hist_fill_bulk_noalloc) */
};

/* Axis kinds. */
enum { HIST_AXIS_FIXED = 0, HIST_AXIS_VARIABLE = 1 };

/* One axis.  FIXED: nbins bins of equal width on [xmin, xmax), both finite,
 * xmin < xmax, (xmax - xmin) finite.  VARIABLE: edges[0..nbins] strictly
 * increasing and finite (host pointer, copied by hist_book; xmin/xmax are
 * ignored). */
typedef struct {
  int32_t kind;
  int32_t nbins;
  double xmin, xmax;
  const double *edges;
} hist_axis_t;

/* Booking flags (bitwise or). */
#define HIST_TRACK_COUNTS (1u << 0)   /* keep per-bin entry counts for weighted fills */
#define HIST_STAT_OVERFLOWS (1u << 1) /* include under/overflow entries in the statistics */
#define HIST_SUMW2 (1u << 2)          /* also keep each bin's sum of squared weights (ROOT's Sumw2) */
/* HIST_STATS_EXACT: the statistics become the exact sums of their rounded
 * terms -- 1D w, fl(w*w), fl(w*x), fl(fl(w*x)*x); 2D adds fl(w*y),
 * fl(fl(w*y)*y), fl(fl(w*x)*y); 3D adds fl(w*z), fl(fl(w*z)*z),
 * fl(fl(w*x)*z), fl(fl(w*y)*z) -- rounded once to binary64:
 * bit-reproducible whatever the launch shape, the order of atomics or the
 * split into fills, and equal to a correctly rounded exact sum (math.fsum)
 * of the same terms.  Extra passes over each bulk (one per four
 * statistics: one in 1D, two in 2D, three in 3D) accumulate them in
 * integer limbs on a per-statistic grid (an escape accumulator takes the
 * terms outside it).  Not with hist_fill_columns or batches
 * (HIST_ERR_UNSUPPORTED). */
#define HIST_STATS_EXACT (1u << 3)
/* Accumulation of weighted bin contents (bits 4-5):
 *   HIST_PREC_FP64   (default) exact fixed-point sums of each weight truncated
 *                    to a multiple of 2^-50 (relative error <= 2^-42 per
 *                    weight with |w| in [2^-8, 2^8); other weights are added
 *                    in binary64); per-bin error <= 2.3e-13 * sum |w|;
 *                    bit-reproducible for in-window weights.
 *   HIST_PREC_FP32C  FP32 compensated partials: each weight split into FP32
 *                    hi + lo (|w - hi - lo| <= 2^-48 |w|); hi added to the
 *                    block's FP32 bin by an atomic whose rounding error is
 *                    recovered exactly (TwoSum on the returned old value) and
 *                    added with lo to an FP32 compensation word; blocks
 *                    flushed and summed in binary64.  Per bin, with m_b the
 *                    bin's entries in block b and A = sum |w|:
 *                      |err| <= 2^-48 ((max_b m_b + 1)^2 + 1) A + B 2^-53 A
 *                    (B blocks); the compensation words' rounding errors
 *                    are random in sign, so measured errors stay far below.
 *                    Weights outside [2^-40, 2^40), and histograms whose bins
 *                    outgrow shared memory, use binary64 atomics.
 *   HIST_PREC_F64ATOMIC  binary64 atomic adds (order-dependent rounding). */
#define HIST_PREC_FP64 (0u << 4)
#define HIST_PREC_FP32C (1u << 4)
#define HIST_PREC_F64ATOMIC (2u << 4)
#define HIST_PREC_MASK (3u << 4)
/* Variable-axis locator (bits 8-9), all exact (the same bins):
 *   HIST_LOCATOR_AUTO     (default) a bucket map when the axis has one: the
 *                         coordinate's bucket under a monotone linear or
 *                         logarithmic map, then that bucket's few thresholds;
 *                         else the binary search over the edges (Sec. 3.1);
 *   HIST_LOCATOR_LEARNED  as AUTO until hist_train_locator installs the
 *                         trained index model (windowed search, full
 *                         binary search on a miss);
 *   HIST_LOCATOR_BSEARCH  always the binary search over the edges. */
#define HIST_LOCATOR_AUTO (0u << 8)
#define HIST_LOCATOR_LEARNED (1u << 8)
#define HIST_LOCATOR_BSEARCH (2u << 8)
#define HIST_LOCATOR_MASK (3u << 8)

typedef struct hist hist_t; /* opaque; owns its device bins, statistics and axis tables */

/* Book a 1D-3D histogram on the current CUDA device (Sec. 3.1: the booking
 * of a histogram model with its axes).  Validates the axes, builds the exact
 * per-axis threshold tables and allocates the device state; no fill is in
 * flight afterwards.  *out receives the new object (owned by the caller,
 * released with hist_free).  Errors: HIST_ERR_ARG, HIST_ERR_AXIS,
 * HIST_ERR_OOM, HIST_ERR_CUDA. */
int hist_book(const hist_axis_t *axes, int ndim, uint32_t flags, hist_t **out);

/* Fill one bulk of n events (Sec. 3.1 steps 1-3; Sec. 3.2 fill per bulk).
 * values: device, column-major [ndim][n] (axis d at values + d*n), binary64.
 * weights: device [n] binary64, or NULL for unit weights.
 * Asynchronous and ordered on `stream`: the caller keeps the inputs alive and
 * unmodified until the stream has passed this call (the paper's Sec. 3.3
 * lesson: a host bulk must not be overwritten while its copy is in flight).
 * Fills accumulate.  n == 0 is a no-op.  Errors: HIST_ERR_ARG (null h or
 * values with n > 0, n < 0), HIST_ERR_ALIGN (pointer not 8-byte aligned),
 * HIST_ERR_CUDA. */
int hist_fill_bulk(hist_t *h, const double *values, const double *weights, int64_t n,
                   hist_stream_t stream);

/* Copy the accumulated result to host memory (the single copy-back of
 * Sec. 3.2).  Synchronises the stream of the last fill.
 * bins: host [nbins_total] binary64 bin contents, ROOT-linearised (x fastest,
 *       flow bins included), or NULL;
 * stats: host [hist_nstats] = [N, sum w, sum w^2, sum wx, sum wx^2
 *        (, sum wy, sum wy^2, sum wxy (, sum wz, sum wz^2, sum wxz, sum wyz))],
 *        or NULL.
 * Non-destructive: later fills keep accumulating. */
int hist_result(hist_t *h, double *bins, double *stats);

/* Host [nbins_total] entry counts per bin (exact).  Unit-weight histograms
 * always have them; weighted ones need HIST_TRACK_COUNTS (else
 * HIST_ERR_STATE). */
int hist_counts(hist_t *h, uint64_t *counts);

/* ---- fused Filter/Define -------------------------------------------------
 * The paper's RDataFrame example (Sec. 2, Listing 1) keeps the rows whose
 * x is nonzero, defines a new column r2 = x^2 + y^2 from two existing ones
 * and fills a histogram with it.  hist_fill_columns does all three in the fill
 * kernel, without writing the defined column: for each event i of the
 * source columns cols[0..ncols) (device [n] binary64 each, ncols <= 4), if
 * every filter holds (cols[col][i] <op> value, binary64 comparison; NaN
 * fails all but HIST_FLT_NE), axis d is filled with defines[d] evaluated in
 * binary64, each operation rounded once, left to right:
 *   HIST_DEF_COL    a                 HIST_DEF_MUL  a * b
 *   HIST_DEF_SUMSQ  a*a + b*b         HIST_DEF_ADD  a + b
 *   HIST_DEF_HYPOT  sqrt(a*a + b*b)   HIST_DEF_SUB  a - b
 * (a = cols[defines[d].a][i], b = cols[defines[d].b][i]; sqrt correctly
 * rounded), with weight weights[i] (device [n], or NULL).  Rows that fail a
 * filter are not entries.  1D and 2D histograms; at most 2 filters.
 * Asynchronous like hist_fill_bulk.  Errors: HIST_ERR_ARG, HIST_ERR_ALIGN,
 * HIST_ERR_UNSUPPORTED (3D, or HIST_SUMW2), HIST_ERR_CUDA. */
enum { HIST_DEF_COL = 0, HIST_DEF_SUMSQ = 1, HIST_DEF_HYPOT = 2, HIST_DEF_MUL = 3, HIST_DEF_ADD = 4, HIST_DEF_SUB = 5 };
enum { HIST_FLT_NE = 0, HIST_FLT_EQ = 1, HIST_FLT_LT = 2, HIST_FLT_LE = 3, HIST_FLT_GT = 4, HIST_FLT_GE = 5 };
typedef struct {
  int32_t op;   /* HIST_DEF_* */
  int32_t a, b; /* source column indices (b unused by HIST_DEF_COL) */
} hist_define_t;
typedef struct {
  int32_t col;  /* source column index */
  int32_t op;   /* HIST_FLT_* */
  double value; /* the constant compared with */
} hist_filter_t;
int hist_fill_columns(hist_t *h, const double *const *cols, int ncols, const hist_define_t *defines,
                      const hist_filter_t *filters, int nfilters, const double *weights, int64_t n,
                      hist_stream_t stream);

/* Per-bin sum of squared weights (the bin errors' input; with HIST_SUMW2),
 * host out [prod(nbins_d + 2)], every entry's w*w (1 for unit-weight
 * entries).  Weighted fills with the bins in shared memory keep it as FP32
 * compensated words (the square formed as an FP32 double-word, within
 * 2^-45 w^2 of fl(w*w)) flushed to binary64, with the error bound of
 * HIST_PREC_FP32C relative to sum w^2; otherwise binary64 atomics of
 * fl(w*w).  Synchronizes like hist_result.  Errors: HIST_ERR_ARG,
 * HIST_ERR_STATE (booked without HIST_SUMW2), HIST_ERR_CUDA.  Histograms
 * with HIST_SUMW2 cannot join a batch (HIST_ERR_UNSUPPORTED there). */
int hist_sumw2(hist_t *h, double *sumw2);

/* Fill from HOST memory, pipelined (Sec. 3.2 transfers bulks of events to
 * the GPU; Sec. 6 names pipelining the bulks as future work): values host
 * column-major [ndim][n], weights host [n] or NULL.  The events are cut into
 * bulks of `bulk` events (0: 2^22); bulk i is copied into one of two
 * library-owned device slots on one of the histogram's two copy streams while the
 * fill of bulk i-1 runs on `stream`, and filled from the slot on `stream`.
 * Pinned host memory makes the copies asynchronous (pageable memory works,
 * with the driver's staging).  Asynchronous: the caller keeps the host
 * buffers alive and unmodified until `stream` has passed the call.  Results
 * are those of hist_fill_bulk over the same events.  Errors: HIST_ERR_ARG,
 * HIST_ERR_OOM, HIST_ERR_CUDA. */
int hist_fill_host(hist_t *h, const double *values, const double *weights, int64_t n, int64_t bulk,
                   hist_stream_t stream);

/* Per-event linear bin index of a bulk (step 1 of Sec. 3.1 alone).
 * values as in hist_fill_bulk; out: device int64 [n].  Asynchronous on
 * `stream`.  Does not change the histogram. */
int hist_locate(hist_t *h, const double *values, int64_t n, int64_t *out, hist_stream_t stream);

/* How the fills find the bin on axis `axis`: 0 the fixed-width estimate with
 * its exact correction, 1 binary search over the thresholds, 2 the trained
 * index model, 3 the bucket map.  Returns the mode, or HIST_ERR_ARG. */
int hist_locator_mode(const hist_t *h, int axis);

/* Kernel timing (measurement aid; the paper has no counterpart): while on,
 * every hist_fill_bulk records a pair of CUDA events on its stream around
 * the fill kernel alone (not the partial-sum reduction that follows).
 * hist_kernel_time waits for the last recorded pair, returns the summed
 * milliseconds and the number of timed launches since the previous call,
 * and starts a new count.  Errors: HIST_ERR_ARG, HIST_ERR_CUDA. */
int hist_set_kernel_timing(hist_t *h, int on);
int hist_kernel_time(hist_t *h, double *ms, int64_t *launches);

/* ---- batched fill: many histograms, one event stream ---------------------
 * The paper's conclusion names computing several histograms from the same
 * data, and its kernels being small and launch-bound, as the next step.  A
 * batch fills up to 128 booked 1D histograms from up to 4 columns and one
 * weight column in one fused pass over the events, with one of three
 * privatisation strategies:
 *   wide   -- every block fills every histogram from its share of the
 *             events; small histograms keep exact per-block bins in shared
 *             memory, large ones use exact global integer atomics;
 *   sliced -- the batch's bins are cut into slices of one block's shared
 *             memory (large histograms span several slices); each block
 *             fills one slice from a share of the events, every bin stays
 *             in shared memory, and the slices sweep the event stream
 *             together so that each event is read from HBM once (from L2
 *             by the other slices);
 *   partitioned -- per column (at most 32 histograms each): the column's
 *             key space is cut into ranges such that every histogram's bins
 *             over one range, the range's merged thresholds of all its
 *             histograms and a row of per-histogram threshold counts per
 *             merged threshold fit one block's shared memory; the events
 *             (and weights) are counted per range, copied into a
 *             partitioned scratch column, and each range's events are filled
 *             by blocks holding that range: one search over the merged
 *             thresholds gives every histogram's bin.  Six kernels per
 *             column, columns one after the other; scratch of 8 bytes per
 *             event (16 weighted), kept by the batch.
 * Histograms that share a column and range share their statistics sums.
 * Results and accuracy per histogram are those of hist_fill_bulk.
 * Precision: a batch whose members are all booked with HIST_PREC_FP32C
 * runs the FP32 compensated form (wide or partitioned strategy): bins in
 * shared memory are FP32 (hi, lo) pairs with TwoSum on the atomic's old
 * value, flushed in binary64 (wide: the small histograms, the large ones
 * take binary64 atomics; partitioned: every histogram's slice of a range).
 * Every other batch keeps exact fixed-point bins (as HIST_PREC_FP64). */
typedef struct hist_batch hist_batch_t;

#define HIST_BATCH_GRAPH (1u << 0)  /* replay the fill's launches as a cached CUDA graph */
#define HIST_BATCH_WIDE (1u << 1)   /* start with the wide strategy (default: sliced when the */
#define HIST_BATCH_SLICED (1u << 2) /* bins outgrow one block's shared memory, else wide) */

/* Build a batch over hists[0..nh) (all 1D, same device); histogram i reads
 * column col_of_hist[i] (0..3).  At most 16 distinct (column, axis range)
 * pairs (statistics groups).
 * The batch references the histograms (they must outlive it) and owns its
 * device descriptors and scratch.  Errors: HIST_ERR_ARG, HIST_ERR_UNSUPPORTED
 * (ND histogram, more than 16 statistics groups, HIST_PREC_FP32C members
 * mixed with others, or all FP32C with HIST_BATCH_SLICED), HIST_ERR_OOM,
 * HIST_ERR_CUDA. */
int hist_batch_create(hist_t *const *hists, int nh, const int32_t *col_of_hist, uint32_t flags,
                      hist_batch_t **out);

/* Fill every histogram of the batch with the same n events: cols is a host
 * array of ncols device column pointers ([n] binary64 each), weights a
 * device [n] array or NULL (unit weights).  Asynchronous on `stream`,
 * ordered after earlier fills of the member histograms; fills accumulate.
 * Errors: HIST_ERR_ARG, HIST_ERR_ALIGN, HIST_ERR_CUDA. */
int hist_batch_fill(hist_batch_t *b, const double *const *cols, int ncols, const double *weights, int64_t n,
                    hist_stream_t stream);

typedef struct {
  int32_t candidates;      /* configurations timed */
  int32_t smem_bytes;      /* chosen shared-memory budget for block-private bins */
  int32_t blocks_per_sm;   /* chosen occupancy */
  int32_t smem_hists;      /* histograms kept in shared memory */
  double best_ms;          /* time of the chosen configuration on the sample */
  double worst_ms;         /* slowest candidate */
  int32_t strategy;        /* chosen strategy: 0 wide, 1 sliced, 2 partitioned */
  int32_t slices;          /* sliced: slices of the chosen plan; partitioned: ranges over all columns; 0 wide */
  int32_t replicas;        /* sliced: blocks per slice */
  int32_t cost_cap_tenths; /* sliced: work cap per slice of the chosen plan, tenths of one histogram */
  int32_t events_per_thread; /* events each fill thread holds at a time: wide, per pass over the
                                members (2 or 4); sliced 4; partitioned 2, or 4 in the kernel
                                compiled for two blocks per SM (tables too large for three) */
} hist_batch_tuning_t;

/* Autotune the batch (for fills like the sample: a unit-weight sample lets
 * the wide strategy keep one word per shared bin, which a later weighted
 * fill widens again): time the candidate strategies, shared-memory budgets
 * (which histograms keep shared-memory bins; the slice size), blocks per SM,
 * events per thread and work caps per slice on the given sample of events,
 * writing into scratch accumulators (the member histograms are not
 * changed), and keep the fastest for later fills.  The sample should be
 * like the later fills in size too: the partitioned strategy stages each
 * range's tables once per work item, a cost that small samples overweight
 * (about 1e7 events per column suffice).  Synchronous.  report may be
 * NULL.  Errors: as hist_batch_fill. */
int hist_batch_tune(hist_batch_t *b, const double *const *cols, int ncols, const double *weights, int64_t n,
                    hist_batch_tuning_t *report);

/* Pin the batch's configuration instead of tuning it: strategy 0 (wide),
 * 1 (sliced) or 2 (partitioned), the shared-memory budget per block in
 * bytes (partitioned: per range); for the sliced
 * strategy the work cap per slice in tenths of one histogram's
 * locate-and-add and the pacing window in tiles of 2048 events (-1 the
 * default, 0 no pacing); for the wide strategy the blocks per SM the kernel
 * is compiled for (2 or 4: its register budget) and the events each thread
 * holds (2 or 4).  info (may be NULL) receives the resulting plan (with
 * best_ms = worst_ms = 0).  Waits for the batch's earlier fills.  Errors:
 * HIST_ERR_ARG, HIST_ERR_UNSUPPORTED (the plan does not fit one block's
 * shared memory; partitioned: more than 32 histograms on a column, or
 * more than 2048 ranges on a column; sliced: an FP32C batch), HIST_ERR_OOM,
 * HIST_ERR_CUDA. */
int hist_batch_configure(hist_batch_t *b, int32_t strategy, int32_t smem_bytes, int32_t cost_cap_tenths,
                         int32_t pace_tiles, int32_t blocks_per_sm, int32_t events_per_thread,
                         hist_batch_tuning_t *info);

/* Release the batch (not its histograms).  NULL is a no-op. */
void hist_batch_free(hist_batch_t *b);

/* ---- learned locator (variable axes) ------------------------------------
 * A trained piecewise-linear index model predicts the bin of a coordinate;
 * an exact search inside a certified window corrects it, and a full binary
 * search judges every window miss, so results stay bit-exact.  The window
 * is certified for every non-NaN coordinate: the model, as the fill
 * evaluates it, is monotone in the coordinate within a segment, so its
 * largest index error lies at an end of a bin, of a segment, or of a
 * monotone piece of the FP32 truncation -- the certifier evaluates every
 * such end (NaN coordinates take the full search).  The model
 * over S uniform segments of u = (xf - u0) * u_scale (xf: the coordinate
 * truncated to FP32) has knots K[j] = base[j] + theta[j] (base: exact int32
 * bin at the knot; theta: a bf16 residual), k^ = K[s] (1 - t) + K[s+1] t.
 * Training: Adam on FP32 master weights minimising the mean squared error
 * against (coordinate, index) pairs taken from the exact binning -- each
 * bin j contributes (e_{j-1}, j - 1/2) and (its midpoint, j). */
typedef struct {
  int32_t segments; /* S; 0 = automatic (a power of two near nbins / 8, 16 .. 2^20) */
  int32_t steps;    /* Adam steps; 0 = 400 */
  float lr;         /* Adam learning rate, in bins; 0 = 0.05 */
  int32_t apply;    /* nonzero: later fills of this axis use the model */
} hist_locator_opts_t;

typedef struct {
  int32_t segments, steps;
  int32_t window_untrained; /* certified half-window of the model before training */
  int32_t window;           /* certified half-window after training */
  double loss_untrained;    /* mean squared index error on the training pairs */
  double loss;
  double train_ms;          /* wall time of training and certification */
} hist_locator_report_t;

/* Train, certify and (opts->apply) install the learned locator of variable
 * axis `axis` (0-based) on the GPU, with the library's own forward, backward
 * and update kernels.  Synchronous.  opts may be NULL (defaults); report may
 * be NULL.  Errors: HIST_ERR_ARG (bad axis index, fixed axis),
 * HIST_ERR_LOCATOR (degenerate axis range in FP32), HIST_ERR_OOM,
 * HIST_ERR_CUDA. */
int hist_train_locator(hist_t *h, int axis, const hist_locator_opts_t *opts, hist_locator_report_t *report);

/* One forward and backward pass of the locator's training loss on the GPU
 * (the kernels hist_train_locator uses), for checking its gradients.  All
 * pointers are host memory: base and theta [nseg + 1], x and target [n],
 * grad [nseg + 1] (out, dL/dtheta), loss (out, mean squared error).
 * Errors: HIST_ERR_ARG, HIST_ERR_OOM, HIST_ERR_CUDA. */
int hist_locator_loss_grad(int nseg, float u0, float u_scale, const int32_t *base, const float *theta,
                           const double *x, const float *target, int64_t n, double *loss, float *grad);

/* Allocation-free 1D fill.  The paper has no counterpart: this entry point
 * serves callers that cannot call cudaMalloc -- code running under another
 * framework's memory manager (which owns all device memory), allocation-free
 * real-time loops, callers that must avoid the synchronisation an allocation
 * may cause.  It fills one bulk of n events on a 1D axis (fixed or variable,
 * nbins + 2 <= 1024) and OVERWRITES the caller's device outputs:
 *   bins_out:  device double [nbins + 2], the bulk's bin contents;
 *   stats_out: device double [5] = [N, sum w, sum w^2, sum wx, sum wx^2].
 * values: device [n]; weights: device [n] or NULL (unit weights); flags: 0
 * or HIST_STAT_OVERFLOWS.  Same semantics and accuracy as hist_book +
 * hist_fill_bulk + hist_result on that bulk.  Asynchronous on `stream`: the
 * call only enqueues kernels (the axis thresholds reach the device as a
 * kernel argument, not by a copy).  The fill runs at most 304 blocks (two
 * per SM of a 152-SM GB300), the size the scratch's per-block region holds.
 * No device or host memory is allocated: the scratch is one fixed library
 * array of about 5 MB per device, held until the process exits.  The first
 * call on a device looks up that array's address (cudaGetSymbolAddress), so
 * make that first call before any stream capture; later calls may be
 * captured into a CUDA graph and replayed.  Calls share the array:
 * calls that overlap on the GPU (unordered streams or threads) race and give
 * wrong results.  Errors: HIST_ERR_ARG, HIST_ERR_AXIS, HIST_ERR_TOO_LARGE
 * (nbins + 2 > 1024), HIST_ERR_ALIGN, HIST_ERR_CUDA. */
int hist_fill_bulk_noalloc(const hist_axis_t *axis, const double *values, const double *weights, int64_t n,
                           uint32_t flags, double *bins_out, double *stats_out, hist_stream_t stream);

/* Zero bins, counts and statistics (synchronous). */
int hist_reset(hist_t *h);

/* Release all device and host state (synchronises first).  NULL is a no-op. */
void hist_free(hist_t *h);

/* Sizes. */
int64_t hist_nbins_total(const hist_t *h);
int hist_nstats(const hist_t *h);
int hist_ndim(const hist_t *h);

/* The exact threshold keys of one axis, as the device compares them (host
 * only; needs no GPU).  out: host int64 [axis->nbins + 3].  key(x) is the
 * int64 that orders like the binary64 x (-0 and +0 -> 0, NaN -> overflow);
 * out[0] = INT64_MIN, out[nbins+2] = INT64_MAX and, for k = 1..nbins+1,
 * out[k] = the least key whose coordinate lands in bin k or above under the
 * Sec. 3.1 rule of this axis.  The bin of x is the largest k with
 * out[k] <= key(x).  Errors: HIST_ERR_ARG, HIST_ERR_AXIS. */
int hist_axis_thresholds(const hist_axis_t *axis, int64_t *out);

/* The FP32 estimate the kernels locate a fixed axis with (host only; needs
 * no GPU).  For a coordinate x with |x| in [2^-126, 2^128) the device forms
 * v = fmaf(x24, scale, offset), x24 = x truncated to its leading 24
 * significant bits, and takes floor(v), clamped to [0, nbins + 1], as the
 * bin when the fraction of v lies more than eps from an integer; otherwise
 * (and for every other x) it compares the key of x with the thresholds of
 * hist_axis_thresholds.  eps bounds |v - (1 + q)|, q the quotient of the
 * Sec. 3.1 fixed-width formula in binary64, wherever that test can pass.
 * Returns HIST_OK when the axis takes the estimate, HIST_ERR_UNSUPPORTED
 * when no useful bound holds (nbins >= 2^21, extreme ranges): the kernels
 * then locate by the thresholds alone.  Errors: HIST_ERR_ARG, HIST_ERR_AXIS
 * (an invalid axis, or a variable one). */
int hist_axis_affine(const hist_axis_t *axis, float *scale, float *offset, float *eps);

/* Static description of a status code. */
const char *hist_strerror(int code);

/* Library version string. */
const char *hist_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HIST_H */
