/*
 * hist_oracle.c -- plain, slow, obviously-correct CPU oracle for bulk
 * histogram filling.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library and its Python binding) never calls it, and it shares no code,
 * header, table or constant with that path.
 *
 * What it computes follows Chen, Dessole and Varbanescu, "Lessons Learned
 * Migrating CUDA to SYCL: A HEP Case Study with ROOT RDataFrame" (2024):
 *
 *   Sec. 3.1 (Histogramming Action): filling one event is three steps --
 *     (1) find the bin of the coordinate, (2) add one, or the event weight,
 *     to that bin, (3) update the sums used for the histogram statistics.
 *     Fixed-width bins: bin = 1 + floor(nbins * (x - min) / (max - min)).
 *     Variable-width bins: a binary search over the edges.
 *     A coordinate outside the range goes to the underflow or overflow bin.
 *     In 2D and 3D every axis is located on its own.
 *   Sec. 3.2 (Native CUDA): in one dimension the statistics are four sums,
 *     the sum of weights, of squared weights, of weight*x and of weight*x^2.
 *
 * Readings taken where the paper is silent or ambiguous (R1-R9; each is
 * pinned by the oracle's tests):
 *   R1  variable bins are lower-inclusive [e_j, e_{j+1}): bin = 1 + the index
 *       of the last edge <= x (an upper-bound search), which matches the
 *       fixed-width formula on its own edges.
 *   R2  fixed formula evaluated left to right in binary64, no fused
 *       multiply-add: d = x - min; t = nbins * d; q = t / (max - min).
 *   R3  a coordinate x < max is never overflow: when rounding makes q reach
 *       nbins the bin is clamped to nbins.
 *   R4  range tests come first, in this order: x < min -> 0;
 *       !(x < max) -> nbins + 1.  NaN therefore lands in the overflow bin.
 *   R5  statistics are summed over events whose every axis bin is in range,
 *       unless stat_overflows is set; the entry count N counts every event.
 *   R6  the 2D and 3D statistics add sum w*y, w*y^2, w*x*y (2D) and
 *       sum w*z, w*z^2, w*x*z, w*y*z (3D); products are rounded left to
 *       right, e.g. w*x*x = (w*x)*x.
 *   R7  ND bins are linearised with x fastest:
 *       g = b0 + (n0 + 2) * (b1 + (n1 + 2) * b2).
 *   R8  no event is dropped: every event lands in one of the
 *       prod(n_d + 2) bins.
 *   R9  NaN or infinite weights propagate by IEEE arithmetic.
 *
 * Two summation orders are produced for every weighted sum:
 *   *_seq  plain binary64 addition in event order (what a sequential
 *          CPU Fill does);
 *   *_acc  Neumaier-compensated addition (sum s plus correction c; the value
 *          is s + c), accurate to a few ulps of the exact sum; this is the
 *          reference that tolerances are measured against.
 * and Sum |term| for every sum (the scale in which tolerances are stated).
 *
 * Compile with -ffp-contract=off: contracting a*b+c into an FMA would change
 * the rounding of the formula in R2 and of the statistic terms in R6.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t kind;        /* 0 = fixed width, 1 = variable edges */
  int32_t nbins;       /* number of in-range bins, >= 1 */
  double xmin, xmax;   /* fixed width: the range [xmin, xmax) */
  const double *edges; /* variable: nbins + 1 strictly increasing edges */
} oracle_axis;

/* Sec. 3.1, fixed-width find-bin, with readings R2-R4. */
int32_t oracle_find_bin_fixed(int32_t nbins, double xmin, double xmax, double x) {
  if (x < xmin) return 0;
  if (!(x < xmax)) return nbins + 1;
  double d = x - xmin;
  double t = (double)nbins * d;
  double q = t / (xmax - xmin);
  if (q >= (double)nbins) return nbins; /* R3 */
  return 1 + (int32_t)q;                /* q >= 0 here, so the cast is floor */
}

/* Sec. 3.1, variable-width find-bin: binary search, reading R1. */
int32_t oracle_find_bin_variable(int32_t nbins, const double *edges, double x) {
  if (x < edges[0]) return 0;
  if (!(x < edges[nbins])) return nbins + 1;
  int32_t lo = 0, hi = nbins; /* invariant: edges[lo] <= x < edges[hi] */
  while (hi - lo > 1) {
    int32_t mid = lo + (hi - lo) / 2;
    if (x < edges[mid])
      hi = mid;
    else
      lo = mid;
  }
  return hi; /* x is in [edges[hi-1], edges[hi]), which is bin number hi */
}

static int32_t find_bin(const oracle_axis *a, double x) {
  if (a->kind == 0) return oracle_find_bin_fixed(a->nbins, a->xmin, a->xmax, x);
  return oracle_find_bin_variable(a->nbins, a->edges, x);
}

/* Number of statistics slots: [N, sum w, sum w^2, sum wx, sum wx^2, ...]. */
int32_t oracle_num_stats(int32_t ndim) {
  if (ndim == 1) return 5;
  if (ndim == 2) return 8;
  return 12;
}

int64_t oracle_num_bins(const oracle_axis *axes, int32_t ndim) {
  int64_t nb = 1;
  for (int32_t d = 0; d < ndim; ++d) nb *= (int64_t)axes[d].nbins + 2;
  return nb;
}

/* Per-event linear bin (steps (1) of Sec. 3.1 for every axis, then R7). */
void oracle_locate(const oracle_axis *axes, int32_t ndim, const double *values,
                   int64_t n, int64_t *out) {
  for (int64_t i = 0; i < n; ++i) {
    int64_t g = 0, stride = 1;
    for (int32_t d = 0; d < ndim; ++d) {
      int32_t b = find_bin(&axes[d], values[(int64_t)d * n + i]);
      g += stride * b;
      stride *= (int64_t)axes[d].nbins + 2;
    }
    out[i] = g;
  }
}

/* Neumaier's compensated addition: (s, c) += v. */
static void neumaier_add(double *s, double *c, double v) {
  double t = *s + v;
  if (isfinite(t)) {
    if (fabs(*s) >= fabs(v))
      *c += (*s - t) + v;
    else
      *c += (v - t) + *s;
  }
  *s = t;
}

typedef struct {
  uint64_t *counts;                 /* [nb] entries per bin */
  double *bins_seq;                 /* [nb] */
  double *bins_acc_s, *bins_acc_c;  /* [nb] */
  double *bins_abs;                 /* [nb] */
  double *stats_seq;                /* [ns] */
  double *stats_acc_s, *stats_acc_c;/* [ns] */
  double *stats_abs;                /* [ns] */
} oracle_out;

/* Sec. 3.1 steps (1)-(3) for events [i0, i1), in event order, accumulating
 * into o (which is not cleared: fills accumulate). */
static void fill_range(const oracle_axis *axes, int32_t ndim, const double *values,
                       const double *weights, int64_t n, int64_t i0, int64_t i1,
                       int32_t stat_overflows, const oracle_out *o) {
  const int32_t ns = oracle_num_stats(ndim);
  double term[12];
  for (int64_t i = i0; i < i1; ++i) {
    /* step (1): find the bin on every axis, then linearise (R7) */
    int64_t g = 0, stride = 1;
    int in_range = 1;
    double c[3] = {0.0, 0.0, 0.0};
    for (int32_t d = 0; d < ndim; ++d) {
      c[d] = values[(int64_t)d * n + i];
      int32_t b = find_bin(&axes[d], c[d]);
      if (b < 1 || b > axes[d].nbins) in_range = 0;
      g += stride * b;
      stride *= (int64_t)axes[d].nbins + 2;
    }
    /* step (2): add one, or the weight, to the bin */
    double w = weights ? weights[i] : 1.0;
    o->counts[g] += 1;
    o->bins_seq[g] += w;
    neumaier_add(&o->bins_acc_s[g], &o->bins_acc_c[g], w);
    o->bins_abs[g] += fabs(w);
    /* step (3): statistics (R5, R6); slot 0 counts every event */
    o->stats_seq[0] += 1.0;
    neumaier_add(&o->stats_acc_s[0], &o->stats_acc_c[0], 1.0);
    o->stats_abs[0] += 1.0;
    if (!in_range && !stat_overflows) continue;
    double x = c[0], y = c[1], z = c[2];
    double wx = w * x;
    term[0] = w;
    term[1] = w * w;
    term[2] = wx;
    term[3] = wx * x;
    if (ndim >= 2) {
      double wy = w * y;
      term[4] = wy;
      term[5] = wy * y;
      term[6] = wx * y;
    }
    if (ndim >= 3) {
      double wy = w * y, wz = w * z;
      term[7] = wz;
      term[8] = wz * z;
      term[9] = wx * z;
      term[10] = wy * z;
    }
    for (int32_t k = 1; k < ns; ++k) {
      double v = term[k - 1];
      o->stats_seq[k] += v;
      neumaier_add(&o->stats_acc_s[k], &o->stats_acc_c[k], v);
      o->stats_abs[k] += fabs(v);
    }
  }
}

static int check_axes(const oracle_axis *axes, int32_t ndim) {
  if (ndim < 1 || ndim > 3) return -1;
  for (int32_t d = 0; d < ndim; ++d) {
    if (axes[d].nbins < 1) return -1;
    if (axes[d].kind == 1 && axes[d].edges == NULL) return -1;
  }
  return 0;
}

/* Single-threaded fill in event order. */
int oracle_fill(const oracle_axis *axes, int32_t ndim, const double *values,
                const double *weights, int64_t n, int32_t stat_overflows,
                uint64_t *counts, double *bins_seq, double *bins_acc_s,
                double *bins_acc_c, double *bins_abs, double *stats_seq,
                double *stats_acc_s, double *stats_acc_c, double *stats_abs) {
  if (check_axes(axes, ndim) != 0 || n < 0) return -1;
  oracle_out o = {counts,    bins_seq,    bins_acc_s,  bins_acc_c, bins_abs,
                  stats_seq, stats_acc_s, stats_acc_c, stats_abs};
  fill_range(axes, ndim, values, weights, n, 0, n, stat_overflows, &o);
  return 0;
}

/* ---- chunk-parallel driver ------------------------------------------------
 * The event range is cut into nthreads contiguous chunks.  Each thread runs
 * the sequential fill above on its own chunk into private arrays; the chunks
 * are then merged in chunk order.  Counts are integers, so they are identical
 * to the sequential result; compensated sums stay compensated (each chunk's s
 * and c are added with the same compensated step); *_seq becomes the
 * chunk-order sum of per-chunk sequential sums. */
typedef struct {
  const oracle_axis *axes;
  int32_t ndim;
  const double *values, *weights;
  int64_t n, i0, i1;
  int32_t stat_overflows;
  oracle_out o;
} chunk_job;

static void *chunk_main(void *arg) {
  chunk_job *j = (chunk_job *)arg;
  fill_range(j->axes, j->ndim, j->values, j->weights, j->n, j->i0, j->i1,
             j->stat_overflows, &j->o);
  return NULL;
}

static int alloc_out(oracle_out *o, int64_t nb, int32_t ns) {
  memset(o, 0, sizeof(*o));
  o->counts = (uint64_t *)calloc((size_t)nb, sizeof(uint64_t));
  o->bins_seq = (double *)calloc((size_t)nb, sizeof(double));
  o->bins_acc_s = (double *)calloc((size_t)nb, sizeof(double));
  o->bins_acc_c = (double *)calloc((size_t)nb, sizeof(double));
  o->bins_abs = (double *)calloc((size_t)nb, sizeof(double));
  o->stats_seq = (double *)calloc((size_t)ns, sizeof(double));
  o->stats_acc_s = (double *)calloc((size_t)ns, sizeof(double));
  o->stats_acc_c = (double *)calloc((size_t)ns, sizeof(double));
  o->stats_abs = (double *)calloc((size_t)ns, sizeof(double));
  return (o->counts && o->bins_seq && o->bins_acc_s && o->bins_acc_c && o->bins_abs &&
          o->stats_seq && o->stats_acc_s && o->stats_acc_c && o->stats_abs)
             ? 0
             : -1;
}

static void free_out(oracle_out *o) {
  free(o->counts);
  free(o->bins_seq);
  free(o->bins_acc_s);
  free(o->bins_acc_c);
  free(o->bins_abs);
  free(o->stats_seq);
  free(o->stats_acc_s);
  free(o->stats_acc_c);
  free(o->stats_abs);
}

int oracle_fill_mt(const oracle_axis *axes, int32_t ndim, const double *values,
                   const double *weights, int64_t n, int32_t stat_overflows,
                   int32_t nthreads, uint64_t *counts, double *bins_seq,
                   double *bins_acc_s, double *bins_acc_c, double *bins_abs,
                   double *stats_seq, double *stats_acc_s, double *stats_acc_c,
                   double *stats_abs) {
  if (check_axes(axes, ndim) != 0 || n < 0 || nthreads < 1) return -1;
  if (nthreads == 1)
    return oracle_fill(axes, ndim, values, weights, n, stat_overflows, counts,
                       bins_seq, bins_acc_s, bins_acc_c, bins_abs, stats_seq,
                       stats_acc_s, stats_acc_c, stats_abs);
  const int64_t nb = oracle_num_bins(axes, ndim);
  const int32_t ns = oracle_num_stats(ndim);
  chunk_job *jobs = (chunk_job *)calloc((size_t)nthreads, sizeof(chunk_job));
  pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !tids) {
    free(jobs);
    free(tids);
    return -2;
  }
  int rc = 0;
  int32_t started = 0;
  for (int32_t t = 0; t < nthreads; ++t) {
    chunk_job *j = &jobs[t];
    j->axes = axes;
    j->ndim = ndim;
    j->values = values;
    j->weights = weights;
    j->n = n;
    j->i0 = n * t / nthreads;
    j->i1 = n * (t + 1) / nthreads;
    j->stat_overflows = stat_overflows;
    if (alloc_out(&j->o, nb, ns) != 0) {
      rc = -2;
      break;
    }
    if (pthread_create(&tids[t], NULL, chunk_main, j) != 0) {
      rc = -3;
      break;
    }
    started = t + 1;
  }
  for (int32_t t = 0; t < started; ++t) pthread_join(tids[t], NULL);
  if (rc == 0) {
    for (int32_t t = 0; t < nthreads; ++t) {
      const oracle_out *p = &jobs[t].o;
      for (int64_t g = 0; g < nb; ++g) {
        counts[g] += p->counts[g];
        bins_seq[g] += p->bins_seq[g];
        neumaier_add(&bins_acc_s[g], &bins_acc_c[g], p->bins_acc_s[g]);
        neumaier_add(&bins_acc_s[g], &bins_acc_c[g], p->bins_acc_c[g]);
        bins_abs[g] += p->bins_abs[g];
      }
      for (int32_t k = 0; k < ns; ++k) {
        stats_seq[k] += p->stats_seq[k];
        neumaier_add(&stats_acc_s[k], &stats_acc_c[k], p->stats_acc_s[k]);
        neumaier_add(&stats_acc_s[k], &stats_acc_c[k], p->stats_acc_c[k]);
        stats_abs[k] += p->stats_abs[k];
      }
    }
  }
  for (int32_t t = 0; t < nthreads; ++t) free_out(&jobs[t].o);
  free(jobs);
  free(tids);
  return rc;
}

/* Chunk-parallel per-event locate (the same find-bin, split over threads). */
typedef struct {
  const oracle_axis *axes;
  int32_t ndim;
  const double *values;
  int64_t n, i0, i1;
  int64_t *out;
} locate_job;

static void *locate_main(void *arg) {
  locate_job *j = (locate_job *)arg;
  for (int64_t i = j->i0; i < j->i1; ++i) {
    int64_t g = 0, stride = 1;
    for (int32_t d = 0; d < j->ndim; ++d) {
      int32_t b = find_bin(&j->axes[d], j->values[(int64_t)d * j->n + i]);
      g += stride * b;
      stride *= (int64_t)j->axes[d].nbins + 2;
    }
    j->out[i] = g;
  }
  return NULL;
}

int oracle_locate_mt(const oracle_axis *axes, int32_t ndim, const double *values,
                     int64_t n, int32_t nthreads, int64_t *out) {
  if (check_axes(axes, ndim) != 0 || n < 0 || nthreads < 1) return -1;
  locate_job *jobs = (locate_job *)calloc((size_t)nthreads, sizeof(locate_job));
  pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !tids) {
    free(jobs);
    free(tids);
    return -2;
  }
  int32_t started = 0;
  int rc = 0;
  for (int32_t t = 0; t < nthreads; ++t) {
    locate_job *j = &jobs[t];
    j->axes = axes;
    j->ndim = ndim;
    j->values = values;
    j->n = n;
    j->i0 = n * t / nthreads;
    j->i1 = n * (t + 1) / nthreads;
    j->out = out;
    if (pthread_create(&tids[t], NULL, locate_main, j) != 0) {
      rc = -3;
      break;
    }
    started = t + 1;
  }
  for (int32_t t = 0; t < started; ++t) pthread_join(tids[t], NULL);
  free(jobs);
  free(tids);
  return rc;
}
