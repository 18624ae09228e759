// axis_compile.cpp -- host-side axis validation and exact threshold tables.
//
// Compiled with -ffp-contract=off: the fixed-width formula below must round
// every operation separately, exactly as Sec. 3.1 of the paper states it
// (bin = 1 + floor(nbins * (x - min) / (max - min)), evaluated left to right
// in binary64), with the range tests first (x < min -> 0, !(x < max) ->
// nbins + 1) and the reading that a coordinate x < max is never overflow.
//
// The formula is monotone in x (each rounded operation is monotone), so the
// set of doubles that land in bin k or above is an up-set; its least element
// T[k] is found by galloping plus bisection over the int64 keys that order
// like doubles.  The device then locates any x exactly by comparing key(x)
// against T -- the fixed formula reproduced bit for bit with integer
// compares.  Variable axes (Sec. 3.1: binary search over the edges) use
// their edges as thresholds directly (lower-inclusive bins).

#include "axis_compile.h"

#include <cmath>
#include <cstdint>
#include <cstring>

namespace hgb {

namespace {
constexpr int64_t kKeyNegInf = -(int64_t)0x7FF0000000000000LL;
constexpr int64_t kKeyPosInf = (int64_t)0x7FF0000000000000LL;
}  // namespace

int64_t host_key(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  const uint64_t mag = b & 0x7FFFFFFFFFFFFFFFull;
  if (mag > 0x7FF0000000000000ull) return 0x7FFFFFFFFFFFFFFELL;  // NaN
  return (b >> 63) ? -(int64_t)mag : (int64_t)mag;
}

double host_double_of_key(int64_t k) {
  uint64_t b = (k >= 0) ? (uint64_t)k : ((uint64_t)(-k) | 0x8000000000000000ull);
  double x;
  std::memcpy(&x, &b, 8);
  return x;
}

int32_t host_fixed_bin(int32_t nbins, double xmin, double xmax, double x) {
  if (x < xmin) return 0;
  if (!(x < xmax)) return nbins + 1;
  const double d = x - xmin;
  const double t = (double)nbins * d;
  const double q = t / (xmax - xmin);
  if (q >= (double)nbins) return nbins;
  return 1 + (int32_t)q;
}

int validate_axis(int32_t kind, int32_t nbins, double xmin, double xmax, const double* edges) {
  if (nbins < 1 || nbins > (1 << 28)) return -1;
  if (kind == 0) {
    if (!std::isfinite(xmin) || !std::isfinite(xmax) || !(xmin < xmax)) return -1;
    if (!std::isfinite(xmax - xmin)) return -1;
    return 0;
  }
  if (kind == 1) {
    if (edges == nullptr) return -1;
    for (int32_t i = 0; i <= nbins; ++i)
      if (!std::isfinite(edges[i])) return -1;
    for (int32_t i = 0; i < nbins; ++i)
      if (!(edges[i] < edges[i + 1])) return -1;
    return 0;
  }
  return -1;
}

namespace {

struct FixedBinOfKey {
  int32_t nbins;
  double xmin, xmax;
  // Keys below key(-inf) / above key(+inf) act as -infinity / +infinity bins.
  int64_t operator()(int64_t K) const {
    if (K < kKeyNegInf) return -1;
    if (K > kKeyPosInf) return (int64_t)nbins + 2;
    return host_fixed_bin(nbins, xmin, xmax, host_double_of_key(K));
  }
};

inline int64_t mid_of(int64_t lo, int64_t hi) {
  const uint64_t span = (uint64_t)hi - (uint64_t)lo;  // < 2^64, no overflow
  return lo + (int64_t)(span / 2);
}

}  // namespace

void build_fixed_thresholds(int32_t nbins, double xmin, double xmax, int64_t* T) {
  const FixedBinOfKey bin{nbins, xmin, xmax};
  T[0] = INT64_MIN;
  T[nbins + 2] = INT64_MAX;
  int64_t prev = kKeyNegInf;  // T[k] >= T[k-1]
  const double width = (xmax - xmin) / (double)nbins;
  for (int32_t k = 1; k <= nbins + 1; ++k) {
    // starting guess: the exact edge position min + (k-1) * width
    double xe = (k == 1) ? xmin : (k == nbins + 1 ? xmax : xmin + (double)(k - 1) * width);
    int64_t g = host_key(xe);
    if (g < prev) g = prev;
    if (g > kKeyPosInf) g = kKeyPosInf;
    // bracket lo < hi with bin(lo) < k <= bin(hi), galloping away from g
    int64_t lo, hi;
    const int64_t floor_lo = prev - 1;  // every key below T[k-1] has bin < k - 1
    if (bin(g) >= k) {
      hi = g;
      uint64_t step = 1;
      for (;;) {
        const bool reach = (uint64_t)(hi - floor_lo) <= step;
        const int64_t cand = reach ? floor_lo : hi - (int64_t)step;
        if (reach || bin(cand) < k) {
          lo = cand;
          break;
        }
        hi = cand;
        step <<= 1;
      }
    } else {
      lo = g;
      uint64_t step = 1;
      const int64_t ceil_hi = kKeyPosInf + 1;
      for (;;) {
        const bool reach = (uint64_t)(ceil_hi - lo) <= step;
        const int64_t cand = reach ? ceil_hi : lo + (int64_t)step;
        if (reach || bin(cand) >= k) {
          hi = cand;
          break;
        }
        lo = cand;
        step <<= 1;
      }
    }
    while ((uint64_t)hi - (uint64_t)lo > 1) {
      const int64_t mid = mid_of(lo, hi);
      if (bin(mid) >= k)
        hi = mid;
      else
        lo = mid;
    }
    T[k] = hi;
    prev = hi;
  }
}

void build_variable_thresholds(int32_t nbins, const double* edges, int64_t* T) {
  T[0] = INT64_MIN;
  for (int32_t j = 0; j <= nbins; ++j) T[j + 1] = host_key(edges[j]);
  T[nbins + 2] = INT64_MAX;
}

bool affine_estimate(int32_t nbins, double xmin, double xmax, float* scale, float* offset, float* eps) {
  // The device evaluates v = fl32(xf * s + o) with xf the coordinate
  // truncated to 24 significant bits, s ~ S = nbins / W_d and o ~ O = 1 - xmin * S
  // (W_d = fl64(xmax - xmin), the width the formula divides by).  The
  // binary64 formula gives 1 + q64 with q64 = (x - xmin) * S * (1 + d),
  // |d| <= 3.01 * 2^-53.  Bound |v - (1 + q64)| over |x| <= X; beyond X the
  // estimate is more than a bin width outside the range and the clamp to
  // bin 0 / nbins + 1 decides correctly.
  const double W = xmax - xmin;
  const double S = (double)nbins / W;
  const double O = 1.0 - xmin * S;
  const float s = (float)S, o = (float)O;
  *scale = s;
  *offset = o;
  *eps = 1.0f;
  if (!std::isfinite(S) || !std::isfinite(O) || !std::isfinite((double)s) || !std::isfinite((double)o)) return false;
  if (nbins >= (1 << 21) || S > std::ldexp(1.0, 100) || S < std::ldexp(1.0, -100)) return false;
  const double X = std::fmax(std::fabs(xmin), std::fabs(xmax)) + W;
  const double u24 = std::ldexp(1.0, -24), u53 = std::ldexp(1.0, -53);
  if (X * S >= std::ldexp(1.0, 21) || std::fabs(O) >= std::ldexp(1.0, 21)) return false;
  const double ds = std::fabs((double)s - S) + u53 * S;                     // |s - exact S|
  const double dO = std::fabs((double)o - O) + 2 * u53 * (std::fabs(xmin) * S + std::fabs(O));
  const double e_trunc = X * std::fabs((double)s) * 2 * u24 + std::ldexp(1.0, -126) * std::fabs((double)s);
  const double e_scale = X * ds;
  const double e_fma = u24 * (X * std::fabs((double)s) * (1 + 4 * u24) + std::fabs((double)o));
  const double e_f64 = 4 * u53 * ((double)nbins + 2) + 2 * u53 * ((double)nbins + 2);
  const double e = 2.0 * (e_trunc + e_scale + dO + e_fma + e_f64);
  if (!(e < 0.25)) return false;
  *eps = (float)(e * (1 + 1e-6)) + std::ldexp(1.0f, -40);
  return true;
}

}  // namespace hgb

namespace hgb {

float host_est_float(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  const uint32_t hi = (uint32_t)(b >> 32);
  const uint32_t sgn = hi & 0x80000000u;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  uint32_t f = ((uint32_t)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu;
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7F000000u : f;
  f |= sgn;
  float r;
  std::memcpy(&r, &f, 4);
  return r;
}

// The device evaluates the same expressions: a shift of the key (key map),
// or __fmaf_rn on the truncated coordinate and a round-down conversion
// (linear map); both clamp.  Each is monotone in the key.
int bucket_of(const BucketMap& m, int64_t key) {
  int64_t b;
  if (m.key_map) {
    b = (key >> m.shift) - m.kbase;
  } else {
    float t = std::fmaf(host_est_float(host_double_of_key(key)), m.scale, m.offset);
    t = std::fmin(std::fmax(t, -1.0f), (float)m.nbk);
    b = (int64_t)std::floor(t);
  }
  return b < 0 ? 0 : (b > m.nbk - 1 ? m.nbk - 1 : (int)b);
}

namespace {

// Bucket of every threshold T[1..nbins+1] under map m; the most in one.
int bucket_histogram(const BucketMap& m, int32_t nbins, const int64_t* T, std::vector<int32_t>* count) {
  count->assign((size_t)m.nbk, 0);
  int most = 0;
  for (int32_t k = 1; k <= nbins + 1; ++k) {
    const int c = ++(*count)[(size_t)bucket_of(m, T[k])];
    if (c > most) most = c;
  }
  return most;
}

}  // namespace

int build_bucket_map(int32_t nbins, const int64_t* T, int32_t nbk, BucketMap* map, std::vector<int32_t>* cnt) {
  const int64_t k0 = T[1], k1 = T[nbins + 1];
  if (!(k1 > k0)) return -1;
  std::vector<int32_t> count, best_count;
  // key map: the smallest shift that spreads [k0, k1] over at most nbk buckets
  BucketMap km;
  std::memset(&km, 0, sizeof(km));
  km.nbk = nbk;
  km.key_map = 1;
  // (the difference in unsigned arithmetic: k1 - k0 can exceed INT64_MAX)
  while (km.shift < 63 && (uint64_t)(k1 >> km.shift) - (uint64_t)(k0 >> km.shift) >= (uint64_t)nbk) ++km.shift;
  km.kbase = k0 >> km.shift;
  int best = bucket_histogram(km, nbins, T, &best_count);
  *map = km;
  // linear map of the truncated coordinate, when the range is finite in FP32
  const float x0 = host_est_float(host_double_of_key(k0));
  const float x1 = host_est_float(host_double_of_key(k1));
  if (std::isfinite(x0) && std::isfinite(x1) && x1 > x0) {
    BucketMap lin;
    std::memset(&lin, 0, sizeof(lin));
    lin.nbk = nbk;
    lin.key_map = 0;
    lin.scale = (float)((double)nbk / ((double)x1 - (double)x0));
    lin.offset = (float)(-(double)x0 * (double)lin.scale);
    if (std::isfinite(lin.scale) && lin.scale > 0.0f && std::isfinite(lin.offset)) {
      const int most = bucket_histogram(lin, nbins, T, &count);
      if (most < best) {
        best = most;
        best_count.swap(count);
        *map = lin;
      }
    }
  }
  cnt->assign((size_t)nbk + 1, 0);
  for (int32_t b = 0; b < nbk; ++b) (*cnt)[(size_t)b + 1] = (*cnt)[(size_t)b] + best_count[(size_t)b];
  int top = 0;
  while (best > 0 && (top == 0 || top * 2 <= best)) top = top ? top * 2 : 1;
  map->top = top;
  return best;
}

}  // namespace hgb
