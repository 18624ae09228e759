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
