// exact_round.cpp -- the host's once-rounding of an exactly summed statistic.
//
// The device leaves each statistic as signed radix-2^32 limbs on a fixed
// grid plus an escape accumulator on the grid 2^-1100; their sum is an exact
// integer multiple of 2^-1100.  Here it is assembled as one signed big
// integer, normalised to a sign and a magnitude, and rounded to the nearest
// binary64 (ties to even) -- the correctly rounded exact sum of the terms.

#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>

#include <cuda_runtime.h>

#include "hist_internal.h"

namespace hgb {

double exact_round(const long long* limbs, int grid, const long long* esc, const unsigned long long* special) {
  const unsigned long long nan = special[0], pinf = special[1], ninf = special[2];
  if (nan || (pinf && ninf)) return std::numeric_limits<double>::quiet_NaN();
  if (pinf) return std::numeric_limits<double>::infinity();
  if (ninf) return -std::numeric_limits<double>::infinity();
  // digits of 32 bits in units of 2^-kEscapeBias, as signed __int128 partial sums
  const int off = grid + kEscapeBias;  // bit offset of the fast limbs (>= 0)
  const int ndig = kEscapeLimbs + kExactLimbs + off / 32 + 4;
  std::vector<__int128> d((size_t)ndig, 0);
  for (int k = 0; k < kEscapeLimbs; ++k) d[(size_t)k] += esc[k];
  const int q = off / 32, r = off % 32;
  for (int j = 0; j < kExactLimbs; ++j) {
    const __int128 v = (__int128)limbs[j] << r;  // |v| < 2^95
    d[(size_t)(q + j)] += v;
  }
  // carry to radix 2^32 digits in [0, 2^32) with a signed top
  for (int k = 0; k + 1 < ndig; ++k) {
    __int128 c = d[(size_t)k] >> 32;
    d[(size_t)k] -= c << 32;
    d[(size_t)(k + 1)] += c;
  }
  const bool neg = d[(size_t)(ndig - 1)] < 0;
  if (neg) {  // the magnitude: negate every digit and carry again
    for (int k = 0; k < ndig; ++k) d[(size_t)k] = -d[(size_t)k];
    for (int k = 0; k + 1 < ndig; ++k) {
      const __int128 c = d[(size_t)k] >> 32;
      d[(size_t)k] -= c << 32;
      d[(size_t)(k + 1)] += c;
    }
  }
  // highest set bit
  int top = -1;
  for (int k = ndig - 1; k >= 0 && top < 0; --k)
    if (d[(size_t)k] != 0) {
      unsigned long long v = (unsigned long long)d[(size_t)k];
      int b = 63;
      while (!((v >> b) & 1ull)) --b;
      top = 32 * k + b;
    }
  if (top < 0) return 0.0;
  auto bit = [&](int pos) -> int {
    if (pos < 0) return 0;
    return (int)(((unsigned long long)d[(size_t)(pos / 32)] >> (pos % 32)) & 1ull);
  };
  // the 53 leading bits, then round to nearest even on the rest
  unsigned long long m = 0;
  for (int i = 0; i < 53; ++i) m = (m << 1) | (unsigned long long)bit(top - i);
  const int rpos = top - 53;  // first dropped bit
  int round = bit(rpos), sticky = 0;
  for (int pos = rpos - 1; pos >= 0 && !sticky; --pos) sticky |= bit(pos);
  // fewer than 53 significant bits: the value is exact
  if (top < 52) {
    m = 0;
    for (int pos = top; pos >= 0; --pos) m = (m << 1) | (unsigned long long)bit(pos);
    const double v = std::ldexp((double)m, -kEscapeBias);
    return neg ? -v : v;
  }
  if (round && (sticky || (m & 1ull))) ++m;  // may carry to 2^53: ldexp handles it exactly
  const double v = std::ldexp((double)m, rpos + 1 - kEscapeBias);
  return neg ? -v : v;
}

}  // namespace hgb
