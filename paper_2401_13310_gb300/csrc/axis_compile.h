// axis_compile.h -- host-side axis validation and exact threshold tables.
#pragma once

#include <cstdint>
#include <vector>

namespace hgb {

// Key that orders like the double (-0 and +0 -> 0; NaN -> just below INT64_MAX).
int64_t host_key(double x);
double host_double_of_key(int64_t k);

// Sec. 3.1 fixed-width find-bin, binary64 without contraction, x < max never overflow.
int32_t host_fixed_bin(int32_t nbins, double xmin, double xmax, double x);

// 0 if the axis is valid (kind 0 fixed, 1 variable), -1 otherwise.
int validate_axis(int32_t kind, int32_t nbins, double xmin, double xmax, const double* edges);

// T must hold nbins + 3 keys: T[0] = INT64_MIN, T[nbins+2] = INT64_MAX and
// T[k] = least key whose coordinate's bin is >= k, k = 1..nbins+1.
void build_fixed_thresholds(int32_t nbins, double xmin, double xmax, int64_t* T);
void build_variable_thresholds(int32_t nbins, const double* edges, int64_t* T);

// FP32 estimate v = xf * scale + offset of 1 + q (q the binary64 quotient of
// the fixed-width formula) with a proven bound eps on |v - (1 + q)|; returns
// false when the axis is outside the range where such a bound stays < 1/4.
bool affine_estimate(int32_t nbins, double xmin, double xmax, float* scale, float* offset, float* eps);

// FP32 value of a binary64 with its significand truncated to 24 bits,
// saturating (|x| < 2^-126 -> +-0, |x| >= 2^128 -> +-2^127), from the bits
// exactly as the device computes it.
float host_est_float(double x);

// The bucket map and counts of a variable axis (T: its nbins + 3 keys) for
// the LOC_BUCKET locate; cnt receives nbk + 1 counts.  Returns the most
// thresholds that share one bucket, or -1 when no map applies.
struct BucketMap {
  int32_t nbk, key_map, shift, top;
  int64_t kbase;
  float scale, offset;
};
int build_bucket_map(int32_t nbins, const int64_t* T, int32_t nbk, BucketMap* map, std::vector<int32_t>* cnt);
int bucket_of(const BucketMap& m, int64_t key);

}  // namespace hgb
