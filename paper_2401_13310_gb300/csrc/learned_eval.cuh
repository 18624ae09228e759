// learned_eval.cuh -- device evaluation of the learned bin-index model.
//
// The model (used by the fill kernels, the trainer and the certifier, so the
// certified error window is measured on exactly the arithmetic the fill
// uses) is a continuous piecewise-linear function of the coordinate:
//   u = (xf - u0) * u_scale          (xf: the coordinate truncated to FP32)
//   s = clamp(floor(u), 0, S - 1),  t = min(u - s, 1)
//   k^ = K[s] + (K[s+1] - K[s]) * t,  K[j] = base[j] + bf16 residual[j]
// base[j] is the exact bin of the segment boundary (an int32), so the
// trainable bf16 residual only carries the shape within a segment.  The
// fill rounds k^ to k0, searches [k0 - W, k0 + W] exactly (W certified) and
// falls back to a full binary search whenever the window misses.
#pragma once

#include <cstdint>

#include "hist_internal.h"

namespace hgb {

__device__ __forceinline__ float lm_knot(int2 kn) {
  return __fadd_rn((float)kn.x, __uint_as_float(((unsigned)kn.y & 0xFFFFu) << 16));
}

// k^ for the FP32 coordinate xf.
__device__ __forceinline__ float lm_eval(const LearnedDev& m, float xf) {
  float u = __fmul_rn(__fsub_rn(xf, m.u0), m.u_scale);
  u = fmaxf(u, 0.0f);  // NaN -> 0
  int s = (int)fminf(u, (float)(m.nseg - 1));
  const float t = fminf(__fsub_rn(u, (float)s), 1.0f);
  const float ka = lm_knot(m.knots[s]);
  const float kb = lm_knot(m.knots[s + 1]);
  return __fmaf_rn(__fsub_rn(kb, ka), t, ka);
}

// Same model with FP32 knot values (training: master weights, no rounding).
__device__ __forceinline__ float lm_eval_master(float u0, float u_scale, int nseg, const int* base,
                                                const float* theta, float xf, int* seg, float* tt) {
  float u = __fmul_rn(__fsub_rn(xf, u0), u_scale);
  u = fmaxf(u, 0.0f);
  int s = (int)fminf(u, (float)(nseg - 1));
  const float t = fminf(__fsub_rn(u, (float)s), 1.0f);
  const float ka = __fadd_rn((float)base[s], theta[s]);
  const float kb = __fadd_rn((float)base[s + 1], theta[s + 1]);
  *seg = s;
  *tt = t;
  return __fmaf_rn(__fsub_rn(kb, ka), t, ka);
}

}  // namespace hgb
