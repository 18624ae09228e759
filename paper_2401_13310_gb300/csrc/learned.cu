// learned.cu -- training and certification kernels of the learned locator.
//
// The locator (see learned_eval.cuh) predicts the bin index of a coordinate
// on a variable-edge axis; an exact search inside a certified window
// corrects it, and a full binary search judges every window miss, so the
// fill stays exact whatever the model predicts.  Training is least squares
// on (coordinate, index) pairs drawn from the exact binning of the axis,
// with the in-bin fraction as a smooth target (edge e_{j-1} -> j - 1/2,
// bin midpoint -> j), by Adam on FP32 master weights:
//   forward   k^_i = K[s_i] (1 - t_i) + K[s_i + 1] t_i,   r_i = k^_i - y_i
//   loss      L = (1/N) sum_i r_i^2
//   backward  dL/dtheta[s_i] += 2 r_i (1 - t_i) / N,
//             dL/dtheta[s_i + 1] += 2 r_i t_i / N
// with K[j] = base[j] + theta[j].  The certifier bounds the index error of
// the stored model (bf16 residuals) over every non-NaN coordinate, with the
// fill's own device function: within one segment the evaluated model is a
// monotone function of the coordinate's key (each step -- truncation to
// FP32, x - u0, the scaling, u - s, the fused multiply-add with fixed knots
// -- is a correctly rounded monotone operation), and so is the rounded
// index; the bin is constant on each bin's key range.  So on every run of
// keys that lies in one bin and one segment, the error is largest at one
// of the run's two ends, and every such end is a bin end, a segment end, or
// an end of a monotone piece of the FP32 truncation (its saturation at
// 2^128).  The certifier evaluates all of them; the largest error is the
// window.  (A NaN coordinate's FP32 value does not follow its key; NaNs,
// like any window miss, take the full binary search.)

#include <cuda_runtime.h>

#include <cstdint>

#include "hist_internal.h"
#include "learned_eval.cuh"

namespace hgb {
namespace {

__device__ __forceinline__ float trunc24(unsigned long long b) {
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned e = (hi >> 20) & 0x7FFu;
  unsigned f = ((unsigned)(b >> 29) - 0xC0000000u) & 0x7FFFFFFFu;
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7F000000u : f;
  return __uint_as_float(f | (hi & 0x80000000u));
}

__global__ void __launch_bounds__(256) k_lm_fwd_bwd(float u0, float u_scale, int nseg, const int* __restrict__ base,
                                                    const float* __restrict__ theta,
                                                    const unsigned long long* __restrict__ x,
                                                    const float* __restrict__ target, long long n,
                                                    float* __restrict__ grad, double* __restrict__ loss) {
  __shared__ double sl[8];
  const float inv_n2 = 2.0f / (float)n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int s;
    float t;
    const float kh = lm_eval_master(u0, u_scale, nseg, base, theta, trunc24(x[i]), &s, &t);
    const float r = __fsub_rn(kh, target[i]);
    acc += (double)r * (double)r;
    const float g = __fmul_rn(r, inv_n2);
    atomicAdd(&grad[s], __fmul_rn(g, __fsub_rn(1.0f, t)));
    atomicAdd(&grad[s + 1], __fmul_rn(g, t));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sl[w];
    atomicAdd(loss, t / (double)n);
  }
}

__global__ void k_lm_adam(float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2,
                          const float* __restrict__ grad, int count, float lr, float b1, float b2, float eps,
                          float corr1, float corr2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float g = grad[i];
  const float a = b1 * m1[i] + (1.0f - b1) * g;
  const float v = b2 * m2[i] + (1.0f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  theta[i] -= lr * (a / corr1) / (sqrtf(v / corr2) + eps);
}

// knots = {base, bf16(theta) rounded to nearest even}
__global__ void k_lm_pack(const int* __restrict__ base, const float* __restrict__ theta, int2* __restrict__ knots,
                          int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const unsigned u = __float_as_uint(theta[i]);
  const unsigned r = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
  knots[i] = make_int2(base[i], (int)r);
}

__device__ __forceinline__ unsigned long long bits_of_key(long long k) {
  return (k >= 0) ? (unsigned long long)k : ((unsigned long long)(-k) | 0x8000000000000000ull);
}

// Segment of the model at the FP32 value xf, as lm_eval computes it.
__device__ __forceinline__ int lm_segment(const LearnedDev& m, float xf) {
  float u = __fmul_rn(__fsub_rn(xf, m.u0), m.u_scale);
  u = fmaxf(u, 0.0f);
  return (int)fminf(u, (float)(m.nseg - 1));
}

// Bin of a key: the largest k in [0, nbins + 1] with T[k] <= key.
__device__ __forceinline__ int bin_of_key(const long long* T, int nbins, long long key) {
  int base = 0, len = nbins + 2;
  while (len > 1) {
    const int half = len >> 1;
    base = (T[base + half] <= key) ? base + half : base;
    len -= half;
  }
  return base;
}

__device__ __forceinline__ int key_error(const LearnedDev& m, const long long* T, int nbins, long long key) {
  const float kh = lm_eval(m, trunc24(bits_of_key(key)));
  const int k0 = (int)floorf(__fadd_rn(kh, 0.5f));
  return abs(k0 - bin_of_key(T, nbins, key));
}

constexpr long long kKeyInf = 0x7FF0000000000000LL;  // key of +inf (-inf: its negation)
constexpr long long kKey2p128 = 0x47F0000000000000LL;  // key of 2^128, where the FP32 truncation saturates

// Segment boundaries and the ends of the truncation's monotone pieces:
// thread b < nseg - 1 finds the first key of segment b + 1 (the model's
// segment is monotone in the key between the saturation points; bisection
// over keys) and evaluates that key and the one before it; the special
// keys (+-inf, +-2^128 and their neighbours) are evaluated by thread 0.
__global__ void __launch_bounds__(256) k_lm_certify_knots(const LearnedDev m, const long long* __restrict__ T,
                                                          int nbins, int* __restrict__ max_err) {
  int worst = 0;
  const int nb = m.nseg - 1;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    // within [-(2^128) + 1 key, 2^128 - 1 key] the truncation is monotone
    long long lo = -kKey2p128 + 1, hi = kKey2p128 - 1;
    if (lm_segment(m, trunc24(bits_of_key(lo))) > b || lm_segment(m, trunc24(bits_of_key(hi))) <= b) continue;
    while (hi - lo > 1) {  // invariant: segment(lo) <= b < segment(hi)
      const long long mid = lo + ((hi - lo) >> 1);
      if (lm_segment(m, trunc24(bits_of_key(mid))) <= b)
        lo = mid;
      else
        hi = mid;
    }
    worst = max(worst, max(key_error(m, T, nbins, lo), key_error(m, T, nbins, hi)));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long sp[8] = {-kKeyInf, -kKey2p128, -kKey2p128 + 1, kKey2p128 - 1, kKey2p128, kKeyInf, 0, -1};
#pragma unroll
    for (int i = 0; i < 8; ++i) worst = max(worst, key_error(m, T, nbins, sp[i]));
  }
  atomicMax(max_err, worst);
}

// Largest |round(k^) - bin| over both ends of every bin (and the two flow
// sides), evaluated with the fill's device function.
__global__ void __launch_bounds__(256) k_lm_certify(const LearnedDev m, const long long* __restrict__ T, int nbins,
                                                    int* __restrict__ max_err) {
  int worst = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= nbins + 1; j += gridDim.x * blockDim.x) {
    // bin j covers keys [T[j], T[j+1]); flows: j = 0 below T[1], j = nbins+1 from T[nbins+1]
    long long lo = T[j], hi = T[j + 1] - 1;
    if (j == 0) lo = hi;                        // the last double below the first edge
    if (j == nbins + 1) hi = lo;                // the last edge itself
    const long long ends[2] = {lo, hi};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float kh = lm_eval(m, trunc24(bits_of_key(ends[e])));
      const int k0 = (int)floorf(__fadd_rn(kh, 0.5f));
      const int err = abs(k0 - j);
      worst = max(worst, err);
    }
  }
  atomicMax(max_err, worst);
}

}  // namespace

int launch_lm_fwd_bwd(float u0, float u_scale, int nseg, const int* base, const float* theta,
                      const unsigned long long* x, const float* target, long long n, float* grad, double* loss,
                      void* stream) {
  if (n <= 0) return 0;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_lm_fwd_bwd<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(u0, u_scale, nseg, base, theta, x, target, n, grad,
                                                              loss);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_lm_adam(float* theta, float* m1, float* m2, const float* grad, int count, float lr, float b1, float b2,
                   float eps, int step, void* stream) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_lm_adam<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, m1, m2, grad, count, lr, b1, b2, eps, c1,
                                                                     c2);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_lm_pack(const int* base, const float* theta, int2* knots, int count, void* stream) {
  k_lm_pack<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(base, theta, knots, count);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_lm_certify(const LearnedDev& m, const long long* T, int nbins, int* max_err, void* stream) {
  long long blocks = ((long long)nbins + 2 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_lm_certify<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(m, T, nbins, max_err);
  if (cudaGetLastError() != cudaSuccess) return -2;
  long long kblocks = ((long long)m.nseg + 255) / 256;
  if (kblocks > 152 * 8) kblocks = 152 * 8;
  k_lm_certify_knots<<<(int)kblocks, 256, 0, (cudaStream_t)stream>>>(m, T, nbins, max_err);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
