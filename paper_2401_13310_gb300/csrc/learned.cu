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
// with K[j] = base[j] + theta[j].  The certifier evaluates the stored model
// (bf16 residuals) at both ends of every bin with the fill's own device
// function and records the largest index error.

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
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace hgb
