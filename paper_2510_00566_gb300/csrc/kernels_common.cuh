// Warp-level helpers shared by the build and search kernels.
#pragma once

#include "device_common.cuh"

namespace pano {

// Exact-as-FP32-allows squared distance sum_j (a_j - b_j)^2 by one warp:
// each lane keeps a Kahan-compensated sum (s, c) of its strided terms (the
// value is s - c); lanes are combined pairwise with an error-free TwoSum of
// the s parts.  Relative error a few FP32 units (compensated summation), far
// below the plain d-term sum's d*u.  Every lane returns the result.
__device__ __forceinline__ float exact_sqdist_warp(const float* __restrict__ a,
                                                   const float* __restrict__ b, int d) {
  const int lane = threadIdx.x & 31;
  float s = 0.f, c = 0.f;
  for (int j = lane; j < d; j += 32) {
    float diff = a[j] - b[j];
    float t = diff * diff;
    float y = t - c;
    float u = s + y;
    c = (u - s) - y;
    s = u;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    float sum = s + s2;
    float bb = sum - s;
    float err = (s - (sum - bb)) + (s2 - bb);
    c = (c + c2) - err;
    s = sum;
  }
  return s - c;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace pano
