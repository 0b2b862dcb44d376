// Warp-level helpers shared by the build and search kernels.
#pragma once

#include "device_common.cuh"

namespace pano {

__device__ __forceinline__ void kahan_add(float t, float& s, float& c) {
  float y = t - c;
  float u = s + y;
  c = (u - s) - y;
  s = u;
}

// Exact-as-FP32-allows squared distance sum_j (a_j - b_j)^2 by one warp:
// each lane keeps a Kahan-compensated sum (s, c) of its terms (the value is
// s - c); lanes are combined pairwise with an error-free TwoSum of the s
// parts.  Relative error a few FP32 units (compensated summation), far below
// the plain d-term sum's d*u.  Loads are issued in batches (several 16-byte
// loads in flight per lane) so the latency is paid a few times per row, not
// once per element.  Every lane returns the result.
__device__ __forceinline__ float exact_sqdist_warp(const float* __restrict__ a,
                                                   const float* __restrict__ b, int d) {
  const int lane = threadIdx.x & 31;
  float s = 0.f, c = 0.f;
  const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(a) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(b) & 15) == 0);
  if (vec) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const int d4 = d >> 2;
    for (int j0 = 0; j0 < d4; j0 += 4 * 32) {
      float4 av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + lane + 32 * u;
        av[u] = j < d4 ? a4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        bv[u] = j < d4 ? b4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float t;
        t = av[u].x - bv[u].x;
        kahan_add(t * t, s, c);
        t = av[u].y - bv[u].y;
        kahan_add(t * t, s, c);
        t = av[u].z - bv[u].z;
        kahan_add(t * t, s, c);
        t = av[u].w - bv[u].w;
        kahan_add(t * t, s, c);
      }
    }
  } else {
    for (int j0 = 0; j0 < d; j0 += 8 * 32) {
      float av[8], bv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + lane + 32 * u;
        av[u] = j < d ? a[j] : 0.f;
        bv[u] = j < d ? b[j] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float t = av[u] - bv[u];
        kahan_add(t * t, s, c);
      }
    }
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

// exact_sqdist_warp with the row fetched in batches of 8 float4 per lane per
// operand (one round of loads for d <= 1024) and two interleaved compensated
// sums per lane (half the dependent chain), combined by TwoSum at the end.
// For the re-ranking flushes, where a warp's distances are latency-bound.
__device__ __forceinline__ float exact_sqdist_warp_wide(const float* __restrict__ a,
                                                        const float* __restrict__ b, int d) {
  const int lane = threadIdx.x & 31;
  if ((d & 3) != 0 || ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15))
    return exact_sqdist_warp(a, b, d);
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  const int d4 = d >> 2;
  for (int j0 = 0; j0 < d4; j0 += 8 * 32) {
    float4 av[8], bv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + lane + 32 * u;
      av[u] = j < d4 ? a4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
      bv[u] = j < d4 ? b4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float t;
      t = av[u].x - bv[u].x;
      kahan_add(t * t, s0, c0);
      t = av[u].y - bv[u].y;
      kahan_add(t * t, s1, c1);
      t = av[u].z - bv[u].z;
      kahan_add(t * t, s0, c0);
      t = av[u].w - bv[u].w;
      kahan_add(t * t, s1, c1);
    }
  }
  // (s0 - c0) + (s1 - c1): TwoSum of the s parts, the c parts and the error
  // term summed plainly (the same pattern as the lane tree below)
  float s = s0 + s1;
  {
    const float bb = s - s0;
    const float err = (s0 - (s - bb)) + (s1 - bb);
    c0 = (c0 + c1) - err;
  }
  float c = c0;
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

// k-th smallest of the nv FP32 values vals[0..nv) (non-negative, +inf for
// absent entries) by one warp: binary search on the bit pattern for the
// least t with #{v <= t} >= k.  Returns +inf when fewer than k are finite.
__device__ __forceinline__ float warp_kth_smallest(const float* vals, int nv, int k) {
  const int lane = threadIdx.x & 31;
  int finite = 0;
  for (int i = lane; i < nv; i += 32) finite += vals[i] < INFINITY;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) finite += __shfl_xor_sync(0xffffffffu, finite, off);
  if (k <= 0 || finite < k) return INFINITY;
  uint32_t lo = 0, hi = 0x7f800000u;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    int cnt = 0;
    for (int i = lane; i < nv; i += 32) cnt += __float_as_uint(vals[i]) <= mid;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (cnt >= k) hi = mid;
    else lo = mid + 1;
  }
  return __uint_as_float(lo);
}

// k-th smallest of nv non-negative bf16 bit patterns (+inf = 0x7f80 for
// absent entries) by one warp; same search as warp_kth_smallest on 16 bits.
// Returns the value as FP32 (+inf when fewer than k are finite).
__device__ __forceinline__ float warp_kth_smallest_bf16(const uint16_t* vals, int nv, int k) {
  const int lane = threadIdx.x & 31;
  int finite = 0;
  for (int i = lane; i < nv; i += 32) finite += vals[i] < 0x7f80u;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) finite += __shfl_xor_sync(0xffffffffu, finite, off);
  if (k <= 0 || finite < k) return INFINITY;
  uint32_t lo = 0, hi = 0x7f80u;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    int cnt = 0;
    for (int i = lane; i < nv; i += 32) cnt += vals[i] <= mid;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (cnt >= k) hi = mid;
    else lo = mid + 1;
  }
  return __uint_as_float(lo << 16);
}

// Compensated FP32 sum of squares after Ogita, Rump & Oishi ("Accurate sum
// and dot product", SIAM J. Sci. Comput. 26(6), 2005): each term v*v is split
// exactly into p + e by an FMA (TwoProduct) and each addition s + p into
// t + err by TwoSum, so s + (exact sum of the error terms) is the exact sum;
// c accumulates those error terms in plain FP32.  The intrinsics keep the
// compiler from fusing the product into the addition, which would break the
// TwoSum identity.  For n terms spread over lanes, a 5-step lane tree and L
// level additions, the error of c is below (2n/32 + 2L + 12)(n/32 + L + 6) u^2
// of the sum, under 2^-30 of it for n <= 8192, L <= 64 (non-negative terms).
struct Acc2 {
  float s, c;
};

// TwoSum: t + err == x + y exactly.
__device__ __forceinline__ float two_sum(float x, float y, float& err) {
  const float t = __fadd_rn(x, y);
  const float bb = __fsub_rn(t, x);
  err = __fadd_rn(__fsub_rn(x, __fsub_rn(t, bb)), __fsub_rn(y, bb));
  return t;
}

__device__ __forceinline__ void acc2_sq(Acc2& a, float v) {
  const float p = __fmul_rn(v, v);
  const float e = __fmaf_rn(v, v, -p);
  float err;
  a.s = two_sum(a.s, p, err);
  a.c = __fadd_rn(a.c, __fadd_rn(err, e));
}

// Adds b into a.  Symmetric in a and b (TwoSum's t and err are, and so is
// a.c + b.c), so both lanes of a shuffle pair hold the same result.
__device__ __forceinline__ void acc2_add(Acc2& a, Acc2 b) {
  float err;
  a.s = two_sum(a.s, b.s, err);
  a.c = __fadd_rn(__fadd_rn(a.c, b.c), err);
}

__device__ __forceinline__ Acc2 warp_sum_acc2(Acc2 a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Acc2 b{__shfl_xor_sync(0xffffffffu, a.s, off), __shfl_xor_sync(0xffffffffu, a.c, off)};
    acc2_add(a, b);
  }
  return a;
}

// Upper bound of the exact sum held by a (relative slack 2^-23 over the
// 2^-30 error bound; FLT_MIN covers terms lost to underflow).
__device__ __forceinline__ float acc2_upper(Acc2 a, float rel) {
  return __fadd_ru(__fmul_ru(__fadd_ru(a.s, a.c), 1.0f + rel), 0x1p-126f);
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace pano
