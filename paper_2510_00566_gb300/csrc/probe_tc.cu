// Coarse-probe distances on the tensor cores (Section 6.1: a query probes its
// nprobe nearest IVF lists).  pd[q][c] = |q|^2 + |c|^2 - 2 q.c for a tile of
// 128 queries x 256 centroids per CTA; the dot products are three bf16
// tcgen05 MMAs per K-step (hi.hi + hi.lo + lo.hi of each operand's bf16 hi +
// lo split), accumulated in FP32 in tensor memory.  The probe selection
// re-scores exactly every centroid within the error bound of the nprobe-th
// (probe_tc_gerr), so the probe sets are those of exact distances.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "probe_tc.h"
#include "tcgen05.cuh"

namespace pano {
namespace {

constexpr int PM = 128;   // queries per tile (MMA M)
constexpr int PN = 256;   // centroids per tile (MMA N)
constexpr int PK = 64;    // K elements per panel (one 128-byte swizzled row)
constexpr int PT = 256;   // threads
constexpr int A_BYTES = PM * PK * 2, B_BYTES = PN * PK * 2;
constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;  // A hi, A lo, B hi, B lo

__device__ __forceinline__ void split2(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Rows [r0, r0 + nr) of a row-major FP32 matrix (row length d), K panel p,
// as bf16 hi and lo tiles of R rows in the swizzled K-major image (rows
// past nr and elements past d are zeros).
// vec: 16-byte loads (d % 4 == 0 and src 16-byte aligned).
__device__ __forceinline__ void stage_rows(const float* __restrict__ src, int64_t r0, int nr,
                                           int d, int p, int R, bool vec, unsigned char* hi,
                                           unsigned char* lo) {
  for (int e = threadIdx.x; e < R * (PK / 8); e += PT) {
    const int r = e / (PK / 8), c8 = e % (PK / 8);
    const int k0 = p * PK + c8 * 8;
    float f[8];
    if (vec && r < nr && k0 + 8 <= d) {
      const float4* s4 = reinterpret_cast<const float4*>(src + (r0 + r) * (int64_t)d + k0);
      const float4 a = __ldg(s4), b = __ldg(s4 + 1);
      f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w;
      f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        f[j] = (r < nr && k0 + j < d) ? __ldg(src + (r0 + r) * (int64_t)d + k0 + j) : 0.f;
    }
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split2(f[j], h[j], l[j]);
    const uint32_t off = tc::swz_offset(r, c8 * 8, R, PK);
    *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
  }
}

__global__ void __launch_bounds__(PT, 1) probe_tc_kernel(const float* __restrict__ Q, int64_t nq,
                                                         const float* __restrict__ C, int nlist,
                                                         int d, const float* __restrict__ qn2,
                                                         const float* __restrict__ cn2,
                                                         float* __restrict__ pd, int* __restrict__ err,
                                                         bool vq, bool vc) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t done[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const int64_t q0 = (int64_t)blockIdx.y * PM;
  const int c0 = blockIdx.x * PN;
  const int nr_q = nq - q0 < PM ? (int)(nq - q0) : PM;
  const int nr_c = nlist - c0 < PN ? nlist - c0 : PN;
  const int N = (nr_c + 15) & ~15;  // MMA N: a multiple of 16
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, PN);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    fence_mbar_init();
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = tc::idesc_bf16(PM, N);
  const int np = (d + PK - 1) / PK;
  uint32_t dpar = 0;
  for (int p = 0; p < np; ++p) {
    const int s = p & 1;
    unsigned char* st = base + (size_t)s * STAGE;
    if (p >= 2) {  // the MMAs that read this stage two panels ago are done
      if (!mbar_wait_bounded(&done[s], (dpar >> s) & 1u)) atomicOr(&s_fail, 1);
      dpar ^= 1u << s;
    }
    stage_rows(Q, q0, nr_q, d, p, PM, vq, st, st + A_BYTES);
    stage_rows(C, c0, nr_c, d, p, N, vc, st + 2 * A_BYTES, st + 2 * A_BYTES + B_BYTES);
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint64_t ah = tc::smem_desc(smem_u32(st), 128);
      const uint64_t al = tc::smem_desc(smem_u32(st + A_BYTES), 128);
      const uint64_t bh = tc::smem_desc(smem_u32(st + 2 * A_BYTES), 128);
      const uint64_t bl = tc::smem_desc(smem_u32(st + 2 * A_BYTES + B_BYTES), 128);
      for (int k = 0; k < PK / 16; ++k) {
        const uint64_t o = tc::kstep_off(k, 0);  // within the panel's one 128-byte row
        tc::mma_bf16(tbase, ah + o, bh + o, idesc, (p > 0 || k > 0) ? 1u : 0u);
        tc::mma_bf16(tbase, ah + o, bl + o, idesc, 1u);
        tc::mma_bf16(tbase, al + o, bh + o, idesc, 1u);
      }
      tc::mma_commit(&done[s]);
    }
  }
  // the last panel's commit covers every MMA of the tile
  {
    const int s = (np - 1) & 1;
    if (!mbar_wait_bounded(&done[s], (dpar >> s) & 1u)) atomicOr(&s_fail, 1);
  }
  tc::fence_after_sync();
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 queries) and
  // columns 128 (w / 4) .. + 127
  const int row = (warp & 3) * 32 + lane;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int col0 = (warp >> 2) * 128;
  const bool ok = __all_sync(0xffffffffu, s_fail == 0);
  if (ok && col0 < N) {
    const int64_t q = q0 + row;
    const float qn = row < nr_q ? qn2[q] : 0.f;
    for (int cb = col0; cb < col0 + 128 && cb < N; cb += 16) {
      float v[16];
      tc::tmem_ld16(tbase + lane_base + (uint32_t)cb, v);
      if (row < nr_q) {
        float* out = pd + q * (int64_t)nlist + c0 + cb;
        if (cb + 16 <= nr_c && ((c0 + cb) & 3) == 0 && (nlist & 3) == 0) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            float4 o;
            o.x = fmaf(-2.f, v[j], qn + __ldg(cn2 + c0 + cb + j));
            o.y = fmaf(-2.f, v[j + 1], qn + __ldg(cn2 + c0 + cb + j + 1));
            o.z = fmaf(-2.f, v[j + 2], qn + __ldg(cn2 + c0 + cb + j + 2));
            o.w = fmaf(-2.f, v[j + 3], qn + __ldg(cn2 + c0 + cb + j + 3));
            *reinterpret_cast<float4*>(out + j) = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < nr_c) out[j] = fmaf(-2.f, v[j], qn + __ldg(cn2 + c0 + cb + j));
        }
      }
    }
  }
  if (tid == 0 && s_fail) atomicOr(err, kErrTimeout);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, PN);
}

}  // namespace

bool probe_tc_supported(int d) { return d >= 8 && d % 8 == 0; }

double probe_tc_gerr(int d) {
  // |pd - exact| <= gerr (|q| + |c|)^2: the dot product loses at most
  // 3 2^-16 sum |q_j c_j| to the split (two splits of 2^-16 each, and the
  // dropped lo.lo product) and 2^-20 of the running sum of |products| per
  // MMA (3 d / 16 MMAs; the accumulation model the verify path uses), with
  // sum |q_j c_j| <= |q| |c| <= (|q| + |c|)^2 / 4; it enters pd twice; the
  // epilogue's two roundings add 2 u of |q|^2 + |c|^2 + 2 |q.c|.  Factor 2
  // of safety on those.
  // The query and centroid norms may come from plain FP32 sums: gamma_{d+4}
  // of |q|^2 + |c|^2 <= (|q| + |c|)^2 covers them.
  const double dot = 3.0 * std::ldexp(1.0, -16) + (3.0 * std::ceil(d / 16.0)) * std::ldexp(1.0, -20);
  return 2.0 * (2.0 * dot / 4.0 + 2.0 * std::ldexp(1.0, -24)) + gamma_n(d + 4);
}

int launch_probe_tc(const float* Q, int64_t nq, const float* C, int nlist, int d,
                    const float* qn2, const float* cn2, float* pd, int* err, cudaStream_t st) {
  static PerDeviceOnce once;
  const size_t smem = (size_t)2 * STAGE + 1024;
  PANO_CUDA(once.run([smem] {
    return cudaFuncSetAttribute((const void*)probe_tc_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }));
  if (nq <= 0 || nlist <= 0) return PANO_OK;
  const dim3 grid((unsigned)((nlist + PN - 1) / PN), (unsigned)((nq + PM - 1) / PM));
  const bool vq = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0;
  const bool vc = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
  probe_tc_kernel<<<grid, PT, smem, st>>>(Q, nq, C, nlist, d, qn2, cn2, pd, err, vq, vc);
  PANO_CUDA(cudaGetLastError());
  return PANO_OK;
}

}  // namespace pano
