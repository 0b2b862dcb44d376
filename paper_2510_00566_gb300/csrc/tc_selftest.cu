// Isolated check of the tensor-core plumbing used by the BF16 verify kernel:
// one CTA stages A (128 x K) and B (N x K) bf16 tiles into the swizzled
// K-major shared-memory layout, runs the K/16 tcgen05 MMAs (twice: the
// second pass accumulates, as the level loop does), reads D back from TMEM
// with 32x32b loads and writes it to global memory.
#include <cuda_bf16.h>

#include "internal.h"
#include "search.h"
#include "tcgen05.cuh"

namespace pano {
namespace {

__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(const __nv_bfloat16* __restrict__ A,
                                                             const __nv_bfloat16* __restrict__ B,
                                                             int N, int K, float* __restrict__ D,
                                                             int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  // swizzled tiles need 1024-byte alignment: round the dynamic base up
  unsigned char* sa = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);
  unsigned char* sb = sa + tc::tile_bytes(128, K);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  // stage A and B: 8 consecutive k per 16-byte chunk
  for (int e = tid; e < 128 * (K / 8); e += blockDim.x) {
    int r = e / (K / 8), c8 = e % (K / 8);
    uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)r * K + c8 * 8);
    *reinterpret_cast<uint4*>(sa + tc::swz_offset(r, c8 * 8, 128, K)) = v;
  }
  for (int e = tid; e < N * (K / 8); e += blockDim.x) {
    int r = e / (K / 8), c8 = e % (K / 8);
    uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + c8 * 8);
    *reinterpret_cast<uint4*>(sb + tc::swz_offset(r, c8 * 8, N, K)) = v;
  }
  fence_proxy_async_smem();
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = tc::idesc_bf16(128, N);
  if (tid == 0) {
    const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
    for (int pass = 0; pass < 2; ++pass)
      for (int s = 0; s < K / 16; ++s)
        tc::mma_bf16(tbase, tc::kstep_desc(a0, s, 128, K), tc::kstep_desc(b0, s, N, K), idesc,
                     (pass | s) ? 1u : 0u);
    tc::mma_commit(&bar);
  }
  bool ok = mbar_wait_bounded(&bar, 0);
  if (!ok && lane == 0) atomicOr(err, kErrTimeout);
  tc::fence_after_sync();
  if (ok) {
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) D[(size_t)tid * N + c0 + j] = v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

}  // namespace
}  // namespace pano

extern "C" int panorama_debug_tc_gemm(const void* A, const void* B, int32_t N, int32_t K,
                                      float* D, void* stream) {
  using namespace pano;
  clear_error();
  PANO_CHECK(A && B && D, PANO_EINVAL, "null argument");
  PANO_CHECK(N >= 16 && N <= 256 && N % 16 == 0, PANO_EINVAL, "N must be a multiple of 16 in [16, 256]");
  PANO_CHECK(K == 16 || K == 32 || (K >= 64 && K <= 256 && K % 64 == 0), PANO_EINVAL,
             "K must be 16, 32 or a multiple of 64 up to 256");
  int rc = check_device(nullptr);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  PANO_CUDA(cudaMallocAsync(&err, 4, st));
  PANO_CUDA(cudaMemsetAsync(err, 0, 4, st));
  size_t smem = tc::tile_bytes(128, K) + tc::tile_bytes(N, K) + 1024;
  PANO_CUDA(cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  tc_selftest_kernel<<<1, 128, smem, st>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, N, K,
                                           D, err);
  PANO_CUDA(cudaGetLastError());
  int herr = 0;
  PANO_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  PANO_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(err, st);
  if (herr) return fail(PANO_ETIMEOUT, "tensor-core self-test wait timed out");
  return PANO_OK;
}
