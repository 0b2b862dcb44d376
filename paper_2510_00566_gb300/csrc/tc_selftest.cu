// Isolated check of the tensor-core plumbing used by the BF16 and FP8 verify
// kernels: one CTA stages A (128 x K) and B (N x K) tiles into the swizzled
// K-major shared-memory layout, runs the tcgen05 MMAs over K (twice: the
// second pass accumulates, as the level loop does), reads D back from TMEM
// with 32x32b loads and writes it to global memory.  BF16 tiles use
// kind::f16 (16 K elements per MMA), E4M3 tiles kind::f8f6f4 (32 per MMA).
#include <cuda_bf16.h>

#include "internal.h"
#include "search.h"
#include "tcgen05.cuh"

namespace pano {
namespace {

template <bool FP8>
__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(const uint8_t* __restrict__ A,
                                                             const uint8_t* __restrict__ B,
                                                             int N, int K, float* __restrict__ D,
                                                             int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  // the byte layout of a K-wide E4M3 tile is that of a K/2-wide bf16 tile
  const int KL = FP8 ? K / 2 : K, rowb = FP8 ? K : 2 * K;
  // swizzled tiles need 1024-byte alignment: round the dynamic base up
  unsigned char* sa = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);
  unsigned char* sb = sa + tc::tile_bytes(128, KL);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  // stage A and B: one 16-byte chunk (8 bf16 / 16 E4M3 elements) at a time
  for (int e = tid; e < 128 * (KL / 8); e += blockDim.x) {
    int r = e / (KL / 8), c8 = e % (KL / 8);
    uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)r * rowb + c8 * 16);
    *reinterpret_cast<uint4*>(sa + tc::swz_offset(r, c8 * 8, 128, KL)) = v;
  }
  for (int e = tid; e < N * (KL / 8); e += blockDim.x) {
    int r = e / (KL / 8), c8 = e % (KL / 8);
    uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * rowb + c8 * 16);
    *reinterpret_cast<uint4*>(sb + tc::swz_offset(r, c8 * 8, N, KL)) = v;
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
  const uint32_t idesc = FP8 ? tc::idesc_e4m3(128, N) : tc::idesc_bf16(128, N);
  if (tid == 0) {
    const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
    for (int pass = 0; pass < 2; ++pass)
      for (int s = 0; s < KL / 16; ++s) {
        const uint64_t ad = tc::kstep_desc(a0, s, 128, KL), bd = tc::kstep_desc(b0, s, N, KL);
        if (FP8)
          tc::mma_e4m3(tbase, ad, bd, idesc, (pass | s) ? 1u : 0u);
        else
          tc::mma_bf16(tbase, ad, bd, idesc, (pass | s) ? 1u : 0u);
      }
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

int run_tc_selftest(bool fp8, const void* A, const void* B, int32_t N, int32_t K, float* D,
                    void* stream) {
  clear_error();
  PANO_CHECK(A && B && D, PANO_EINVAL, "null argument");
  PANO_CHECK(N >= 16 && N <= 256 && N % 16 == 0, PANO_EINVAL,
             "N must be a multiple of 16 in [16, 256]");
  // K in the layout's bf16-equivalent width (E4M3: K / 2)
  const int KL = fp8 ? K / 2 : K;
  const bool k_ok = KL == 16 || KL == 32 || (KL >= 64 && KL <= 256 && KL % 64 == 0);
  PANO_CHECK((!fp8 || K % 2 == 0) && k_ok, PANO_EINVAL,
             fp8 ? "K must be 32, 64 or a multiple of 128 up to 512"
                 : "K must be 16, 32 or a multiple of 64 up to 256");
  int rc = check_device(nullptr);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  PANO_CUDA(cudaMallocAsync(&err, 4, st));
  PANO_CUDA(cudaMemsetAsync(err, 0, 4, st));
  size_t smem = tc::tile_bytes(128, KL) + tc::tile_bytes(N, KL) + 1024;
  const void* kern =
      fp8 ? (const void*)tc_selftest_kernel<true> : (const void*)tc_selftest_kernel<false>;
  PANO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (fp8)
    tc_selftest_kernel<true><<<1, 128, smem, st>>>((const uint8_t*)A, (const uint8_t*)B, N, K, D,
                                                   err);
  else
    tc_selftest_kernel<false><<<1, 128, smem, st>>>((const uint8_t*)A, (const uint8_t*)B, N, K, D,
                                                    err);
  PANO_CUDA(cudaGetLastError());
  int herr = 0;
  PANO_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  PANO_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(err, st);
  if (herr) return fail(PANO_ETIMEOUT, "tensor-core self-test wait timed out");
  return PANO_OK;
}

}  // namespace
}  // namespace pano

extern "C" int panorama_debug_tc_gemm(const void* A, const void* B, int32_t N, int32_t K,
                                      float* D, void* stream) {
  return pano::run_tc_selftest(false, A, B, N, K, D, stream);
}

extern "C" int panorama_debug_tc_gemm_fp8(const void* A, const void* B, int32_t N, int32_t K,
                                          float* D, void* stream) {
  return pano::run_tc_selftest(true, A, B, N, K, D, stream);
}

namespace pano {
namespace {
__global__ void sqrt_up_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sqrt_up(x[i]);
}
}  // namespace
}  // namespace pano

extern "C" int panorama_debug_sqrt_up(const float* x, int64_t n, float* out, void* stream) {
  using namespace pano;
  clear_error();
  PANO_CHECK(n >= 0 && (n == 0 || (x && out)), PANO_EINVAL, "bad arguments");
  if (n == 0) return PANO_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  sqrt_up_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, out);
  PANO_CUDA(cudaGetLastError());
  PANO_CUDA(cudaStreamSynchronize(st));
  return PANO_OK;
}
