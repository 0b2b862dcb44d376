/*
 * panorama_debug.h -- self-test entry points of libpanorama (not part of the
 * search API).  They exist so that tests can check building blocks of the
 * GB300 kernels in isolation.
 */
#ifndef PANORAMA_DEBUG_H
#define PANORAMA_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* panorama_debug_tc_gemm -- one CTA computes D = 2 * A * B^T with the
 * tensor-core path of the BF16 verify kernel (swizzled K-major shared-memory
 * tiles, tcgen05.mma into tensor memory, accumulation over two passes,
 * tcgen05.ld read-back).  The paper has no counterpart: it is a unit check of
 * the kernel's building blocks.
 *   A: device, 128 x K bf16 row-major;  B: device, N x K bf16 row-major;
 *   D: device, 128 x N FP32 row-major (written).
 *   N: multiple of 16 in [16, 256];  K: 16, 32 or a multiple of 64 <= 256.
 * Errors: PANO_EINVAL (sizes, null pointers), PANO_ENODEV, PANO_ECUDA,
 *         PANO_ETIMEOUT (the completion wait gave up). */
int panorama_debug_tc_gemm(const void* A, const void* B, int32_t N, int32_t K,
                           float* D, void* stream);

/* panorama_debug_tc_gemm_fp8 -- the same with E4M3 tiles and the FP8 verify
 * kernel's MMA (tcgen05.mma kind::f8f6f4, 32 K elements per instruction; the
 * tile of K E4M3 bytes per row has the byte layout of a K/2-wide bf16 tile).
 *   A: device, 128 x K E4M3 bytes row-major;  B: device, N x K E4M3 bytes;
 *   D: device, 128 x N FP32 row-major (written).
 *   N: multiple of 16 in [16, 256];  K: 32, 64 or a multiple of 128 <= 512.
 * Errors: as panorama_debug_tc_gemm. */
int panorama_debug_tc_gemm_fp8(const void* A, const void* B, int32_t N, int32_t K,
                               float* D, void* stream);

/* panorama_debug_sqrt_up -- out[i] = the verify kernels' rounded-up square
 * root of x[i] (x[i] >= 0): the approximate square root times 1 + 2^-18,
 * rounded up, which the upper bounds of the last level use.  The paper has
 * no counterpart: it lets a test check that the result bounds the exact
 * root from above.
 *   x, out: device, n floats.
 * Errors: PANO_EINVAL (n < 0, null pointers with n > 0), PANO_ECUDA. */
int panorama_debug_sqrt_up(const float* x, int64_t n, float* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PANORAMA_DEBUG_H */
