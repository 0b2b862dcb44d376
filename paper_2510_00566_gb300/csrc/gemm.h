// Launchers of the FP32 SIMT GEMM (see gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define GEMM_KT_DEV 16

namespace pano {

enum { kStore = 0, kDist = 1 };

// C[m][n] = sum_k (A[m][k] - mu[k]) * B[n][k]      (mode kStore; mu may be 0)
// C[m][n] = an[m] + bn[n] - 2 * sum_k A[m][k] B[n][k]   (mode kDist)
cudaError_t gemm_nt(int mode, int M, int N, int K, const float* A, int lda, const float* mu,
                    const float* B, int ldb, float* C, int64_t ldc, const float* an,
                    const float* bn, cudaStream_t st);

// For each row m: the two smallest keys (ordered(an[m] + bn[n] - 2 a_m.b_n) << 32 | n)
// over n < N, written to out2[2m], out2[2m+1].
cudaError_t gemm_argmin2(int M, int N, int K, const float* A, int lda, const float* mu,
                         const float* B, int ldb, const float* an, const float* bn,
                         unsigned long long* out2, cudaStream_t st);

}  // namespace pano
