// FP32 SIMT "NT" GEMM used by the query/database transform (q~ = T~(q-mu~)),
// the coarse IVF probe and k-means:  C[m][n] = sum_k (A[m][k] - mu[k]) B[n][k].
//
// kStore / kDist: 128x64 CTA tile (8x4 register tile per thread, so two
// CTAs fit an SM's registers), float4 global loads when rows are 16-byte
// aligned.  kArgmin2: 128x128 tile (8x8 per thread).  Both use a 16-deep K
// tile double-buffered through shared memory, and every K tile is
// accumulated in a fresh register before being added to the running total,
// which bounds the roundings a product sees by GEMM_KT + ceil(K/GEMM_KT) + 1
// (used by the rigorous error terms of the bounds).
//
// Epilogues: kStore (C = acc), kDist (C = an[m] + bn[n] - 2 acc, the squared
// distance expansion) and kArgmin2 (no C: each row's two smallest expansion
// distances over all n, written as (dist, n) keys; one CTA walks all of N for
// its 128 rows so no cross-CTA reduction is needed).
#include "device_common.cuh"
#include "gemm.h"

namespace pano {

namespace {

constexpr int BM = 128, BN = 128, BK = GEMM_KT_DEV, NT = 256, PAD = 4;

struct Tile {
  float a[2][BK][BM + PAD];
  float b[2][BK][BN + PAD];
};

__device__ __forceinline__ void load_tile(const float* __restrict__ A, int lda,
                                          const float* __restrict__ mu,
                                          const float* __restrict__ B, int ldb,
                                          int M, int N, int K, int m0, int n0,
                                          int k0, float (&ra)[8], float (&rb)[8]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int e = tid + NT * i;
    int r = e >> 4, kk = e & 15;
    int gk = k0 + kk;
    int gm = m0 + r, gn = n0 + r;
    float va = 0.f, vb = 0.f;
    if (gk < K) {
      if (gm < M) va = A[(int64_t)gm * lda + gk] - (mu ? mu[gk] : 0.f);
      if (gn < N) vb = B[(int64_t)gn * ldb + gk];
    }
    ra[i] = va;
    rb[i] = vb;
  }
}

__device__ __forceinline__ void store_tile(Tile& s, int buf, const float (&ra)[8],
                                           const float (&rb)[8]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int e = tid + NT * i;
    int r = e >> 4, kk = e & 15;
    s.a[buf][kk][r] = ra[i];
    s.b[buf][kk][r] = rb[i];
  }
}

// acc += A_tile x B_tile^T over the whole K range for the CTA tile (m0, n0);
// result in tot[8][8] (rows ty*4+{0..3}, 64+ty*4+{0..3}; same for columns).
__device__ __forceinline__ void mainloop(Tile& s, const float* __restrict__ A, int lda,
                                         const float* __restrict__ mu,
                                         const float* __restrict__ B, int ldb, int M,
                                         int N, int K, int m0, int n0,
                                         float (&tot)[8][8]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float ra[8], rb[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) tot[i][j] = 0.f;
  const int nk = (K + BK - 1) / BK;
  load_tile(A, lda, mu, B, ldb, M, N, K, m0, n0, 0, ra, rb);
  store_tile(s, 0, ra, rb);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load_tile(A, lda, mu, B, ldb, M, N, K, m0, n0, (t + 1) * BK, ra, rb);
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&s.a[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&s.a[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&s.b[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&s.b[buf][kk][64 + tx * 4]);
      float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) tot[i][j] += acc[i][j];
    if (t + 1 < nk) store_tile(s, buf ^ 1, ra, rb);
    __syncthreads();
  }
}

__device__ __forceinline__ int row_of(int i) {
  return (i < 4) ? ((threadIdx.x >> 4) * 4 + i) : (64 + (threadIdx.x >> 4) * 4 + i - 4);
}
__device__ __forceinline__ int col_of(int j) {
  return (j < 4) ? ((threadIdx.x & 15) * 4 + j) : (64 + (threadIdx.x & 15) * 4 + j - 4);
}

// ---- 128 x 64 tile (kStore, kDist)
constexpr int BN2 = 64;

struct Tile2 {
  float a[2][BK][BM + PAD];
  float b[2][BK][BN2 + PAD];
};

// thread's share of one K tile: rows r_a(i) of A (2 x float4 or 8 scalars)
// and rows of B (1 x float4 or 4 scalars)
template <bool VEC>
__device__ __forceinline__ void load_tile2(const float* __restrict__ A, int lda,
                                           const float* __restrict__ mu,
                                           const float* __restrict__ B, int ldb, int M, int N,
                                           int K, int m0, int n0, int k0, float (&ra)[8],
                                           float (&rb)[4]) {
  const int tid = threadIdx.x;
  if (VEC) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = tid + NT * i, r = e >> 2, k4 = (e & 3) * 4, gm = m0 + r, gk = k0 + k4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < M && gk < K) {
        v = *reinterpret_cast<const float4*>(A + (int64_t)gm * lda + gk);
        if (mu) {
          const float4 u = *reinterpret_cast<const float4*>(mu + gk);
          v.x -= u.x;
          v.y -= u.y;
          v.z -= u.z;
          v.w -= u.w;
        }
      }
      ra[4 * i] = v.x;
      ra[4 * i + 1] = v.y;
      ra[4 * i + 2] = v.z;
      ra[4 * i + 3] = v.w;
    }
    const int r = tid >> 2, k4 = (tid & 3) * 4, gn = n0 + r, gk = k0 + k4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gn < N && gk < K) v = *reinterpret_cast<const float4*>(B + (int64_t)gn * ldb + gk);
    rb[0] = v.x;
    rb[1] = v.y;
    rb[2] = v.z;
    rb[3] = v.w;
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = tid + NT * i, r = e >> 4, kk = e & 15, gm = m0 + r, gk = k0 + kk;
      ra[i] = (gm < M && gk < K) ? A[(int64_t)gm * lda + gk] - (mu ? mu[gk] : 0.f) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + NT * i, r = e >> 4, kk = e & 15, gn = n0 + r, gk = k0 + kk;
      rb[i] = (gn < N && gk < K) ? B[(int64_t)gn * ldb + gk] : 0.f;
    }
  }
}

template <bool VEC>
__device__ __forceinline__ void store_tile2(Tile2& s, int buf, const float (&ra)[8],
                                            const float (&rb)[4]) {
  const int tid = threadIdx.x;
  if (VEC) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = tid + NT * i, r = e >> 2, k4 = (e & 3) * 4;
#pragma unroll
      for (int j = 0; j < 4; ++j) s.a[buf][k4 + j][r] = ra[4 * i + j];
    }
    const int r = tid >> 2, k4 = (tid & 3) * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) s.b[buf][k4 + j][r] = rb[j];
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = tid + NT * i;
      s.a[buf][e & 15][e >> 4] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + NT * i;
      s.b[buf][e & 15][e >> 4] = rb[i];
    }
  }
}

// rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns tx*4 + {0..3}
template <int MODE, bool VEC>
__global__ void __launch_bounds__(NT, 2) gemm_nt64_kernel(int M, int N, int K,
                                                          const float* __restrict__ A, int lda,
                                                          const float* __restrict__ mu,
                                                          const float* __restrict__ B, int ldb,
                                                          float* __restrict__ C, int64_t ldc,
                                                          const float* __restrict__ an,
                                                          const float* __restrict__ bn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tile2& s = *reinterpret_cast<Tile2*>(smem_raw);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN2;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float tot[8][4], ra[8], rb[4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) tot[i][j] = 0.f;
  const int nk = (K + BK - 1) / BK;
  load_tile2<VEC>(A, lda, mu, B, ldb, M, N, K, m0, n0, 0, ra, rb);
  store_tile2<VEC>(s, 0, ra, rb);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load_tile2<VEC>(A, lda, mu, B, ldb, M, N, K, m0, n0, (t + 1) * BK, ra, rb);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&s.a[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&s.a[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&s.b[buf][kk][tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) tot[i][j] += acc[i][j];
    if (t + 1 < nk) store_tile2<VEC>(s, buf ^ 1, ra, rb);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gm >= M) continue;
    const float am = (MODE == kDist) ? an[gm] : 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = tot[i][j];
      if (MODE == kDist) v = am + bn[gn] - 2.0f * v;
      C[(int64_t)gm * ldc + gn] = v;
    }
  }
}

__device__ __forceinline__ void top2_push(unsigned long long& k0, unsigned long long& k1,
                                          unsigned long long key) {
  if (key < k0) {
    k1 = k0;
    k0 = key;
  } else if (key < k1) {
    k1 = key;
  }
}

// Each CTA owns 128 rows and loops over all column tiles.
__global__ void __launch_bounds__(NT) gemm_argmin2_kernel(
    int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ mu,
    const float* __restrict__ B, int ldb, const float* __restrict__ an,
    const float* __restrict__ bn, unsigned long long* __restrict__ out2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tile& s = *reinterpret_cast<Tile*>(smem_raw);
  const int m0 = blockIdx.x * BM;
  unsigned long long best0[8], best1[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) best0[i] = best1[i] = kEmptyKey;
  for (int n0 = 0; n0 < N; n0 += BN) {
    float tot[8][8];
    mainloop(s, A, lda, mu, B, ldb, M, N, K, m0, n0, tot);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int gm = m0 + row_of(i);
      float am = gm < M ? an[gm] : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int gn = n0 + col_of(j);
        if (gn >= N) continue;
        float v = am + bn[gn] - 2.0f * tot[i][j];
        unsigned long long key =
            (static_cast<unsigned long long>(float_ordered(v)) << 32) | (uint32_t)gn;
        top2_push(best0[i], best1[i], key);
      }
    }
  }
  // the 16 threads sharing a row group are lanes of one half-warp
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
      unsigned long long o0 = __shfl_xor_sync(0xffffffffu, best0[i], off);
      unsigned long long o1 = __shfl_xor_sync(0xffffffffu, best1[i], off);
      top2_push(best0[i], best1[i], o0);
      top2_push(best0[i], best1[i], o1);
    }
    int gm = m0 + row_of(i);
    if ((threadIdx.x & 15) == 0 && gm < M) {
      out2[2 * (int64_t)gm] = best0[i];
      out2[2 * (int64_t)gm + 1] = best1[i];
    }
  }
}

}  // namespace

// 33.8 KB: below the 48 KB default, no opt-in attribute needed.
static size_t tile_smem() { return sizeof(Tile); }

cudaError_t gemm_nt(int mode, int M, int N, int K, const float* A, int lda, const float* mu,
                    const float* B, int ldb, float* C, int64_t ldc, const float* an,
                    const float* bn, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + BM - 1) / BM, (N + BN2 - 1) / BN2);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  // float4 loads need 16-byte aligned rows (and mu)
  const bool vec = ((K | lda | ldb) & 3) == 0 && ((uintptr_t)A & 15) == 0 &&
                   ((uintptr_t)B & 15) == 0 && ((uintptr_t)mu & 15) == 0;
  const size_t sm = sizeof(Tile2);  // 25.3 KB
  if (mode == kStore) {
    if (vec)
      gemm_nt64_kernel<kStore, true><<<grid, NT, sm, st>>>(M, N, K, A, lda, mu, B, ldb, C, ldc, an, bn);
    else
      gemm_nt64_kernel<kStore, false><<<grid, NT, sm, st>>>(M, N, K, A, lda, mu, B, ldb, C, ldc, an, bn);
  } else {
    if (vec)
      gemm_nt64_kernel<kDist, true><<<grid, NT, sm, st>>>(M, N, K, A, lda, mu, B, ldb, C, ldc, an, bn);
    else
      gemm_nt64_kernel<kDist, false><<<grid, NT, sm, st>>>(M, N, K, A, lda, mu, B, ldb, C, ldc, an, bn);
  }
  return cudaGetLastError();
}

cudaError_t gemm_argmin2(int M, int N, int K, const float* A, int lda, const float* mu,
                         const float* B, int ldb, const float* an, const float* bn,
                         unsigned long long* out2, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  dim3 grid((M + BM - 1) / BM);
  gemm_argmin2_kernel<<<grid, NT, tile_smem(), st>>>(M, N, K, A, lda, mu, B, ldb, an, bn,
                                                     out2);
  return cudaGetLastError();
}

}  // namespace pano
