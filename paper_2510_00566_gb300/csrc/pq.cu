// IVFPQ Panorama: spectrum shaping (Section 4.3), the IVFPQ build and the
// level-wise bounded asymmetric-distance search (Section 6.3).
//
// Search: one thread block per (query, probed list) pair.  The block forms
// the query residual r = q~ - c~ in shared memory and its level tail
// energies (FP64), then walks the list in slabs of PQ_S candidates.  A
// level's subvector terms e_m = ||r_m - C_m[code_m]||^2 come from a table of
// the 256 terms of each of the level's subquantisers in shared memory (the
// paper's per-level look-up tables) while many candidates are live, and
// straight from the codebook once few are (the same arithmetic, so the same
// values).  The codes of one level of a block of 256 vectors are M / L rows
// of 256 bytes (subquantiser-major): at level 0 every thread takes four
// consecutive candidates, whose codes of one subquantiser are one 32-bit
// word.  Survivors are compacted with warp ballots into the next level's
// list; levels stay in step across the block while more than PQ_DEEP
// candidates live, after which each thread walks its survivors through the
// remaining levels alone.  The query's top-k is a sorted array of
// (distance, id) keys shared by all of its pairs; its k-th key is the
// pruning threshold (Algorithm 1's running k-th distance), seeded before the
// scan with the first members of the query's nearest list.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/panorama_pq.h"
#include "device_common.cuh"
#include "gemm.h"
#include "internal.h"
#include "search.h"

namespace pano {
namespace {

constexpr int PQ_KSUB = 256;     // codewords per subquantiser (8-bit codes)
constexpr int PQ_B = 256;        // vector slots per layout block
constexpr int PQ_S = 2048;       // candidates per slab of one (query, list) pair
constexpr int PQ_NT = 256;       // threads of the verify kernel
constexpr int PQ_MAXML = 64;     // subquantisers per level
constexpr int PQ_MAXDSUB = 32;   // coordinates per subvector
constexpr int PQ_LUT_MIN = 128;  // live candidates from which a level's table is built
constexpr int PQ_SEED = 64;      // nearest-list members that seed each query's top-k
constexpr int PQ_DEEP = 128;     // live candidates from which a slab finishes depth-first
constexpr int PQ_MAXL = 64;

// ------------------------------------------------------------------ host
// Q of G = QR with diag(R) > 0 (Householder reflections in FP64), G the
// n x n block at g with row stride ld: a Haar-distributed rotation when G
// is standard normal (Mezzadri 2007).  Q row-major n x n.
void haar_q(const double* g, int64_t ld, int n, std::vector<double>& Q) {
  std::vector<double> A((size_t)n * n), V((size_t)n * n, 0.0), beta(n, 0.0), rdiag(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = g[(size_t)i * ld + j];
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = k; i < n; ++i) nrm += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    nrm = std::sqrt(nrm);
    const double x0 = A[(size_t)k * n + k];
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    double vn = 0.0;
    for (int i = k; i < n; ++i) {
      double v = A[(size_t)i * n + k] - (i == k ? alpha : 0.0);
      V[(size_t)i * n + k] = v;
      vn += v * v;
    }
    beta[k] = vn > 0.0 ? 2.0 / vn : 0.0;
    for (int j = k; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < n; ++i) s += V[(size_t)i * n + k] * A[(size_t)i * n + j];
      s *= beta[k];
      for (int i = k; i < n; ++i) A[(size_t)i * n + j] -= s * V[(size_t)i * n + k];
    }
    rdiag[k] = A[(size_t)k * n + k];
  }
  // Q = H_0 H_1 ... H_{n-1}
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int k = n - 1; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < n; ++i) s += V[(size_t)i * n + k] * Q[(size_t)i * n + j];
      s *= beta[k];
      for (int i = k; i < n; ++i) Q[(size_t)i * n + j] -= s * V[(size_t)i * n + k];
    }
  }
  for (int j = 0; j < n; ++j)
    if (rdiag[j] < 0.0)
      for (int i = 0; i < n; ++i) Q[(size_t)i * n + j] = -Q[(size_t)i * n + j];
}

// rows a..a+n of M (d columns) <- Q * rows a..a+n of M
void rotate_rows(std::vector<double>& Mx, int d, int a, int n, const std::vector<double>& Q) {
  std::vector<double> out((size_t)n * d, 0.0);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      double* o = out.data() + i * d;
      for (int t = 0; t < n; ++t) {
        const double q = Q[(size_t)i * n + t];
        const double* src = Mx.data() + (size_t)(a + t) * d;
        for (int j = 0; j < d; ++j) o[j] += q * src[j];
      }
    }
  });
  std::memcpy(Mx.data() + (size_t)a * d, out.data(), out.size() * 8);
}

void finish_transform(pano_transform& t) {
  const int d = t.d;
  t.T32.resize((size_t)d * d);
  t.mu32.resize(d);
  for (size_t i = 0; i < t.T.size(); ++i) t.T32[i] = (float)t.T[i];
  for (int i = 0; i < d; ++i) t.mu32[i] = (float)t.mu[i];
  t.eta = orthogonality_defect(t.T32.data(), d) * (1.0 + 1e-6) + 1e-15;
}

uint64_t mix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// k distinct indices of [0, n), ascending (partial Fisher-Yates).
std::vector<int64_t> sample_rows(int64_t n, int64_t k, uint64_t seed) {
  k = std::min(k, n);
  std::vector<int64_t> out;
  if (k == n) {
    out.resize(n);
    std::iota(out.begin(), out.end(), 0);
    return out;
  }
  std::vector<int64_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  uint64_t s = seed;
  for (int64_t i = 0; i < k; ++i) {
    int64_t j = i + (int64_t)(mix64(s) % (uint64_t)(n - i));
    std::swap(perm[i], perm[j]);
  }
  out.assign(perm.begin(), perm.begin() + k);
  std::sort(out.begin(), out.end());
  return out;
}

struct DTmp {
  void* p = nullptr;
  ~DTmp() {
    if (p) cudaFree(p);
  }
};

// ---------------------------------------------------------------- device
// The subvector term sum_t fl(fl(r_t - c_t)^2), left to right (no fused
// multiply-add: every kernel, and the encoder, gets the same bits).
__device__ __forceinline__ float pq_term(const float* __restrict__ r,
                                         const float* __restrict__ c, int dsub) {
  float t = __fsub_rn(r[0], c[0]);
  float s = __fmul_rn(t, t);
  for (int j = 1; j < dsub; ++j) {
    t = __fsub_rn(r[j], c[j]);
    s = __fadd_rn(s, __fmul_rn(t, t));
  }
  return s;
}

__global__ void pq_gather_kernel(const float* __restrict__ X, int d,
                                 const int64_t* __restrict__ rows, int64_t n,
                                 float* __restrict__ out) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t r = rows[i];
  for (int j = threadIdx.x; j < d; j += blockDim.x)
    out[i * d + j] = r >= 0 ? X[r * d + j] : 0.f;
}

// R[i] = xt[i] - ct[list[i]] (rows with list -1: zero)
__global__ void pq_residual_kernel(float* __restrict__ xt, int64_t n, int d,
                                   const float* __restrict__ ct,
                                   const int32_t* __restrict__ list) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int c = list[i];
  for (int j = threadIdx.x; j < d; j += blockDim.x)
    xt[i * d + j] = c >= 0 ? __fsub_rn(xt[i * d + j], ct[(size_t)c * d + j]) : 0.f;
}

// Nearest codeword of each (row, subquantiser), ties to the lower index.
// Grid (ceil(n / 256), M); the subquantiser's codebook in shared memory.
// layout != 0: codes go to [(i / 256) * M + m][256] + i % 256 (the index
// layout, i = slot), else to [i][M].  Rows with skip[i] < 0 are left alone.
__global__ void __launch_bounds__(256) pq_encode_kernel(const float* __restrict__ R, int64_t n,
                                                        int d, int M, int dsub,
                                                        const float* __restrict__ cb,
                                                        const int32_t* __restrict__ skip,
                                                        int layout, uint8_t* __restrict__ codes) {
  extern __shared__ float s_cb[];
  const int m = blockIdx.y;
  for (int t = threadIdx.x; t < PQ_KSUB * dsub; t += blockDim.x)
    s_cb[t] = cb[(size_t)m * PQ_KSUB * dsub + t];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (skip && skip[i] < 0)) return;
  float r[PQ_MAXDSUB];
  for (int t = 0; t < dsub; ++t) r[t] = R[i * d + (int64_t)m * dsub + t];
  float best = INFINITY;
  int bj = 0;
  for (int j = 0; j < PQ_KSUB; ++j) {
    const float e = pq_term(r, s_cb + j * dsub, dsub);
    if (e < best) {
      best = e;
      bj = j;
    }
  }
  if (layout)
    codes[((i / PQ_B) * M + m) * PQ_B + (i % PQ_B)] = (uint8_t)bj;
  else
    codes[i * M + m] = (uint8_t)bj;
}

// One Lloyd step of every subquantiser: assign each sampled subvector to its
// nearest codeword (as the encoder) and accumulate FP64 sums and counts.
__global__ void __launch_bounds__(256) pq_kmeans_accum_kernel(
    const float* __restrict__ R, int64_t n, int d, int dsub, const float* __restrict__ cb,
    double* __restrict__ sums, int* __restrict__ cnt) {
  extern __shared__ float s_cb[];
  const int m = blockIdx.y;
  for (int t = threadIdx.x; t < PQ_KSUB * dsub; t += blockDim.x)
    s_cb[t] = cb[(size_t)m * PQ_KSUB * dsub + t];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r[PQ_MAXDSUB];
  for (int t = 0; t < dsub; ++t) r[t] = R[i * d + (int64_t)m * dsub + t];
  float best = INFINITY;
  int bj = 0;
  for (int j = 0; j < PQ_KSUB; ++j) {
    const float e = pq_term(r, s_cb + j * dsub, dsub);
    if (e < best) {
      best = e;
      bj = j;
    }
  }
  const size_t cell = (size_t)m * PQ_KSUB + bj;
  for (int t = 0; t < dsub; ++t) atomicAdd(sums + cell * dsub + t, (double)r[t]);
  atomicAdd(cnt + cell, 1);
}

__global__ void pq_kmeans_update_kernel(int M, int dsub, const double* __restrict__ sums,
                                        const int* __restrict__ cnt, float* __restrict__ cb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * PQ_KSUB * dsub) return;
  const int c = cnt[i / dsub];
  if (c > 0) cb[i] = (float)(sums[i] / c);  // an empty cell keeps its codeword
}

// ||C_m[j]||^2 in FP64
__global__ void pq_cnorm_kernel(int M, int dsub, const float* __restrict__ cb,
                                double* __restrict__ cn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * PQ_KSUB) return;
  double s = 0.0;
  for (int t = 0; t < dsub; ++t) {
    const double v = cb[i * dsub + t];
    s += v * v;
  }
  cn[i] = s;
}

// Scatter caller codes (vector-id order) into the block layout.
__global__ void pq_scatter_codes_kernel(const uint8_t* __restrict__ src, int M,
                                        const int64_t* __restrict__ perm, int64_t nslots,
                                        uint8_t* __restrict__ codes) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nslots * M) return;
  const int64_t slot = i / M;
  const int m = (int)(i % M);
  const int64_t id = perm[slot];
  codes[((slot / PQ_B) * M + m) * PQ_B + (slot % PQ_B)] = id >= 0 ? src[id * M + m] : 0;
}

// ids and tail norms of every slot: tails[(block L + l) 256 + lane] =
// sqrt(sum over the subquantisers of levels > l of ||C_m[code_m]||^2).
__global__ void pq_tails_kernel(const uint8_t* __restrict__ codes,
                                const int64_t* __restrict__ perm, int64_t nslots, int M,
                                int L, const double* __restrict__ cn, float* __restrict__ tails,
                                int32_t* __restrict__ ids) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  const int64_t blk = slot / PQ_B;
  const int lane = (int)(slot % PQ_B);
  const int64_t id = perm[slot];
  ids[slot] = (int32_t)id;
  const int ML = M / L;
  double acc = 0.0;
  for (int l = L - 1; l >= 0; --l) {
    tails[(blk * L + l) * PQ_B + lane] = id >= 0 ? (float)sqrt(acc) : 0.f;
    if (id < 0) continue;
    for (int mm = 0; mm < ML; ++mm) {
      const int m = l * ML + mm;
      acc += cn[(size_t)m * PQ_KSUB + codes[(blk * M + m) * PQ_B + lane]];
    }
  }
}

// ---- search
struct PqArgs {
  const uint8_t* codes;
  const float* xtail;
  const int32_t* ids;
  const int64_t* blk_off;
  const int32_t* list_size;
  const float* codebook;
  const float* cent_t;
  const float* qt;
  const int2* pairs;  // (query, list), nearest lists first, then by list; x < 0: none
  const int32_t* kq;  // per-query k (<= k_max); a query's top-k row holds k_max slots
  unsigned long long* topk;
  unsigned long long* stats;
  int d, M, dsub, L, ML, b, k_max, prune, collect;
  float lo;    // (1 - gamma) factor of the lower bound, rounded down
  float erel;  // relative allowance for the roundings of s_q, s_x and |s_q - s_x|
  float eps;   // Eq. 4 (1 = the exact, margined test)
};

// Bytes of dynamic shared memory of the verify kernel.
size_t pq_verify_smem(int d, int L, int ML) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    o = (o + 15) & ~(size_t)15;
    o += bytes;
  };
  take((size_t)d * 4);                 // r
  take((size_t)L * 8);                 // level energies (FP64)
  take((size_t)L * 4);                 // s_q per level
  take((size_t)ML * PQ_KSUB * 4);      // level table
  take((size_t)2 * PQ_S * 4);          // partial distances (two lists)
  take((size_t)2 * PQ_S * 2);          // live candidates (two lists)
  take(64);                            // counters, threshold
  return o;
}

__device__ __forceinline__ float threshold_of(const unsigned long long* slots, int k) {
  const unsigned long long key = ld_volatile_u64(slots + k - 1);
  return key == kEmptyKey ? INFINITY : key_dist(key);
}

// Table of one level: lut[mm][j] = term(r_m, C_m[j]) for m = m0 + mm.  Four
// consecutive codewords per thread (their DS-float rows arrive as DS float4
// loads, 16-byte aligned since j0 % 4 == 0), stored as one float4.
template <int DS>
__device__ __forceinline__ void build_table_v(float* lut, const float* r,
                                              const float* __restrict__ cb, int m0, int ML) {
  for (int e4 = threadIdx.x; e4 < ML * (PQ_KSUB / 4); e4 += blockDim.x) {
    const int mm = e4 / (PQ_KSUB / 4), j0 = (e4 % (PQ_KSUB / 4)) * 4;
    const int m = m0 + mm;
    const float4* c4 = reinterpret_cast<const float4*>(cb + ((size_t)m * PQ_KSUB + j0) * DS);
    float cv[4 * DS];
#pragma unroll
    for (int t = 0; t < DS; ++t) {
      const float4 v = __ldg(c4 + t);
      cv[4 * t] = v.x;
      cv[4 * t + 1] = v.y;
      cv[4 * t + 2] = v.z;
      cv[4 * t + 3] = v.w;
    }
    float rv[DS];
#pragma unroll
    for (int t = 0; t < DS; ++t) rv[t] = r[m * DS + t];
    float o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = pq_term(rv, cv + u * DS, DS);
    *reinterpret_cast<float4*>(lut + mm * PQ_KSUB + j0) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

__device__ __forceinline__ void build_table(float* lut, const float* r,
                                            const float* __restrict__ cb, int m0, int ML,
                                            int dsub) {
  switch (dsub) {
    case 1: build_table_v<1>(lut, r, cb, m0, ML); break;
    case 2: build_table_v<2>(lut, r, cb, m0, ML); break;
    case 4: build_table_v<4>(lut, r, cb, m0, ML); break;
    case 8: build_table_v<8>(lut, r, cb, m0, ML); break;
    default:
      for (int e = threadIdx.x; e < ML * PQ_KSUB; e += blockDim.x) {
        const int m = m0 + e / PQ_KSUB;
        lut[e] = pq_term(r + m * dsub, cb + ((size_t)m * PQ_KSUB + (e % PQ_KSUB)) * dsub, dsub);
      }
  }
}

// Eq. 3 in partial-distance form, margined (see search_pq): keep unless
// (1 - gamma) (P + max(0, |s_q - s_x| - 8u (s_q + s_x))^2) > tau.
// eps < 1: Eq. 4, the Cauchy-Schwarz term scaled by eps,
// LB_eps = P + s_q^2 + s_x^2 - 2 eps s_q s_x (approximate by design: no
// rounding allowance; what is returned still carries its computed distance).
__device__ __forceinline__ bool pq_keep(float P, float sx, float sql, float tau, float erel,
                                        float lo, float eps) {
  float lb;
  if (eps < 1.f) {
    lb = P + fmaxf(0.f, fmaf(sql, sql, sx * sx) - 2.f * eps * sql * sx);
  } else {
    float gap = fabsf(__fsub_rn(sql, sx)) - erel * (sql + sx);
    gap = fmaxf(gap, 0.f);
    lb = __fmaf_rn(gap, gap, P);
  }
  return !(lb * lo > tau);
}

// One level's partial distance of one candidate whose codes start at cp
// (subquantiser rows PQ_B bytes apart), terms added in subquantiser order;
// codes are loaded eight at a time so their latencies overlap.
template <bool LUT>
__device__ __forceinline__ float level_sum1(const uint8_t* __restrict__ cp, int ML, int m0,
                                            const float* lut, const float* r,
                                            const float* __restrict__ cb, int dsub) {
  float S = 0.f;
  for (int mm0 = 0; mm0 < ML; mm0 += 8) {
    int code[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) code[u] = mm0 + u < ML ? __ldg(cp + (size_t)(mm0 + u) * PQ_B) : 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (mm0 + u < ML) {
        const int m = m0 + mm0 + u;
        const float e = LUT ? lut[(mm0 + u) * PQ_KSUB + code[u]]
                            : pq_term(r + m * dsub, cb + ((size_t)m * PQ_KSUB + code[u]) * dsub,
                                      dsub);
        S = mm0 + u == 0 ? e : __fadd_rn(S, e);
      }
    }
  }
  return S;
}

// level_sum1 without a table for a compile-time subvector width: the eight
// codewords of a round are loaded together (after their codes) before any
// term is formed, so a round costs two load latencies, not eight.
template <int DS>
__device__ __forceinline__ float level_sum1_direct(const uint8_t* __restrict__ cp, int ML, int m0,
                                                   const float* r,
                                                   const float* __restrict__ cb) {
  float S = 0.f;
  for (int mm0 = 0; mm0 < ML; mm0 += 8) {
    int code[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) code[u] = mm0 + u < ML ? __ldg(cp + (size_t)(mm0 + u) * PQ_B) : 0;
    float cv[8][DS];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int m = min(m0 + mm0 + u, m0 + ML - 1);
      const float* c = cb + ((size_t)m * PQ_KSUB + code[u]) * DS;
#pragma unroll
      for (int t = 0; t < DS; ++t) cv[u][t] = __ldg(c + t);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (mm0 + u < ML) {
        const int m = m0 + mm0 + u;
        float rv[DS];
#pragma unroll
        for (int t = 0; t < DS; ++t) rv[t] = r[m * DS + t];
        const float e = pq_term(rv, cv[u], DS);
        S = mm0 + u == 0 ? e : __fadd_rn(S, e);
      }
    }
  }
  return S;
}

// A level's partial distance without a table, any subvector width.
__device__ __forceinline__ float level_sum_direct(const uint8_t* __restrict__ cp, int ML, int m0,
                                                  const float* r,
                                                  const float* __restrict__ cb, int dsub) {
  switch (dsub) {
    case 1: return level_sum1_direct<1>(cp, ML, m0, r, cb);
    case 2: return level_sum1_direct<2>(cp, ML, m0, r, cb);
    case 4: return level_sum1_direct<4>(cp, ML, m0, r, cb);
    default: return level_sum1<false>(cp, ML, m0, nullptr, r, cb, dsub);
  }
}

// The same for four consecutive candidates (one 32-bit load carries their
// four codes of a subquantiser), eight subquantisers per round, the next
// round's codes loaded while the current round's terms are summed.
template <bool LUT>
__device__ __forceinline__ void level_sum4(const uint32_t* __restrict__ cp, int ML, int m0,
                                           const float* lut, const float* r,
                                           const float* __restrict__ cb, int dsub, float S[4]) {
  constexpr int G = 8;
  uint32_t w[G];
#pragma unroll
  for (int u = 0; u < G; ++u) w[u] = u < ML ? __ldg(cp + (size_t)u * (PQ_B / 4)) : 0u;
#pragma unroll 1
  for (int mm0 = 0; mm0 < ML; mm0 += G) {
    uint32_t wn[G];
#pragma unroll
    for (int u = 0; u < G; ++u)
      wn[u] = mm0 + G + u < ML ? __ldg(cp + (size_t)(mm0 + G + u) * (PQ_B / 4)) : 0u;
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if (mm0 + u < ML) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int code = (w[u] >> (8 * c)) & 255;
          const int m = m0 + mm0 + u;
          const float e = LUT ? lut[(mm0 + u) * PQ_KSUB + code]
                              : pq_term(r + m * dsub, cb + ((size_t)m * PQ_KSUB + code) * dsub,
                                        dsub);
          S[c] = mm0 + u == 0 ? e : __fadd_rn(S[c], e);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) w[u] = wn[u];
  }
}

__global__ void __launch_bounds__(PQ_NT, 3) pq_verify_kernel(const PqArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int d = a.d, L = a.L, ML = a.ML, M = a.M, dsub = a.dsub;
  size_t o = 0;
  auto carve = [&](size_t bytes) {
    o = (o + 15) & ~(size_t)15;
    unsigned char* p = smem + o;
    o += bytes;
    return p;
  };
  float* r = (float*)carve((size_t)d * 4);
  double* eq = (double*)carve((size_t)L * 8);
  float* sq = (float*)carve((size_t)L * 4);
  float* lut = (float*)carve((size_t)ML * PQ_KSUB * 4);
  float* pacc = (float*)carve((size_t)2 * PQ_S * 4);
  uint16_t* live = (uint16_t*)carve((size_t)2 * PQ_S * 2);
  int* ctr = (int*)carve(64);  // [0] survivors of the level, [2] threshold bits, [3] k,
                               // [8..15] four 64-bit section clocks
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // section clocks in shared memory (thread 0's view: the block's barriers
  // align the phases): prologue, level-0 tables, level-0 scan, deeper levels
  unsigned long long* sec = reinterpret_cast<unsigned long long*>(ctr + 8);
  long long t_mark = 0;
  if (a.collect && threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) sec[i] = 0;
    t_mark = clock64();
  }
  auto lap = [&](int i) {
    if (a.collect && threadIdx.x == 0) {
      const long long t = clock64();
      sec[i] += (unsigned long long)(t - t_mark);
      t_mark = t;
    }
  };
  const int2 pr = a.pairs[blockIdx.x];
  if (pr.x < 0) return;  // a slot of a query that probes fewer lists
  const int q = pr.x, c = pr.y;
  const int nc = a.list_size[c];
  if (nc == 0 || a.kq[q] == 0) return;
  const int64_t blk0 = a.blk_off[c];
  unsigned long long* slots = a.topk + (size_t)q * a.k_max;
  // the query's k, read from shared memory where it is used (kept out of
  // the registers the level loops need)
  volatile int* s_kq = ctr + 3;
  if (tid == 0) *s_kq = a.kq[q];

  for (int j = tid; j < d; j += PQ_NT)
    r[j] = __fsub_rn(a.qt[(size_t)q * d + j], a.cent_t[(size_t)c * d + j]);
  __syncthreads();
  // FP64 level energies of the residual (one warp per level) while the whole
  // block builds level 0's table (the first slab needs it when it is large)
  for (int l = warp; l < L; l += PQ_NT / 32) {
    double s = 0.0;
    for (int j = lane; j < a.b; j += 32) {
      const double v = r[l * a.b + j];
      s += v * v;
    }
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) eq[l] = s;
  }
  int lut_level = -1;  // the level whose table `lut` holds (uniform)
  unsigned long long n_lut = 0;
  if (min(PQ_S, nc) >= PQ_LUT_MIN) {
    build_table(lut, r, a.codebook, 0, ML, dsub);
    lut_level = 0;
    n_lut = 1;
  }
  __syncthreads();
  // tail after level l: one lane per level, FP64 sum, sqrt rounded to FP32
  if (warp == 0)
    for (int l = lane; l < L; l += 32) {
      double tail = 0.0;
      for (int l2 = L - 1; l2 > l; --l2) tail += eq[l2];
      sq[l] = (float)sqrt(tail);
    }
  __syncthreads();

  lap(0);
  // counters (every thread keeps its own; summed at the end when collecting)
  unsigned long long n_dims = 0, n_lv = 0, n_full = 0;
  for (int s0 = 0; s0 < nc; s0 += PQ_S) {
    const int ns = min(PQ_S, nc - s0);
    int nl = ns, cur = 0;
    for (int l = 0; l < L && nl > 0; ++l) {
      const bool last = l == L - 1;
      if (l > 0 && a.prune && nl <= PQ_DEEP) {
        // few survivors: each thread walks its own through the remaining
        // levels (terms straight from the codebook, the same bits as the
        // tables), stopping at the first level whose test fails; no block
        // barrier per level
        for (int i = tid; i < nl; i += PQ_NT) {
          const int cand = live[cur * PQ_S + i];
          float P = pacc[cur * PQ_S + i];
          const int g = s0 + cand;
          const int64_t blk = blk0 + g / PQ_B;
          const int ln = g % PQ_B;
          for (int ll = l; ll < L; ++ll) {
            const float tq = threshold_of(slots, *s_kq);
            const uint8_t* cp = a.codes + (blk * M + (int64_t)ll * ML) * PQ_B + ln;
            P = __fadd_rn(P, level_sum_direct(cp, ML, ll * ML, r, a.codebook, dsub));
            n_dims += a.b;
            ++n_lv;
            if (ll == L - 1) {
              ++n_full;
              const unsigned long long key = make_key(P, a.ids[blk * PQ_B + ln]);
              if (key < ld_volatile_u64(slots + *s_kq - 1)) topk_insert_thread(slots, *s_kq, key);
            } else if (!pq_keep(P, a.xtail[(blk * L + ll) * PQ_B + ln], sq[ll], tq, a.erel,
                                a.lo, a.eps)) {
              break;
            }
          }
        }
        __syncthreads();  // the next slab reuses the live list
        lap(3);
        break;
      }
      if (tid == 0) {
        ctr[0] = 0;
        ctr[2] = __float_as_int(threshold_of(slots, *s_kq));
      }
      const bool use_lut = nl >= PQ_LUT_MIN;
      if (use_lut && lut_level != l) {
        build_table(lut, r, a.codebook, l * ML, ML, dsub);
        lut_level = l;
        if (tid == 0) ++n_lut;
      }
      __syncthreads();
      lap(l == 0 ? 1 : 3);
      const float tau = __int_as_float(ctr[2]);
      const float sql = sq[l];
      const int nxt = cur ^ 1;
      auto passes = [&](float P, float sx) {
        return !a.prune || pq_keep(P, sx, sql, tau, a.erel, a.lo, a.eps);
      };
      // level 0 visits every candidate of the slab: four consecutive ones per
      // thread (one 32-bit code load per subquantiser); deeper levels visit
      // the live list, one candidate per thread
      const bool dense = l == 0;
      const int nunits = dense ? (ns + 3) >> 2 : nl;
      for (int i0 = 0; i0 < nunits; i0 += PQ_NT) {
        const int i = i0 + tid;
        bool keep[4] = {false, false, false, false};
        float Pv[4] = {0.f, 0.f, 0.f, 0.f};
        int cand0 = 0;
        if (i < nunits && dense) {
          cand0 = 4 * i;
          const int g = s0 + cand0;
          const int64_t blk = blk0 + g / PQ_B;
          const int ln = g % PQ_B;
          const uint32_t* cp = reinterpret_cast<const uint32_t*>(a.codes + blk * M * PQ_B + ln);
          float S[4];
          if (use_lut)
            level_sum4<true>(cp, ML, 0, lut, r, a.codebook, dsub, S);
          else
            level_sum4<false>(cp, ML, 0, lut, r, a.codebook, dsub, S);
          float sxv[4] = {0.f, 0.f, 0.f, 0.f};
          if (!last) {
            const float4 t4 = *reinterpret_cast<const float4*>(a.xtail + blk * L * PQ_B + ln);
            sxv[0] = t4.x;
            sxv[1] = t4.y;
            sxv[2] = t4.z;
            sxv[3] = t4.w;
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (cand0 + c >= ns) continue;
            const float P = __fadd_rn(0.f, S[c]);
            Pv[c] = P;
            if (last) {
              const unsigned long long key = make_key(P, a.ids[blk * PQ_B + ln + c]);
              if (key < ld_volatile_u64(slots + *s_kq - 1)) topk_insert_thread(slots, *s_kq, key);
            } else {
              keep[c] = passes(P, sxv[c]);
            }
          }
        } else if (i < nunits) {
          cand0 = live[cur * PQ_S + i];
          const int g = s0 + cand0;
          const int64_t blk = blk0 + g / PQ_B;
          const int ln = g % PQ_B;
          const uint8_t* cp = a.codes + (blk * M + (int64_t)l * ML) * PQ_B + ln;
          const float S = use_lut ? level_sum1<true>(cp, ML, l * ML, lut, r, a.codebook, dsub)
                                  : level_sum_direct(cp, ML, l * ML, r, a.codebook, dsub);
          const float P = __fadd_rn(pacc[cur * PQ_S + i], S);
          Pv[0] = P;
          if (last) {
            const unsigned long long key = make_key(P, a.ids[blk * PQ_B + ln]);
            if (key < ld_volatile_u64(slots + *s_kq - 1)) topk_insert_thread(slots, *s_kq, key);
          } else {
            keep[0] = passes(P, a.xtail[(blk * L + l) * PQ_B + ln]);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c > 0 && !dense) break;
          const unsigned ball = __ballot_sync(0xffffffffu, keep[c]);
          if (ball) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&ctr[0], __popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (keep[c]) {
              const int at = base + __popc(ball & ((1u << lane) - 1));
              live[nxt * PQ_S + at] = (uint16_t)(cand0 + c);
              pacc[nxt * PQ_S + at] = Pv[c];
            }
          }
        }
      }
      __syncthreads();
      if (a.collect && tid == 0) {
        n_dims += (unsigned long long)nl * a.b;
        n_lv += nl;
        if (last) n_full += nl;
      }
      nl = last ? 0 : ctr[0];
      cur = nxt;
      __syncthreads();
      lap(l == 0 ? 2 : 3);
    }
  }
  if (a.collect) {
    for (int off = 16; off; off >>= 1) {
      n_dims += __shfl_xor_sync(0xffffffffu, n_dims, off);
      n_lv += __shfl_xor_sync(0xffffffffu, n_lv, off);
      n_full += __shfl_xor_sync(0xffffffffu, n_full, off);
    }
    if (lane == 0 && n_lv) {
      atomicAdd(a.stats + 1, n_dims);
      atomicAdd(a.stats + 2, n_lv);
      atomicAdd(a.stats + 3, n_full);
    }
    if (tid == 0) {
      atomicAdd(a.stats + 0, (unsigned long long)nc);
      atomicAdd(a.stats + 4, n_lut);
      atomicAdd(a.stats + 5, 1ULL);
      for (int i = 0; i < 4; ++i) atomicAdd(a.stats + 8 + i, sec[i]);
    }
  }
}

// Seeds each query's top-k with the first PQ_SEED members of its nearest
// list, distances computed exactly as pq_verify_kernel computes them (level
// sums in subquantiser order, added in level order), so that the verify
// kernel's insert of the same candidate meets an equal key and is dropped.
__global__ void __launch_bounds__(256) pq_seed_kernel(const PqArgs a,
                                                      const int32_t* __restrict__ probes,
                                                      int nprobe) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int d = a.d, L = a.L, ML = a.ML, dsub = a.dsub;
  float* r = (float*)smem;
  float* part = r + ((d + 3) & ~3);  // [PQ_SEED][L]
  const int q = blockIdx.x;
  const int c = probes[(size_t)q * nprobe];
  const int ns = min(PQ_SEED, a.list_size[c]);
  const int kq = a.kq[q];
  if (ns == 0 || kq == 0) return;
  const int64_t blk0 = a.blk_off[c];
  for (int j = threadIdx.x; j < d; j += blockDim.x)
    r[j] = __fsub_rn(a.qt[(size_t)q * d + j], a.cent_t[(size_t)c * d + j]);
  __syncthreads();
  // neighbouring lanes take neighbouring candidates of one level, so a warp's
  // code loads hit one 32-byte run per subquantiser
  for (int e = threadIdx.x; e < ns * L; e += blockDim.x) {
    const int cand = e % ns, l = e / ns;
    const int64_t blk = blk0 + cand / PQ_B;
    const int ln = cand % PQ_B;
    const uint8_t* cp = a.codes + (blk * a.M + (int64_t)l * ML) * PQ_B + ln;
    part[cand * L + l] = level_sum_direct(cp, ML, l * ML, r, a.codebook, dsub);
  }
  __syncthreads();
  for (int cand = threadIdx.x; cand < ns; cand += blockDim.x) {
    float P = 0.f;
    for (int l = 0; l < L; ++l) P = __fadd_rn(P, part[cand * L + l]);
    const int64_t blk = blk0 + cand / PQ_B;
    topk_insert_thread(a.topk + (size_t)q * a.k_max, kq,
                       make_key(P, a.ids[blk * PQ_B + cand % PQ_B]));
  }
}

// Pair order: each query's nearest list first (grouped by list), then the
// other probes (grouped by list).  bucket b = (rank > 0) * nlist + list.
// Per-query probe counts and k, clamped to [1, cap] and [0, k_max].
__global__ void pq_prep_kernel(int64_t nq, const int32_t* __restrict__ npq_in, int cap,
                               const int32_t* __restrict__ kq_in, int k, int k_max,
                               int32_t* __restrict__ npq, int32_t* __restrict__ kq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  npq[i] = npq_in ? min(max(npq_in[i], 1), cap) : cap;
  kq[i] = kq_in ? min(max(kq_in[i], 0), k_max) : k;
}

// A probe slot makes a pair when its rank is below the query's nprobe and
// the query wants at least one result.
__device__ __forceinline__ bool pq_pair_live(int64_t i, int nprobe, const int32_t* npq,
                                             const int32_t* kq) {
  const int64_t q = i / nprobe;
  return (int)(i % nprobe) < npq[q] && kq[q] > 0;
}

__global__ void pq_pair_count_kernel(const int32_t* __restrict__ probes, int64_t nq, int nprobe,
                                     int nlist, const int32_t* __restrict__ npq,
                                     const int32_t* __restrict__ kq, int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe || !pq_pair_live(i, nprobe, npq, kq)) return;
  const int rank = (int)(i % nprobe);
  atomicAdd(cnt + (rank > 0) * nlist + probes[i], 1);
}

__global__ void __launch_bounds__(1024) pq_pair_scan_kernel(const int* __restrict__ cnt, int nb,
                                                            int* __restrict__ off) {
  __shared__ int s_part[1024];
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int sum = 0;
  for (int b = b0; b < min(nb, b0 + per); ++b) sum += cnt[b];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  for (int st = 1; st < 1024; st <<= 1) {
    const int v = threadIdx.x >= st ? s_part[threadIdx.x - st] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s_part[threadIdx.x] - sum;
  for (int b = b0; b < min(nb, b0 + per); ++b) {
    off[b] = run;
    run += cnt[b];
  }
}

__global__ void pq_pair_scatter_kernel(const int32_t* __restrict__ probes, int64_t nq, int nprobe,
                                       int nlist, const int32_t* __restrict__ npq,
                                       const int32_t* __restrict__ kq, int* __restrict__ fill,
                                       const int* __restrict__ off, int2* __restrict__ pairs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe || !pq_pair_live(i, nprobe, npq, kq)) return;
  const int rank = (int)(i % nprobe);
  const int c = probes[i];
  const int b = (rank > 0) * nlist + c;
  const int at = off[b] + atomicAdd(fill + b, 1);
  pairs[at] = make_int2((int)(i / nprobe), c);
}

__global__ void pq_decode_kernel(const unsigned long long* __restrict__ topk, int64_t n,
                                 int64_t* __restrict__ ids, float* __restrict__ dists) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long key = topk[i];
  ids[i] = key == kEmptyKey ? -1 : (int64_t)key_id(key);
  dists[i] = key == kEmptyKey ? INFINITY : key_dist(key);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
}

}  // namespace

// ------------------------------------------------------------------ build
int build_ivfpq(const pano_transform* t, const float* X, int64_t n, int nlist,
                const pano_pq_build_opts* o, cudaStream_t st, pano_index** out) {
  PANO_CHECK(t && X && out && o, PANO_EINVAL, "null argument");
  const int d = t->d, M = o->M, L = o->n_levels;
  PANO_CHECK(n >= 1 && nlist >= 1 && nlist <= n, PANO_EINVAL, "need 1 <= nlist <= n");
  PANO_CHECK(n < ((int64_t)1 << 31) - 1, PANO_EINVAL, "at most 2^31-2 vectors");
  PANO_CHECK(L >= 1 && L <= PQ_MAXL && d % L == 0, PANO_EINVAL,
             "n_levels must divide d (at most 64 levels)");
  PANO_CHECK(M >= 1 && d % M == 0 && M % L == 0, PANO_EINVAL,
             "M must divide d and be a multiple of n_levels");
  const int dsub = d / M, ML = M / L;
  PANO_CHECK(ML <= PQ_MAXML, PANO_EINVAL, "at most 64 subquantisers per level");
  PANO_CHECK(dsub <= PQ_MAXDSUB, PANO_EINVAL, "at most 32 coordinates per subvector");
  PANO_CHECK(o->codebooks || n >= PQ_KSUB, PANO_EINVAL,
             "training codebooks needs at least 256 vectors");
  if (o->assign) {
    PANO_CHECK(o->centroids, PANO_EINVAL, "an assignment needs its centroids");
    for (int64_t i = 0; i < n; ++i)
      PANO_CHECK(o->assign[i] >= 0 && o->assign[i] < nlist, PANO_EINVAL,
                 "assignment out of range");
  }
  int dev = 0;
  int rc = check_device(&dev);
  if (rc) return rc;
  auto idx = std::make_unique<pano_index>();
  pano_index& I = *idx;
  I.device = dev;
  I.n = n;
  I.d = d;
  I.nlist = nlist;
  I.precision = PANO_PQ;
  I.chunk = PQ_B;
  I.L = L;
  I.pq_M = M;
  I.pq_dsub = dsub;
  I.tf = *t;
  I.eta = t->eta;
  I.widths.assign(L, d / L);
  I.offs.assign(L + 1, 0);
  for (int l = 0; l < L; ++l) I.offs[l + 1] = I.offs[l] + d / L;
  I.max_w = d / L;

  const float* Xd = X;
  DTmp t_x;
  if (!is_device_ptr(X)) {
    PANO_CUDA(cudaMalloc(&t_x.p, (size_t)n * d * 4));
    PANO_CUDA(cudaMemcpyAsync(t_x.p, X, (size_t)n * d * 4, cudaMemcpyHostToDevice, st));
    Xd = (const float*)t_x.p;
  }

  // ---- coarse quantiser and lists
  pano_build_opts co;
  std::memset(&co, 0, sizeof(co));
  co.kmeans_iters = o->kmeans_iters;
  co.kmeans_sample = o->kmeans_sample;
  co.seed = o->seed ? o->seed : 1234;
  co.centroids = o->centroids;
  if (o->assign) {
    // centroids and lists given: only the centroid arrays are needed
    I.centroids.assign(o->centroids, o->centroids + (size_t)nlist * d);
    std::vector<float> hcn(nlist);
    float cmax = 0.f;
    for (int c = 0; c < nlist; ++c) {
      double s = 0;
      for (int j = 0; j < d; ++j)
        s += (double)I.centroids[(size_t)c * d + j] * I.centroids[(size_t)c * d + j];
      hcn[c] = (float)s;
      cmax = std::max(cmax, (float)std::sqrt(s));
    }
    I.cmax = cmax;
    if ((rc = I.cent.alloc((size_t)nlist * d * 4)) || (rc = I.cent_n2.alloc(nlist * 4))) return rc;
    PANO_CUDA(cudaMemcpyAsync(I.cent.p, I.centroids.data(), (size_t)nlist * d * 4,
                              cudaMemcpyHostToDevice, st));
    PANO_CUDA(cudaMemcpyAsync(I.cent_n2.p, hcn.data(), nlist * 4, cudaMemcpyHostToDevice, st));
    I.assign.assign(o->assign, o->assign + n);
  } else {
    rc = coarse_lists(Xd, n, d, nlist, &co, st, I);
    if (rc) return rc;
  }

  // ---- list layout (host): blocks of PQ_B slots, ascending id within a list
  I.list_size.assign(nlist, 0);
  for (int64_t i = 0; i < n; ++i) I.list_size[I.assign[i]]++;
  I.list_chunk_off.assign(nlist + 1, 0);
  for (int c = 0; c < nlist; ++c)
    I.list_chunk_off[c + 1] = I.list_chunk_off[c] + (I.list_size[c] + PQ_B - 1) / PQ_B;
  I.n_chunks = I.list_chunk_off[nlist];
  const int64_t nslots = I.n_chunks * PQ_B;
  std::vector<int64_t> perm(nslots, -1);
  std::vector<int32_t> slot_list(nslots, -1);
  {
    std::vector<int64_t> fill(nlist, 0);
    for (int64_t i = 0; i < n; ++i) {
      const int c = I.assign[i];
      const int64_t s = I.list_chunk_off[c] * PQ_B + fill[c]++;
      perm[s] = i;
      slot_list[s] = c;
    }
  }
  if ((rc = I.chunk_off_d.alloc((nlist + 1) * 8)) || (rc = I.list_size_d.alloc(nlist * 4)) ||
      (rc = I.level_off_d.alloc((L + 1) * 4)) || (rc = I.T32.alloc((size_t)d * d * 4)) ||
      (rc = I.mu32.alloc(d * 4)) || (rc = I.pq_cent_t.alloc((size_t)nlist * d * 4)) ||
      (rc = I.pq_codebook.alloc((size_t)M * PQ_KSUB * dsub * 4)) ||
      (rc = I.pq_codes.alloc((size_t)std::max<int64_t>(nslots, 1) * M)) ||
      (rc = I.tails.alloc((size_t)std::max<int64_t>(nslots, 1) * L * 4)) ||
      (rc = I.ids.alloc((size_t)std::max<int64_t>(nslots, 1) * 4)))
    return rc;
  PANO_CUDA(cudaMemcpyAsync(I.chunk_off_d.p, I.list_chunk_off.data(), (nlist + 1) * 8,
                            cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.list_size_d.p, I.list_size.data(), nlist * 4,
                            cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.level_off_d.p, I.offs.data(), (L + 1) * 4, cudaMemcpyHostToDevice,
                            st));
  PANO_CUDA(cudaMemcpyAsync(I.T32.p, t->T32.data(), (size_t)d * d * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.mu32.p, t->mu32.data(), d * 4, cudaMemcpyHostToDevice, st));
  // c~ = T~(c - mu~)
  PANO_CUDA(gemm_nt(kStore, nlist, d, d, I.cent.as<float>(), d, I.mu32.as<float>(),
                    I.T32.as<float>(), d, I.pq_cent_t.as<float>(), d, nullptr, nullptr, st));

  DTmp t_perm, t_sl;
  PANO_CUDA(cudaMalloc(&t_perm.p, std::max<int64_t>(nslots, 1) * 8));
  PANO_CUDA(cudaMalloc(&t_sl.p, std::max<int64_t>(nslots, 1) * 4));
  PANO_CUDA(cudaMemcpyAsync(t_perm.p, perm.data(), nslots * 8, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(t_sl.p, slot_list.data(), nslots * 4, cudaMemcpyHostToDevice, st));
  const size_t cbsm = (size_t)PQ_KSUB * dsub * 4;

  // rows (or sampled rows) -> transformed residuals, in blocks of rows
  auto residuals = [&](const int64_t* rows_d, const int32_t* lists_d, int64_t m,
                       float* out_r) -> int {
    if (m == 0) return PANO_OK;
    pq_gather_kernel<<<(unsigned)m, 128, 0, st>>>(Xd, d, rows_d, m, out_r);
    PANO_CUDA(cudaGetLastError());
    // in place: the GEMM reads rows and writes x~ to a second buffer
    DTmp t_xt;
    PANO_CUDA(cudaMalloc(&t_xt.p, (size_t)m * d * 4));
    PANO_CUDA(gemm_nt(kStore, (int)m, d, d, out_r, d, I.mu32.as<float>(), I.T32.as<float>(), d,
                      (float*)t_xt.p, d, nullptr, nullptr, st));
    pq_residual_kernel<<<(unsigned)m, 128, 0, st>>>((float*)t_xt.p, m, d,
                                                    I.pq_cent_t.as<float>(), lists_d);
    PANO_CUDA(cudaGetLastError());
    PANO_CUDA(cudaMemcpyAsync(out_r, t_xt.p, (size_t)m * d * 4, cudaMemcpyDeviceToDevice, st));
    PANO_CUDA(cudaStreamSynchronize(st));
    return PANO_OK;
  };

  // ---- codebooks
  if (o->codebooks) {
    PANO_CUDA(cudaMemcpyAsync(I.pq_codebook.p, o->codebooks, (size_t)M * PQ_KSUB * dsub * 4,
                              cudaMemcpyHostToDevice, st));
  } else {
    const int64_t ns = std::min<int64_t>(n, o->pq_sample > 0 ? o->pq_sample : 65536);
    std::vector<int64_t> rows = sample_rows(n, std::max<int64_t>(ns, PQ_KSUB),
                                            (o->seed ? o->seed : 1234) ^ 0x5051ULL);
    const int64_t m = (int64_t)rows.size();
    std::vector<int32_t> lists(m);
    for (int64_t i = 0; i < m; ++i) lists[i] = I.assign[rows[i]];
    DTmp t_rows, t_lists, t_r, t_sums, t_cnt;
    PANO_CUDA(cudaMalloc(&t_rows.p, m * 8));
    PANO_CUDA(cudaMalloc(&t_lists.p, m * 4));
    PANO_CUDA(cudaMalloc(&t_r.p, (size_t)m * d * 4));
    PANO_CUDA(cudaMalloc(&t_sums.p, (size_t)M * PQ_KSUB * dsub * 8));
    PANO_CUDA(cudaMalloc(&t_cnt.p, (size_t)M * PQ_KSUB * 4));
    PANO_CUDA(cudaMemcpyAsync(t_rows.p, rows.data(), m * 8, cudaMemcpyHostToDevice, st));
    PANO_CUDA(cudaMemcpyAsync(t_lists.p, lists.data(), m * 4, cudaMemcpyHostToDevice, st));
    rc = residuals((const int64_t*)t_rows.p, (const int32_t*)t_lists.p, m, (float*)t_r.p);
    if (rc) return rc;
    // initial codewords: 256 distinct sampled rows' subvectors
    std::vector<int64_t> init = sample_rows(m, PQ_KSUB, (o->seed ? o->seed : 1234) ^ 0xC0DEULL);
    std::vector<float> hr((size_t)m * d);
    PANO_CUDA(cudaMemcpyAsync(hr.data(), t_r.p, hr.size() * 4, cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaStreamSynchronize(st));
    std::vector<float> cb((size_t)M * PQ_KSUB * dsub);
    for (int mq = 0; mq < M; ++mq)
      for (int j = 0; j < PQ_KSUB; ++j)
        for (int tt = 0; tt < dsub; ++tt)
          cb[((size_t)mq * PQ_KSUB + j) * dsub + tt] = hr[(size_t)init[j] * d + mq * dsub + tt];
    PANO_CUDA(cudaMemcpyAsync(I.pq_codebook.p, cb.data(), cb.size() * 4, cudaMemcpyHostToDevice,
                              st));
    const int iters = o->pq_iters > 0 ? o->pq_iters : 16;
    for (int it = 0; it < iters; ++it) {
      PANO_CUDA(cudaMemsetAsync(t_sums.p, 0, (size_t)M * PQ_KSUB * dsub * 8, st));
      PANO_CUDA(cudaMemsetAsync(t_cnt.p, 0, (size_t)M * PQ_KSUB * 4, st));
      pq_kmeans_accum_kernel<<<dim3((unsigned)((m + 255) / 256), M), 256, cbsm, st>>>(
          (const float*)t_r.p, m, d, dsub, I.pq_codebook.as<float>(), (double*)t_sums.p,
          (int*)t_cnt.p);
      PANO_CUDA(cudaGetLastError());
      const int64_t tot = (int64_t)M * PQ_KSUB * dsub;
      pq_kmeans_update_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
          M, dsub, (const double*)t_sums.p, (const int*)t_cnt.p, I.pq_codebook.as<float>());
      PANO_CUDA(cudaGetLastError());
    }
  }

  // ---- codes, in the block layout
  if (o->codes) {
    DTmp t_codes;
    PANO_CUDA(cudaMalloc(&t_codes.p, (size_t)n * M));
    PANO_CUDA(cudaMemcpyAsync(t_codes.p, o->codes, (size_t)n * M, cudaMemcpyHostToDevice, st));
    const int64_t tot = nslots * M;
    if (tot > 0)
      pq_scatter_codes_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
          (const uint8_t*)t_codes.p, M, (const int64_t*)t_perm.p, nslots,
          I.pq_codes.as<uint8_t>());
    PANO_CUDA(cudaGetLastError());
    PANO_CUDA(cudaStreamSynchronize(st));
  } else {
    PANO_CUDA(cudaMemsetAsync(I.pq_codes.p, 0, (size_t)std::max<int64_t>(nslots, 1) * M, st));
    // blocks of slots (a multiple of PQ_B): 64 MB of residuals each
    const int64_t step =
        std::max<int64_t>(PQ_B, (((int64_t)1 << 24) / d) / PQ_B * PQ_B);
    DTmp t_r;
    PANO_CUDA(cudaMalloc(&t_r.p, (size_t)std::min(step, std::max<int64_t>(nslots, 1)) * d * 4));
    for (int64_t s0 = 0; s0 < nslots; s0 += step) {
      const int64_t m = std::min(step, nslots - s0);
      rc = residuals((const int64_t*)t_perm.p + s0, (const int32_t*)t_sl.p + s0, m,
                     (float*)t_r.p);
      if (rc) return rc;
      pq_encode_kernel<<<dim3((unsigned)((m + 255) / 256), M), 256, cbsm, st>>>(
          (const float*)t_r.p, m, d, M, dsub, I.pq_codebook.as<float>(),
          (const int32_t*)t_sl.p + s0, 1, I.pq_codes.as<uint8_t>() + s0 * M);
      PANO_CUDA(cudaGetLastError());
    }
  }

  // ---- ids and tail norms
  {
    DTmp t_cn;
    PANO_CUDA(cudaMalloc(&t_cn.p, (size_t)M * PQ_KSUB * 8));
    pq_cnorm_kernel<<<(unsigned)((M * PQ_KSUB + 255) / 256), 256, 0, st>>>(
        M, dsub, I.pq_codebook.as<float>(), (double*)t_cn.p);
    if (nslots > 0)
      pq_tails_kernel<<<(unsigned)((nslots + 255) / 256), 256, 0, st>>>(
          I.pq_codes.as<uint8_t>(), (const int64_t*)t_perm.p, nslots, M, L,
          (const double*)t_cn.p, I.tails.as<float>(), I.ids.as<int32_t>());
    PANO_CUDA(cudaGetLastError());
    PANO_CUDA(cudaStreamSynchronize(st));
  }
  *out = idx.release();
  return PANO_OK;
}

// ----------------------------------------------------------------- search
// npq_in / kq_in: device per-query nprobe / k (clamped), or null for the
// scalars; with npq_in, nprobe is the cap of every query's probes.
int search_pq(const pano_index* ip, const float* queries, int64_t nq, const int32_t* npq_in,
              int nprobe, const int32_t* kq_in, int k, int k_max, int64_t* out_ids,
              float* out_dists, int mode, int collect, float epsilon, cudaStream_t st) {
  PANO_CHECK(ip, PANO_EINVAL, "null index");
  const pano_index& I = *ip;
  PANO_CHECK(I.pq_M > 0, PANO_EINVAL, "not an IVFPQ index (panorama_build_ivfpq)");
  PANO_CHECK(nq >= 0 && nq < (1LL << 31), PANO_EINVAL, "nq out of range");
  PANO_CHECK(nq == 0 || (queries && out_ids && out_dists), PANO_EINVAL, "null argument");
  PANO_CHECK(k_max >= 1 && k_max <= 1024, PANO_EINVAL, "k_max must be in [1, 1024]");
  if (!kq_in) PANO_CHECK(k >= 0 && k <= k_max, PANO_EINVAL, "k must be in [0, k_max]");
  if (npq_in) nprobe = nprobe >= 1 ? std::min(nprobe, I.nlist) : I.nlist;
  PANO_CHECK(nprobe >= 1 && nprobe <= I.nlist, PANO_EINVAL, "nprobe must be in [1, nlist]");
  PANO_CHECK((int64_t)nq * nprobe < (1LL << 31), PANO_EINVAL, "too many (query, list) pairs");
  pano_search_stats& S = stats_slot();
  std::memset(&S, 0, sizeof(S));
  S.n_queries = nq;
  if (nq == 0) return PANO_OK;
  const bool counts = (collect & 1) != 0, timing = (collect & 2) != 0;
  int cur = 0;
  PANO_CUDA(cudaGetDevice(&cur));
  PANO_CHECK(cur == I.device, PANO_EINVAL, "current device differs from the index's device");
  const int d = I.d, L = I.L, M = I.pq_M, dsub = I.pq_dsub, ML = M / L, nlist = I.nlist;
  const int64_t npairs = nq * nprobe;

  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    size_t at = off;
    off += bytes;
    return at;
  };
  const size_t o_qt = take((size_t)nq * d * 4);
  const size_t o_pr = take((size_t)npairs * 4);
  const size_t o_pairs = take((size_t)npairs * 8);
  const size_t o_cnt = take((size_t)2 * nlist * 4);
  const size_t o_fill = take((size_t)2 * nlist * 4);
  const size_t o_off = take((size_t)2 * nlist * 4);
  const size_t o_topk = take((size_t)nq * k_max * 8);
  const size_t o_npq = take((size_t)nq * 4);
  const size_t o_kq = take((size_t)nq * 4);
  const size_t o_stats = take(16 * 8);
  void* ws = nullptr;
  PANO_CUDA(cudaMallocAsync(&ws, off, st));
  char* W = (char*)ws;
  float* qt = (float*)(W + o_qt);
  int32_t* probes = (int32_t*)(W + o_pr);
  int2* pairs = (int2*)(W + o_pairs);
  int* cnt = (int*)(W + o_cnt);
  int* fill = (int*)(W + o_fill);
  int* poff = (int*)(W + o_off);
  unsigned long long* topk = (unsigned long long*)(W + o_topk);
  unsigned long long* stats = (unsigned long long*)(W + o_stats);
  int32_t* npq = (int32_t*)(W + o_npq);
  int32_t* kq = (int32_t*)(W + o_kq);

  cudaEvent_t ev[6] = {};
  if (timing)
    for (auto& e : ev) PANO_CUDA(cudaEventCreate(&e));
  auto mark = [&](int i) {
    if (timing) cudaEventRecord(ev[i], st);
  };
  auto body = [&]() -> int {
    PANO_CUDA(cudaMemsetAsync(cnt, 0, (size_t)2 * nlist * 4, st));
    PANO_CUDA(cudaMemsetAsync(fill, 0, (size_t)2 * nlist * 4, st));
    PANO_CUDA(cudaMemsetAsync(topk, 0xff, (size_t)nq * k_max * 8, st));
    PANO_CUDA(cudaMemsetAsync(pairs, 0xff, (size_t)npairs * 8, st));  // (-1, -1): no pair
    PANO_CUDA(cudaMemsetAsync(stats, 0, 16 * 8, st));
    pq_prep_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(nq, npq_in, nprobe, kq_in, k,
                                                                k_max, npq, kq);
    // q~ = T~(q - mu~)
    mark(0);
    PANO_CUDA(gemm_nt(kStore, (int)nq, d, d, queries, d, I.mu32.as<float>(), I.T32.as<float>(),
                      d, qt, d, nullptr, nullptr, st));
    mark(1);
    int rc = probe_only(ip, queries, nq, nprobe, probes, st);
    if (rc) return rc;
    mark(2);
    const unsigned pg = (unsigned)((npairs + 255) / 256);
    pq_pair_count_kernel<<<pg, 256, 0, st>>>(probes, nq, nprobe, nlist, npq, kq, cnt);
    pq_pair_scan_kernel<<<1, 1024, 0, st>>>(cnt, 2 * nlist, poff);
    pq_pair_scatter_kernel<<<pg, 256, 0, st>>>(probes, nq, nprobe, nlist, npq, kq, fill, poff,
                                               pairs);
    PANO_CUDA(cudaGetLastError());

    PqArgs a;
    std::memset(&a, 0, sizeof(a));
    a.codes = I.pq_codes.as<uint8_t>();
    a.xtail = I.tails.as<float>();
    a.ids = I.ids.as<int32_t>();
    a.blk_off = I.chunk_off_d.as<int64_t>();
    a.list_size = I.list_size_d.as<int32_t>();
    a.codebook = I.pq_codebook.as<float>();
    a.cent_t = I.pq_cent_t.as<float>();
    a.qt = qt;
    a.pairs = pairs;
    a.topk = topk;
    a.stats = stats;
    a.d = d;
    a.M = M;
    a.dsub = dsub;
    a.L = L;
    a.ML = ML;
    a.b = d / L;
    a.kq = kq;
    a.k_max = k_max;
    a.prune = mode == 0 ? 1 : 0;
    a.collect = counts ? 1 : 0;
    // D~ >= (1-u)^(L + ML + dsub + 2) (D_head~ + (sqrt R_q - sqrt R_x)^2) (level
    // and subquantiser sums of non-negative terms, each term's subtraction,
    // square and additions); the computed bound and its scaling add three
    // roundings up: lo = 1 - gamma_{L + ML + dsub + 6}, rounded down.
    const double lo = 1.0 - gamma_n((double)L + ML + dsub + 6);
    float lo32 = (float)lo;
    if ((double)lo32 > lo) lo32 = std::nextafter(lo32, 0.f);
    a.lo = lo32;
    // s_q, s_x: FP64 sums rounded to FP32 (u each), |s_q - s_x| and the
    // allowance itself (u each): 8u of (s_q + s_x) covers them with margin.
    a.erel = (float)(8.0 * kU32);
    a.eps = (epsilon > 0.f && epsilon < 1.f) ? epsilon : 1.f;

    const size_t ssm = (size_t)((d + 3) & ~3) * 4 + (size_t)PQ_SEED * L * 4;
    PANO_CUDA(cudaFuncSetAttribute(pq_seed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)ssm));
    pq_seed_kernel<<<(unsigned)nq, 256, ssm, st>>>(a, probes, nprobe);
    PANO_CUDA(cudaGetLastError());
    mark(3);
    const size_t vsm = pq_verify_smem(d, L, ML);
    PANO_CUDA(cudaFuncSetAttribute(pq_verify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)vsm));
    pq_verify_kernel<<<(unsigned)npairs, PQ_NT, vsm, st>>>(a);
    PANO_CUDA(cudaGetLastError());
    mark(4);
    pq_decode_kernel<<<(unsigned)((nq * k_max + 255) / 256), 256, 0, st>>>(topk, nq * k_max, out_ids,
                                                                      out_dists);
    PANO_CUDA(cudaGetLastError());
    mark(5);
    unsigned long long hs[16] = {};
    PANO_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaStreamSynchronize(st));
    if (timing) {
      // stage_ms: transform, probe, pair order + seeds, -, verify, decode
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      S.stage_ms[0] = ms;
      cudaEventElapsedTime(&ms, ev[1], ev[2]);
      S.stage_ms[1] = ms;
      cudaEventElapsedTime(&ms, ev[2], ev[3]);
      S.stage_ms[2] = ms;
      cudaEventElapsedTime(&ms, ev[3], ev[4]);
      S.stage_ms[4] = ms;
      cudaEventElapsedTime(&ms, ev[4], ev[5]);
      S.stage_ms[5] = ms;
    }
    if (counts) {
      S.pairs = (int64_t)hs[0];
      S.dims_scanned = (int64_t)hs[1];
      S.pair_levels = (int64_t)hs[2];
      S.reranked = (int64_t)hs[3];
      S.tile_levels = (int64_t)hs[4];
      S.work_items = (int64_t)hs[5];
      // block clocks: prologue, level-0 tables, level-0 scan, deeper levels
      for (int i = 0; i < 4; ++i) S.section_cycles[i] = (int64_t)hs[8 + i];
    }
    return PANO_OK;
  };
  int rc = body();
  cudaFreeAsync(ws, st);
  if (timing)
    for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

int debug_pq_encode(const float* R, int64_t n, int d, int M, const float* cb, uint8_t* codes,
                    cudaStream_t st) {
  PANO_CHECK(R && cb && codes, PANO_EINVAL, "null argument");
  PANO_CHECK(n >= 0 && M >= 1 && d % M == 0 && d / M <= PQ_MAXDSUB, PANO_EINVAL,
             "M must divide d with at most 32 coordinates per subvector");
  if (n == 0) return PANO_OK;
  const int dsub = d / M;
  pq_encode_kernel<<<dim3((unsigned)((n + 255) / 256), M), 256, (size_t)PQ_KSUB * dsub * 4, st>>>(
      R, n, d, M, dsub, cb, nullptr, 0, codes);
  PANO_CUDA(cudaGetLastError());
  PANO_CUDA(cudaStreamSynchronize(st));
  return PANO_OK;
}

}  // namespace pano

using namespace pano;

extern "C" {

int panorama_transform_import(const double* T, const double* mu, const double* lam, int32_t d,
                              pano_transform** out) {
  clear_error();
  PANO_CHECK(T && mu && lam && out && d >= 1, PANO_EINVAL, "bad arguments to transform_import");
  auto t = std::make_unique<pano_transform>();
  t->d = d;
  t->T.assign(T, T + (size_t)d * d);
  t->mu.assign(mu, mu + d);
  t->lam.assign(lam, lam + d);
  for (double v : t->T) PANO_CHECK(std::isfinite(v), PANO_EINVAL, "non-finite T");
  for (double v : t->mu) PANO_CHECK(std::isfinite(v), PANO_EINVAL, "non-finite mu");
  for (double v : t->lam) PANO_CHECK(std::isfinite(v) && v >= 0, PANO_EINVAL, "bad lam");
  finish_transform(*t);
  *out = t.release();
  return PANO_OK;
}

int panorama_shape_transform(const pano_transform* t, int32_t n_levels, double kappa,
                             const double* gauss, int32_t* blocks, pano_transform** out) {
  clear_error();
  PANO_CHECK(t && gauss && out, PANO_EINVAL, "null argument");
  const int d = t->d, L = n_levels;
  PANO_CHECK(L >= 1 && d % L == 0, PANO_EINVAL, "n_levels must divide d");
  PANO_CHECK(std::isfinite(kappa) && kappa >= 1.0, PANO_EINVAL, "kappa must be >= 1");
  PANO_CHECK((int)t->lam.size() == d, PANO_EINVAL, "the transform has no coordinate variances");
  for (size_t i = 0; i < (size_t)2 * d * d; ++i)
    PANO_CHECK(std::isfinite(gauss[i]), PANO_EINVAL, "non-finite Gaussian draw");
  const int b = d / L;
  const double* G1 = gauss;
  const double* G2 = gauss + (size_t)d * d;
  std::vector<double> v(t->lam);
  double tot = 0.0;
  for (double x : v) tot += x;
  const double cap = kappa * tot / L;
  const double tie = 1e-12;
  auto tn = std::make_unique<pano_transform>();
  tn->d = d;
  tn->mu = t->mu;
  tn->T = t->T;
  std::vector<std::pair<int, int>> bl;
  std::vector<double> Q;
  // Procedure 1: Robin Hood inter-level shaping
  for (int l = 0; l < L; ++l) {
    const int a = l * b;
    double E = 0.0;
    for (int j = a; j < a + b; ++j) E += v[j];
    if (E <= cap * (1 + tie)) continue;
    int s = 1;
    double sum = E + v[a + b];
    while (a + b + s < d && (double)b * sum > cap * (b + s) * (1 + tie)) {
      sum += v[a + b + s];
      ++s;
    }
    const int nb = b + s;
    haar_q(G1 + (size_t)a * d + a, d, nb, Q);
    rotate_rows(tn->T, d, a, nb, Q);
    double bs = 0.0;
    for (int j = a; j < a + nb; ++j) bs += v[j];
    for (int j = a; j < a + nb; ++j) v[j] = bs / nb;
    bl.emplace_back(a, nb);
  }
  // Procedure 2: intra-level isotropisation
  for (int l = 0; l < L; ++l) {
    const int a = l * b;
    haar_q(G2 + (size_t)a * d + a, d, b, Q);
    rotate_rows(tn->T, d, a, b, Q);
    double E = 0.0;
    for (int j = a; j < a + b; ++j) E += v[j];
    for (int j = a; j < a + b; ++j) v[j] = E / b;
  }
  tn->lam = v;
  finish_transform(*tn);
  if (blocks) {
    for (int i = 0; i < 2 * L; ++i) blocks[i] = -1;
    for (size_t i = 0; i < bl.size() && (int)i < L; ++i) {
      blocks[2 * i] = bl[i].first;
      blocks[2 * i + 1] = bl[i].second;
    }
  }
  *out = tn.release();
  return PANO_OK;
}

int panorama_build_ivfpq(const pano_transform* t, const float* X, int64_t n, int32_t nlist,
                         const pano_pq_build_opts* opts, void* stream, pano_index** out) {
  clear_error();
  return build_ivfpq(t, X, n, nlist, opts, (cudaStream_t)stream, out);
}

int panorama_search_pq(const pano_index* idx, const float* queries, int64_t nq, int32_t nprobe,
                       int32_t k, int64_t* out_ids, float* out_dists, int32_t mode,
                       int32_t collect_stats, float epsilon, void* stream) {
  clear_error();
  PANO_CHECK(k >= 1 && k <= 1024, PANO_EINVAL, "k must be in [1, 1024]");
  return search_pq(idx, queries, nq, nullptr, nprobe, nullptr, k, k, out_ids, out_dists, mode,
                   collect_stats, epsilon, (cudaStream_t)stream);
}

int panorama_search_pq_ex(const pano_index* idx, const float* queries, int64_t nq,
                          const int32_t* nprobe, int32_t nprobe_scalar, const int32_t* k,
                          int32_t k_scalar, int32_t k_max, int64_t* out_ids, float* out_dists,
                          const pano_search_opts* opts, void* stream) {
  clear_error();
  const int collect = opts ? ((opts->collect_stats ? 1 : 0) | (opts->collect_timing ? 2 : 0)) : 0;
  return search_pq(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max, out_ids,
                   out_dists, opts ? opts->mode : 0, collect, opts ? opts->epsilon : 1.f,
                   (cudaStream_t)stream);
}

int panorama_pq_export(const pano_index* idx, float* codebooks, uint8_t* codes, int32_t* M_out) {
  clear_error();
  PANO_CHECK(idx && idx->pq_M > 0, PANO_EINVAL, "not an IVFPQ index");
  const pano_index& I = *idx;
  const int M = I.pq_M;
  if (M_out) *M_out = M;
  if (codebooks)
    PANO_CUDA(cudaMemcpy(codebooks, I.pq_codebook.p, (size_t)M * PQ_KSUB * I.pq_dsub * 4,
                         cudaMemcpyDeviceToHost));
  if (codes) {
    const int64_t nslots = I.n_chunks * PQ_B;
    std::vector<uint8_t> lay((size_t)std::max<int64_t>(nslots, 1) * M);
    std::vector<int32_t> ids((size_t)std::max<int64_t>(nslots, 1));
    PANO_CUDA(cudaMemcpy(lay.data(), I.pq_codes.p, (size_t)nslots * M, cudaMemcpyDeviceToHost));
    PANO_CUDA(cudaMemcpy(ids.data(), I.ids.p, (size_t)nslots * 4, cudaMemcpyDeviceToHost));
    for (int64_t s = 0; s < nslots; ++s) {
      if (ids[s] < 0) continue;
      for (int m = 0; m < M; ++m)
        codes[(size_t)ids[s] * M + m] = lay[((s / PQ_B) * M + m) * PQ_B + s % PQ_B];
    }
  }
  return PANO_OK;
}

int panorama_debug_pq_encode(const float* R, int64_t n, int32_t d, int32_t M,
                             const float* codebooks, uint8_t* codes, void* stream) {
  clear_error();
  return debug_pq_encode(R, n, d, M, codebooks, codes, (cudaStream_t)stream);
}

}  // extern "C"
