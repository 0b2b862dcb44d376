// panorama_search: the device hot path.
//
//   a1 transform_queries   q~ = T~(q - mu~) (FP32 GEMM) + per-query norms,
//                          rounded-up tail norms sqrt(R_q^{(l,d)}) and the
//                          transform-error bound e_q                  [Alg. 1]
//   a2 probe + select      original-space expansion distances to every
//                          centroid, radix select of the nprobe-th, exact
//                          re-score of the boundary band    [Section 6.1]
//   a3 work inversion      probes -> per-list query buckets -> work items
//                          (list, segment, query group); rank-0 probes (each
//                          query's nearest list) form phase A, the rest B
//   a4-a8 verify           level-wise partial products, bound update,
//                          pruning and survivor compaction   [Eq. 2-3, Alg. 1]
//   a9 re-rank             survivors' exact distances on the original rows
//   a10 top-k              lock-free k-smallest insertion per query; its k-th
//                          key is the running threshold d_k      [Alg. 1]
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "gemm.h"
#include "internal.h"
#include "kernels_common.cuh"
#include "probe_tc.h"
#include "search.h"
#include "verify_tc.h"

namespace pano {

namespace {

constexpr int CH = 64;
// Device statistics words: [0] pair-levels, [1] tile-levels, [2] slice bytes,
// [3] reranked, [4] pairs, [5] unused, [6] / [7] dims of phase A / B,
// [8..15] section cycles, [16..23] their phase-A part, [24] phase-A pairs,
// [25] live-row bytes (tensor-core path).
constexpr int kStatWords = 26;
constexpr int SEG_CHUNKS = 32;  // chunks per work-item segment
constexpr int NT = 256;

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// --------------------------------------------------------------- a1: norms
// One warp per query.  The transformed row is first staged in shared memory
// with one batch of coalesced loads (so the level loop below does not wait
// on global memory L times).  Level energies are summed from the last level
// backwards in compensated FP32 (Acc2: the FP64 pipe is a small fraction of
// the FP32 one), giving the rounded-up tail norms directly; the rounded
// norms keep the accuracy of one rounding of the exact value.
constexpr int kNormRows = 8;      // queries (warps) per CTA
constexpr int kNormMaxD = 1536;   // staged row length (48 KB per CTA); longer rows read global memory

__global__ void __launch_bounds__(kNormRows * 32) query_norms_kernel(
    const float* __restrict__ q, const float* __restrict__ qt, int64_t nq, int d, int L,
    const int32_t* __restrict__ level_off, const float* __restrict__ mu, float c_trans_up,
    float4* __restrict__ qinfo, float* __restrict__ qtail, float* __restrict__ qn2) {
  extern __shared__ float qrow_s[];  // [kNormRows][d] when d <= kNormMaxD
  const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * kNormRows + w;
  if (row >= nq) return;
  const float* x = qt + row * d;
  if (d <= kNormMaxD) {
    float* xs = qrow_s + (size_t)w * d;
    for (int j = lane; j < d; j += 32) xs[j] = x[j];
    __syncwarp();
    x = xs;
  }
  Acc2 suffix{0.f, 0.f};
  float xmax = 0.f;  // largest |q~_j| (the FP8 path's query scale)
  for (int l = L - 1; l >= 0; --l) {
    Acc2 e{0.f, 0.f};
    for (int j = level_off[l] + lane; j < level_off[l + 1]; j += 32) {
      acc2_sq(e, x[j]);
      xmax = fmaxf(xmax, fabsf(x[j]));
    }
    acc2_add(suffix, warp_sum_acc2(e));
    if (lane == 0) qtail[row * (L + 1) + l] = __fsqrt_ru(acc2_upper(suffix, 0x1p-23f));
  }
  // deviation from the mean: each fl(q_j - mu_j) is within u of the exact
  // difference, so the slack 4u covers the squares' 2u and Acc2's 2^-30
  Acc2 dev{0.f, 0.f}, on{0.f, 0.f};
  for (int j = lane; j < d; j += 32) {
    const float v = q[row * d + j];
    acc2_sq(dev, __fsub_rn(v, mu[j]));
    acc2_sq(on, v);
  }
  dev = warp_sum_acc2(dev);
  on = warp_sum_acc2(on);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, off));
  if (lane == 0) {
    qtail[row * (L + 1) + L] = 0.f;
    const float nqf = __fadd_rn(suffix.s, suffix.c);
    qinfo[row] = make_float4(nqf, sqrtf(nqf),
                             __fmul_ru(c_trans_up, __fsqrt_ru(acc2_upper(dev, 0x1p-21f))), xmax);
    qn2[row] = __fadd_rn(on.s, on.c);
  }
}

// FP32 squared norms of rows (compensated FP32 sums, rounded once).
__global__ void row_sqnorm_kernel(const float* __restrict__ X, int64_t m, int d,
                                  float* __restrict__ out) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= m) return;
  Acc2 s{0.f, 0.f};
  for (int j = threadIdx.x & 31; j < d; j += 32) acc2_sq(s, X[row * d + j]);
  s = warp_sum_acc2(s);
  if ((threadIdx.x & 31) == 0) out[row] = __fadd_rn(s.s, s.c);
}

// nprobe / k per query, clamped to [1, nlist] and [0, k_max].
__global__ void prep_kernel(int64_t nq, const int32_t* __restrict__ nprobe, int nprobe_scalar,
                            int nprobe_cap, const int32_t* __restrict__ k, int k_scalar,
                            int k_max, int32_t* __restrict__ npq, int32_t* __restrict__ kq,
                            int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  int np = nprobe ? nprobe[i] : nprobe_scalar;
  int kk = k ? k[i] : k_scalar;
  if (np < 1 || np > nprobe_cap || kk < 0 || kk > k_max) atomicOr(err, kErrBadInput);
  npq[i] = min(max(np, 1), nprobe_cap);
  kq[i] = min(max(kk, 0), k_max);
}

// ------------------------------------------------------ a2: probe selection
// One CTA per query.  The nprobe-th smallest expansion distance v is found by
// an 8-bit radix select on order-preserving keys.  With e the expansion's
// rounding bound (|expansion - exact| <= e for every centroid), the nprobe-th
// smallest exact distance D* lies in [v - e, v + e]: a centroid whose
// expansion is above v + 2e is beyond D*, and one below v - 2e is strictly
// inside it, so only the band [v - 2e, v + 2e] needs the compensated
// difference form, and the probe set is the centroids below the band plus
// the band's first ones by (exact distance, list id).  exact_order: every
// centroid up to v + 2e is re-scored and the nprobe are written in ascending
// (exact distance, list id) order; otherwise the ones below the band come
// first, by (expansion distance, list id), then the band's.
constexpr int kBandCap = 1024;

__global__ void __launch_bounds__(NT) probe_select_kernel(
    const float* __restrict__ pdist, int nlist, const float* __restrict__ q,
    const float* __restrict__ cent, int d, const float* __restrict__ qn2, float cmax,
    float gerr, const int32_t* __restrict__ npq, int nprobe_stride,
    int32_t* __restrict__ probes, int* __restrict__ err, int exact_order) {
  extern __shared__ uint32_t keys[];  // nlist
  __shared__ int hist[256];
  __shared__ int s_bin, s_below;
  // below the band: [0, n_in); the band: [kBandCap - n_band, kBandCap)
  __shared__ int n_in, n_band;
  __shared__ int band_id[kBandCap];
  __shared__ float band_d[kBandCap];
  const int64_t row = blockIdx.x;
  const int m = npq[row];
  const float* pd = pdist + row * (int64_t)nlist;
  for (int i = threadIdx.x; i < nlist; i += NT) keys[i] = float_ordered(pd[i]);
  if (threadIdx.x == 0) n_in = n_band = 0;
  uint32_t prefix = 0, mask = 0;
  int remaining = m;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += NT) hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nlist; i += NT) {
      uint32_t k = keys[i];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // first bin b with (count below b) + hist[b] >= remaining: lane l
      // holds bins 8l..8l+7; a warp scan of the lane totals and a ballot
      // find the lane, which walks its eight bins (b = 256 if none)
      const int lane = threadIdx.x;
      int h[8], tot = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        h[u] = hist[lane * 8 + u];
        tot += h[u];
      }
      int inc = tot;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, inc >= remaining);
      if (lane == (hit ? __ffs(hit) - 1 : 31)) {
        int acc = inc - tot, b = lane * 8 + 8;
        bool found = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (!found) {
            if (acc + h[u] >= remaining) {
              found = true;
              b = lane * 8 + u;
            } else {
              acc += h[u];
            }
          }
        }
        s_bin = b;
        s_below = acc;
      }
    }
    __syncthreads();
    prefix |= (uint32_t)s_bin << shift;
    mask |= 255u << shift;
    remaining -= s_below;
    __syncthreads();
  }
  // decode v and split the centroids up to v + 2e into "below the band" and
  // "in the band"
  uint32_t u = (prefix & 0x80000000u) ? (prefix & 0x7fffffffu) : ~prefix;
  float v = __uint_as_float(u);
  float s = sqrtf(qn2[row]) + cmax;
  const float e2 = 2.f * gerr * s * s;
  float hi = v + e2;
  const float lo = exact_order ? -INFINITY : v - e2;
  for (int i = threadIdx.x; i < nlist; i += NT) {
    const float di = pd[i];
    if (di <= hi) {
      if (di < lo) {
        const int pos = atomicAdd(&n_in, 1);
        if (pos < kBandCap) {
          band_id[pos] = i;
          band_d[pos] = di;
        }
      } else {
        const int pos = atomicAdd(&n_band, 1);
        if (pos < kBandCap) band_id[kBandCap - 1 - pos] = i;
      }
    }
  }
  __syncthreads();
  const bool over = n_in + n_band > kBandCap;
  if (threadIdx.x == 0 && over) atomicOr(err, kErrOverflow);
  const int ni = over ? 0 : n_in;
  const int nb = over ? min(n_band, kBandCap) : n_band;
  const int b0 = kBandCap - nb;  // the band occupies [b0, kBandCap)
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  for (int b = b0 + warp; b < kBandCap; b += NT / 32) {
    float e = exact_sqdist_warp(q + row * d, cent + (int64_t)band_id[b] * d, d);
    if (lane == 0) band_d[b] = e;
  }
  __syncthreads();
  // ranks: below the band among themselves, the band among itself after them
  int32_t* out = probes + row * (int64_t)nprobe_stride;
  for (int b = threadIdx.x; b < ni; b += NT) {
    const float db = band_d[b];
    const int ib = band_id[b];
    int rank = 0;
    for (int o = 0; o < ni; ++o) {
      const float dd = band_d[o];
      rank += (dd < db) || (dd == db && band_id[o] < ib);
    }
    if (rank < m) out[rank] = ib;
  }
  for (int b = b0 + threadIdx.x; b < kBandCap; b += NT) {
    const float db = band_d[b];
    const int ib = band_id[b];
    int rank = ni;
    for (int o = b0; o < kBandCap; ++o) {
      const float dd = band_d[o];
      rank += (dd < db) || (dd == db && band_id[o] < ib);
    }
    if (rank < m) out[rank] = ib;
  }
  for (int r = ni + nb + threadIdx.x; r < m; r += NT) out[r] = -1;  // unreachable unless nlist < m
}

// ------------------------------------------------------- a3: work inversion
__global__ void inv_count_kernel(int64_t nq, const int32_t* __restrict__ probes, int stride,
                                 const int32_t* __restrict__ npq, int* __restrict__ cnt,
                                 int nlist, int first_rank_b) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * stride) return;
  int64_t qi = e / stride;
  int r = (int)(e % stride);
  if (r >= npq[qi]) return;
  int c = probes[e];
  if (c < 0) return;
  atomicAdd(&cnt[(r < first_rank_b ? 0 : nlist) + c], 1);
}

// Single CTA: exclusive scans of bucket sizes and of work items per list for
// both phases.  items(c) = ceil(cnt / QB_phase) * nseg(c).
__global__ void __launch_bounds__(1024) inv_scan_kernel(const int* __restrict__ cnt, int nlist,
                                                        const int64_t* __restrict__ chunk_off,
                                                        int seg, int qbA, int qbB,
                                                        int* __restrict__ boff,
                                                        int* __restrict__ ioff,
                                                        int* __restrict__ totals) {
  __shared__ int part_b[1024], part_i[1024];
  for (int ph = 0; ph < 2; ++ph) {
    const int* cn = cnt + ph * nlist;
    const int qb = ph == 0 ? qbA : qbB;
    int per = (nlist + 1023) / 1024;
    int b0 = threadIdx.x * per, b1 = min(nlist, b0 + per);
    int sb = 0, si = 0;
    for (int c = b0; c < b1; ++c) {
      int nch = (int)(chunk_off[c + 1] - chunk_off[c]);
      int nseg = (nch + seg - 1) / seg;
      sb += cn[c];
      si += ((cn[c] + qb - 1) / qb) * nseg;
    }
    part_b[threadIdx.x] = sb;
    part_i[threadIdx.x] = si;
    __syncthreads();
    if (threadIdx.x == 0) {
      int ab = 0, ai = 0;
      for (int t = 0; t < 1024; ++t) {
        int xb = part_b[t], xi = part_i[t];
        part_b[t] = ab;
        part_i[t] = ai;
        ab += xb;
        ai += xi;
      }
      totals[2 * ph] = ab;
      totals[2 * ph + 1] = ai;
    }
    __syncthreads();
    int ab = part_b[threadIdx.x], ai = part_i[threadIdx.x];
    for (int c = b0; c < b1; ++c) {
      int nch = (int)(chunk_off[c + 1] - chunk_off[c]);
      int nseg = (nch + seg - 1) / seg;
      boff[ph * (nlist + 1) + c] = ab;
      ioff[ph * (nlist + 1) + c] = ai;
      ab += cn[c];
      ai += ((cn[c] + qb - 1) / qb) * nseg;
    }
    if (threadIdx.x == 1023) {
      boff[ph * (nlist + 1) + nlist] = ab;
      ioff[ph * (nlist + 1) + nlist] = ai;
    }
    __syncthreads();
  }
}

__global__ void inv_scatter_kernel(int64_t nq, const int32_t* __restrict__ probes, int stride,
                                   const int32_t* __restrict__ npq, const int* __restrict__ boff,
                                   const int* __restrict__ totals, int* __restrict__ fill,
                                   int nlist, int first_rank_b, int32_t* __restrict__ bucket) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * stride) return;
  int64_t qi = e / stride;
  int r = (int)(e % stride);
  if (r >= npq[qi]) return;
  int c = probes[e];
  if (c < 0) return;
  int ph = r < first_rank_b ? 0 : 1;
  int base = ph == 1 ? totals[0] : 0;  // phase-B buckets follow the phase-A ones
  int pos = base + boff[ph * (nlist + 1) + c] + atomicAdd(&fill[ph * nlist + c], 1);
  bucket[pos] = (int32_t)qi;
}

// Work item i of a phase -> (list, segment, bucket offset, group size).
__global__ void inv_emit_kernel(int ph, const int* __restrict__ cnt, int nlist,
                                const int64_t* __restrict__ chunk_off, int seg, int qb,
                                const int* __restrict__ boff, const int* __restrict__ ioff,
                                const int* __restrict__ totals, int64_t cap,
                                int4* __restrict__ items, int* __restrict__ err) {
  const int n_items = totals[2 * ph + 1];
  const int* io = ioff + ph * (nlist + 1);
  const int* bo = boff + ph * (nlist + 1);
  if (n_items > cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrOverflow);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < imin64(n_items, cap);
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nlist;  // largest c with io[c] <= i
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (io[mid] <= i) lo = mid;
      else hi = mid;
    }
    int c = lo;
    while (c + 1 < nlist && io[c + 1] <= i) ++c;  // skip empty lists
    int local = (int)(i - io[c]);
    int nch = (int)(chunk_off[c + 1] - chunk_off[c]);
    int nseg = (nch + seg - 1) / seg;
    int g = local / nseg, s = local % nseg;
    int n_in = cnt[ph * nlist + c];
    int base = (ph == 1 ? totals[0] : 0) + bo[c] + g * qb;
    items[i] = make_int4(c, s, base, min(qb, n_in - g * qb));
  }
}

// ------------------------------------------------- Alg. 1 warm start (a6)
// Per query: distances to the first max(4k, 64) (at most 256) members of its
// nearest list; the k-th smallest is an upper bound on d_k and seeds the
// threshold before any tile is verified.  Algorithm 1 also fills its heap
// with k candidates before pruning anything; that matters once the
// epsilon-relaxed bound of Eq. 4 can prune every candidate of a query, so
// an epsilon-relaxed search (topk != nullptr) also enters the seeds whose
// bound is at most that k-th one (at least k of them) into the top-k with
// their exact distances, computed by the re-ranking's own routine on the
// same rows (a later re-rank of the same candidate yields the same key and
// is kept once).  With exact pruning they would change no result, so exact
// searches skip those k exact distances.
//
// The query row sits in shared memory; a warp loads a whole row (up to 1024
// dims) in one batch and sums fl(q_j - x_j)^2 by FMA into four interleaved
// sums per lane.  Each term meets at most m = ceil(d/128) + 8 roundings, so
// with the differences' relative error u the exact distance is at most the
// computed one times 1 / ((1 - gamma_m)(1 - u)^2) <= slack = 1 + 2(m + 3)u
// (host-computed, rounded up); multiplying by it (rounding up) keeps every
// seed distance an upper bound on the exact one.
constexpr int kSeedMax = 256;
constexpr int kSeedWarps = 8;

__global__ void __launch_bounds__(kSeedWarps * 32) seed_tau_kernel(
    const float* __restrict__ q, int d, const int32_t* __restrict__ probes, int stride,
    const int64_t* __restrict__ chunk_off, const int32_t* __restrict__ list_size, int chunk,
    const float* __restrict__ rows, const int32_t* __restrict__ kq,
    const int32_t* __restrict__ order, float slack, float* __restrict__ tau_seed,
    const int32_t* __restrict__ ids, unsigned long long* __restrict__ topk, int k_max) {
  extern __shared__ float4 qs4[];  // the query row (d floats)
  __shared__ float dist[kSeedMax];
  __shared__ float s_t;
  const int64_t row = order ? order[blockIdx.x] : blockIdx.x;
  const int k = kq[row];
  const int c = probes[row * stride];
  const int n = c >= 0 ? list_size[c] : 0;
  const int ns = min(n, min(kSeedMax, max(4 * k, 64)));
  if (k <= 0 || ns < k) {
    if (threadIdx.x == 0) tau_seed[row] = k <= 0 ? -1.f : INFINITY;
    return;
  }
  float* qs = reinterpret_cast<float*>(qs4);
  for (int j = threadIdx.x; j < d; j += kSeedWarps * 32) qs[j] = q[row * d + j];
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t base = chunk_off[c] * chunk;  // a list's members are its first slots
  const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(rows) & 15) == 0;
  for (int i = warp; i < ns; i += kSeedWarps) {
    const float* x = rows + (base + i) * d;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (vec) {
      const float4* x4 = reinterpret_cast<const float4*>(x);
      const int d4 = d >> 2;
      for (int j0 = 0; j0 < d4; j0 += 8 * 32) {
        float4 xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + lane + 32 * u;
          xv[u] = j < d4 ? x4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + lane + 32 * u;
          if (j < d4) {
            const float4 qv = qs4[j];
            float t;
            t = qv.x - xv[u].x;
            acc[0] = fmaf(t, t, acc[0]);
            t = qv.y - xv[u].y;
            acc[1] = fmaf(t, t, acc[1]);
            t = qv.z - xv[u].z;
            acc[2] = fmaf(t, t, acc[2]);
            t = qv.w - xv[u].w;
            acc[3] = fmaf(t, t, acc[3]);
          }
        }
      }
    } else {
      for (int j0 = 0; j0 < d; j0 += 8 * 32) {
        float xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + lane + 32 * u;
          xv[u] = j < d ? x[j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + lane + 32 * u;
          if (j < d) {
            const float t = qs[j] - xv[u];
            acc[u & 3] = fmaf(t, t, acc[u & 3]);
          }
        }
      }
    }
    float s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) dist[i] = __fadd_ru(__fmul_ru(s, slack), 0x1p-126f);
  }
  __syncthreads();
  if (warp == 0) {
    const float t = warp_kth_smallest(dist, ns, k);
    if (lane == 0) {
      tau_seed[row] = t;
      s_t = t;
    }
  }
  __syncthreads();
  if (!topk) return;
  const float t = s_t;
  for (int i = warp; i < ns; i += kSeedWarps) {
    if (!(dist[i] <= t)) continue;
    const float e = exact_sqdist_warp_wide(q + row * d, rows + (base + i) * d, d);
    topk_insert_warp(topk + row * k_max, k, make_key(e, ids[base + i]));
  }
}

// The same seeds for up to 16 queries of one phase-A work item at once
// (two-phase searches, d <= 1024, d % 4 == 0): the queries sit in shared
// memory and each warp reads one of the list's first rows into registers
// (8 float4 per lane) and computes its distances to all of them, so a list's
// rows are read once per 16 queries instead of once per query.  Per query
// and row, each lane sums fl(q_j - x_j)^2 by FMA over its (at most 32) dims
// into four interleaved sums, then the warp adds the lanes' sums: each term
// meets at most m = ceil(d/128) + 8 roundings, as in seed_tau_kernel, whose
// slack is reused.  CTA b takes sub-group b % nsub of item b / nsub; only
// an item's first segment computes (the queries of a group are the same in
// every segment).
constexpr int kSeedSub = 16;

__global__ void __launch_bounds__(kSeedWarps * 32) seed_group_kernel(
    const float* __restrict__ q, int d, const int4* __restrict__ items,
    const int* __restrict__ n_items, int64_t items_cap, int nsub,
    const int32_t* __restrict__ bucket, const int64_t* __restrict__ chunk_off,
    const int32_t* __restrict__ list_size, int chunk, const float* __restrict__ rows,
    const int32_t* __restrict__ kq, float slack, float* __restrict__ tau_seed,
    const int32_t* __restrict__ ids, unsigned long long* __restrict__ topk, int k_max) {
  extern __shared__ float4 sg_raw[];
  const int64_t item = blockIdx.x / nsub;
  const int sub = blockIdx.x % nsub;
  if (item >= imin64(*n_items, items_cap)) return;
  const int4 it = items[item];
  if (it.y != 0) return;
  const int g0 = sub * kSeedSub, G = min(kSeedSub, it.w - g0);
  if (G <= 0) return;
  const int c = it.x, n = list_size[c];
  const int d4 = d >> 2;
  float4* qs = sg_raw;                                                // [G][d/4]
  float* dist = reinterpret_cast<float*>(sg_raw + (size_t)kSeedSub * d4);  // [G][kSeedMax]
  __shared__ int s_q[kSeedSub], s_k[kSeedSub], s_ns[kSeedSub];
  __shared__ float s_t[kSeedSub];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  if (tid < G) {
    const int qi = bucket[it.z + g0 + tid];
    const int k = kq[qi];
    s_q[tid] = qi;
    s_k[tid] = k;
    s_ns[tid] = min(n, min(kSeedMax, max(4 * k, 64)));
  }
  __syncthreads();
  int nsmax = 0;
  for (int g = 0; g < G; ++g) nsmax = max(nsmax, s_ns[g]);
  for (int e = tid; e < G * d4; e += kSeedWarps * 32) {
    const int g = e / d4, j = e % d4;
    qs[e] = reinterpret_cast<const float4*>(q + (int64_t)s_q[g] * d)[j];
  }
  __syncthreads();
  const int64_t base = chunk_off[c] * chunk;  // a list's members are its first slots
  // two rows per warp in registers: each query float4 read from shared
  // memory serves both (the loop is bound by those reads)
  for (int r0 = 2 * warp; r0 < nsmax; r0 += 2 * kSeedWarps) {
    float4 xv[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4* x4 = reinterpret_cast<const float4*>(rows + (base + r0 + h) * d);
      const bool ok = r0 + h < nsmax;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = lane + 32 * u;
        xv[h][u] = ok && j < d4 ? x4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    for (int g = 0; g < G; ++g) {
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = lane + 32 * u;
        if (j < d4) {
          const float4 qv = qs[g * d4 + j];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float t;
            t = qv.x - xv[h][u].x;
            acc[h][0] = fmaf(t, t, acc[h][0]);
            t = qv.y - xv[h][u].y;
            acc[h][1] = fmaf(t, t, acc[h][1]);
            t = qv.z - xv[h][u].z;
            acc[h][2] = fmaf(t, t, acc[h][2]);
            t = qv.w - xv[h][u].w;
            acc[h][3] = fmaf(t, t, acc[h][3]);
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float sum = (acc[h][0] + acc[h][1]) + (acc[h][2] + acc[h][3]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0 && r0 + h < s_ns[g])
          dist[g * kSeedMax + r0 + h] = __fadd_ru(__fmul_ru(sum, slack), 0x1p-126f);
      }
    }
  }
  __syncthreads();
  for (int g = warp; g < G; g += kSeedWarps) {
    const int k = s_k[g], ns = s_ns[g];
    const float t = (k <= 0) ? -1.f : (ns < k ? INFINITY : warp_kth_smallest(dist + g * kSeedMax, ns, k));
    if (lane == 0) {
      tau_seed[s_q[g]] = t;
      s_t[g] = t;
    }
  }
  if (!topk) return;
  __syncthreads();
  // the seeds within each query's k-th bound enter its top-k (a warp each)
  for (int e = warp; e < G * kSeedMax; e += kSeedWarps) {
    const int g = e / kSeedMax, i = e % kSeedMax;
    if (i >= s_ns[g] || !(dist[g * kSeedMax + i] <= s_t[g])) continue;
    const int64_t qi = s_q[g];
    const float ex = exact_sqdist_warp_wide(q + qi * d, rows + (base + i) * d, d);
    topk_insert_warp(topk + qi * k_max, s_k[g], make_key(ex, ids[base + i]));
  }
}

// ------------------------------------------------------------ a4-a10 verify
struct VerifyArgs {
  const float* slices;
  const float* rows;
  const int64_t* chunk_off;
  const float* qt;
  const float* qorig;
  const float4* qinfo;
  const float* qtail;
  const int32_t* kq;
  float* tau_seed;  // per-query threshold: warm start, lowered by any tile
  const int4* items;
  const int* n_items;  // device count
  int* counter;
  const int32_t* bucket;
  unsigned long long* topk;
  int* err;
  unsigned long long* stats;  // kStatWords counters (layout at kStatWords)
  int64_t items_cap;
  int d, L, max_w, k_max;
  float gslack;    // slack factor: |computed - exact| <= gslack (|q~|+|x~|)^2
  float lb_scale;  // (1 - 8u) / (1 + eta): lower bound in T~ space -> original
  float ub_scale;  // (1 + 8u) / (1 - eta): upper bound in T~ space -> original
  int prune;       // 0: plain scan (prune only after the last level)
  int test_every;  // with prune: test at level l when l % test_every == 0 (and the last)
  int collect;
  int phase;        // 0: phase A (its dims are also counted apart)
  float eps;        // Eq. 4: the query tail term of the pruning test is scaled by eps
  float inv_lb_up;  // 1 / lb_scale rounded up
  int32_t level_off[65];
  int32_t row_off[65];  // first row (of 64 floats) of level l's block in a chunk
  int64_t chunk_rows;   // rows per chunk in the slice array
};

// Shared-memory plan of the FP32 verify kernel, identical on host and device.
// NST stage buffers rotate through (tile, level) steps; each holds, per
// chunk of the tile, one level block of the slice array: the level slice,
// the tail row of the next level and (level 0) the norms, error bounds and
// ids, (max_w + 4) rows of 64 floats.  Query slices are kept
// row-major per query with a row stride of 4 x (odd) floats, so the 128-bit
// reads of four queries' rows by neighbouring threads hit distinct banks.
struct FpSmem {
  uint32_t stage_f;  // floats per stage (also the last level's UB scratch)
  uint32_t qstride;  // floats between two queries' rows in a query slice
  uint32_t qbuf_f;   // floats per query-slice buffer
  uint32_t off_qb, off_cterm, off_qterm, off_qtl, off_ids, off_q, off_pend, total;
  static constexpr int kPend = 256;  // deferred re-rank entries
  __host__ __device__ FpSmem(int QB, int CB, int max_w, int L, int NST) {
    uint32_t sf = (uint32_t)(CB * (max_w + 4));
    if (sf < (uint32_t)(QB * CB)) sf = (uint32_t)(QB * CB);
    stage_f = (sf + 31u) & ~31u;
    qstride = (uint32_t)((max_w + 3) & ~3);
    if (((qstride / 4) & 1u) == 0) qstride += 4;
    qbuf_f = ((uint32_t)QB * qstride + 31u) & ~31u;
    off_qb = (uint32_t)NST * stage_f * 4u;  // two buffers: levels by parity
    off_cterm = off_qb + 2u * qbuf_f * 4u;
    off_qterm = off_cterm + CB * 16u;
    off_qtl = off_qterm + QB * 16u;
    off_ids = off_qtl + (((uint32_t)QB * (L + 1) * 4u + 15u) & ~15u);
    off_q = off_ids + CB * 4u;
    off_pend = off_q + QB * 6u * 4u;
    // slot (8); query, id, lower and upper bound, this tile's bounds (4 each);
    // kept (2)
    total = off_pend + kPend * 34u;
  }
};

// Evaluation slack of the separable test below (FP32 rounding of its three
// products and two sums, relative to (|q~| + E)(|x~| + e_x)).
constexpr float kEvalSlack = 32.f * 5.9604645e-08f;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// sqrt(tau / lb_scale) rounded up, from hardware-rounded operations: y is
// rounded up, rsqrtf has at most 2 ulp error (CUDA's documented bound) and
// the product one rounding; the factor 1 + 2^-19 covers both.
__device__ __forceinline__ float sqrt_ratio_up(float tau, float inv_lb_up) {
  const float y = __fmul_ru(tau, inv_lb_up);
  if (!(y > 0.f)) return 0.f;
  if (y > 1e36f) return 1e18f;
  return __fmul_ru(y * rsqrtf(y), 1.0000019f);
}

// One CTA per work item at a time (persistent).  A tile is CB candidates
// (CB / 64 chunks) x the item's query group (<= QB); thread (tq, tc) owns a
// 4 x 4 register tile of partial products: queries tq + TQ*i, candidates
// 4tc + j.  The tile walks the levels (Algorithm 1's batch step), and the
// staging of the next step runs behind the arithmetic of the current one:
// when level l of tile t starts, level l+1 of the chunks still live (and the
// group's level-(l+1) query slice) is copied speculatively into a second
// stage, and level 0 of tile t+1 (with its norms, bounds and ids) into the
// third.  A tile that dies at level l leaves its speculative copy unused.
// Survivors are re-ranked in batches (those whose lower bound exceeds the
// threshold by then are dropped); the delayed top-k insertions only leave
// the threshold larger for a while, which is still a valid threshold.
template <int QB, int CB, int NTH, int NST>
__global__ void __launch_bounds__(NTH, 2) verify_fp32_kernel(const VerifyArgs a) {
  constexpr int NCH = CB / CH;
  constexpr int TQ = QB / 4;
  constexpr int NW = NTH / 32;
  static_assert(TQ * (CB / 4) == NTH, "4x4 register tile per thread");
  static_assert(TQ <= 32 && (32 % TQ) == 0 && (TQ < 8 || TQ % 8 == 0),
                "a warp holds whole query-row groups");
  static_assert(NCH <= 32, "live-chunk mask");
  // the thread that issues bulk copies: a warp with no per-query setup work
  constexpr int ISSUER = 32 * ((QB + 31) / 32 < NW ? (QB + 31) / 32 : NW - 1);
  extern __shared__ __align__(128) unsigned char smem[];
  const int L = a.L, d = a.d, max_w = a.max_w;
  const FpSmem lay(QB, CB, max_w, L, NST);
  const int QS = (int)lay.qstride;
  float4* cterm = reinterpret_cast<float4*>(smem + lay.off_cterm);    // (ex, rx, Hx, |x|^2)
  float4* qterm = reinterpret_cast<float4*>(smem + lay.off_qterm);    // (E, g rq, Hq, tau)
  float* qtl = reinterpret_cast<float*>(smem + lay.off_qtl);          // [QB][L+1]
  int32_t* ids_s = reinterpret_cast<int32_t*>(smem + lay.off_ids);    // [CB]
  int32_t* qid = reinterpret_cast<int32_t*>(smem + lay.off_q);        // [QB]
  float* qnq = reinterpret_cast<float*>(qid + QB);
  float* qrq = qnq + QB;
  float* qeq = qrq + QB;
  float* qtau = qeq + QB;
  int32_t* qk = reinterpret_cast<int32_t*>(qtau + QB);
  int64_t* pslot = reinterpret_cast<int64_t*>(smem + lay.off_pend);   // deferred re-rank
  int32_t* pq = reinterpret_cast<int32_t*>(pslot + FpSmem::kPend);
  int32_t* pid = pq + FpSmem::kPend;
  float* plb = reinterpret_cast<float*>(pid + FpSmem::kPend);  // the pair's lower bound
  float* pub = plb + FpSmem::kPend;                             // the pair's upper bound
  float* lbt = pub + FpSmem::kPend;                             // this tile's, by survivor
  float* ubt = lbt + FpSmem::kPend;
  uint16_t* keep = reinterpret_cast<uint16_t*>(ubt + FpSmem::kPend);  // entries to re-rank
  const int BR = (max_w + 4) * CH;  // floats per chunk block in a stage
  auto stage_x = [&](int b) { return reinterpret_cast<float*>(smem + (uint32_t)b * lay.stage_f * 4u); };
  auto qslice = [&](int l) {
    return reinterpret_cast<float*>(smem + lay.off_qb + (uint32_t)(l & 1) * lay.qbuf_f * 4u);
  };
  static_assert(NST == 3 || NST == 4, "stage count");
  __shared__ __align__(8) uint64_t bar[NST];
  __shared__ int s_item, s_nsurv, s_npend, s_nkeep;
  __shared__ uint32_t s_live[2];

  const int tid = threadIdx.x;
  // thread -> (tq, tc): a warp holds WQ = min(TQ, 8) query rows x 32 / WQ
  // candidate blocks, so its float4 query loads touch at most 8 rows (one
  // 128-byte wavefront with the odd row stride) and its candidate loads
  // 16 B x 32 / WQ; a warp's candidates (16 or 32) lie in one chunk
  constexpr int WQ = TQ >= 8 ? 8 : TQ, WC = 32 / WQ, NWQ = TQ / WQ;
  const int tq = (tid & 31) % WQ + WQ * ((tid >> 5) % NWQ);
  const int tc = (tid & 31) / WQ + WC * ((tid >> 5) / NWQ);
  const int warp = tid / 32, lane = tid & 31;
  // counters (collect_stats) live in shared memory, off the registers:
  // [0] pair-levels, [1] dims, [2] tile-levels, [3] bytes, [4] reranked
  __shared__ unsigned long long s_stat[5], s_sec[8];
  // per warp: its live pairs (lane << 4 | bit) and their level dot products
  // when few are live (the sparse path of the level loop)
  __shared__ uint16_t s_pair[NTH / 32][32];
  __shared__ float s_pdot[NTH / 32][32];
  __shared__ long long s_tmark, s_tkernel;
  if (tid == 0) {
    for (int b = 0; b < NST; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
    s_nsurv = 0;
    s_npend = 0;
    s_live[0] = s_live[1] = 0u;
    for (int i = 0; i < 5; ++i) s_stat[i] = 0;
    for (int i = 0; i < 8; ++i) s_sec[i] = 0;
    s_tkernel = s_tmark = clock64();
  }
  __syncthreads();
  // stage-buffer state, identical in every thread: phase and pending bits,
  // and a FIFO of free stages (2 bits each, front in the low bits) so that a
  // stage released with an unused speculative copy in flight is reused last
  uint32_t ph = 0, pend = 0, fq = 0;
  int fn = 0;
  bool failed = false;
  auto wait_stage = [&](int b) {
    if (!((pend >> b) & 1u)) return;
    if (!mbar_wait_bounded(&bar[b], (ph >> b) & 1u)) failed = true;
    ph ^= 1u << b;
    pend &= ~(1u << b);
  };
  auto push_free = [&](int b) {
    fq |= (uint32_t)b << (2 * fn);
    ++fn;
  };
  auto pop_free = [&]() {
    const int b = (int)(fq & 3u);
    fq >>= 2;
    --fn;
    return b;
  };
  // stage level l of tile `tile` (chunks in `live`) into buffer b; one
  // thread issues, every thread records the pending copy
  auto issue = [&](int b, int64_t tile, int nch, int l, uint32_t live) {
    const int w = a.level_off[l + 1] - a.level_off[l];
    if ((pend >> b) & 1u) {
      // An earlier (unused) copy into b must have landed, and every thread
      // must have seen that phase complete before the barrier is re-armed:
      // a thread still waiting on the old parity after the next phase had
      // completed too would wait for a phase that never comes.
      wait_stage(b);
      __syncthreads();
    }
    if (tid == ISSUER) {
      const uint32_t blk = (uint32_t)(w + (l == 0 ? 4 : 1)) * CH * 4;  // one level block
      mbar_arrive_expect_tx(&bar[b], (uint32_t)__popc(live) * blk);
      float* xs = stage_x(b);
      for (int c = 0; c < nch; ++c)
        if ((live >> c) & 1u)
          bulk_g2s(xs + (size_t)c * BR, a.slices + ((tile + c) * a.chunk_rows + a.row_off[l]) * CH,
                   blk, &bar[b]);
      if (a.collect) s_stat[3] += (unsigned long long)__popc(live) * w * CH * 4;
    }
    pend |= 1u << b;
  };
  // the group's query slice of level l -> [QB][QS], asynchronously when the
  // rows are 16-byte aligned (completion: cp_async_wait_all + a barrier)
  auto load_qslice = [&](int l, int G) {
    const int m = a.level_off[l], w = a.level_off[l + 1] - m;
    float* dst = qslice(l);
    if (((d | m | w) & 3) == 0) {
      const int nv = w / 4;
      for (int e = tid; e < G * nv; e += NTH) {
        const int g = e / nv, v = e - g * nv;
        cp_async16(dst + g * QS + 4 * v, a.qt + (int64_t)qid[g] * d + m + 4 * v);
      }
      cp_async_commit();
    } else {
      for (int e = tid; e < G * w; e += NTH) {
        const int g = e / w, j = e - g * w;
        dst[g * QS + j] = a.qt[(int64_t)qid[g] * d + m + j];
      }
    }
  };
  auto section = [&](int i) {  // charge the time since the last mark to section i
    if (a.collect && tid == 0) {
      const long long now = clock64();
      s_sec[i] += (unsigned long long)(now - s_tmark);
      s_tmark = now;
    }
  };
  const float gs = a.gslack;
  // per-query terms of the separable form of the margined Eq. 3 test:
  // the pair is pruned when  p + sq sx + (g rq) rx + E ex  <  Hq + Hx, with
  // E = e_q + sqrt(tau / lb_scale) rounded up (see the candidate terms)
  auto set_query_terms = [&](int g, float tau) {
    const float st = tau == INFINITY ? 1e18f : sqrt_ratio_up(tau, a.inv_lb_up);
    const float E = __fadd_ru(qeq[g], st);
    const float nq = qnq[g], rq = qrq[g];
    qterm[g] = make_float4(E, gs * rq, 0.5f * (nq - gs * nq - E * E - kEvalSlack * (rq + E) * (rq + E)),
                           tau);
  };
  // The running threshold of query slot g: k-th key of its top-k (rounded
  // up) and its warm-start seed.  The loads are issued one tile ahead and
  // combined when the tile that uses them starts; a value read early is an
  // older, larger threshold: still a valid one.
  struct TauRead {
    unsigned long long key;
    float seed;
  };
  auto read_tau = [&](int g, int G) {
    TauRead r{kEmptyKey, -1.f};  // k == 0: nothing can enter
    if (g < G && qk[g] > 0) {
      r.key = ld_volatile_u64(a.topk + (int64_t)qid[g] * a.k_max + qk[g] - 1);
      r.seed = __ldcg(a.tau_seed + qid[g]);
    }
    return r;
  };
  auto tau_of = [&](const TauRead& r) {
    if (r.seed < 0.f) return -1.f;
    const float t = r.key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(r.key), 1.000001f);
    return fminf(t, r.seed);
  };
  // exact distances of the deferred survivors (their rows were prefetched
  // into L2 one tile earlier) and their top-k insertion
  // (all threads call it)
  auto rerank_pending = [&]() {
    const int np = s_npend;
    if (tid == 0) s_nkeep = 0;
    __syncthreads();
    // the threshold may have dropped since a pair survived: a lower bound
    // above it rules the pair out without its exact distance; so do k
    // pending pairs of the same query whose upper bounds lie below it (all
    // k are closer; the pair's own upper bound is never below its lower one)
    for (int s = tid; s < np; s += NTH) {
      const int q = pq[s], kk = a.kq[q];
      const unsigned long long key = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + kk - 1);
      const float tau = fminf(key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f),
                              __ldcg(a.tau_seed + q));
      const float lb = plb[s];
      bool keep_s = !(lb > tau);
      if (keep_s) {
        int below = 0;
        for (int o = 0; o < np && below < kk; ++o)
          below += (pq[o] == q) & (__fmul_ru(pub[o], 1.000001f) < lb);
        keep_s = below < kk;
      }
      if (keep_s) keep[atomicAdd(&s_nkeep, 1)] = (uint16_t)s;
    }
    __syncthreads();
    const int nk = s_nkeep;
    if ((d & 3) == 0)  // all kept rows head for L2 at once
      for (int i = tid; i < nk; i += NTH) {
        prefetch_l2(a.rows + pslot[keep[i]] * d, (uint32_t)d * 4);
        prefetch_l2(a.qorig + (int64_t)pq[keep[i]] * d, (uint32_t)d * 4);
      }
    // exact distances (a warp each; they replace the lower bounds), then
    // the top-k insertions (a thread each, so their chains overlap)
    for (int i = warp; i < nk; i += NW) {
      const int s = keep[i];
      const float dist =
          exact_sqdist_warp_wide(a.qorig + (int64_t)pq[s] * d, a.rows + pslot[s] * d, d);
      if (lane == 0) plb[s] = dist;
    }
    __syncthreads();
    for (int i = tid; i < nk; i += NTH) {
      const int s = keep[i], q = pq[s];
      topk_insert_thread(a.topk + (int64_t)q * a.k_max, a.kq[q], make_key(plb[s], pid[s]));
    }
    if (a.collect && tid == 0) s_stat[4] += nk;
  };

  while (true) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    const int n_items = (int)imin64(*a.n_items, a.items_cap);
    if (item >= n_items || failed) break;
    const int4 it = a.items[item];
    const int64_t ch0 = a.chunk_off[it.x] + (int64_t)it.y * SEG_CHUNKS;
    const int64_t ch1 = imin64(a.chunk_off[it.x + 1], ch0 + SEG_CHUNKS);
    const int G = it.w;
    fq = 0u;
    fn = 0;
    for (int b = 0; b < NST; ++b) push_free(b);
    // Levels 0 .. PRE-1 of tile t+1 are staged while tile t runs (with four
    // stages also level 1: nearly every tile reaches it); deeper levels are
    // staged speculatively one level ahead.
    constexpr int PRE = NST - 2;
    const bool pre1 = PRE == 2 && L > 1;
    int cur = pop_free(), c1 = -1;  // this tile's level-0 and level-1 stages
    {
      const int nch0 = (int)imin64(NCH, ch1 - ch0);
      issue(cur, ch0, nch0, 0, (1u << nch0) - 1u);
      if (pre1) {
        c1 = pop_free();
        issue(c1, ch0, nch0, 1, (1u << nch0) - 1u);
      }
    }
    // levels 0 and 1's query slices stay in their buffers (by level parity)
    // unless a deeper level reuses one
    bool qok0 = true, qok1 = true;
    for (int g = tid; g < QB; g += NTH) {
      if (g < G) {
        int q = a.bucket[it.z + g];
        qid[g] = q;
        float4 inf = a.qinfo[q];
        qnq[g] = inf.x;
        qrq[g] = inf.y;
        qeq[g] = inf.z;
        qk[g] = a.kq[q];
      } else {
        qid[g] = -1;
        qnq[g] = qrq[g] = qeq[g] = 0.f;
        qk[g] = 0;
      }
    }
    __syncthreads();
    for (int e = tid; e < QB * (L + 1); e += NTH) {
      int g = e / (L + 1), l = e % (L + 1);
      qtl[e] = g < G ? a.eps * a.qtail[(int64_t)qid[g] * (L + 1) + l] : 0.f;
    }
    load_qslice(0, G);
    if (L > 1) load_qslice(1, G);
    cp_async_wait_all();
    TauRead tau_next = read_tau(tid, G);
    section(0);

    for (int64_t tile = ch0; tile < ch1; tile += NCH) {
      const int nch = (int)imin64(NCH, ch1 - tile);
      section(0);
      wait_stage(cur);
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
      section(1);  // the tile's first stage landed: a staging wait
      // the next tile's first levels go out before this tile's arithmetic
      const bool has_next = tile + NCH < ch1;
      int n0 = -1, n1 = -1;
      if (has_next) {
        const int nch_n = (int)imin64(NCH, ch1 - tile - NCH);
        n0 = pop_free();
        issue(n0, tile + NCH, nch_n, 0, (1u << nch_n) - 1u);
        if (pre1) {
          n1 = pop_free();
          issue(n1, tile + NCH, nch_n, 1, (1u << nch_n) - 1u);
        }
      }
      if (tid < QB) {
        // the global threshold, or the one this item's last tile reached
        float tau = tau_of(tau_next);
        if (tau >= 0.f && tile != ch0) tau = fminf(tau, qtau[tid]);
        qtau[tid] = tau;
        if (tau >= 0.f) set_query_terms(tid, tau);
        else qterm[tid] = make_float4(0.f, 0.f, -INFINITY, tau);
        if (has_next) tau_next = read_tau(tid, G);
      }
      // candidate terms by the highest threads (the lowest hold queries)
      for (int e = NTH - 1 - tid; e < CB; e += NTH) {
        if (e / CH < nch) {
          const float* meta = stage_x(cur) + (e / CH) * BR + (a.level_off[1] + 1) * CH + (e % CH);
          const float nx = meta[0], rx = sqrtf(nx), exv = meta[CH];
          cterm[e] = make_float4(
              exv, rx, 0.5f * (nx - gs * nx - exv * exv - kEvalSlack * (rx + exv) * (rx + exv)), nx);
          ids_s[e] = __float_as_int(meta[2 * CH]);
        } else {
          cterm[e] = make_float4(0.f, 0.f, 0.f, 0.f);
          ids_s[e] = -1;
        }
      }
      __syncthreads();

      uint32_t alive = 0;  // bit 4*ai + bi: pair (query tq + TQ ai, cand 4tc + bi)
#pragma unroll
      for (int ai = 0; ai < 4; ++ai)
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) {
          int g = tq + TQ * ai, e = 4 * tc + bi;
          if (g < G && qk[g] > 0 && ids_s[e] >= 0) alive |= 1u << (4 * ai + bi);
        }
      float p[4][4];
#pragma unroll
      for (int ai = 0; ai < 4; ++ai)
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) p[ai][bi] = 0.f;
      const int my_ch = (4 * tc) / CH, my_i = (4 * tc) % CH;
      bool completed = true;
      section(0);

      for (int l = 0; l < L; ++l) {
        // chunks with a live pair (a warp's pairs all lie in chunk my_ch)
        const bool wl = __any_sync(0xffffffffu, alive != 0);
        if ((tid & 31) == 0 && wl) atomicOr(&s_live[l & 1], 1u << my_ch);
        const int any = __syncthreads_or(alive != 0);
        if (!any) {
          completed = false;
          break;
        }
        const uint32_t live = s_live[l & 1];
        if (tid == 0) s_live[(l + 1) & 1] = 0u;  // last read at level l - 1
        const int w = a.level_off[l + 1] - a.level_off[l];
        // this level's query slice landed (issued one level ago) ...
        cp_async_wait_all();
        // ... and level l+1 goes out speculatively for the chunks live now
        // (unless it was staged with the tile)
        int nb = -1;
        if (l + 1 < L) {
          if (l == 0 && pre1) {
            nb = c1;
            c1 = -1;
          } else {
            nb = pop_free();
            issue(nb, tile, nch, l + 1, live);
          }
          if (l + 1 >= 2) {
            load_qslice(l + 1, G);
            if ((l + 1) & 1) qok1 = false;
            else qok0 = false;
          }
        }
        if (a.collect && tid == 0) s_stat[2] += 1;
        if (l > 0) wait_stage(cur);
        if (__syncthreads_or(failed)) {
          failed = true;
          completed = false;
          break;
        }
        section(1);
        const float* xb = stage_x(cur) + (size_t)my_ch * BR + my_i;  // this thread's candidates
        const int nalive = wl ? (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(alive)) : 0;
        if (wl && l > 0 && nalive <= 32) {
          // few live pairs in the warp: they are listed in lane order and each
          // lane computes one pair's level dot product, which its owner adds
          // (the same sequential sum over the level's dims as the dense path
          // below, so the partial products are identical)
          const int lane = tid & 31, wrp = tid >> 5, cnt = __popc(alive);
          int pre = cnt;
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, pre, off);
            if (lane >= off) pre += y;
          }
          const int base = pre - cnt;
          uint16_t* slot = s_pair[wrp];
          float* res = s_pdot[wrp];
          {
            uint32_t m = alive;
            for (int k = base; m; ++k) {
              slot[k] = (uint16_t)((lane << 4) | (__ffs(m) - 1));
              m &= m - 1;
            }
          }
          __syncwarp();
          if (lane < nalive) {
            const int code = slot[lane], src = code >> 4, bit = code & 15;
            const int stq = src % WQ + WQ * (wrp % NWQ), stc = src / WQ + WC * (wrp / NWQ);
            const float* qr = qslice(l) + (size_t)(stq + TQ * (bit >> 2)) * QS;
            const float* xc =
                stage_x(cur) + (size_t)((4 * stc) / CH) * BR + (4 * stc) % CH + (bit & 3);
            float dt = 0.f;
            for (int j = 0; j < w; ++j) dt = fmaf(qr[j], xc[j * CH], dt);
            res[lane] = dt;
          }
          __syncwarp();
#pragma unroll
          for (int ai = 0; ai < 4; ++ai)
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) {
              const int b = 4 * ai + bi;
              if (alive & (1u << b)) p[ai][bi] += res[base + __popc(alive & ((1u << b) - 1u))];
            }
        } else if (wl) {
          float acc[4][4];
#pragma unroll
          for (int ai = 0; ai < 4; ++ai)
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) acc[ai][bi] = 0.f;
          const float* qb = qslice(l) + tq * QS;
          const int w4 = w & ~3;
#pragma unroll 2
          for (int j = 0; j < w4; j += 4) {
            float qv[4][4], xv[4][4];
#pragma unroll
            for (int ai = 0; ai < 4; ++ai) {
              const float4 t = *reinterpret_cast<const float4*>(qb + ai * TQ * QS + j);
              qv[ai][0] = t.x;
              qv[ai][1] = t.y;
              qv[ai][2] = t.z;
              qv[ai][3] = t.w;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 t = *reinterpret_cast<const float4*>(xb + (j + u) * CH);
              xv[u][0] = t.x;
              xv[u][1] = t.y;
              xv[u][2] = t.z;
              xv[u][3] = t.w;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int ai = 0; ai < 4; ++ai)
#pragma unroll
                for (int bi = 0; bi < 4; ++bi) acc[ai][bi] = fmaf(qv[ai][u], xv[u][bi], acc[ai][bi]);
          }
          for (int j = w4; j < w; ++j) {
            const float4 t = *reinterpret_cast<const float4*>(xb + j * CH);
            const float xx[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int ai = 0; ai < 4; ++ai) {
              const float qq = qb[ai * TQ * QS + j];
#pragma unroll
              for (int bi = 0; bi < 4; ++bi) acc[ai][bi] = fmaf(qq, xx[bi], acc[ai][bi]);
            }
          }
#pragma unroll
          for (int ai = 0; ai < 4; ++ai)
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) p[ai][bi] += acc[ai][bi];
        }
        if (wl) {
          if (a.collect) {
            const unsigned np = __reduce_add_sync(__activemask(), (unsigned)__popc(alive));
            if ((threadIdx.x & 31) == __ffs(__activemask()) - 1) {
              atomicAdd(&s_stat[0], (unsigned long long)np);
              atomicAdd(&s_stat[1], (unsigned long long)np * w);
            }
          }
          // bound update and pruning (Eq. 3 with rounding margins)
          if ((a.prune && l % a.test_every == 0) || l == L - 1) {
            const float4 sx = *reinterpret_cast<const float4*>(xb + w * CH);
            const float sxv[4] = {sx.x, sx.y, sx.z, sx.w};
            float4 ct[4];
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) ct[bi] = cterm[4 * tc + bi];
#pragma unroll
            for (int ai = 0; ai < 4; ++ai) {
              const int g = tq + TQ * ai;
              const float4 t = qterm[g];
              const float sq = qtl[g * (L + 1) + l + 1];
#pragma unroll
              for (int bi = 0; bi < 4; ++bi) {
                const float P = fmaf(t.x, ct[bi].x, fmaf(t.y, ct[bi].y, fmaf(sq, sxv[bi], p[ai][bi])));
                if (P < t.z + ct[bi].z) alive &= ~(1u << (4 * ai + bi));
              }
            }
          }
        }
        __syncthreads();  // the stage and the query slice are refilled next
        section(l == 0 ? 2 : 3);
        if (l + 1 < L) {  // the next level's stage becomes current
          push_free(cur);
          cur = nb;
        }
      }
      if (failed) break;
      cp_async_wait_all();  // an unused speculative query slice
      // The k-th smallest upper bound of the tile tightens each query's
      // threshold before re-ranking (at the last level UB ~ LB ~ exact, so
      // only ~k pairs per query survive even while the running top-k is
      // still empty).  The last level's stage is free: it is the scratch.
      const int done = __syncthreads_or(completed && alive != 0);
      // every thread's copies have landed: levels 0 and 1's query slices
      // can be restaged for the next tile
      if (has_next && !qok0) {
        load_qslice(0, G);
        qok0 = true;
      }
      if (has_next && !qok1) {
        load_qslice(1, G);
        qok1 = true;
      }
      if (done) {
        float* ub = stage_x(cur);  // [QB][CB]
        for (int e = tid; e < QB * CB; e += NTH) ub[e] = INFINITY;
        __syncthreads();
        if (completed) {
#pragma unroll
          for (int ai = 0; ai < 4; ++ai) {
            const int g = tq + TQ * ai;
            const float nq = qnq[g], rq = qrq[g], eq = qeq[g];
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) {
              if (!(alive & (1u << (4 * ai + bi)))) continue;
              const int e = 4 * tc + bi;
              const float4 ct = cterm[e];
              const float A = nq + ct.w - 2.f * p[ai][bi];
              const float S = rq + ct.y;
              const float ubs = fmaxf(A + gs * S * S, 0.f);
              const float r = __fadd_ru(__fsqrt_ru(ubs), eq + ct.x);
              ub[g * CB + e] = __fmul_ru(__fmul_ru(r, r), a.ub_scale);
            }
          }
        }
        __syncthreads();
        // k candidates with upper bounds <= t: t bounds the query's k-th
        // distance, so it is published for every later tile of the query
        for (int g = warp; g < G; g += NW) {
          const float t = warp_kth_smallest(ub + g * CB, CB, qk[g]);
          if (lane == 0 && qk[g] > 0 && t < qtau[g]) {
            qtau[g] = t;
            atomicMin(reinterpret_cast<unsigned int*>(a.tau_seed) + qid[g], __float_as_uint(t));
          }
        }
        __syncthreads();
        for (int g = tid; g < G; g += NTH)
          if (qk[g] > 0) set_query_terms(g, qtau[g]);
        __syncthreads();
        if (completed) {
          float4 ct[4];
#pragma unroll
          for (int bi = 0; bi < 4; ++bi) ct[bi] = cterm[4 * tc + bi];
#pragma unroll
          for (int ai = 0; ai < 4; ++ai) {
            const float4 t = qterm[tq + TQ * ai];
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) {
              const float P = fmaf(t.x, ct[bi].x, fmaf(t.y, ct[bi].y, p[ai][bi]));
              if (P < t.z + ct[bi].z) alive &= ~(1u << (4 * ai + bi));
            }
          }
        }
      }
      section(4);
      // survivors of all L levels join the deferred list; a full list is
      // checked against the thresholds of the moment and the rest re-ranked
      // by all warps at once.
      // The list [QB*CB] is kept in the tile's last stage, read by now (a
      // tile with survivors completed every level: no copy is landing).
      uint16_t* surv = reinterpret_cast<uint16_t*>(stage_x(cur));
      if (completed && alive) {
#pragma unroll
        for (int ai = 0; ai < 4; ++ai)
#pragma unroll
          for (int bi = 0; bi < 4; ++bi)
            if (alive & (1u << (4 * ai + bi))) {
              const int g = tq + TQ * ai, e = 4 * tc + bi;
              const int pos = atomicAdd(&s_nsurv, 1);
              surv[pos] = (uint16_t)((g << 8) | e);
              if (pos < FpSmem::kPend) {  // its Eq. 3 bounds (C = 0 at the end)
                const float4 ct = cterm[e];
                const float A = qnq[g] + ct.w - 2.f * p[ai][bi];
                const float S = qrq[g] + ct.y;
                const float r = sqrtf(fmaxf(A - gs * S * S, 0.f)) - (qeq[g] + ct.x);
                lbt[pos] = r > 0.f ? r * r * a.lb_scale : 0.f;
                const float ru = __fadd_ru(__fsqrt_ru(fmaxf(A + gs * S * S, 0.f)), qeq[g] + ct.x);
                ubt[pos] = __fmul_ru(__fmul_ru(ru, ru), a.ub_scale);
              }
            }
      }
      __syncthreads();
      const int ns = s_nsurv;
      int np = s_npend;
      if (np + ns > FpSmem::kPend) {  // the list is full: re-rank it (all warps)
        rerank_pending();
        np = 0;
        __syncthreads();
      }
      if (ns <= FpSmem::kPend) {
        for (int s = tid; s < ns; s += NTH) {
          const int g = surv[s] >> 8, e = surv[s] & 255;
          const int64_t slot = (tile + e / CH) * CH + (e % CH);
          pslot[np + s] = slot;
          pq[np + s] = qid[g];
          pid[np + s] = ids_s[e];
          plb[np + s] = lbt[s];
          pub[np + s] = ubt[s];
        }
      } else {  // too many to defer: re-rank them now
        for (int s = warp; s < ns; s += NW) {
          const int g = surv[s] >> 8, e = surv[s] & 255;
          const int64_t slot = (tile + e / CH) * CH + (e % CH);
          const float dist =
              exact_sqdist_warp_wide(a.qorig + (int64_t)qid[g] * d, a.rows + slot * d, d);
          topk_insert_warp(a.topk + (int64_t)qid[g] * a.k_max, qk[g], make_key(dist, ids_s[e]));
        }
        if (a.collect && tid == 0) s_stat[4] += ns;
      }
      // the stages go back to the free list (an unused speculative copy may
      // still be landing: it is drained when the stage is reused)
      push_free(cur);
      if (c1 >= 0) push_free(c1);
      // generic-proxy writes (scratch) precede later bulk-async refills
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        s_npend = ns <= FpSmem::kPend ? np + ns : np;
        s_nsurv = 0;
        s_live[0] = s_live[1] = 0u;
      }
      cur = n0;
      c1 = n1;
      section(5);
    }
    // nothing may stay in flight past the item
    for (int b = 0; b < NST; ++b) wait_stage(b);
    cp_async_wait_all();
    failed = __syncthreads_or(failed) != 0;
  }
  if (!failed) {  // the last deferred survivors
    __syncthreads();
    rerank_pending();
  }
  for (int b = 0; b < NST; ++b) wait_stage(b);  // bounded; after a failure too
  cp_async_wait_all();
  if (failed && tid == 0) atomicOr(a.err, kErrTimeout);
  __syncthreads();
  if (a.collect && tid == 0) {
    s_sec[6] = (unsigned long long)(clock64() - s_tkernel);
    s_sec[7] = 1;  // CTAs that ran
    for (int i = 0; i < 8; ++i) atomicAdd(&a.stats[8 + i], s_sec[i]);
    if (a.phase == 0)
      for (int i = 0; i < 8; ++i) atomicAdd(&a.stats[16 + i], s_sec[i]);
    atomicAdd(&a.stats[0], s_stat[0]);
    atomicAdd(&a.stats[a.phase == 0 ? 6 : 7], s_stat[1]);
    atomicAdd(&a.stats[1], s_stat[2]);
    atomicAdd(&a.stats[2], s_stat[3]);
    atomicAdd(&a.stats[3], s_stat[4]);
  }
}

__global__ void decode_kernel(int64_t nq, int k_max, const int32_t* __restrict__ kq,
                              const unsigned long long* __restrict__ topk,
                              int64_t* __restrict__ out_ids, float* __restrict__ out_d) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * k_max) return;
  int64_t qi = e / k_max;
  int j = (int)(e % k_max);
  unsigned long long key = j < kq[qi] ? topk[e] : kEmptyKey;
  if (key == kEmptyKey) {
    out_ids[e] = -1;
    out_d[e] = INFINITY;
  } else {
    out_ids[e] = key_id(key);
    out_d[e] = key_dist(key);
  }
}

// Pairs in all candidate sets (stats): sum over (q, r < nprobe_q) of list sizes.
// Pairs of all probes into out[0]; those of phase A (rank 0, when the search
// runs two phases) into out_a[0].
__global__ void pair_count_kernel(int64_t nq, const int32_t* __restrict__ probes, int stride,
                                  const int32_t* __restrict__ npq, const int32_t* __restrict__ lsz,
                                  int two_phase, unsigned long long* __restrict__ out,
                                  unsigned long long* __restrict__ out_a) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0, va = 0;
  if (e < nq * stride) {
    int64_t qi = e / stride;
    int r = (int)(e % stride);
    if (r < npq[qi] && probes[e] >= 0) v = lsz[probes[e]];
    if (r == 0 && two_phase) va = v;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v += __shfl_xor_sync(0xffffffffu, v, off);
    va += __shfl_xor_sync(0xffffffffu, va, off);
  }
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
  if ((threadIdx.x & 31) == 0 && va) atomicAdd(out_a, va);
}

// Lets `kern` use all the dynamic shared memory the device allows next to its
// static shared memory.
cudaError_t allow_dynamic_smem(const void* kern) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

// FP32 verify tiles (QB queries x CB candidates, NTH threads).  Phase A
// (each query's nearest list: small groups) prefers wide candidate tiles,
// phase B (many queries per list) 64-query groups; narrower tiles serve wide
// levels whose stage buffers would not fit otherwise.
// Phase B's tiles are short (most die after a level or two), so levels 0
// and 1 of the next tile are staged ahead (four stages); phase A's run deep.
struct TileCfg {
  int QB, CB, NTH, NST;
};
constexpr TileCfg kTilesA[] = {{16, 256, 256, 3}, {16, 128, 128, 3}, {16, 64, 64, 3}};
constexpr TileCfg kTilesB[] = {{64, 64, 256, 4}, {32, 64, 128, 4}, {16, 64, 64, 3}};

template <int QB, int CB, int NTH, int NST>
cudaError_t tile_kernel_attrs(const void** kern, size_t* static_smem) {
  static PerDeviceOnce once;
  auto k = verify_fp32_kernel<QB, CB, NTH, NST>;
  cudaError_t err = once.run([&] {
    cudaError_t e = allow_dynamic_smem((const void*)k);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
  });
  cudaFuncAttributes fa;
  if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, k);
  *kern = (const void*)k;
  *static_smem = err == cudaSuccess ? fa.sharedSizeBytes : 0;
  return err;
}

cudaError_t tile_attrs(const TileCfg& c, const void** kern, size_t* static_smem) {
  if (c.QB == 16 && c.CB == 256) return tile_kernel_attrs<16, 256, 256, 3>(kern, static_smem);
  if (c.QB == 16 && c.CB == 128) return tile_kernel_attrs<16, 128, 128, 3>(kern, static_smem);
  if (c.QB == 64) return tile_kernel_attrs<64, 64, 256, 4>(kern, static_smem);
  if (c.QB == 32) return tile_kernel_attrs<32, 64, 128, 4>(kern, static_smem);
  return tile_kernel_attrs<16, 64, 64, 3>(kern, static_smem);
}

// First tile of `list` whose stage buffers fit (blocks per SM in *bps).
int pick_tile(const TileCfg* list, int n, int max_w, int L, TileCfg* out, int* bps) {
  int dev = 0, optin = 0, per_sm = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  PANO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PANO_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  for (int i = 0; i < n; ++i) {
    const void* k = nullptr;
    size_t ss = 0;
    PANO_CUDA(tile_attrs(list[i], &k, &ss));
    const size_t smem = FpSmem(list[i].QB, list[i].CB, max_w, L, list[i].NST).total;
    const long two = (long)per_sm / 2 - 1024 - (long)ss, one = (long)optin - (long)ss;
    const int b = (long)smem <= two ? 2 : ((long)smem <= one ? 1 : 0);
    if (b) {
      *out = list[i];
      *bps = b;
      return PANO_OK;
    }
  }
  return fail(PANO_EINVAL, "verify tile does not fit in shared memory");
}

// Launches the picked tile.  The grid is sized from the shared-memory plan,
// not from the occupancy API, whose answer follows the SM's current
// shared-memory carveout.
int launch_verify(const VerifyArgs& a, const TileCfg& c, int bps, cudaStream_t st) {
  const void* k = nullptr;
  size_t ss = 0;
  PANO_CUDA(tile_attrs(c, &k, &ss));
  int dev = 0, sms = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  PANO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = FpSmem(c.QB, c.CB, a.max_w, a.L, c.NST).total;
  void* args[] = {const_cast<VerifyArgs*>(&a)};
  PANO_CUDA(cudaLaunchKernel(k, dim3(sms * bps), dim3(c.NTH), args, smem, st));
  return PANO_OK;
}

// Carves one stream-ordered allocation into aligned pieces.
struct Carver {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

thread_local pano_search_stats t_stats;

// Pieces of one search's workspace (byte offsets into one allocation): the
// tiles of the FP32 verify phases, the work-item capacities and the carve.
struct SearchLayout {
  TileCfg tileA{TC_QG, 0, 0, 0}, tileB{TC_QG, 0, 0, 0};
  int bpsA = 0, bpsB = 0;
  int64_t capA = 0, capB = 0;
  size_t o_qt, o_qinfo, o_qtail, o_qn2, o_pd, o_pr, o_npq, o_kq, o_seed, o_cnt, o_fill, o_boff,
      o_ioff, o_tot, o_bucket, o_itA, o_itB, o_topk, o_err, o_stats;
  size_t total = 0;
};

int plan_layout(const pano_index& I, int64_t nq, int stride, int k_max, SearchLayout* out) {
  SearchLayout& y = *out;
  const int d = I.d, L = I.L, nlist = I.nlist;
  const bool tcpath = I.precision != PANO_FP32;
  if (!tcpath) {
    int r = pick_tile(kTilesA, 3, I.max_w, L, &y.tileA, &y.bpsA);
    if (!r) r = pick_tile(kTilesB, 3, I.max_w, L, &y.tileB, &y.bpsB);
    if (r) return r;
  }
  const int QBA = y.tileA.QB, QBB = y.tileB.QB;
  const int SEG = tcpath ? TC_SEG : SEG_CHUNKS;
  // work-item capacity: groups x segments, plus one partial group per list
  int64_t max_seg = 1, tot_seg = 0;
  for (int c = 0; c < nlist; ++c) {
    int64_t nch = I.list_chunk_off[c + 1] - I.list_chunk_off[c];
    int64_t s = (nch + SEG - 1) / SEG;
    max_seg = std::max(max_seg, s);
    tot_seg += s;
  }
  y.capA = ((nq + QBA - 1) / QBA) * max_seg + tot_seg;
  y.capB = ((nq * stride + QBB - 1) / QBB) * max_seg + tot_seg;
  Carver cv;
  y.o_qt = cv.take<float>((size_t)nq * d);
  y.o_qinfo = cv.take<float4>(nq);
  y.o_qtail = cv.take<float>((size_t)nq * (L + 1));
  y.o_qn2 = cv.take<float>(nq);
  y.o_pd = nlist > 1 ? cv.take<float>((size_t)nq * nlist) : 0;
  y.o_pr = cv.take<int32_t>((size_t)nq * stride);
  y.o_npq = cv.take<int32_t>(nq);
  y.o_kq = cv.take<int32_t>(nq);
  y.o_seed = cv.take<float>(nq);
  y.o_cnt = cv.take<int>(2 * (size_t)nlist);
  y.o_fill = cv.take<int>(2 * (size_t)nlist);
  y.o_boff = cv.take<int>(2 * (size_t)(nlist + 1));
  y.o_ioff = cv.take<int>(2 * (size_t)(nlist + 1));
  y.o_tot = cv.take<int>(8);
  y.o_bucket = cv.take<int32_t>((size_t)nq * stride);
  y.o_itA = cv.take<int4>(y.capA);
  y.o_itB = cv.take<int4>(std::max<int64_t>(y.capB, 1));
  y.o_topk = cv.take<unsigned long long>((size_t)nq * k_max);
  y.o_err = cv.take<int>(4);
  y.o_stats = cv.take<unsigned long long>(kStatWords);
  y.total = cv.off;
  return PANO_OK;
}


}  // namespace

int search(const pano_index* ip, const float* queries, int64_t nq, const int32_t* nprobe,
           int32_t nprobe_scalar, const int32_t* k, int32_t k_scalar, int32_t k_max,
           int64_t* out_ids, float* out_dists, cudaStream_t st, const pano_search_opts* opts,
           void* ext_ws, size_t ext_cap, int* err_host) {
  PANO_CHECK(ip, PANO_EINVAL, "null index");
  const pano_index& I = *ip;
  PANO_CHECK(!I.flat, PANO_EINVAL, "a flat index is searched with panorama_refine");
  PANO_CHECK(!I.pq_M, PANO_EINVAL, "an IVFPQ index is searched with panorama_search_pq");
  PANO_CHECK(nq >= 0 && nq < (1LL << 31), PANO_EINVAL, "nq out of range");
  PANO_CHECK(nq == 0 || (queries && out_ids && out_dists), PANO_EINVAL, "null argument");
  PANO_CHECK(k_max >= 1 && k_max <= 1024, PANO_EINVAL, "k_max must be in [1, 1024]");
  if (!nprobe)
    PANO_CHECK(nprobe_scalar >= 1 && nprobe_scalar <= I.nlist, PANO_EINVAL,
               "nprobe must be in [1, nlist]");
  if (!k) PANO_CHECK(k_scalar >= 0 && k_scalar <= k_max, PANO_EINVAL, "k must be in [0, k_max]");
  const int mode = opts ? opts->mode : 0;
  // Eq. 4: LB_eps = A - 2 eps C (0 and 1 mean the exact Eq. 3)
  const float eps = (opts && opts->epsilon > 0.f && opts->epsilon < 1.f) ? opts->epsilon : 1.f;
  // bound-test schedule: 0 = the storage format's default (FP32 every level;
  // tensor-core formats every kTcTestEvery-th level plus nearly dead chunks)
  const int te_opt = (opts && opts->test_every > 0) ? opts->test_every : 0;
  const int test_every =
      te_opt > 0 ? te_opt : (I.precision == PANO_FP32 ? 1 : kTcTestEvery);
  const bool timing = opts ? opts->collect_timing != 0 : false;
  const bool sync = (opts ? opts->synchronize != 0 : true) || timing;
  const bool collect = opts ? opts->collect_stats != 0 : false;
  std::memset(&t_stats, 0, sizeof(t_stats));
  t_stats.n_queries = nq;
  if (nq == 0) return PANO_OK;
  int cur = 0;
  PANO_CUDA(cudaGetDevice(&cur));
  PANO_CHECK(cur == I.device, PANO_EINVAL, "current device differs from the index's device");

  const int d = I.d, L = I.L, nlist = I.nlist;
  const int np_cap = nprobe ? ((nprobe_scalar >= 1) ? std::min(nprobe_scalar, nlist) : nlist)
                            : nprobe_scalar;
  const int stride = np_cap;
  const bool tcpath = I.precision != PANO_FP32;
  SearchLayout lay;
  if (int r = plan_layout(I, nq, stride, k_max, &lay)) return r;
  const TileCfg tileA = lay.tileA, tileB = lay.tileB;
  const int bpsA = lay.bpsA, bpsB = lay.bpsB;
  const int QBA = tileA.QB, QBB = tileB.QB;
  const int SEG = tcpath ? TC_SEG : SEG_CHUNKS;
  const int64_t capA = lay.capA, capB = lay.capB;
  const size_t o_qt = lay.o_qt, o_qinfo = lay.o_qinfo, o_qtail = lay.o_qtail, o_qn2 = lay.o_qn2,
               o_pd = lay.o_pd, o_pr = lay.o_pr, o_npq = lay.o_npq, o_kq = lay.o_kq,
               o_seed = lay.o_seed, o_cnt = lay.o_cnt, o_fill = lay.o_fill, o_boff = lay.o_boff,
               o_ioff = lay.o_ioff, o_tot = lay.o_tot, o_bucket = lay.o_bucket, o_itA = lay.o_itA,
               o_itB = lay.o_itB, o_topk = lay.o_topk, o_err = lay.o_err, o_stats = lay.o_stats;
  Carver cv;
  cv.off = lay.total;
  void* ws = ext_ws;
  if (ext_ws) {
    PANO_CHECK(cv.off <= ext_cap, PANO_EINVAL,
               "search workspace of " + std::to_string(cv.off) + " bytes exceeds the " +
                   std::to_string(ext_cap) + "-byte static scratch");
  } else {
    PANO_CUDA(cudaMallocAsync(&ws, cv.off, st));
  }
  char* W = static_cast<char*>(ws);
  auto P = [&](size_t o) { return (void*)(W + o); };
  float* qt = (float*)P(o_qt);
  float4* qinfo = (float4*)P(o_qinfo);
  float* qtail = (float*)P(o_qtail);
  float* qn2 = (float*)P(o_qn2);
  int32_t* probes = (int32_t*)P(o_pr);
  int32_t* npq = (int32_t*)P(o_npq);
  int32_t* kq = (int32_t*)P(o_kq);
  float* tau_seed = (float*)P(o_seed);
  int* cnt = (int*)P(o_cnt);
  int* fillc = (int*)P(o_fill);
  int* boff = (int*)P(o_boff);
  int* ioff = (int*)P(o_ioff);
  int* tot = (int*)P(o_tot);
  int32_t* bucket = (int32_t*)P(o_bucket);
  int4* itA = (int4*)P(o_itA);
  int4* itB = (int4*)P(o_itB);
  unsigned long long* topk = (unsigned long long*)P(o_topk);
  int* err = (int*)P(o_err);
  unsigned long long* stats = (unsigned long long*)P(o_stats);
  int rc = PANO_OK;
  cudaEvent_t ev[7] = {};
  if (timing)
    for (auto& e : ev) PANO_CUDA(cudaEventCreate(&e));
  auto mark = [&](int i) {
    if (timing) cudaEventRecord(ev[i], st);
  };
  auto body = [&]() -> int {
    PANO_CUDA(cudaMemsetAsync(cnt, 0, 2 * (size_t)nlist * 4, st));
    PANO_CUDA(cudaMemsetAsync(fillc, 0, 2 * (size_t)nlist * 4, st));
    PANO_CUDA(cudaMemsetAsync(tot, 0, 8 * 4, st));  // [4..5] verify counters
    PANO_CUDA(cudaMemsetAsync(topk, 0xff, (size_t)nq * k_max * 8, st));
    PANO_CUDA(cudaMemsetAsync(err, 0, 16, st));
    PANO_CUDA(cudaMemsetAsync(stats, 0, kStatWords * 8, st));
    prep_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(nq, nprobe, nprobe_scalar, np_cap, k,
                                                              k_scalar, k_max, npq, kq, err);
    PANO_CUDA(cudaGetLastError());
    // a1
    mark(0);
    PANO_CUDA(gemm_nt(kStore, (int)nq, d, d, queries, d, I.mu32.as<float>(), I.T32.as<float>(), d,
                      qt, d, nullptr, nullptr, st));
    float c_trans_up = (float)I.c_trans;  // rounded up: the e_q bound stays an upper bound
    if ((double)c_trans_up < I.c_trans) c_trans_up = std::nextafter(c_trans_up, INFINITY);
    query_norms_kernel<<<(unsigned)((nq + kNormRows - 1) / kNormRows), kNormRows * 32,
                         d <= kNormMaxD ? (size_t)kNormRows * d * 4 : 0, st>>>(
        queries, qt, nq, d, L, I.level_off_d.as<int32_t>(), I.mu32.as<float>(), c_trans_up, qinfo,
        qtail, qn2);
    PANO_CUDA(cudaGetLastError());
    // a2
    mark(1);
    if (nlist > 1) {
      float* pd = (float*)P(o_pd);
      // query x centroid distances: tensor cores (bf16 hi/lo) where d allows,
      // with the wider error band they need; the band is re-scored exactly
      float gerr;
      if (probe_tc_supported(d)) {
        int r = launch_probe_tc(queries, nq, I.cent.as<float>(), nlist, d, qn2,
                                I.cent_n2.as<float>(), pd, err, st);
        if (r) return r;
        gerr = (float)probe_tc_gerr(d);
        if ((double)gerr < probe_tc_gerr(d)) gerr = std::nextafter(gerr, INFINITY);
      } else {
        PANO_CUDA(gemm_nt(kDist, (int)nq, nlist, d, queries, d, nullptr, I.cent.as<float>(), d,
                          pd, nlist, qn2, I.cent_n2.as<float>(), st));
        gerr = (float)(2.0 * gamma_n(gemm_rounds(d) + 4));
      }
      const float cmax = I.cmax;
      size_t psm = (size_t)nlist * 4;
      PANO_CUDA(allow_dynamic_smem((const void*)probe_select_kernel));
      probe_select_kernel<<<(unsigned)nq, NT, psm, st>>>(pd, nlist, queries, I.cent.as<float>(), d,
                                                         qn2, cmax, gerr, npq, stride, probes, err,
                                                         0);
      PANO_CUDA(cudaGetLastError());
    } else {
      PANO_CUDA(cudaMemsetAsync(probes, 0, (size_t)nq * stride * 4, st));
    }
    // a3 (and the Alg. 1 warm start of the threshold)
    mark(2);
    const int64_t ne = nq * stride;
    // Phase A (each query's nearest list, verified first for a tight
    // threshold) pays off unless its query groups are nearly empty: on the
    // tensor-core path a group fills MMA columns, so fewer than 8 queries per
    // list on average make one pass the better choice.
    const int sp = opts ? opts->single_phase : 0;
    const bool one_pass = sp == 1 || (sp == 0 && tcpath && nq < 8 * (int64_t)nlist);
    const int first_rank_b = one_pass ? 0 : 1;
    inv_count_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(nq, probes, stride, npq, cnt,
                                                                   nlist, first_rank_b);
    inv_scan_kernel<<<1, 1024, 0, st>>>(cnt, nlist, I.chunk_off_d.as<int64_t>(), SEG, QBA, QBB,
                                        boff, ioff, tot);
    inv_scatter_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
        nq, probes, stride, npq, boff, tot, fillc, nlist, first_rank_b, bucket);
    PANO_CUDA(cudaGetLastError());
    inv_emit_kernel<<<1024, 256, 0, st>>>(0, cnt, nlist, I.chunk_off_d.as<int64_t>(), SEG, QBA,
                                          boff, ioff, tot, capA, itA, err);
    inv_emit_kernel<<<1024, 256, 0, st>>>(1, cnt, nlist, I.chunk_off_d.as<int64_t>(), SEG, QBB,
                                          boff, ioff, tot, capB, itB, err);
    PANO_CUDA(cudaGetLastError());
    // the warm-start seeds, in phase A's order when there is a phase A (its
    // bucket lists every query once, grouped by nearest list, so the CTAs
    // that read one list's first rows run together and share them in L2)
    const double seed_m = (d + 127) / 128 + 8;
    const double seed_sl = 1.0 + 2.0 * (seed_m + 3.0) * kU32;
    float seed_slack = (float)seed_sl;
    if ((double)seed_slack < seed_sl) seed_slack = std::nextafter(seed_slack, INFINITY);
    if (!one_pass && d <= 1024 && (d & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(queries) & 15) == 0) {
      const int nsub = (QBA + kSeedSub - 1) / kSeedSub;
      const size_t gsm = (size_t)kSeedSub * d * 4 + (size_t)kSeedSub * kSeedMax * 4;
      PANO_CUDA(allow_dynamic_smem((const void*)seed_group_kernel));
      seed_group_kernel<<<(unsigned)(capA * nsub), kSeedWarps * 32, gsm, st>>>(
          queries, d, itA, tot + 1, capA, nsub, bucket, I.chunk_off_d.as<int64_t>(),
          I.list_size_d.as<int32_t>(), I.chunk, I.rows.as<float>(), kq, seed_slack, tau_seed,
          I.ids.as<int32_t>(), eps < 1.f ? topk : nullptr, k_max);
    } else {
      seed_tau_kernel<<<(unsigned)nq, kSeedWarps * 32, (size_t)d * 4, st>>>(
          queries, d, probes, stride, I.chunk_off_d.as<int64_t>(), I.list_size_d.as<int32_t>(),
          I.chunk, I.rows.as<float>(), kq, one_pass ? nullptr : bucket, seed_slack, tau_seed,
          I.ids.as<int32_t>(), eps < 1.f ? topk : nullptr, k_max);
    }
    PANO_CUDA(cudaGetLastError());
    // a4-a10
    if (tcpath) {
      VerifyTCArgs ta;
      std::memset(&ta, 0, sizeof(ta));
      ta.slices = I.slices.as<uint8_t>();
      ta.tails = I.tails.as<float>();
      ta.xn2 = I.xn2.as<float>();
      ta.ex = I.ex.as<float>();
      ta.ids = I.ids.as<int32_t>();
      ta.fp8 = I.precision == PANO_FP8 ? 1 : 0;
      ta.xscale = ta.fp8 ? I.xscale.as<float>() : nullptr;
      ta.rows = I.rows.as<float>();
      ta.chunk_off = I.chunk_off_d.as<int64_t>();
      ta.qt = qt;
      ta.qorig = queries;
      ta.qinfo = qinfo;
      ta.qtail = qtail;
      ta.kq = kq;
      ta.tau_seed = tau_seed;
      ta.topk = topk;
      ta.err = err;
      ta.stats = stats;
      ta.d = d;
      ta.L = L;
      ta.max_w = I.max_w;
      ta.k_max = k_max;
      // p error: bf16 hi/lo query split (2^-16 |q~_j| per term) plus the
      // tensor-core accumulation (2^-20 of the running sum of |products| per
      // MMA instruction, 2 d / 16 instructions); FP32 evaluation of the
      // remaining terms: gamma_{L+8}; factor 2 of safety on the last two.
      // BF16: the query's hi/lo split (2^-16 of |q|), d/8 MMAs at 2^-20 of
      // the running sum of |products| each, the FP32 epilogue.  FP8: the
      // three-term E4M3 split (2^-12 of |q| doubled; its underflow is a
      // separate per-group term), 3d/32 MMAs on products of at most
      // (1 + 2^-4 + 2^-8) |x^| |q|, one more rounding for the row factor.
      ta.gslack = ta.fp8 ? (float)(std::ldexp(1.0, -11) +
                                   (3.0 * d / 32.0 + 1.0) * 1.1 * std::ldexp(1.0, -20) +
                                   2.0 * gamma_n(L + 9))
                         : (float)(std::ldexp(1.0, -16) + (d / 8.0) * std::ldexp(1.0, -20) +
                                   2.0 * gamma_n(L + 8));
      ta.lb_scale = (float)((1.0 - 8.0 * kU32) / (1.0 + I.eta));
      {
        // inv is the double nearest 1 / lb_scale: a float at or below it
        // moves up one step, so f exceeds the exact reciprocal
        const double inv = 1.0 / (double)ta.lb_scale;
        float f = (float)inv;
        if ((double)f <= inv) f = std::nextafter(f, INFINITY);
        ta.inv_lb_up = f;
      }
      ta.ub_scale = (float)((1.0 + 8.0 * kU32) / (1.0 - I.eta) * (1.0 + 1e-7));
      ta.prune = mode == 0 ? 1 : 0;
      ta.test_every = test_every;
      ta.eps = eps;
      ta.collect = collect ? 1 : 0;
      for (int l = 0; l <= L; ++l) ta.level_off[l] = I.offs[l];
      ta.bucket = bucket;
      mark(3);
      ta.items = itA;
      ta.n_items = tot + 1;
      ta.counter = tot + 4;
      ta.items_cap = capA;
      ta.phase = 0;
      int r = one_pass ? PANO_OK : launch_verify_tc(ta, st);  // one pass: phase A is empty
      if (r) return r;
      mark(4);
      ta.items = itB;
      ta.n_items = tot + 3;
      ta.counter = tot + 5;
      ta.items_cap = capB;
      ta.phase = 1;
      r = launch_verify_tc(ta, st);
      if (r) return r;
    } else {
    VerifyArgs va;
    std::memset(&va, 0, sizeof(va));
    va.slices = I.slices.as<float>();
    va.rows = I.rows.as<float>();
    va.chunk_off = I.chunk_off_d.as<int64_t>();
    va.qt = qt;
    va.qorig = queries;
    va.qinfo = qinfo;
    va.qtail = qtail;
    va.kq = kq;
    va.tau_seed = tau_seed;
    va.topk = topk;
    va.err = err;
    va.stats = stats;
    va.d = d;
    va.L = L;
    va.max_w = I.max_w;
    va.k_max = k_max;
    va.gslack = (float)(2.0 * gamma_n(I.max_w + L + 8));
    va.lb_scale = (float)((1.0 - 8.0 * kU32) / (1.0 + I.eta));
    {
      const double inv = 1.0 / (double)va.lb_scale;
      float f = (float)inv;
      if ((double)f <= inv) f = std::nextafter(f, INFINITY);
      va.inv_lb_up = f;
    }
    va.ub_scale = (float)((1.0 + 8.0 * kU32) / (1.0 - I.eta) * (1.0 + 1e-7));
    va.prune = mode == 0 ? 1 : 0;
    va.test_every = test_every;
    va.eps = eps;
    va.collect = collect ? 1 : 0;
    for (int l = 0; l <= L; ++l) va.level_off[l] = I.offs[l];
    for (int l = 0; l < L; ++l) va.row_off[l] = I.fp32_row_off(l);
    va.chunk_rows = I.fp32_chunk_rows();
    va.bucket = bucket;
    // phase A
    mark(3);
    va.items = itA;
    va.n_items = tot + 1;
    va.counter = tot + 4;
    va.items_cap = capA;
    va.phase = 0;
    int r = one_pass ? PANO_OK : launch_verify(va, tileA, bpsA, st);  // one pass: phase A is empty
    if (r) return r;
    // phase B
    mark(4);
    va.items = itB;
    va.n_items = tot + 3;
    va.counter = tot + 5;
    va.items_cap = capB;
    va.phase = 1;
    r = launch_verify(va, tileB, bpsB, st);
    if (r) return r;
    }
    mark(5);
    const int64_t no = nq * k_max;
    decode_kernel<<<(unsigned)((no + 255) / 256), 256, 0, st>>>(nq, k_max, kq, topk, out_ids,
                                                                out_dists);
    PANO_CUDA(cudaGetLastError());
    mark(6);
    // the device error word for a caller that does not synchronize (it maps
    // the word to a status once the stream has passed this copy)
    if (err_host) PANO_CUDA(cudaMemcpyAsync(err_host, err, 4, cudaMemcpyDeviceToHost, st));
    if (collect) {
      pair_count_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
          nq, probes, stride, npq, I.list_size_d.as<int32_t>(), one_pass ? 0 : 1, stats + 4,
          stats + 24);
      PANO_CUDA(cudaGetLastError());
    }
    if (sync || collect) {
      int herr[4];
      unsigned long long hst[kStatWords];
      int htot[8];
      PANO_CUDA(cudaMemcpyAsync(herr, err, 16, cudaMemcpyDeviceToHost, st));
      PANO_CUDA(cudaMemcpyAsync(hst, stats, kStatWords * 8, cudaMemcpyDeviceToHost, st));
      PANO_CUDA(cudaMemcpyAsync(htot, tot, 32, cudaMemcpyDeviceToHost, st));
      PANO_CUDA(cudaStreamSynchronize(st));
      t_stats.pair_levels = (int64_t)hst[0];
      t_stats.tile_levels = (int64_t)hst[1];
      t_stats.slice_bytes = (int64_t)hst[2];
      t_stats.reranked = (int64_t)hst[3];
      t_stats.pairs = (int64_t)hst[4];
      t_stats.work_items = (int64_t)htot[1] + htot[3];
      t_stats.device_error = herr[0];
      t_stats.dims_scanned = (int64_t)(hst[5] + hst[6] + hst[7]);
      t_stats.dims_scanned_a = (int64_t)hst[6];
      for (int i = 0; i < 8; ++i) t_stats.section_cycles[i] = (int64_t)hst[8 + i];
      for (int i = 0; i < 8; ++i) t_stats.section_cycles_a[i] = (int64_t)hst[16 + i];
      t_stats.pairs_a = (int64_t)hst[24];
      t_stats.live_row_bytes = (int64_t)hst[25];
      if (timing)
        for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&t_stats.stage_ms[i], ev[i], ev[i + 1]);
      if (herr[0] & kErrTimeout) return fail(PANO_ETIMEOUT, "a device-side wait timed out");
    }
    return PANO_OK;
  };
  rc = body();
  if (timing)
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  cudaError_t fe = ext_ws ? cudaSuccess : cudaFreeAsync(ws, st);
  if (rc == PANO_OK && fe != cudaSuccess) return cuda_fail(fe, "cudaFreeAsync");
  return rc;
}

int search_workspace_bytes(const pano_index* ip, int64_t nq, int32_t stride, int32_t k_max,
                           size_t* out) {
  PANO_CHECK(ip && out && nq >= 0 && stride >= 1 && k_max >= 1, PANO_EINVAL, "bad argument");
  SearchLayout lay;
  if (int r = plan_layout(*ip, nq, std::min(stride, ip->nlist), k_max, &lay)) return r;
  *out = lay.total;
  return PANO_OK;
}

int status_of_device_error(int word) {
  if (word & kErrTimeout) return PANO_ETIMEOUT;
  if (word & kErrBadInput) return PANO_EINVAL;
  return PANO_OK;
}

int probe_only(const pano_index* ip, const float* queries, int64_t nq, int32_t nprobe,
               int32_t* out, cudaStream_t st) {
  PANO_CHECK(ip, PANO_EINVAL, "null index");
  const pano_index& I = *ip;
  PANO_CHECK(nprobe >= 1 && nprobe <= I.nlist, PANO_EINVAL, "nprobe must be in [1, nlist]");
  PANO_CHECK(nq >= 0 && nq < (1LL << 31), PANO_EINVAL, "nq out of range");
  PANO_CHECK(nq == 0 || (queries && out), PANO_EINVAL, "null argument");
  if (nq == 0) return PANO_OK;
  const int d = I.d, nlist = I.nlist;
  if (nlist == 1) {
    PANO_CUDA(cudaMemsetAsync(out, 0, nq * 4, st));
    return PANO_OK;
  }
  Carver cv;
  size_t o_pd = cv.take<float>((size_t)nq * nlist);
  size_t o_qn = cv.take<float>(nq);
  size_t o_np = cv.take<int32_t>(2 * nq);
  size_t o_err = cv.take<int>(4);
  void* ws = nullptr;
  PANO_CUDA(cudaMallocAsync(&ws, cv.off, st));
  char* W = (char*)ws;
  float* pd = (float*)(W + o_pd);
  float* qn2 = (float*)(W + o_qn);
  int32_t* npq = (int32_t*)(W + o_np);
  int* err = (int*)(W + o_err);
  auto body = [&]() -> int {
    PANO_CUDA(cudaMemsetAsync(err, 0, 16, st));
    prep_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(nq, nullptr, nprobe, nlist, nullptr,
                                                              0, 1, npq, npq + nq, err);
    row_sqnorm_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(queries, nq, d, qn2);
    float gerr;
    if (probe_tc_supported(d)) {
      int r = launch_probe_tc(queries, nq, I.cent.as<float>(), nlist, d, qn2,
                              I.cent_n2.as<float>(), pd, err, st);
      if (r) return r;
      gerr = (float)probe_tc_gerr(d);
      if ((double)gerr < probe_tc_gerr(d)) gerr = std::nextafter(gerr, INFINITY);
    } else {
      PANO_CUDA(gemm_nt(kDist, (int)nq, nlist, d, queries, d, nullptr, I.cent.as<float>(), d,
                        pd, nlist, qn2, I.cent_n2.as<float>(), st));
      gerr = (float)(2.0 * gamma_n(gemm_rounds(d) + 4));
    }
    size_t psm = (size_t)nlist * 4;
    PANO_CUDA(allow_dynamic_smem((const void*)probe_select_kernel));
    probe_select_kernel<<<(unsigned)nq, NT, psm, st>>>(pd, nlist, queries, I.cent.as<float>(), d,
                                                       qn2, I.cmax, gerr, npq, nprobe, out, err, 1);
    PANO_CUDA(cudaGetLastError());
    PANO_CUDA(cudaStreamSynchronize(st));
    return PANO_OK;
  };
  int rc = body();
  cudaFreeAsync(ws, st);
  return rc;
}

const pano_search_stats& last_stats() { return t_stats; }
pano_search_stats& stats_slot() { return t_stats; }

// a1 for callers outside the IVF search (the refine path): q~ = T~(q - mu~),
// then norms, rounded-up tails and e_q (query_norms_kernel).
int transform_queries(const pano_index& I, const float* queries, int64_t nq, float* qt,
                      float4* qinfo, float* qtail, float* qn2, cudaStream_t st) {
  const int d = I.d, L = I.L;
  if (nq == 0) return PANO_OK;
  PANO_CUDA(gemm_nt(kStore, (int)nq, d, d, queries, d, I.mu32.as<float>(), I.T32.as<float>(), d,
                    qt, d, nullptr, nullptr, st));
  float c_trans_up = (float)I.c_trans;
  if ((double)c_trans_up < I.c_trans) c_trans_up = std::nextafter(c_trans_up, INFINITY);
  query_norms_kernel<<<(unsigned)((nq + kNormRows - 1) / kNormRows), kNormRows * 32,
                       d <= kNormMaxD ? (size_t)kNormRows * d * 4 : 0, st>>>(
      queries, qt, nq, d, L, I.level_off_d.as<int32_t>(), I.mu32.as<float>(), c_trans_up, qinfo,
      qtail, qn2);
  PANO_CUDA(cudaGetLastError());
  return PANO_OK;
}

}  // namespace pano
