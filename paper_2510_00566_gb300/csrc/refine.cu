// Point-centric refinement of candidate-id lists (the paper's no-batch
// variant, B = 1: IndexFlatPanorama behind IndexRefinePanorama, Section 6.4
// and Table 1): another index's top-k' ids per query are re-ranked exactly,
// each candidate being abandoned at the first level whose Eq. 3 lower bound
// exceeds the query's running k-th distance (Algorithm 1).
//
// Flat layout (build_flat): the transformed rows x~ = T~(x - mu~) row-major
// [n][d] FP32 (a candidate's level slice is contiguous, so a scattered id list
// costs one gather per level), rounded-up tails sqrt(R^{(l,d)}) [n][L+1],
// ||x~||^2 and the transform error bound e_x [n], and the original rows [n][d]
// for the exact re-ranking.  The id of a vector is its row.
//
// Search (refine_kernel, one CTA per query): Algorithm 1 seeds the heap with
// the first k candidates' exact distances; the rest go in rounds of 256, one
// candidate per thread, refined level by level against the round's
// threshold with the margined separable test of the IVF kernels.  The
// survivors of a round are checked against the threshold of the moment and
// against each other (k survivors with upper bounds below a lower bound rule
// it out), then re-ranked on the original rows (a warp each) and inserted
// into the query's top-k in shared memory (a thread each).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "gemm.h"
#include "internal.h"
#include "kernels_common.cuh"
#include "search.h"

namespace pano {
namespace {

constexpr int RT = 256;           // threads per query: one candidate each per round
constexpr int RW = RT / 32;
constexpr int kRefineMaxK = 1024;
constexpr int kSeedScan = 2048;  // candidates ranked for the seed (shared memory)
constexpr float kEval = 32.f * 5.9604645e-08f;  // evaluation slack of the separable test

// Tails, norms and transform-error bounds of the flat rows (FP64 sums; the
// same quantities as the IVF packers, per row instead of per chunk slot).
__global__ void __launch_bounds__(256) flat_stats_kernel(
    const float* __restrict__ xt, const float* __restrict__ rows, int64_t n, int d, int L,
    const int32_t* __restrict__ level_off, const float* __restrict__ mu, double c_trans,
    float* __restrict__ tails, float* __restrict__ xn2, float* __restrict__ ex) {
  const int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float* x = xt + i * d;
  double suffix = 0.0;
  for (int l = L - 1; l >= 0; --l) {
    double e = 0.0;
    for (int j = level_off[l] + lane; j < level_off[l + 1]; j += 32) {
      const double v = x[j];
      e += v * v;
    }
    suffix += warp_sum_f64(e);
    if (lane == 0) tails[i * (L + 1) + l] = __double2float_ru(sqrt(suffix * (1.0 + 1e-12)));
  }
  double dev = 0.0;
  const float* r = rows + i * d;
  for (int j = lane; j < d; j += 32) {
    const double v = (double)r[j] - (double)mu[j];
    dev += v * v;
  }
  dev = warp_sum_f64(dev);
  if (lane == 0) {
    tails[i * (L + 1) + L] = 0.f;
    xn2[i] = (float)suffix;
    ex[i] = __double2float_ru(c_trans * sqrt(dev) * (1.0 + 1e-9));
  }
}

struct RefineArgs {
  const float* xt;     // [n][d] x~
  const float* tails;  // [n][L+1]
  const float* xn2;
  const float* ex;
  const float* rows;   // [n][d] original
  const float* qt;     // [nq][d] q~
  const float* qorig;  // [nq][d]
  const float4* qinfo;
  const float* qtail;  // [nq][L+1]
  const int64_t* cand;  // [nq][kp], -1 = none
  int64_t* out_ids;
  float* out_dists;
  int* err;
  unsigned long long* stats;  // [0] candidates, [1] dims read, [2] re-ranked
  int64_t n;
  int d, L, kp, k;
  float gslack, lb_scale, ub_scale, inv_lb_up, eps;
  int32_t level_off[65];
};

__device__ __forceinline__ float threshold_of(const unsigned long long* topk, int k) {
  const unsigned long long key = topk[k - 1];
  return key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f);
}

// sqrt(tau / lb_scale) rounded up (rsqrtf: at most 2 ulp; the factor
// 1 + 2^-19 covers it and the products' roundings).
__device__ __forceinline__ float sqrt_ratio_up_r(float tau, float inv_lb_up) {
  const float y = __fmul_ru(tau, inv_lb_up);
  if (y == 0.f) return 0.f;
  return __fmul_ru(__fmul_ru(y, rsqrtf(y)), 1.0f + 0x1p-19f);
}

__global__ void __launch_bounds__(RT) refine_kernel(const RefineArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = a.d, L = a.L, k = a.k, kp = a.kp;
  float* qs = reinterpret_cast<float*>(sm);  // q~ [d], 16-byte aligned for float4 reads
  unsigned long long* topk = reinterpret_cast<unsigned long long*>(qs + ((d + 3) & ~3));  // [k]
  __shared__ float qtl[65];
  __shared__ int64_t pslot[RT];
  __shared__ float plb[RT], pub[RT];
  __shared__ uint16_t keep[RT];
  __shared__ int s_np, s_nk;
  __shared__ float4 s_qterm;  // (E, g rq, H_q, tau)
  __shared__ unsigned long long s_dims, s_cands, s_rer;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const int64_t q = blockIdx.x;
  for (int i = tid; i < k; i += RT) topk[i] = kEmptyKey;
  for (int j = tid; j < d; j += RT) qs[j] = a.qt[q * d + j];
  for (int l = tid; l <= L; l += RT) qtl[l] = a.eps * a.qtail[q * (L + 1) + l];
  if (tid == 0) s_dims = s_cands = s_rer = 0;
  const float4 inf = a.qinfo[q];
  const float nq = inf.x, rq = inf.y, eq = inf.z, gs = a.gslack;
  const int64_t* cl = a.cand + q * (int64_t)kp;
  const float* qo = a.qorig + q * (int64_t)d;
  const bool vec = (d & 3) == 0;
  __syncthreads();

  auto valid_id = [&](int64_t id) {
    if (id < -1 || id >= a.n) {
      atomicOr(a.err, kErrBadInput);
      return false;
    }
    return id >= 0;
  };
  // Algorithm 1 seeds the heap with k candidates' exact distances; which k
  // is free, so they are the k of smallest approximate distance after the
  // first level, A^(1) = ||q~||^2 + ||x~||^2 - 2 p^(0,1) (>= 0: the first
  // level's squared distance plus both tail energies), among the first
  // kSeedScan candidates.  A seed is marked -1 in akey and skipped later.
  const int ns = min(kp, kSeedScan);
  const int m1 = a.level_off[1];
  float* akey = reinterpret_cast<float*>(topk + k);  // [ns]
  unsigned long long dims0 = 0;
  for (int c = tid; c < ns; c += RT) {
    const int64_t id = cl[c];
    float key = INFINITY;
    if (valid_id(id)) {
      const float* x = a.xt + id * d;
      float p0 = 0.f;
      for (int j = 0; j < m1; ++j) p0 = fmaf(qs[j], x[j], p0);
      key = fmaxf(nq + a.xn2[id] - 2.f * p0, 0.f);
      dims0 += (unsigned long long)m1;
    }
    akey[c] = key;
  }
  __syncthreads();
  __shared__ float s_tk;
  if (warp == 0) {
    const float tk = warp_kth_smallest(akey, ns, k);
    if (lane == 0) s_tk = tk;
  }
  __syncthreads();
  const float tk = s_tk;
  for (int c = warp; c < ns; c += RW) {
    // absent or invalid ids carry +inf, which tk = +inf (fewer than k valid
    // candidates) would otherwise admit
    if (akey[c] == INFINITY || !(akey[c] <= tk)) continue;
    const int64_t id = cl[c];
    const float dist = exact_sqdist_warp_wide(qo, a.rows + id * d, d);
    __syncwarp();
    if (lane == 0) {
      // a repeat of a seed id is a seed too: equal keys are kept once
      topk_insert_thread(topk, k, make_key(dist, (int32_t)id));
      akey[c] = -1.f;
      atomicAdd(&s_rer, 1ull);
      atomicAdd(&s_cands, 1ull);
      atomicAdd(&s_dims, (unsigned long long)d);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) dims0 += __shfl_xor_sync(0xffffffffu, dims0, off);
  if (lane == 0 && dims0) atomicAdd(&s_dims, dims0);
  __syncthreads();

  for (int r0 = 0; r0 < kp; r0 += RT) {
    if (tid == 0) {
      s_np = 0;
      const float tau = threshold_of(topk, k);
      const float st = tau == INFINITY ? 1e18f : sqrt_ratio_up_r(tau, a.inv_lb_up);
      const float E = __fadd_ru(eq, st);
      s_qterm = make_float4(E, gs * rq, 0.5f * (nq - gs * nq - E * E - kEval * (rq + E) * (rq + E)),
                            tau);
    }
    __syncthreads();
    const float4 t = s_qterm;
    const int c = r0 + tid;
    const bool seeded = c < ns && akey[c] < 0.f;
    const int64_t id = c < kp && !seeded ? cl[c] : -1;
    unsigned long long dims = 0;
    if (c < kp && !seeded && valid_id(id)) {
      const float* x = a.xt + id * d;
      const float* tx = a.tails + id * (L + 1);
      const float nx = a.xn2[id], rx = sqrtf(nx), exv = a.ex[id];
      const float Hx = 0.5f * (nx - gs * nx - exv * exv - kEval * (rx + exv) * (rx + exv));
      float p = 0.f;
      bool alive = true;
      for (int l = 0; l < L && alive; ++l) {
        const int m0 = a.level_off[l], m1 = a.level_off[l + 1];
        float acc = 0.f;
        if (vec && ((m0 | m1) & 3) == 0) {
          for (int j = m0; j < m1; j += 4) {
            const float4 xv = *reinterpret_cast<const float4*>(x + j);
            const float4 qv = *reinterpret_cast<const float4*>(qs + j);
            acc = fmaf(qv.x, xv.x, acc);
            acc = fmaf(qv.y, xv.y, acc);
            acc = fmaf(qv.z, xv.z, acc);
            acc = fmaf(qv.w, xv.w, acc);
          }
        } else {
          for (int j = m0; j < m1; ++j) acc = fmaf(qs[j], x[j], acc);
        }
        p += acc;
        dims += (unsigned long long)(m1 - m0);
        // margined Eq. 3 (separable form): pruned when LB > tau
        const float P = fmaf(t.x, exv, fmaf(t.y, rx, fmaf(qtl[l + 1], tx[l + 1], p)));
        if (P < t.z + Hx) alive = false;
      }
      if (alive) {  // its Eq. 3 bounds after the last level (C = 0)
        const float A = nq + nx - 2.f * p, S = rq + rx;
        const float lr = sqrtf(fmaxf(A - gs * S * S, 0.f)) - (eq + exv);
        const float ru = __fadd_ru(__fsqrt_ru(fmaxf(A + gs * S * S, 0.f)), eq + exv);
        const int pos = atomicAdd(&s_np, 1);
        pslot[pos] = id;
        plb[pos] = lr > 0.f ? lr * lr * a.lb_scale : 0.f;
        pub[pos] = __fmul_ru(__fmul_ru(ru, ru), a.ub_scale);
      }
      atomicAdd(&s_cands, 1ull);
    }
    // coordinates read (one atomic per warp)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dims += __shfl_xor_sync(0xffffffffu, dims, off);
    if (lane == 0 && dims) atomicAdd(&s_dims, dims);
    if (tid == 0) s_nk = 0;
    __syncthreads();
    // the round's survivors: dropped if above the threshold of the moment or
    // if k survivors have upper bounds below its lower bound
    const int np = s_np;
    if (tid < np) {
      const float lb = plb[tid];
      bool keep_s = !(lb > threshold_of(topk, k));
      if (keep_s) {
        int below = 0;
        for (int o = 0; o < np && below < k; ++o) below += __fmul_ru(pub[o], 1.000001f) < lb;
        keep_s = below < k;
      }
      if (keep_s) keep[atomicAdd(&s_nk, 1)] = (uint16_t)tid;
    }
    __syncthreads();
    const int nk = s_nk;
    for (int i = warp; i < nk; i += RW) {
      const int s = keep[i];
      const float dist = exact_sqdist_warp_wide(qo, a.rows + pslot[s] * d, d);
      if (lane == 0) plb[s] = dist;
    }
    __syncthreads();
    if (tid < nk) {
      const int s = keep[tid];
      topk_insert_thread(topk, k, make_key(plb[s], (int32_t)pslot[s]));
    }
    if (tid == 0) s_rer += (unsigned long long)nk;
    __syncthreads();
  }
  for (int i = tid; i < k; i += RT) {
    const unsigned long long key = topk[i];
    a.out_ids[q * k + i] = key == kEmptyKey ? -1 : (int64_t)key_id(key);
    a.out_dists[q * k + i] = key == kEmptyKey ? INFINITY : key_dist(key);
  }
  if (tid == 0 && a.stats) {
    atomicAdd(&a.stats[0], s_cands);
    atomicAdd(&a.stats[1], s_dims);
    atomicAdd(&a.stats[2], s_rer);
  }
}

struct Buf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~Buf() {
    if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace

int build_flat(const pano_transform* t, const float* X, int64_t n, const pano_build_opts* o,
               cudaStream_t st, pano_index** out) {
  PANO_CHECK(t && X && out, PANO_EINVAL, "null argument");
  const int d = t->d;
  PANO_CHECK(n >= 1 && n < ((int64_t)1 << 31) - 1, PANO_EINVAL, "need 1 <= n < 2^31 - 1");
  PANO_CHECK(!o || o->precision == PANO_FP32, PANO_EINVAL, "a flat index stores FP32 rows");
  PANO_CHECK(d <= 8192, PANO_EINVAL, "dimension must be at most 8192");
  int dev = 0;
  int rc = check_device(&dev);
  if (rc) return rc;
  auto idx = std::make_unique<pano_index>();
  pano_index& I = *idx;
  I.device = dev;
  I.n = n;
  I.d = d;
  I.nlist = 1;
  I.precision = PANO_FP32;
  I.chunk = 1;
  I.flat = 1;
  I.n_chunks = n;
  I.tf = *t;
  rc = make_levels(d, o, I.widths, I.offs);
  if (rc) return rc;
  I.L = (int)I.widths.size();
  I.max_w = *std::max_element(I.widths.begin(), I.widths.end());
  I.eta = t->eta;
  const double nu = std::sqrt((double)d * (1.0 + t->eta));
  I.c_trans = t->identity ? 0.0 : (gamma_n(gemm_rounds(d)) * nu + 1.01 * kU32 * (1.0 + t->eta));
  // one list holding every row (the IVF tables stay consistent: save/load,
  // index inspection); the id of a vector is its row
  I.list_size.assign(1, (int32_t)n);
  I.list_chunk_off = {0, n};
  I.centroids.assign(d, 0.f);
  I.assign.assign(n, 0);
  std::vector<int32_t> ident(n);
  for (int64_t i = 0; i < n; ++i) ident[i] = (int32_t)i;
  if ((rc = I.level_off_d.alloc((I.L + 1) * 4)) || (rc = I.T32.alloc((size_t)d * d * 4)) ||
      (rc = I.mu32.alloc(d * 4)) || (rc = I.slices.alloc(I.slices_bytes())) ||
      (rc = I.tails.alloc((size_t)n * (I.L + 1) * 4)) || (rc = I.xn2.alloc(n * 4)) ||
      (rc = I.ex.alloc(n * 4)) || (rc = I.rows.alloc((size_t)n * d * 4)) ||
      (rc = I.ids.alloc(n * 4)) || (rc = I.cent.alloc(d * 4)) || (rc = I.cent_n2.alloc(4)) ||
      (rc = I.chunk_off_d.alloc(16)) || (rc = I.list_size_d.alloc(4)))
    return rc;
  PANO_CUDA(cudaMemcpyAsync(I.ids.p, ident.data(), n * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemsetAsync(I.cent.p, 0, d * 4, st));
  PANO_CUDA(cudaMemsetAsync(I.cent_n2.p, 0, 4, st));
  PANO_CUDA(cudaMemcpyAsync(I.chunk_off_d.p, I.list_chunk_off.data(), 16, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.list_size_d.p, I.list_size.data(), 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.level_off_d.p, I.offs.data(), (I.L + 1) * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.T32.p, t->T32.data(), (size_t)d * d * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.mu32.p, t->mu32.data(), d * 4, cudaMemcpyHostToDevice, st));
  // host or device input: cudaMemcpyDefault picks the direction
  PANO_CUDA(cudaMemcpyAsync(I.rows.p, X, (size_t)n * d * 4, cudaMemcpyDefault, st));
  const int64_t blk = std::max<int64_t>(1, ((int64_t)1 << 26) / ((int64_t)d * 4));
  for (int64_t s = 0; s < n; s += blk) {
    const int64_t m = std::min(blk, n - s);
    PANO_CUDA(gemm_nt(kStore, (int)m, d, d, I.rows.as<float>() + s * d, d, I.mu32.as<float>(),
                      I.T32.as<float>(), d, I.slices.as<float>() + s * d, d, nullptr, nullptr, st));
  }
  flat_stats_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(
      I.slices.as<float>(), I.rows.as<float>(), n, d, I.L, I.level_off_d.as<int32_t>(),
      I.mu32.as<float>(), I.c_trans, I.tails.as<float>(), I.xn2.as<float>(), I.ex.as<float>());
  PANO_CUDA(cudaGetLastError());
  PANO_CUDA(cudaStreamSynchronize(st));
  *out = idx.release();
  return PANO_OK;
}

int refine(const pano_index* ip, const float* queries, int64_t nq, const int64_t* cand,
           int32_t kprime, int32_t k, int64_t* out_ids, float* out_dists, float epsilon,
           cudaStream_t st) {
  PANO_CHECK(ip, PANO_EINVAL, "null index");
  const pano_index& I = *ip;
  PANO_CHECK(I.flat, PANO_EINVAL, "refine needs a flat index (panorama_build_flat)");
  PANO_CHECK(nq >= 0 && nq < (1LL << 31), PANO_EINVAL, "nq out of range");
  PANO_CHECK(k >= 1 && k <= kRefineMaxK, PANO_EINVAL, "k must be in [1, 1024]");
  PANO_CHECK(kprime >= 0 && kprime <= (1 << 20), PANO_EINVAL, "kprime must be in [0, 2^20]");
  PANO_CHECK(nq == 0 || (queries && out_ids && out_dists && (kprime == 0 || cand)), PANO_EINVAL,
             "null argument");
  PANO_CHECK(epsilon >= 0.f && epsilon <= 1.f, PANO_EINVAL, "epsilon must be in [0, 1]");
  int cur = -1;
  PANO_CUDA(cudaGetDevice(&cur));
  PANO_CHECK(cur == I.device, PANO_EINVAL, "current device differs from the index's device");
  pano_search_stats& stats = stats_slot();
  std::memset(&stats, 0, sizeof(stats));
  stats.n_queries = nq;
  if (nq == 0) return PANO_OK;
  const int d = I.d, L = I.L;
  // workspace: q~, qinfo, qtail, qn2, error flag, counters
  const size_t o_qt = 0, o_qi = (o_qt + (size_t)nq * d * 4 + 255) & ~(size_t)255;
  const size_t o_qtl = (o_qi + (size_t)nq * 16 + 255) & ~(size_t)255;
  const size_t o_qn = (o_qtl + (size_t)nq * (L + 1) * 4 + 255) & ~(size_t)255;
  const size_t o_err = (o_qn + (size_t)nq * 4 + 255) & ~(size_t)255;
  const size_t total = o_err + 256;
  Buf ws;
  ws.st = st;
  PANO_CUDA(cudaMallocAsync(&ws.p, total, st));
  char* W = (char*)ws.p;
  PANO_CUDA(cudaMemsetAsync(W + o_err, 0, 256, st));
  int rc = transform_queries(I, queries, nq, (float*)(W + o_qt), (float4*)(W + o_qi),
                             (float*)(W + o_qtl), (float*)(W + o_qn), st);
  if (rc) return rc;
  RefineArgs a;
  std::memset(&a, 0, sizeof(a));
  a.xt = I.slices.as<float>();
  a.tails = I.tails.as<float>();
  a.xn2 = I.xn2.as<float>();
  a.ex = I.ex.as<float>();
  a.rows = I.rows.as<float>();
  a.qt = (const float*)(W + o_qt);
  a.qorig = queries;
  a.qinfo = (const float4*)(W + o_qi);
  a.qtail = (const float*)(W + o_qtl);
  a.cand = cand;
  a.out_ids = out_ids;
  a.out_dists = out_dists;
  a.err = (int*)(W + o_err);
  a.stats = (unsigned long long*)(W + o_err + 64);
  a.n = I.n;
  a.d = d;
  a.L = L;
  a.kp = kprime;
  a.k = k;
  // the FP32 IVF kernel's margins: per-level dot products then a running sum
  a.gslack = (float)(2.0 * gamma_n(I.max_w + L + 8));
  a.lb_scale = (float)((1.0 - 8.0 * kU32) / (1.0 + I.eta));
  a.ub_scale = (float)((1.0 + 8.0 * kU32) / (1.0 - I.eta) * (1.0 + 1e-7));
  {
    const double inv = 1.0 / (double)a.lb_scale;
    float f = (float)inv;
    if ((double)f < inv) f = std::nextafter(f, INFINITY);
    a.inv_lb_up = f;
  }
  a.eps = epsilon > 0.f ? epsilon : 1.f;
  for (int l = 0; l <= L; ++l) a.level_off[l] = I.offs[l];
  const size_t smem =
      (size_t)((d + 3) & ~3) * 4 + (size_t)k * 8 + (size_t)std::min(kprime, kSeedScan) * 4;
  PANO_CUDA(cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(smem, 48 * 1024)));
  refine_kernel<<<(unsigned)nq, RT, smem, st>>>(a);
  PANO_CUDA(cudaGetLastError());
  int herr = 0;
  unsigned long long hst[3];
  PANO_CUDA(cudaMemcpyAsync(&herr, a.err, 4, cudaMemcpyDeviceToHost, st));
  PANO_CUDA(cudaMemcpyAsync(hst, a.stats, 24, cudaMemcpyDeviceToHost, st));
  PANO_CUDA(cudaStreamSynchronize(st));
  stats.pairs = (int64_t)hst[0];
  stats.dims_scanned = (int64_t)hst[1];
  stats.reranked = (int64_t)hst[2];
  if (herr & kErrBadInput) return fail(PANO_EINVAL, "candidate id outside [-1, n)");
  return PANO_OK;
}

}  // namespace pano
