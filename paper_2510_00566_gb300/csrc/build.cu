// panorama_build_ivf: k-means coarse quantiser, nearest-centroid assignment,
// transform and level-major packing of every IVF list (Sections 6.1, 6.5).
//
// Device layout of a built FP32 index (CH = 64 vectors per chunk, chunks of
// one list are consecutive, lists in id order, a list's last chunk padded):
//   slices [chunk][d+L+3][CH] x~ transposed per chunk, level by level: the
//                           level-l block is the [w_l][CH] slice at dims
//                           m_l..m_{l+1}-1 (the paper's level-major batch,
//                           with B = CH) followed by the tail row
//                           sqrt(R_x^{(l+1,d)}); level 0's block also holds
//                           ||x~||^2, e_x and the ids, so one bulk copy
//                           stages everything a (chunk, level) step reads;
//   tails  [chunk][L+1][CH] sqrt(R_x^{(l,d)}) rounded up (FP64 sums);
//   xn2    [chunk][CH]      ||x~||^2;  ex [chunk][CH] bound on the transform
//                           error ||x~ - T~(x - mu~)||;  ids [chunk][CH];
//   rows   [chunk*CH][d]    the original FP32 rows (exact re-ranking).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "gemm.h"
#include "internal.h"
#include "kernels_common.cuh"
#include "search.h"
#include "verify_tc.h"

namespace pano {

namespace {

constexpr int CH = 64;

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// k distinct indices of [0, n) (partial Fisher-Yates on an index map).
std::vector<int64_t> sample_without_replacement(int64_t n, int64_t k, uint64_t seed) {
  std::vector<int64_t> out(k);
  if (k >= n) {
    std::iota(out.begin(), out.end(), 0);
    return out;
  }
  std::vector<int64_t> perm;
  if (n <= (int64_t)1 << 26) {
    perm.resize(n);
    std::iota(perm.begin(), perm.end(), 0);
    for (int64_t i = 0; i < k; ++i) {
      int64_t j = i + (int64_t)(splitmix64(seed) % (uint64_t)(n - i));
      std::swap(perm[i], perm[j]);
      out[i] = perm[i];
    }
  } else {  // sparse: rejection of repeats
    std::vector<int64_t> seen;
    seen.reserve(k);
    while ((int64_t)seen.size() < k) {
      int64_t v = (int64_t)(splitmix64(seed) % (uint64_t)n);
      seen.push_back(v);
      if ((int64_t)seen.size() == k) {
        std::sort(seen.begin(), seen.end());
        seen.erase(std::unique(seen.begin(), seen.end()), seen.end());
      }
    }
    out = seen;
  }
  std::sort(out.begin(), out.end());
  return out;
}

__global__ void gather_rows_kernel(const float* __restrict__ X, int d,
                                   const int64_t* __restrict__ idx, int64_t m,
                                   float* __restrict__ out) {
  int64_t row = blockIdx.x;
  if (row >= m) return;
  int64_t src = idx[row];
  for (int j = threadIdx.x; j < d; j += blockDim.x)
    out[row * d + j] = src >= 0 ? X[src * d + j] : 0.f;
}

// FP32 squared norms of rows (accumulated in FP64, rounded once).
__global__ void row_norms_kernel(const float* __restrict__ X, int64_t m, int d,
                                 float* __restrict__ out) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= m) return;
  double s = 0.0;
  for (int j = threadIdx.x & 31; j < d; j += 32) {
    double v = X[row * d + j];
    s += v * v;
  }
  s = warp_sum_f64(s);
  if ((threadIdx.x & 31) == 0) out[row] = (float)s;
}

// Sums of member rows per centroid (FP64 atomics) and member counts.
__global__ void kmeans_accum_kernel(const float* __restrict__ X, int64_t m, int d,
                                    const unsigned long long* __restrict__ best2,
                                    double* __restrict__ sums, int* __restrict__ counts) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= m) return;
  int c = (int)(uint32_t)(best2[2 * row] & 0xffffffffULL);
  int lane = threadIdx.x & 31;
  for (int j = lane; j < d; j += 32) atomicAdd(&sums[(int64_t)c * d + j], (double)X[row * d + j]);
  if (lane == 0) atomicAdd(&counts[c], 1);
}

// Final assignment: the expansion-form best centroid unless the runner-up is
// within twice the expansion's rounding bound, in which case both are
// re-scored with the compensated difference form (ties -> lower id).
__global__ void assign_resolve_kernel(const float* __restrict__ X, int64_t m, int d,
                                      const float* __restrict__ C, const float* __restrict__ xn2,
                                      const float* __restrict__ cn2, float cmax,
                                      const unsigned long long* __restrict__ best2, float gerr,
                                      int32_t* __restrict__ out) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= m) return;
  unsigned long long k0 = best2[2 * row], k1 = best2[2 * row + 1];
  int c0 = (int)(uint32_t)(k0 & 0xffffffffULL);
  int choice = c0;
  if (k1 != kEmptyKey) {
    int c1 = (int)(uint32_t)(k1 & 0xffffffffULL);
    uint32_t o0 = (uint32_t)(k0 >> 32), o1 = (uint32_t)(k1 >> 32);
    auto dec = [](uint32_t o) {
      uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
      return __uint_as_float(u);
    };
    float d0 = dec(o0), d1 = dec(o1);
    float s = sqrtf(xn2[row]) + cmax;
    float band = 2.f * gerr * s * s;
    if (d1 - d0 <= band) {
      float e0 = exact_sqdist_warp(X + row * d, C + (int64_t)c0 * d, d);
      float e1 = exact_sqdist_warp(X + row * d, C + (int64_t)c1 * d, d);
      if (e1 < e0 || (e1 == e0 && c1 < c0)) choice = c1;
    }
  }
  if ((threadIdx.x & 31) == 0) out[row] = choice;
}

// x~ for 64 slots (one chunk) per CTA -> transposed slices, tail norms,
// norms, transform-error bounds and ids.
// xt, rows and perm point at the block's first chunk; chunk0 is its global
// index (outputs are global arrays).
__global__ void __launch_bounds__(256) pack_fp32_kernel(
    const float* __restrict__ xt, const float* __restrict__ rows,
    const int64_t* __restrict__ perm, int64_t chunk0, int d, int L,
    const int32_t* __restrict__ level_off, const float* __restrict__ mu, double c_trans,
    float* __restrict__ slices, float* __restrict__ tails, float* __restrict__ xn2,
    float* __restrict__ ex, int32_t* __restrict__ ids) {
  __shared__ float tile[CH][33];
  __shared__ int16_t lvl_of[8192];  // level of each dimension
  const int64_t lc = blockIdx.x;  // chunk within the block
  const int64_t g = chunk0 + lc;  // global chunk
  const float* xblk = xt + lc * CH * d;
  const int64_t* pb = perm + lc * CH;
  float* sl = slices + g * (int64_t)(d + L + 3) * CH;
  // row of dimension j in the chunk's block sequence
  auto row_of = [&](int j) { const int l = lvl_of[j]; return j + (l == 0 ? 0 : l + 3); };
  auto tail_row = [&](int l) { return level_off[l + 1] + (l == 0 ? 0 : l + 3); };
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    int l = 0;
    while (level_off[l + 1] <= j) ++l;
    lvl_of[j] = (int16_t)l;
  }
  __syncthreads();
  for (int j0 = 0; j0 < d; j0 += 32) {
    for (int e = threadIdx.x; e < CH * 32; e += blockDim.x) {
      int i = e / 32, jj = e % 32;
      float v = 0.f;
      if (j0 + jj < d && pb[i] >= 0) v = xblk[(int64_t)i * d + j0 + jj];
      tile[i][jj] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CH * 32; e += blockDim.x) {
      int jj = e / CH, i = e % CH;
      if (j0 + jj < d) sl[(int64_t)row_of(j0 + jj) * CH + i] = tile[i][jj];
    }
    __syncthreads();
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  for (int i = warp; i < CH; i += blockDim.x / 32) {
    int64_t slot = g * CH + i;
    bool valid = pb[i] >= 0;
    const float* x = xblk + (int64_t)i * d;
    double suffix = 0.0;
    // level energies from the last level backwards give the tails directly
    for (int l = L - 1; l >= 0; --l) {
      double e = 0.0;
      if (valid)
        for (int j = level_off[l] + lane; j < level_off[l + 1]; j += 32) {
          double v = x[j];
          e += v * v;
        }
      e = warp_sum_f64(e);
      suffix += e;
      if (lane == 0) {
        const float t = __double2float_ru(sqrt(suffix * (1.0 + 1e-12)));
        tails[(g * (L + 1) + l) * CH + i] = t;
        if (l > 0) sl[(int64_t)tail_row(l - 1) * CH + i] = t;
      }
    }
    double dev = 0.0;  // ||x - mu~||
    if (valid) {
      const float* r = rows + (lc * CH + i) * (int64_t)d;  // rows of this block
      for (int j = lane; j < d; j += 32) {
        double v = (double)r[j] - (double)mu[j];
        dev += v * v;
      }
    }
    dev = warp_sum_f64(dev);
    if (lane == 0) {
      const float exv = valid ? __double2float_ru(c_trans * sqrt(dev) * (1.0 + 1e-9)) : 0.f;
      const int32_t id = valid ? (int32_t)pb[i] : -1;
      tails[(g * (L + 1) + L) * CH + i] = 0.f;
      sl[(int64_t)tail_row(L - 1) * CH + i] = 0.f;
      xn2[slot] = (float)suffix;
      ex[slot] = exv;
      ids[slot] = id;
      const int64_t r0 = tail_row(0);  // level 0's extra rows
      sl[(r0 + 1) * CH + i] = (float)suffix;
      sl[(r0 + 2) * CH + i] = exv;
      sl[(r0 + 3) * CH + i] = __int_as_float(id);
    }
  }
}

// k-means++ seeding (D^2 sampling, Arthur & Vassilvitskii 2007) over m
// sample rows, on the device.  Round r: every row's squared distance to the
// newest seed lowers its running minimum d2; each block adds up its rows'
// d2 (FP64); then one thread draws u ~ U[0, sum d2) from a counter-based
// hash of (seed, r) and picks the row where the running sum crosses u.
constexpr int kKppBlocks = 512;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) kpp_update_kernel(const float* __restrict__ xs, int64_t m,
                                                         int d, const int64_t* __restrict__ picks,
                                                         int r, int64_t rpb, float* __restrict__ d2,
                                                         double* __restrict__ bsum) {
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
  const float* c = xs + picks[r] * (int64_t)d;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  double part = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += blockDim.x / 32) {
    const float* x = xs + i * (int64_t)d;
    float s = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float t = x[j] - c[j];
      s = fmaf(t, t, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const float v = r == 0 ? s : fminf(d2[i], s);
    if (lane == 0) d2[i] = v;
    part += (double)v;
  }
  __shared__ double red[8];
  if (lane == 0) red[warp] = part;  // lane 0 holds the warp's rows (all lanes add the same)
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void kpp_pick_kernel(const float* __restrict__ d2, int64_t m, int64_t rpb, int nblk,
                                const double* __restrict__ bsum, uint64_t seed, int r,
                                int64_t* __restrict__ picks) {
  if (threadIdx.x != 0) return;
  double total = 0.0;
  for (int b = 0; b < nblk; ++b) total += bsum[b];
  const double u = (double)(mix64(seed ^ mix64((uint64_t)r + 1)) >> 11) * 0x1.0p-53 * total;
  int64_t pick = (int64_t)((mix64(seed + 7 * (uint64_t)r) >> 1) % (uint64_t)m);  // all d2 zero
  if (total > 0.0) {
    double acc = 0.0;
    int b = 0;
    while (b < nblk - 1 && acc + bsum[b] <= u) acc += bsum[b++];
    const int64_t i0 = (int64_t)b * rpb, i1 = i0 + rpb < m ? i0 + rpb : m;
    pick = i1 - 1;
    for (int64_t i = i0; i < i1; ++i) {
      acc += (double)d2[i];
      if (acc > u && d2[i] > 0.f) {
        pick = i;
        break;
      }
    }
  }
  picks[r + 1] = pick;
}

struct Tmp {
  void* p = nullptr;
  ~Tmp() {
    if (p) cudaFree(p);
  }
};

int kmeans(const float* Xd, int64_t n, int d, int nlist, int iters, int64_t ns,
           uint64_t seed, cudaStream_t st, std::vector<float>& cent) {
  std::vector<int64_t> sidx = sample_without_replacement(n, ns, seed);
  ns = (int64_t)sidx.size();
  Tmp t_idx, t_xs, t_xn, t_c, t_cn, t_best, t_sums, t_cnt;
  PANO_CUDA(cudaMalloc(&t_idx.p, ns * sizeof(int64_t)));
  PANO_CUDA(cudaMalloc(&t_xs.p, (size_t)ns * d * sizeof(float)));
  PANO_CUDA(cudaMalloc(&t_xn.p, ns * sizeof(float)));
  PANO_CUDA(cudaMalloc(&t_c.p, (size_t)nlist * d * sizeof(float)));
  PANO_CUDA(cudaMalloc(&t_cn.p, nlist * sizeof(float)));
  PANO_CUDA(cudaMalloc(&t_best.p, 2 * ns * sizeof(unsigned long long)));
  PANO_CUDA(cudaMalloc(&t_sums.p, (size_t)nlist * d * sizeof(double)));
  PANO_CUDA(cudaMalloc(&t_cnt.p, nlist * sizeof(int)));
  PANO_CUDA(cudaMemcpyAsync(t_idx.p, sidx.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  float* xs = (float*)t_xs.p;
  gather_rows_kernel<<<(unsigned)ns, 128, 0, st>>>(Xd, d, (int64_t*)t_idx.p, ns, xs);
  row_norms_kernel<<<(unsigned)((ns + 7) / 8), 256, 0, st>>>(xs, ns, d, (float*)t_xn.p);
  // initial centroids: k-means++ (D^2) seeding over the first m sample rows
  // (the sample is already a uniform draw of the data)
  {
    const int64_t m = std::min<int64_t>(ns, (int64_t)64 * nlist);
    const int64_t rpb = (m + kKppBlocks - 1) / kKppBlocks;
    const int nblk = (int)((m + rpb - 1) / rpb);
    Tmp t_d2, t_bs, t_pk;
    PANO_CUDA(cudaMalloc(&t_d2.p, m * sizeof(float)));
    PANO_CUDA(cudaMalloc(&t_bs.p, nblk * sizeof(double)));
    PANO_CUDA(cudaMalloc(&t_pk.p, (size_t)(nlist + 1) * sizeof(int64_t)));
    uint64_t s0 = seed ^ 0xA5A5A5A5ULL;
    const int64_t first = (int64_t)(splitmix64(s0) % (uint64_t)m);
    PANO_CUDA(cudaMemcpyAsync(t_pk.p, &first, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    for (int r = 0; r + 1 < nlist; ++r) {
      kpp_update_kernel<<<nblk, 256, 0, st>>>(xs, m, d, (const int64_t*)t_pk.p, r, rpb,
                                              (float*)t_d2.p, (double*)t_bs.p);
      kpp_pick_kernel<<<1, 32, 0, st>>>((const float*)t_d2.p, m, rpb, nblk,
                                        (const double*)t_bs.p, s0, r, (int64_t*)t_pk.p);
    }
    PANO_CUDA(cudaGetLastError());
    gather_rows_kernel<<<(unsigned)nlist, 128, 0, st>>>(xs, d, (const int64_t*)t_pk.p, nlist,
                                                        (float*)t_c.p);
    PANO_CUDA(cudaGetLastError());
    cent.resize((size_t)nlist * d);
    PANO_CUDA(cudaMemcpyAsync(cent.data(), t_c.p, cent.size() * sizeof(float),
                              cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<double> hsums((size_t)nlist * d);
  std::vector<int> hcnt(nlist);
  std::vector<float> hcn(nlist);
  uint64_t pert = seed ^ 0x5EED5EEDULL;
  for (int it = 0; it < iters; ++it) {
    for (int c = 0; c < nlist; ++c) {
      double s = 0.0;
      for (int j = 0; j < d; ++j) s += (double)cent[(size_t)c * d + j] * cent[(size_t)c * d + j];
      hcn[c] = (float)s;
    }
    PANO_CUDA(cudaMemcpyAsync(t_c.p, cent.data(), cent.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    PANO_CUDA(cudaMemcpyAsync(t_cn.p, hcn.data(), nlist * sizeof(float), cudaMemcpyHostToDevice, st));
    PANO_CUDA(gemm_argmin2((int)ns, nlist, d, xs, d, nullptr, (float*)t_c.p, d, (float*)t_xn.p,
                           (float*)t_cn.p, (unsigned long long*)t_best.p, st));
    PANO_CUDA(cudaMemsetAsync(t_sums.p, 0, (size_t)nlist * d * sizeof(double), st));
    PANO_CUDA(cudaMemsetAsync(t_cnt.p, 0, nlist * sizeof(int), st));
    kmeans_accum_kernel<<<(unsigned)((ns + 7) / 8), 256, 0, st>>>(
        xs, ns, d, (unsigned long long*)t_best.p, (double*)t_sums.p, (int*)t_cnt.p);
    PANO_CUDA(cudaGetLastError());
    PANO_CUDA(cudaMemcpyAsync(hsums.data(), t_sums.p, hsums.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaMemcpyAsync(hcnt.data(), t_cnt.p, nlist * sizeof(int), cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < nlist; ++c)
      if (hcnt[c] > 0)
        for (int j = 0; j < d; ++j)
          cent[(size_t)c * d + j] = (float)(hsums[(size_t)c * d + j] / hcnt[c]);
    // empty lists: split the currently largest one (symmetric perturbation)
    for (int c = 0; c < nlist; ++c) {
      if (hcnt[c] > 0) continue;
      int big = (int)(std::max_element(hcnt.begin(), hcnt.end()) - hcnt.begin());
      for (int j = 0; j < d; ++j) {
        float base = cent[(size_t)big * d + j];
        float eps = (float)(1e-4 * ((splitmix64(pert) & 1) ? 1.0 : -1.0)) * (std::fabs(base) + 1e-3f);
        cent[(size_t)c * d + j] = base + eps;
        cent[(size_t)big * d + j] = base - eps;
      }
      hcnt[c] = hcnt[big] / 2;
      hcnt[big] -= hcnt[c];
    }
    // balance: while a list holds under half the mean and another over 1.5
    // times it, the small list's centroid moves to split the large one (at
    // most nlist / 16 moves per iteration; the last two iterations settle)
    if (it + 2 < iters && nlist > 1) {
      const double mean = (double)ns / nlist;
      std::vector<int> order(nlist);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](int x, int y) { return hcnt[x] < hcnt[y]; });
      int lo = 0, hi = nlist - 1, moves = 0;
      while (lo < hi && moves < std::max(1, nlist / 16) && hcnt[order[lo]] < 0.5 * mean &&
             hcnt[order[hi]] > 1.5 * mean) {
        const int small = order[lo++], big = order[hi--];
        for (int j = 0; j < d; ++j) {
          float base = cent[(size_t)big * d + j];
          float eps = (float)(1e-4 * ((splitmix64(pert) & 1) ? 1.0 : -1.0)) * (std::fabs(base) + 1e-3f);
          cent[(size_t)small * d + j] = base + eps;
          cent[(size_t)big * d + j] = base - eps;
        }
        ++moves;
      }
    }
  }
  return PANO_OK;
}

}  // namespace

int DevBuf::alloc(size_t n) {
  release();
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    return cuda_fail(e, "cudaMalloc(index)");
  }
  bytes = n;
  return PANO_OK;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

int check_device(int* dev_out) {
  int dev = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  PANO_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(PANO_ENODEV, "this library is built for sm_103 (GB300); device is sm_" +
                                 std::to_string(prop.major) + std::to_string(prop.minor));
  if (dev_out) *dev_out = dev;
  return PANO_OK;
}

// Level split from the options (shared with load).
int make_levels(int d, const pano_build_opts* o, std::vector<int32_t>& widths,
                std::vector<int32_t>& offs) {
  int L = (o && o->n_levels > 0) ? o->n_levels : 8;
  if (L > d) L = d;
  if (L > 64) return fail(PANO_EINVAL, "at most 64 levels are supported");
  widths.assign(L, 0);
  if (o && o->level_widths) {
    int64_t s = 0;
    for (int l = 0; l < L; ++l) {
      widths[l] = o->level_widths[l];
      if (widths[l] < 1) return fail(PANO_EINVAL, "level widths must be >= 1");
      s += widths[l];
    }
    if (s != d) return fail(PANO_EINVAL, "level widths must sum to d");
  } else {
    if (d % L != 0)
      return fail(PANO_EINVAL, "d must be divisible by n_levels when level_widths is NULL");
    for (int l = 0; l < L; ++l) widths[l] = d / L;
  }
  offs.assign(L + 1, 0);
  for (int l = 0; l < L; ++l) offs[l + 1] = offs[l] + widths[l];
  return PANO_OK;
}

// Centroids (given, the sample mean for one list, or k-means) and each
// vector's nearest centroid (IVF, Section 6.1): fills I.centroids, I.cmax,
// I.cent, I.cent_n2 and I.assign.  Xd: device rows n x d.
int coarse_lists(const float* Xd, int64_t n, int d, int nlist, const pano_build_opts* o,
                 cudaStream_t st, pano_index& I) {
  int rc = PANO_OK;
  if (o && o->centroids) {
    I.centroids.assign(o->centroids, o->centroids + (size_t)nlist * d);
  } else if (nlist == 1) {
    I.centroids.assign(d, 0.f);
    std::vector<float> h((size_t)std::min<int64_t>(n, 65536) * d);
    // a flat index: the centroid is irrelevant to search; keep the sample mean
    PANO_CUDA(cudaMemcpyAsync(h.data(), Xd, h.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaStreamSynchronize(st));
    int64_t m = h.size() / d;
    for (int j = 0; j < d; ++j) {
      double s = 0;
      for (int64_t r = 0; r < m; ++r) s += h[r * d + j];
      I.centroids[j] = (float)(s / m);
    }
  } else {
    int iters = (o && o->kmeans_iters > 0) ? o->kmeans_iters : 20;
    int64_t ns = (o && o->kmeans_sample > 0) ? o->kmeans_sample : (int64_t)256 * nlist;
    ns = std::min(ns, n);
    ns = std::max<int64_t>(ns, nlist);
    rc = kmeans(Xd, n, d, nlist, iters, ns, o ? o->seed : 1234, st, I.centroids);
    if (rc) return rc;
  }
  std::vector<float> hcn(nlist);
  float cmax = 0.f;
  for (int c = 0; c < nlist; ++c) {
    double s = 0;
    for (int j = 0; j < d; ++j) s += (double)I.centroids[(size_t)c * d + j] * I.centroids[(size_t)c * d + j];
    hcn[c] = (float)s;
    cmax = std::max(cmax, (float)std::sqrt(s));
  }
  I.cmax = cmax;
  if ((rc = I.cent.alloc((size_t)nlist * d * 4)) || (rc = I.cent_n2.alloc(nlist * 4))) return rc;
  PANO_CUDA(cudaMemcpyAsync(I.cent.p, I.centroids.data(), (size_t)nlist * d * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.cent_n2.p, hcn.data(), nlist * 4, cudaMemcpyHostToDevice, st));

  // ---- assignment
  I.assign.assign(n, 0);
  if (nlist > 1) {
    Tmp t_xn, t_best, t_asg;
    const int64_t blk = 1 << 20;
    PANO_CUDA(cudaMalloc(&t_xn.p, blk * sizeof(float)));
    PANO_CUDA(cudaMalloc(&t_best.p, 2 * blk * sizeof(unsigned long long)));
    PANO_CUDA(cudaMalloc(&t_asg.p, n * sizeof(int32_t)));
    float gerr = (float)(2.0 * gamma_n(gemm_rounds(d) + 4));
    for (int64_t s = 0; s < n; s += blk) {
      int64_t m = std::min(blk, n - s);
      row_norms_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(Xd + s * d, m, d, (float*)t_xn.p);
      PANO_CUDA(gemm_argmin2((int)m, nlist, d, Xd + s * d, d, nullptr, I.cent.as<float>(), d,
                             (float*)t_xn.p, I.cent_n2.as<float>(), (unsigned long long*)t_best.p, st));
      assign_resolve_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(
          Xd + s * d, m, d, I.cent.as<float>(), (float*)t_xn.p, I.cent_n2.as<float>(), cmax,
          (unsigned long long*)t_best.p, gerr, (int32_t*)t_asg.p + s);
      PANO_CUDA(cudaGetLastError());
    }
    PANO_CUDA(cudaMemcpyAsync(I.assign.data(), t_asg.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PANO_CUDA(cudaStreamSynchronize(st));
  }
  return PANO_OK;
}

int build_ivf(const pano_transform* t, const float* X, int64_t n, int nlist,
              const pano_build_opts* o, cudaStream_t st, pano_index** out) {
  PANO_CHECK(t && X && out, PANO_EINVAL, "null argument");
  const int d = t->d;
  PANO_CHECK(n >= 1 && nlist >= 1 && nlist <= n, PANO_EINVAL, "need 1 <= nlist <= n");
  PANO_CHECK(n < ((int64_t)1 << 31) - 1, PANO_EINVAL, "at most 2^31-2 vectors");
  int precision = o ? o->precision : PANO_FP32;
  PANO_CHECK(precision == PANO_FP32 || precision == PANO_BF16 || precision == PANO_FP8,
             PANO_EINVAL, "storage precision must be PANO_FP32, PANO_BF16 or PANO_FP8");
  PANO_CHECK(d <= 8192, PANO_EINVAL, "dimension must be at most 8192");
  int dev = 0;
  int rc = check_device(&dev);
  if (rc) return rc;
  auto idx = std::make_unique<pano_index>();
  pano_index& I = *idx;
  I.device = dev;
  I.n = n;
  I.d = d;
  I.nlist = nlist;
  I.precision = precision;
  const int CHK = precision == PANO_FP32 ? CH : TC_CHUNK;  // vectors per chunk
  I.chunk = CHK;
  I.tf = *t;
  rc = make_levels(d, o, I.widths, I.offs);
  if (rc) return rc;
  if (precision == PANO_BF16)
    for (int w : I.widths)
      PANO_CHECK(w == 16 || w == 32 || w % 64 == 0, PANO_EINVAL,
                 "bf16 level widths must be 16, 32 or multiples of 64");
  if (precision == PANO_FP8)  // the byte layout of bf16 tiles of half the width
    for (int w : I.widths)
      PANO_CHECK(w == 32 || w == 64 || w % 128 == 0, PANO_EINVAL,
                 "fp8 level widths must be 32, 64 or multiples of 128");
  I.L = (int)I.widths.size();
  I.max_w = *std::max_element(I.widths.begin(), I.widths.end());
  I.eta = t->eta;
  // transform error: blocked FP32 dot products of |T~| rows with |v - mu~|
  // (||T~||_F <= sqrt(d (1 + eta)) bounds the 2-norm of |T~|) plus the
  // rounding of the subtraction.
  double nu = std::sqrt((double)d * (1.0 + t->eta));
  I.c_trans = t->identity ? 0.0 : (gamma_n(gemm_rounds(d)) * nu + 1.01 * kU32 * (1.0 + t->eta));

  // ---- data on the device
  const float* Xd = X;
  Tmp t_x;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, X) != cudaSuccess || pa.type == cudaMemoryTypeHost ||
      pa.type == cudaMemoryTypeUnregistered) {
    cudaGetLastError();
    PANO_CUDA(cudaMalloc(&t_x.p, (size_t)n * d * sizeof(float)));
    PANO_CUDA(cudaMemcpyAsync(t_x.p, X, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, st));
    Xd = (const float*)t_x.p;
  }

  // ---- coarse quantiser and assignment
  rc = coarse_lists(Xd, n, d, nlist, o, st, I);
  if (rc) return rc;

  // ---- list layout (host)
  I.list_size.assign(nlist, 0);
  for (int64_t i = 0; i < n; ++i) I.list_size[I.assign[i]]++;
  I.list_chunk_off.assign(nlist + 1, 0);
  for (int c = 0; c < nlist; ++c)
    I.list_chunk_off[c + 1] = I.list_chunk_off[c] + (I.list_size[c] + CHK - 1) / CHK;
  I.n_chunks = I.list_chunk_off[nlist];
  const int64_t nslots = I.n_chunks * CHK;
  std::vector<int64_t> perm(nslots, -1);
  {
    std::vector<int64_t> fill(nlist, 0);
    for (int64_t i = 0; i < n; ++i) {  // ascending id within each list
      int c = I.assign[i];
      perm[I.list_chunk_off[c] * CHK + fill[c]++] = i;
    }
  }
  std::vector<int64_t> hco(I.list_chunk_off);
  if ((rc = I.chunk_off_d.alloc((nlist + 1) * 8)) || (rc = I.list_size_d.alloc(nlist * 4)) ||
      (rc = I.level_off_d.alloc((I.L + 1) * 4)) || (rc = I.T32.alloc((size_t)d * d * 4)) ||
      (rc = I.mu32.alloc(d * 4)))
    return rc;
  PANO_CUDA(cudaMemcpyAsync(I.chunk_off_d.p, hco.data(), (nlist + 1) * 8, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.list_size_d.p, I.list_size.data(), nlist * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.level_off_d.p, I.offs.data(), (I.L + 1) * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.T32.p, t->T32.data(), (size_t)d * d * 4, cudaMemcpyHostToDevice, st));
  PANO_CUDA(cudaMemcpyAsync(I.mu32.p, t->mu32.data(), d * 4, cudaMemcpyHostToDevice, st));

  // ---- packed arrays
  if ((rc = I.slices.alloc(I.slices_bytes())) ||
      (rc = I.tails.alloc((size_t)I.n_chunks * (I.L + 1) * CHK * 4)) ||
      (rc = I.xn2.alloc(nslots * 4)) || (rc = I.ex.alloc(nslots * 4)) ||
      (rc = I.ids.alloc(nslots * 4)) || (rc = I.rows.alloc((size_t)nslots * d * 4)) ||
      (precision == PANO_FP8 && (rc = I.xscale.alloc(nslots * 4))))
    return rc;
  Tmp t_perm, t_xt;
  PANO_CUDA(cudaMalloc(&t_perm.p, nslots * sizeof(int64_t)));
  PANO_CUDA(cudaMemcpyAsync(t_perm.p, perm.data(), nslots * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (nslots > 0) {
    gather_rows_kernel<<<(unsigned)nslots, 128, 0, st>>>(Xd, d, (int64_t*)t_perm.p, nslots,
                                                          I.rows.as<float>());
    PANO_CUDA(cudaGetLastError());
  }
  // chunks per transform/pack block (64 MB of transformed rows)
  const int64_t cblk = std::max<int64_t>(1, ((int64_t)1 << 26) / ((int64_t)CHK * d * 4));
  PANO_CUDA(cudaMalloc(&t_xt.p, (size_t)std::min(cblk, std::max<int64_t>(I.n_chunks, 1)) * CHK * d * 4));
  for (int64_t c0 = 0; c0 < I.n_chunks; c0 += cblk) {
    int64_t nc = std::min(cblk, I.n_chunks - c0);
    const float* rows_blk = I.rows.as<float>() + c0 * CHK * d;
    PANO_CUDA(gemm_nt(kStore, (int)(nc * CHK), d, d, rows_blk, d, I.mu32.as<float>(),
                      I.T32.as<float>(), d, (float*)t_xt.p, d, nullptr, nullptr, st));
    if (precision == PANO_FP32) {
      pack_fp32_kernel<<<(unsigned)nc, 256, 0, st>>>(
          (float*)t_xt.p, rows_blk, (int64_t*)t_perm.p + c0 * CHK, c0, d, I.L,
          I.level_off_d.as<int32_t>(), I.mu32.as<float>(), I.c_trans, I.slices.as<float>(),
          I.tails.as<float>(), I.xn2.as<float>(), I.ex.as<float>(), I.ids.as<int32_t>());
      PANO_CUDA(cudaGetLastError());
    } else if (precision == PANO_BF16) {
      rc = launch_pack_bf16((float*)t_xt.p, rows_blk, (int64_t*)t_perm.p + c0 * CHK, c0, nc, d,
                            I.L, I.level_off_d.as<int32_t>(), I.mu32.as<float>(), I.c_trans,
                            I.slices.as<uint8_t>(), I.tails.as<float>(), I.xn2.as<float>(),
                            I.ex.as<float>(), I.ids.as<int32_t>(), st);
      if (rc) return rc;
    } else {
      rc = launch_pack_fp8((float*)t_xt.p, rows_blk, (int64_t*)t_perm.p + c0 * CHK, c0, nc, d,
                           I.L, I.level_off_d.as<int32_t>(), I.mu32.as<float>(), I.c_trans,
                           I.slices.as<uint8_t>(), I.tails.as<float>(), I.xn2.as<float>(),
                           I.ex.as<float>(), I.xscale.as<float>(), I.ids.as<int32_t>(), st);
      if (rc) return rc;
    }
  }
  PANO_CUDA(cudaStreamSynchronize(st));
  *out = idx.release();
  return PANO_OK;
}

}  // namespace pano

size_t pano_index::device_bytes() const {
  return T32.bytes + mu32.bytes + cent.bytes + cent_n2.bytes + chunk_off_d.bytes +
         list_size_d.bytes + level_off_d.bytes + slices.bytes + tails.bytes + xn2.bytes +
         ex.bytes + ids.bytes + rows.bytes + xscale.bytes + pq_codes.bytes + pq_codebook.bytes +
         pq_cent_t.bytes;
}
