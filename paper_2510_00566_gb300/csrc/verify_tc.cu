// BF16 storage + tensor-core level-wise verification (Eq. 2-3, Algorithm 1)
// for sm_103a.
//
// Index layout (precision PANO_BF16): chunks of 128 vectors; the level-l
// slice of a chunk is a 128 x w_l bf16 tile stored exactly as the swizzled
// K-major shared-memory image a tcgen05.mma operand needs (see tcgen05.cuh),
// so one bulk-async copy stages a whole level slice and one 32/64/128-byte
// copy stages a single row.  Widths are 16, 32 or multiples of 64.  The tail
// norms, norms and error bounds are those of the dequantised vector
// x^ = bf16(x~), with e_x bounding ||x^ - T~(x - mu~)||.
//
// Work item: (list, segment of <= 4 chunks, group of <= 64 queries).  The CTA
// walks the segment level by level (the paper's batch: every candidate moves
// one level before the next level starts, the threshold is refreshed per
// level).  Per (chunk, level) the partial products of all 128 candidates x
// the group's queries are one MMA chain: A = level tile of the chunk, B = the
// queries' level slices split into bf16 hi + lo parts (two MMAs into the same
// accumulator), accumulated across levels in tensor memory (4 chunks x 64
// columns = 256 TMEM columns; two CTAs share an SM).  The epilogue thread of TMEM lane t owns
// candidate row t: it reads its accumulators with tcgen05.ld and applies the
// separable form of the margined Eq. 3 test, which costs three FMAs and a
// compare per (candidate, query) pair.  Dead rows are not re-staged: at deep
// levels only live rows are copied (a row-granular gather), or the whole
// slice when most rows live.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "kernels_common.cuh"
#include "search.h"
#include "tcgen05.cuh"
#include "verify_tc.h"

namespace pano {
namespace {

constexpr int CH = TC_CHUNK;  // 128 rows (MMA M)
constexpr int QG = TC_QG;     // 64 queries per group (MMA N, padded to 16)
constexpr int S = TC_SEG;     // chunks per segment (4 x 64 = 256 TMEM columns)
constexpr int NBUF = 3;       // staged A tiles in flight
constexpr int NT = 128;       // thread t <-> TMEM lane t <-> chunk row t

// ------------------------------------------------------------------ build
// One CTA per chunk: bf16 tiles, tail norms / norms of the dequantised
// vectors and the bound on their distance to the exact transform.
__global__ void __launch_bounds__(256) pack_bf16_kernel(
    const float* __restrict__ xt, const float* __restrict__ rows,
    const int64_t* __restrict__ perm, int64_t chunk0, int d, int L,
    const int32_t* __restrict__ level_off, const float* __restrict__ mu, double c_trans,
    uint8_t* __restrict__ slices, float* __restrict__ tails, float* __restrict__ xn2,
    float* __restrict__ ex, int32_t* __restrict__ ids) {
  __shared__ int16_t lvl_of[8192 / 8];  // level of each 8-element chunk of a row
  const int64_t lc = blockIdx.x, g = chunk0 + lc;
  const float* xblk = xt + lc * CH * d;
  const int64_t* pb = perm + lc * CH;
  uint8_t* cbase = slices + g * (int64_t)CH * d * 2;
  for (int c8 = threadIdx.x; c8 < d / 8; c8 += blockDim.x) {
    int l = 0;
    while (level_off[l + 1] <= c8 * 8) ++l;
    lvl_of[c8] = (int16_t)l;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CH * (d / 8); e += blockDim.x) {
    const int r = e / (d / 8), c8 = e % (d / 8);
    const int l = lvl_of[c8];
    const int m = level_off[l], w = level_off[l + 1] - m;
    const bool valid = pb[r] >= 0;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = __float2bfloat16_rn(valid ? xblk[(int64_t)r * d + c8 * 8 + j] : 0.f);
    *reinterpret_cast<uint4*>(cbase + (size_t)m * CH * 2 + tc::swz_offset(r, c8 * 8 - m, CH, w)) =
        *reinterpret_cast<const uint4*>(v);
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  for (int i = warp; i < CH; i += blockDim.x / 32) {
    const int64_t slot = g * CH + i;
    const bool valid = pb[i] >= 0;
    const float* x = xblk + (int64_t)i * d;
    double suffix = 0.0, qerr = 0.0;
    for (int l = L - 1; l >= 0; --l) {
      double e = 0.0;
      if (valid)
        for (int j = level_off[l] + lane; j < level_off[l + 1]; j += 32) {
          double xf = x[j];
          double xh = __bfloat162float(__float2bfloat16_rn(x[j]));
          e += xh * xh;
          qerr += (xh - xf) * (xh - xf);
        }
      suffix += warp_sum_f64(e);
      if (lane == 0)
        tails[(g * (L + 1) + l) * CH + i] = __double2float_ru(sqrt(suffix * (1.0 + 1e-12)));
    }
    qerr = warp_sum_f64(qerr);
    double dev = 0.0;
    if (valid) {
      const float* r = rows + (lc * CH + i) * (int64_t)d;
      for (int j = lane; j < d; j += 32) {
        double v = (double)r[j] - (double)mu[j];
        dev += v * v;
      }
    }
    dev = warp_sum_f64(dev);
    if (lane == 0) {
      tails[(g * (L + 1) + L) * CH + i] = 0.f;
      xn2[slot] = (float)suffix;
      ex[slot] = valid ? __double2float_ru((sqrt(qerr) + c_trans * sqrt(dev)) * (1.0 + 1e-9)) : 0.f;
      ids[slot] = valid ? (int32_t)pb[i] : -1;
    }
  }
}

// ------------------------------------------------------------------ search
constexpr int TMEM_COLS = S * QG;  // 256: two CTAs can share an SM's tensor memory

struct Smem {
  uint32_t abytes, bbytes;
  uint32_t off_b_hi, off_b_lo, off_alive, off_cand, off_q, off_surv, total;
  __host__ __device__ Smem(int max_w) {
    // A buffers double as the [QG][CH] upper-bound scratch of the last level
    uint32_t a = (uint32_t)(CH * max_w * 2);
    const uint32_t ub_need = (uint32_t)(QG * CH * 4 + NBUF - 1) / NBUF;
    if (a < ub_need) a = ub_need;
    abytes = (a + 1023) & ~1023u;
    bbytes = (uint32_t)(QG * max_w * 2 + 1023) & ~1023u;
    off_b_hi = NBUF * abytes;
    off_b_lo = off_b_hi + bbytes;
    off_alive = off_b_lo + bbytes;                   // [S][CH][2] u32
    off_cand = off_alive + S * CH * 2 * 4;           // 5 x [S][CH] (Hx, rx, ex, id, sx)
    off_q = off_cand + 5 * S * CH * 4;               // 10 x [QG]
    off_surv = off_q + 10 * QG * 4;                  // [CH * QG] u16
    total = off_surv + CH * QG * 2;
  }
};

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t& bits, int b, int* fail) {
  const uint32_t par = (bits >> b) & 1u;
  bits ^= 1u << b;
  if (mbar_wait_bounded(bar, par)) return true;
  atomicOr(fail, 1);
  return false;
}

__global__ void __launch_bounds__(NT, 2) verify_tc_kernel(const VerifyTCArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const Smem lay(a.max_w);
  unsigned char* abuf = base;
  unsigned char* bhi = base + lay.off_b_hi;
  unsigned char* blo = base + lay.off_b_lo;
  uint32_t* alive = reinterpret_cast<uint32_t*>(base + lay.off_alive);
  float* cHx = reinterpret_cast<float*>(base + lay.off_cand);
  float* crx = cHx + S * CH;
  float* cex = crx + S * CH;
  int32_t* cid = reinterpret_cast<int32_t*>(cex + S * CH);
  float* csx = reinterpret_cast<float*>(cid + S * CH);
  int32_t* qid = reinterpret_cast<int32_t*>(base + lay.off_q);
  int32_t* qk = qid + QG;
  float* qnq = reinterpret_cast<float*>(qk + QG);
  float* qrq = qnq + QG;
  float* qeq = qrq + QG;
  float* qH = qeq + QG;
  float* qsq = qH + QG;
  float* qgr = qsq + QG;
  float* qE = qgr + QG;
  float* qtau = qE + QG;
  uint16_t* surv = reinterpret_cast<uint16_t*>(base + lay.off_surv);
  __shared__ __align__(8) uint64_t load_bar[NBUF], mma_bar[NBUF];
  __shared__ uint32_t tmem_base;
  __shared__ int s_item, s_nlive, s_nsurv, s_fail;
  __shared__ int live_list[S];
  __shared__ uint32_t rowlive[S][4];

  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&load_bar[b], 1);
      mbar_init(&mma_bar[b], 1);
    }
    fence_mbar_init();
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int L = a.L, d = a.d;
  uint32_t load_bits = 0, mma_bits = 0;
  unsigned long long st_pairs = 0, st_dims = 0, st_tiles = 0, st_bytes = 0, st_rerank = 0;
  const float g_slack = a.gslack;
  constexpr float kEval = 32.f * 5.9604645e-08f;  // evaluation slack of the separable test

  // per-query terms of the separable test for threshold tau (thread g < QG)
  auto set_query_terms = [&](int g, float tau, float sq) {
    const float st = tau == INFINITY ? 1e18f : fminf(__fsqrt_ru(__fdiv_ru(tau, a.lb_scale)), 1e18f);
    const float E = __fadd_ru(qeq[g], st);
    const float nq = qnq[g], rq = qrq[g];
    qH[g] = 0.5f * (nq - g_slack * nq - E * E - kEval * (rq + E) * (rq + E));
    qE[g] = E;
    qsq[g] = sq;
    qgr[g] = g_slack * rq;
  };

  while (true) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    const int64_t n_items = *a.n_items < a.items_cap ? *a.n_items : a.items_cap;
    if (item >= n_items || s_fail) break;
    const int4 it = a.items[item];
    const int64_t ch0 = a.chunk_off[it.x] + (int64_t)it.y * S;
    const int64_t chE = a.chunk_off[it.x + 1];
    const int nch = (int)((chE - ch0) < S ? (chE - ch0) : S);
    const int G = it.w;
    const int Npad = G <= 16 ? 16 : ((G + 15) & ~15);
    const uint32_t idesc = tc::idesc_bf16(CH, Npad);
    if (tid < QG) {
      int q = tid < G ? a.bucket[it.z + tid] : -1;
      qid[tid] = q;
      if (q >= 0) {
        float4 inf = a.qinfo[q];
        qnq[tid] = inf.x;
        qrq[tid] = inf.y;
        qeq[tid] = inf.z;
        qk[tid] = a.kq[q];
      } else {
        qnq[tid] = qrq[tid] = qeq[tid] = 0.f;
        qk[tid] = 0;
      }
    }
    for (int e = tid; e < S * CH; e += NT) {
      const int c = e / CH;
      if (c < nch) {
        const int64_t slot = (ch0 + c) * CH + (e % CH);
        const float nx = a.xn2[slot], rx = sqrtf(nx), exv = a.ex[slot];
        const float s2 = (rx + exv) * (rx + exv);
        cHx[e] = 0.5f * (nx - g_slack * nx - exv * exv - kEval * s2);
        crx[e] = rx;
        cex[e] = exv;
        cid[e] = a.ids[slot];
      } else {
        cHx[e] = crx[e] = cex[e] = 0.f;
        cid[e] = -1;
      }
    }
    __syncthreads();
    // initial liveness: valid candidate x query with k > 0
    uint32_t gm0 = 0, gm1 = 0;
    for (int g = 0; g < G; ++g)
      if (qk[g] > 0) {
        if (g < 32) gm0 |= 1u << g;
        else gm1 |= 1u << (g - 32);
      }
    for (int c = 0; c < S; ++c) {
      const bool v = c < nch && cid[c * CH + tid] >= 0;
      alive[(c * CH + tid) * 2] = v ? gm0 : 0u;
      alive[(c * CH + tid) * 2 + 1] = v ? gm1 : 0u;
      const unsigned bal = __ballot_sync(0xffffffffu, v && (gm0 | gm1));
      if (lane == 0) rowlive[c][warp] = bal;
    }
    bool completed = true;

    for (int l = 0; l < L; ++l) {
      const int m = a.level_off[l], w = a.level_off[l + 1] - m;
      const bool test = a.prune || l == L - 1;
      if (tid == 0) {
        int n = 0;
        for (int c = 0; c < nch; ++c)
          if (rowlive[c][0] | rowlive[c][1] | rowlive[c][2] | rowlive[c][3]) live_list[n++] = c;
        s_nlive = n;
      }
      __syncthreads();
      const int nlive = s_nlive;
      if (nlive == 0) {
        completed = false;
        break;
      }
      const uint8_t* lvl_src = a.slices + (size_t)m * CH * 2;
      const uint32_t tbytes = (uint32_t)w * CH * 2;
      const int rb = tc::row_bytes(w), npan = w >= 64 ? w / 64 : 1;
      // warp 0 stages live chunk i of this level into buffer i % NBUF
      auto issue_load = [&](int i) {
        const int c = live_list[i], b = i % NBUF;
        unsigned char* dst = abuf + (size_t)b * lay.abytes;
        const uint8_t* src = lvl_src + (ch0 + c) * (int64_t)CH * d * 2;
        const int nrows = __popc(rowlive[c][0]) + __popc(rowlive[c][1]) +
                          __popc(rowlive[c][2]) + __popc(rowlive[c][3]);
        if (nrows * 2 >= CH || l == 0) {
          if (lane == 0) {
            mbar_arrive_expect_tx(&load_bar[b], tbytes);
            bulk_g2s(dst, src, tbytes, &load_bar[b]);
          }
          st_bytes += (lane == 0) ? tbytes : 0;
        } else {
          if (lane == 0) mbar_arrive_expect_tx(&load_bar[b], (uint32_t)nrows * w * 2);
          __syncwarp();
          for (int r = lane; r < CH; r += 32)
            if ((rowlive[c][r >> 5] >> (r & 31)) & 1u)
              for (int p = 0; p < npan; ++p) {
                const uint32_t o = (uint32_t)p * CH * 128 + (uint32_t)r * rb;
                bulk_g2s(dst + o, src + o, (uint32_t)rb, &load_bar[b]);
              }
          st_bytes += (lane == 0) ? (unsigned long long)nrows * w * 2 : 0;
        }
      };
      auto issue_mma = [&](int i) {
        const int c = live_list[i], b = i % NBUF;
        const uint32_t a0 = smem_u32(abuf + (size_t)b * lay.abytes);
        const uint32_t h0 = smem_u32(bhi), l0 = smem_u32(blo);
        const uint32_t dt = tbase + (uint32_t)(c * QG);
        for (int s = 0; s < w / 16; ++s) {
          const uint64_t ad = tc::kstep_desc(a0, s, CH, w);
          tc::mma_bf16(dt, ad, tc::kstep_desc(h0, s, Npad, w), idesc, (l > 0 || s > 0) ? 1u : 0u);
          tc::mma_bf16(dt, ad, tc::kstep_desc(l0, s, Npad, w), idesc, 1u);
        }
        tc::mma_commit(&mma_bar[b]);
      };
      // the first tiles are in flight while the query tiles are built
      if (warp == 0)
        for (int i = 0; i < nlive && i < NBUF; ++i) issue_load(i);
      // candidates' tail norms after level l (all loads issued first)
      {
        float tv[S * CH / NT];
#pragma unroll
        for (int u = 0; u < S * CH / NT; ++u) {
          const int e = tid + u * NT;
          tv[u] = e < nch * CH ? a.tails[((ch0 + e / CH) * (L + 1) + l + 1) * CH + (e % CH)] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < S * CH / NT; ++u) csx[tid + u * NT] = tv[u];
      }
      // threshold refresh: running top-k and the warm-start seed
      if (tid < QG) {
        const int q = qid[tid];
        if (q >= 0 && qk[tid] > 0) {
          unsigned long long key = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + qk[tid] - 1);
          float tau = key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f);
          tau = fminf(tau, a.tau_seed[q]);
          qtau[tid] = tau;
          set_query_terms(tid, tau, a.qtail[(int64_t)q * (L + 1) + l + 1]);
        } else {
          qtau[tid] = -1.f;
          qH[tid] = -INFINITY;
          qE[tid] = qsq[tid] = qgr[tid] = 0.f;
        }
      }
      // B tiles: the group's level-l query slices as bf16 hi / lo
      for (int e = tid; e < Npad * (w / 8); e += NT) {
        const int g = e / (w / 8), c8 = e % (w / 8);
        __align__(16) __nv_bfloat16 hi[8], lo[8];
        if (g < G) {
          const float* src = a.qt + (int64_t)qid[g] * d + m + c8 * 8;
          const float4 f0 = *reinterpret_cast<const float4*>(src);
          const float4 f1 = *reinterpret_cast<const float4*>(src + 4);
          const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
          for (int j = 0; j < 8; ++j) tc::split_bf16(f[j], hi[j], lo[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) hi[j] = lo[j] = __float2bfloat16_rn(0.f);
        }
        const uint32_t off = tc::swz_offset(g, c8 * 8, Npad, w);
        *reinterpret_cast<uint4*>(bhi + off) = *reinterpret_cast<const uint4*>(hi);
        *reinterpret_cast<uint4*>(blo + off) = *reinterpret_cast<const uint4*>(lo);
      }
      fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        if (wait_phase(&load_bar[0], load_bits, 0, &s_fail)) issue_mma(0);
      }
      st_tiles += (tid == 0) ? nlive : 0;
      for (int i = 0; i < nlive; ++i) {
        const int c = live_list[i], b = i % NBUF;
        if (tid == 0 && i + 1 < nlive) {
          const int b1 = (i + 1) % NBUF;
          if (wait_phase(&load_bar[b1], load_bits, b1, &s_fail)) issue_mma(i + 1);
        }
        const bool ok = wait_phase(&mma_bar[b], mma_bits, b, &s_fail);
        tc::fence_after_sync();
        // epilogue: candidate row `tid` of chunk c against the group
        uint32_t w0 = alive[(c * CH + tid) * 2], w1 = alive[(c * CH + tid) * 2 + 1];
        const bool any_warp =
            __any_sync(0xffffffffu, (w0 | w1) != 0) && __all_sync(0xffffffffu, ok);
        if (any_warp) {
          const float sx = csx[c * CH + tid], rx = crx[c * CH + tid], exv = cex[c * CH + tid];
          const float Hx = cHx[c * CH + tid];
          if (a.collect) {
            st_pairs += __popc(w0) + __popc(w1);
            st_dims += (unsigned long long)(__popc(w0) + __popc(w1)) * w;
          }
          float v[32];
          tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG), v);
          if (test) {
#pragma unroll
            for (int g = 0; g < 32; ++g)
              if ((w0 >> g) & 1u) {
                const float P = fmaf(qE[g], exv, fmaf(qgr[g], rx, fmaf(qsq[g], sx, v[g])));
                if (P < qH[g] + Hx) w0 &= ~(1u << g);
              }
          }
          if (Npad > 32) {
            tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG + 32), v);
            if (test) {
#pragma unroll
              for (int g = 0; g < 32; ++g)
                if ((w1 >> g) & 1u) {
                  const float P =
                      fmaf(qE[g + 32], exv, fmaf(qgr[g + 32], rx, fmaf(qsq[g + 32], sx, v[g])));
                  if (P < qH[g + 32] + Hx) w1 &= ~(1u << g);
                }
            }
          }
          alive[(c * CH + tid) * 2] = w0;
          alive[(c * CH + tid) * 2 + 1] = w1;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, (w0 | w1) != 0);
        if (lane == 0) rowlive[c][warp] = bal;
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
          const int go = __shfl_sync(0xffffffffu, (i + NBUF < nlive && !s_fail) ? 1 : 0, 0);
          if (go) issue_load(i + NBUF);
        }
      }
      if (s_fail) {
        completed = false;
        break;
      }
    }
    if (s_fail) break;
    if (!completed) continue;

    // Last level done: per chunk, the k-th smallest upper bound of each
    // query tightens its threshold (at the last level UB ~ LB ~ exact), then
    // the pairs are tested again, so only ~k per query reach re-ranking.
    float* ub = reinterpret_cast<float*>(abuf);  // [QG][CH]
    for (int c = 0; c < nch; ++c) {
      if (!(rowlive[c][0] | rowlive[c][1] | rowlive[c][2] | rowlive[c][3])) continue;
      const uint32_t w0 = alive[(c * CH + tid) * 2], w1 = alive[(c * CH + tid) * 2 + 1];
      const bool any_warp = __any_sync(0xffffffffu, (w0 | w1) != 0);
      if (any_warp) {
        const float rx = crx[c * CH + tid], exv = cex[c * CH + tid];
        const float nx2 = a.xn2[(ch0 + c) * CH + tid];
        float v[32];
        for (int half = 0; half < (Npad > 32 ? 2 : 1); ++half) {
          tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG + 32 * half), v);
          const uint32_t wm = half ? w1 : w0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int g = 32 * half + j;
            float u = INFINITY;
            if ((wm >> j) & 1u) {
              const float A = qnq[g] + nx2 - 2.f * v[j];
              const float Ss = qrq[g] + rx;
              const float r = __fadd_ru(__fsqrt_ru(fmaxf(A + g_slack * Ss * Ss, 0.f)),
                                        qeq[g] + exv);
              u = __fmul_ru(__fmul_ru(r, r), a.ub_scale);
            }
            ub[g * CH + tid] = u;
          }
        }
        if (Npad <= 32)
          for (int g = 32; g < 64; ++g) ub[g * CH + tid] = INFINITY;
      } else {
        for (int g = 0; g < 64; ++g) ub[g * CH + tid] = INFINITY;
      }
      __syncthreads();
      for (int g = warp; g < G; g += NT / 32) {
        const float t = warp_kth_smallest(ub + g * CH, CH, qk[g]);
        if (lane == 0 && t < qtau[g]) qtau[g] = t;
      }
      __syncthreads();
    }
    if (tid < G && qk[tid] > 0) set_query_terms(tid, qtau[tid], 0.f);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // survivors of the tightened test: exact distances on the original rows
    for (int c = 0; c < nch; ++c) {
      if (tid == 0) s_nsurv = 0;
      uint32_t w0 = alive[(c * CH + tid) * 2], w1 = alive[(c * CH + tid) * 2 + 1];
      const bool any_warp = __any_sync(0xffffffffu, (w0 | w1) != 0);
      if (any_warp) {
        const float rx = crx[c * CH + tid], exv = cex[c * CH + tid], Hx = cHx[c * CH + tid];
        float v[32];
        for (int half = 0; half < (Npad > 32 ? 2 : 1); ++half) {
          tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG + 32 * half), v);
          uint32_t& wm = half ? w1 : w0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int g = 32 * half + j;
            if ((wm >> j) & 1u) {
              const float P = fmaf(qE[g], exv, fmaf(qgr[g], rx, v[j]));
              if (P < qH[g] + Hx) wm &= ~(1u << j);
            }
          }
        }
      }
      __syncthreads();
      for (int g = 0; g < 64; ++g) {
        const uint32_t bit = g < 32 ? (w0 >> g) & 1u : (w1 >> (g - 32)) & 1u;
        if (bit) surv[atomicAdd(&s_nsurv, 1)] = (uint16_t)((tid << 6) | g);
      }
      __syncthreads();
      const int ns = s_nsurv;
      for (int s = warp; s < ns; s += NT / 32) {
        const int row = surv[s] >> 6, g = surv[s] & 63;
        const int q = qid[g];
        const int64_t slot = (ch0 + c) * CH + row;
        const float dist = exact_sqdist_warp(a.qorig + (int64_t)q * d, a.rows + slot * d, d);
        if (lane == 0)
          topk_insert(a.topk + (int64_t)q * a.k_max, qk[g], make_key(dist, cid[c * CH + row]));
      }
      st_rerank += (tid == 0) ? ns : 0;
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
    // the scratch written through the generic proxy is refilled by
    // bulk-async copies in the next item
    fence_proxy_async_smem();
  }
  if (s_fail && tid == 0) atomicOr(a.err, kErrTimeout);
  if (a.collect) {
    unsigned long long v = st_pairs, dv = st_dims;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, off);
      dv += __shfl_xor_sync(0xffffffffu, dv, off);
    }
    if (lane == 0) {
      atomicAdd(&a.stats[0], v);
      atomicAdd(&a.stats[5], dv);
    }
    if (tid == 0) {
      atomicAdd(&a.stats[1], st_tiles);
      atomicAdd(&a.stats[3], st_rerank);
    }
    if (lane == 0) atomicAdd(&a.stats[2], st_bytes);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace

int launch_pack_bf16(const float* xt, const float* rows, const int64_t* perm, int64_t chunk0,
                     int64_t nchunks, int d, int L, const int32_t* level_off, const float* mu,
                     double c_trans, uint8_t* slices, float* tails, float* xn2, float* ex,
                     int32_t* ids, cudaStream_t st) {
  PANO_CHECK(d % 8 == 0 && d <= 8192, PANO_EINVAL, "bf16 storage needs d % 8 == 0, d <= 8192");
  pack_bf16_kernel<<<(unsigned)nchunks, 256, 0, st>>>(xt, rows, perm, chunk0, d, L, level_off,
                                                      mu, c_trans, slices, tails, xn2, ex, ids);
  PANO_CUDA(cudaGetLastError());
  return PANO_OK;
}

size_t verify_tc_smem(int max_w) {
  // at most two CTAs per SM: each owns 256 of the 512 TMEM columns
  return std::max<size_t>(Smem(max_w).total + 1024, 80 * 1024);
}

int launch_verify_tc(const VerifyTCArgs& a, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    attr_err = cudaFuncGetAttributes(&fa, verify_tc_kernel);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(verify_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin - (int)fa.sharedSizeBytes);
  });
  PANO_CUDA(attr_err);
  const size_t smem = verify_tc_smem(a.max_w);
  int dev = 0, sms = 0, bps = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  PANO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PANO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, verify_tc_kernel, NT, smem));
  if (bps < 1) return fail(PANO_EINVAL, "tensor-core verify tile does not fit in shared memory");
  bps = std::min(bps, 2);  // two CTAs x 256 TMEM columns fill the SM's tensor memory
  verify_tc_kernel<<<sms * bps, NT, smem, st>>>(a);
  PANO_CUDA(cudaGetLastError());
  return PANO_OK;
}

}  // namespace pano
