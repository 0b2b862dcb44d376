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
// columns = 256 TMEM columns; two CTAs share an SM).  One warp of the CTA
// issues the MMA chains and the tile copies; the other eight test: candidate
// row t is owned by two epilogue threads (warps w and w + 4 read the same
// TMEM lane quarter), one per half of the query group, each reading its 32
// accumulators with tcgen05.ld and applying the separable form of the
// margined Eq. 3 test (three FMAs and a compare per (candidate, query) pair)
// at the levels of the bound-test schedule.  A chunk whose rows are all dead
// is neither copied nor multiplied again.
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
// epilogue thread t < NE: TMEM lane / chunk row t % 128 and query half
// t / 128 (queries 32h .. 32h+31 are TMEM columns 32h.. of each chunk's
// accumulator); warps w and w + 4 share a lane quarter.  Warp NE / 32 issues
// the MMA chains and the tile copies.
constexpr int NE = 256;
constexpr int NT = NE + 32;
constexpr int kIssuer = NE / 32;

// Barrier of the NE epilogue threads alone (named barrier 1).
__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NE) : "memory");
}
__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

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

// FP8 storage: each vector gets a power-of-two scale s_x = 2^e (the least with
// max |x~_j| / s_x <= 448, E4M3's largest finite value; e clamped to [-60,
// 60]) and its elements are stored as E4M3 of x~ / s_x, rounded to nearest.
// Level tiles have the byte layout of bf16 tiles of half the width; tail
// norms, norms and e_x are those of x^ = s_x e4m3(x~ / s_x).  Widths are 32,
// 64 or multiples of 128, so 16-element groups never straddle a level.
__global__ void __launch_bounds__(256) pack_fp8_kernel(
    const float* __restrict__ xt, const float* __restrict__ rows,
    const int64_t* __restrict__ perm, int64_t chunk0, int d, int L,
    const int32_t* __restrict__ level_off, const float* __restrict__ mu, double c_trans,
    uint8_t* __restrict__ slices, float* __restrict__ tails, float* __restrict__ xn2,
    float* __restrict__ ex, float* __restrict__ xscale, int32_t* __restrict__ ids) {
  __shared__ int16_t lvl_of[8192 / 16];  // level of each 16-element group of a row
  __shared__ float s_scale[CH], s_inv[CH];
  const int64_t lc = blockIdx.x, g = chunk0 + lc;
  const float* xblk = xt + lc * CH * d;
  const int64_t* pb = perm + lc * CH;
  uint8_t* cbase = slices + g * (int64_t)CH * d;
  for (int c16 = threadIdx.x; c16 < d / 16; c16 += blockDim.x) {
    int l = 0;
    while (level_off[l + 1] <= c16 * 16) ++l;
    lvl_of[c16] = (int16_t)l;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  for (int i = warp; i < CH; i += blockDim.x / 32) {
    float m = 0.f;
    if (pb[i] >= 0)
      for (int j = lane; j < d; j += 32) m = fmaxf(m, fabsf(xblk[(int64_t)i * d + j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    int e = 0;
    if (m > 0.f) frexpf(m / 448.f, &e);  // m / 448 < 2^e, so m / 2^e < 448
    e = max(-60, min(60, e));
    if (lane == 0) {
      s_scale[i] = ldexpf(1.f, e);
      s_inv[i] = ldexpf(1.f, -e);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CH * (d / 16); e += blockDim.x) {
    const int r = e / (d / 16), c16 = e % (d / 16);
    const int l = lvl_of[c16];
    const int m = level_off[l], w = level_off[l + 1] - m;
    const bool valid = pb[r] >= 0;
    const float inv = s_inv[r];
    __align__(16) uint8_t v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = tc::f32_to_e4m3(valid ? xblk[(int64_t)r * d + c16 * 16 + j] * inv : 0.f);
    *reinterpret_cast<uint4*>(cbase + (size_t)m * CH +
                              tc::swz_offset(r, (c16 * 16 - m) / 2, CH, w / 2)) =
        *reinterpret_cast<const uint4*>(v);
  }
  for (int i = warp; i < CH; i += blockDim.x / 32) {
    const int64_t slot = g * CH + i;
    const bool valid = pb[i] >= 0;
    const float* x = xblk + (int64_t)i * d;
    const float sc = s_scale[i], inv = s_inv[i];
    double suffix = 0.0, qerr = 0.0;
    for (int l = L - 1; l >= 0; --l) {
      double e = 0.0;
      if (valid)
        for (int j = level_off[l] + lane; j < level_off[l + 1]; j += 32) {
          const double xf = x[j];
          const double xh = (double)(tc::e4m3_to_f32(tc::f32_to_e4m3(x[j] * inv)) * sc);
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
      xscale[slot] = sc;
      ids[slot] = valid ? (int32_t)pb[i] : -1;
    }
  }
}

// ------------------------------------------------------------------ search
// One work item = (list, segment of S chunks, group of <= QG queries).  Each
// chunk owns an A buffer.  Per level the issue warp issues every live
// chunk's MMA chain as soon as its tile has landed; the epilogue warps test
// the chunks in order as their accumulators complete and tell the issue warp
// (an mbarrier per chunk) when all of them have read one, whereupon a chunk
// that stays live has its next level's tile staged into its buffer while the
// other chunks are still tested.  The next level's tail norms and threshold
// terms are loaded into the epilogue threads' registers at the start of a
// level; they and the next level's B tiles (built from the query slices in
// global memory) are written to shared memory at its end: for BF16 by each
// epilogue warp once its own tests are done, before the level's one CTA
// barrier; for FP8 after that barrier, with a second one.  A live chunk's
// bound is tested at the levels of the schedule (l % test_every == 0), at the
// last level, and at every level once it is nearly dead.
constexpr int TMEM_COLS = S * QG;  // 256: two CTAs share an SM's tensor memory
constexpr int AW = (QG + 31) / 32;  // alive-mask words per candidate row
// a chunk with at most this many live rows is tested at every level: only a
// test that leaves no live row retires the chunk's copies and MMAs
constexpr int kTestRows = 16;
static_assert(QG == 64 && AW == 2 && TMEM_COLS <= 256, "two query halves; two CTAs per SM");

struct Smem {
  uint32_t abytes, bbytes;
  uint32_t off_b_hi, off_b_lo, off_alive, off_cand, off_q, total;
  static constexpr int kPend = 256;  // deferred re-rank entries (static shared memory)
  // eb: bytes per stored element (2 BF16, 1 FP8).  The B buffers hold the
  // bf16 hi and lo tiles, or the three E4M3 term tiles (two in the first).
  __host__ __device__ Smem(int max_w, int eb) {
    // after the last level the A buffers hold the [QG][S*CH] bf16 upper
    // bounds, then the [CH * QG] survivor list and their lower bounds
    uint32_t a = (uint32_t)(CH * max_w * eb);
    const uint32_t per = (uint32_t)(QG * S * CH * 2 + S - 1) / S;
    if (a < per) a = per;
    abytes = (a + 1023) & ~1023u;
    bbytes = (uint32_t)(QG * max_w * 2 + 1023) & ~1023u;
    off_b_hi = S * abytes;
    off_b_lo = off_b_hi + bbytes;
    off_alive = off_b_lo + bbytes;                   // [S][AW][CH] u32 (a warp's rows: consecutive words)
    off_cand = off_alive + S * CH * AW * 4;  // 7 x [S][CH] (Hx, rx, ex, id, sx, FP8 factor, sx')
    off_q = off_cand + 7 * S * CH * 4;       // 2 x [QG] float4 + 6 x [QG]
    total = off_q + 14 * QG * 4;
  }
};

// The deferred pairs are checked against their queries' thresholds of the
// moment and against each other (below); the rest get their exact distance
// and top-k insertion, in two passes: first each query's k kept pairs of
// smallest lower bound (ties by entry), whose exact distances usually set
// its threshold, then the others that still pass the threshold.  All threads
// epilogue threads call it (one thread per entry at most: kPend <= NE); kept out of
// line so that it does not add to the level loop's registers.  Returns the
// number re-ranked (thread 0; 0 elsewhere).
__device__ __noinline__ int flush_pending(const VerifyTCArgs& a, int np,
                                          const int64_t* __restrict__ pslot,
                                          const int32_t* __restrict__ pq,
                                          const int32_t* __restrict__ pid,
                                          float* __restrict__ plb,
                                          const float* __restrict__ pub, uint16_t* keep,
                                          uint16_t* rank, int* s_cnt) {
  const int tid = threadIdx.x, warp = tid / 32, nw = NE / 32;
  if (tid == 0) s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
  epi_sync();
  auto tau_of = [&](int q, int kk) {
    const unsigned long long key = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + kk - 1);
    return fminf(key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f),
                 __ldcg(a.tau_seed + q));
  };
  // a pair is re-ranked unless its lower bound exceeds the threshold or the
  // upper bounds of k pending pairs of the same query (all k are closer)
  if (tid < np) {
    const int s = tid, q = pq[s], kk = a.kq[q];
    const float lb = plb[s];
    bool keep_s = !(lb > tau_of(q, kk));
    if (keep_s) {
      int below = 0;
      for (int o = 0; o < np && below < kk; ++o)
        below += (pq[o] == q) & (__fmul_ru(pub[o], 1.000001f) < lb);
      keep_s = below < kk;
    }
    if (keep_s) keep[atomicAdd(&s_cnt[0], 1)] = (uint16_t)s;
  }
  epi_sync();
  const int nk = s_cnt[0];
  if (tid < nk && (a.d & 3) == 0)  // all kept rows head for L2 at once
    prefetch_l2(a.rows + pslot[keep[tid]] * a.d, (uint32_t)a.d * 4);
  bool first = false;
  if (tid < nk) {  // rank among the kept pairs of its query
    const int s = keep[tid], q = pq[s];
    const float lb = plb[s];
    int r = 0;
    for (int j = 0; j < nk; ++j) {
      const int o = keep[j];
      r += (pq[o] == q) & ((plb[o] < lb) | ((plb[o] == lb) & (o < s)));
    }
    first = r < a.kq[q];
    rank[tid] = first ? 1 : 0;
    if (first) atomicAdd(&s_cnt[1], 1);
  }
  epi_sync();
  // exact distances (a warp each; they replace the lower bounds), then the
  // top-k insertions (a thread each, so their chains overlap)
  auto rerank = [&](const uint16_t* list, int n, const uint16_t* sel) {
    for (int i = warp; i < n; i += nw) {
      if (sel && !sel[i]) continue;
      const int s = list[i];
      const float dist =
          exact_sqdist_warp_wide(a.qorig + (int64_t)pq[s] * a.d, a.rows + pslot[s] * a.d, a.d);
      if ((tid & 31) == 0) plb[s] = dist;
    }
    epi_sync();
    if (tid < n && (!sel || sel[tid])) {
      const int s = list[tid], q = pq[s];
      topk_insert_thread(a.topk + (int64_t)q * a.k_max, a.kq[q], make_key(plb[s], pid[s]));
    }
    epi_sync();
  };
  rerank(keep, nk, rank);
  // the others, against the thresholds of the moment (rank now lists them)
  if (tid < nk && !first) {
    const int s = keep[tid], q = pq[s];
    if (!(plb[s] > tau_of(q, a.kq[q]))) rank[atomicAdd(&s_cnt[2], 1)] = (uint16_t)s;
  }
  epi_sync();
  rerank(rank, s_cnt[2], nullptr);
  return tid == 0 ? s_cnt[1] + s_cnt[2] : 0;
}

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t& bits, int b, int* fail) {
  const uint32_t par = (bits >> b) & 1u;
  bits ^= 1u << b;
  if (mbar_wait_bounded(bar, par)) return true;
  atomicOr(fail, 1);
  return false;
}

// FP8 = false: BF16 tiles, kind::f16 MMAs with the query split into bf16 hi +
// lo.  FP8 = true: E4M3 tiles (the byte layout of bf16 tiles of half the
// width), kind::f8f6f4 MMAs with the query split into three E4M3 terms at one
// power-of-two scale per group; the accumulator times the row's factor
// s_x / (group scale) is the partial product.
template <bool FP8>
__global__ void __launch_bounds__(NT, 2) verify_tc_kernel(const VerifyTCArgs a) {
  constexpr int EB = FP8 ? 1 : 2;  // bytes per stored element
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const Smem lay(a.max_w, EB);
  unsigned char* abuf = base;
  unsigned char* bhi = base + lay.off_b_hi;
  unsigned char* blo = base + lay.off_b_lo;
  uint32_t* alive = reinterpret_cast<uint32_t*>(base + lay.off_alive);
  float* cHx = reinterpret_cast<float*>(base + lay.off_cand);
  float* crx = cHx + S * CH;
  float* cex = crx + S * CH;
  int32_t* cid = reinterpret_cast<int32_t*>(cex + S * CH);
  float* csx = reinterpret_cast<float*>(cid + S * CH);
  float* cfr = csx + S * CH;  // FP8: s_x / group scale, the accumulator's factor
  // per-query terms of the separable test: (E, g*rq, sq, H)
  float4* qterm = reinterpret_cast<float4*>(base + lay.off_q);  // [2][QG]
  int32_t* qid = reinterpret_cast<int32_t*>(qterm + 2 * QG);
  // BF16: each epilogue warp writes the next level's B tiles, tail norms and
  // query terms as soon as its own tests of the level are done (the level's
  // MMAs have completed by then), into a second tail / query-term buffer
  // chosen by level parity, so one CTA barrier per level suffices.  FP8 (its
  // three-term B tiles) measured faster with the writes after the level's
  // barrier and a second barrier.
  constexpr bool kEarly = !FP8;
  // level l's tail norms and query terms (two buffers by level parity when
  // the next level's are written while this level is still being tested)
  float* const csx1 = cfr + S * CH;
  auto csx_of = [&](int l) { return (kEarly && (l & 1)) ? csx1 : csx; };
  auto qterm_of = [&](int l) { return (kEarly && (l & 1)) ? qterm + QG : qterm; };
  int32_t* qk = qid + QG;
  float* qnq = reinterpret_cast<float*>(qk + QG);
  float* qrq = qnq + QG;
  float* qeq = qrq + QG;
  float* qtau = qeq + QG;
  uint16_t* ub16 = reinterpret_cast<uint16_t*>(abuf);  // [QG][S*CH] bf16 bits
  uint16_t* surv = reinterpret_cast<uint16_t*>(abuf);  // [CH * QG], after ub16 is read
  // [32][NE] each thread's last accumulators (slot j of thread t at j*NE + t)
  float* vdump = reinterpret_cast<float*>(abuf + CH * QG * 2);
  // deferred re-rank list: (slot, query, id, lower bound) per pair
  __shared__ int64_t pslot[Smem::kPend];
  __shared__ int32_t pq[Smem::kPend], pid[Smem::kPend];
  __shared__ float plb[Smem::kPend], pub[Smem::kPend];
  __shared__ uint16_t keep[Smem::kPend], rnk[Smem::kPend];
  __shared__ int s_flush[3];
  static_assert(Smem::kPend <= NE, "the flush gives each pending pair one thread");
  // per chunk: its tile has landed / its MMAs are done / every epilogue warp
  // has read its accumulator (count NE / 32)
  __shared__ __align__(8) uint64_t load_bar[S], mma_bar[S], epi_bar[S];
  __shared__ uint32_t tmem_base;
  __shared__ int s_item, s_nsurv, s_fail, s_npend;
  // FP8: the group's largest |q~_j| (as bits), query scale and the absolute
  // bound of the query split's underflow per unit of |x|_2
  __shared__ unsigned int s_qmax;
  __shared__ float s_qs, s_cunder;
  __shared__ uint32_t rowlive[S][NE / 32];  // per epilogue warp: its rows live in its half
  // the chunks live at level l and the chunks whose bound is tested there
  // (bit c), by level parity: written by the issue warp from the liveness
  // words it has acquired (before the CTA barrier that ends the previous
  // level), so every thread reads the same masks even while fast warps
  // already update rowlive for level l
  __shared__ uint32_t s_live[2], s_test[2];
  __shared__ uint32_t s_gm[2];  // the group's queries with k > 0 (two halves)

  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const int row = tid & (CH - 1), half = tid / CH;
  const bool epi = tid < NE;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int c = 0; c < S; ++c) {
      mbar_init(&load_bar[c], 1);
      mbar_init(&mma_bar[c], 1);
      mbar_init(&epi_bar[c], NE / 32);
    }
    fence_mbar_init();
    s_fail = 0;
    s_npend = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int L = a.L, d = a.d;
  uint32_t load_bits = 0, mma_bits = 0, epi_bits = 0;
  // counters (collect_stats) live in shared memory, off the registers:
  // [0] pairs, [1] dims, [2] tiles, [3] bytes, [4] reranked, [5] live-row
  // bytes; section cycles
  __shared__ unsigned long long s_stat[6], s_sec[8];
  __shared__ long long s_tmark, s_tkernel;
  if (tid == 0) {
    for (int i = 0; i < 6; ++i) s_stat[i] = 0;
    for (int i = 0; i < 8; ++i) s_sec[i] = 0;
    s_tkernel = s_tmark = clock64();
  }
  auto section = [&](int i) {  // charge the time since the last mark to section i
    if (a.collect && tid == 0) {
      const long long now = clock64();
      s_sec[i] += (unsigned long long)(now - s_tmark);
      s_tmark = now;
    }
  };
  const float g_slack = a.gslack;
  constexpr float kEval = 32.f * 5.9604645e-08f;  // evaluation slack of the separable test

  // threshold -> per-query terms of the separable test (thread g < QG)
  auto set_query_terms = [&](int g, float tau, float sq, float4* qt) {
    // sqrt(tau / lb_scale), bounded from above (a product by the rounded-up
    // reciprocal, itself rounded up, bounds the quotient from above)
    const float st = tau == INFINITY ? 1e18f : fminf(sqrt_up(__fmul_ru(tau, a.inv_lb_up)), 1e18f);
    const float E = __fadd_ru(qeq[g], st);
    const float nq = qnq[g], rq = qrq[g];
    // FP8: the query split's underflow error (at most s_cunder |x|_2 on the
    // partial product) joins the g rq coefficient of rx
    qt[g] = make_float4(E, FP8 ? fmaf(g_slack, rq, s_cunder) : g_slack * rq, sq,
                           0.5f * (nq - g_slack * nq - E * E - kEval * (rq + E) * (rq + E)));
    qtau[g] = tau;
  };
  auto rerank_pending = [&](int np) {
    const int nk = flush_pending(a, np, pslot, pq, pid, plb, pub, keep, rnk, s_flush);
    if (a.collect && tid == 0) s_stat[4] += nk;
  };
  auto chunk_live = [&](int c) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < NE / 32; ++i) m |= rowlive[c][i];
    return m != 0u;
  };

  while (true) {
    if (tid == 0) {
      s_item = atomicAdd(a.counter, 1);
      s_qmax = 0u;
    }
    __syncthreads();
    const int item = s_item;
    const int64_t n_items = *a.n_items < a.items_cap ? *a.n_items : a.items_cap;
    if (item >= n_items || s_fail) break;
    if (a.collect && tid == 0) s_tmark = clock64();
    const int4 it = a.items[item];
    const int64_t ch0 = a.chunk_off[it.x] + (int64_t)it.y * S;
    const int64_t chE = a.chunk_off[it.x + 1];
    const int nch = (int)((chE - ch0) < S ? (chE - ch0) : S);
    const int G = it.w;
    const int Npad = G <= 16 ? 16 : ((G + 15) & ~15);
    const uint32_t idesc = FP8 ? tc::idesc_e4m3(CH, Npad) : tc::idesc_bf16(CH, Npad);
    const uint8_t* item_src = a.slices + ch0 * (int64_t)CH * d * EB;

    // stage chunk c's level-l tile: one bulk-async copy of the whole tile
    // (issue warp).  Copying only the 8-row atoms that still hold a live row
    // saves bytes, but its one copy instruction per atom on the issue warp's
    // path cost more than the bytes (HBM is far from busy here), so every
    // live chunk's tile is copied whole.
    auto issue_load = [&](int c, int l) {
      const int m = a.level_off[l], w = a.level_off[l + 1] - m;
      const uint32_t tbytes = (uint32_t)w * CH * EB;
      unsigned char* dst = abuf + (size_t)c * lay.abytes;
      const uint8_t* src = item_src + (int64_t)c * CH * d * EB + (size_t)m * CH * EB;
      if (lane == 0) {
        mbar_arrive_expect_tx(&load_bar[c], tbytes);
        bulk_g2s(dst, src, tbytes, &load_bar[c]);
        if (a.collect) atomicAdd(&s_stat[3], (unsigned long long)tbytes);
      }
    };
    // B tiles for level l, 8 query elements at a time: bf16 hi / lo parts,
    // or (FP8) three E4M3 terms of the scaled query in three tiles
    auto store_b = [&](int g, int c8, int w, const float (&f)[8]) {
      if (FP8) {
        const float qs = s_qs;
        __align__(8) uint8_t t0[8], t1[8], t2[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) tc::split3_e4m3(f[j] * qs, t0[j], t1[j], t2[j]);
        const uint32_t off = tc::swz_offset(g, c8 * 4, Npad, w / 2);
        *reinterpret_cast<uint2*>(bhi + off) = *reinterpret_cast<const uint2*>(t0);
        *reinterpret_cast<uint2*>(bhi + QG * a.max_w + off) = *reinterpret_cast<const uint2*>(t1);
        *reinterpret_cast<uint2*>(blo + off) = *reinterpret_cast<const uint2*>(t2);
      } else {
        __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) tc::split_bf16(f[j], hi[j], lo[j]);
        const uint32_t off = tc::swz_offset(g, c8 * 8, Npad, w);
        *reinterpret_cast<uint4*>(bhi + off) = *reinterpret_cast<const uint4*>(hi);
        *reinterpret_cast<uint4*>(blo + off) = *reinterpret_cast<const uint4*>(lo);
      }
    };
    // (two 8-element groups per thread per round: both loads are in flight
    // before either is converted)
    auto build_b = [&](int l, int first_chunk) {
      const int m = a.level_off[l], w = a.level_off[l + 1] - m;
      const int n8 = w / 8, total = Npad * n8;
      const bool p2 = (n8 & (n8 - 1)) == 0;  // widths 16, 32, 64, 128, 256: a shift
      const int sh = __ffs(n8) - 1;
      for (int e0 = tid + first_chunk * NE; e0 < total; e0 += 2 * NE) {
        float f[2][8];
        int gg[2], cc[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int e = e0 + u * NE;
          gg[u] = p2 ? e >> sh : e / n8;
          cc[u] = p2 ? e & (n8 - 1) : e % n8;
#pragma unroll
          for (int j = 0; j < 8; ++j) f[u][j] = 0.f;
          if (e < total && gg[u] < G) {
            const float* src = a.qt + (int64_t)qid[gg[u]] * d + m + cc[u] * 8;
            const float4 f0 = *reinterpret_cast<const float4*>(src);
            const float4 f1 = *reinterpret_cast<const float4*>(src + 4);
            f[u][0] = f0.x, f[u][1] = f0.y, f[u][2] = f0.z, f[u][3] = f0.w;
            f[u][4] = f1.x, f[u][5] = f1.y, f[u][6] = f1.z, f[u][7] = f1.w;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (e0 + u * NE < total) store_b(gg[u], cc[u], w, f[u]);
      }
    };

    // the next level's B tiles (query slices read from global memory here:
    // holding them in registers since the level's start cost more in spills
    // than the load latency), tail norms and query terms (epilogue threads)
    auto next_level_setup = [&](int l, const float (&tail_pf)[S * CH / NE],
                                unsigned long long key_pf, float seed_pf, float sq_pf) {
      build_b(l + 1, 0);
      float* const cs = csx_of(l + 1);
#pragma unroll
      for (int u = 0; u < S * CH / NE; ++u) cs[tid + u * NE] = tail_pf[u];
      if (tid < QG && qid[tid] >= 0 && qk[tid] > 0) {
        const float tau = key_pf == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key_pf), 1.000001f);
        set_query_terms(tid, fminf(tau, seed_pf), a.eps * sq_pf, qterm_of(l + 1));
      }
      fence_proxy_async_smem();
    };

    // ---- item prologue: group, candidates, liveness, level-0 tiles
    // the level-0 tiles of every chunk are staged first, so that their copies
    // overlap the rest of the prologue (the previous item's last-level work,
    // which used the A buffers, ended at the barrier above)
    if (warp == kIssuer)
      for (int c = 0; c < nch; ++c) issue_load(c, 0);
    if (tid < QG) {
      int q = tid < G ? a.bucket[it.z + tid] : -1;
      qid[tid] = q;
      int kk = 0;
      if (q >= 0) {
        float4 inf = a.qinfo[q];
        qnq[tid] = inf.x;
        qrq[tid] = inf.y;
        qeq[tid] = inf.z;
        kk = a.kq[q];
        if (FP8) atomicMax(&s_qmax, __float_as_uint(inf.w));  // inf.w = max_j |q~_j| >= 0
      } else {
        qnq[tid] = qrq[tid] = qeq[tid] = 0.f;
      }
      qk[tid] = kk;
      // the group's queries with k > 0: warp 0 holds queries 0-31, warp 1 32-63
      const unsigned b = __ballot_sync(0xffffffffu, kk > 0);
      if (lane == 0) s_gm[warp] = b;
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
        csx[e] = a.tails[((ch0 + c) * (L + 1) + 1) * CH + (e % CH)];
      } else {
        cHx[e] = crx[e] = cex[e] = csx[e] = 0.f;
        cid[e] = -1;
      }
    }
    __syncthreads();
    if (FP8 && tid == 0) {
      // query scale 2^-e: the group's largest |q~_j| times it is at most 448
      // (no E4M3 term saturates); a smaller e (at most -60) only adds
      // underflow, which s_cunder bounds: each element loses at most 2^-10
      // of the scaled unit, so the partial product at most
      // 2^-10 2^e sqrt(d) |x|_2
      const float qm = __uint_as_float(s_qmax);
      int e = 0;
      if (qm > 0.f) frexpf(qm / 448.f, &e);
      if (e > 60) atomicOr(a.err, kErrBadInput);
      e = max(-60, min(60, e));
      s_qs = ldexpf(1.f, -e);
      s_cunder = __fmul_ru(ldexpf(1.f, e - 10), __fsqrt_ru((float)d));
    }
    if (epi) {
      const uint32_t gm = s_gm[half];
      for (int c = 0; c < S; ++c) {
        const bool v = c < nch && cid[c * CH + row] >= 0;
        alive[(c * AW + half) * CH + row] = v ? gm : 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, v && gm);
        if (lane == 0) rowlive[c][warp] = bal;
      }
    }
    __syncthreads();
    if (warp == kIssuer) {
      // a chunk with no live row at level 0 (no valid row, or no query with
      // k > 0) is not multiplied: its copy is waited for here instead
      uint32_t m = 0;
      for (int c = 0; c < nch; ++c) {
        if (chunk_live(c)) {
          m |= 1u << c;
        } else if (lane == 0) {
          wait_phase(&load_bar[c], load_bits, c, &s_fail);
        }
      }
      if (lane == 0) {
        s_live[0] = m;
        s_test[0] = (a.prune || L == 1) ? m : 0u;  // level 0: a test level of every schedule
      }
    }
    if (tid < QG) {
      const int q = qid[tid];
      if (q >= 0 && qk[tid] > 0) {
        unsigned long long key = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + qk[tid] - 1);
        float tau = key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f);
        set_query_terms(tid, fminf(tau, __ldcg(a.tau_seed + q)),
                        a.eps * a.qtail[(int64_t)q * (L + 1) + 1], qterm);
      } else {
        qterm[tid] = qterm[QG + tid] = make_float4(0.f, 0.f, 0.f, -INFINITY);
        qtau[tid] = -1.f;
      }
    }
    if (FP8) {
      const float qinv = 1.f / s_qs;  // a power of two: exact
      for (int e = tid; e < S * CH; e += NT)
        cfr[e] = e / CH < nch ? a.xscale[(ch0 + e / CH) * CH + (e % CH)] * qinv : 0.f;
    }
    if (epi) build_b(0, 0);
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    bool completed = true;
    section(0);
    for (int l = 0; l < L; ++l) {
      const int w = a.level_off[l + 1] - a.level_off[l];
      const bool has_next = l + 1 < L;
      const float* const csx_l = csx_of(l);
      const float4* const qterm_l = qterm_of(l);
      const uint32_t live_mask = s_live[l & 1];
      const uint32_t test_mask = s_test[l & 1];
      if (!live_mask) {
        completed = false;
        break;
      }
      if (a.collect && tid == 0) {
        // algorithmic bytes of the level: every candidate still live for
        // some query of the group reads its level slice and tail norm
        unsigned long long n = 0;
        for (int c = 0; c < nch; ++c)
          for (int q = 0; q < 4; ++q) n += __popc(rowlive[c][q] | rowlive[c][q + 4]);
        s_stat[5] += n * (unsigned long long)(w * EB + 4);
      }
      // prefetch the next level's tails and thresholds (raw loads: no
      // arithmetic on them here, so no thread waits for them before its
      // tests)
      float tail_pf[S * CH / NE];
      unsigned long long key_pf = kEmptyKey;
      float seed_pf = INFINITY, sq_pf = 0.f;
      if (has_next && epi) {
#pragma unroll
        for (int u = 0; u < S * CH / NE; ++u) {
          const int e = tid + u * NE;
          tail_pf[u] = 0.f;
          if (e < nch * CH) tail_pf[u] = a.tails[((ch0 + e / CH) * (L + 1) + l + 2) * CH + (e % CH)];
        }
        if (tid < QG) {
          const int q = qid[tid];
          if (q >= 0 && qk[tid] > 0) {
            key_pf = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + qk[tid] - 1);
            seed_pf = __ldcg(a.tau_seed + q);
            sq_pf = a.qtail[(int64_t)q * (L + 1) + l + 2];
          }
        }
      }
      // chunk c's test (epilogue warps): its accumulator once its MMAs are
      // done, then its liveness for the issue warp
      auto epilogue = [&](int c) {
        const bool test = (test_mask >> c) & 1u;
        const bool ok = wait_phase(&mma_bar[c], mma_bits, c, &s_fail);
        tc::fence_after_sync();
        uint32_t wm = alive[(c * AW + half) * CH + row];
        const bool any_live = __any_sync(0xffffffffu, wm != 0);
        if (a.collect && any_live) {
          const unsigned np = __reduce_add_sync(0xffffffffu, (unsigned)__popc(wm));
          if (lane == 0) {
            atomicAdd(&s_stat[0], (unsigned long long)np);
            atomicAdd(&s_stat[1], (unsigned long long)np * w);
          }
        }
        // a level without a test (the plain scan's levels before the last)
        // changes no liveness: its accumulator is not read
        const bool any_warp = test && any_live && __all_sync(0xffffffffu, ok);
        if (any_warp) {
          const float sx = csx_l[c * CH + row], rx = crx[c * CH + row], exv = cex[c * CH + row];
          const float Hx = cHx[c * CH + row];
          const float fr = FP8 ? cfr[c * CH + row] : 1.f;
          if (Npad <= 16) {  // a group of <= 16 queries: 16 columns (half 0 only)
            float v[16];
            tc::tmem_ld16(tbase + lane_base + (uint32_t)(c * QG + 32 * half), v);
            if (test && wm) {
              const float4* qt = qterm_l + 32 * half;
              uint32_t pruned = 0;
#pragma unroll
              for (int g = 0; g < 16; ++g) {
                const float4 t = qt[g];
                const float p = FP8 ? v[g] * fr : v[g];
                const float P = fmaf(t.x, exv, fmaf(t.y, rx, fmaf(t.z, sx, p)));
                pruned |= (P < t.w + Hx ? 1u : 0u) << g;
              }
              wm &= ~pruned;
            }
          } else {
            float v[32];
            tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG + 32 * half), v);
            if (test && wm) {  // every slot is tested (no branches); dead ones stay dead
              const float4* qt = qterm_l + 32 * half;
              uint32_t pruned = 0;
#pragma unroll
              for (int g = 0; g < 32; ++g) {
                const float4 t = qt[g];
                const float p = FP8 ? v[g] * fr : v[g];
                const float P = fmaf(t.x, exv, fmaf(t.y, rx, fmaf(t.z, sx, p)));
                pruned |= (P < t.w + Hx ? 1u : 0u) << g;
              }
              wm &= ~pruned;
            }
          }
          alive[(c * AW + half) * CH + row] = wm;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, wm != 0);
        if (lane == 0) rowlive[c][warp] = bal;
        // every lane's accumulator reads are complete before lane 0 tells
        // the issue warp (which then overwrites the chunk's tile and, at the
        // next level, its accumulator)
        tc::fence_before_sync();
        __syncwarp();
        if (has_next && lane == 0) mbar_arrive_plain(&epi_bar[c]);
      };
      if (warp == kIssuer) {
        // every live chunk's MMA chain as soon as its tile has landed (the
        // epilogue warps test chunk c while chunk c + 1's MMAs run) ...
        if (lane == 0) {
          // the level's descriptors; K-step s adds its offset (16-byte
          // units) to the start-address field
          const int rb = tc::row_bytes(FP8 ? w / 2 : w);
          const uint64_t dh = tc::smem_desc(smem_u32(bhi), rb);
          const uint64_t dl = tc::smem_desc(smem_u32(blo), rb);
          const uint64_t dm = tc::smem_desc(smem_u32(bhi) + (uint32_t)(QG * a.max_w), rb);
          (void)dm;
          for (int c = 0; c < nch; ++c) {
            if (!((live_mask >> c) & 1u)) continue;
            if (wait_phase(&load_bar[c], load_bits, c, &s_fail)) {
              const uint32_t dt = tbase + (uint32_t)(c * QG);
              const uint64_t da = tc::smem_desc(smem_u32(abuf + (size_t)c * lay.abytes), rb);
              if (FP8) {  // 32 elements per K-step; tiles addressed at half width
                for (int s = 0; s < w / 32; ++s) {
                  const uint64_t ad = da + tc::kstep_off(s, CH);
                  const uint64_t bo = tc::kstep_off(s, Npad);
                  tc::mma_e4m3(dt, ad, dh + bo, idesc, (l > 0 || s > 0) ? 1u : 0u);
                  tc::mma_e4m3(dt, ad, dm + bo, idesc, 1u);
                  tc::mma_e4m3(dt, ad, dl + bo, idesc, 1u);
                }
              } else {
                for (int s = 0; s < w / 16; ++s) {
                  const uint64_t ad = da + tc::kstep_off(s, CH);
                  const uint64_t bo = tc::kstep_off(s, Npad);
                  tc::mma_bf16(dt, ad, dh + bo, idesc, (l > 0 || s > 0) ? 1u : 0u);
                  tc::mma_bf16(dt, ad, dl + bo, idesc, 1u);
                }
              }
            }
            // committed even after a failed wait, so the epilogue's wait ends
            tc::mma_commit(&mma_bar[c]);
          }
        }
        __syncwarp();
        // ... then each chunk that stays live gets its next level's tile as
        // soon as every epilogue warp has read its accumulator
        if (has_next) {
          uint32_t next_live = 0, next_test = 0;
          for (int c = 0; c < nch; ++c) {
            if (!((live_mask >> c) & 1u)) continue;
            int ok = 1;
            if (lane == 0) ok = wait_phase(&epi_bar[c], epi_bits, c, &s_fail) ? 1 : 0;
            tc::fence_after_sync();
            // lane 0 (which acquired the chunk's liveness words) decides for
            // the warp (s_fail may change under it)
            const int go = __shfl_sync(0xffffffffu, (ok && !s_fail && chunk_live(c)) ? 1 : 0, 0);
            if (go) {
              issue_load(c, l + 1);
              next_live |= 1u << c;
              // the bound-test schedule: chunk c is tested at level l + 1 if
              // that is a level of the schedule or the last, or if at most
              // kTestRows of its rows are still live
              int n = 0;
              for (int q = 0; q < 4; ++q) n += __popc(rowlive[c][q] | rowlive[c][q + 4]);
              if (l + 1 == L - 1 ||
                  (a.prune && ((l + 1) % a.test_every == 0 || n <= kTestRows)))
                next_test |= 1u << c;
            }
          }
          if (lane == 0) {
            s_live[(l + 1) & 1] = next_live;
            s_test[(l + 1) & 1] = next_test;
          }
        }
      } else {
        for (int c = 0; c < nch; ++c)
          if ((live_mask >> c) & 1u) epilogue(c);
        // every MMA of the level has completed (this warp saw the last live
        // chunk's commit), so its B tiles are free: the next level's B
        // tiles, tails and thresholds go in now, into the other tail and
        // query-term buffers, while other warps may still be testing
        if (kEarly && has_next) next_level_setup(l, tail_pf, key_pf, seed_pf, sq_pf);
      }
      // the level's accumulators have been read, its B tiles are free and
      // the next level's tiles are on their way; a failed wait anywhere ends
      // the item for every thread alike
      tc::fence_before_sync();
      const int failed = __syncthreads_or(s_fail != 0);
      tc::fence_after_sync();
      if (a.collect && tid == 0) s_stat[2] += __popc(live_mask);
      section(2);
      if (failed) {
        completed = false;
        break;
      }
      if (!kEarly && has_next) {
        if (epi) next_level_setup(l, tail_pf, key_pf, seed_pf, sq_pf);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
      }
      section(3);
    }
    if (s_fail) break;
    if (!completed) continue;
    if (!epi) continue;  // the rest of the item is the epilogue warps' (named barrier 1)

    // Last level done: the k-th smallest upper bound of each query over the
    // whole segment tightens its threshold (at the last level UB ~ LB ~
    // exact), then the pairs are tested again, so about k pairs per query
    // reach re-ranking.  The bounds are kept as bf16 rounded up (still upper
    // bounds) so that all S x CH of them fit next to each other.
    for (int c = 0; c < S; ++c) {
      uint32_t wm = 0;
      if (c < nch && chunk_live(c)) wm = alive[(c * AW + half) * CH + row];
      const bool any_warp = __any_sync(0xffffffffu, wm != 0);
      uint16_t* col = ub16 + (32 * half) * S * CH + c * CH + row;  // stride S*CH per query
      if (any_warp) {
        const float rx = crx[c * CH + row], exv = cex[c * CH + row];
        const float nx2 = a.xn2[(ch0 + c) * CH + row];
        const float fr = FP8 ? cfr[c * CH + row] : 1.f;
        const float under = FP8 ? 2.f * s_cunder * rx : 0.f;  // FP8 query split
        float v[32];
        tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG + 32 * half), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int g = 32 * half + j;
          uint16_t u = 0x7f80u;
          if ((wm >> j) & 1u) {
            const float A = qnq[g] + nx2 - 2.f * (FP8 ? v[j] * fr : v[j]);
            const float Ss = qrq[g] + rx;
            const float r = __fadd_ru(sqrt_up(fmaxf(A + fmaf(g_slack * Ss, Ss, under), 0.f)),
                                      qeq[g] + exv);
            u = __bfloat16_as_ushort(__float2bfloat16_ru(__fmul_ru(__fmul_ru(r, r), a.ub_scale)));
          }
          col[j * S * CH] = u;
        }
      } else {
        for (int j = 0; j < 32; ++j) col[j * S * CH] = 0x7f80u;
      }
    }
    epi_sync();
    for (int g = warp; g < G; g += NE / 32) {
      const float t = warp_kth_smallest_bf16(ub16 + g * S * CH, S * CH, qk[g]);
      // k candidates with upper bounds <= t: a threshold for every later
      // work item of the query too
      if (lane == 0 && qk[g] > 0 && t < qtau[g]) {
        qtau[g] = t;
        atomicMin(reinterpret_cast<unsigned int*>(a.tau_seed) + qid[g], __float_as_uint(t));
      }
    }
    epi_sync();
    float4* const qterm_last = qterm_of(L - 1);
    if (tid < G && qk[tid] > 0) set_query_terms(tid, qtau[tid], 0.f, qterm_last);
    tc::fence_before_sync();
    epi_sync();
    tc::fence_after_sync();
    section(4);
    // survivors of the tightened test join the deferred re-rank list with
    // their Eq. 3 lower bound (C = 0 after the last level); a full list is
    // checked and re-ranked by all warps at once
    for (int c = 0; c < nch; ++c) {
      if (tid == 0) s_nsurv = 0;
      epi_sync();
      uint32_t wm = alive[(c * AW + half) * CH + row];
      const bool any_warp = __any_sync(0xffffffffu, wm != 0);
      if (any_warp) {
        const float rx = crx[c * CH + row], exv = cex[c * CH + row], Hx = cHx[c * CH + row];
        const float fr = FP8 ? cfr[c * CH + row] : 1.f;
        float v[32];
        tc::tmem_ld32(tbase + lane_base + (uint32_t)(c * QG + 32 * half), v);
        const float4* qt = qterm_last + 32 * half;
        uint32_t pruned = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float4 t = qt[j];
          const float P = fmaf(t.x, exv, fmaf(t.y, rx, FP8 ? v[j] * fr : v[j]));
          pruned |= (P < t.w + Hx ? 1u : 0u) << j;
        }
        wm &= ~pruned;
        if (wm) {
#pragma unroll
          for (int j = 0; j < 32; ++j) vdump[j * NE + tid] = v[j];
        }
      }
      for (uint32_t m = wm; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        surv[atomicAdd(&s_nsurv, 1)] = (uint16_t)((row << 6) | (32 * half + j));
      }
      epi_sync();
      const int ns = s_nsurv;
      int np = s_npend;
      // all survivors go through the deferred list, a full list being
      // checked and re-ranked before more join (the survivor list and the
      // accumulators dumped above stay untouched by a flush)
      for (int b0 = 0; b0 < ns;) {
        if (np == Smem::kPend) {
          epi_sync();
          rerank_pending(np);
          np = 0;
        }
        const int nb = min(ns - b0, Smem::kPend - np);
        for (int s = tid; s < nb; s += NE) {
          const int e = surv[b0 + s], r = e >> 6, g = e & 63;
          const int64_t slot = (ch0 + c) * CH + r;
          const float rx = crx[c * CH + r], exv = cex[c * CH + r];
          float p = vdump[(g & 31) * NE + r + CH * (g >> 5)];  // all levels
          if (FP8) p *= cfr[c * CH + r];
          const float under = FP8 ? 2.f * s_cunder * rx : 0.f;
          const float A = qnq[g] + a.xn2[slot] - 2.f * p;
          const float Ss = qrq[g] + rx;
          const float slack = fmaf(g_slack * Ss, Ss, under);
          const float lr = sqrtf(fmaxf(A - slack, 0.f)) - (qeq[g] + exv);
          pslot[np + s] = slot;
          pq[np + s] = qid[g];
          pid[np + s] = cid[c * CH + r];
          plb[np + s] = lr > 0.f ? lr * lr * a.lb_scale : 0.f;
          const float ru = __fadd_ru(sqrt_up(fmaxf(A + slack, 0.f)), qeq[g] + exv);
          pub[np + s] = __fmul_ru(__fmul_ru(ru, ru), a.ub_scale);
        }
        np += nb;
        b0 += nb;
      }
      tc::fence_before_sync();
      epi_sync();
      tc::fence_after_sync();
      if (tid == 0) s_npend = np;
    }
    // the scratch written through the generic proxy is refilled by
    // bulk-async copies in the next item
    fence_proxy_async_smem();
    section(5);
  }
  if (!s_fail && epi) {  // the last deferred survivors
    epi_sync();
    rerank_pending(s_npend);
  }
  if (s_fail && tid == 0) atomicOr(a.err, kErrTimeout);
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
    atomicAdd(&a.stats[25], s_stat[5]);
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

int launch_pack_fp8(const float* xt, const float* rows, const int64_t* perm, int64_t chunk0,
                    int64_t nchunks, int d, int L, const int32_t* level_off, const float* mu,
                    double c_trans, uint8_t* slices, float* tails, float* xn2, float* ex,
                    float* xscale, int32_t* ids, cudaStream_t st) {
  PANO_CHECK(d % 32 == 0 && d <= 8192, PANO_EINVAL, "fp8 storage needs d % 32 == 0, d <= 8192");
  pack_fp8_kernel<<<(unsigned)nchunks, 256, 0, st>>>(xt, rows, perm, chunk0, d, L, level_off, mu,
                                                     c_trans, slices, tails, xn2, ex, xscale, ids);
  PANO_CUDA(cudaGetLastError());
  return PANO_OK;
}

size_t verify_tc_smem(int max_w, bool fp8) {
  // at most two CTAs per SM: each owns 256 of the 512 TMEM columns
  return std::max<size_t>(Smem(max_w, fp8 ? 1 : 2).total + 1024, 80 * 1024);
}

int launch_verify_tc(const VerifyTCArgs& a, cudaStream_t st) {
  static PerDeviceOnce once;
  PANO_CUDA(once.run([] {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (const void* k : {(const void*)verify_tc_kernel<false>, (const void*)verify_tc_kernel<true>}) {
      cudaFuncAttributes fa;
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return e;
  }));
  const size_t smem = verify_tc_smem(a.max_w, a.fp8 != 0);
  int dev = 0, sms = 0, optin = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  PANO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PANO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)optin)
    return fail(PANO_EINVAL, "tensor-core verify tile does not fit in shared memory");
  // Two CTAs x 256 TMEM columns fill an SM's tensor memory.  The grid is
  // not sized from the occupancy API: it reports the SM's current shared
  // memory carveout, which switches only when a launch asks for more.  A
  // persistent CTA that cannot be resident yet starts later and finds the
  // queue drained, so over-provisioning is harmless.
  if (a.fp8)
    verify_tc_kernel<true><<<sms * 2, NT, smem, st>>>(a);
  else
    verify_tc_kernel<false><<<sms * 2, NT, smem, st>>>(a);
  PANO_CUDA(cudaGetLastError());
  return PANO_OK;
}

}  // namespace pano
