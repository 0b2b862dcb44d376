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
// columns = 256 TMEM columns; two CTAs share an SM).  Candidate row t is
// owned by two epilogue threads (warps w and w + 4 read the same TMEM lane
// quarter), one per half of the query group: each reads its 32 accumulators
// with tcgen05.ld and applies the separable form of the margined Eq. 3 test,
// which costs three FMAs and a compare per (candidate, query) pair.  Dead rows are not re-staged: at deep
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
// Work item = (list, segment of <= S chunks, group of <= QG queries).  The
// CTA walks the segment level by level (the paper's batch: every candidate
// moves one level before the next level starts; the threshold terms are
// refreshed per level) with three roles that hand work to each other
// through mbarriers, so no CTA-wide barrier sits in the level loop:
//
// * producer warp: takes work items from the queue and, for each level and
//   chunk not known to be dead, stages the chunk's level tile into a ring of
//   NA shared-memory stages with bulk-async copies (only the 8-row atoms
//   holding a live row once few rows live).  It runs up to NA steps ahead of
//   the tensor core: at level l it uses the liveness the epilogue published
//   for the latest finished level of the chunk (a superset of the rows live
//   at level l), so copies are issued a level ahead of their use.
// * MMA warp (one thread): for each staged (chunk, level) step passes the
//   step descriptor on to the epilogue's ring, then waits for the tile, the
//   level's query tiles and the epilogue of the chunk's previous level (its
//   accumulator is read before it is accumulated into again),
//   then issues the chunk's MMA chain (A = level tile, B = the queries' level
//   slices split into bf16 hi + lo, or three E4M3 terms; D = the chunk's 64
//   TMEM columns, accumulated across levels) and commits it to the stage's
//   "empty" and the chunk's "done" barriers; a chunk whose rows all died is
//   skipped with plain arrivals.
// * epilogue warps (16, four per TMEM lane quarter): one thread per
//   (candidate row, 16-query slice of the group).  Per step: tcgen05.ld of
//   16 accumulators, the separable margined Eq. 3 test (three FMAs and a
//   compare per pair; query columns no lane of the warp still holds are
//   skipped), alive masks and per-warp row liveness; the last warp to finish
//   a step publishes the chunk's live 8-row atoms for the producer.  The
//   warps do not keep step with each other: they meet only at level
//   boundaries (per-query threshold terms refreshed, the query tiles of the
//   level after next built, double-buffered), at item starts (the group and
//   the candidates loaded) and at last-level steps, whose survivors' lower
//   and upper bounds go to a deferred re-rank list that is checked and
//   re-ranked when full.  Those meetings are mbarriers with bounded waits,
//   so a failed role can never leave the others waiting for ever.
constexpr int S = TC_SEG;           // chunks per work item (8 x 64 = 512 TMEM columns)
constexpr int EW = 16;              // epilogue warps
constexpr int NSL = EW / 4;         // query slices (warps per TMEM lane quarter)
constexpr int QS = QG / NSL;        // 16 query columns per epilogue thread
constexpr int NEPI = EW * 32;       // epilogue threads
constexpr int NT = 64 + NEPI;       // producer warp, MMA warp, epilogue warps
constexpr int TMEM_COLS = S * QG;   // 512: one CTA per SM
constexpr int RING = 32;            // step descriptors MMA warp -> epilogue (>= S + 1)
constexpr int kMaxStages = 16;      // A-tile ring stages
constexpr int kPend = 256;          // deferred re-rank entries (one epilogue thread each)
constexpr int PF_CHUNKS = 1;        // 8-element query chunks prefetched per epilogue thread
constexpr int TPF = S * CH / NEPI;  // tail norms prefetched per epilogue thread
static_assert(QG == 64 && QS == 16 && TMEM_COLS == 512 && kPend <= NEPI &&
                  TPF * NEPI == S * CH && PF_CHUNKS * NEPI * 8 == QG * 64,
              "layout of the tensor-core verify kernel");
// the producer runs at most kMaxStages steps ahead of the MMA warp, which
// runs at most S steps ahead of the slowest epilogue warp
static_assert(RING > kMaxStages + S + 1, "step ring too short");

// Dynamic shared memory: the A ring and the query-tile buffers (hi and lo
// halves each); the fixed-size arrays are static shared memory.
struct Lay {
  uint32_t abytes, bbytes, off_b, total;
  // nb: query-tile buffers (2: the next level's tiles are built while the
  // current level runs; 1 for wide levels, built at the level boundary)
  __host__ __device__ Lay(int max_w, int eb, int na, int nb) {
    abytes = (uint32_t)(CH * max_w * eb + 1023) & ~1023u;
    bbytes = (uint32_t)(QG * max_w * 2 + 1023) & ~1023u;
    off_b = (uint32_t)na * abytes;
    total = off_b + 2 * nb * bbytes;  // [nb buffers][hi, lo]
  }
};

__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait that also gives up as soon as another role has failed.
__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, volatile int* fail) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*fail) return false;
    if (clock64() - t0 > kWaitCycles) {
      atomicOr(const_cast<int*>(fail), 1);
      return false;
    }
  }
}

// wait_or_fail that adds the cycles it waited to *acc when acc is set.
__device__ __forceinline__ bool timed_wait(uint64_t* bar, uint32_t parity, volatile int* fail,
                                           unsigned long long* acc) {
  if (!acc) return wait_or_fail(bar, parity, fail);
  const long long t0 = clock64();
  const bool ok = wait_or_fail(bar, parity, fail);
  *acc += (unsigned long long)(clock64() - t0);
  return ok;
}

// Meetings of the epilogue threads on an mbarrier (count NEPI) with bounded
// waits; any_of also ORs a predicate over them through three flags used in
// rotation (the flag of the meeting before last is cleared, which no thread
// can still be reading or already setting again).
struct EpiSync {
  uint64_t* bar;
  int* flags;  // [3]
  volatile int* fail;
  uint32_t par;
  int k;
  __device__ bool sync() {
    mbar_arrive_plain(bar);
    const bool ok = wait_or_fail(bar, par, fail);
    par ^= 1u;
    return ok;
  }
  __device__ bool any_of(bool p, int etid) {
    volatile int* f = flags + k % 3;
    if (p) *f = 1;
    sync();
    const bool r = *f != 0;
    if (etid == 0) flags[(k + 2) % 3] = 0;
    ++k;
    return r;
  }
};

// The deferred pairs are checked against their queries' thresholds of the
// moment and against each other: a pair whose lower bound exceeds the
// upper bounds of k pending pairs of its query is dropped (all k are
// closer), and the k-th smallest pending upper bound of a query is a
// threshold for all its later work (k distinct candidates lie below it).
// The rest get their exact distance and top-k insertion, in two passes:
// first each query's k kept pairs of smallest lower bound (ties by entry),
// whose exact distances usually set its threshold, then the others that
// still pass it.  All epilogue threads call it (one thread per entry at
// most); kept out of line so that it does not add to the step loop's
// registers.  Returns the number re-ranked (epilogue thread 0; 0 elsewhere).
__device__ __noinline__ int flush_pending(const VerifyTCArgs& a, EpiSync& es, int np, int etid,
                                          const int64_t* __restrict__ pslot,
                                          const int32_t* __restrict__ pq,
                                          const int32_t* __restrict__ pid,
                                          float* __restrict__ plb,
                                          const float* __restrict__ pub, uint16_t* keep,
                                          uint16_t* rank, int* s_cnt) {
  const int warp = etid / 32;
  if (etid == 0) s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
  es.sync();
  auto tau_of = [&](int q, int kk) {
    const unsigned long long key = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + kk - 1);
    return fminf(key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f),
                 __ldcg(a.tau_seed + q));
  };
  if (etid < np) {
    const int s = etid, q = pq[s], kk = a.kq[q];
    const float lb = plb[s], ub = pub[s];
    bool keep_s = !(lb > tau_of(q, kk));
    int below = 0, ub_rank = 0;
    for (int o = 0; o < np; ++o) {
      const bool same = pq[o] == q;
      below += same & (__fmul_ru(pub[o], 1.000001f) < lb);
      ub_rank += same & ((pub[o] < ub) | ((pub[o] == ub) & (o <= s)));
    }
    keep_s = keep_s && below < kk;
    if (kk > 0 && ub_rank >= kk)  // k pending candidates with upper bounds <= ub
      atomicMin(reinterpret_cast<unsigned int*>(a.tau_seed) + q, __float_as_uint(ub));
    if (keep_s) keep[atomicAdd(&s_cnt[0], 1)] = (uint16_t)s;
  }
  es.sync();
  const int nk = s_cnt[0];
  if (etid < nk && (a.d & 3) == 0)  // all kept rows head for L2 at once
    prefetch_l2(a.rows + pslot[keep[etid]] * a.d, (uint32_t)a.d * 4);
  bool first = false;
  if (etid < nk) {  // rank among the kept pairs of its query
    const int s = keep[etid], q = pq[s];
    const float lb = plb[s];
    int r = 0;
    for (int j = 0; j < nk; ++j) {
      const int o = keep[j];
      r += (pq[o] == q) & ((plb[o] < lb) | ((plb[o] == lb) & (o < s)));
    }
    first = r < a.kq[q];
    rank[etid] = first ? 1 : 0;
    if (first) atomicAdd(&s_cnt[1], 1);
  }
  es.sync();
  // exact distances (a warp each; they replace the lower bounds), then the
  // top-k insertions (a thread each, so their chains overlap)
  auto rerank = [&](const uint16_t* list, int n, const uint16_t* sel) {
    for (int i = warp; i < n; i += EW) {
      if (sel && !sel[i]) continue;
      const int s = list[i];
      const float dist =
          exact_sqdist_warp_wide(a.qorig + (int64_t)pq[s] * a.d, a.rows + pslot[s] * a.d, a.d);
      if ((etid & 31) == 0) plb[s] = dist;
    }
    es.sync();
    if (etid < n && (!sel || sel[etid])) {
      const int s = list[etid], q = pq[s];
      topk_insert_thread(a.topk + (int64_t)q * a.k_max, a.kq[q], make_key(plb[s], pid[s]));
    }
    es.sync();
  };
  rerank(keep, nk, rank);
  // the others, against the thresholds of the moment (rank now lists them)
  if (etid < nk && !first) {
    const int s = keep[etid], q = pq[s];
    if (!(plb[s] > tau_of(q, a.kq[q]))) rank[atomicAdd(&s_cnt[2], 1)] = (uint16_t)s;
  }
  es.sync();
  rerank(rank, s_cnt[2], nullptr);
  return etid == 0 ? s_cnt[1] + s_cnt[2] : 0;
}

// FP8 = false: BF16 tiles, kind::f16 MMAs with the query split into bf16 hi +
// lo.  FP8 = true: E4M3 tiles (the byte layout of bf16 tiles of half the
// width), kind::f8f6f4 MMAs with the query split into three E4M3 terms at one
// power-of-two scale per group; the accumulator times the row's factor
// s_x / (group scale) is the partial product.
template <bool FP8>
__global__ void __launch_bounds__(NT, 1) verify_tc_kernel(const VerifyTCArgs a) {
  constexpr int EB = FP8 ? 1 : 2;  // bytes per stored element
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const int NA = a.na;
  const int NB = a.nb;       // query-tile buffers
  const int AHEAD = NB - 1;  // levels the query tiles are built ahead
  const Lay lay(a.max_w, EB, NA, NB);
  auto bidx = [&](int lv) { return NB == 2 ? (lv & 1) : 0; };
  unsigned char* abuf = base;
  unsigned char* bbuf = base + lay.off_b;
  // per candidate row of the item's chunks: alive masks of the query
  // slices, Eq. 3 terms, the current level's tail norm sqrt(R_x^(l+1,d)),
  // the FP8 accumulator factor s_x / (group scale) and the id
  __shared__ uint16_t alive[S * CH * NSL];
  __shared__ float cHx[S * CH], crx[S * CH], cex[S * CH], cxn[S * CH], csx[S * CH], cfr[S * CH];
  __shared__ int32_t cid[S * CH];
  // per query of the group: terms of the separable test (E, g*rq, sq, H)
  __shared__ float4 qterm[QG];
  __shared__ int32_t qid[QG], qk[QG];
  __shared__ float qnq[QG], qrq[QG], qeq[QG], qtau[QG];

  __shared__ __align__(8) uint64_t a_full[kMaxStages], a_empty[kMaxStages];
  __shared__ __align__(8) uint64_t mma_done[S], epi_done[S], b_full[2], desc_full[RING], drain,
      epi_bar;
  __shared__ int s_any[3];
  __shared__ int4 stage_desc[kMaxStages], epi_desc[RING];
  __shared__ __align__(16) uint32_t rowlive[S][EW];  // per epilogue warp: its live rows
  __shared__ unsigned long long atom_word[S];  // item << 32 | level << 16 | live 8-row atoms
  __shared__ int last_item[S], last_level[S];  // MMA warp: each chunk's latest step
  __shared__ int64_t pslot[kPend];
  __shared__ int32_t pq[kPend], pid[kPend];
  __shared__ float plb[kPend], pub[kPend];
  __shared__ uint16_t keep[kPend], rnk[kPend];
  __shared__ int s_flush[3];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_np;
  // FP8: the group's largest |q~_j| (as bits), query scale and the absolute
  // bound of the query split's underflow per unit of |x|_2
  __shared__ unsigned int s_qmax;
  __shared__ float s_qs, s_cunder;
  // counters (collect_stats): [0] pairs, [1] dims, [2] steps, [3] staged
  // bytes, [4] reranked, [5] live-row bytes; section cycles
  __shared__ unsigned long long s_stat[6], s_sec[8], s_wait[4];

  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  volatile int* vfail = &s_fail;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 32) {
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int c = 0; c < S; ++c) {
      mbar_init(&mma_done[c], 1);
      mbar_init(&epi_done[c], EW);
      atom_word[c] = ~0ULL;
      last_item[c] = -1;
      last_level[c] = 0;
      for (int e = 0; e < EW; ++e) rowlive[c][e] = 0u;
    }
    for (int i = 0; i < 2; ++i) mbar_init(&b_full[i], NEPI);
    for (int i = 0; i < RING; ++i) mbar_init(&desc_full[i], 1);
    mbar_init(&drain, 1);
    mbar_init(&epi_bar, NEPI);
    s_any[0] = s_any[1] = s_any[2] = 0;
    fence_mbar_init();
    s_fail = 0;
    s_np = 0;
    for (int i = 0; i < 6; ++i) s_stat[i] = 0;
    for (int i = 0; i < 4; ++i) s_wait[i] = 0;
    for (int i = 0; i < 8; ++i) s_sec[i] = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const int L = a.L, d = a.d;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    uint32_t filled = 0, empty_par = 0, fill_par = 0;
    int st = 0, pstep = 0;
    // a step's descriptor goes to the MMA warp (with its stage) and to the
    // epilogue's ring (a new item's prologue there builds the query tiles
    // the MMA warp waits for)
    auto publish = [&](int4 dsc) {
      stage_desc[st] = dsc;
      const int slot = pstep % RING;
      epi_desc[slot] = dsc;
      mbar_arrive_plain(&desc_full[slot]);
      ++pstep;
    };
    auto acquire = [&](int s) {
      if (!((filled >> s) & 1u)) {
        filled |= 1u << s;
        return true;
      }
      const bool ok = timed_wait(&a_empty[s], (empty_par >> s) & 1u, vfail,
                                 a.collect && lane == 0 ? &s_wait[3] : nullptr);
      empty_par ^= 1u << s;
      return ok;
    };
    bool ok = true;
    while (ok) {
      int item = 0;
      if (lane == 0) item = atomicAdd(a.counter, 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      const int64_t n_items = *a.n_items < a.items_cap ? *a.n_items : a.items_cap;
      const bool stop = __shfl_sync(0xffffffffu, (item >= n_items || *vfail) ? 1 : 0, 0) != 0;
      if (stop) {  // no more work: the terminal step
        ok = __all_sync(0xffffffffu, acquire(st));
        if (ok) {
          if (lane == 0) {
            publish(make_int4(-1, 0, 0, 0));
            mbar_arrive_plain(&a_full[st]);
          }
          fill_par ^= 1u << st;
        }
        break;
      }
      const int4 it = a.items[item];
      const int64_t ch0 = a.chunk_off[it.x] + (int64_t)it.y * S;
      const int64_t chE = a.chunk_off[it.x + 1];
      const int nch = (int)((chE - ch0) < S ? (chE - ch0) : S);
      const uint8_t* item_src = a.slices + ch0 * (int64_t)CH * d * EB;
      for (int l = 0; l < L && ok; ++l) {
        const int m = a.level_off[l], w = a.level_off[l + 1] - m;
        const int wl = FP8 ? w / 2 : w;  // width of the bf16 tile with the same bytes
        const uint32_t tbytes = (uint32_t)w * CH * EB;
        const int rb = tc::row_bytes(wl), npan = wl >= 64 ? wl / 64 : 1;
        bool any = false;
        for (int c = 0; c < nch; ++c) {
          uint32_t atoms = 0xffffu;
          if (l > 0) {  // liveness of the chunk's latest finished level of this item
            const unsigned long long wd =
                *reinterpret_cast<volatile unsigned long long*>(&atom_word[c]);
            if ((int)(wd >> 32) == item && (int)((wd >> 16) & 0xffffu) < l)
              atoms = (uint32_t)(wd & 0xffffu);
            if (!atoms) continue;  // every row of the chunk is dead
          }
          if (!__all_sync(0xffffffffu, acquire(st))) {
            ok = false;
            break;
          }
          unsigned char* dst = abuf + (size_t)st * lay.abytes;
          const uint8_t* src = item_src + (int64_t)c * CH * d * EB + (size_t)m * CH * EB;
          const int na = __popc(atoms);
          if (lane == 0) publish(make_int4(item, c | (l << 8), it.w, nch));
          if (l == 0 || na * 4 >= 3 * 16) {
            if (lane == 0) {
              mbar_arrive_expect_tx(&a_full[st], tbytes);
              bulk_g2s(dst, src, tbytes, &a_full[st]);
              if (a.collect) s_stat[3] += tbytes;
            }
          } else {
            const uint32_t atom_bytes = (uint32_t)(8 * rb);  // one 8-row atom of one panel
            if (lane == 0) {
              mbar_arrive_expect_tx(&a_full[st], (uint32_t)na * npan * atom_bytes);
              if (a.collect) s_stat[3] += (unsigned long long)na * npan * atom_bytes;
            }
            __syncwarp();
            for (int t = lane; t < 16 * npan; t += 32) {
              const int at = t % 16, p = t / 16;
              if ((atoms >> at) & 1u) {
                const uint32_t o = (uint32_t)p * CH * 128 + (uint32_t)at * atom_bytes;
                bulk_g2s(dst + o, src + o, atom_bytes, &a_full[st]);
              }
            }
          }
          fill_par ^= 1u << st;
          any = true;
          st = st + 1 == NA ? 0 : st + 1;
        }
        if (!any) break;  // every chunk of the item is dead
      }
    }
    // copies still in flight land before the CTA can exit
    for (int s = 0; s < NA; ++s)
      if ((filled >> s) & 1u) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&a_full[s], ((fill_par >> s) & 1u) ^ 1u) &&
               clock64() - t0 < kWaitCycles) {
        }
      }
  } else if (warp == 1) {
    // ----------------------------------------------------------- MMA issue
    if (lane == 0) {
      uint32_t full_par = 0, epi_par = 0, epi_pend = 0, bpar = 0;
      int cur_item = -1, cur_level = -1, st = 0, Npad = 16;
      uint32_t idesc = 0;
      bool issued = false;
      while (true) {
        if (!timed_wait(&a_full[st], (full_par >> st) & 1u, vfail, a.collect ? &s_wait[0] : nullptr))
          break;
        full_par ^= 1u << st;
        const int4 dsc = stage_desc[st];
        if (dsc.x < 0) break;  // terminal
        const int c = dsc.y & 0xff, l = (dsc.y >> 8) & 0xff;
        bool ok = true;
        if (dsc.x != cur_item) {
          // the query tiles of the level after the previous item's last
          // level were built but not used: take that phase too
          if (NB == 2 && cur_item >= 0 && cur_level + 1 < L) {
            const int bi = (cur_level + 1) & 1;
            ok = wait_or_fail(&b_full[bi], (bpar >> bi) & 1u, vfail);
            bpar ^= 1u << bi;
          }
          cur_item = dsc.x;
          cur_level = -1;
          const int G = dsc.z;
          Npad = G <= 16 ? 16 : ((G + 15) & ~15);
          idesc = FP8 ? tc::idesc_e4m3(CH, Npad) : tc::idesc_bf16(CH, Npad);
        }
        if (ok && l != cur_level) {
          const int bi = bidx(l);
          ok = wait_or_fail(&b_full[bi], (bpar >> bi) & 1u, vfail);
          bpar ^= 1u << bi;
          cur_level = l;
        }
        const bool had_step = (epi_pend >> c) & 1u;
        if (ok && had_step) {  // the chunk's accumulator has been read
          ok = timed_wait(&epi_done[c], (epi_par >> c) & 1u, vfail,
                          a.collect ? &s_wait[1] : nullptr);
          epi_par ^= 1u << c;
        }
        if (!ok) break;
        tc::fence_after_sync();
        // rows of the chunk live after its latest finished step, per lane
        // quarter: the OR of the quarter's four query-slice warps (word e of
        // rowlive[c] belongs to epilogue warp e: slice e / 4, quarter
        // (e + 2) % 4)
        const uint4* rl = reinterpret_cast<const uint4*>(&rowlive[c][0]);
        const uint4 u0 = rl[0], u1 = rl[1], u2 = rl[2], u3 = rl[3];
        const uint32_t qm[4] = {u0.z | u1.z | u2.z | u3.z, u0.w | u1.w | u2.w | u3.w,
                                u0.x | u1.x | u2.x | u3.x, u0.y | u1.y | u2.y | u3.y};
        const uint32_t live = qm[0] | qm[1] | qm[2] | qm[3];
        if (had_step && last_item[c] == dsc.x) {
          // publish the live 8-row atoms of that step for the producer, and
          // count the rows entering level l (algorithmic bytes)
          uint32_t atoms = 0, nlive = 0;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            nlive += __popc(qm[qq]);
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if ((qm[qq] >> (8 * b)) & 0xffu) atoms |= 1u << (qq * 4 + b);
          }
          *reinterpret_cast<volatile unsigned long long*>(&atom_word[c]) =
              ((unsigned long long)(uint32_t)dsc.x << 32) |
              ((unsigned long long)last_level[c] << 16) | atoms;
          if (a.collect)
            atomicAdd(&s_stat[5], (unsigned long long)nlive *
                                      (unsigned long long)((a.level_off[l + 1] - a.level_off[l]) *
                                                               EB + 4));
        }
        last_item[c] = dsc.x;
        last_level[c] = l;
        if (live) {
          if (a.collect) s_stat[2] += 1;
          const int w = a.level_off[l + 1] - a.level_off[l];
          const int rb = tc::row_bytes(FP8 ? w / 2 : w);
          const uint32_t a0 = smem_u32(abuf + (size_t)st * lay.abytes);
          const uint32_t h0 = smem_u32(bbuf + (size_t)bidx(l) * 2 * lay.bbytes);
          const uint32_t dt = tbase + (uint32_t)(c * QG);
          // descriptors of the first K-step; K-step s adds (s % 4) 32-byte
          // chunks and (s / 4) 128-byte panels of R rows (R * 8 in units of
          // 16 bytes) to the start-address field
          const uint64_t ad = tc::smem_desc(a0, rb);
          const uint64_t hd = tc::smem_desc(h0, rb);
          const uint64_t ld = tc::smem_desc(h0 + lay.bbytes, rb);
          const uint32_t pa = (uint32_t)CH * 8u, pb = (uint32_t)Npad * 8u;
          if (FP8) {  // 32 elements per K-step; tiles addressed at half width
            const uint64_t md = tc::smem_desc(h0 + (uint32_t)(QG * a.max_w), rb);
            for (int k = 0; k < w / 32; ++k) {
              const uint64_t oa = (uint64_t)((k & 3) * 2 + (k >> 2) * pa);
              const uint64_t ob = (uint64_t)((k & 3) * 2 + (k >> 2) * pb);
              tc::mma_e4m3(dt, ad + oa, hd + ob, idesc, (l > 0 || k > 0) ? 1u : 0u);
              tc::mma_e4m3(dt, ad + oa, md + ob, idesc, 1u);
              tc::mma_e4m3(dt, ad + oa, ld + ob, idesc, 1u);
            }
          } else {
            for (int k = 0; k < w / 16; ++k) {
              const uint64_t oa = (uint64_t)((k & 3) * 2 + (k >> 2) * pa);
              const uint64_t ob = (uint64_t)((k & 3) * 2 + (k >> 2) * pb);
              tc::mma_bf16(dt, ad + oa, hd + ob, idesc, (l > 0 || k > 0) ? 1u : 0u);
              tc::mma_bf16(dt, ad + oa, ld + ob, idesc, 1u);
            }
          }
          tc::mma_commit(&a_empty[st]);
          tc::mma_commit(&mma_done[c]);
          issued = true;
        } else {
          mbar_arrive_plain(&a_empty[st]);
          mbar_arrive_plain(&mma_done[c]);
        }
        epi_pend |= 1u << c;
        st = st + 1 == NA ? 0 : st + 1;
      }
      if (issued) {  // every MMA has completed before TMEM is released
        tc::mma_commit(&drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(&drain, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue
    const int etid = tid - 64, e = etid >> 5;
    const int quarter = (e + 2) & 3;  // TMEM lanes a warp may read: 32 * (warp % 4)
    const int slice = e >> 2;         // query columns QS * slice .. + QS - 1
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const float g_slack = a.gslack;
    constexpr float kEval = 32.f * 5.9604645e-08f;  // evaluation slack of the separable test
    EpiSync es{&epi_bar, s_any, vfail, 0u, 0};
    long long t_mark = clock64();
    const long long t_kernel = t_mark;
    auto section = [&](int i) {  // charge the time since the last mark to section i
      if (a.collect && etid == 0) {
        const long long now = clock64();
        s_sec[i] += (unsigned long long)(now - t_mark);
        t_mark = now;
      }
    };
    // threshold -> per-query terms of the separable test (thread g < QG)
    auto set_query_terms = [&](int g, float tau, float sq) {
      const float stq = tau == INFINITY ? 1e18f : fminf(__fsqrt_ru(__fdiv_ru(tau, a.lb_scale)), 1e18f);
      const float E = __fadd_ru(qeq[g], stq);
      const float nq = qnq[g], rq = qrq[g];
      // FP8: the query split's underflow error (at most s_cunder |x|_2 on the
      // partial product) joins the g rq coefficient of rx
      qterm[g] = make_float4(E, FP8 ? fmaf(g_slack, rq, s_cunder) : g_slack * rq, sq,
                             0.5f * (nq - g_slack * nq - E * E - kEval * (rq + E) * (rq + E)));
      qtau[g] = tau;
    };
    auto tau_now = [&](unsigned long long key, float seed) {
      const float t = key == kEmptyKey ? INFINITY : __fmul_ru(key_dist(key), 1.000001f);
      return fminf(t, seed);
    };
    int cur_item = -1, cur_level = -1, G = 0, Npad = 16, nch = 0;
    int64_t ch0 = 0;
    uint32_t mpar = 0;
    // prefetch registers: the next boundary's query slices, tails and
    // threshold inputs
    float4 pf[2 * PF_CHUNKS];
    float tpf[TPF];
    unsigned long long key_pf = kEmptyKey;
    float seed_pf = INFINITY, sq_pf = 0.f;

    // B tiles for level l, 8 query elements at a time: bf16 hi / lo parts,
    // or (FP8) three E4M3 terms of the scaled query in three tiles
    auto store_b = [&](unsigned char* bhi, int g, int c8, int w, const float (&f)[8]) {
      unsigned char* blo = bhi + lay.bbytes;
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
    auto build_b = [&](int l, int first_chunk) {  // straight from global memory
      const int m = a.level_off[l], w = a.level_off[l + 1] - m;
      unsigned char* bhi = bbuf + (size_t)bidx(l) * 2 * lay.bbytes;
      for (int i = etid + first_chunk * NEPI; i < Npad * (w / 8); i += NEPI) {
        const int g = i / (w / 8), c8 = i % (w / 8);
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (g < G) {
          const float* src = a.qt + (int64_t)qid[g] * d + m + c8 * 8;
          const float4 f0 = *reinterpret_cast<const float4*>(src);
          const float4 f1 = *reinterpret_cast<const float4*>(src + 4);
          f[0] = f0.x, f[1] = f0.y, f[2] = f0.z, f[3] = f0.w;
          f[4] = f1.x, f[5] = f1.y, f[6] = f1.z, f[7] = f1.w;
        }
        store_b(bhi, g, c8, w, f);
      }
    };
    // loads for the boundary into level l + 1: the query slices of level
    // l + 1 + AHEAD (the B tile built there), the tails that level l + 1
    // tests with and the threshold inputs
    auto prefetch = [&](int l) {
      const int lb = l + 1 + AHEAD;
      if (lb < L) {
        const int m1 = a.level_off[lb], w1 = a.level_off[lb + 1] - m1;
#pragma unroll
        for (int i = 0; i < PF_CHUNKS; ++i) {
          const int e2 = etid + i * NEPI;
          const int g = e2 / (w1 / 8), c8 = e2 % (w1 / 8);
          if (e2 < Npad * (w1 / 8) && g < G) {
            const float* src = a.qt + (int64_t)qid[g] * d + m1 + c8 * 8;
            pf[2 * i] = *reinterpret_cast<const float4*>(src);
            pf[2 * i + 1] = *reinterpret_cast<const float4*>(src + 4);
          } else {
            pf[2 * i] = pf[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
      if (l + 1 < L) {
#pragma unroll
        for (int u = 0; u < TPF; ++u) {
          const int e2 = etid + u * NEPI;
          tpf[u] = e2 < nch * CH ? a.tails[((ch0 + e2 / CH) * (L + 1) + l + 2) * CH + (e2 % CH)]
                                 : 0.f;
        }
        if (etid < QG && qid[etid] >= 0 && qk[etid] > 0) {
          const int q = qid[etid];
          key_pf = ld_volatile_u64(a.topk + (int64_t)q * a.k_max + qk[etid] - 1);
          seed_pf = __ldcg(a.tau_seed + q);
          sq_pf = a.eps * a.qtail[(int64_t)q * (L + 1) + l + 2];
        }
      }
    };
    auto prologue = [&](int item) {
      es.sync();  // the previous item's per-item data is no longer read
      const int4 it = a.items[item];
      ch0 = a.chunk_off[it.x] + (int64_t)it.y * S;
      const int64_t chE = a.chunk_off[it.x + 1];
      nch = (int)((chE - ch0) < S ? (chE - ch0) : S);
      G = it.w;
      Npad = G <= 16 ? 16 : ((G + 15) & ~15);
      if (etid == 0) s_qmax = 0u;
      es.sync();
      if (etid < QG) {
        const int q = etid < G ? a.bucket[it.z + etid] : -1;
        qid[etid] = q;
        if (q >= 0) {
          const float4 inf = a.qinfo[q];
          qnq[etid] = inf.x;
          qrq[etid] = inf.y;
          qeq[etid] = inf.z;
          qk[etid] = a.kq[q];
          if (FP8) atomicMax(&s_qmax, __float_as_uint(inf.w));  // inf.w = max_j |q~_j| >= 0
        } else {
          qnq[etid] = qrq[etid] = qeq[etid] = 0.f;
          qk[etid] = 0;
        }
      }
      for (int i = etid; i < S * CH; i += NEPI) {
        const int c = i / CH;
        if (c < nch) {
          const int64_t slot = (ch0 + c) * CH + (i % CH);
          const float nx = a.xn2[slot], rx = sqrtf(nx), exv = a.ex[slot];
          const float s2 = (rx + exv) * (rx + exv);
          cHx[i] = 0.5f * (nx - g_slack * nx - exv * exv - kEval * s2);
          crx[i] = rx;
          cex[i] = exv;
          cxn[i] = nx;
          cid[i] = a.ids[slot];
          csx[i] = a.tails[((ch0 + c) * (L + 1) + 1) * CH + (i % CH)];
        } else {
          cHx[i] = crx[i] = cex[i] = cxn[i] = csx[i] = 0.f;
          cid[i] = -1;
        }
      }
      es.sync();
      if (FP8 && etid == 0) {
        // query scale 2^-e: the group's largest |q~_j| times it is at most
        // 448 (no E4M3 term saturates); a smaller e (at most -60) only adds
        // underflow, which s_cunder bounds: each element loses at most
        // 2^-10 of the scaled unit, so the partial product at most
        // 2^-10 2^e sqrt(d) |x|_2
        const float qm = __uint_as_float(s_qmax);
        int ex2 = 0;
        if (qm > 0.f) frexpf(qm / 448.f, &ex2);
        if (ex2 > 60) atomicOr(a.err, kErrBadInput);
        ex2 = max(-60, min(60, ex2));
        s_qs = ldexpf(1.f, -ex2);
        s_cunder = __fmul_ru(ldexpf(1.f, ex2 - 10), __fsqrt_ru((float)d));
      }
      {
        uint32_t gm = 0;  // this thread's query slice: members with k > 0
        for (int j = 0; j < QS; ++j) {
          const int g = QS * slice + j;
          if (g < G && qk[g] > 0) gm |= 1u << j;
        }
        for (int c = 0; c < S; ++c) {
          const bool v = c < nch && cid[c * CH + row] >= 0;
          alive[(c * CH + row) * NSL + slice] = (uint16_t)(v ? gm : 0u);
          const unsigned bal = __ballot_sync(0xffffffffu, v && gm);
          if (lane == 0) rowlive[c][e] = bal;
        }
      }
      es.sync();
      if (etid < QG) {
        const int q = qid[etid];
        if (q >= 0 && qk[etid] > 0) {
          const unsigned long long key =
              ld_volatile_u64(a.topk + (int64_t)q * a.k_max + qk[etid] - 1);
          set_query_terms(etid, tau_now(key, __ldcg(a.tau_seed + q)),
                          a.eps * a.qtail[(int64_t)q * (L + 1) + 1]);
        } else {
          qterm[etid] = make_float4(0.f, 0.f, 0.f, -INFINITY);
          qtau[etid] = -1.f;
        }
      }
      if (FP8) {
        const float qinv = 1.f / s_qs;  // a power of two: exact
        for (int i = etid; i < S * CH; i += NEPI)
          cfr[i] = i / CH < nch ? a.xscale[(ch0 + i / CH) * CH + (i % CH)] * qinv : 0.f;
      }
      if (a.collect && etid == 0) {  // level 0's live rows (algorithmic bytes)
        const int w0 = a.level_off[1] - a.level_off[0];
        unsigned long long n = 0;
        for (int c = 0; c < nch; ++c)
          for (int qq = 0; qq < 4; ++qq) {
            uint32_t m = 0;
            for (int j = 0; j < NSL; ++j) m |= rowlive[c][((qq + 2) & 3) + 4 * j];
            n += __popc(m);
          }
        atomicAdd(&s_stat[5], n * (unsigned long long)(w0 * EB + 4));
      }
      for (int lv = 0; lv <= AHEAD && lv < L; ++lv) build_b(lv, 0);
      fence_proxy_async_smem();
      for (int lv = 0; lv <= AHEAD && lv < L; ++lv) mbar_arrive_plain(&b_full[bidx(lv)]);
      prefetch(0);
      es.sync();
    };
    auto boundary = [&](int l) {  // into level l >= 1
      es.sync();  // level l - 1 is finished: its query terms, tails and B buffer are free
      if (etid < QG && qid[etid] >= 0 && qk[etid] > 0)
        set_query_terms(etid, tau_now(key_pf, seed_pf), sq_pf);
#pragma unroll
      for (int u = 0; u < TPF; ++u) csx[etid + u * NEPI] = tpf[u];
      const int lb = l + AHEAD;  // the level whose query tiles are built here
      if (lb < L) {
        const int m1 = a.level_off[lb], w1 = a.level_off[lb + 1] - m1;
        unsigned char* bhi = bbuf + (size_t)bidx(lb) * 2 * lay.bbytes;
#pragma unroll
        for (int i = 0; i < PF_CHUNKS; ++i) {
          const int e2 = etid + i * NEPI;
          if (e2 < Npad * (w1 / 8)) {
            const int g = e2 / (w1 / 8), c8 = e2 % (w1 / 8);
            const float f[8] = {pf[2 * i].x, pf[2 * i].y, pf[2 * i].z, pf[2 * i].w,
                                pf[2 * i + 1].x, pf[2 * i + 1].y, pf[2 * i + 1].z,
                                pf[2 * i + 1].w};
            store_b(bhi, g, c8, w1, f);
          }
        }
        if (Npad * (w1 / 8) > PF_CHUNKS * NEPI) build_b(lb, PF_CHUNKS);  // wide levels
        fence_proxy_async_smem();
        mbar_arrive_plain(&b_full[bidx(lb)]);
      }
      prefetch(l);
      es.sync();
    };

    int step = 0;
    while (true) {
      const int slot = step % RING;
      const bool ok = __all_sync(
          0xffffffffu, wait_or_fail(&desc_full[slot], (uint32_t)(step / RING) & 1u, vfail));
      const int4 dsc = ok ? epi_desc[slot] : make_int4(-1, 0, 0, 0);
      if (dsc.x < 0) break;  // the terminal step (or a failed role)
      const int c = dsc.y & 0xff, l = (dsc.y >> 8) & 0xff;
      section(2);
      if (dsc.x != cur_item) {
        prologue(dsc.x);
        cur_item = dsc.x;
        cur_level = 0;
        section(0);
      } else if (l != cur_level) {
        boundary(l);
        cur_level = l;
        section(3);
      }
      const int w = a.level_off[l + 1] - a.level_off[l];
      const bool test = a.prune || l == L - 1;
      const bool okm = __all_sync(
          0xffffffffu, timed_wait(&mma_done[c], (mpar >> c) & 1u, vfail,
                                  a.collect && etid == 0 ? &s_wait[2] : nullptr));
      mpar ^= 1u << c;
      tc::fence_after_sync();
      const int r0 = c * CH + row;
      uint32_t wm = alive[r0 * NSL + slice];
      const bool any_warp = okm && __any_sync(0xffffffffu, wm != 0);
      float v[QS];
      float rx = 0.f, exv = 0.f, fr = 1.f;
      if (any_warp) {
        const float sx = csx[r0], Hx = cHx[r0];
        rx = crx[r0];
        exv = cex[r0];
        if (FP8) fr = cfr[r0];
        if (a.collect) {
          const unsigned np = __reduce_add_sync(0xffffffffu, (unsigned)__popc(wm));
          if (lane == 0) {
            atomicAdd(&s_stat[0], (unsigned long long)np);
            atomicAdd(&s_stat[1], (unsigned long long)np * w);
          }
        }
        tc::tmem_ld16(tbase + lane_base + (uint32_t)(c * QG + QS * slice), v);
        if (test) {
          // query columns some lane of the warp still holds (warp-uniform)
          const uint32_t wany = __reduce_or_sync(0xffffffffu, wm);
          const float4* qt = qterm + QS * slice;
          uint32_t pruned = 0;
#pragma unroll
          for (int g = 0; g < QS; ++g) {
            if ((wany >> g) & 1u) {
              const float4 t = qt[g];
              const float p = FP8 ? v[g] * fr : v[g];
              const float P = fmaf(t.x, exv, fmaf(t.y, rx, fmaf(t.z, sx, p)));
              pruned |= (P < t.w + Hx ? 1u : 0u) << g;
            }
          }
          wm &= ~pruned;
        }
        alive[r0 * NSL + slice] = (uint16_t)wm;
      } else {
        wm = 0u;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, wm != 0);
      tc::fence_before_sync();
      if (lane == 0) {
        rowlive[c][e] = bal;
        mbar_arrive_plain(&epi_done[c]);
      }
      if (l == L - 1) {
        // survivors of the last level join the deferred re-rank list with
        // their Eq. 3 bounds (C = 0 after the last level); a full list is
        // checked and re-ranked by all epilogue threads, then the rest join
        uint32_t rem = wm;
        while (true) {
          if (rem) {
            const float xn2v = cxn[r0];
            const int32_t idv = cid[r0];
            const int64_t xslot = (ch0 + c) * CH + row;
            const float under = FP8 ? 2.f * s_cunder * rx : 0.f;  // FP8 query split
#pragma unroll
            for (int g = 0; g < QS; ++g) {
              if ((rem >> g) & 1u) {
                const int pos = atomicAdd(&s_np, 1);
                if (pos < kPend) {
                  const int gq = QS * slice + g;
                  const float p = FP8 ? v[g] * fr : v[g];
                  const float A = qnq[gq] + xn2v - 2.f * p;
                  const float Ss = qrq[gq] + rx;
                  const float slack = fmaf(g_slack * Ss, Ss, under);
                  const float lr = sqrtf(fmaxf(A - slack, 0.f)) - (qeq[gq] + exv);
                  const float ru = __fadd_ru(__fsqrt_ru(fmaxf(A + slack, 0.f)), qeq[gq] + exv);
                  pslot[pos] = xslot;
                  pq[pos] = qid[gq];
                  pid[pos] = idv;
                  plb[pos] = lr > 0.f ? lr * lr * a.lb_scale : 0.f;
                  pub[pos] = __fmul_ru(__fmul_ru(ru, ru), a.ub_scale);
                  rem &= ~(1u << g);
                }
              }
            }
          }
          if (!es.any_of(rem != 0, etid)) break;
          if (*vfail) break;  // a failed meeting: the list is not flushed
          section(2);
          const int nk = flush_pending(a, es, kPend, etid, pslot, pq, pid, plb, pub, keep, rnk,
                                       s_flush);
          if (a.collect && etid == 0) s_stat[4] += nk;
          if (etid == 0) s_np = 0;
          es.sync();
          section(5);
        }
      }
      ++step;
    }
    section(2);
    // the last deferred survivors
    es.sync();
    const int np = s_np < kPend ? s_np : kPend;
    if (np > 0 && !*vfail) {
      const int nk = flush_pending(a, es, np, etid, pslot, pq, pid, plb, pub, keep, rnk, s_flush);
      if (a.collect && etid == 0) s_stat[4] += nk;
    }
    section(5);
    if (a.collect && etid == 0) s_sec[6] = (unsigned long long)(clock64() - t_kernel);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 64) {
    if (s_fail) atomicOr(a.err, kErrTimeout);
    if (a.collect) {
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
      for (int i = 0; i < 4; ++i) atomicAdd(&a.stats[26 + i], s_wait[i]);
    }
  }
  tc::fence_after_sync();
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

// Stages of the A ring that fit next to the fixed part of the layout.
static int ring_stages(int max_w, bool fp8, int nb, size_t budget) {
  const int eb = fp8 ? 1 : 2;
  const Lay fixed(max_w, eb, 0, nb);
  if (budget <= fixed.total) return 0;
  return (int)std::min<size_t>(kMaxStages, (budget - fixed.total) / fixed.abytes);
}

size_t verify_tc_smem(int max_w, bool fp8) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  const size_t budget = (size_t)optin - 16 * 1024;
  for (int nb = 2; nb >= 1; --nb) {
    const int na = ring_stages(max_w, fp8, nb, budget);
    if (na >= 3) return Lay(max_w, fp8 ? 1 : 2, na, nb).total + 1024;
  }
  return 0;
}

int launch_verify_tc(const VerifyTCArgs& a_in, cudaStream_t st) {
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
  const bool fp8 = a_in.fp8 != 0;
  const void* kern = fp8 ? (const void*)verify_tc_kernel<true> : (const void*)verify_tc_kernel<false>;
  cudaFuncAttributes fa;
  PANO_CUDA(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, sms = 0, optin = 0, per_sm = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  PANO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PANO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PANO_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  const size_t budget = (size_t)optin - fa.sharedSizeBytes - 1024;  // 1024: alignment slack
  VerifyTCArgs a = a_in;
  // double-buffered query tiles with at least three A stages, else single
  a.nb = 2;
  a.na = ring_stages(a.max_w, fp8, 2, budget);
  if (a.na < 3) {
    a.nb = 1;
    a.na = ring_stages(a.max_w, fp8, 1, budget);
  }
  if (a.na < 3) return fail(PANO_EINVAL, "tensor-core verify tiles do not fit in shared memory");
  // One CTA per SM holds all 512 TMEM columns: the request is kept above
  // half of the SM's shared memory so that a second CTA never lands there.
  size_t smem = Lay(a.max_w, fp8 ? 1 : 2, a.na, a.nb).total + 1024;
  smem = std::max(smem, (size_t)per_sm / 2 + 1024);
  smem = std::min(smem, budget + 1024);
  void* args[] = {&a};
  PANO_CUDA(cudaLaunchKernel(kern, dim3(sms), dim3(NT), args, smem, st));
  return PANO_OK;
}

}  // namespace pano
