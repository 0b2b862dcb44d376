// Device helpers shared by the library's kernels: bulk-async (TMA engine)
// copies with mbarrier completion, bounded waits, (distance, id) keys and the
// lock-free k-smallest insertion used for the running top-k.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pano {

// Error bits written into the per-call device status word.
enum : int {
  kErrTimeout = 1,   // a bounded wait gave up
  kErrOverflow = 2,  // a capacity bound was exceeded (result still valid)
  kErrBadInput = 4,  // an out-of-range per-query value was clamped
};

// Roughly one second of spinning at GB300 clocks before a wait gives up.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// One bulk-async copy global -> shared completing on `bar` (TMA engine,
// non-tensor form).  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar`; false after ~kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// ------------------------------------------------------- (dist, id) keys
// Non-negative FP32 distances order like their bit patterns, so a 64-bit key
// (dist bits << 32 | id) orders by (distance, id).  The empty key is ~0.
constexpr unsigned long long kEmptyKey = ~0ULL;

__device__ __forceinline__ unsigned long long make_key(float dist, int32_t id) {
  dist = fmaxf(dist, 0.0f);
  return (static_cast<unsigned long long>(__float_as_uint(dist)) << 32) |
         static_cast<uint32_t>(id);
}
__device__ __forceinline__ float key_dist(unsigned long long k) {
  return __uint_as_float(static_cast<uint32_t>(k >> 32));
}
__device__ __forceinline__ int32_t key_id(unsigned long long k) {
  return static_cast<int32_t>(static_cast<uint32_t>(k & 0xffffffffULL));
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Insert `key` into the ascending k-slot array `slots` shared by concurrent
// inserters.  Each step is an atomic compare-exchange between the carried
// key and one slot (atomicMin keeps the smaller, the larger moves on), so
// once all inserts have finished the slots hold the k smallest keys ever
// inserted, in ascending order.  A slot whose current value is already below
// the carried key would keep it, so those steps are skipped.
__device__ __forceinline__ void topk_insert(unsigned long long* slots, int k,
                                            unsigned long long key) {
  int j = 0;
  while (j < k && ld_volatile_u64(slots + j) < key) ++j;
  for (; j < k; ++j) {
    unsigned long long old = atomicMin(slots + j, key);
    if (old == kEmptyKey || old == key) return;  // an equal key is the same pair: kept once
    key = old > key ? old : key;
  }
}

// topk_insert by one thread whose slot reads go out in batches of eight
// independent loads (one round per eight slots, not one per slot), so that
// many threads can each insert a key at once and their compare-exchange
// chains overlap.  A read may be stale: slots only ever decrease, so the
// first slot found not below the key is never past the key's place, and
// starting early only adds steps that leave a slot unchanged.
__device__ __forceinline__ void topk_insert_thread(unsigned long long* slots, int k,
                                                   unsigned long long key) {
  int start = k;
  for (int j0 = 0; j0 < k && start == k; j0 += 8) {
    unsigned long long v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = j0 + u < k ? ld_volatile_u64(slots + j0 + u) : kEmptyKey;
#pragma unroll
    for (int u = 7; u >= 0; --u)
      if (v[u] >= key) start = j0 + u;
  }
  for (int j = start; j < k; ++j) {
    unsigned long long old = atomicMin(slots + j, key);
    if (old == kEmptyKey || old == key) return;  // an equal key is the same pair: kept once
    key = old > key ? old : key;
  }
}

// topk_insert issued by a whole warp: the slots are read once in parallel
// (one round instead of a chain of dependent reads) to find the first slot
// not below the key; lane 0 then runs the compare-exchange chain from there.
// All 32 lanes must call it with the same arguments.
__device__ __forceinline__ void topk_insert_warp(unsigned long long* slots, int k,
                                                 unsigned long long key) {
  const int lane = threadIdx.x & 31;
  int start = k;
  for (int j0 = 0; j0 < k; j0 += 32) {
    const int j = j0 + lane;
    const bool ge = j < k && ld_volatile_u64(slots + j) >= key;
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    if (m) {
      start = j0 + __ffs(m) - 1;
      break;
    }
  }
  if (lane == 0)
    for (int j = start; j < k; ++j) {
      unsigned long long old = atomicMin(slots + j, key);
      if (old == kEmptyKey || old == key) return;  // an equal key is the same pair: kept once
      key = old > key ? old : key;
    }
}

// Hint that `bytes` (a multiple of 16, 16-byte aligned) at p will be read
// soon: a bulk prefetch into L2 (no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// sqrt(x) rounded up, for x >= 0 where only an upper bound is needed: the
// approximate square root (sqrt.approx.f32, whose relative error is a few
// units of 2^-23) times 1 + 2^-18, rounded up.  One multiply on top of the
// approximation, against the longer sequence of the IEEE directed-rounding
// square root.  Inputs below 2^-126 (zero and subnormals) are raised to it,
// so the result there is 2^-63 (times 1 + 2^-18), still an upper bound.
// panorama_debug_sqrt_up exposes it so that a test checks the bound against
// FP64 over the whole range.
__device__ __forceinline__ float sqrt_up(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fmaxf(x, 0x1p-126f)));
  return __fmul_ru(r, 1.0f + 0x1p-18f);
}

// Order-preserving map of any FP32 value to uint32.
__device__ __forceinline__ uint32_t float_ordered(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace pano
