// Blackwell (sm_100a/sm_103a) 5th-generation tensor-core primitives written
// as inline PTX: tensor-memory (TMEM) allocation, single-thread MMA issue with
// shared-memory matrix descriptors, completion tracking through mbarriers and
// warp-wide TMEM loads for the epilogue.
//
// Shared-memory operand layout used throughout (K-major, "swizzled"): a tile
// of R rows x K bf16 elements (or 2K FP8 elements: the layout is one of bytes,
// so an FP8 tile of width w is addressed as a bf16 tile of width w / 2, and
// one 32-byte K-step holds 16 bf16 or 32 FP8 elements) is stored as row-major
// rows of RB bytes
// (RB = 32, 64 or 128); wider K is split into panels of 64 elements
// (128-byte rows) stored one after another (panel stride R * 128 bytes).
// Within each 8-row atom the 16-byte chunk c of row r sits at chunk position
// c ^ f(r), f = (r & 7) for 128-byte rows, (r >> 1) & 3 for 64-byte rows and
// (r >> 2) & 1 for 32-byte rows -- the three swizzle modes of the matrix
// descriptor.  Tiles are 1024-byte aligned.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "device_common.cuh"

namespace pano {
namespace tc {

// Row width in bytes of one K panel for a level of `w` bf16 elements.
__host__ __device__ __forceinline__ int row_bytes(int w) { return w >= 64 ? 128 : 2 * w; }
// Descriptor layout code of the swizzle mode (128B = 2, 64B = 4, 32B = 6).
__host__ __device__ __forceinline__ uint32_t layout_code(int rb) {
  return rb == 128 ? 2u : (rb == 64 ? 4u : 6u);
}
// Byte offset of element (row, k) of an R-row tile (bf16).
__host__ __device__ __forceinline__ uint32_t swz_offset(int row, int k, int R, int w) {
  const int rb = row_bytes(w);
  const int panel = k >> 6;
  const int kk = k & 63;
  const int chunk = kk >> 3, within = kk & 7;
  int f;
  if (rb == 128)
    f = row & 7;
  else if (rb == 64)
    f = (row >> 1) & 3;
  else
    f = (row >> 2) & 1;
  return (uint32_t)(panel * R * 128 + row * rb + ((chunk ^ f) << 4) + within * 2);
}
// Bytes of an R x w tile.
__host__ __device__ __forceinline__ uint32_t tile_bytes(int R, int w) {
  return (uint32_t)(w >= 64 ? (w / 64) * R * 128 : R * 2 * w);
}

// Shared-memory matrix descriptor (tcgen05 form): start address >> 4 in bits
// [0,14), leading byte offset >> 4 in [16,30) (unused by swizzled K-major
// tiles, set to 1), stride byte offset >> 4 in [32,46) (distance between
// 8-row groups), descriptor version 1 in [46,48), swizzle mode in [61,64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int rb) {
  const uint64_t sbo = (uint64_t)(8 * rb) >> 4;
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= sbo << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout_code(rb) << 61;
  return d;
}
// Start-address offset of K-step s (16 bf16 / 32 E4M3 elements) of an R-row
// tile, in the descriptor's 16-byte units: (s % 4) 32-byte chunks within a
// 128-byte panel row and (s / 4) panels of R rows.  Added to a descriptor of
// the tile's base (the field cannot carry: shared addresses are < 2^18).
__device__ __forceinline__ uint64_t kstep_off(int s, int R) {
  return (uint64_t)((uint32_t)(s & 3) * 2u + (uint32_t)(s >> 2) * (uint32_t)R * 8u);
}
// Descriptor of K-step s (16 elements) of an R-row tile at `base`.
__device__ __forceinline__ uint64_t kstep_desc(uint32_t base, int s, int R, int w) {
  const int rb = row_bytes(w);
  const uint32_t panel = (uint32_t)(s >> 2);
  const uint32_t off = panel * (uint32_t)R * 128u + (uint32_t)(s & 3) * 32u;
  return smem_desc(base + off, rb);
}

// Instruction descriptor of kind::f16: bf16 x bf16 -> f32, both K-major,
// M x N (M = 128, N multiple of 16 in [16, 256]).  Bits: D format [4,6) = 1
// (f32), A format [7,10) = 1 (bf16), B format [10,13) = 1 (bf16), N >> 3 in
// [17,23), M >> 4 in [24,29).
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f8f6f4 with E4M3 A and B (format code 0 in
// [7,10) and [10,13)), f32 D, both K-major; one MMA covers 32 K elements.
__host__ __device__ __forceinline__ uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------------ TMEM
// Allocate `ncols` (power of two >= 32) columns; the address is written to
// *dst_smem.  Executed by one full warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same for E4M3 operands (kind::f8f6f4).
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once all previously issued MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive f32 columns of this thread's TMEM lane (warp w reads lanes
// 32*(w%4) .. +31; `taddr` carries the lane base in bits [16,32)).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive f32 columns (same lane rule).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// bf16 hi/lo split of an FP32 value: x ~= hi + lo with |x - hi - lo| <=
// 2^-16 |x| (both round to nearest).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no
// infinities) of an FP32 value, rounded to nearest even and saturated to
// +-448; and the exact FP32 value of an E4M3 byte.
__device__ __forceinline__ uint8_t f32_to_e4m3(float x) {
  return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float e4m3_to_f32(uint8_t b) {
  // normal: exponent rebiased (7 -> 127), mantissa to FP32's top bits;
  // subnormal (exponent field 0): mantissa * 2^-9
  const uint32_t e = (b >> 3) & 0xfu, mm = b & 7u;
  const float m = e ? __uint_as_float(((e + 120u) << 23) | (mm << 20)) : (float)mm * 0x1p-9f;
  return (b & 0x80u) ? -m : m;
}

// Three-term E4M3 split of an FP32 value y with |y| <= 448: y ~= t0 + t1 + t2,
// each term the E4M3 rounding of the remainder (the remainders are exact in
// FP32).  |y - t0 - t1 - t2| <= max(2^-12 |y|, 2^-10): each rounding loses at
// most 2^-4 of a normal value or 2^-10 below E4M3's normal range.
__device__ __forceinline__ void split3_e4m3(float y, uint8_t& t0, uint8_t& t1, uint8_t& t2) {
  t0 = f32_to_e4m3(y);
  const float r1 = y - e4m3_to_f32(t0);
  t1 = f32_to_e4m3(r1);
  const float r2 = r1 - e4m3_to_f32(t1);
  t2 = f32_to_e4m3(r2);
}

}  // namespace tc
}  // namespace pano
