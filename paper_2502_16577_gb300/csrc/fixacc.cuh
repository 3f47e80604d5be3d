// Exact accumulation of the Gray-code terms in a 192-bit fixed-point integer
// (an alternative to the double-double "quad" outer sum of Sec. 5 that uses
// no FP64 instruction at all).
//
// A term is sign * M * 2^E with the 63-bit product mantissa M in [2^62, 2^63)
// (see prod_mul).  The accumulator A is a two's-complement integer of six
// 32-bit words that represents A * 2^L0.  L0 is fixed per launch from the
// bound |term| < 2^(bound_log2 + 1) (Sec. 5's scaling argument): with
// L0 = bound_log2 + n - 190, the sum of all 2^(n-1) terms stays below 2^190 in
// magnitude and every term is added without rounding, only bits below 2^L0
// (more than 2^(190 - 62 - n) below the largest possible term) being dropped.
// Integer sums are associative, so the lane, warp and CTA reductions are
// exact and independent of their order.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace permgpu {

struct Fix192 {
  uint32_t w[6];
};

__device__ __forceinline__ void fix_zero(Fix192& a) {
#pragma unroll
  for (int k = 0; k < 6; ++k) a.w[k] = 0u;
}

// The unit exponent of a launch (see above); n >= 1.
__device__ __forceinline__ int fix_l0(int bound_log2, int n) { return bound_log2 + (n < 2 ? 2 : n) - 190; }

// a += (-1)^neg * M * 2^s for M = m1:m0 < 2^63 and s <= 127 (s < 0 shifts M
// right, dropping the bits below the unit).
__device__ __forceinline__ void fix_add(Fix192& a, uint32_t m0, uint32_t m1, int s, uint32_t neg) {
  unsigned long long M = ((unsigned long long)m1 << 32) | m0;
  if (s < 0) {
    M = s > -64 ? M >> (-s) : 0ull;
    s = 0;
  }
  const unsigned long long lo = M << (s & 63);
  const unsigned long long hi = (s & 63) ? M >> (64 - (s & 63)) : 0ull;
  const bool up = s >= 64;  // the addend occupies 64-bit words (0, 1) or (1, 2)
  const unsigned long long w0 = up ? 0ull : lo, w1 = up ? lo : hi, w2 = up ? hi : 0ull;
  const uint32_t m = 0u - neg;  // subtract: add the complement plus one
  uint32_t x[6] = {(uint32_t)w0 ^ m, (uint32_t)(w0 >> 32) ^ m, (uint32_t)w1 ^ m,
                   (uint32_t)(w1 >> 32) ^ m, (uint32_t)w2 ^ m, (uint32_t)(w2 >> 32) ^ m};
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "add.cc.u32 t, %6, 0xFFFFFFFF;\n\t"  // carry = neg (0 or 1)
      "addc.cc.u32 %0, %0, %7;\n\t"
      "addc.cc.u32 %1, %1, %8;\n\t"
      "addc.cc.u32 %2, %2, %9;\n\t"
      "addc.cc.u32 %3, %3, %10;\n\t"
      "addc.cc.u32 %4, %4, %11;\n\t"
      "addc.u32 %5, %5, %12;\n\t"
      "}"
      : "+r"(a.w[0]), "+r"(a.w[1]), "+r"(a.w[2]), "+r"(a.w[3]), "+r"(a.w[4]), "+r"(a.w[5])
      : "r"(neg), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]));
}

// a += b (192-bit).
__device__ __forceinline__ void fix_add_fix(Fix192& a, const Fix192& b) {
  asm("add.cc.u32 %0, %0, %6;\n\t"
      "addc.cc.u32 %1, %1, %7;\n\t"
      "addc.cc.u32 %2, %2, %8;\n\t"
      "addc.cc.u32 %3, %3, %9;\n\t"
      "addc.cc.u32 %4, %4, %10;\n\t"
      "addc.u32 %5, %5, %11;"
      : "+r"(a.w[0]), "+r"(a.w[1]), "+r"(a.w[2]), "+r"(a.w[3]), "+r"(a.w[4]), "+r"(a.w[5])
      : "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
}

__device__ __forceinline__ Fix192 fix_shfl_down(const Fix192& v, int off) {
  Fix192 r;
#pragma unroll
  for (int k = 0; k < 6; ++k) r.w[k] = __shfl_down_sync(0xffffffffu, v.w[k], off);
  return r;
}

// Warp sum (lane 0 holds it).
__device__ __forceinline__ Fix192 fix_warp_sum(Fix192 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const Fix192 o = fix_shfl_down(v, off);
    fix_add_fix(v, o);
  }
  return v;
}

// Block sum for a block of `warps` warps (thread 0 holds it).
template <int WARPS>
__device__ __forceinline__ Fix192 fix_block_sum(Fix192 v) {
  __shared__ Fix192 s_w[WARPS];
  v = fix_warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_w[w] = v;
  __syncthreads();
  Fix192 r;
  fix_zero(r);
  if (threadIdx.x == 0)
    for (int k = 0; k < WARPS; ++k) fix_add_fix(r, s_w[k]);
  return r;
}

// 2^e as binary64 for -1074 <= e <= 1023 (0 below, +inf above).
__device__ __forceinline__ double pow2_exact(int e) {
  if (e > 1023) return __longlong_as_double(0x7ff0000000000000ll);
  if (e >= -1022) return __longlong_as_double((long long)(e + 1023) << 52);
  if (e >= -1074) return __longlong_as_double(1ll << (e + 1074));
  return 0.0;
}

// A * 2^L0 as a double-double: the six words are exact binary64 values,
// added from the most significant down (faithful to about 2^-104).
__device__ __forceinline__ dd fix_to_dd(const Fix192& a, int L0) {
  dd r = {0.0, 0.0};
  r = dd_add_d(r, (double)(int32_t)a.w[5] * pow2_exact(L0 + 160));
#pragma unroll
  for (int k = 4; k >= 0; --k) r = dd_add_d(r, (double)a.w[k] * pow2_exact(L0 + 32 * k));
  return dd_make(r.hi, r.lo);
}

}  // namespace permgpu
