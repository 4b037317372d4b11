// Conversions of FP64 numbers done with integer instructions only.
//
// On this GPU the FP64 pipe (which also executes FP64 <-> FP32 conversions)
// runs at a small fraction of the integer and FP32 rates, and the split of
// every input element would otherwise be bound by it.  Both routines read the
// IEEE-754 binary64 fields (sign, 11-bit biased exponent, 52-bit fraction)
// and assemble the narrower formats from the significand bits.  Values below
// 2^-126 in magnitude become zero; inputs are finite.
#pragma once

#include <cstdint>

namespace bse {

// Split x into P BF16 numbers, x = h_0 + ... + h_{P-1} + r: each of the first
// P-1 pieces takes the next 8 significant bits of what remains (truncation,
// so the remainder stays exactly representable), the last piece rounds to
// nearest, so |r| <= 2^-(8P+1) |x| (2^-25 for P = 3).
__device__ __forceinline__ void split_bf16_bits(double x, int P, uint16_t* h) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint16_t sign = (uint16_t)((b >> 48) & 0x8000u);
  const int e = (int)((b >> 52) & 0x7FF);
  uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // |x| = M * 2^(e - 1075)
  if (e == 0) M = 0;                                     // zero or FP64 subnormal
  for (int i = 0; i < P; ++i) {
    uint16_t out = 0;
    if (M != 0) {
      const int lead = 63 - __clzll((long long)M);
      const int sh = lead - 7;                           // keep bits [lead, lead - 7]
      uint32_t v;
      if (sh > 0) {
        v = (uint32_t)(M >> sh);
        if (i == P - 1) {
          v += (uint32_t)((M >> (sh - 1)) & 1u);         // round half up
        } else {
          M -= (uint64_t)v << sh;
        }
      } else {
        v = (uint32_t)(M << (-sh));                      // fewer than 8 bits left: exact
        M = 0;
      }
      // value = v * 2^(sh + e - 1075), v in [128, 256]
      int be = 7 + sh + e - 1075 + 127;
      if (v == 256u) {
        v = 128u;
        be += 1;
      }
      if (be > 0 && be < 255) out = (uint16_t)(sign | ((uint32_t)be << 7) | (v & 0x7Fu));
    }
    h[i] = out;
  }
}

// FP64 -> FP32, round half up on the 24-bit significand.
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  int be = e - 1023 + 127;
  if (e == 0 || be <= 0) return __uint_as_float(sign);
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint32_t v = (uint32_t)(M >> 29) + (uint32_t)((M >> 28) & 1u);   // 24 bits, rounded
  if (v == (1u << 24)) {
    v >>= 1;
    be += 1;
  }
  if (be >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((uint32_t)be << 23) | (v & 0x7FFFFFu));
}

}  // namespace bse

namespace bse {

// FP32 -> FP64 with integer instructions (exact; FP32 subnormals become zero).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0) return __longlong_as_double((long long)sign);
  const uint64_t be = e == 0xFFu ? 0x7FFull : (uint64_t)(e + 896u);
  return __longlong_as_double((long long)(sign | (be << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// sc * (hi + lo) for a compensated sum, formed as sc*hi + sc*lo with every
// rounding explicit (no contraction into an FMA), so that every kernel that
// finishes such a sum gives the same bits.
__device__ __forceinline__ float scale_hi_lo(float sc, float hi, float lo) {
  return __fadd_rn(__fmul_rn(sc, hi), __fmul_rn(sc, lo));
}

// Error-free sum of two FP32 numbers (Knuth's TwoSum): s + err == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bp = s - a;
  err = (a - (s - bp)) + (b - bp);
}

}  // namespace bse

namespace bse {

// FP64 (given as its two 32-bit words) -> FP32, round half up, 32-bit
// integer instructions only.  |x| < 2^-126 becomes a signed zero.
__device__ __forceinline__ uint32_t f64w_to_f32_bits(uint32_t lo, uint32_t hi) {
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int be = e - 896;                                     // FP32 biased exponent
  uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);            // top 23 fraction bits
  uint32_t f = ((uint32_t)be << 23) + m + ((lo >> 28) & 1u);   // rounding carries into the exponent
  f = be <= 0 ? 0u : (be >= 255 ? 0x7F800000u : f);
  return sign | f;
}

// FP32 -> BF16 bit pattern, round to nearest even (finite inputs).
__device__ __forceinline__ uint32_t f32_to_bf16_rn_bits(uint32_t u) {
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

// x (FP32) = h_0 + ... + h_{P-1} + r with every h_i a BF16 number taken to
// nearest from what remains; the remainders are exact in FP32.
template <int P>
__device__ __forceinline__ void split_f32_bf16(uint32_t u, uint32_t* h) {
  float r = __uint_as_float(u);
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const uint32_t b = f32_to_bf16_rn_bits(__float_as_uint(r));
    h[i] = b;
    if (i + 1 < P) r -= __uint_as_float(b << 16);
  }
}

}  // namespace bse
