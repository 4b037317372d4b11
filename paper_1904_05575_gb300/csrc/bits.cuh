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
