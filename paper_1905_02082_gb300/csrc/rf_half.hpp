// IEEE 754 binary16 <-> binary32 conversions on the host, written from the
// format's definition (1 sign bit, 5 exponent bits with bias 15, 10 fraction
// bits; exponent 0 = zero/subnormal, 31 = infinity/NaN).  Used by volume
// export/import of the compact FP16 storage mode; the kernels use the
// hardware conversions, which follow the same definition.
#pragma once

#include <cstdint>
#include <cstring>

namespace rf {

inline float half_bits_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h >> 15) << 31;
  const uint32_t e = (h >> 10) & 0x1Fu;
  uint32_t m = h & 0x3FFu;
  uint32_t bits;
  if (e == 0x1Fu) {
    bits = sign | 0x7F800000u | (m << 13);  // infinity or NaN (payload kept)
  } else if (e != 0) {
    bits = sign | ((e + 112u) << 23) | (m << 13);  // normal: rebias 15 -> 127
  } else if (m == 0) {
    bits = sign;  // signed zero
  } else {
    // subnormal m * 2^-24: normalise the fraction into a float
    int ex = -1;
    do {
      m <<= 1;
      ++ex;
    } while ((m & 0x400u) == 0);
    bits = sign | ((uint32_t)(112 - ex) << 23) | ((m & 0x3FFu) << 13);
  }
  float f;
  std::memcpy(&f, &bits, 4);
  return f;
}

// Round to nearest, ties to even; overflow to infinity; NaN stays NaN.
inline uint16_t float_to_half_bits(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint16_t sign = (uint16_t)((x >> 16) & 0x8000u);
  const uint32_t ax = x & 0x7FFFFFFFu;
  if (ax >= 0x7F800000u) return (uint16_t)(sign | 0x7C00u | (ax > 0x7F800000u ? 0x200u : 0u));
  if (ax >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u);  // >= 65520 rounds to infinity
  const int e = (int)(ax >> 23) - 127;
  if (e >= -14) {  // normal half
    const uint32_t mant = ax & 0x7FFFFFu;
    uint32_t h = ((uint32_t)(e + 15) << 10) | (mant >> 13);
    const uint32_t rest = mant & 0x1FFFu;
    if (rest > 0x1000u || (rest == 0x1000u && (h & 1u))) ++h;  // carries into the exponent correctly
    return (uint16_t)(sign | h);
  }
  if (e < -25) return sign;  // below half the smallest subnormal: zero
  // subnormal half: value / 2^-24, rounded to nearest even
  const uint32_t mant = (ax & 0x7FFFFFu) | 0x800000u;  // 24-bit significand, value = mant * 2^(e-23)
  const int shift = -e - 1;                            // h = mant >> (shift) with value 2^-24 units
  const uint32_t h = mant >> shift;
  const uint32_t rest = mant & ((1u << shift) - 1u);
  const uint32_t halfway = 1u << (shift - 1);
  uint32_t r = h;
  if (rest > halfway || (rest == halfway && (h & 1u))) ++r;
  return (uint16_t)(sign | r);
}

}  // namespace rf
