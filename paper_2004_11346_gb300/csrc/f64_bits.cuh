// IEEE 754 binary64 <-> binary32 conversions in integer arithmetic (device).
#pragma once

#include <cstdint>

namespace sht {

// Round to nearest even; subnormals, infinities and NaN per the standard.
// GB300's FP64 pipe runs at a small fraction of its integer and FP32 rates,
// and the FP32 and tensor-core paths convert every FP64 input and output value
// once: on the FP64 pipe the conversions alone take milliseconds per call.
// These agree bit for bit with the hardware conversions (checked on 2^30
// patterns, including subnormal, overflow and rounding-tie cases).
__device__ __forceinline__ uint64_t rne_shift(uint64_t x, int s) {
  // x >> s rounded to nearest, ties to even (1 <= s <= 63)
  const uint64_t q = x >> s, rem = x & ((1ull << s) - 1), half = 1ull << (s - 1);
  return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}
__device__ __forceinline__ float f64_to_f32_slow(double d) {
  const uint64_t b = (uint64_t)__double_as_longlong(d);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;  // binary32 biased exponent
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  if (fe >= 1) return __uint_as_float(sign | (uint32_t)(((uint64_t)fe << 23) + rne_shift(m, 29)));
  // binary32 subnormal (or zero): value = (2^52 + m) 2^(e - 1075) = k 2^-149
  if (e == 0 || fe < -24) return __uint_as_float(sign);
  return __uint_as_float(sign | (uint32_t)rne_shift((1ull << 52) | m, 29 + 1 - fe));
}
__device__ __forceinline__ double f32_to_f64_slow(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  uint32_t e = (u >> 23) & 0xFF, m = u & 0x7FFFFFu;
  if (e == 0xFF) return __hiloint2double((int)(sign | 0x7FF00000u | (m >> 3)), (int)(m << 29));
  if (e == 0) {
    if (m == 0) return __hiloint2double((int)sign, 0);
    const int sh = __clz(m) - 8;  // bring the leading one to bit 23
    m = (m << sh) & 0x7FFFFFu;
    e = 1 - sh + 896;
  } else {
    e += 896;
  }
  return __hiloint2double((int)(sign | (e << 20) | (m >> 3)), (int)(m << 29));
}

// The same conversions with a short path for the common case, in 32-bit
// integer arithmetic on the two halves of the binary64 pattern.
// binary64 -> binary32 when the result is a normal binary32 before rounding
// (biased binary64 exponent 897..1150): the 23 result mantissa bits are the
// 20 of the high word and the top 3 of the low word, the low 29 bits decide
// the rounding (to nearest, ties to even), and a carry out of the mantissa
// moves into the exponent (up to infinity), as rounding requires.
__device__ __forceinline__ float f64_to_f32_bits(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t ex = (hi >> 20) & 0x7FFu;
  if (ex - 897u < 254u) {
    uint32_t r = (((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1FFFFFFFu;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | r);
  }
  return f64_to_f32_slow(d);
}
// binary32 -> binary64 for normal inputs: rebias the exponent (+896) and
// widen the mantissa.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u)
    return __hiloint2double((int)((u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + (896u << 20))), (int)(u << 29));
  return f32_to_f64_slow(f);
}

}  // namespace sht
