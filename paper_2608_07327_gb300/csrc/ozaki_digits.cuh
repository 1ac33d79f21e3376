// Exact splitting of FP64 values into signed base-128 digits for the tensor-core products (Ozaki et
// al., "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012). A value x of a group (a row or a
// column) whose largest biased exponent is emax is written as
//     x = 2^(emax - 1022) * sum_{t=0..7} d_t 2^(-7 - 7t)   (+ rounding below 2^-56 of the scale),
// d_t an integer in [-127, 127] taken straight from the 53-bit significand (integer shifts): exact
// in FP16. A product of two such digits is below 2^14.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace mbpcg {

constexpr int kOzDigits = 8;

__device__ __forceinline__ int biased_exponent(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// |x| 2^(1022 - emax) 2^56 as an integer below 2^56 (the 8 digits' bits), and the sign of x.
__device__ __forceinline__ unsigned long long ozaki_magnitude(double x, int emax, int& sgn) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (e != 0 && e != 0x7FF && emax != 0) {
    const unsigned long long mant = ((unsigned long long)bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int shift = e - emax + 3;  // X = |x| 2^(1022 - emax) 2^56 < 2^56
    // below 2^-3 of the group's largest value the significand is shifted out at the bottom: round
    // to nearest there (a truncation would bias every product towards zero)
    X = shift >= 0 ? (mant << shift) : (shift > -60 ? ((mant + (1ull << (-shift - 1))) >> (-shift)) : 0ull);
  }
  sgn = bits < 0 ? -1 : 1;
  return X;
}

// Digit t of a magnitude from ozaki_magnitude.
__device__ __forceinline__ int ozaki_digit(unsigned long long X, int sgn, int t) {
  return sgn * (int)((X >> (49 - 7 * t)) & 127ull);
}

// The 8 signed base-128 digits of x relative to the scale 2^(emax - 1022).
__device__ __forceinline__ void ozaki_digits(double x, int emax, int (&d)[kOzDigits]) {
  int sgn;
  const unsigned long long X = ozaki_magnitude(x, emax, sgn);
#pragma unroll
  for (int t = 0; t < kOzDigits; ++t) d[t] = ozaki_digit(X, sgn, t);
}

// The digits of a magnitude from ozaki_magnitude, one per byte: hi holds digits 0..3 (digit t in byte
// 3 - t), lo digits 4..7 (digit t in byte 7 - t); every byte is below 128.
__device__ __forceinline__ uint32_t oz_spread4(uint32_t v) {  // v < 2^28: its 7-bit fields to bytes
  return (v & 0x7Fu) | ((v << 1) & 0x7F00u) | ((v << 2) & 0x7F0000u) | ((v << 3) & 0x7F000000u);
}
__device__ __forceinline__ void oz_digit_bytes(unsigned long long X, uint32_t& hi, uint32_t& lo) {
  hi = oz_spread4((uint32_t)(X >> 28));
  lo = oz_spread4((uint32_t)X & 0xFFFFFFFu);
}

// Signs of two values as the FP16 pairs (s_a, s_b) and (-1024 s_a, -1024 s_b) (s = +-1) that
// oz_f16_digit_pair takes.
__device__ __forceinline__ void oz_sign_pair(int sa, int sb, uint32_t& s2, uint32_t& c2) {
  s2 = (sa < 0 ? 0xBC00u : 0x3C00u) | ((sb < 0 ? 0xBC00u : 0x3C00u) << 16);
  c2 = (sa < 0 ? 0x6400u : 0xE400u) | ((sb < 0 ? 0x6400u : 0xE400u) << 16);
}

// Digit t of two values as an FP16 pair (value a in the low half), from their digit bytes (wa, wb:
// the hi or lo word of each, by t) and their signs: one byte permutation puts the two digit bytes in
// the low bytes of the halves with zero high bytes (the selector's sign-replicate bit copies the top
// bit of a byte below 128), an OR makes them 1024 + d (exact in FP16), and one FP16 multiply-add
// s (1024 + d) - 1024 s leaves s d exactly.
__device__ __forceinline__ uint32_t oz_f16_digit_pair(uint32_t wa, uint32_t wb, int t, uint32_t s2, uint32_t c2) {
  const uint32_t b = 3u - (uint32_t)(t & 3);
  const uint32_t sel = b | ((8u | b) << 4) | ((4u + b) << 8) | ((12u + b) << 12);
  uint32_t w;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(w) : "r"(wa), "r"(wb), "r"(sel));
  w |= 0x64006400u;
  const __half2 v = __hfma2(*reinterpret_cast<const __half2*>(&w), *reinterpret_cast<const __half2*>(&s2),
                            *reinterpret_cast<const __half2*>(&c2));
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Two digits (|d| <= 127) as an FP16 pair (the first in the low half), with integer operations and
// one half-precision subtraction: 1024 + (d + 128) is an FP16 with bits 0x6400 + d + 128 (exact for
// 0 <= d + 128 < 1024), and subtracting 1024 + 128 from both halves at once leaves d exactly.
__device__ __forceinline__ uint32_t oz_f16_pair_of_ints(int d0, int d1) {
  const uint32_t b = (uint32_t)(0x6480 + d0) | ((uint32_t)(0x6480 + d1) << 16);
  const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&b), __half2half2(__ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&v);
}

}  // namespace mbpcg
