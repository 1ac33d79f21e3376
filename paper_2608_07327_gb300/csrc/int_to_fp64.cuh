// Conversion of a 64-bit integer to the nearest FP64 value (ties to even, IEEE 754 roundTiesToEven)
// with integer operations only: on this GPU the integer-to-FP64 conversion instruction runs on the
// FP64 pipe (2 per clock per SM), which makes it the slowest step of an epilogue that converts one
// value per output. Host-compilable, so that it can be checked against the C conversion on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define MBPCG_HD __host__ __device__ __forceinline__
#else
#define MBPCG_HD inline
#endif

namespace mbpcg {

MBPCG_HD int clz64(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)u);
#else
  return __builtin_clzll(u);
#endif
}

MBPCG_HD double bits_as_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// (double)t, rounded to nearest with ties to even: the leading one is moved to bit 63, the top 53
// bits are the significand, the 11 below decide the rounding (above half, or exactly half with an
// odd significand, round up); a carry out of the significand raises the exponent.
MBPCG_HD double ll_to_double_rn(long long t) {
  if (t == 0) return 0.0;
  const uint64_t sign = t < 0 ? (1ull << 63) : 0ull;
  uint64_t u = t < 0 ? 0ull - (uint64_t)t : (uint64_t)t;
  const int lz = clz64(u);
  u <<= lz;
  uint64_t m = u >> 11;
  const uint64_t rest = u & 0x7FFull;
  m += (rest > 0x400ull || (rest == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  uint64_t e = (uint64_t)(1023 + 63 - lz);
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  return bits_as_double(sign | (e << 52) | (m & ((1ull << 52) - 1)));
}

// (double)t 2^k in one step when that is a normal number or zero (ok = true: the exponent of the
// rounded t is raised by k, no second rounding); ok = false when it would leave the normal range.
MBPCG_HD double ll_to_double_scaled_rn(long long t, int k, bool& ok) {
  ok = true;
  if (t == 0) return 0.0;
  const uint64_t sign = t < 0 ? (1ull << 63) : 0ull;
  uint64_t u = t < 0 ? 0ull - (uint64_t)t : (uint64_t)t;
  const int lz = clz64(u);
  u <<= lz;
  uint64_t m = u >> 11;
  const uint64_t rest = u & 0x7FFull;
  m += (rest > 0x400ull || (rest == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  int e = 1023 + 63 - lz + k;
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  ok = e >= 1 && e <= 2046;
  return bits_as_double(sign | ((uint64_t)(ok ? e : 1) << 52) | (m & ((1ull << 52) - 1)));
}

}  // namespace mbpcg
