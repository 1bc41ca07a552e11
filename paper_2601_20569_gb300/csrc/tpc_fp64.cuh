// Exact FP32 <-> FP64 conversions with integer operations.
//
// GB300's FP64 unit is narrow, and a hardware conversion occupies it like an
// FP64 multiply: the looper update of the final fit would spend about a third
// of its FP64 issue on conversions.  widen() is exact for every finite float;
// narrow() rounds to nearest even exactly as the hardware conversion does.
// Values outside the normal float range (widen: denormals, infinities, NaN;
// narrow: non-zero results below the smallest normal float or above the
// largest float exponent) take the hardware conversion; zeros do not (fresh
// covariances have many exact zeros).  Host-compilable so that a CPU test
// can check both against the host's IEEE conversions.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define TPC_HD __host__ __device__ __forceinline__
#else
#define TPC_HD inline
#endif

namespace tpc {

TPC_HD uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

TPC_HD float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

TPC_HD double bitsd(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double d;
  std::memcpy(&d, &b, 8);
  return d;
#endif
}

TPC_HD void dbits(double d, uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
  hi = (uint32_t)__double2hiint(d);
  lo = (uint32_t)__double2loint(d);
#else
  uint64_t b;
  std::memcpy(&b, &d, 8);
  hi = (uint32_t)(b >> 32);
  lo = (uint32_t)b;
#endif
}

// float -> double: sign, exponent rebiased by 1023 - 127, mantissa shifted
// into the top of the 52-bit field.
TPC_HD double widen(float f) {
  const uint32_t u = fbits(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((u & 0x7fffffffu) == 0u) return bitsd(u & 0x80000000u, 0u);
    return (double)f;
  }
  return bitsd((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3), u << 29);
}

// double -> float, round to nearest even: keep mantissa bits 51..29, round on
// bits 28..0 (a carry into the exponent is the correct rounding).
TPC_HD float narrow(double d) {
  uint32_t hi, lo;
  dbits(d, hi, lo);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (((hi & 0x7fffffffu) | lo) == 0u) return bitsf(hi & 0x80000000u);  // signed zero
  if (e < 897u || e > 1150u) return (float)d;
  const uint32_t m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  uint32_t f = (hi & 0x80000000u) | ((e - 896u) << 23) | m23;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) f += 1u;
  return bitsf(f);
}

}  // namespace tpc
