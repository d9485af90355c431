// fp_bits.cuh -- exact IEEE 754 binary32 <-> binary64 conversions done on the
// integer pipe.
//
// On this GPU the FP64 pipe also executes the conversions to and from
// binary64, at about two lanes per SM and clock.  The pseudo-time update of
// an FP32-bulk grid widens nine FP32 residuals and narrows nine new FP64
// master values to the FP32 shadow per cell; issued as conversion
// instructions they, not HBM, bound the kernel.  These functions build the
// result's sign, exponent and significand fields with integer instructions
// for every operand class (normal, subnormal, zero, infinity, NaN), so that
// no conversion instruction is issued at all.  They give the IEEE 754 results
// -- exact widening, and narrowing rounded to nearest, ties to even -- bit for
// bit; a NaN comes out quiet with as much of its payload as fits.
//
// Field layout (IEEE 754-2008, Sect. 3.4): binary32 = 1 sign, 8 exponent
// (bias 127), 23 significand bits; binary64 = 1 sign, 11 exponent (bias
// 1023), 52 significand bits.  A normal binary32 exponent field e32 in
// 1..254 maps to e64 = e32 + 896.
//
// The file is also compiled by a host C++ compiler (no CUDA), which checks it
// against the host's own conversions.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define CRN_FPB_FN __host__ __device__ __forceinline__
#else
#define CRN_FPB_FN inline
#endif

namespace crn {

CRN_FPB_FN uint32_t fpb_bits32(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}

CRN_FPB_FN float fpb_float(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}

CRN_FPB_FN uint64_t fpb_bits64(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}

CRN_FPB_FN double fpb_double(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

CRN_FPB_FN int fpb_clz32(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

// binary32 -> binary64, exact.  NaNs keep their payload and come out quiet.
CRN_FPB_FN double widen_f32(float x) {
  const uint32_t b = fpb_bits32(x);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t m = b & 0x7fffffu;
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  if (e - 1u < 254u)  // normal
    return fpb_double(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29));
  if (e == 0xffu)     // infinity, NaN
    return fpb_double(sign | (0x7ffull << 52) | ((uint64_t)m << 29) | (m ? (1ull << 51) : 0ull));
  if (m == 0u) return fpb_double(sign);  // +-0
  // subnormal m * 2^-149 with its leading one at bit p: normal in binary64
  const int p = 31 - fpb_clz32(m);
  return fpb_double(sign | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & 0xfffffffffffffull));
}

// binary64 -> binary32, rounded to nearest, ties to even.  NaNs come out
// quiet with the leading 22 bits of their payload.
CRN_FPB_FN float narrow_f64(double x) {
  const uint64_t b = fpb_bits64(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  const uint64_t f = b & 0xfffffffffffffull;
  if (e - 897u < 254u) {  // binary32 normal range before rounding
    const uint32_t m = (uint32_t)(f >> 29);                 // leading 23 significand bits
    const uint32_t rest = (uint32_t)f & 0x1fffffffu;        // the 29 bits dropped
    // round up above the halfway point, and at it when the kept part is odd;
    // a carry out of the significand raises the exponent (to infinity from
    // the largest binade), as rounding to nearest requires
    const uint32_t r = sign | ((e - 896u) << 23) | m;
    return fpb_float(r + (uint32_t)((rest > 0x10000000u) || (rest == 0x10000000u && (m & 1u))));
  }
  if (e == 0x7ffu)        // infinity, NaN
    return fpb_float(sign | 0x7f800000u | (uint32_t)(f >> 29) | (f ? 0x400000u : 0u));
  if (e > 1150u) return fpb_float(sign | 0x7f800000u);     // |x| >= 2^128: overflow
  // binary32 subnormal or zero: k = M 2^(e' - 926) units of 2^-149, with the
  // full significand M and e' = max(e, 1)
  const uint64_t M = e ? (f | (1ull << 52)) : f;
  const uint32_t s = 926u - (e ? e : 1u);                   // >= 30
  if (s >= 54u) return fpb_float(sign);                     // below half the least subnormal
  const uint64_t q = M >> s;
  const uint64_t rem = M & ((1ull << s) - 1u), half = 1ull << (s - 1u);
  // a carry into bit 23 gives the least normal number, as it should
  return fpb_float(sign | (uint32_t)(q + (uint64_t)((rem > half) || (rem == half && (q & 1u)))));
}

}  // namespace crn

#undef CRN_FPB_FN
