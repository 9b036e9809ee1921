// Rounding an FP64 value to FP32, and its hi/lo split (hi = RN(v),
// lo = RN(v - hi)), in integer arithmetic on the bit patterns. The split
// feeds the force kernel's group-relative coordinates: (x_hi - c_hi) +
// (x_lo - c_lo) stands for the FP64 subtraction x - c run on FP32 units.
// GB300's FP64 unit is narrow; the integer form gives the same values from
// the integer pipe for every |v| in [2^-74, 2^100) (the moments' final pass,
// 251k cells at 2^20 particles: 25 -> 20 us), and falls back to the FP64
// conversions outside that range (zeros, tiny or huge values, non-finite
// values).
//
// This header compiles as CUDA (host and device) and as plain C, so that
// the host tests run the same code against the FP64 conversions.
#ifndef AFD_SPLIT_CUH
#define AFD_SPLIT_CUH

#include <stdint.h>

#if defined(__CUDACC__)
#define AFD_SPLIT_FN __host__ __device__ __forceinline__
#else
#include <string.h>
#define AFD_SPLIT_FN static inline
#endif

AFD_SPLIT_FN uint64_t afd_split_dbits(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  memcpy(&u, &v, sizeof u);
  return u;
#endif
}

AFD_SPLIT_FN float afd_split_fval(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}

AFD_SPLIT_FN float afd_split_i2f(int32_t r) {
#if defined(__CUDA_ARCH__)
  return __int2float_rn(r);
#else
  return (float)r;  // round to nearest even, the default mode
#endif
}

AFD_SPLIT_FN float afd_split_d2f(double v) {
#if defined(__CUDA_ARCH__)
  return __double2float_rn(v);
#else
  return (float)v;
#endif
}

// Biased FP64 exponents of the range the integer form covers: [2^-74, 2^100).
#define AFD_SPLIT_EMIN 949u
#define AFD_SPLIT_EMAX 1123u

// hi = RN(v) in FP32 and lo = RN(v - hi) in FP32. With the 53-bit
// significand F of v (implicit bit included) and its exponent e: the top 24
// bits q = F >> 29 round to nearest, ties to even, on the 29 bits below
// (a carry to 2^24 moves hi to the next binade); the residual r = F - q 2^29
// is exact, |r| <= 2^28, and lo = RN(r) 2^(e - 1075), the power-of-two scale
// exact because lo stays a normal FP32 number in this range. A zero residual
// gives lo = +0, as the FP64 subtraction v - hi does.
AFD_SPLIT_FN void afd_split2(double v, float *hi, float *lo) {
  const uint64_t u = afd_split_dbits(v);
  const uint32_t e = (uint32_t)(u >> 52) & 0x7ffu;
  if (e < AFD_SPLIT_EMIN || e >= AFD_SPLIT_EMAX) {
    const float h = afd_split_d2f(v);
    *hi = h;
    *lo = afd_split_d2f(v - (double)h);
    return;
  }
  const uint32_t sgn = (uint32_t)(u >> 63);
  const uint64_t F = (u & ((1ull << 52) - 1ull)) | (1ull << 52);
  uint64_t q = F >> 29;
  const uint64_t rem = F & ((1ull << 29) - 1ull);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (q & 1ull))) q += 1ull;
  const int32_t r = (int32_t)((int64_t)F - (int64_t)(q << 29));
  uint32_t eh = e - 896u;  // e - 1023 + 127
  if (q == (1ull << 24)) {
    q >>= 1;
    eh += 1u;
  }
  *hi = afd_split_fval((sgn << 31) | (eh << 23) | ((uint32_t)q & 0x7fffffu));
  const float scale = afd_split_fval((e - 948u) << 23);  // 2^(e - 1075)
  *lo = afd_split_i2f(sgn ? -r : r) * scale;
}

// RN(v) in FP32 (the hi part of the split alone).
AFD_SPLIT_FN float afd_round_f32(double v) {
  const uint64_t u = afd_split_dbits(v);
  const uint32_t e = (uint32_t)(u >> 52) & 0x7ffu;
  if (e < AFD_SPLIT_EMIN || e >= AFD_SPLIT_EMAX) return afd_split_d2f(v);
  const uint32_t sgn = (uint32_t)(u >> 63);
  const uint64_t F = (u & ((1ull << 52) - 1ull)) | (1ull << 52);
  uint64_t q = F >> 29;
  const uint64_t rem = F & ((1ull << 29) - 1ull);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (q & 1ull))) q += 1ull;
  uint32_t eh = e - 896u;
  if (q == (1ull << 24)) {
    q >>= 1;
    eh += 1u;
  }
  return afd_split_fval((sgn << 31) | (eh << 23) | ((uint32_t)q & 0x7fffffu));
}

// Finite test on the exponent bits (no FP64 instruction).
AFD_SPLIT_FN int afd_finite_bits(double v) {
  return ((uint32_t)(afd_split_dbits(v) >> 52) & 0x7ffu) != 0x7ffu;
}

#endif  // AFD_SPLIT_CUH
