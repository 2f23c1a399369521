// IEEE-754 binary64 multiplication (and a faithful reciprocal) on the integer pipes.
//
// GB300 issues FP64 arithmetic at 2 lane-operations per SM per cycle, while its integer and FP32
// pipes, which the FP64-bound kernels of this library leave almost idle, issue tens of times more.
// f64_mul_int() forms the binary64 product x*y rounded to nearest, ties to even (IEEE 754-2019,
// Sec. 4.3.1 and 5.4.1) from the two 53-bit significands with 64-bit integer multiplies, so its
// result is bit-identical to the hardware DMUL instruction, and a kernel can move a share of its
// multiplications off the FP64 pipe.
//
// Method (the schoolbook significand product of software floating-point, as described for example
// in Muller et al., Handbook of Floating-Point Arithmetic): with significands Ma, Mb in [2^52, 2^53)
// shifted left by 10 bits, the exact 128-bit product lies in [2^124, 2^126); its high word holds the
// 53 result bits plus 8 or 9 lower bits, and the low word only contributes to the sticky bit. One
// normalising shift, a round-to-nearest-even increment and the biased exponent sum (whose carry
// absorbs a significand that rounds up to 2^53) give the result word.
//
// Zero operands (with a finite other operand) are handled on the fast path. The function reports
// failure (and leaves `out` unspecified) when an operand is subnormal, infinite or NaN, or when the
// product leaves the normal range; callers then recompute with the FP64 pipe. The header compiles as
// CUDA (device and host) and as plain C++ for host-side checks against the host's own multiply.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define HW_FP64_INT_FN __host__ __device__ __forceinline__
#else
#define HW_FP64_INT_FN static inline
#endif

namespace hw {

// The two 32-bit words of a double. On the device this is a register move the compiler cannot see
// through, so integer tests on the words are not turned back into FP64 comparisons.
HW_FP64_INT_FN void f64_words(double x, uint32_t& lo, uint32_t& hi) {
#if defined(__CUDA_ARCH__)
  asm("mov.b64 {%0,%1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  lo = (uint32_t)u;
  hi = (uint32_t)(u >> 32);
#endif
}

HW_FP64_INT_FN double f64_from_words(uint32_t lo, uint32_t hi) {
#if defined(__CUDA_ARCH__)
  double x;
  asm("mov.b64 %0, {%1,%2};" : "=d"(x) : "r"(lo), "r"(hi));
  return x;
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}

HW_FP64_INT_FN uint64_t u64_mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// The words of a compile-time constant, through a cast the compiler folds.
HW_FP64_INT_FN void f64_const_words(double x, uint32_t& lo, uint32_t& hi) {
#if defined(__CUDA_ARCH__)
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
#endif
  lo = (uint32_t)u;
  hi = (uint32_t)(u >> 32);
}

// x*y rounded to nearest even on the integer pipes; false when the fast path does not apply.
// YCONST: y is a compile-time constant (its significand and exponent fold into the code).
template <bool YCONST = false>
HW_FP64_INT_FN bool f64_mul_int(double x, double y, double& out) {
  uint32_t al, ah, bl, bh;
  f64_words(x, al, ah);
  if (YCONST) f64_const_words(y, bl, bh);
  else f64_words(y, bl, bh);
  const uint32_t ea = (ah >> 20) & 0x7ffu, eb = (bh >> 20) & 0x7ffu;
  // significands with the hidden bit, shifted so that they lie in [2^62, 2^63)
  const uint64_t ma = ((uint64_t)((ah & 0xfffffu) | 0x100000u) << 42) | ((uint64_t)al << 10);
  const uint64_t mb = ((uint64_t)((bh & 0xfffffu) | 0x100000u) << 42) | ((uint64_t)bl << 10);
  uint64_t hi = u64_mulhi(ma, mb);   // [2^60, 2^62)
  const uint64_t lo = ma * mb;       // below the rounding position: sticky only
  const uint32_t n = (uint32_t)(hi >> 61) ^ 1u;  // 1 when the significand product is below 2
  hi <<= n;                                      // [2^61, 2^62): result bits 61..9, guard bit 8
  hi |= (uint64_t)(lo != 0);
  const uint64_t m = (hi + 0xffu + ((hi >> 9) & 1u)) >> 9;  // round to nearest even, in [2^52, 2^53]
  const int E = (int)(ea + eb) - 1022 - (int)n;              // biased exponent of the result
  const bool zero = (((ah << 1) | al) == 0u) | (((bh << 1) | bl) == 0u);
  const bool ok = (ea != 0x7ffu) & (eb != 0x7ffu) &
                  (zero | ((ea != 0u) & (eb != 0u) & ((unsigned)(E - 1) < 2045u)));
  const uint32_t s = (ah ^ bh) & 0x80000000u;
  const uint64_t packed = ((uint64_t)(uint32_t)(E - 1) << 52) + m;  // hidden bit carries into E
  out = f64_from_words(zero ? 0u : (uint32_t)packed, zero ? s : (s | (uint32_t)(packed >> 32)));
  return ok;
}

// Seed of the reciprocal: 1/mf for mf in [1, 2) to about 22 bits (the SFU's approximation on the device).
HW_FP64_INT_FN float f32_rcp_seed(float mf) {
#if defined(__CUDA_ARCH__)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(mf));
  return r;
#else
  return 1.0f / mf;
#endif
}

HW_FP64_INT_FN uint32_t f32_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}

HW_FP64_INT_FN float f32_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}

HW_FP64_INT_FN int64_t s64_mulhi(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

// 1/x on the integer pipes, within one ulp (faithfully rounded; round to nearest of an approximation
// accurate to about 2^-60). False (out unspecified) unless x is normal with a biased exponent of at
// most 2044, i.e. the reciprocal is normal. Method (Newton-Raphson iteration with a third-order step,
// a textbook division algorithm): a seed Y0 ~ 2^83/M (22 bits) of the significand M in [2^52, 2^53)
// from the single-precision reciprocal; the residual E = 2^83 - M*Y0 (exact in 64-bit two's
// complement for a seed error below 2^-20); then 2^116/M ~ Y0 (2^33 + (E + E^2/2^83) / 2^50), rounded
// to 53 bits. SEED_ERR perturbs the seed by that many single-precision ulps (host tests only).
template <int SEED_ERR = 0>
HW_FP64_INT_FN bool f64_rcp_int(double x, double& out) {
  uint32_t al, ah;
  f64_words(x, al, ah);
  const uint32_t ex = (ah >> 20) & 0x7ffu;
  const uint32_t fh = ah & 0xfffffu;
  const bool ok = (ex - 1u) < 2044u;
  // seed from the leading 23 fraction bits: mf in [1, 2), r ~ 1/mf (about 1/2 to 1)
  const float mf = f32_from_bits(0x3f800000u | (fh << 3) | (al >> 29));
  const uint32_t rb = f32_bits(f32_rcp_seed(mf)) + (uint32_t)SEED_ERR;
  // Y0 = r 2^31 from r's significand and exponent (125..127)
  const uint32_t Y0 = ((rb & 0x7fffffu) | 0x800000u) << ((rb >> 23) - 119u);
  const uint32_t mh = fh | 0x100000u;
  // E = 2^83 - M Y0 mod 2^64, with M = mh 2^32 + al
  const uint64_t Plo = ((uint64_t)(mh * Y0) << 32) + (uint64_t)al * Y0;
  const int64_t E = -(int64_t)Plo;
  const uint64_t aE = (uint64_t)(E < 0 ? -E : E);
  const int64_t T = E + (int64_t)(u64_mulhi(aE, aE) >> 19);              // E + E^2 / 2^83
  const int64_t corr = s64_mulhi(T, (int64_t)((uint64_t)Y0 << 31)) >> 17;  // Y0 T / 2^50
  const uint64_t Y = ((uint64_t)Y0 << 33) + (uint64_t)corr;  // ~ 2^116 / M (mod 2^64), in (2^63, 2^64)
  const uint64_t Q = (Y + 0x400u) >> 11;                       // 53-bit significand of 2^53/M
  const bool pow2 = (fh | al) == 0u;
  const uint32_t s = ah & 0x80000000u;
  // result exponent: 2045 - ex (2046 - ex for a power-of-two significand, whose reciprocal is exact)
  const uint64_t packed = ((uint64_t)(2044u - ex) << 52) + Q;
  out = f64_from_words(pow2 ? 0u : (uint32_t)packed, s | (pow2 ? (2046u - ex) << 20 : (uint32_t)(packed >> 32)));
  return ok;
}

}  // namespace hw
