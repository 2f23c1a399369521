// IEEE-754 binary64 multiplication on the integer pipes.
//
// GB300 issues FP64 arithmetic at 2 lane-operations per SM per cycle, while its integer and FP32
// pipes, which the FP64-bound kernels of this library leave almost idle, issue tens of times more.
// f64_mul_int() forms the binary64 product x*y rounded to nearest, ties to even (IEEE 754-2019,
// Sec. 4.3.1 and 5.4.1) from the two 53-bit significands with 64-bit integer multiplies, so its
// result is bit-identical to the hardware DMUL instruction, and a kernel can move a share of its
// multiplications off the FP64 pipe.
//
// Method (the schoolbook significand product, e.g. Muller et al., Handbook of Floating-Point
// Arithmetic, Sec. 8.4): with significands Ma, Mb in [2^52, 2^53) shifted left by 10 bits, the exact
// 128-bit product lies in [2^124, 2^126); its high word holds the 53 result bits plus 8 or 9 lower
// bits, and the low word only contributes to the sticky bit. One normalising shift, a round-to-
// nearest-even increment and the biased exponent sum (whose carry absorbs a significand that rounds
// up to 2^53) give the result word.
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

}  // namespace hw
