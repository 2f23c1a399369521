// IEEE-754 binary64 multiplication and addition on the integer pipes.
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

HW_FP64_INT_FN int u64_clz(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// x+y rounded to nearest even on the integer pipes; false (out unspecified) when an operand is
// infinite or NaN or the sum is subnormal or overflows. Zero and subnormal operands are exact on the
// fast path. Method: order the operands by magnitude, align the smaller significand (10 guard bits,
// the bits shifted out folded into a sticky bit), add or subtract, normalise with a leading-zero
// count and round to nearest even at the 53rd bit (Muller et al., Sec. 8.3).
HW_FP64_INT_FN bool f64_add_int(double x, double y, double& out) {
  uint32_t al, ah, bl, bh;
  f64_words(x, al, ah);
  f64_words(y, bl, bh);
  const uint64_t A = ((uint64_t)(ah & 0x7fffffffu) << 32) | al, B = ((uint64_t)(bh & 0x7fffffffu) << 32) | bl;
  const bool sw = B > A;
  const uint64_t P = sw ? B : A, Q = sw ? A : B;  // |P| >= |Q|
  const uint32_t sp = (sw ? bh : ah) & 0x80000000u;
  const bool sub = ((ah ^ bh) & 0x80000000u) != 0;
  const uint32_t ph = (uint32_t)(P >> 32), qh = (uint32_t)(Q >> 32);
  const int ep = (int)(ph >> 20), eq = (int)(qh >> 20);
  // significands (hidden bit only for normal numbers) in [2^62, 2^63) for normal operands
  const uint64_t mp = ((uint64_t)((ph & 0xfffffu) | ((uint32_t)(ep != 0) << 20)) << 42) | ((uint64_t)(uint32_t)P << 10);
  const uint64_t mq = ((uint64_t)((qh & 0xfffffu) | ((uint32_t)(eq != 0) << 20)) << 42) | ((uint64_t)(uint32_t)Q << 10);
  const int epp = ep + (ep == 0), eqq = eq + (eq == 0);  // subnormals scale like exponent 1
  int d = epp - eqq;
  d = d < 63 ? d : 63;
  const uint64_t kept = mq >> d;
  const uint64_t mqs = kept | (uint64_t)((kept << d) != mq);  // sticky
  const uint64_t S0 = sub ? mp - mqs : mp + mqs;
  const int lz = u64_clz(S0);
  const uint64_t S = S0 << (lz & 63);                        // leading one at bit 63
  const int E = epp + 1 - lz;                                 // biased exponent of the result
  const uint32_t low = (uint32_t)S;
  const uint64_t up = ((low >> 10) & 1u) & (((low & 0x3ffu) != 0u) | ((low >> 11) & 1u));
  const uint64_t m = (S >> 11) + up;                          // [2^52, 2^53]
  const bool zero = S0 == 0;                                  // exact cancellation or two zeros
  const bool ok = (ep != 0x7ff) & (eq != 0x7ff) & (zero | ((unsigned)(E - 1) < 2045u));
  const uint64_t packed = ((uint64_t)(uint32_t)(E - 1) << 52) + m;
  out = f64_from_words(zero ? 0u : (uint32_t)packed, zero ? (ah & bh & 0x80000000u) : (sp | (uint32_t)(packed >> 32)));
  return ok;
}

}  // namespace hw
