// Host check of the integer-pipe binary64 multiply and reciprocal (paper_2208_01260_gb300/csrc/
// hw_fp64_int.h) against the host's IEEE-754 arithmetic: every product the fast path accepts must
// equal x*y bit for bit, every reciprocal must be within one ulp of 1/x (with seeds perturbed by up to
// six single-precision ulps, beyond the device approximation's error). Usage: fp64_int_check N SEED
// [rcp]; prints "accepted mismatches rejected" and exits non-zero on a mismatch or when the fast path
// rejected an operand it must take.
#include "hw_fp64_int.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

static double as_double(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }
static uint64_t as_bits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }

template <int SE>
static void check_rcp(long n, std::mt19937_64& rng, long& accepted, long& bad, long& missed) {
  for (long i = 0; i < n; ++i) {
    uint64_t a = rng();
    if (i % 3 == 1) a = (a & 0x800fffffffffffffull) | (uint64_t)(1000 + rng() % 48) << 52;
    if (i % 3 == 2)  // significands near 1 and near 2, all exponents of the fast path
      a = (a & 0x80000000000fffffull) | (uint64_t)(1 + rng() % 2044) << 52 |
          ((rng() & 1) ? 0 : 0x000ffffffff00000ull);
    const double x = as_double(a);
    double r = 0.0;
    const unsigned ex = (unsigned)(a >> 52) & 0x7ffu;
    if (!hw::f64_rcp_int<SE>(x, r)) {
      if (ex >= 1 && ex <= 2044) ++missed;
      continue;
    }
    ++accepted;
    const double t = 1.0 / x;
    if (r != t && r != std::nextafter(t, INFINITY) && r != std::nextafter(t, -INFINITY)) {
      if (bad < 5) printf("reciprocal of %a: %a vs %a\n", x, r, t);
      ++bad;
    }
  }
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  std::mt19937_64 rng(argc > 2 ? strtoull(argv[2], nullptr, 10) : 1);
  if (argc > 3 && strcmp(argv[3], "rcp") == 0) {
    long accepted = 0, bad = 0, missed = 0;
    check_rcp<0>(n, rng, accepted, bad, missed);
    check_rcp<3>(n / 4, rng, accepted, bad, missed);
    check_rcp<-3>(n / 4, rng, accepted, bad, missed);
    check_rcp<6>(n / 4, rng, accepted, bad, missed);
    check_rcp<-6>(n / 4, rng, accepted, bad, missed);
    printf("%ld %ld %ld\n", accepted, bad, missed);
    return (bad || missed) ? 1 : 0;
  }
  const uint64_t SGN_FRAC = 0x800fffffffffffffull;
  long accepted = 0, bad = 0, missed = 0;
  for (long i = 0; i < n; ++i) {
    uint64_t a = rng(), b = rng();
    switch (i % 7) {
      case 1:  // exponents near 1 (the scheme's data)
        a = (a & SGN_FRAC) | (uint64_t)(1000 + rng() % 48) << 52;
        b = (b & SGN_FRAC) | (uint64_t)(1000 + rng() % 48) << 52;
        break;
      case 2:  // short significands: exact products and rounding ties
        a = (a & 0x800fff0000000000ull) | (uint64_t)1023 << 52;
        b = (b & 0x800ffffff0000000ull) | (uint64_t)1023 << 52;
        break;
      case 3:  // nearly equal operands (squares)
        b = a ^ (rng() & 0xfff);
        break;
      case 4:  // signed zeros against anything
        if (rng() & 1) a &= 0x8000000000000000ull; else b &= 0x8000000000000000ull;
        break;
      case 5:  // products at the edges of the normal range
        a = (a & SGN_FRAC) | (uint64_t)(1 + rng() % 40) << 52;
        b = (b & SGN_FRAC) | (uint64_t)(1000 + rng() % 40) << 52;
        if (rng() & 1) { a ^= (uint64_t)0x7fe0000000000000ull & a; a |= (uint64_t)(2000 + rng() % 46) << 52; }
        break;
      case 6:  // subnormal, infinite and NaN operands
        a = (a & SGN_FRAC) | (uint64_t)((rng() % 3 == 0) ? 2047 : 0) << 52;
        break;
      default:
        break;
    }
    const double x = as_double(a), y = as_double(b);
    double r = 0.0;
    const double t = x * y;
    if (hw::f64_mul_int(x, y, r)) {
      ++accepted;
      if (as_bits(r) != as_bits(t)) {
        if (bad < 5) printf("mismatch %a * %a: %a vs %a\n", x, y, r, t);
        ++bad;
      }
    } else if (std::fpclassify(x) == FP_NORMAL && std::fpclassify(y) == FP_NORMAL &&
               std::fabs(t) >= 0x1p-1021 && std::fabs(t) < 0x1p1022) {
      if (missed < 5) printf("rejected %a * %a = %a\n", x, y, t);
      ++missed;
    }
  }
  printf("%ld %ld %ld\n", accepted, bad, missed);
  return (bad || missed) ? 1 : 0;
}
