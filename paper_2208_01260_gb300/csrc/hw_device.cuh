// Device-side building blocks of the well-balanced fifth-order FD HWENO scheme (Zhao & Zhang,
// arXiv:2208.01260) for sm_103a, written for an FP64-pipe-bound kernel: every FP64 add, mul and
// fma counts, memory traffic is cheap.
//
// Conventions shared by all kernels (each one mathematically identical to the paper's formulas):
//   * Derivative planes are stored multiplied by the grid spacing of their direction: the state holds
//     V' = dx V and Q' = dy Q, and the static planes hold b, dx b_x, dy b_y. Every Hermite formula of
//     Sec. 2.1-2.2 uses the derivative only as dx*phi, so the scaling removes those multiplications.
//   * The Lax-Friedrichs split F^+- = (F +- alpha U)/2 (Sec. 2.1 Step 1) is used without the 1/2, and
//     the characteristic projection uses the rows of L = R^{-1} without their 1/(2c) factor. Both are
//     per-interface scalings s_k of a characteristic field (s = (4c, 2, 4c) in a sweep, (2c, 1, 2c) in the
//     limiter). The smoothness indicators are quadratic in the data, so the nonlinear weights of
//     eq. (GHYZZ) are unchanged when epsilon is replaced by s_k^2 epsilon; the scaling is undone at the
//     back-projection.
//   * The weights are normalised with one reciprocal: omega_l = gamma_l p_l / sum(gamma_m p_m) with
//     p_1 = s_2 s_3, p_2 = s_1 s_3, p_3 = s_1 s_2, s_l = (beta_l + eps)^2, equal to eq. (GHYZZ).
//   * Reciprocals and square roots use the hardware approximation plus one cubically convergent
//     Newton step (Householder order 3 for 1/x and for 1/sqrt(x)), accurate to a few ulp.
//   * The functions are templates on the working precision R: double for the scheme, float for the
//     single-precision variant, which uses the hardware approximations alone and normalises the
//     weights by the smallest beta_l + eps (products of four of them overflow float on large jumps).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include "hw_fp64_int.h"

namespace hw {

enum { BC_PERIODIC = 0, BC_REFLECTIVE = 1, BC_OUTFLOW = 2 };

// State planes: 0 eta, 1 m, 2 w, 3 H1', 4 M1', 5 W1', 6 H2', 7 M2', 8 W2' (2D);
//               0 eta, 1 m, 2 H', 3 M' (1D).
// Static planes: 0 b, 1 dx b_x, 2 dy b_y (2D); 0 b, 1 dx b_x (1D).
// Reflective parity of the 12 planes (state then static) across an x-wall and a y-wall
// (mirror image of the SWE: u odd across x-walls, v odd across y-walls).
__host__ __device__ constexpr double par_x2d(int q) {
  return (q == 1 || q == 3 || q == 5 || q == 7 || q == 10) ? -1.0 : 1.0;
}
__host__ __device__ constexpr double par_y2d(int q) {
  return (q == 2 || q == 5 || q == 6 || q == 7 || q == 11) ? -1.0 : 1.0;
}
// 1D: eta +, m -, H' -, M' +, b +, dx b_x -.
__host__ __device__ constexpr double par_1d(int q) { return (q == 1 || q == 2 || q == 5) ? -1.0 : 1.0; }

// Map a node index that may lie up to n outside [0, n) onto the grid. flip = reflected (the caller
// applies the parity table); a transmissive boundary copies the boundary node.
__device__ __forceinline__ int map_index(int i, int n, int bc, bool& flip) {
  flip = false;
  if (i < 0) {
    if (bc == BC_PERIODIC) return i + n;
    if (bc == BC_OUTFLOW) return 0;
    flip = true;
    return -1 - i;
  }
  if (i >= n) {
    if (bc == BC_PERIODIC) return i - n;
    if (bc == BC_OUTFLOW) return n - 1;
    flip = true;
    return 2 * n - 1 - i;
  }
  return i;
}

// ---------------------------------------------------------------------------------------------
// Reciprocal and reciprocal square root: hardware seed (about 20 bits) refined by one cubically
// convergent step, so the relative error is below 2^-52 plus rounding.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double rcp_seed(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_seed(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
// 1/x: e = 1 - x r, r' = r (1 + e + e^2) (Householder iteration of order 3 for f(r) = 1/r - x).
__device__ __forceinline__ double fast_rcp(double x) {
  double r = rcp_seed(x);
  double e = fma(-x, r, 1.0);
  double t = fma(e, e, e);
  return fma(r, t, r);
}
// 1/sqrt(x): e = 1 - x r^2, r' = r (1 + e/2 + 3 e^2 / 8) (third-order Householder step).
__device__ __forceinline__ double fast_rsqrt(double x) {
  double r = rsqrt_seed(x);
  double r2 = r * r;
  double e = fma(-x, r2, 1.0);
  double t = fma(0.375, e, 0.5);
  double u = e * t;
  return fma(r, u, r);
}

// Single precision (the FP32 variant): the hardware approximations alone, within about one float ulp,
// one instruction each (the correctly rounded forms cost several, and the float kernels are bound by
// instruction issue and memory, not by the FP32 pipe).
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fast_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Non-negative double -> ordered 64-bit key (for an exact, order-independent atomicMax).
__device__ __forceinline__ unsigned long long dkey(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double dabs(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }

// ---------------------------------------------------------------------------------------------
// One characteristic field, one upwind side, scaled data (Sec. 2.1 Step 1).
//   f0, f1, f2 = scaled f_{i-1}, f_i, f_{i+1};  p0, p1, p2 = scaled dx*phi (mirrored for the '-' side).
// Returns the weighted value sum(w_l q_l) and the unnormalised weight numerators p (times 1/den)
// for the source reconstruction with the same weights (Step 2).
//
// Algebra (exact rearrangement of the printed q_l and beta_l):
//   d1 = f0 - f1, d2 = f1 - f2, B1 = 2 d1 + p0 + p1, A1 = B1 + d1 + p1, B2 = 2 d2 + p1 + p2,
//   A2 = B2 + d2 + p1, e = d1 - d2 = f0 - 2 f1 + f2, g3 = f0 - f2 + 2 p1, P = f1 + p1/2;
//   q1 = P + A1/6, q2 = P - A2/6, q3 = P + e/12 (weights summing to 1 leave P outside the weighted sum);
//   beta1 = p1^2 + 13/3 A1^2 + 781/20 B1^2, beta2 = p1^2 + 13/3 A2^2 + 781/20 B2^2,
//   beta3 = p1^2 + 13/12 e^2 + 781/80 g3^2.
// ---------------------------------------------------------------------------------------------
// R is the working precision: double for the scheme, float for the single-precision variant. Constants
// are written as R(...) so that a float instantiation does no double arithmetic.
template <class R>
struct WeightsT {
  // omega_l = n_l * r (n_3 already carries gamma_3 / gamma_1 = 4/3)
  R n1, n2, n3, r;
};
using Weights = WeightsT<double>;

// Arithmetic policies for products and reciprocals. MulFP64: the plain product on the FP64 pipe (the
// compiler may fuse it with a following add into an fma) and fast_rcp. MulIntT: the correctly rounded
// product on the integer pipes (hw_fp64_int.h, bit-identical to DMUL) and, with IRCP, the integer-pipe
// reciprocal (within one ulp; else fast_rcp); it records whether any operation left its fast path, in
// which case the caller recomputes the block with MulFP64. k(c, x) multiplies by a literal constant c.
// Float data is handled natively by both.
struct MulFP64 {
  static constexpr bool bad = false;
  template <class R>
  __device__ __forceinline__ R operator()(R x, R y) { return x * y; }
  template <class R>
  __device__ __forceinline__ R k(R c, R x) { return c * x; }
  template <class R>
  __device__ __forceinline__ R rcp(R x) { return fast_rcp(x); }
};
template <bool IRCP>
struct MulIntT {
  bool bad = false;
  __device__ __forceinline__ double operator()(double x, double y) {
    double r;
    bad |= !f64_mul_int(x, y, r);
    return r;
  }
  __device__ __forceinline__ float operator()(float x, float y) { return x * y; }
  __device__ __forceinline__ double k(double c, double x) {
    double r;
    bad |= !f64_mul_int<true>(x, c, r);
    return r;
  }
  __device__ __forceinline__ float k(float c, float x) { return c * x; }
  __device__ __forceinline__ double rcp(double x) {
    if constexpr (!IRCP) return fast_rcp(x);
    double r;
    bad |= !f64_rcp_int(x, r);
    return r;
  }
  __device__ __forceinline__ float rcp(float x) { return fast_rcp(x); }
};
using MulInt = MulIntT<true>;

// Unnormalised weights proportional to w_1/t_1^2, w_2/t_2^2, w_3/t_3^2 (t_l = beta_l + eps). In double the
// products of the other two squares (one reciprocal); in float, where t^4 can overflow on large jumps,
// (t_min/t_l)^2, each at most 1.
template <class R, class M>
__device__ __forceinline__ void inverse_square_weights(R t1, R t2, R t3, R& n1, R& n2, R& n3, M& mul) {
  if constexpr (std::is_same<R, double>::value) {
    const R s1 = mul(t1, t1), s2 = mul(t2, t2), s3 = mul(t3, t3);
    n1 = mul(s2, s3);
    n2 = mul(s1, s3);
    n3 = mul(s1, s2);
  } else {
    const R m = fminf(fminf(t1, t2), t3);
    const R a1 = m * fast_rcp(t1), a2 = m * fast_rcp(t2), a3 = m * fast_rcp(t3);
    n1 = a1 * a1;
    n2 = a2 * a2;
    n3 = a3 * a3;
  }
}

template <bool LINEAR, class R, class M>
__device__ __forceinline__ R hweno_side_m(R f0, R f1, R f2, R p0, R p1, R p2, R eps, WeightsT<R>& W, M& mul) {
  const R d1 = f0 - f1, d2 = f1 - f2;
  const R B1 = fma(R(2.0), d1, p0 + p1);
  const R A1 = B1 + (d1 + p1);
  const R B2 = fma(R(2.0), d2, p1 + p2);
  const R A2 = B2 + (d2 + p1);
  const R P = fma(R(0.5), p1, f1);
  const R e = d1 - d2;  // f0 - 2 f1 + f2
  if (LINEAR) {
    const R q1 = fma(R(1.0 / 6.0), A1, P);
    const R q2 = fma(R(-1.0 / 6.0), A2, P);
    const R q3 = fma(R(1.0 / 12.0), e, P);
    W.n1 = R(0.3); W.n2 = R(0.3); W.n3 = R(0.4); W.r = R(1.0);
    return fma(R(0.3), q1, fma(R(0.3), q2, mul.k(R(0.4), q3)));
  }
  const R g3 = fma(R(2.0), p1, f0 - f2);
  // t_l = beta_l + eps, with eps added once to the common term p1^2
  const R ppe = fma(p1, p1, eps);  // an fma either way: no product to move off the FP64 pipe
  const R t1 = fma(mul.k(R(781.0 / 20.0), B1), B1, fma(mul.k(R(13.0 / 3.0), A1), A1, ppe));
  const R t2 = fma(mul.k(R(781.0 / 20.0), B2), B2, fma(mul.k(R(13.0 / 3.0), A2), A2, ppe));
  const R t3 = fma(mul.k(R(781.0 / 80.0), g3), g3, fma(mul.k(R(13.0 / 12.0), e), e, ppe));
  R n3;
  inverse_square_weights(t1, t2, t3, W.n1, W.n2, n3, mul);
  // gamma = (3, 3, 4)/10 -> proportional to (1, 1, 4/3)
  W.n3 = mul.k(R(4.0 / 3.0), n3);
  W.r = mul.rcp(W.n1 + W.n2 + W.n3);
  // sum(omega_l q_l) = P + (n1 A1 - n2 A2 + (n3'/2) e) / (6 (n1 + n2 + n3')), n3' = W.n3
  const R z = fma(mul.k(R(0.5), W.n3), e, fma(-W.n2, A2, mul(W.n1, A1)));
  return fma(mul.k(R(1.0 / 6.0), W.r), z, P);
}

// One side on the FP64 pipe (the 1D kernels, the batched form and the adjoint's recomputation).
template <bool LINEAR, class R>
__device__ __forceinline__ R hweno_side(R f0, R f1, R f2, R p0, R p1, R p2, R eps, WeightsT<R>& W) {
  MulFP64 mf;
  return hweno_side_m<LINEAR>(f0, f1, f2, p0, p1, p2, eps, W, mf);
}

// The source reconstructed with the same weights (Sec. 2.1 Step 2) from precomputed candidates.
template <class R, class M>
__device__ __forceinline__ R weighted_m(const WeightsT<R>& W, R c1, R c2, R c3, M& mul) {
  return mul(fma(W.n1, c1, fma(W.n2, c2, mul(W.n3, c3))), W.r);
}
template <class R>
__device__ __forceinline__ R weighted(const WeightsT<R>& W, R c1, R c2, R c3) {
  MulFP64 mf;
  return weighted_m(W, c1, c2, c3, mf);
}

// Limiter for one characteristic field (eqs. step1-dxi, limiter-1d), scaled data:
//   m0, m1, m2 = scaled mu_{i-1}, mu_i, mu_{i+1};  nl, nr = scaled dx*nu_{i-1}, dx*nu_{i+1}.
// Returns the scaled dx*nu^mod. p'_1 = 2(m1-m0) - nl, p'_2 = 2(m2-m1) - nr, p'_3 = (m2-m0)/2,
// beta^L_1 = p'_1^2 + 13/3 (m1-m0-nl)^2, beta^L_2 = p'_2^2 + 13/3 (m2-m1-nr)^2,
// beta^L_3 = p'_3^2 + 13/12 (m2 - 2 m1 + m0)^2, d = (1,1,2)/4.
template <bool LINEAR, class R, class M>
__device__ __forceinline__ R limiter_field_m(R m0, R m1, R m2, R nl, R nr, R eps, M& mul) {
  const R dl = m1 - m0, dr = m2 - m1;
  const R pl = fma(R(2.0), dl, -nl);
  const R pr = fma(R(2.0), dr, -nr);
  const R pc2 = dl + dr;  // 2 p'_3
  if (LINEAR) return fma(R(0.25), pl + pr, mul.k(R(0.25), pc2));
  const R al = dl - nl, ar = dr - nr, ac = dr - dl;
  const R b1 = fma(mul.k(R(13.0 / 3.0), al), al, mul(pl, pl));
  const R b2 = fma(mul.k(R(13.0 / 3.0), ar), ar, mul(pr, pr));
  const R b3 = fma(mul.k(R(13.0 / 12.0), ac), ac, mul(mul.k(R(0.25), pc2), pc2));
  // d = (1, 1, 2)/4 -> proportional to (1, 1, 2); p'_3 = pc2 / 2 so its term is n3 pc2
  R n1, n2, n3;
  inverse_square_weights(b1 + eps, b2 + eps, b3 + eps, n1, n2, n3, mul);
  const R den = fma(R(2.0), n3, n1 + n2);
  const R num = fma(n1, pl, fma(n2, pr, mul(n3, pc2)));
  return mul(num, mul.rcp(den));
}
template <bool LINEAR, class R>
__device__ __forceinline__ R limiter_field(R m0, R m1, R m2, R nl, R nr, R eps) {
  MulFP64 mf;
  return limiter_field_m<LINEAR>(m0, m1, m2, nl, nr, eps, mf);
}

}  // namespace hw
