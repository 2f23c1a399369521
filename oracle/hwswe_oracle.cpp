// CPU ORACLE — TEST INFRASTRUCTURE ONLY.
//
// Plain, slow FP64 restatement of the well-balanced fifth-order finite-difference Hermite WENO
// (HWENO) scheme for the shallow water equations in pre-balanced form (Zhao & Zhang,
// arXiv:2208.01260). Only the test suite, the smoke check and the benchmark's CPU-baseline leg load
// this library. The CUDA library never calls it, shares no code with it, and this file includes
// nothing from the CUDA side.
//
// Everything is written in the paper's order and notation with ghost-padded arrays and plain loops:
//   Sec. 2, eq. (swe-form-1d-e)/(swe-form-1d-h)  1D pre-balanced system and its derivative system
//   Sec. 2.1 Step 1                              LF splitting, Hermite candidates, weights (eq. GHYZZ),
//                                                derivative flux Q' (eq. Rec-phi)
//   Sec. 2.1 Step 2, eq. (swe-form-1d-semi)      source balance with the same weights
//   Sec. 2.2, eq. (RK), eqs. (step1-dxi), (limiter-1d)  SSP-RK3 and the HWENO limiter
//   Sec. 3, eqs. (swe-form-2d-e), (swe-form-2d-h), (mixed), (swe-form-2d-dis)  2D extension
//
// Readings where the paper is silent or garbled (each also listed in the design notes):
//   * alpha: global per direction and per RK stage, max(|u|+c) over the stage's input state.
//   * eigenvectors: R = [[1,0,1],[u-c,0,u+c],[v,1,v]] (x), L = R^{-1}; y likewise; evaluated at the
//     interface from h = (h_i+h_{i+1})/2, u = (m_i+m_{i+1})/(h_i+h_{i+1}), v likewise.
//   * weight sum index printed as 0..2 in eq. (GHYZZ) read as 1..3.
//   * source split printed with a bold b read as the tilde-b of the sweep.
//   * 2D semi-discrete source terms printed with '+' read with '-' (Sec. 3 continuous form and the
//     1D scheme fix the sign).
//   * limiter: V along x with x-eigenvectors at the node, Q along y with y-eigenvectors at the node.
//   * boundary conditions: periodic, or reflective walls at the cell faces with the parity table.
//
// The scalar type is a template parameter: double for the reference values, a counting type for
// the operation tally, a forward-mode dual number for directional derivatives, and single and
// double-double precision for the lake-at-rest rows of Tables 1-3.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <limits>

namespace orc {

// ---------------------------------------------------------------------------------------------
// Scalar types
// ---------------------------------------------------------------------------------------------

// Operation counter: carries the double value so that comparisons branch exactly as in double.
struct OpCount { double add, mul, div, sqrt, cmp; };
static OpCount g_ops = {0, 0, 0, 0, 0};

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline bool operator<(Cnt a, Cnt b) { g_ops.cmp++; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { g_ops.cmp++; return a.v > b.v; }
inline Cnt sqrt(Cnt a) { g_ops.sqrt++; return Cnt(std::sqrt(a.v)); }
inline double val(Cnt a) { return a.v; }

// Forward-mode dual number: value and one directional derivative.
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline double val(Dual a) { return a.v; }

// Double-double number hi + lo (|lo| <= ulp(hi)/2), about 106 significant bits, for the well-balance
// pin against the quadruple-precision rows of Tables 1-3. Error-free transformations: Knuth's TwoSum,
// the FMA form of Dekker's TwoProduct; division and square root take one correction step each.
// The file is compiled with -ffp-contract=off, which TwoSum needs.
struct DD {
  double hi, lo;
  DD() : hi(0), lo(0) {}
  DD(double x) : hi(x), lo(0) {}
  DD(double h, double l) : hi(h), lo(l) {}
};
inline DD dd_two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return DD(s, (a - (s - bb)) + (b - bb));
}
inline DD dd_fast_two_sum(double a, double b) {  // needs |a| >= |b| (or a == 0)
  const double s = a + b;
  return DD(s, b - (s - a));
}
inline DD dd_two_prod(double a, double b) {
  const double p = a * b;
  return DD(p, std::fma(a, b, -p));
}
inline DD operator+(DD a, DD b) {
  DD s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = dd_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return dd_fast_two_sum(s.hi, s.lo);
}
inline DD operator-(DD a) { return DD(-a.hi, -a.lo); }
inline DD operator-(DD a, DD b) { return a + (-b); }
inline DD operator*(DD a, DD b) {
  DD p = dd_two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return dd_fast_two_sum(p.hi, p.lo);
}
inline DD operator/(DD a, DD b) {
  const double q1 = a.hi / b.hi;
  const DD r1 = a - b * DD(q1);
  const double q2 = r1.hi / b.hi;
  const DD r2 = r1 - b * DD(q2);
  const double q3 = r2.hi / b.hi;
  return dd_fast_two_sum(q1, q2) + DD(q3);
}
inline DD& operator+=(DD& a, DD b) { a = a + b; return a; }
inline bool operator<(DD a, DD b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline bool operator>(DD a, DD b) { return b < a; }
inline DD sqrt(DD a) {
  if (!(a.hi > 0.0)) return DD(std::sqrt(a.hi));
  const double x = std::sqrt(a.hi);
  const DD r = a - dd_two_prod(x, x);  // Newton: sqrt(a) ~ x + (a - x^2) / (2x)
  return dd_fast_two_sum(x, r.hi / (2.0 * x));
}
inline double val(DD a) { return a.hi + a.lo; }

// Single precision with every operation and constant in float (a plain float would let double
// literals promote whole expressions to double).
struct F32 {
  float v;
  F32() : v(0) {}
  F32(double x) : v((float)x) {}
};
inline F32 f32(float x) { F32 r; r.v = x; return r; }
inline F32 operator+(F32 a, F32 b) { return f32(a.v + b.v); }
inline F32 operator-(F32 a, F32 b) { return f32(a.v - b.v); }
inline F32 operator*(F32 a, F32 b) { return f32(a.v * b.v); }
inline F32 operator/(F32 a, F32 b) { return f32(a.v / b.v); }
inline F32 operator-(F32 a) { return f32(-a.v); }
inline F32& operator+=(F32& a, F32 b) { a = a + b; return a; }
inline bool operator<(F32 a, F32 b) { return a.v < b.v; }
inline bool operator>(F32 a, F32 b) { return a.v > b.v; }
inline F32 sqrt(F32 a) { return f32(std::sqrt(a.v)); }
inline double val(F32 a) { return a.v; }

inline double val(double a) { return a; }
using std::sqrt;

// Build a scalar from a value and (for the dual type) a seed direction.
template <class T> inline T make_scalar(double x, double dx);
template <> inline double make_scalar<double>(double x, double) { return x; }
template <> inline Cnt make_scalar<Cnt>(double x, double) { return Cnt(x); }
template <> inline Dual make_scalar<Dual>(double x, double dx) { return Dual(x, dx); }
template <> inline DD make_scalar<DD>(double x, double) { return DD(x); }
template <> inline F32 make_scalar<F32>(double x, double) { return F32(x); }
inline double dpart(double) { return 0.0; }
inline double dpart(Cnt) { return 0.0; }
inline double dpart(Dual a) { return a.d; }

template <class T> inline T sq(T a) { return a * a; }
// SSP-RK3 coefficient p/q in the working precision, so that a_k + b_k = 1 holds to that precision
// (in double-double, 1/3 and 2/3 rounded to double would add a drift of 5.6e-17 per step); the
// operation counter does not count it (it is a per-stage constant).
template <class T> inline T rk_ratio(double p, double q) { return T(p) / T(q); }
template <> inline double rk_ratio<double>(double p, double q) { return p / q; }
template <> inline Cnt rk_ratio<Cnt>(double p, double q) { return Cnt(p / q); }
// |x| with the derivative convention d|x| = dx for x >= 0.
template <class T> inline T absv(T a) { return (a < T(0.0)) ? -a : a; }
template <class T> inline T maxv(T a, T b) { return (b > a) ? b : a; }

// ---------------------------------------------------------------------------------------------
// Problem description
// ---------------------------------------------------------------------------------------------

enum { BC_PERIODIC = 0, BC_REFLECTIVE = 1, BC_OUTFLOW = 2 };

struct Grid {
  int dim, nx, ny;
  double x0, x1, y0, y1;
  int bc_x, bc_y;
  double dx() const { return (x1 - x0) / nx; }
  double dy() const { return (y1 - y0) / ny; }
};

struct Params {
  double g, cfl, eps_w, eps_lim;
  int char_decomp, limiter, linear_weights;
};

// Linear weights of the reconstruction (Sec. 2.1, after eq. GHYZZ) and of the limiter (Sec. 2.2).
static const double GAMMA[3] = {3.0 / 10.0, 3.0 / 10.0, 4.0 / 10.0};
static const double DLIM[3] = {1.0 / 4.0, 1.0 / 4.0, 1.0 / 2.0};

// ---------------------------------------------------------------------------------------------
// Scalar building blocks of Sec. 2.1 Step 1 (stencil data f[0..2] = f_{i-1}, f_i, f_{i+1})
// ---------------------------------------------------------------------------------------------

// Values of the three cubic Hermite candidates q_1, q_2, q_3 at x_{i+1/2} (eq. HWEp1).
template <class T>
void hermite_candidates(const T f[3], const T phi[3], double dx, T q[3]) {
  q[0] = 0.5 * (f[0] + f[1]) + dx / 6.0 * (phi[0] + 5.0 * phi[1]);
  q[1] = 0.5 * (f[1] + f[2]) + dx / 6.0 * (phi[1] - phi[2]);
  q[2] = (f[0] + 10.0 * f[1] + f[2]) / 12.0 + dx / 2.0 * phi[1];
}

// Smoothness indicators beta_1..beta_3 (Sec. 2.1, printed after eq. GHYZZ).
template <class T>
void smoothness(const T f[3], const T phi[3], double dx, T beta[3]) {
  T a = dx * phi[1];
  beta[0] = a * a + 13.0 / 3.0 * sq(3.0 * (f[0] - f[1]) + dx * (phi[0] + 2.0 * phi[1])) +
            781.0 / 20.0 * sq(2.0 * (f[0] - f[1]) + dx * (phi[0] + phi[1]));
  beta[1] = a * a + 13.0 / 3.0 * sq(3.0 * (f[1] - f[2]) + dx * (phi[2] + 2.0 * phi[1])) +
            781.0 / 20.0 * sq(2.0 * (f[1] - f[2]) + dx * (phi[2] + phi[1]));
  beta[2] = a * a + 13.0 / 12.0 * sq(f[0] - 2.0 * f[1] + f[2]) +
            781.0 / 80.0 * sq(f[0] - f[2] + 2.0 * dx * phi[1]);
}

// Nonlinear weights omega = omega~ / sum(omega~), omega~ = gamma / (beta + eps)^2 (eq. GHYZZ).
template <class T>
void nonlinear_weights(const T beta[3], const double lin[3], double eps, int linear, T w[3]) {
  if (linear) {
    for (int l = 0; l < 3; ++l) w[l] = T(lin[l]);
    return;
  }
  T wt[3];
  T s = T(0.0);
  for (int l = 0; l < 3; ++l) {
    wt[l] = T(lin[l]) / sq(beta[l] + eps);
    s = s + wt[l];
  }
  for (int l = 0; l < 3; ++l) w[l] = wt[l] / s;
}

// Weighted HWENO value f^_{i+1/2} = sum omega_l q_l(x_{i+1/2}) (eq. Rec-f), upwind side f'(u) >= 0.
template <class T>
T hweno_value(const T f[3], const T phi[3], double dx, double eps, int linear, T w_out[3]) {
  T q[3], beta[3];
  hermite_candidates(f, phi, dx, q);
  smoothness(f, phi, dx, beta);
  nonlinear_weights(beta, GAMMA, eps, linear, w_out);
  return w_out[0] * q[0] + w_out[1] * q[1] + w_out[2] * q[2];
}

// Derivative of the quintic Hermite polynomial Q at x_{i+1/2} (eq. Rec-phi).
template <class T>
T qprime(const T f[3], const T phi[3], double dx) {
  return (f[0] - 8.0 * f[1] + 7.0 * f[2]) / (4.0 * dx) + (phi[0] - 2.0 * phi[1] - 5.0 * phi[2]) / 12.0;
}

// HWENO limiter at one node for scalar data mu_{i-1..i+1}, nu_{i-1}, nu_{i+1}
// (eqs. step1-dxi and limiter-1d; nu_i is not used).
template <class T>
T limiter_value(const T mu[3], const T nu[3], double dx, double eps, int linear) {
  T p[3], beta[3], w[3];
  p[0] = 2.0 / dx * (mu[1] - mu[0]) - nu[0];
  p[1] = 2.0 / dx * (mu[2] - mu[1]) - nu[2];
  p[2] = 1.0 / (2.0 * dx) * (mu[2] - mu[0]);
  beta[0] = sq(2.0 * mu[1] - 2.0 * mu[0] - nu[0] * dx) + 13.0 / 3.0 * sq(mu[1] - mu[0] - nu[0] * dx);
  beta[1] = sq(2.0 * mu[2] - 2.0 * mu[1] - nu[2] * dx) + 13.0 / 3.0 * sq(mu[2] - mu[1] - nu[2] * dx);
  beta[2] = 1.0 / 4.0 * sq(mu[2] - mu[0]) + 13.0 / 12.0 * sq(mu[0] - 2.0 * mu[1] + mu[2]);
  nonlinear_weights(beta, DLIM, eps, linear, w);
  return w[0] * p[0] + w[1] * p[1] + w[2] * p[2];
}

// ---------------------------------------------------------------------------------------------
// Eigenvectors of the flux Jacobian (reading: standard SWE eigenvectors; pre-balanced variables
// have the same Jacobian with h = eta - b).
// ---------------------------------------------------------------------------------------------

// NC = 2 (1D) or 3 (2D). dir = 0 for x, 1 for y. identity if char_decomp is off.
template <class T, int NC>
void eigenvectors(int dir, T u, T v, T c, int char_decomp, T L[NC][NC], T R[NC][NC]) {
  for (int a = 0; a < NC; ++a)
    for (int b = 0; b < NC; ++b) {
      L[a][b] = T(a == b ? 1.0 : 0.0);
      R[a][b] = T(a == b ? 1.0 : 0.0);
    }
  if (!char_decomp) return;
  T ic = 1.0 / (2.0 * c);
  if (NC == 2) {
    // R = [[1,1],[u-c,u+c]], L = (1/2c)[[u+c,-1],[-(u-c),1]]
    R[0][0] = T(1.0); R[0][1] = T(1.0);
    R[1][0] = u - c;  R[1][1] = u + c;
    L[0][0] = ic * (u + c);    L[0][1] = -ic;
    L[1][0] = -ic * (u - c);   L[1][1] = ic;
    return;
  }
  if (dir == 0) {
    // R_x = [[1,0,1],[u-c,0,u+c],[v,1,v]], L_x = (1/2c)[[u+c,-1,0],[-2cv,0,2c],[-(u-c),1,0]]
    R[0][0] = T(1.0); R[0][1] = T(0.0); R[0][2] = T(1.0);
    R[1][0] = u - c;  R[1][1] = T(0.0); R[1][2] = u + c;
    R[2][0] = v;      R[2][1] = T(1.0); R[2][2] = v;
    L[0][0] = ic * (u + c);           L[0][1] = -ic;       L[0][2] = T(0.0);
    L[1][0] = ic * (-2.0 * c * v);    L[1][1] = T(0.0);    L[1][2] = ic * (2.0 * c);
    L[2][0] = -ic * (u - c);          L[2][1] = ic;        L[2][2] = T(0.0);
  } else {
    // R_y = [[1,0,1],[u,1,u],[v-c,0,v+c]], L_y = (1/2c)[[v+c,0,-1],[-2cu,2c,0],[-(v-c),0,1]]
    R[0][0] = T(1.0); R[0][1] = T(0.0); R[0][2] = T(1.0);
    R[1][0] = u;      R[1][1] = T(1.0); R[1][2] = u;
    R[2][0] = v - c;  R[2][1] = T(0.0); R[2][2] = v + c;
    L[0][0] = ic * (v + c);           L[0][1] = T(0.0);    L[0][2] = -ic;
    L[1][0] = ic * (-2.0 * c * u);    L[1][1] = ic * (2.0 * c); L[1][2] = T(0.0);
    L[2][0] = -ic * (v - c);          L[2][1] = T(0.0);    L[2][2] = ic;
  }
}

// ---------------------------------------------------------------------------------------------
// One interface x_{i+1/2} of one sweep (Sec. 2.1 Steps 1-2; in 2D Sec. 3, applied along x or y).
// Stencil nodes s = 0..3 are i-1, i, i+1, i+2 along the sweep.
//   U  : state (eta, m[, w])          D  : its derivative along the sweep (V or Q)
//   F  : flux along the sweep (F or F1 or F2)
//   G  : derivative flux along the sweep (Phi, Phi1 or Psi2)
//   bs : tilde-b or bar-b              Bs : its derivative along the sweep
// Outputs: Fhat, Ghat (derivative-equation flux), bhat (source), Bhat (derivative-equation source).
// ---------------------------------------------------------------------------------------------
template <class T, int NC>
struct Stencil {
  T U[4][NC], D[4][NC], F[4][NC], G[4][NC], bs[4][NC], Bs[4][NC];
};

template <class T, int NC>
void interface_flux(const Stencil<T, NC>& st, const T L[NC][NC], const T R[NC][NC], T alpha, double dx,
                    double eps, int linear, T Fhat[NC], T Ghat[NC], T bhat[NC], T Bhat[NC]) {
  T fchar[NC], bchar[NC];
  for (int c = 0; c < NC; ++c) {
    fchar[c] = T(0.0); bchar[c] = T(0.0); Ghat[c] = T(0.0); Bhat[c] = T(0.0);
  }
  for (int side = 0; side < 2; ++side) {
    const double sgn = side == 0 ? 1.0 : -1.0;  // F^+ = (F + alpha U)/2, F^- = (F - alpha U)/2
    // Split fluxes at the four stencil nodes (Sec. 2.1 Step 1) and split source (Step 2).
    T Fs[4][NC], Gs[4][NC], bh[4][NC], Bh[4][NC];
    for (int s = 0; s < 4; ++s)
      for (int c = 0; c < NC; ++c) {
        Fs[s][c] = 0.5 * (st.F[s][c] + sgn * alpha * st.U[s][c]);
        Gs[s][c] = 0.5 * (st.G[s][c] + sgn * alpha * st.D[s][c]);
        bh[s][c] = 0.5 * st.bs[s][c];
        Bh[s][c] = 0.5 * st.Bs[s][c];
      }
    // Upwind stencil for this side: '+' uses i-1, i, i+1; '-' is the mirror image about x_{i+1/2}
    // (nodes i+2, i+1, i, with derivatives changing sign under the reflection).
    int idx[3];
    double dsgn;
    if (side == 0) { idx[0] = 0; idx[1] = 1; idx[2] = 2; dsgn = 1.0; }
    else           { idx[0] = 3; idx[1] = 2; idx[2] = 1; dsgn = -1.0; }
    // Nonlinear reconstruction of each characteristic field (eqs. HWEp1, GHYZZ, Rec-f) and the
    // source with the same projection and the same weights (Step 2).
    for (int k = 0; k < NC; ++k) {
      T f[3], phi[3], fb[3], phib[3], w[3];
      for (int t = 0; t < 3; ++t) {
        int s = idx[t];
        T a = T(0.0), b = T(0.0), ab = T(0.0), bb = T(0.0);
        for (int c = 0; c < NC; ++c) {
          a = a + L[k][c] * Fs[s][c];
          b = b + L[k][c] * Gs[s][c];
          ab = ab + L[k][c] * bh[s][c];
          bb = bb + L[k][c] * Bh[s][c];
        }
        f[t] = a; phi[t] = dsgn * b; fb[t] = ab; phib[t] = dsgn * bb;
      }
      T fv = hweno_value(f, phi, dx, eps, linear, w);
      T qb[3];
      hermite_candidates(fb, phib, dx, qb);
      T bv = w[0] * qb[0] + w[1] * qb[1] + w[2] * qb[2];
      fchar[k] = fchar[k] + fv;
      bchar[k] = bchar[k] + bv;
    }
    // Derivative-equation fluxes: component-wise Q' (eq. Rec-phi); the mirror flips its sign.
    for (int c = 0; c < NC; ++c) {
      T f[3], phi[3], fb[3], phib[3];
      for (int t = 0; t < 3; ++t) {
        int s = idx[t];
        f[t] = Fs[s][c]; phi[t] = dsgn * Gs[s][c];
        fb[t] = bh[s][c]; phib[t] = dsgn * Bh[s][c];
      }
      Ghat[c] = Ghat[c] + dsgn * qprime(f, phi, dx);
      Bhat[c] = Bhat[c] + dsgn * qprime(fb, phib, dx);
    }
  }
  // Back to physical components: F^ = R (f^+ + f^-), likewise b^.
  for (int c = 0; c < NC; ++c) {
    T a = T(0.0), b = T(0.0);
    for (int k = 0; k < NC; ++k) {
      a = a + R[c][k] * fchar[k];
      b = b + R[c][k] * bchar[k];
    }
    Fhat[c] = a;
    bhat[c] = b;
  }
}

// Mixed-derivative interface value (eq. mixed): (-X_{i-1} + 7 X_i + 7 X_{i+1} - X_{i+2}) / 12.
template <class T>
T mixed_value(T xm1, T x0, T xp1, T xp2) {
  return -1.0 / 12.0 * xm1 + 7.0 / 12.0 * x0 + 7.0 / 12.0 * xp1 - 1.0 / 12.0 * xp2;
}

// ---------------------------------------------------------------------------------------------
// Padded planes and boundary ghosts
// ---------------------------------------------------------------------------------------------
static const int PAD = 2;

template <class T>
struct Plane {
  int nx, ny, padx, pady;
  std::vector<T> a;
  Plane() : nx(0), ny(0), padx(0), pady(0) {}
  Plane(int nx_, int ny_, int px, int py)
      : nx(nx_), ny(ny_), padx(px), pady(py), a((size_t)(nx_ + 2 * px) * (ny_ + 2 * py),
                                                 T(std::numeric_limits<double>::quiet_NaN())) {}
  T& at(int i, int j) { return a[(size_t)(j + pady) * (nx + 2 * padx) + (i + padx)]; }
  const T& at(int i, int j) const { return a[(size_t)(j + pady) * (nx + 2 * padx) + (i + padx)]; }
};

// Fill ghosts: periodic wrap; mirror about the wall faces with parity +1 (even) / -1 (odd); or, for
// transmissive boundaries, a copy of the boundary node (zero-order extrapolation of every variable).
template <class T>
void fill_ghosts(Plane<T>& p, int bc_x, int bc_y, double par_x, double par_y) {
  for (int j = 0; j < p.ny; ++j)
    for (int k = 0; k < p.padx; ++k) {
      if (bc_x == BC_PERIODIC) {
        p.at(-1 - k, j) = p.at(p.nx - 1 - k, j);
        p.at(p.nx + k, j) = p.at(k, j);
      } else if (bc_x == BC_OUTFLOW) {
        p.at(-1 - k, j) = p.at(0, j);
        p.at(p.nx + k, j) = p.at(p.nx - 1, j);
      } else {
        p.at(-1 - k, j) = par_x * p.at(k, j);
        p.at(p.nx + k, j) = par_x * p.at(p.nx - 1 - k, j);
      }
    }
  for (int i = 0; i < p.nx; ++i)
    for (int k = 0; k < p.pady; ++k) {
      if (bc_y == BC_PERIODIC) {
        p.at(i, -1 - k) = p.at(i, p.ny - 1 - k);
        p.at(i, p.ny + k) = p.at(i, k);
      } else if (bc_y == BC_OUTFLOW) {
        p.at(i, -1 - k) = p.at(i, 0);
        p.at(i, p.ny + k) = p.at(i, p.ny - 1);
      } else {
        p.at(i, -1 - k) = par_y * p.at(i, k);
        p.at(i, p.ny + k) = par_y * p.at(i, p.ny - 1 - k);
      }
    }
}

// ---------------------------------------------------------------------------------------------
// 2D scheme (Sec. 3)
// ---------------------------------------------------------------------------------------------
// State planes: 0 eta, 1 m, 2 w, 3 H1, 4 M1, 5 W1, 6 H2, 7 M2, 8 W2. Static: 0 b, 1 b_x, 2 b_y.
// Reflective parities (x-walls, y-walls), reading of the mirror symmetry of the SWE:
static const double PAR2X[12] = {+1, -1, +1, -1, +1, -1, +1, -1, +1, /*b*/ +1, /*bx*/ -1, /*by*/ +1};
static const double PAR2Y[12] = {+1, +1, -1, +1, +1, -1, -1, -1, +1, /*b*/ +1, /*bx*/ +1, /*by*/ -1};

template <class T>
struct State2D {
  Plane<T> p[12];  // 9 state + 3 static, padded
};

template <class T>
void load_state2d(const Grid& gr, const double* const* st, const double* const* stat, State2D<T>& S,
                  const double* const* dst = nullptr, const double* const* dstat = nullptr) {
  for (int q = 0; q < 12; ++q) {
    S.p[q] = Plane<T>(gr.nx, gr.ny, PAD, PAD);
    const double* src = q < 9 ? st[q] : stat[q - 9];
    const double* dsrc = nullptr;
    if (q < 9 && dst) dsrc = dst[q];
    if (q >= 9 && dstat) dsrc = dstat[q - 9];
    for (int j = 0; j < gr.ny; ++j)
      for (int i = 0; i < gr.nx; ++i) {
        size_t o = (size_t)j * gr.nx + i;
        S.p[q].at(i, j) = make_scalar<T>(src[o], dsrc ? dsrc[o] : 0.0);
      }
    fill_ghosts(S.p[q], gr.bc_x, gr.bc_y, PAR2X[q], PAR2Y[q]);
  }
}


// Pointwise fluxes of the 2D pre-balanced system (eq. swe-form-2d-e) and the derivative fluxes
// of eq. (swe-form-2d-h), written out with the chain rule:
//   d_d F1 = (M_d, 2u M_d + (gh-u^2) H_d + (u^2-g eta) B_d, -uv H_d + v M_d + u W_d + uv B_d)
//   d_d F2 = (W_d, -uv H_d + v M_d + u W_d + uv B_d, 2v W_d + (gh-v^2) H_d + (v^2-g eta) B_d)
// with Phi1 = d_x F1, Phi2 = d_x F2, Psi1 = d_y F1, Psi2 = d_y F2.
template <class T>
struct Point2D {
  T F1[3], F2[3], Phi1[3], Phi2[3], Psi1[3], Psi2[3];
};

template <class T>
void pointwise2d(double g, T eta, T m, T w, T H1, T M1, T W1, T H2, T M2, T W2, T b, T bx, T by,
                 Point2D<T>& P) {
  T h = eta - b;
  T u = m / h, v = w / h;
  T pres = 0.5 * g * (eta * eta - 2.0 * eta * b);
  P.F1[0] = m;
  P.F1[1] = m * m / h + pres;
  P.F1[2] = m * w / h;
  P.F2[0] = w;
  P.F2[1] = m * w / h;
  P.F2[2] = w * w / h + pres;
  const T Hd[2] = {H1, H2}, Md[2] = {M1, M2}, Wd[2] = {W1, W2}, Bd[2] = {bx, by};
  T* dF1[2] = {P.Phi1, P.Psi1};
  T* dF2[2] = {P.Phi2, P.Psi2};
  for (int d = 0; d < 2; ++d) {
    T cross = -u * v * Hd[d] + v * Md[d] + u * Wd[d] + u * v * Bd[d];
    dF1[d][0] = Md[d];
    dF1[d][1] = 2.0 * u * Md[d] + (g * h - u * u) * Hd[d] + (u * u - g * eta) * Bd[d];
    dF1[d][2] = cross;
    dF2[d][0] = Wd[d];
    dF2[d][1] = cross;
    dF2[d][2] = 2.0 * v * Wd[d] + (g * h - v * v) * Hd[d] + (v * v - g * eta) * Bd[d];
  }
}

// Global Lax-Friedrichs constants alpha_x = max(|u|+c), alpha_y = max(|v|+c) over the nodes.
template <class T>
void alpha2d(const Grid& gr, const Params& pr, const State2D<T>& S, T& ax, T& ay) {
  ax = T(0.0);
  ay = T(0.0);
  for (int j = 0; j < gr.ny; ++j)
    for (int i = 0; i < gr.nx; ++i) {
      T h = S.p[0].at(i, j) - S.p[9].at(i, j);
      T u = S.p[1].at(i, j) / h, v = S.p[2].at(i, j) / h;
      T c = sqrt(pr.g * h);
      ax = maxv(ax, absv(u) + c);
      ay = maxv(ay, absv(v) + c);
    }
}

// Interface values of one sweep at one interface (Sec. 2.1 Steps 1-2 along x or y, eq. mixed).
template <class T>
struct Iface2D {
  T Fh[3], Gh[3], Mh[3], bh[3], Bh[3], BMh[3];
};

// x-interface (i+1/2, j): Step 1 and Step 2 along x for (F1, Phi1, tilde-b, tilde-B1); mixed terms
// Psi1 and tilde-B2. PointAt(i, j) returns the pointwise fluxes of a node.
template <class T, class PointAt>
void x_interface(const Grid& gr, const Params& pr, const State2D<T>& S, const PointAt& P, T ax, int i, int j,
                 Iface2D<T>& o) {
  const double g = pr.g;
  Stencil<T, 3> st;
  Point2D<T> pt[4];
  for (int s = 0; s < 4; ++s) {
    int ii = i - 1 + s;
    pt[s] = P(ii, j);
    for (int c = 0; c < 3; ++c) {
      st.U[s][c] = S.p[c].at(ii, j);
      st.D[s][c] = S.p[3 + c].at(ii, j);
      st.F[s][c] = pt[s].F1[c];
      st.G[s][c] = pt[s].Phi1[c];
    }
    st.bs[s][0] = T(0.0); st.bs[s][1] = S.p[9].at(ii, j);  st.bs[s][2] = T(0.0);
    st.Bs[s][0] = T(0.0); st.Bs[s][1] = S.p[10].at(ii, j); st.Bs[s][2] = T(0.0);
  }
  T hl = S.p[0].at(i, j) - S.p[9].at(i, j), hr = S.p[0].at(i + 1, j) - S.p[9].at(i + 1, j);
  T hbar = 0.5 * (hl + hr);
  T ubar = (S.p[1].at(i, j) + S.p[1].at(i + 1, j)) / (hl + hr);
  T vbar = (S.p[2].at(i, j) + S.p[2].at(i + 1, j)) / (hl + hr);
  T cbar = sqrt(g * hbar);
  T L[3][3], R[3][3];
  eigenvectors<T, 3>(0, ubar, vbar, cbar, pr.char_decomp, L, R);
  interface_flux<T, 3>(st, L, R, ax, gr.dx(), pr.eps_w, pr.linear_weights, o.Fh, o.Gh, o.bh, o.Bh);
  for (int c = 0; c < 3; ++c) o.Mh[c] = mixed_value(pt[0].Psi1[c], pt[1].Psi1[c], pt[2].Psi1[c], pt[3].Psi1[c]);
  o.BMh[0] = T(0.0);
  o.BMh[1] = mixed_value(S.p[11].at(i - 1, j), S.p[11].at(i, j), S.p[11].at(i + 1, j), S.p[11].at(i + 2, j));
  o.BMh[2] = T(0.0);
}

// y-interface (i, j+1/2): Step 1 and Step 2 along y for (F2, Psi2, bar-b, bar-B2); mixed terms Phi2
// and bar-B1.
template <class T, class PointAt>
void y_interface(const Grid& gr, const Params& pr, const State2D<T>& S, const PointAt& P, T ay, int i, int j,
                 Iface2D<T>& o) {
  const double g = pr.g;
  Stencil<T, 3> st;
  Point2D<T> pt[4];
  for (int s = 0; s < 4; ++s) {
    int jj = j - 1 + s;
    pt[s] = P(i, jj);
    for (int c = 0; c < 3; ++c) {
      st.U[s][c] = S.p[c].at(i, jj);
      st.D[s][c] = S.p[6 + c].at(i, jj);
      st.F[s][c] = pt[s].F2[c];
      st.G[s][c] = pt[s].Psi2[c];
    }
    st.bs[s][0] = T(0.0); st.bs[s][1] = T(0.0); st.bs[s][2] = S.p[9].at(i, jj);
    st.Bs[s][0] = T(0.0); st.Bs[s][1] = T(0.0); st.Bs[s][2] = S.p[11].at(i, jj);
  }
  T hl = S.p[0].at(i, j) - S.p[9].at(i, j), hr = S.p[0].at(i, j + 1) - S.p[9].at(i, j + 1);
  T hbar = 0.5 * (hl + hr);
  T ubar = (S.p[1].at(i, j) + S.p[1].at(i, j + 1)) / (hl + hr);
  T vbar = (S.p[2].at(i, j) + S.p[2].at(i, j + 1)) / (hl + hr);
  T cbar = sqrt(g * hbar);
  T L[3][3], R[3][3];
  eigenvectors<T, 3>(1, ubar, vbar, cbar, pr.char_decomp, L, R);
  interface_flux<T, 3>(st, L, R, ay, gr.dy(), pr.eps_w, pr.linear_weights, o.Fh, o.Gh, o.bh, o.Bh);
  for (int c = 0; c < 3; ++c) o.Mh[c] = mixed_value(pt[0].Phi2[c], pt[1].Phi2[c], pt[2].Phi2[c], pt[3].Phi2[c]);
  o.BMh[0] = T(0.0);
  o.BMh[1] = T(0.0);
  o.BMh[2] = mixed_value(S.p[10].at(i, j - 1), S.p[10].at(i, j), S.p[10].at(i, j + 1), S.p[10].at(i, j + 2));
}

// Assembly of eq. (swe-form-2d-dis) at one node from its four interfaces; r[0..8] = d/dt of
// (eta, m, w, H1, M1, W1, H2, M2, W2).
template <class T>
void assemble2d(const Grid& gr, const Params& pr, const State2D<T>& S, int i, int j, const Iface2D<T>& xl,
                const Iface2D<T>& xr, const Iface2D<T>& yl, const Iface2D<T>& yr, T r[9]) {
  const double dx = gr.dx(), dy = gr.dy(), g = pr.g;
  T eta = S.p[0].at(i, j), H1 = S.p[3].at(i, j), H2 = S.p[6].at(i, j);
  for (int c = 0; c < 3; ++c) {
    T db = (xr.bh[c] - xl.bh[c]) / dx + (yr.bh[c] - yl.bh[c]) / dy;
    r[c] = -(xr.Fh[c] - xl.Fh[c]) / dx - (yr.Fh[c] - yl.Fh[c]) / dy - g * eta * db;
    r[3 + c] = -(xr.Gh[c] - xl.Gh[c]) / dx - (yr.Mh[c] - yl.Mh[c]) / dy -
               g * eta * ((xr.Bh[c] - xl.Bh[c]) / dx + (yr.BMh[c] - yl.BMh[c]) / dy) - g * H1 * db;
    r[6 + c] = -(xr.Mh[c] - xl.Mh[c]) / dx - (yr.Gh[c] - yl.Gh[c]) / dy -
               g * eta * ((xr.BMh[c] - xl.BMh[c]) / dx + (yr.Bh[c] - yl.Bh[c]) / dy) - g * H2 * db;
  }
}

template <class T>
Point2D<T> point_at(const Params& pr, const State2D<T>& S, int i, int j) {
  Point2D<T> P;
  pointwise2d(pr.g, S.p[0].at(i, j), S.p[1].at(i, j), S.p[2].at(i, j), S.p[3].at(i, j), S.p[4].at(i, j),
              S.p[5].at(i, j), S.p[6].at(i, j), S.p[7].at(i, j), S.p[8].at(i, j), S.p[9].at(i, j),
              S.p[10].at(i, j), S.p[11].at(i, j), P);
  return P;
}

template <class T> struct Parallel { static const bool ok = true; };
template <> struct Parallel<Cnt> { static const bool ok = false; };

// Right-hand side R, R_x, R_y of eq. (swe-form-2d-dis) on the whole grid, source signs read as '-'.
// out[0..8]: d/dt of (eta, m, w, H1, M1, W1, H2, M2, W2), each nx*ny, row-major.
template <class T>
void rhs2d(const Grid& gr, const Params& pr, const State2D<T>& S, T ax, T ay, std::vector<T> out[9]) {
  const int nx = gr.nx, ny = gr.ny;
  // Pointwise fluxes on every node a sweep reads (row j: i in [-2, nx+2); column i: j in [-2, ny+2)).
  Plane<Point2D<T>> P;
  P.nx = nx; P.ny = ny; P.padx = PAD; P.pady = PAD;
  P.a.resize((size_t)(nx + 2 * PAD) * (ny + 2 * PAD));
#pragma omp parallel for if (Parallel<T>::ok)
  for (int j = -PAD; j < ny + PAD; ++j) {
    if (j >= 0 && j < ny) {
      for (int i = -PAD; i < nx + PAD; ++i) P.at(i, j) = point_at(pr, S, i, j);
    } else {
      for (int i = 0; i < nx; ++i) P.at(i, j) = point_at(pr, S, i, j);
    }
  }
  auto PA = [&](int i, int j) { return P.at(i, j); };
  // Interface values. x-interface i+1/2 is stored at index i (i = -1..nx-1), y likewise.
  Plane<Iface2D<T>> X, Y;
  X.nx = nx; X.ny = ny; X.padx = 1; X.pady = 0; X.a.resize((size_t)(nx + 2) * ny);
  Y.nx = nx; Y.ny = ny; Y.padx = 0; Y.pady = 1; Y.a.resize((size_t)nx * (ny + 2));
#pragma omp parallel for if (Parallel<T>::ok)
  for (int j = 0; j < ny; ++j)
    for (int i = -1; i < nx; ++i) x_interface(gr, pr, S, PA, ax, i, j, X.at(i, j));
#pragma omp parallel for if (Parallel<T>::ok)
  for (int j = -1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) y_interface(gr, pr, S, PA, ay, i, j, Y.at(i, j));
  for (int q = 0; q < 9; ++q) out[q].assign((size_t)nx * ny, T(0.0));
#pragma omp parallel for if (Parallel<T>::ok)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      T r[9];
      assemble2d(gr, pr, S, i, j, X.at(i - 1, j), X.at(i, j), Y.at(i, j - 1), Y.at(i, j), r);
      for (int q = 0; q < 9; ++q) out[q][(size_t)j * nx + i] = r[q];
    }
}

// The same right-hand side at one node only, every interface recomputed from the padded state.
template <class T>
void rhs2d_at(const Grid& gr, const Params& pr, const State2D<T>& S, T ax, T ay, int i, int j, T r[9]) {
  auto PA = [&](int ii, int jj) { return point_at(pr, S, ii, jj); };
  Iface2D<T> xl, xr, yl, yr;
  x_interface(gr, pr, S, PA, ax, i - 1, j, xl);
  x_interface(gr, pr, S, PA, ax, i, j, xr);
  y_interface(gr, pr, S, PA, ay, i, j - 1, yl);
  y_interface(gr, pr, S, PA, ay, i, j, yr);
  assemble2d(gr, pr, S, i, j, xl, xr, yl, yr, r);
}

// HWENO limiter in 2D (Sec. 2.2 applied dimension by dimension, end of Sec. 3) at one node: V along x
// with the x-eigenvectors at the node, Q along y with the y-eigenvectors at the node.
// mod[0..5] = V^mod, Q^mod.
template <class T>
void limiter2d_at(const Grid& gr, const Params& pr, const State2D<T>& S, int i, int j, T mod[6]) {
  if (!pr.limiter) {
    for (int q = 0; q < 6; ++q) mod[q] = S.p[3 + q].at(i, j);
    return;
  }
  T h = S.p[0].at(i, j) - S.p[9].at(i, j);
  T u = S.p[1].at(i, j) / h, v = S.p[2].at(i, j) / h, c = sqrt(pr.g * h);
  for (int d = 0; d < 2; ++d) {
    T L[3][3], R[3][3];
    eigenvectors<T, 3>(d, u, v, c, pr.char_decomp, L, R);
    const double del = d == 0 ? gr.dx() : gr.dy();
    T numod[3];
    for (int k = 0; k < 3; ++k) {
      T mu[3], nu[3];
      for (int t = 0; t < 3; ++t) {
        int ii = d == 0 ? i - 1 + t : i, jj = d == 0 ? j : j - 1 + t;
        T a = T(0.0), b = T(0.0);
        for (int cc = 0; cc < 3; ++cc) {
          a = a + L[k][cc] * S.p[cc].at(ii, jj);
          b = b + L[k][cc] * S.p[3 + 3 * d + cc].at(ii, jj);
        }
        mu[t] = a;
        nu[t] = b;
      }
      numod[k] = limiter_value(mu, nu, del, pr.eps_lim, pr.linear_weights);
    }
    for (int cc = 0; cc < 3; ++cc) {
      T a = T(0.0);
      for (int k = 0; k < 3; ++k) a = a + R[cc][k] * numod[k];
      mod[3 * d + cc] = a;
    }
  }
}

template <class T>
void limiter2d(const Grid& gr, const Params& pr, const State2D<T>& S, std::vector<T> mod[6]) {
  const int nx = gr.nx, ny = gr.ny;
  for (int q = 0; q < 6; ++q) mod[q].assign((size_t)nx * ny, T(0.0));
#pragma omp parallel for if (Parallel<T>::ok)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      T m[6];
      limiter2d_at(gr, pr, S, i, j, m);
      for (int q = 0; q < 6; ++q) mod[q][(size_t)j * nx + i] = m[q];
    }
}

// One SSP-RK3 stage (eq. RK). R is evaluated on the unmodified stage state; the combination uses
// the limited derivatives. Stage 1 stores the step's base U^n and the limited V^{n,mod}, Q^{n,mod}.
// (a_k, b_k) = (0,1), (3/4,1/4), (1/3,2/3): S^(k) = a_k base + b_k (S^(k-1),mod + dt R(S^(k-1))).
template <class T>
void stage2d(const Grid& gr, const Params& pr, int k, double dt, const State2D<T>& S,
             std::vector<T> base[9], std::vector<T> out[9], T* alpha_used) {
  const size_t n = (size_t)gr.nx * gr.ny;
  T ax, ay;
  alpha2d(gr, pr, S, ax, ay);
  if (alpha_used) { alpha_used[0] = ax; alpha_used[1] = ay; }
  std::vector<T> R[9], mod[6];
  rhs2d(gr, pr, S, ax, ay, R);
  limiter2d(gr, pr, S, mod);
  if (k == 1) {
    for (int q = 0; q < 9; ++q) base[q].resize(n);
    for (int j = 0; j < gr.ny; ++j)
      for (int i = 0; i < gr.nx; ++i) {
        size_t o = (size_t)j * gr.nx + i;
        for (int q = 0; q < 3; ++q) base[q][o] = S.p[q].at(i, j);
        for (int q = 0; q < 6; ++q) base[3 + q][o] = mod[q][o];
      }
  }
  const T a = k == 1 ? T(0.0) : (k == 2 ? rk_ratio<T>(3.0, 4.0) : rk_ratio<T>(1.0, 3.0));
  const T b = k == 1 ? T(1.0) : (k == 2 ? rk_ratio<T>(1.0, 4.0) : rk_ratio<T>(2.0, 3.0));
  for (int q = 0; q < 9; ++q) out[q].resize(n);
  for (int j = 0; j < gr.ny; ++j)
    for (int i = 0; i < gr.nx; ++i) {
      size_t o = (size_t)j * gr.nx + i;
      for (int q = 0; q < 9; ++q) {
        T cur = q < 3 ? S.p[q].at(i, j) : mod[q - 3][o];
        if (k == 1)
          out[q][o] = cur + dt * R[q][o];
        else
          out[q][o] = a * base[q][o] + b * (cur + dt * R[q][o]);
      }
    }
}

// ---------------------------------------------------------------------------------------------
// 1D scheme (Sec. 2)
// ---------------------------------------------------------------------------------------------
// State planes: 0 eta, 1 m, 2 H, 3 M. Static: 0 b, 1 b_x.
static const double PAR1[6] = {+1, -1, -1, +1, /*b*/ +1, /*bx*/ -1};

template <class T>
struct State1D {
  Plane<T> p[6];
};

template <class T>
void load_state1d(const Grid& gr, const double* const* st, const double* const* stat, State1D<T>& S,
                  const double* const* dst = nullptr, const double* const* dstat = nullptr) {
  for (int q = 0; q < 6; ++q) {
    S.p[q] = Plane<T>(gr.nx, 1, PAD, 0);
    const double* src = q < 4 ? st[q] : stat[q - 4];
    const double* dsrc = nullptr;
    if (q < 4 && dst) dsrc = dst[q];
    if (q >= 4 && dstat) dsrc = dstat[q - 4];
    for (int i = 0; i < gr.nx; ++i) S.p[q].at(i, 0) = make_scalar<T>(src[i], dsrc ? dsrc[i] : 0.0);
    fill_ghosts(S.p[q], gr.bc_x, BC_PERIODIC, PAR1[q], 1.0);
  }
}

template <class T>
T alpha1d(const Grid& gr, const Params& pr, const State1D<T>& S) {
  T a = T(0.0);
  for (int i = 0; i < gr.nx; ++i) {
    T h = S.p[0].at(i, 0) - S.p[4].at(i, 0);
    T u = S.p[1].at(i, 0) / h;
    a = maxv(a, absv(u) + sqrt(pr.g * h));
  }
  return a;
}

// F (eq. swe-form-1d-e) and Phi (printed after eq. swe-form-1d-h) at one node.
template <class T>
void pointwise1d(double g, T eta, T m, T H, T M, T b, T bx, T F[2], T Phi[2]) {
  T h = eta - b;
  F[0] = m;
  F[1] = m * m / h + 0.5 * g * (eta * eta - 2.0 * eta * b);
  Phi[0] = M;
  Phi[1] = (g * h - m * m / (h * h)) * H + 2.0 * m / h * M + (m * m / (h * h) - g * eta) * bx;
}

// R, R_x of eq. (swe-form-1d-semi). out[0..3] = d/dt (eta, m, H, M).
template <class T>
void rhs1d(const Grid& gr, const Params& pr, const State1D<T>& S, T alpha, std::vector<T> out[4]) {
  const int nx = gr.nx;
  const double dx = gr.dx(), g = pr.g;
  std::vector<T> F((size_t)(nx + 4) * 2), Phi((size_t)(nx + 4) * 2);
  for (int i = -PAD; i < nx + PAD; ++i)
    pointwise1d(g, S.p[0].at(i, 0), S.p[1].at(i, 0), S.p[2].at(i, 0), S.p[3].at(i, 0), S.p[4].at(i, 0),
                S.p[5].at(i, 0), &F[(size_t)(i + PAD) * 2], &Phi[(size_t)(i + PAD) * 2]);
  std::vector<T> Fh((size_t)(nx + 1) * 2), Gh((size_t)(nx + 1) * 2), bh((size_t)(nx + 1) * 2),
      Bh((size_t)(nx + 1) * 2);
  for (int i = -1; i < nx; ++i) {
    Stencil<T, 2> st;
    for (int s = 0; s < 4; ++s) {
      int ii = i - 1 + s;
      for (int c = 0; c < 2; ++c) {
        st.U[s][c] = S.p[c].at(ii, 0);
        st.D[s][c] = S.p[2 + c].at(ii, 0);
        st.F[s][c] = F[(size_t)(ii + PAD) * 2 + c];
        st.G[s][c] = Phi[(size_t)(ii + PAD) * 2 + c];
      }
      st.bs[s][0] = T(0.0); st.bs[s][1] = S.p[4].at(ii, 0);
      st.Bs[s][0] = T(0.0); st.Bs[s][1] = S.p[5].at(ii, 0);
    }
    T hl = S.p[0].at(i, 0) - S.p[4].at(i, 0), hr = S.p[0].at(i + 1, 0) - S.p[4].at(i + 1, 0);
    T hbar = 0.5 * (hl + hr);
    T ubar = (S.p[1].at(i, 0) + S.p[1].at(i + 1, 0)) / (hl + hr);
    T cbar = sqrt(g * hbar);
    T L[2][2], R[2][2];
    eigenvectors<T, 2>(0, ubar, T(0.0), cbar, pr.char_decomp, L, R);
    size_t o = (size_t)(i + 1) * 2;
    interface_flux<T, 2>(st, L, R, alpha, dx, pr.eps_w, pr.linear_weights, &Fh[o], &Gh[o], &bh[o], &Bh[o]);
  }
  for (int q = 0; q < 4; ++q) out[q].assign(nx, T(0.0));
  for (int i = 0; i < nx; ++i) {
    size_t r = (size_t)(i + 1) * 2, l = (size_t)i * 2;
    T eta = S.p[0].at(i, 0), H = S.p[2].at(i, 0);
    for (int c = 0; c < 2; ++c) {
      out[c][i] = -g * eta * (bh[r + c] - bh[l + c]) / dx - (Fh[r + c] - Fh[l + c]) / dx;
      out[2 + c][i] = -g * H * (bh[r + c] - bh[l + c]) / dx - g * eta * (Bh[r + c] - Bh[l + c]) / dx -
                      (Gh[r + c] - Gh[l + c]) / dx;
    }
  }
}

template <class T>
void limiter1d(const Grid& gr, const Params& pr, const State1D<T>& S, std::vector<T> mod[2]) {
  const int nx = gr.nx;
  for (int q = 0; q < 2; ++q) mod[q].assign(nx, T(0.0));
  for (int i = 0; i < nx; ++i) {
    if (!pr.limiter) {
      mod[0][i] = S.p[2].at(i, 0);
      mod[1][i] = S.p[3].at(i, 0);
      continue;
    }
    T h = S.p[0].at(i, 0) - S.p[4].at(i, 0);
    T u = S.p[1].at(i, 0) / h, c = sqrt(pr.g * h);
    T L[2][2], R[2][2];
    eigenvectors<T, 2>(0, u, T(0.0), c, pr.char_decomp, L, R);
    T numod[2];
    for (int k = 0; k < 2; ++k) {
      T mu[3], nu[3];
      for (int t = 0; t < 3; ++t) {
        mu[t] = L[k][0] * S.p[0].at(i - 1 + t, 0) + L[k][1] * S.p[1].at(i - 1 + t, 0);
        nu[t] = L[k][0] * S.p[2].at(i - 1 + t, 0) + L[k][1] * S.p[3].at(i - 1 + t, 0);
      }
      numod[k] = limiter_value(mu, nu, gr.dx(), pr.eps_lim, pr.linear_weights);
    }
    for (int cc = 0; cc < 2; ++cc) mod[cc][i] = R[cc][0] * numod[0] + R[cc][1] * numod[1];
  }
}

template <class T>
void stage1d(const Grid& gr, const Params& pr, int k, double dt, const State1D<T>& S, std::vector<T> base[4],
             std::vector<T> out[4], T* alpha_used) {
  const int nx = gr.nx;
  T al = alpha1d(gr, pr, S);
  if (alpha_used) alpha_used[0] = al;
  std::vector<T> R[4], mod[2];
  rhs1d(gr, pr, S, al, R);
  limiter1d(gr, pr, S, mod);
  if (k == 1) {
    for (int q = 0; q < 4; ++q) base[q].resize(nx);
    for (int i = 0; i < nx; ++i) {
      base[0][i] = S.p[0].at(i, 0);
      base[1][i] = S.p[1].at(i, 0);
      base[2][i] = mod[0][i];
      base[3][i] = mod[1][i];
    }
  }
  const T a = k == 1 ? T(0.0) : (k == 2 ? rk_ratio<T>(3.0, 4.0) : rk_ratio<T>(1.0, 3.0));
  const T b = k == 1 ? T(1.0) : (k == 2 ? rk_ratio<T>(1.0, 4.0) : rk_ratio<T>(2.0, 3.0));
  for (int q = 0; q < 4; ++q) out[q].resize(nx);
  for (int i = 0; i < nx; ++i)
    for (int q = 0; q < 4; ++q) {
      T cur = q < 2 ? S.p[q].at(i, 0) : mod[q - 2][i];
      if (k == 1)
        out[q][i] = cur + dt * R[q][i];
      else
        out[q][i] = a * base[q][i] + b * (cur + dt * R[q][i]);
    }
}

}  // namespace orc

// =============================================================================================
// C ABI (loaded with ctypes by the tests, the smoke check and the CPU-baseline leg only)
// =============================================================================================
using orc::Grid;
using orc::Params;

namespace {
template <class T>
void to_ptrs(std::vector<T>* v, int n, double* const* out) {
  for (int q = 0; q < n; ++q)
    for (size_t o = 0; o < v[q].size(); ++o) out[q][o] = orc::val(v[q][o]);
}
int check_grid(const Grid* g) {
  if (!g || g->nx < 1 || g->ny < 1) return -1;
  if (g->dim == 1 && g->ny != 1) return -1;
  if (g->dim != 1 && g->dim != 2) return -1;
  if (g->bc_x < 0 || g->bc_x > 2 || g->bc_y < 0 || g->bc_y > 2) return -1;
  if (g->nx < 2 || (g->dim == 2 && g->ny < 2)) return -1;  // reflective/periodic halo of 2 needs >= 2 nodes
  return 0;
}
}  // namespace

// One RHS / one stage of the 2D scheme in the scalar type T, from and to double planes.
template <class T>
int rhs2d_as(const Grid* g, const Params* p, const double* const* st, const double* const* stat, double* const* out,
             double* a2) {
  if (check_grid(g) || g->dim != 2) return -1;
  orc::State2D<T> S;
  orc::load_state2d(*g, st, stat, S);
  T ax, ay;
  orc::alpha2d(*g, *p, S, ax, ay);
  std::vector<T> R[9];
  orc::rhs2d(*g, *p, S, ax, ay, R);
  to_ptrs(R, 9, out);
  if (a2) { a2[0] = orc::val(ax); a2[1] = orc::val(ay); }
  return 0;
}
template <class T>
int stage2d_as(const Grid* g, const Params* p, int k, double dt, const double* const* st, const double* const* stat,
               double* const* base, double* const* out, double* a2) {
  if (check_grid(g) || g->dim != 2 || k < 1 || k > 3) return -1;
  const size_t n = (size_t)g->nx * g->ny;
  orc::State2D<T> S;
  orc::load_state2d(*g, st, stat, S);
  std::vector<T> B[9], O[9];
  if (k > 1)
    for (int q = 0; q < 9; ++q)
      for (size_t o = 0; o < n; ++o) B[q].push_back(T(base[q][o]));
  T al[2];
  orc::stage2d(*g, *p, k, dt, S, B, O, al);
  if (k == 1) to_ptrs(B, 9, base);
  to_ptrs(O, 9, out);
  if (a2) { a2[0] = orc::val(al[0]); a2[1] = orc::val(al[1]); }
  return 0;
}

extern "C" {

// ---- scalar pieces (pins) ----
void orc_candidates(const double* f, const double* phi, double dx, double* q) { orc::hermite_candidates(f, phi, dx, q); }
void orc_smoothness(const double* f, const double* phi, double dx, double* b) { orc::smoothness(f, phi, dx, b); }
double orc_hweno_value(const double* f, const double* phi, double dx, double eps, int linear, double* w) {
  double ww[3];
  double r = orc::hweno_value(f, phi, dx, eps, linear, ww);
  if (w) for (int l = 0; l < 3; ++l) w[l] = ww[l];
  return r;
}
double orc_qprime(const double* f, const double* phi, double dx) { return orc::qprime(f, phi, dx); }
double orc_limiter_value(const double* mu, const double* nu, double dx, double eps, int linear) {
  return orc::limiter_value(mu, nu, dx, eps, linear);
}
void orc_eigenvectors(int nc, int dir, double u, double v, double c, double* L, double* R) {
  if (nc == 2) {
    double l[2][2], r[2][2];
    orc::eigenvectors<double, 2>(dir, u, v, c, 1, l, r);
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) { L[a * 2 + b] = l[a][b]; R[a * 2 + b] = r[a][b]; }
  } else {
    double l[3][3], r[3][3];
    orc::eigenvectors<double, 3>(dir, u, v, c, 1, l, r);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) { L[a * 3 + b] = l[a][b]; R[a * 3 + b] = r[a][b]; }
  }
}
// Pointwise 2D fluxes: out[18] = F1, F2, Phi1, Phi2, Psi1, Psi2.
void orc_pointwise2d(double g, const double* s12, double* out) {
  orc::Point2D<double> P;
  orc::pointwise2d(g, s12[0], s12[1], s12[2], s12[3], s12[4], s12[5], s12[6], s12[7], s12[8], s12[9], s12[10],
                   s12[11], P);
  for (int c = 0; c < 3; ++c) {
    out[c] = P.F1[c]; out[3 + c] = P.F2[c]; out[6 + c] = P.Phi1[c];
    out[9 + c] = P.Phi2[c]; out[12 + c] = P.Psi1[c]; out[15 + c] = P.Psi2[c];
  }
}

// ---- 2D ----
int orc_alpha2d(const Grid* g, const Params* p, const double* const* st, const double* const* stat, double* a2) {
  if (check_grid(g) || g->dim != 2) return -1;
  orc::State2D<double> S;
  orc::load_state2d(*g, st, stat, S);
  orc::alpha2d(*g, *p, S, a2[0], a2[1]);
  return 0;
}
int orc_rhs2d(const Grid* g, const Params* p, const double* const* st, const double* const* stat, double* const* out,
              double* a2) {
  return rhs2d_as<double>(g, p, st, stat, out, a2);
}
// The same in single precision (every operation in float; inputs rounded to float, outputs widened).
int orc_rhs2d_f32(const Grid* g, const Params* p, const double* const* st, const double* const* stat,
                  double* const* out, double* a2) {
  return rhs2d_as<orc::F32>(g, p, st, stat, out, a2);
}
int orc_limiter2d(const Grid* g, const Params* p, const double* const* st, const double* const* stat,
                  double* const* mod) {
  if (check_grid(g) || g->dim != 2) return -1;
  orc::State2D<double> S;
  orc::load_state2d(*g, st, stat, S);
  std::vector<double> M[6];
  orc::limiter2d(*g, *p, S, M);
  to_ptrs(M, 6, mod);
  return 0;
}
// One RK stage. base[9] is written for k == 1 and read for k = 2, 3.
int orc_stage2d(const Grid* g, const Params* p, int k, double dt, const double* const* st,
                const double* const* stat, double* const* base, double* const* out, double* a2) {
  return stage2d_as<double>(g, p, k, dt, st, stat, base, out, a2);
}
int orc_stage2d_f32(const Grid* g, const Params* p, int k, double dt, const double* const* st,
                    const double* const* stat, double* const* base, double* const* out, double* a2) {
  return stage2d_as<orc::F32>(g, p, k, dt, st, stat, base, out, a2);
}
// Stage output at selected nodes only (sampled parity at sizes the full oracle grid would be slow
// on). alpha2 gives the stage's alpha (computed over the full grid by orc_alpha2d); base holds the
// step's base planes (U^n, V^{n,mod}, Q^{n,mod}) at the selected nodes for k = 2, 3 (ignored for k == 1).
int orc_stage2d_points(const Grid* g, const Params* p, int k, double dt, const double* const* st,
                       const double* const* stat, const double* a2, int npts, const int* pi, const int* pj,
                       const double* base_pts, double* out_pts, double* mod_pts) {
  if (check_grid(g) || g->dim != 2 || k < 1 || k > 3) return -1;
  orc::State2D<double> S;
  orc::load_state2d(*g, st, stat, S);
  const double a = k == 1 ? 0.0 : (k == 2 ? 3.0 / 4.0 : 1.0 / 3.0);
  const double b = k == 1 ? 1.0 : (k == 2 ? 1.0 / 4.0 : 2.0 / 3.0);
#pragma omp parallel for
  for (int n = 0; n < npts; ++n) {
    int i = pi[n], j = pj[n];
    double r[9], m[6];
    orc::rhs2d_at(*g, *p, S, a2[0], a2[1], i, j, r);
    orc::limiter2d_at(*g, *p, S, i, j, m);
    for (int q = 0; q < 9; ++q) {
      double cur = q < 3 ? S.p[q].at(i, j) : m[q - 3];
      if (k == 1)
        out_pts[(size_t)n * 9 + q] = cur + dt * r[q];
      else
        out_pts[(size_t)n * 9 + q] = a * base_pts[(size_t)n * 9 + q] + b * (cur + dt * r[q]);
    }
    if (mod_pts)
      for (int q = 0; q < 6; ++q) mod_pts[(size_t)n * 6 + q] = m[q];
  }
  return 0;
}
int orc_rk3_step2d(const Grid* g, const Params* p, double dt, double* const* st, const double* const* stat) {
  if (check_grid(g) || g->dim != 2) return -1;
  const size_t n = (size_t)g->nx * g->ny;
  std::vector<double> B[9], cur[9], nxt[9];
  for (int q = 0; q < 9; ++q) cur[q].assign(st[q], st[q] + n);
  for (int k = 1; k <= 3; ++k) {
    const double* cp[9];
    for (int q = 0; q < 9; ++q) cp[q] = cur[q].data();
    orc::State2D<double> S;
    orc::load_state2d(*g, cp, stat, S);
    orc::stage2d(*g, *p, k, dt, S, B, nxt, (double*)nullptr);
    for (int q = 0; q < 9; ++q) cur[q].swap(nxt[q]);
  }
  to_ptrs(cur, 9, st);
  return 0;
}
// CFL time step from the state (Sec. 4: CFL number 0.6): dt = cfl / (alpha_x/dx + alpha_y/dy).
double orc_cfl_dt2d(const Grid* g, const Params* p, const double* const* st, const double* const* stat) {
  double a2[2];
  if (orc_alpha2d(g, p, st, stat, a2)) return -1.0;
  return p->cfl / (a2[0] / g->dx() + a2[1] / g->dy());
}
// Operation tally of one RK stage (k = 2: RHS, limiter and the full combination) on the given
// state: counts[0..4] = add/sub, mul, div, sqrt, compare.
int orc_count_stage2d(const Grid* g, const Params* p, const double* const* st, const double* const* stat,
                      double* counts) {
  if (check_grid(g) || g->dim != 2) return -1;
  const size_t n = (size_t)g->nx * g->ny;
  orc::State2D<orc::Cnt> S;
  orc::load_state2d(*g, st, stat, S);
  std::vector<orc::Cnt> B[9], O[9];
  for (int q = 0; q < 9; ++q) B[q].assign(n, orc::Cnt(0.0));
  orc::g_ops = {0, 0, 0, 0, 0};
  orc::stage2d(*g, *p, 2, 1e-4, S, B, O, (orc::Cnt*)nullptr);
  counts[0] = orc::g_ops.add; counts[1] = orc::g_ops.mul; counts[2] = orc::g_ops.div;
  counts[3] = orc::g_ops.sqrt; counts[4] = orc::g_ops.cmp;
  return 0;
}

// ---- 1D ----
int orc_alpha1d(const Grid* g, const Params* p, const double* const* st, const double* const* stat, double* a) {
  if (check_grid(g) || g->dim != 1) return -1;
  orc::State1D<double> S;
  orc::load_state1d(*g, st, stat, S);
  *a = orc::alpha1d(*g, *p, S);
  return 0;
}
int orc_rhs1d(const Grid* g, const Params* p, const double* const* st, const double* const* stat, double* const* out,
              double* a) {
  if (check_grid(g) || g->dim != 1) return -1;
  orc::State1D<double> S;
  orc::load_state1d(*g, st, stat, S);
  double al = orc::alpha1d(*g, *p, S);
  std::vector<double> R[4];
  orc::rhs1d(*g, *p, S, al, R);
  to_ptrs(R, 4, out);
  if (a) *a = al;
  return 0;
}
int orc_limiter1d(const Grid* g, const Params* p, const double* const* st, const double* const* stat,
                  double* const* mod) {
  if (check_grid(g) || g->dim != 1) return -1;
  orc::State1D<double> S;
  orc::load_state1d(*g, st, stat, S);
  std::vector<double> M[2];
  orc::limiter1d(*g, *p, S, M);
  to_ptrs(M, 2, mod);
  return 0;
}
int orc_stage1d(const Grid* g, const Params* p, int k, double dt, const double* const* st,
                const double* const* stat, double* const* base, double* const* out, double* a) {
  if (check_grid(g) || g->dim != 1 || k < 1 || k > 3) return -1;
  const size_t n = (size_t)g->nx;
  orc::State1D<double> S;
  orc::load_state1d(*g, st, stat, S);
  std::vector<double> B[4], O[4];
  if (k > 1)
    for (int q = 0; q < 4; ++q) B[q].assign(base[q], base[q] + n);
  double al;
  orc::stage1d(*g, *p, k, dt, S, B, O, &al);
  if (k == 1) to_ptrs(B, 4, base);
  to_ptrs(O, 4, out);
  if (a) *a = al;
  return 0;
}
int orc_rk3_step1d(const Grid* g, const Params* p, double dt, double* const* st, const double* const* stat) {
  if (check_grid(g) || g->dim != 1) return -1;
  const size_t n = (size_t)g->nx;
  std::vector<double> B[4], cur[4], nxt[4];
  for (int q = 0; q < 4; ++q) cur[q].assign(st[q], st[q] + n);
  for (int k = 1; k <= 3; ++k) {
    const double* cp[4];
    for (int q = 0; q < 4; ++q) cp[q] = cur[q].data();
    orc::State1D<double> S;
    orc::load_state1d(*g, cp, stat, S);
    orc::stage1d(*g, *p, k, dt, S, B, nxt, (double*)nullptr);
    for (int q = 0; q < 4; ++q) cur[q].swap(nxt[q]);
  }
  to_ptrs(cur, 4, st);
  return 0;
}
double orc_cfl_dt1d(const Grid* g, const Params* p, const double* const* st, const double* const* stat) {
  double a;
  if (orc_alpha1d(g, p, st, stat, &a)) return -1.0;
  return p->cfl * g->dx() / a;
}

}  // extern "C"

// =============================================================================================
// Gauge-misfit loss of a 2D run and its directional derivative (forward-mode dual numbers): the
// independent reference for the adjoint. L = sum_{n=1..N} sum_g (eta^n[g] - obs[n-1][g])^2.
// =============================================================================================
namespace orc {
template <class T>
void set_state2d(const Grid& gr, State2D<T>& S, std::vector<T>* planes) {
  for (int q = 0; q < 9; ++q) {
    for (int j = 0; j < gr.ny; ++j)
      for (int i = 0; i < gr.nx; ++i) S.p[q].at(i, j) = planes[q][(size_t)j * gr.nx + i];
    fill_ghosts(S.p[q], gr.bc_x, gr.bc_y, PAR2X[q], PAR2Y[q]);
  }
}

template <class T>
T gauge_loss2d(const Grid& gr, const Params& pr, State2D<T>& S, int nsteps, const double* dts, const int* gidx, int ng,
               const double* obs) {
  T L = T(0.0);
  std::vector<T> B[9], O[9];
  for (int n = 0; n < nsteps; ++n) {
    for (int k = 1; k <= 3; ++k) {
      stage2d(gr, pr, k, dts[n], S, B, O, (T*)nullptr);
      set_state2d(gr, S, O);
    }
    for (int g = 0; g < ng; ++g) {
      const int i = gidx[g] % gr.nx, j = gidx[g] / gr.nx;
      T e = S.p[0].at(i, j) - obs[(size_t)n * ng + g];
      L = L + e * e;
    }
  }
  return L;
}
}  // namespace orc

extern "C" int orc_gauge_loss_dual2d(const Grid* g, const Params* p, const double* const* st, const double* const* stat,
                                     const double* const* dst, const double* const* dstat, int nsteps, const double* dts,
                                     const int* gidx, int ng, const double* obs, double* out2) {
  if (check_grid(g) || g->dim != 2 || nsteps < 1 || ng < 1) return -1;
  orc::State2D<orc::Dual> S;
  orc::load_state2d(*g, st, stat, S, dst, dstat);
  orc::Dual L = orc::gauge_loss2d(*g, *p, S, nsteps, dts, gidx, ng, obs);
  out2[0] = L.v;
  out2[1] = L.d;
  return 0;
}

// =============================================================================================
// Lake at rest in single, double and double-double precision (Sec. 4, Ex. 4.2 Tables 1-2 and
// Ex. 4.7 Table 3): the run to t_end at the CFL time step and the L1 / Linf deviations of h and the
// discharges from the initial state (whose exact solution it is).
// =============================================================================================
namespace orc {
template <class T>
void set_state1d(const Grid& gr, State1D<T>& S, std::vector<T>* planes) {
  for (int q = 0; q < 4; ++q) {
    for (int i = 0; i < gr.nx; ++i) S.p[q].at(i, 0) = planes[q][i];
    fill_ghosts(S.p[q], gr.bc_x, BC_PERIODIC, PAR1[q], 1.0);
  }
}

inline bool last_step(double t, double dt, double t_end) { return dt >= (t_end - t) - 1e-12 * t_end; }

// out: for each of the nq conserved planes (h first, then the discharges) its L1 and Linf deviation.
template <class T>
int lake_run1d(const Grid& gr, const Params& pr, const double* const* st, const double* const* stat, double t_end,
               double* out, int* steps) {
  State1D<T> S;
  load_state1d(gr, st, stat, S);
  std::vector<T> init[2];
  for (int q = 0; q < 2; ++q)
    for (int i = 0; i < gr.nx; ++i) init[q].push_back(S.p[q].at(i, 0));
  double t = 0.0;
  int n = 0;
  while (t < t_end && n < 1000000) {
    double dt = pr.cfl * gr.dx() / val(alpha1d(gr, pr, S));
    const bool last = last_step(t, dt, t_end);
    if (last) dt = t_end - t;
    std::vector<T> B[4], O[4];
    for (int k = 1; k <= 3; ++k) {
      stage1d(gr, pr, k, dt, S, B, O, (T*)nullptr);
      set_state1d(gr, S, O);
    }
    t = last ? t_end : t + dt;
    ++n;
  }
  for (int q = 0; q < 2; ++q) {
    double l1 = 0.0, li = 0.0;
    for (int i = 0; i < gr.nx; ++i) {
      const double e = std::fabs(val(S.p[q].at(i, 0) - init[q][i]));  // h - h0 = eta - eta0 (b is fixed)
      l1 += e;
      li = std::max(li, e);
    }
    out[2 * q] = l1 / gr.nx;
    out[2 * q + 1] = li;
  }
  *steps = n;
  return 0;
}

template <class T>
int lake_run2d(const Grid& gr, const Params& pr, const double* const* st, const double* const* stat, double t_end,
               double* out, int* steps) {
  State2D<T> S;
  load_state2d(gr, st, stat, S);
  std::vector<T> init[3];
  for (int q = 0; q < 3; ++q)
    for (int j = 0; j < gr.ny; ++j)
      for (int i = 0; i < gr.nx; ++i) init[q].push_back(S.p[q].at(i, j));
  double t = 0.0;
  int n = 0;
  while (t < t_end && n < 1000000) {
    T ax, ay;
    alpha2d(gr, pr, S, ax, ay);
    double dt = pr.cfl / (val(ax) / gr.dx() + val(ay) / gr.dy());
    const bool last = last_step(t, dt, t_end);
    if (last) dt = t_end - t;
    std::vector<T> B[9], O[9];
    for (int k = 1; k <= 3; ++k) {
      stage2d(gr, pr, k, dt, S, B, O, (T*)nullptr);
      set_state2d(gr, S, O);
    }
    t = last ? t_end : t + dt;
    ++n;
  }
  const size_t nn = (size_t)gr.nx * gr.ny;
  for (int q = 0; q < 3; ++q) {
    double l1 = 0.0, li = 0.0;
    for (int j = 0; j < gr.ny; ++j)
      for (int i = 0; i < gr.nx; ++i) {
        const double e = std::fabs(val(S.p[q].at(i, j) - init[q][(size_t)j * gr.nx + i]));
        l1 += e;
        li = std::max(li, e);
      }
    out[2 * q] = l1 / nn;
    out[2 * q + 1] = li;
  }
  *steps = n;
  return 0;
}
}  // namespace orc

// precision: 0 single, 1 double, 2 double-double. out: L1, Linf of h, then of the discharge(s).
extern "C" int orc_lake_run(const Grid* g, const Params* p, const double* const* st, const double* const* stat,
                            double t_end, int precision, double* out, int* steps) {
  if (check_grid(g) || !(t_end > 0.0) || !out || !steps) return -1;
  if (g->dim == 1) {
    if (precision == 0) return orc::lake_run1d<orc::F32>(*g, *p, st, stat, t_end, out, steps);
    if (precision == 1) return orc::lake_run1d<double>(*g, *p, st, stat, t_end, out, steps);
    if (precision == 2) return orc::lake_run1d<orc::DD>(*g, *p, st, stat, t_end, out, steps);
  } else {
    if (precision == 0) return orc::lake_run2d<orc::F32>(*g, *p, st, stat, t_end, out, steps);
    if (precision == 1) return orc::lake_run2d<double>(*g, *p, st, stat, t_end, out, steps);
    if (precision == 2) return orc::lake_run2d<orc::DD>(*g, *p, st, stat, t_end, out, steps);
  }
  return -1;
}
