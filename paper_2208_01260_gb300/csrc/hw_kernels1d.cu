// 1D kernels of the well-balanced fifth-order FD HWENO scheme (Zhao & Zhang, arXiv:2208.01260,
// Sec. 2): state (eta, m, dx H, dx M), static (b, dx b_x). Same conventions as the 2D kernels
// (see hw_device.cuh): split without 1/2, projection rows without 1/(2c), epsilon rescaled.
#include "hw_device.cuh"
#include "hw_internal.h"

namespace hw {

enum { Q_FP = 0, Q_FM = 2, Q_GP = 4, Q_GM = 6, Q_H = 8, Q_M = 9, NREC1 = 10 };

struct Node6 {
  double v[6];  // eta m H' M' b bxs
};

__device__ __forceinline__ void load_node1d(const Dev1D& d, int i, Node6& n) {
  bool f;
  const int ii = map_index(i, d.nx, d.bc, f);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double x = __ldg(d.S[q] + ii);
    n.v[q] = f ? x * par_1d(q) : x;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    double x = __ldg(d.stat[q] + ii);
    n.v[4 + q] = f ? x * par_1d(4 + q) : x;
  }
}

// F and Phi of Sec. 2 (eq. swe-form-1d-e and the printed Phi), split with alpha (no 1/2).
__device__ __forceinline__ void node_record1d(const Node6& n, double g, double alpha, double rec[NREC1]) {
  const double eta = n.v[0], m = n.v[1], H = n.v[2], M = n.v[3], b = n.v[4], B = n.v[5];
  const double h = eta - b;
  const double u = m * fast_rcp(h);
  const double gh = g * h, ge = g * eta;
  const double pres = ge * fma(0.5, eta, -b);
  const double uu = u * u;
  const double F0 = m, F1 = fma(m, u, pres);
  const double G0 = M, G1 = fma(u + u, M, fma(gh - uu, H, (uu - ge) * B));
  rec[Q_FP] = fma(alpha, eta, F0);
  rec[Q_FP + 1] = fma(alpha, m, F1);
  rec[Q_FM] = fma(-alpha, eta, F0);
  rec[Q_FM + 1] = fma(-alpha, m, F1);
  rec[Q_GP] = fma(alpha, H, G0);
  rec[Q_GP + 1] = fma(alpha, M, G1);
  rec[Q_GM] = fma(-alpha, H, G0);
  rec[Q_GM + 1] = fma(-alpha, M, G1);
  rec[Q_H] = h;
  rec[Q_M] = m;
}

// Outputs (6): 2 Fhat (2), 2 bhat (2), 24 dx Phihat (2).
template <bool LINEAR, bool CHAR>
__device__ __forceinline__ void interface_values1d(const double* r0, const double* r1, const double* r2,
                                                   const double* r3, int stride, const double qb[6], double g,
                                                   double eps_w, double out[6]) {
#define RV(r, f) (r)[(f) * stride]
  const double hs = RV(r1, Q_H) + RV(r2, Q_H);
  const double ub = (RV(r1, Q_M) + RV(r2, Q_M)) * fast_rcp(hs);
  const double gh = (0.5 * g) * hs;
  const double rs = fast_rsqrt(gh);
  const double cb = gh * rs, ic2 = 0.5 * rs;
  const double upc = ub + cb, umc = ub - cb;
  const double eps = CHAR ? (8.0 * g * eps_w) * hs : 4.0 * eps_w;
  const double* rp[4] = {r0, r1, r2, r3};
  double G[2], GB1 = 0.0, GB2 = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int os[3] = {side == 0 ? 0 : 3, side == 0 ? 1 : 2, side == 0 ? 2 : 1};
    const int fo = side == 0 ? Q_FP : Q_FM, go = side == 0 ? Q_GP : Q_GM;
    const double sg = side == 0 ? 1.0 : -1.0;
    double f[2][3], p[2][3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const double* r = rp[os[t]];
      const double F0 = RV(r, fo), F1 = RV(r, fo + 1);
      const double G0 = sg * RV(r, go), G1 = sg * RV(r, go + 1);
      if (CHAR) {
        // rows of L without 1/(2c): (u+c, -1), (-(u-c), 1)
        f[0][t] = fma(upc, F0, -F1);
        f[1][t] = fma(-umc, F0, F1);
        p[0][t] = fma(upc, G0, -G1);
        p[1][t] = fma(-umc, G0, G1);
      } else {
        f[0][t] = F0; f[1][t] = F1; p[0][t] = G0; p[1][t] = G1;
      }
    }
    const double* qbs = qb + 3 * side;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      Weights W;
      const double v = hweno_side<LINEAR>(f[k][0], f[k][1], f[k][2], p[k][0], p[k][1], p[k][2], eps, W);
      G[k] = side == 0 ? v : G[k] + v;
      if (CHAR) {
        if (k == 0) GB1 -= weighted(W, qbs[0], qbs[1], qbs[2]);
        else GB2 += weighted(W, qbs[0], qbs[1], qbs[2]);
      } else if (k == 1) {
        GB2 += weighted(W, qbs[0], qbs[1], qbs[2]);
      }
    }
  }
  if (CHAR) {
    const double A = (G[0] + G[1]) * ic2;
    out[0] = A;
    out[1] = fma(ub, A, 0.5 * (G[1] - G[0]));
    const double B = (GB1 + GB2) * ic2;
    out[2] = B;
    out[3] = fma(ub, B, 0.5 * (GB2 - GB1));
  } else {
    out[0] = G[0]; out[1] = G[1];
    out[2] = 0.0;  out[3] = GB2;
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const double fpart =
        fma(7.0, RV(r2, Q_FP + c) - RV(r1, Q_FM + c),
            fma(8.0, RV(r2, Q_FM + c) - RV(r1, Q_FP + c), RV(r0, Q_FP + c) - RV(r3, Q_FM + c)));
    const double gpart = fma(-5.0, RV(r2, Q_GP + c) + RV(r1, Q_GM + c),
                             fma(-2.0, RV(r1, Q_GP + c) + RV(r2, Q_GM + c), RV(r0, Q_GP + c) + RV(r3, Q_GM + c)));
    out[4 + c] = fma(3.0, fpart, gpart);
  }
#undef RV
}

constexpr int X1_T = 128;
constexpr int X1_N = X1_T + 3;

template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(X1_T) k_sweep1d(Dev1D d, const double* __restrict__ alpha) {
  __shared__ double sm[NREC1 * X1_N];
  const int k0 = blockIdx.x * X1_T;
  const double a = alpha[0];
  for (int t = threadIdx.x; t < X1_N; t += X1_T) {
    const int i = k0 - 2 + t;
    if (i > d.nx + 1) break;
    Node6 n;
    load_node1d(d, i, n);
    double rec[NREC1];
    node_record1d(n, d.g, a, rec);
#pragma unroll
    for (int f = 0; f < NREC1; ++f) sm[f * X1_N + t] = rec[f];
  }
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (k > d.nx) return;
  const int t = threadIdx.x;
  double qb[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) qb[q] = __ldg(d.qb[q] + k);
  double out[6];
  interface_values1d<LINEAR, CHAR>(sm + t, sm + t + 1, sm + t + 2, sm + t + 3, X1_N, qb, d.g, d.eps_w, out);
#pragma unroll
  for (int q = 0; q < 6; ++q) d.X[q][k] = out[q];
}

template <int MODE, bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(128) k_node1d(Dev1D d, StageArgs1D sa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nx) return;
  double cur[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) cur[q] = __ldg(d.S[q] + i);
  if (MODE == MODE_STAGE && !(*sa.dt > 0.0)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) sa.out[q][i] = cur[q];
    return;
  }
  const double eta = cur[0], H = cur[2];
  const double g = d.g, ge = g * eta;
  double R[4];
  // eq. (swe-form-1d-semi): R = -g eta [b^]/dx - [F^]/dx; dx R_x = -g (dx H)[b^]/dx - g eta [B^] - [Phi^]
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const double dF = __ldg(d.X[c] + i + 1) - __ldg(d.X[c] + i);
    const double db = d.c_b * (__ldg(d.X[2 + c] + i + 1) - __ldg(d.X[2 + c] + i));
    const double dG = __ldg(d.X[4 + c] + i + 1) - __ldg(d.X[4 + c] + i);
    R[c] = fma(-ge, db, -d.c_b * dF);
    double rv = fma(-g * H, db, -d.c_g * dG);
    if (c == 1) rv = fma(-ge, __ldg(d.sv + i), rv);
    R[2 + c] = rv;
  }
  if (MODE == MODE_RHS) {
#pragma unroll
    for (int q = 0; q < 4; ++q) sa.rhs_out[q][i] = q < 2 ? R[q] : R[q] * d.inv_dx;
    return;
  }
  double mod[2];
  if (sa.limiter) {
    const double b0 = __ldg(d.stat[0] + i);
    const double h = eta - b0, gh = g * h;
    const double u = cur[1] * fast_rcp(h);
    const double rs = fast_rsqrt(gh);
    const double c = gh * rs, ic2 = 0.5 * rs;
    Node6 nm, np;
    load_node1d(d, i - 1, nm);
    load_node1d(d, i + 1, np);
    double nu[2];
    if (CHAR) {
      const double upc = u + c, umc = u - c;
      const double e = (4.0 * d.eps_lim) * gh;
      const double m0a = fma(upc, nm.v[0], -nm.v[1]), m1a = fma(upc, cur[0], -cur[1]), m2a = fma(upc, np.v[0], -np.v[1]);
      const double nla = fma(upc, nm.v[2], -nm.v[3]), nra = fma(upc, np.v[2], -np.v[3]);
      const double m0b = fma(-umc, nm.v[0], nm.v[1]), m1b = fma(-umc, cur[0], cur[1]), m2b = fma(-umc, np.v[0], np.v[1]);
      const double nlb = fma(-umc, nm.v[2], nm.v[3]), nrb = fma(-umc, np.v[2], np.v[3]);
      nu[0] = limiter_field<LINEAR>(m0a, m1a, m2a, nla, nra, e);
      nu[1] = limiter_field<LINEAR>(m0b, m1b, m2b, nlb, nrb, e);
      const double A = (nu[0] + nu[1]) * ic2;
      mod[0] = A;
      mod[1] = fma(u, A, 0.5 * (nu[1] - nu[0]));
    } else {
      mod[0] = limiter_field<LINEAR>(nm.v[0], cur[0], np.v[0], nm.v[2], np.v[2], d.eps_lim);
      mod[1] = limiter_field<LINEAR>(nm.v[1], cur[1], np.v[1], nm.v[3], np.v[3], d.eps_lim);
    }
  } else {
    mod[0] = cur[2];
    mod[1] = cur[3];
  }
  const double dt = *sa.dt;
  if (sa.k == 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double cq = q < 2 ? cur[q] : mod[q - 2];
      if (sa.base) sa.base[q][i] = cq;
      sa.out[q][i] = fma(dt, R[q], cq);
    }
  } else {
    const double a = sa.k == 2 ? 0.75 : 1.0 / 3.0;
    const double b = sa.k == 2 ? 0.25 : 2.0 / 3.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double cq = q < 2 ? cur[q] : mod[q - 2];
      sa.out[q][i] = fma(a, __ldg(sa.base[q] + i), b * fma(dt, R[q], cq));
    }
  }
}

__global__ void __launch_bounds__(256) k_alpha1d(Dev1D d, unsigned long long* amax, int* status) {
  unsigned long long k = 0;
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.nx; i += gridDim.x * blockDim.x) {
    const double h = __ldg(d.S[0] + i) - __ldg(d.stat[0] + i);
    if (!(h > 0.0) || !(h < 1e300)) { bad |= h == h ? HW_STATUS_DEPTH : HW_STATUS_NONFINITE; continue; }
    const double gh = d.g * h;
    const double a = dabs(__ldg(d.S[1] + i) * fast_rcp(h)) + gh * fast_rsqrt(gh);
    if (!(a < 1e300)) { bad |= HW_STATUS_NONFINITE; continue; }
    k = max(k, dkey(a));
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, s));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, k);
  if (bad) atomicOr(status, bad);
}

__global__ void k_finish_alpha1d(const unsigned long long* amax, double* alpha, double* dt_out, double cfl,
                                 double dx, const double* t_now, double t_end) {
  const double a = __longlong_as_double((long long)amax[0]);
  alpha[0] = a;
  alpha[1] = 0.0;
  if (dt_out) {
    double dt = cfl * dx / a;
    double t_next = t_now ? *t_now + dt : 0.0;
    if (t_now && t_end > 0.0) {
      // the step that reaches t_end (within a relative 1e-12) ends exactly on it
      const double rem = t_end - *t_now;
      if (dt >= rem - 1e-12 * t_end) {
        dt = rem > 0.0 ? rem : 0.0;
        t_next = rem > 0.0 ? t_end : *t_now;
      }
    }
    *dt_out = dt;
    if (t_now) dt_out[1] = t_next;
  }
}

__global__ void k_init1d(Dev1D d, PhysIn1D in, int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.nx; i += gridDim.x * blockDim.x) {
    const double h = in.p[0][i], b = in.p[2][i], bx = in.p[5][i];
    if (!(h > 0.0) || !(h < 1e300)) atomicOr(status, h == h ? HW_STATUS_DEPTH : HW_STATUS_NONFINITE);
    d.S[0][i] = h + b;
    d.S[1][i] = in.p[1][i];
    d.S[2][i] = d.dx * (in.p[3][i] + bx);
    d.S[3][i] = d.dx * in.p[4][i];
    d.stat[0][i] = b;
    d.stat[1][i] = d.dx * bx;
    d.bx[i] = bx;
  }
}

__device__ __forceinline__ double bval1d(const Dev1D& d, int q, int i) {
  bool f;
  const int ii = map_index(i, d.nx, d.bc, f);
  double x = q == 0 ? d.stat[0][ii] : d.bx[ii];
  return (f && q == 1) ? -x : x;
}

__global__ void k_static1d(Dev1D d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= d.nx) {
    double b[4], s[4];
    for (int t = 0; t < 4; ++t) {
      b[t] = bval1d(d, 0, k - 2 + t);
      s[t] = d.dx * bval1d(d, 1, k - 2 + t);
    }
    d.qb[0][k] = 0.5 * (b[0] + b[1]) + (s[0] + 5.0 * s[1]) / 6.0;
    d.qb[1][k] = 0.5 * (b[1] + b[2]) + (s[1] - s[2]) / 6.0;
    d.qb[2][k] = (b[0] + 10.0 * b[1] + b[2]) / 12.0 + 0.5 * s[1];
    d.qb[3][k] = 0.5 * (b[3] + b[2]) + (-s[3] - 5.0 * s[2]) / 6.0;
    d.qb[4][k] = 0.5 * (b[2] + b[1]) + (-s[2] + s[1]) / 6.0;
    d.qb[5][k] = (b[3] + 10.0 * b[2] + b[1]) / 12.0 - 0.5 * s[2];
  }
  if (k < d.nx) {
    auto Bh = [&](int kk) {  // (Q'+ + Q'-) on (b/2, b_x/2) at interface kk-1/2 (eq. Rec-phi)
      const double b0 = bval1d(d, 0, kk - 2), b1 = bval1d(d, 0, kk - 1), b2 = bval1d(d, 0, kk), b3 = bval1d(d, 0, kk + 1);
      const double s0 = bval1d(d, 1, kk - 2), s1 = bval1d(d, 1, kk - 1), s2 = bval1d(d, 1, kk), s3 = bval1d(d, 1, kk + 1);
      const double qp = (b0 - 8.0 * b1 + 7.0 * b2) / (4.0 * d.dx) + (s0 - 2.0 * s1 - 5.0 * s2) / 12.0;
      const double qm = (-7.0 * b1 + 8.0 * b2 - b3) / (4.0 * d.dx) + (-5.0 * s1 - 2.0 * s2 + s3) / 12.0;
      return 0.5 * (qp + qm);
    };
    d.sv[k] = Bh(k + 1) - Bh(k);
  }
}

__global__ void k_convert1d(Dev1D d, Ptr9 src4, Ptr9 dst4, int layout, int dir) {
  double* const* S = d.S;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.nx; i += gridDim.x * blockDim.x) {
    const double b = d.stat[0][i], bx = d.bx[i];
    if (dir == 0) {
      const double x0 = S[0][i], x1 = S[1][i], x2 = S[2][i], x3 = S[3][i];
      dst4.p[0][i] = layout == 0 ? x0 - b : x0;
      dst4.p[1][i] = x1;
      dst4.p[2][i] = layout == 0 ? x2 * d.inv_dx - bx : x2 * d.inv_dx;
      dst4.p[3][i] = x3 * d.inv_dx;
    } else {
      const double x0 = src4.p[0][i], x1 = src4.p[1][i], x2 = src4.p[2][i], x3 = src4.p[3][i];
      S[0][i] = layout == 0 ? x0 + b : x0;
      S[1][i] = x1;
      S[2][i] = d.dx * (layout == 0 ? x2 + bx : x2);
      S[3][i] = d.dx * x3;
    }
  }
}

// ---- launchers ----
void launch_alpha1d(const Dev1D& d, unsigned long long* amax, int* status, cudaStream_t st) {
  cudaMemsetAsync(amax, 0, sizeof(unsigned long long), st);
  int blocks = std::min((d.nx + 255) / 256, 152 * 4);
  k_alpha1d<<<blocks, 256, 0, st>>>(d, amax, status);
}
void launch_finish_alpha1d(const Dev1D& d, const unsigned long long* amax, double* alpha, double* dt_out,
                           double cfl, const double* t_now, double t_end, cudaStream_t st) {
  k_finish_alpha1d<<<1, 1, 0, st>>>(amax, alpha, dt_out, cfl, d.dx, t_now, t_end);
}
void launch_sweep1d(const Dev1D& d, const double* alpha, bool linear, bool chr, cudaStream_t st) {
  const int g = (d.nx + 1 + X1_T - 1) / X1_T;
  if (linear) { if (chr) k_sweep1d<true, true><<<g, X1_T, 0, st>>>(d, alpha); else k_sweep1d<true, false><<<g, X1_T, 0, st>>>(d, alpha); }
  else        { if (chr) k_sweep1d<false, true><<<g, X1_T, 0, st>>>(d, alpha); else k_sweep1d<false, false><<<g, X1_T, 0, st>>>(d, alpha); }
}
void launch_node1d(const Dev1D& d, const StageArgs1D& sa, int mode, bool linear, bool chr, cudaStream_t st) {
  const int g = (d.nx + 127) / 128;
#define L1(M, A, B) k_node1d<M, A, B><<<g, 128, 0, st>>>(d, sa)
  if (mode == MODE_RHS) {
    if (linear) { if (chr) L1(MODE_RHS, true, true); else L1(MODE_RHS, true, false); }
    else        { if (chr) L1(MODE_RHS, false, true); else L1(MODE_RHS, false, false); }
  } else {
    if (linear) { if (chr) L1(MODE_STAGE, true, true); else L1(MODE_STAGE, true, false); }
    else        { if (chr) L1(MODE_STAGE, false, true); else L1(MODE_STAGE, false, false); }
  }
#undef L1
}
void launch_init1d(const Dev1D& d, const PhysIn1D& in, int* status, cudaStream_t st) {
  const int blocks = std::min((d.nx + 255) / 256, 152 * 4);
  k_init1d<<<blocks, 256, 0, st>>>(d, in, status);
  k_static1d<<<(d.nx + 1 + 127) / 128, 128, 0, st>>>(d);
}
void launch_convert1d(const Dev1D& d, const Ptr9& src, const Ptr9& dst, int layout, int dir, cudaStream_t st) {
  const int blocks = std::min((d.nx + 255) / 256, 152 * 4);
  k_convert1d<<<blocks, 256, 0, st>>>(d, src, dst, layout, dir);
}

}  // namespace hw
