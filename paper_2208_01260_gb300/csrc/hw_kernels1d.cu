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

// The same interface with its four independent nonlinear reconstructions (field k on side s, Sec. 2.1
// Step 1) on four lanes of a warp: lanes 4j .. 4j + 3 compute interface j, lane r taking field r >> 1 on
// side r & 1, and exchange their values by shuffles in the order interface_values1d adds them, so the
// outputs are the same values. Lane r returns output components {0, 1}, {2, 3}, {4} or {5} for
// r = 0, 1, 2, 3 in o[0..1]. Every lane of the warp must call (the shuffles take the full warp).
// For grids whose sweep has too few interfaces to occupy the GPU: one warp's chain of FP64 instructions,
// not the GPU's FP64 throughput, then sets the kernel's duration, and this chain is about a third as long.
template <bool LINEAR, bool CHAR>
__device__ __forceinline__ void interface_values1d_lanes(const double* r0, const double* r1, const double* r2,
                                                         const double* r3, int stride, const Dev1D& d, int kq,
                                                         int lane, double o[2]) {
#define RV(r, f) (r)[(f) * stride]
  const double g = d.g, eps_w = d.eps_w;
  const double hs = RV(r1, Q_H) + RV(r2, Q_H);
  const double ub = (RV(r1, Q_M) + RV(r2, Q_M)) * fast_rcp(hs);
  const double gh = (0.5 * g) * hs;
  const double rs = fast_rsqrt(gh);
  const double cb = gh * rs, ic2 = 0.5 * rs;
  const double upc = ub + cb, umc = ub - cb;
  const double eps = CHAR ? (8.0 * g * eps_w) * hs : 4.0 * eps_w;
  const int k = lane >> 1, side = lane & 1;
  // '+': nodes 0, 1, 2 of (F+, G+); '-': nodes 3, 2, 1 of (F-, G-) with the derivative negated
  const double* a0 = side == 0 ? r0 : r3;
  const double* a1 = side == 0 ? r1 : r2;
  const double* a2 = side == 0 ? r2 : r1;
  const int fo = side == 0 ? Q_FP : Q_FM, go = side == 0 ? Q_GP : Q_GM;
  const double sg = side == 0 ? 1.0 : -1.0;
  // rows of L without 1/(2c): (u+c, -1), (-(u-c), 1)
  const double ca = k == 0 ? upc : -umc, cs = k == 0 ? -1.0 : 1.0;
  const double* ap[3] = {a0, a1, a2};
  double f[3], p[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const double F0 = RV(ap[t], fo), F1 = RV(ap[t], fo + 1);
    const double G0 = sg * RV(ap[t], go), G1 = sg * RV(ap[t], go + 1);
    if (CHAR) {
      f[t] = fma(ca, F0, cs * F1);
      p[t] = fma(ca, G0, cs * G1);
    } else {
      f[t] = k == 0 ? F0 : F1;
      p[t] = k == 0 ? G0 : G1;
    }
  }
  Weights W;
  const double v = hweno_side<LINEAR>(f[0], f[1], f[2], p[0], p[1], p[2], eps, W);
  double w = 0.0;
  if (CHAR || k == 1) {
    const int qo = 3 * side;
    w = weighted(W, __ldg(d.qb[qo] + kq), __ldg(d.qb[qo + 1] + kq), __ldg(d.qb[qo + 2] + kq));
  }
  // the two sides of a field (lanes r, r ^ 1), in the order '+' then '-'
  const double vo = __shfl_xor_sync(0xffffffffu, v, 1), wo = __shfl_xor_sync(0xffffffffu, w, 1);
  const double Gk = side == 0 ? v + vo : vo + v;
  const double w0 = side == 0 ? w : wo, w1 = side == 0 ? wo : w;
  const double Bk = (CHAR && k == 0) ? (0.0 - w0) - w1 : (0.0 + w0) + w1;  // field 1: GB1 -= ..., field 2: GB2 += ...
  // the other field (lanes r, r ^ 2)
  const double Gx = __shfl_xor_sync(0xffffffffu, Gk, 2), Bx = __shfl_xor_sync(0xffffffffu, Bk, 2);
  const double G0 = k == 0 ? Gk : Gx, G1 = k == 0 ? Gx : Gk;
  const double GB1 = CHAR ? (k == 0 ? Bk : Bx) : 0.0, GB2 = k == 0 ? Bx : Bk;
  if (lane == 0) {
    if (CHAR) {
      const double A = (G0 + G1) * ic2;
      o[0] = A;
      o[1] = fma(ub, A, 0.5 * (G1 - G0));
    } else {
      o[0] = G0;
      o[1] = G1;
    }
  } else if (lane == 1) {
    if (CHAR) {
      const double B = (GB1 + GB2) * ic2;
      o[0] = B;
      o[1] = fma(ub, B, 0.5 * (GB2 - GB1));
    } else {
      o[0] = 0.0;
      o[1] = GB2;
    }
  } else {
    const int c = lane - 2;
    const double fpart =
        fma(7.0, RV(r2, Q_FP + c) - RV(r1, Q_FM + c),
            fma(8.0, RV(r2, Q_FM + c) - RV(r1, Q_FP + c), RV(r0, Q_FP + c) - RV(r3, Q_FM + c)));
    const double gpart = fma(-5.0, RV(r2, Q_GP + c) + RV(r1, Q_GM + c),
                             fma(-2.0, RV(r1, Q_GP + c) + RV(r2, Q_GM + c), RV(r0, Q_GP + c) + RV(r3, Q_GM + c)));
    o[0] = fma(3.0, fpart, gpart);
    o[1] = 0.0;
  }
#undef RV
}

constexpr int X1_T = 128;
constexpr int X1_N = X1_T + 3;
// The four-lane sweep: XL_I interfaces per block of 4 XL_I threads, used while the grid has at most
// kLaneSweepMax interfaces (up to one such warp per SM partition: 152 SMs x 4 partitions x 8 interfaces).
constexpr int XL_I = 32;
constexpr int XL_T = 4 * XL_I;
constexpr int XL_N = XL_I + 3;
constexpr int kLaneSweepMax = 152 * 4 * 8;

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

template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(XL_T) k_sweep1d_lanes(Dev1D d, const double* __restrict__ alpha) {
  __shared__ double sm[NREC1 * XL_N];
  const int k0 = blockIdx.x * XL_I;
  const double a = alpha[0];
  for (int t = threadIdx.x; t < XL_N; t += XL_T) {
    const int i = k0 - 2 + t;
    if (i > d.nx + 1) break;
    Node6 n;
    load_node1d(d, i, n);
    double rec[NREC1];
    node_record1d(n, d.g, a, rec);
#pragma unroll
    for (int f = 0; f < NREC1; ++f) sm[f * XL_N + t] = rec[f];
  }
  __syncthreads();
  const int j = threadIdx.x >> 2, lane = threadIdx.x & 3;
  const int k = k0 + j;
  const bool live = k <= d.nx;
  const int jj = live ? j : 0;  // past the last interface: the block's first interface again, not written
  double o[2];
  interface_values1d_lanes<LINEAR, CHAR>(sm + jj, sm + jj + 1, sm + jj + 2, sm + jj + 3, XL_N, d, k0 + jj, lane, o);
  if (!live) return;
  if (lane < 2) {
    d.X[2 * lane][k] = o[0];
    d.X[2 * lane + 1][k] = o[1];
  } else {
    d.X[2 + lane][k] = o[0];
  }
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

// The node update with two lanes per node, for grids with few nodes (as the four-lane sweep): lane 0
// forms the U components (eta, m), lane 1 the V components; the limiter's two characteristic fields
// (without the projection: its two components) run one on each lane and meet by a shuffle. Both lanes
// run one instruction stream (the lane picks operands, never a branch), with the same operations on the
// same values as k_node1d. Every lane of the warp must call (the shuffle takes the full warp).
constexpr int NL_N = 64;                    // nodes per block of 2 NL_N threads
constexpr int kLaneNodeMax = 152 * 4 * 16;  // up to one such warp per SM partition

template <int MODE, bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(2 * NL_N) k_node1d_lanes(Dev1D d, StageArgs1D sa) {
  const int lane = threadIdx.x & 1;
  const int ir = blockIdx.x * NL_N + (threadIdx.x >> 1);
  const bool live = ir < d.nx;
  const int i = live ? ir : d.nx - 1;  // past the last node: the last node again, not written
  double cur[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) cur[q] = __ldg(d.S[q] + i);
  if (MODE == MODE_STAGE && !(*sa.dt > 0.0)) {
    if (live) {
      (lane ? sa.out[2] : sa.out[0])[i] = lane ? cur[2] : cur[0];
      (lane ? sa.out[3] : sa.out[1])[i] = lane ? cur[3] : cur[1];
    }
    return;
  }
  const double eta = cur[0], H = cur[2];
  const double g = d.g, ge = g * eta;
  // eq. (swe-form-1d-semi) as in k_node1d; this lane's components: R[c] (lane 0) or R[2 + c] (lane 1)
  double R2[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const double db = d.c_b * (__ldg(d.X[2 + c] + i + 1) - __ldg(d.X[2 + c] + i));
    const double* Xd = lane ? d.X[4 + c] : d.X[c];
    const double dd = __ldg(Xd + i + 1) - __ldg(Xd + i);
    const double A = lane ? -g * H : -ge;
    double r = fma(A, db, -(lane ? d.c_g : d.c_b) * dd);
    if (c == 1) {
      const double rs1 = fma(-ge, __ldg(d.sv + i), r);
      r = lane ? rs1 : r;
    }
    R2[c] = r;
  }
  if (MODE == MODE_RHS) {
    if (live) {
      (lane ? sa.rhs_out[2] : sa.rhs_out[0])[i] = lane ? R2[0] * d.inv_dx : R2[0];
      (lane ? sa.rhs_out[3] : sa.rhs_out[1])[i] = lane ? R2[1] * d.inv_dx : R2[1];
    }
    return;
  }
  double mod0, mod1;
  if (sa.limiter) {
    const double b0 = __ldg(d.stat[0] + i);
    const double h = eta - b0, gh = g * h;
    const double u = cur[1] * fast_rcp(h);
    const double rs = fast_rsqrt(gh);
    const double c = gh * rs, ic2 = 0.5 * rs;
    Node6 nm, np;
    load_node1d(d, i - 1, nm);
    load_node1d(d, i + 1, np);
    double nu;
    if (CHAR) {
      const double upc = u + c, umc = u - c;
      const double e = (4.0 * d.eps_lim) * gh;
      // field a: row (u+c, -1); field b: row (-(u-c), 1)
      const double ca = lane ? -umc : upc, cs = lane ? 1.0 : -1.0;
      const double m0 = fma(ca, nm.v[0], cs * nm.v[1]), m1 = fma(ca, cur[0], cs * cur[1]), m2 = fma(ca, np.v[0], cs * np.v[1]);
      const double nl = fma(ca, nm.v[2], cs * nm.v[3]), nr = fma(ca, np.v[2], cs * np.v[3]);
      nu = limiter_field<LINEAR>(m0, m1, m2, nl, nr, e);
    } else {
      nu = limiter_field<LINEAR>(lane ? nm.v[1] : nm.v[0], lane ? cur[1] : cur[0], lane ? np.v[1] : np.v[0],
                                 lane ? nm.v[3] : nm.v[2], lane ? np.v[3] : np.v[2], d.eps_lim);
    }
    const double nuo = __shfl_xor_sync(0xffffffffu, nu, 1);
    const double nu0 = lane ? nuo : nu, nu1 = lane ? nu : nuo;
    if (CHAR) {
      const double A = (nu0 + nu1) * ic2;
      mod0 = A;
      mod1 = fma(u, A, 0.5 * (nu1 - nu0));
    } else {
      mod0 = nu0;
      mod1 = nu1;
    }
  } else {
    mod0 = cur[2];
    mod1 = cur[3];
  }
  const double dt = *sa.dt;
  const double c0 = lane ? mod0 : cur[0], c1 = lane ? mod1 : cur[1];
  double* o0 = lane ? sa.out[2] : sa.out[0];
  double* o1 = lane ? sa.out[3] : sa.out[1];
  if (!live) return;
  if (sa.k == 1) {
    if (sa.base) {
      (lane ? sa.base[2] : sa.base[0])[i] = c0;
      (lane ? sa.base[3] : sa.base[1])[i] = c1;
    }
    o0[i] = fma(dt, R2[0], c0);
    o1[i] = fma(dt, R2[1], c1);
  } else {
    const double a = sa.k == 2 ? 0.75 : 1.0 / 3.0;
    const double b = sa.k == 2 ? 0.25 : 2.0 / 3.0;
    o0[i] = fma(a, __ldg((lane ? sa.base[2] : sa.base[0]) + i), b * fma(dt, R2[0], c0));
    o1[i] = fma(a, __ldg((lane ? sa.base[3] : sa.base[1]) + i), b * fma(dt, R2[1], c1));
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

// alpha from its key; with dt_out, dt = CFL dx / alpha, the step that reaches t_end ending on it.
__device__ __forceinline__ void finish_alpha1d(unsigned long long key, double* alpha, double* dt_out, double cfl,
                                               double dx, const double* t_now, double t_end) {
  const double a = __longlong_as_double((long long)key);
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

__global__ void k_finish_alpha1d(const unsigned long long* amax, double* alpha, double* dt_out, double cfl,
                                 double dx, const double* t_now, double t_end) {
  finish_alpha1d(amax[0], alpha, dt_out, cfl, dx, t_now, t_end);
}

// The reduction and its finish in one launch (a solver's stages; the reset kernel and the finish launch
// of the separate form cost more than the arithmetic on the paper's 1D grids): slot[0] accumulates the
// key, slot[1] counts the blocks done; the last block to arrive finishes and clears both for the next
// launch (both are zero before the first). No block waits for another.
__global__ void __launch_bounds__(256) k_alpha_finish1d(Dev1D d, unsigned long long* slot, int* status, double* alpha,
                                                        double* dt_out, double cfl, const double* t_now, double t_end) {
  __shared__ unsigned long long wk[8];
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
  if ((threadIdx.x & 31) == 0) wk[threadIdx.x >> 5] = k;
  if (bad) atomicOr(status, bad);
  __syncthreads();
  if (threadIdx.x != 0) return;
  // one thread per block: the block's maximum, a fence, then the arrival count, so the last block to arrive
  // finds every block's maximum in slot[0]
  unsigned long long bk = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bk = max(bk, wk[w]);
  atomicMax(slot, bk);
  __threadfence();
  if (atomicAdd(slot + 1, 1ull) != (unsigned long long)gridDim.x - 1) return;
  __threadfence();
  finish_alpha1d(atomicMax(slot, 0ull), alpha, dt_out, cfl, d.dx, t_now, t_end);
  slot[0] = 0;
  slot[1] = 0;
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
void launch_alpha_finish1d(const Dev1D& d, unsigned long long* slot, int* status, double* alpha, double* dt_out,
                           double cfl, const double* t_now, double t_end, cudaStream_t st) {
  const int blocks = std::min((d.nx + 255) / 256, 152 * 4);
  k_alpha_finish1d<<<blocks, 256, 0, st>>>(d, slot, status, alpha, dt_out, cfl, t_now, t_end);
}
void launch_sweep1d(const Dev1D& d, const double* alpha, bool linear, bool chr, cudaStream_t st) {
  if (d.nx + 1 <= kLaneSweepMax) {
    const int gl = (d.nx + 1 + XL_I - 1) / XL_I;
    if (linear) { if (chr) k_sweep1d_lanes<true, true><<<gl, XL_T, 0, st>>>(d, alpha); else k_sweep1d_lanes<true, false><<<gl, XL_T, 0, st>>>(d, alpha); }
    else        { if (chr) k_sweep1d_lanes<false, true><<<gl, XL_T, 0, st>>>(d, alpha); else k_sweep1d_lanes<false, false><<<gl, XL_T, 0, st>>>(d, alpha); }
    return;
  }
  const int g = (d.nx + 1 + X1_T - 1) / X1_T;
  if (linear) { if (chr) k_sweep1d<true, true><<<g, X1_T, 0, st>>>(d, alpha); else k_sweep1d<true, false><<<g, X1_T, 0, st>>>(d, alpha); }
  else        { if (chr) k_sweep1d<false, true><<<g, X1_T, 0, st>>>(d, alpha); else k_sweep1d<false, false><<<g, X1_T, 0, st>>>(d, alpha); }
}
void launch_node1d(const Dev1D& d, const StageArgs1D& sa, int mode, bool linear, bool chr, cudaStream_t st) {
  const bool lanes = d.nx <= kLaneNodeMax;
  const int g = lanes ? (d.nx + NL_N - 1) / NL_N : (d.nx + 127) / 128;
#define L1(M, A, B) \
  (lanes ? (void)(k_node1d_lanes<M, A, B><<<g, 2 * NL_N, 0, st>>>(d, sa)) : (void)(k_node1d<M, A, B><<<g, 128, 0, st>>>(d, sa)))
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
