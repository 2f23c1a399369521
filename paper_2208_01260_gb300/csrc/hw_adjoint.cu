// Discrete adjoint of hw_rk3_step (2D, nonlinear weights, characteristic projection, limiter on or
// off) and the gauge-misfit loss with binomial checkpointing over time steps.
//
// Reverse of one RK stage (eq. RK with the right-hand side of eq. swe-form-2d-dis):
//   k_adj_node_pre   RK combination, node-local terms of the assembly (g eta, g H1, g H2 times the
//                    source differences), the adjoint of the limited derivatives
//   k_adj_sweep_x/y  adjoint of each interface's 12 values (from the two neighbouring nodes), reverse
//                    of the reconstruction (Sec. 2.1 Steps 1-2, eq. mixed) into the four stencil records
//   k_adj_records    reverse of the per-node records (fluxes, chain-rule derivatives, LF split), ghost
//                    records mapped back to the mirrored or periodic node with the parity table
//   k_adj_limiter    reverse of the HWENO limiter (Sec. 2.2) in x and y
//   k_adj_alpha_*    alpha = max(|u| + c): its adjoint goes to the first node attaining the maximum
// Scatters use FP64 atomics (sums in an unspecified order; the gradient tolerance is far above
// rounding). The parts of the source balance that depend on b only (candidates, Q' and mixed terms
// of b_x, b_y) are reversed by k_adj_static.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hwswe.h"
#include "hw_adjoint.cuh"
#include "hw_halo.h"
#include "hw_internal.h"

namespace hw {

struct AdjDev {
  Dev2D d;                // stage input state, static planes, grid constants
  const double* alpha;    // alpha of this stage [2]
  int k;
  double dt, a, b;
  int limiter;
  const double* lout[9];  // adjoint of the stage output
  double* lin[9];         // adjoint of the stage input (written)
  double* lbase[9];       // adjoint of the step base (accumulated over stages 3, 2; consumed at stage 1)
  double* lR[9];          // adjoint of the right-hand side (scratch)
  double* lmod[6];        // adjoint of the limited derivatives (scratch)
  double* lrecx[NREC];    // record adjoints, x: rows of nx + 4 (raw index -2 .. nx+1)
  double* lrecy[NREC];    // record adjoints, y: ny + 4 rows of nx
  double* lstat[3];       // adjoint of b, dx b_x, dy b_y (direct dependences), accumulated
  double* lqbx[6];
  double* lqby[6];
  double* lsv[2];
  double* lsq[2];
  double* lalpha;         // [2], accumulated within the stage
  const double* dbx[3];   // forward 2 bhat (x-interfaces) of this stage
  const double* dby[3];   // forward 2 bhat (y-interfaces)
  const double* fax;      // forward first component of 2 Fhat (x-interfaces) of this stage
  const double* fay;      // forward first component of 2 Fhat (y-interfaces)
  int* argmax;            // [2]
};

// atomically add parity-mapped adjoints of a (possibly ghost) node's 12 entries to the real node
__device__ __forceinline__ void scatter_node(const AdjDev& A, int i, int j, const double ln[12], bool with_state,
                                             bool with_stat) {
  bool fx, fy;
  const int ii = map_index(i, A.d.nx, A.d.bc_x, fx);
  const int jj = map_index(j, A.d.ny, A.d.bc_y, fy);
  const size_t o = (size_t)jj * A.d.nx + ii;
  if (with_state)
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      double x = ln[q];
      if (fx) x *= par_x2d(q);
      if (fy) x *= par_y2d(q);
      if (x != 0.0) atomicAdd(A.lin[q] + o, x);
    }
  if (with_stat)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double x = ln[9 + q];
      if (fx) x *= par_x2d(9 + q);
      if (fy) x *= par_y2d(9 + q);
      if (x != 0.0) atomicAdd(A.lstat[q] + o, x);
    }
}

__device__ __forceinline__ double block_sum(double v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  return v;  // lane 0 of each warp holds the warp sum
}

// ---- 1. node pre-pass ----
__global__ void __launch_bounds__(256) k_adj_node_pre(AdjDev A) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  const Dev2D& d = A.d;
  if (i >= d.nx || j >= d.ny) return;
  const size_t o = (size_t)j * d.nx + i;
  double lc[9], lR[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const double lo = A.lout[q][o];
    if (A.k == 1) {
      lc[q] = lo + A.lbase[q][o];
      lR[q] = A.dt * lo;
    } else {
      lc[q] = A.b * lo;
      lR[q] = A.b * A.dt * lo;
      A.lbase[q][o] += A.a * lo;
    }
  }
  const double eta = d.S[0][o], g = d.g, ge = g * eta;
  // source differences db_c = [b~^]_x/dx + [b-^]_y/dy from the forward interface values
  double db[3];
  const size_t ox = (size_t)j * (d.nx + 1) + i, oy = (size_t)j * d.nx + i;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    db[c] = fma(d.c_bx, A.dbx[c][ox + 1] - A.dbx[c][ox], d.c_by * (A.dby[c][oy + d.nx] - A.dby[c][oy]));
  double leta = 0.0, lH1 = 0.0, lH2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    leta -= g * db[c] * lR[c];
    lH1 -= g * db[c] * lR[3 + c];
    lH2 -= g * db[c] * lR[6 + c];
  }
#pragma unroll
  for (int c = 1; c < 3; ++c) {
    const double sv = d.sv[c - 1][o], sq = d.sq[c - 1][o];
    leta -= g * (sv * lR[3 + c] + sq * lR[6 + c]);
    A.lsv[c - 1][o] -= ge * lR[3 + c];
    A.lsq[c - 1][o] -= ge * lR[6 + c];
  }
  A.lin[0][o] = lc[0] + leta;
  A.lin[1][o] = lc[1];
  A.lin[2][o] = lc[2];
  if (A.limiter) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      A.lmod[q][o] = lc[3 + q];
      A.lin[3 + q][o] = 0.0;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) A.lin[3 + q][o] = lc[3 + q];
  }
  A.lin[3][o] += lH1;
  A.lin[6][o] += lH2;
#pragma unroll
  for (int q = 0; q < 9; ++q) A.lR[q][o] = lR[q];
}

// adjoint of the 12 values of the x-interface k of row j (from nodes k-1 and k)
__device__ __forceinline__ void interface_adjoint_x(const AdjDev& A, int k, int j, double lX[12]) {
  const Dev2D& d = A.d;
  for (int q = 0; q < 12; ++q) lX[q] = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int p = side == 0 ? k - 1 : k;  // node seeing k as its right (side 0) or left (side 1) interface
    if (p < 0 || p >= d.nx) continue;
    const double sgn = side == 0 ? -1.0 : 1.0;
    const size_t o = (size_t)j * d.nx + p;
    const double g = d.g, ge = g * d.S[0][o], gH1 = g * d.S[3][o], gH2 = g * d.S[6][o];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double lu = A.lR[c][o], lv = A.lR[3 + c][o], lq = A.lR[6 + c][o];
      lX[c] += sgn * d.c_bx * lu;
      lX[3 + c] += sgn * d.c_bx * (ge * lu + gH1 * lv + gH2 * lq);
      lX[6 + c] += sgn * d.c_gx * lv;
      lX[9 + c] += sgn * d.c_mx * lq;
    }
  }
}

__device__ __forceinline__ void interface_adjoint_y(const AdjDev& A, int i, int k, double lY[12]) {
  const Dev2D& d = A.d;
  for (int q = 0; q < 12; ++q) lY[q] = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int p = side == 0 ? k - 1 : k;
    if (p < 0 || p >= d.ny) continue;
    const double sgn = side == 0 ? -1.0 : 1.0;
    const size_t o = (size_t)p * d.nx + i;
    const double g = d.g, ge = g * d.S[0][o], gH1 = g * d.S[3][o], gH2 = g * d.S[6][o];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double lu = A.lR[c][o], lv = A.lR[3 + c][o], lq = A.lR[6 + c][o];
      lY[c] += sgn * d.c_by * lu;
      lY[3 + c] += sgn * d.c_by * (ge * lu + gH1 * lv + gH2 * lq);
      lY[6 + c] += sgn * d.c_gy * lq;  // Psi2 hat feeds the Q equations
      lY[9 + c] += sgn * d.c_my * lv;  // mixed Phi2 hat feeds the V equations
    }
  }
}

// ---- 2. x-interfaces (a block of AX_T threads: AX_I = AX_T - 3 consecutive interfaces of one row and
// their AX_N = AX_T node records, one per thread) ----
// The four record adjoints of each interface collect in a shared-memory slab; after the block has
// finished, each record sums its (up to) four contributions, so only the three records a block shares
// with each neighbour are added atomically.
constexpr int AX_T = 64;
constexpr int AX_I = AX_T - 3;
constexpr int AX_N = AX_T;

__global__ void __launch_bounds__(AX_T) k_adj_sweep_x(AdjDev A) {
  __shared__ double sm[NREC * AX_N];
  __shared__ double slab[4 * NREC * AX_T];
  const Dev2D& d = A.d;
  const int j = blockIdx.y, k0 = blockIdx.x * AX_I;
  const double ax = A.alpha[0];
  const int t = threadIdx.x;
  for (int u = t; u < AX_N; u += AX_T) {
    const int i = k0 - 2 + u;
    if (i > d.nx + 1) break;
    Node12 n;
    load_node(d, i, j, n);
    double rec[NREC];
    node_record<0>(n, d.g, ax, rec);
#pragma unroll
    for (int f = 0; f < NREC; ++f) sm[f * AX_N + u] = rec[f];
  }
  __syncthreads();
  const int k = k0 + t;
  if (t < AX_I && k <= d.nx) {
    const size_t o = (size_t)j * (d.nx + 1) + k;
    double qb[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) qb[q] = d.qbx[q][o];
    double lX[12];
    interface_adjoint_x(A, k, j, lX);
    double lqb[6] = {0, 0, 0, 0, 0, 0};
    interface_values_rev<0>(sm + t, 1, AX_N, qb, A.fax[o], A.dbx[0][o], d.g, d.eps_w, lX,
                            SlabAcc{slab + t, AX_T}, lqb);
#pragma unroll
    for (int q = 0; q < 6; ++q) A.lqbx[q][o] += lqb[q];
  } else {
    for (int e = 0; e < 4 * NREC; ++e) slab[e * AX_T + t] = 0.0;  // no interface (tile or row end)
  }
  __syncthreads();
  const size_t row = (size_t)j * (d.nx + 4);
  for (int u = t; u < AX_N; u += AX_T) {
    const int r = k0 - 2 + u;  // raw record index, -2 .. nx+1
    if (r > d.nx + 1) break;
    const bool shared_slot = u < 3 || u >= AX_I;
    for (int f = 0; f < NREC; ++f) {
      double acc = 0.0;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int tt = u - s;
        if (tt >= 0 && tt < AX_T) acc += slab[(s * NREC + f) * AX_T + tt];
      }
      double* dst = A.lrecx[f] + row + (r + 2);
      if (shared_slot) {
        if (acc != 0.0) atomicAdd(dst, acc);
      } else {
        *dst = acc;
      }
    }
  }
}

// ---- 2'. y-interfaces (a block: AY_R interface rows of 32 columns; records of AY_R + 3 node rows) ----
constexpr int AY_R = 8;
constexpr int AY_NR = AY_R + 3;
constexpr int AY_T = 32 * AY_R;
constexpr size_t AY_SMEM = (size_t)(NREC * AY_NR * 32 + 4 * NREC * AY_T) * sizeof(double);

__global__ void __launch_bounds__(AY_T) k_adj_sweep_y(AdjDev A) {
  extern __shared__ double ysm[];
  double* recs = ysm;                      // [NREC][AY_NR][32]
  double* slab = ysm + NREC * AY_NR * 32;  // [4][NREC][AY_T]
  const Dev2D& d = A.d;
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * AY_R;
  const int tid = threadIdx.x, c = tid & 31, ty = tid >> 5;
  const double ay = A.alpha[1];
  for (int idx = tid; idx < AY_NR * 32; idx += AY_T) {
    const int u = idx >> 5, cc = idx & 31;
    const int i = i0 + cc, r = k0 - 2 + u;
    if (i >= d.nx || r > d.ny + 1) continue;
    Node12 n;
    load_node(d, i, r, n);
    double rec[NREC];
    node_record<1>(n, d.g, ay, rec);
#pragma unroll
    for (int f = 0; f < NREC; ++f) recs[(f * AY_NR + u) * 32 + cc] = rec[f];
  }
  __syncthreads();
  const int i = i0 + c, k = k0 + ty;
  if (i < d.nx && k <= d.ny) {
    const size_t o = (size_t)k * d.nx + i;
    double qb[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) qb[q] = d.qby[q][o];
    double lY[12];
    interface_adjoint_y(A, i, k, lY);
    double lqb[6] = {0, 0, 0, 0, 0, 0};
    const double* r0 = recs + ty * 32 + c;
    interface_values_rev<1>(r0, 32, AY_NR * 32, qb, A.fay[o], A.dby[0][o], d.g, d.eps_w, lY,
                            SlabAcc{slab + tid, AY_T}, lqb);
#pragma unroll
    for (int q = 0; q < 6; ++q) A.lqby[q][o] += lqb[q];
  } else {
    for (int e = 0; e < 4 * NREC; ++e) slab[e * AY_T + tid] = 0.0;  // past the grid's edge
  }
  __syncthreads();
  for (int idx = tid; idx < AY_NR * 32; idx += AY_T) {
    const int u = idx >> 5, cc = idx & 31;
    const int ii = i0 + cc, r = k0 - 2 + u;  // raw record row, -2 .. ny+1
    if (ii >= d.nx || r > d.ny + 1) continue;
    const bool shared_row = u < 3 || u >= AY_R;
    const size_t pos = (size_t)(r + 2) * d.nx + ii;
    for (int f = 0; f < NREC; ++f) {
      double acc = 0.0;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int uu = u - s;
        if (uu >= 0 && uu < AY_R) acc += slab[(s * NREC + f) * AY_T + uu * 32 + cc];
      }
      double* dst = A.lrecy[f] + pos;
      if (shared_row) {
        if (acc != 0.0) atomicAdd(dst, acc);
      } else {
        *dst = acc;
      }
    }
  }
}

// ---- 3. records: raw x-records (r = -2..nx+1, row j) and raw y-records (column i, r = -2..ny+1) ----
__global__ void __launch_bounds__(256) k_adj_records(AdjDev A) {
  const Dev2D& d = A.d;
  const int nxr = (d.nx + 4) * d.ny, nyr = d.nx * (d.ny + 4);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double la = 0.0;
  int dir = -1;
  if (tid < nxr) {
    dir = 0;
    const int j = tid / (d.nx + 4), r = tid - j * (d.nx + 4) - 2;
    double lrec[NREC];
    bool any = false;
#pragma unroll
    for (int f = 0; f < NREC; ++f) {
      lrec[f] = A.lrecx[f][tid];
      any |= lrec[f] != 0.0;
    }
    if (any) {
      Node12 n;
      load_node(d, r, j, n);
      double ln[12] = {};
      la = node_record_rev<0>(n, d.g, A.alpha[0], lrec, ln);
      scatter_node(A, r, j, ln, true, true);
    }
  } else if (tid < nxr + nyr) {
    dir = 1;
    const int u = tid - nxr;
    const int rr = u / d.nx, i = u - rr * d.nx, r = rr - 2;
    double lrec[NREC];
    bool any = false;
#pragma unroll
    for (int f = 0; f < NREC; ++f) {
      lrec[f] = A.lrecy[f][u];
      any |= lrec[f] != 0.0;
    }
    if (any) {
      Node12 n;
      load_node(d, i, r, n);
      double ln[12] = {};
      la = node_record_rev<1>(n, d.g, A.alpha[1], lrec, ln);
      scatter_node(A, i, r, ln, true, true);
    }
  }
  // alpha adjoints: warps may straddle the x/y boundary, so reduce per direction
  const double lx = block_sum(dir == 0 ? la : 0.0), ly = block_sum(dir == 1 ? la : 0.0);
  if ((threadIdx.x & 31) == 0) {
    if (lx != 0.0) atomicAdd(A.lalpha, lx);
    if (ly != 0.0) atomicAdd(A.lalpha + 1, ly);
  }
}

// ---- 4. limiter ----
__global__ void __launch_bounds__(256) k_adj_limiter(AdjDev A) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  const Dev2D& d = A.d;
  if (i >= d.nx || j >= d.ny) return;
  const size_t o = (size_t)j * d.nx + i;
  double cur[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) cur[q] = d.S[q][o];
  const double g = d.g;
  const double b0 = d.stat[0][o];
  const double h = cur[0] - b0, gh = g * h, rh = fast_rcp(h);
  const double u = cur[1] * rh, v = cur[2] * rh;
  const double rs = fast_rsqrt(gh), c = gh * rs, ic2 = 0.5 * rs;
  double lu = 0.0, lv = 0.0, lc = 0.0, lic2 = 0.0, lgh = 0.0;
  double l0[12] = {};
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    double lo[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) lo[q] = A.lmod[3 * dir + q][o];
    if (lo[0] == 0.0 && lo[1] == 0.0 && lo[2] == 0.0) continue;
    Node12 nm, np;
    const int im = dir == 0 ? i - 1 : i, jm = dir == 0 ? j : j - 1;
    const int ip = dir == 0 ? i + 1 : i, jp = dir == 0 ? j : j + 1;
    load_node(d, im, jm, nm);
    load_node(d, ip, jp, np);
    const int qd = dir == 0 ? 3 : 6;
    double lUm[3] = {}, lU0[3] = {}, lUp[3] = {}, lDm[3] = {}, lDp[3] = {};
    if (dir == 0)
      limit_dir_rev<0>(nm.v, cur, np.v, nm.v + qd, np.v + qd, u, v, c, ic2, gh, d.eps_lim, lo, lUm, lU0, lUp, lDm, lDp,
                       lu, lv, lc, lic2, lgh);
    else
      limit_dir_rev<1>(nm.v, cur, np.v, nm.v + qd, np.v + qd, u, v, c, ic2, gh, d.eps_lim, lo, lUm, lU0, lUp, lDm, lDp,
                       lu, lv, lc, lic2, lgh);
    double lm12[12] = {}, lp12[12] = {};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      lm12[q] = lUm[q];
      lm12[qd + q] = lDm[q];
      lp12[q] = lUp[q];
      lp12[qd + q] = lDp[q];
      l0[q] += lU0[q];
    }
    scatter_node(A, im, jm, lm12, true, false);
    scatter_node(A, ip, jp, lp12, true, false);
    asm volatile("" ::: "memory");  // one direction's data live at a time
  }
  // node eigen quantities: u = m/h, v = w/h, c = gh rs, ic2 = rs/2, rs = gh^-1/2, gh = g h, h = eta - b
  const double lrs = 0.5 * lic2 + gh * lc;
  const double lght = lgh + rs * lc - 0.5 * rs * rs * rs * lrs;
  const double lh = g * lght - rh * rh * (cur[1] * lu + cur[2] * lv);
  l0[0] += lh;
  l0[1] += rh * lu;
  l0[2] += rh * lv;
  l0[9] = -lh;
  scatter_node(A, i, j, l0, true, true);
}

// ---- 5. alpha: the first node attaining the maximum receives the adjoint ----
__global__ void __launch_bounds__(256) k_adj_alpha_find(AdjDev A) {
  const Dev2D& d = A.d;
  const int n = d.nx * d.ny;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    const double h = d.S[0][o] - d.stat[0][o];
    const double rh = fast_rcp(h), gh = d.g * h, c = gh * fast_rsqrt(gh);
    const double ax = dabs(d.S[1][o] * rh) + c, ay = dabs(d.S[2][o] * rh) + c;
    // the forward reduction may round the last bit differently (FMA contraction): 4e-16 relative window
    if (fabs(ax - A.alpha[0]) <= 4e-16 * A.alpha[0]) atomicMin(A.argmax, o);
    if (fabs(ay - A.alpha[1]) <= 4e-16 * A.alpha[1]) atomicMin(A.argmax + 1, o);
  }
}

__global__ void k_adj_alpha_apply(AdjDev A) {
  const Dev2D& d = A.d;
  for (int dir = 0; dir < 2; ++dir) {
    const int o = A.argmax[dir];
    const double la = A.lalpha[dir];
    if (o == INT_MAX || la == 0.0) continue;
    const double h = d.S[0][o] - d.stat[0][o];
    const double rh = fast_rcp(h), gh = d.g * h, rs = fast_rsqrt(gh), c = gh * rs;
    const double mom = d.S[1 + dir][o];
    const double un = mom * rh;
    const double sg = un < 0.0 ? -1.0 : 1.0;  // d|x| = dx at x = 0 (same convention as the oracle)
    // alpha = |mom/h| + sqrt(g h)
    const double lmom = la * sg * rh;
    const double lh = la * (-sg * un * rh + 0.5 * d.g * rs);
    (void)c;
    atomicAdd(A.lin[0] + o, lh);
    atomicAdd(A.lin[1 + dir] + o, lmom);
    atomicAdd(A.lstat[0] + o, -lh);
  }
}

// ---- static terms (once per call): candidates, Q' of (b, b_x) and (b, b_y), mixed terms ----
struct StatAdj {
  Dev2D d;
  const double* lqbx[6];
  const double* lqby[6];
  const double* lsv[2];
  const double* lsq[2];
  double* lb;   // adjoint of b (physical)
  double* lbx;  // of b_x
  double* lby;  // of b_y
};

__device__ __forceinline__ void add_b(const StatAdj& S, int q, int i, int j, double x) {
  if (x == 0.0) return;
  bool fx, fy;
  const int ii = map_index(i, S.d.nx, S.d.bc_x, fx);
  const int jj = map_index(j, S.d.ny, S.d.bc_y, fy);
  if (fx && q == 1) x = -x;
  if (fy && q == 2) x = -x;
  double* dst = q == 0 ? S.lb : (q == 1 ? S.lbx : S.lby);
  atomicAdd(dst + (size_t)jj * S.d.nx + ii, x);
}

// candidates q_1..q_3 of (b, s) with s = spacing * b_s, '+' side from nodes 0,1,2 and mirrored '-' side
__device__ __forceinline__ void cands_rev(const double lq[6], double lb[4], double ls[4]) {
  // + : q1 = (b0+b1)/2 + (s0 + 5 s1)/6, q2 = (b1+b2)/2 + (s1 - s2)/6, q3 = (b0 + 10 b1 + b2)/12 + s1/2
  lb[0] += 0.5 * lq[0] + lq[2] / 12.0;
  lb[1] += 0.5 * lq[0] + 0.5 * lq[1] + 10.0 * lq[2] / 12.0;
  lb[2] += 0.5 * lq[1] + lq[2] / 12.0;
  ls[0] += lq[0] / 6.0;
  ls[1] += 5.0 * lq[0] / 6.0 + lq[1] / 6.0 + 0.5 * lq[2];
  ls[2] += -lq[1] / 6.0;
  // - : nodes (3, 2, 1) with s negated
  lb[3] += 0.5 * lq[3] + lq[5] / 12.0;
  lb[2] += 0.5 * lq[3] + 0.5 * lq[4] + 10.0 * lq[5] / 12.0;
  lb[1] += 0.5 * lq[4] + lq[5] / 12.0;
  ls[3] -= lq[3] / 6.0;
  ls[2] -= 5.0 * lq[3] / 6.0 + lq[4] / 6.0 + 0.5 * lq[5];
  ls[1] -= -lq[4] / 6.0;
}

// adjoint of qprime_sum(b0..b3, s0..s3, del) = ((b0-8b1+7b2) + (-7b1+8b2-b3))/(8 del) + ((s0-2s1-5s2) + (-5s1-2s2+s3))/24
__device__ __forceinline__ void qps_rev(double l, double del, double lb[4], double ls[4]) {
  const double cb = l / (8.0 * del), cs = l / 24.0;
  lb[0] += cb; lb[1] -= 15.0 * cb; lb[2] += 15.0 * cb; lb[3] -= cb;
  ls[0] += cs; ls[1] -= 7.0 * cs; ls[2] -= 7.0 * cs; ls[3] += cs;
}

__global__ void k_adj_static(StatAdj S) {
  const Dev2D& d = S.d;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  // x-interface k = i of row j: candidates (b, dx b_x); Q' of (b, b_x) from sv[0]; mixed b_y from sq[0]
  if (j < d.ny && i <= d.nx) {
    const int k = i;
    const size_t o = (size_t)j * (d.nx + 1) + k;
    double lq[6];
    for (int q = 0; q < 6; ++q) lq[q] = S.lqbx[q][o];
    double lb[4] = {}, ls[4] = {}, lby[4] = {};
    cands_rev(lq, lb, ls);
    for (int t = 0; t < 4; ++t) ls[t] *= d.dx;  // s = dx b_x
    // B1x(k) enters sv[0] of node k-1 with + and of node k with -
    double lB1 = 0.0, lB2 = 0.0;
    if (k - 1 >= 0 && k - 1 < d.nx) {
      lB1 += S.lsv[0][(size_t)j * d.nx + k - 1];
      lB2 += S.lsq[0][(size_t)j * d.nx + k - 1] * d.dy * d.inv_dx;
    }
    if (k < d.nx) {
      lB1 -= S.lsv[0][(size_t)j * d.nx + k];
      lB2 -= S.lsq[0][(size_t)j * d.nx + k] * d.dy * d.inv_dx;
    }
    qps_rev(lB1, d.dx, lb, ls);
    // mixed (-x0 + 7 x1 + 7 x2 - x3)/12 of b_y
    lby[0] -= lB2 / 12.0; lby[1] += 7.0 * lB2 / 12.0; lby[2] += 7.0 * lB2 / 12.0; lby[3] -= lB2 / 12.0;
    for (int t = 0; t < 4; ++t) {
      add_b(S, 0, k - 2 + t, j, lb[t]);
      add_b(S, 1, k - 2 + t, j, ls[t]);
      add_b(S, 2, k - 2 + t, j, lby[t]);
    }
  }
  // y-interface k = j of column i: candidates (b, dy b_y); Q' of (b, b_y) from sq[1]; mixed b_x from sv[1]
  if (i < d.nx && j <= d.ny) {
    const int k = j;
    const size_t o = (size_t)k * d.nx + i;
    double lq[6];
    for (int q = 0; q < 6; ++q) lq[q] = S.lqby[q][o];
    double lb[4] = {}, ls[4] = {}, lbx[4] = {};
    cands_rev(lq, lb, ls);
    for (int t = 0; t < 4; ++t) ls[t] *= d.dy;
    double lB2 = 0.0, lB1 = 0.0;
    if (k - 1 >= 0 && k - 1 < d.ny) {
      lB2 += S.lsq[1][(size_t)(k - 1) * d.nx + i];
      lB1 += S.lsv[1][(size_t)(k - 1) * d.nx + i] * d.dx * d.inv_dy;
    }
    if (k < d.ny) {
      lB2 -= S.lsq[1][(size_t)k * d.nx + i];
      lB1 -= S.lsv[1][(size_t)k * d.nx + i] * d.dx * d.inv_dy;
    }
    qps_rev(lB2, d.dy, lb, ls);
    lbx[0] -= lB1 / 12.0; lbx[1] += 7.0 * lB1 / 12.0; lbx[2] += 7.0 * lB1 / 12.0; lbx[3] -= lB1 / 12.0;
    for (int t = 0; t < 4; ++t) {
      add_b(S, 0, i, k - 2 + t, lb[t]);
      add_b(S, 2, i, k - 2 + t, ls[t]);
      add_b(S, 1, i, k - 2 + t, lbx[t]);
    }
  }
}

// user gradient (equilibrium layout, physical derivatives) <-> internal adjoint (scaled derivatives)
__global__ void k_adj_convert(int n, double dx, double dy, Ptr9 src, Ptr9 dst, int to_internal) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const double sc = q < 3 ? 1.0 : (q < 6 ? dx : dy);
      // eta_x = H1'/dx: dL/dH1' = dL/deta_x / dx, and back
      dst.p[q][o] = to_internal ? src.p[q][o] / sc : src.p[q][o] * sc;
    }
  }
}

// lb, lbx, lby (physical) += direct static adjoints (b, dx b_x, dy b_y)
__global__ void k_adj_static_direct(int n, double dx, double dy, const double* l0, const double* l1, const double* l2,
                                    double* lb, double* lbx, double* lby) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    lb[o] += l0[o];
    lbx[o] += dx * l1[o];
    lby[o] += dy * l2[o];
  }
}

__global__ void k_gather_eta(const double* eta, const int* idx, int ng, double* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng) out[g] = eta[idx[g]];
}

__global__ void k_loss_seed(const double* gval, const double* obs, const int* idx, int ng, double* leta) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng) atomicAdd(leta + idx[g], 2.0 * (gval[g] - obs[g]));
}

// ---- block decomposition: gauges by (local node, global slot), alpha over the blocks ----
__global__ void k_gather_eta_map(const double* eta, const int* idx, const int* slot, int n, double* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[slot[g]] = eta[idx[g]];
}

__global__ void k_loss_seed_map(const double* gval, const double* obs, const int* idx, const int* slot, int n,
                                double* leta) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) atomicAdd(leta + idx[g], 2.0 * (gval[slot[g]] - obs[slot[g]]));
}

// out[d] = maximum over the rows of the blocks' alpha keys (rows[2 p + d])
__global__ void k_keys_max(const unsigned long long* rows, int np, unsigned long long* out) {
  const int d = threadIdx.x;
  if (d >= 2) return;
  unsigned long long m = 0;
  for (int p = 0; p < np; ++p) m = max(m, rows[2 * p + d]);
  out[d] = m;
}

// The first node of the global grid (index gj gnx + gi) attaining the stage's alpha, over the block's own
// nodes (extended indices [2, nxl + 2) x [2, nyl + 2), block origin (i0, j0)); the minimum over the
// blocks is the undecomposed grid's first maximising node.
__global__ void __launch_bounds__(256) k_adj_alpha_find_block(AdjDev A, int nxl, int nyl, int i0, int j0, int gnx) {
  const Dev2D& d = A.d;
  const int n = nxl * nyl;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int li = t % nxl, lj = t / nxl;
    const size_t o = (size_t)(lj + 2) * d.nx + (li + 2);
    const double h = d.S[0][o] - d.stat[0][o];
    const double rh = fast_rcp(h), gh = d.g * h, c = gh * fast_rsqrt(gh);
    const double ax = dabs(d.S[1][o] * rh) + c, ay = dabs(d.S[2][o] * rh) + c;
    const int gidx = (j0 + lj) * gnx + (i0 + li);
    if (fabs(ax - A.alpha[0]) <= 4e-16 * A.alpha[0]) atomicMin(A.argmax, gidx);
    if (fabs(ay - A.alpha[1]) <= 4e-16 * A.alpha[1]) atomicMin(A.argmax + 1, gidx);
  }
}

// The alpha adjoint of all blocks (A.lalpha, summed) applied by the block that owns that node.
__global__ void k_adj_alpha_apply_block(AdjDev A, int nxl, int nyl, int i0, int j0, int gnx) {
  const Dev2D& d = A.d;
  for (int dir = 0; dir < 2; ++dir) {
    const int gidx = A.argmax[dir];
    const double la = A.lalpha[dir];
    if (gidx == INT_MAX || la == 0.0) continue;
    const int gi = gidx % gnx - i0, gj = gidx / gnx - j0;
    if (gi < 0 || gi >= nxl || gj < 0 || gj >= nyl) continue;
    const size_t o = (size_t)(gj + 2) * d.nx + (gi + 2);
    const double h = d.S[0][o] - d.stat[0][o];
    const double rh = fast_rcp(h), gh = d.g * h, rs = fast_rsqrt(gh);
    const double un = d.S[1 + dir][o] * rh;
    const double sg = un < 0.0 ? -1.0 : 1.0;
    const double lmom = la * sg * rh;
    const double lh = la * (-sg * un * rh + 0.5 * d.g * rs);
    atomicAdd(A.lin[0] + o, lh);
    atomicAdd(A.lin[1 + dir] + o, lmom);
    atomicAdd(A.lstat[0] + o, -lh);
  }
}

}  // namespace hw

// =============================================================================================
// Host side: one step's reverse, the loss, checkpointing
// =============================================================================================
namespace {

int afail(int code, const std::string& m) { return hw::set_last_error(code, m.c_str()); }
#define ACUDA(call)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return afail(HW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct AdjBuffers {
  hw_solver* owner = nullptr;
  size_t n = 0;
  int nx = 0, ny = 0;
  std::vector<void*> allocs;
  double* stage_in[3][9] = {};
  double* stage_out[9] = {};
  double* alpha_st = nullptr;  // [3][2]
  double* dbx[3][3] = {};
  double* dby[3][3] = {};
  double* fx[3] = {};  // first component of 2 Fhat per stage, x- and y-interfaces
  double* fy[3] = {};
  double* lam[2][9] = {};
  double* lbase[9] = {};
  double* lR[9] = {};
  double* lmod[6] = {};
  double* lrecx[hw::NREC] = {};
  double* lrecy[hw::NREC] = {};
  double* lstat[3] = {};
  double* lqbx[6] = {};
  double* lqby[6] = {};
  double* lsv[2] = {};
  double* lsq[2] = {};
  double* lalpha = nullptr;
  int* argmax = nullptr;
  double* lstatic_phys[3] = {};
  unsigned long long* amax = nullptr;  // the forward alpha reduction's keys and scratch (kAlpha2dScratch)
};

std::mutex g_adj_mu;
std::vector<AdjBuffers*> g_adj;  // one per live solver that used the adjoint (released by hw_destroy)

// Zeroed on the solver's stream: the static adjoints accumulate into their buffers from the first use on
// (each use clears them when it is done), so they must start at zero, not at whatever the memory held.
int adj_alloc(AdjBuffers* B, double** p, size_t cnt, cudaStream_t st) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, cnt * sizeof(double));
  if (e != cudaSuccess) return afail(HW_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  B->allocs.push_back(q);
  *p = (double*)q;
  e = cudaMemsetAsync(q, 0, cnt * sizeof(double), st);
  if (e != cudaSuccess) return afail(HW_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  return HW_OK;
}

int get_buffers(hw_solver* s, const hw::SolverView& v, AdjBuffers** out) {
  std::lock_guard<std::mutex> lk(g_adj_mu);
  for (AdjBuffers* B : g_adj)
    if (B->owner == s) {
      if (B->n != v.n || B->nx != v.d2->nx || B->ny != v.d2->ny)
        return afail(HW_ERR_STATE, "adjoint: working buffers do not match the solver's grid");
      *out = B;
      return HW_OK;
    }
  AdjBuffers* B = new AdjBuffers();
  B->owner = s;
  B->n = v.n;
  B->nx = v.d2->nx;
  B->ny = v.d2->ny;
  const size_t n = v.n, nxi = (size_t)(B->nx + 1) * B->ny, nyi = (size_t)B->nx * (B->ny + 1);
  int rc = HW_OK;
  auto A = [&](double** p, size_t c) { if (rc == HW_OK) rc = adj_alloc(B, p, c, v.stream); };
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 9; ++q) A(&B->stage_in[k][q], n);
  for (int q = 0; q < 9; ++q) { A(&B->stage_out[q], n); A(&B->lam[0][q], n); A(&B->lam[1][q], n); A(&B->lbase[q], n); A(&B->lR[q], n); }
  A(&B->alpha_st, 8);
  for (int k = 0; k < 3; ++k) {
    for (int c = 0; c < 3; ++c) { A(&B->dbx[k][c], nxi); A(&B->dby[k][c], nyi); }
    A(&B->fx[k], nxi);
    A(&B->fy[k], nyi);
  }
  for (int q = 0; q < 6; ++q) { A(&B->lmod[q], n); A(&B->lqbx[q], nxi); A(&B->lqby[q], nyi); }
  for (int f = 0; f < hw::NREC; ++f) { A(&B->lrecx[f], (size_t)(B->nx + 4) * B->ny); A(&B->lrecy[f], (size_t)B->nx * (B->ny + 4)); }
  for (int q = 0; q < 3; ++q) { A(&B->lstat[q], n); A(&B->lstatic_phys[q], n); }
  for (int q = 0; q < 2; ++q) { A(&B->lsv[q], n); A(&B->lsq[q], n); }
  double* misc = nullptr;
  A(&misc, 8);
  A(reinterpret_cast<double**>(&B->amax), hw::kAlpha2dScratch);
  if (rc != HW_OK) {
    for (void* p : B->allocs) cudaFree(p);
    delete B;
    return rc;
  }
  B->lalpha = misc;
  B->argmax = (int*)(misc + 4);
  g_adj.push_back(B);
  *out = B;
  return HW_OK;
}

}  // namespace

void hw::adjoint_release(hw_solver* s) {
  std::lock_guard<std::mutex> lk(g_adj_mu);
  for (size_t k = 0; k < g_adj.size(); ++k)
    if (g_adj[k]->owner == s) {
      for (void* p : g_adj[k]->allocs) cudaFree(p);
      delete g_adj[k];
      g_adj.erase(g_adj.begin() + k);
      return;
    }
}

namespace {

// The gauge misfit sum over (step, gauge) of (eta - obs)^2, in that order: one function, so that every
// entry point (single grid, blocks on one GPU, blocks over processes) rounds it alike.
double misfit_loss(const double* g, const double* obs, size_t n) {
  double L = 0.0;
  for (size_t q = 0; q < n; ++q) L += (g[q] - obs[q]) * (g[q] - obs[q]);
  return L;
}

int zero_planes(double* const* p, int count, size_t n, cudaStream_t st) {
  for (int q = 0; q < count; ++q) ACUDA(cudaMemsetAsync(p[q], 0, n * sizeof(double), st));
  return HW_OK;
}

// What the reverse of one step reads: every stage's input, the step's output, the stage alphas, the
// stages' source interface values 2 bhat and the first components of their fluxes 2 Fhat. Points into AdjBuffers (one step, recomputed from a
// checkpoint) or into a whole-run tape.
struct StepTape {
  double* in[3][9];
  double* out[9];
  double* alpha;  // [3][2]
  double* dbx[3][3];
  double* dby[3][3];
  double* fx[3];
  double* fy[3];
};

StepTape buffer_tape(AdjBuffers* B) {
  StepTape T{};
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 9; ++q) T.in[k][q] = B->stage_in[k][q];
  for (int q = 0; q < 9; ++q) T.out[q] = B->stage_out[q];
  T.alpha = B->alpha_st;
  for (int k = 0; k < 3; ++k) {
    for (int c = 0; c < 3; ++c) { T.dbx[k][c] = B->dbx[k][c]; T.dby[k][c] = B->dby[k][c]; }
    T.fx[k] = B->fx[k];
    T.fy[k] = B->fy[k];
  }
  return T;
}

// One forward step from T.in[0] recording into T (the sweeps write the source interface values straight
// into the tape); the solver's state is not touched.
int forward_record(const hw::SolverView& v, AdjBuffers* B, const StepTape& T, double dt) {
  cudaStream_t st = v.stream;
  ACUDA(cudaMemcpyAsync(v.dt, &dt, sizeof(double), cudaMemcpyHostToDevice, st));
  hw::Dev2D d = *v.d2;
  const bool lin = false, chr = true;
  for (int k = 1; k <= 3; ++k) {
    for (int q = 0; q < 9; ++q) d.S[q] = T.in[k - 1][q];
    for (int c = 0; c < 3; ++c) { d.X[3 + c] = T.dbx[k - 1][c]; d.Y[3 + c] = T.dby[k - 1][c]; }
    d.X[0] = T.fx[k - 1];
    d.Y[0] = T.fy[k - 1];
    hw::launch_alpha2d(d, B->amax, (int*)(B->lalpha + 2), st);
    hw::launch_finish_alpha2d(d, B->amax, T.alpha + 2 * (k - 1), nullptr, v.params->cfl,
                              nullptr, -1.0, st);
    hw::launch_sweep_x2d(d, T.alpha + 2 * (k - 1), lin, chr, st);
    hw::launch_sweep_y2d(d, T.alpha + 2 * (k - 1), lin, chr, st);
    hw::StageArgs sa{};
    sa.k = k;
    sa.limiter = v.params->limiter;
    sa.dt = v.dt;
    for (int q = 0; q < 9; ++q) {
      sa.out[q] = k < 3 ? T.in[k][q] : T.out[q];
      sa.base[q] = v.base[q];
    }
    hw::launch_node2d(d, sa, hw::MODE_STAGE, lin, chr, st);
  }
  ACUDA(cudaGetLastError());
  return HW_OK;
}

// The reverse of stage k of the recorded step T: its arguments (the adjoint of the stage output in lam[cur],
// of its input written to lam[cur ^ 1]).
hw::AdjDev stage_args(const hw::SolverView& v, AdjBuffers* B, const StepTape& T, double dt, int k, int cur) {
  const double ak[4] = {0.0, 0.0, 0.75, 1.0 / 3.0}, bk[4] = {0.0, 1.0, 0.25, 2.0 / 3.0};
  hw::Dev2D d = *v.d2;
  for (int q = 0; q < 9; ++q) d.S[q] = T.in[k - 1][q];
  hw::AdjDev A{};
  A.d = d;
  A.alpha = T.alpha + 2 * (k - 1);
  A.k = k;
  A.dt = dt;
  A.a = ak[k];
  A.b = bk[k];
  A.limiter = v.params->limiter;
  for (int q = 0; q < 9; ++q) {
    A.lout[q] = B->lam[cur][q];
    A.lin[q] = B->lam[cur ^ 1][q];
    A.lbase[q] = B->lbase[q];
    A.lR[q] = B->lR[q];
  }
  for (int q = 0; q < 6; ++q) { A.lmod[q] = B->lmod[q]; A.lqbx[q] = B->lqbx[q]; A.lqby[q] = B->lqby[q]; }
  for (int f = 0; f < hw::NREC; ++f) { A.lrecx[f] = B->lrecx[f]; A.lrecy[f] = B->lrecy[f]; }
  for (int q = 0; q < 3; ++q) { A.lstat[q] = B->lstat[q]; A.dbx[q] = T.dbx[k - 1][q]; A.dby[q] = T.dby[k - 1][q]; }
  A.fax = T.fx[k - 1];
  A.fay = T.fy[k - 1];
  for (int q = 0; q < 2; ++q) { A.lsv[q] = B->lsv[q]; A.lsq[q] = B->lsq[q]; }
  A.lalpha = B->lalpha;
  A.argmax = B->argmax;
  return A;
}

// Stage k's reverse up to alpha: the record adjoints cleared, then the node pre-pass, the sweeps, the
// records and the limiter (the alpha adjoint accumulates in A.lalpha, which the caller clears).
int reverse_stage_body(const hw::SolverView& v, AdjBuffers* B, const hw::AdjDev& A) {
  int rc = HW_OK;
  cudaStream_t st = v.stream;
  const hw::Dev2D& d = A.d;
  if ((rc = zero_planes(B->lrecx, hw::NREC, (size_t)(d.nx + 4) * d.ny, st))) return rc;
  if ((rc = zero_planes(B->lrecy, hw::NREC, (size_t)d.nx * (d.ny + 4), st))) return rc;
  const dim3 gn((d.nx + 31) / 32, (d.ny + 7) / 8), bn(32, 8);
  hw::k_adj_node_pre<<<gn, bn, 0, st>>>(A);
  hw::k_adj_sweep_x<<<dim3((d.nx + 1 + hw::AX_I - 1) / hw::AX_I, d.ny), hw::AX_T, 0, st>>>(A);
  hw::k_adj_sweep_y<<<dim3((d.nx + 31) / 32, (d.ny + 1 + hw::AY_R - 1) / hw::AY_R), hw::AY_T, hw::AY_SMEM, st>>>(A);
  const int nrec = (d.nx + 4) * d.ny + d.nx * (d.ny + 4);
  hw::k_adj_records<<<(nrec + 255) / 256, 256, 0, st>>>(A);
  if (A.limiter) hw::k_adj_limiter<<<gn, bn, 0, st>>>(A);
  ACUDA(cudaGetLastError());
  return HW_OK;
}

// Reverse of one recorded step: lam[cur] holds the adjoint of the step's output on entry and of its input
// on return (in lam[*cur]); static adjoints accumulate.
int reverse_recorded(const hw::SolverView& v, AdjBuffers* B, const StepTape& T, double dt, int* cur) {
  int rc = HW_OK;
  ACUDA(cudaFuncSetAttribute(hw::k_adj_sweep_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hw::AY_SMEM));
  cudaStream_t st = v.stream;
  const size_t n = v.n;
  if ((rc = zero_planes(B->lbase, 9, n, st))) return rc;
  for (int k = 3; k >= 1; --k) {
    const hw::AdjDev A = stage_args(v, B, T, dt, k, *cur);
    ACUDA(cudaMemsetAsync(B->lalpha, 0, 2 * sizeof(double), st));
    ACUDA(cudaMemsetAsync(B->argmax, 0x7f, 2 * sizeof(int), st));
    if ((rc = reverse_stage_body(v, B, A))) return rc;
    hw::k_adj_alpha_find<<<std::min((int)((n + 255) / 256), 152 * 8), 256, 0, st>>>(A);
    hw::k_adj_alpha_apply<<<1, 1, 0, st>>>(A);
    ACUDA(cudaGetLastError());
    *cur ^= 1;
  }
  return HW_OK;
}

// Reverse of one step from the solver's current state (recomputed into the one-step buffers).
int reverse_step(const hw::SolverView& v, AdjBuffers* B, double dt, int* cur) {
  const StepTape T = buffer_tape(B);
  const size_t bytes = v.n * sizeof(double);
  for (int q = 0; q < 9; ++q)
    ACUDA(cudaMemcpyAsync(T.in[0][q], v.state[q], bytes, cudaMemcpyDeviceToDevice, v.stream));
  int rc = forward_record(v, B, T, dt);
  if (rc) return rc;
  return reverse_recorded(v, B, T, dt, cur);
}

// static adjoints -> (b, b_x, b_y) and clear the accumulators
int finish_static(const hw::SolverView& v, AdjBuffers* B, double* const* out) {
  int rc = HW_OK;
  cudaStream_t st = v.stream;
  const hw::Dev2D& d = *v.d2;
  hw::StatAdj S{};
  S.d = d;
  for (int q = 0; q < 6; ++q) { S.lqbx[q] = B->lqbx[q]; S.lqby[q] = B->lqby[q]; }
  for (int q = 0; q < 2; ++q) { S.lsv[q] = B->lsv[q]; S.lsq[q] = B->lsq[q]; }
  S.lb = out[0];
  S.lbx = out[1];
  S.lby = out[2];
  hw::k_adj_static<<<dim3((d.nx + 1 + 31) / 32, (d.ny + 1 + 7) / 8), dim3(32, 8), 0, st>>>(S);
  const int blocks = std::min((int)((v.n + 255) / 256), 152 * 8);
  hw::k_adj_static_direct<<<blocks, 256, 0, st>>>((int)v.n, d.dx, d.dy, B->lstat[0], B->lstat[1], B->lstat[2],
                                                  out[0], out[1], out[2]);
  ACUDA(cudaGetLastError());
  if ((rc = zero_planes(B->lqbx, 6, (size_t)(d.nx + 1) * d.ny, st))) return rc;
  if ((rc = zero_planes(B->lqby, 6, (size_t)d.nx * (d.ny + 1), st))) return rc;
  if ((rc = zero_planes(B->lsv, 2, v.n, st))) return rc;
  if ((rc = zero_planes(B->lsq, 2, v.n, st))) return rc;
  if ((rc = zero_planes(B->lstat, 3, v.n, st))) return rc;
  return HW_OK;
}

int check_adjoint_solver(hw_solver* s, hw::SolverView* v) {
  if (!s) return afail(HW_ERR_ARG, "adjoint: null solver");
  int rc = hw::solver_view(s, v);
  if (rc) return rc;
  if (!v->d2) return afail(HW_ERR_ARG, "adjoint: 2D solvers only");
  if (v->params->linear_weights || !v->params->char_decomp)
    return afail(HW_ERR_ARG, "adjoint: needs nonlinear weights and characteristic projection");
  // the record-adjoint kernel indexes (nx+4) ny + nx (ny+4) records with 32-bit integers
  if (2 * ((long long)v->n + 2LL * (v->d2->nx + v->d2->ny)) >= (long long)INT_MAX)
    return afail(HW_ERR_ARG, "adjoint: grid too large (more than about 2^30 nodes)");
  return HW_OK;
}

// DP table of binomial checkpointing: cost[n][s] = extra forward steps to reverse n steps holding s
// free snapshots (besides the one at the start), split[n][s] = steps to advance before the next
// snapshot.
struct Schedule {
  int N, S;
  std::vector<long long> cost;
  std::vector<int> split;
  long long& c(int n, int s) { return cost[(size_t)n * (S + 1) + s]; }
  int& m(int n, int s) { return split[(size_t)n * (S + 1) + s]; }
  Schedule(int N_, int S_) : N(N_), S(S_), cost((size_t)(N_ + 1) * (S_ + 1), 0), split((size_t)(N_ + 1) * (S_ + 1), 0) {
    for (int s = 0; s <= S; ++s) c(1, s) = 0;
    for (int n = 2; n <= N; ++n) {
      c(n, 0) = (long long)n * (n - 1) / 2;
      for (int s = 1; s <= S; ++s) {
        long long best = -1;
        int bm = 1;
        for (int mm = 1; mm < n; ++mm) {
          const long long v = mm + c(n - mm, s - 1) + c(mm, s);
          if (best < 0 || v < best) { best = v; bm = mm; }
        }
        c(n, s) = best;
        m(n, s) = bm;
      }
    }
  }
};

// Whole-run tape: for each step its three stage inputs, the stages' source interface values and first
// flux components, and the stage alphas, then the final state; step j's output is step j+1's first stage input. Planes start on 256-byte
// boundaries.
struct RunTape {
  size_t pn, pxi, pyi, step_d;
  int nsteps;
  static size_t up(size_t x) { return (x + 31) & ~(size_t)31; }
  RunTape(const hw::SolverView& v, int N) : nsteps(N) {
    pn = up(v.n);
    pxi = up((size_t)(v.d2->nx + 1) * v.d2->ny);
    pyi = up((size_t)v.d2->nx * (v.d2->ny + 1));
    step_d = 27 * pn + 12 * pxi + 12 * pyi + 32;
  }
  size_t bytes() const { return ((size_t)nsteps * step_d + 9 * pn) * sizeof(double); }
  StepTape step(double* base, int j) const {
    StepTape T{};
    double* p = base + (size_t)j * step_d;
    for (int k = 0; k < 3; ++k)
      for (int q = 0; q < 9; ++q) T.in[k][q] = p + (size_t)(9 * k + q) * pn;
    double* next = base + (size_t)(j + 1) * step_d;  // the final state sits where step nsteps would begin
    for (int q = 0; q < 9; ++q) T.out[q] = next + (size_t)q * pn;
    double* x = p + 27 * pn;
    for (int k = 0; k < 3; ++k) {
      for (int c = 0; c < 3; ++c) {
        T.dbx[k][c] = x + (size_t)(4 * k + c) * pxi;
        T.dby[k][c] = x + 12 * pxi + (size_t)(4 * k + c) * pyi;
      }
      T.fx[k] = x + (size_t)(4 * k + 3) * pxi;
      T.fy[k] = x + 12 * pxi + (size_t)(4 * k + 3) * pyi;
    }
    T.alpha = x + 12 * pxi + 12 * pyi;
    return T;
  }
};

struct RunCtx {
  hw_solver* s;
  hw::SolverView v;
  AdjBuffers* B;
  const double* dts;
  double* d_gvals;     // [N][ng]
  const double* d_obs; // [N][ng]
  const int* d_idx;
  int ng;
  std::vector<double*> slots;  // snapshots: 9 planes each
  int cur;
  long long fwd_steps;
};

int load_slot(RunCtx& R, int slot) {
  double* src[9];
  for (int q = 0; q < 9; ++q) src[q] = R.slots[slot] + (size_t)q * R.v.n;
  return hw::solver_set_state_planes(R.s, src);
}

int save_slot(RunCtx& R, int slot) {
  for (int q = 0; q < 9; ++q)
    ACUDA(cudaMemcpyAsync(R.slots[slot] + (size_t)q * R.v.n, R.v.state[q], R.v.n * sizeof(double),
                          cudaMemcpyDeviceToDevice, R.v.stream));
  return HW_OK;
}

int advance(RunCtx& R, int from, int steps) {
  for (int j = 0; j < steps; ++j) {
    int rc = hw_rk3_step(R.s, R.dts[from + j]);
    if (rc) return rc;
    hw::solver_view(R.s, &R.v);
    ++R.fwd_steps;
  }
  return HW_OK;
}

int reverse_one(RunCtx& R, int j) {
  // adjoint of the loss at S^{j+1}, then the reverse of step j (state S^j is loaded)
  hw::k_loss_seed<<<(R.ng + 127) / 128, 128, 0, R.v.stream>>>(R.d_gvals + (size_t)j * R.ng, R.d_obs + (size_t)j * R.ng,
                                                             R.d_idx, R.ng, R.B->lam[R.cur][0]);
  hw::solver_view(R.s, &R.v);
  return reverse_step(R.v, R.B, R.dts[j], &R.cur);
}

int reverse_range(RunCtx& R, Schedule& P, int a, int n, int s, int slot_a) {
  int rc;
  if (n == 1) {
    if ((rc = load_slot(R, slot_a))) return rc;
    return reverse_one(R, a);
  }
  if (s == 0) {
    for (int j = a + n - 1; j >= a; --j) {
      if ((rc = load_slot(R, slot_a))) return rc;
      if ((rc = advance(R, a, j - a))) return rc;
      if ((rc = reverse_one(R, j))) return rc;
    }
    return HW_OK;
  }
  const int m = P.m(n, s);
  const int slot_b = slot_a + 1;
  if ((rc = load_slot(R, slot_a))) return rc;
  if ((rc = advance(R, a, m))) return rc;
  if ((rc = save_slot(R, slot_b))) return rc;
  if ((rc = reverse_range(R, P, a + m, n - m, s - 1, slot_b))) return rc;
  return reverse_range(R, P, a, m, s, slot_a);
}

}  // namespace

extern "C" {

int hw_adjoint_step(hw_solver* s, double dt, double* const* lam_state, double* const* lam_static) {
  hw::SolverView v;
  int rc = check_adjoint_solver(s, &v);
  if (rc) return rc;
  if (!lam_state || !lam_static) return afail(HW_ERR_ARG, "hw_adjoint_step: null adjoint planes");
  for (int q = 0; q < 9; ++q)
    if (!lam_state[q]) return afail(HW_ERR_ARG, "hw_adjoint_step: null state adjoint plane");
  for (int q = 0; q < 3; ++q)
    if (!lam_static[q]) return afail(HW_ERR_ARG, "hw_adjoint_step: null static adjoint plane");
  if (!(dt >= 0) || !(dt < 1e300)) return afail(HW_ERR_ARG, "hw_adjoint_step: bad dt");
  AdjBuffers* B = nullptr;
  if ((rc = get_buffers(s, v, &B))) return rc;
  const int blocks = std::min((int)((v.n + 255) / 256), 152 * 8);
  hw::Ptr9 src{}, dst{};
  for (int q = 0; q < 9; ++q) { src.p[q] = lam_state[q]; dst.p[q] = B->lam[0][q]; }
  hw::k_adj_convert<<<blocks, 256, 0, v.stream>>>((int)v.n, v.d2->dx, v.d2->dy, src, dst, 1);
  int cur = 0;
  if ((rc = reverse_step(v, B, dt, &cur))) return rc;
  for (int q = 0; q < 9; ++q) { src.p[q] = B->lam[cur][q]; dst.p[q] = lam_state[q]; }
  hw::k_adj_convert<<<blocks, 256, 0, v.stream>>>((int)v.n, v.d2->dx, v.d2->dy, src, dst, 0);
  if ((rc = finish_static(v, B, lam_static))) return rc;
  ACUDA(cudaGetLastError());
  return HW_OK;
}

int hw_gauge_loss(hw_solver* s, int nsteps, const double* dts, const int* gauge_idx, int ngauge,
                  const double* eta_obs, double* loss_out, double* eta_gauges) {
  hw::SolverView v;
  int rc = check_adjoint_solver(s, &v);
  if (rc) return rc;
  if (nsteps < 1 || !dts || !gauge_idx || ngauge < 1 || !eta_obs || !loss_out)
    return afail(HW_ERR_ARG, "hw_gauge_loss: bad argument");
  for (int g = 0; g < ngauge; ++g)
    if (gauge_idx[g] < 0 || (size_t)gauge_idx[g] >= v.n) return afail(HW_ERR_ARG, "hw_gauge_loss: gauge out of range");
  cudaStream_t st = v.stream;
  double *d_save = nullptr, *d_g = nullptr;
  int* d_idx = nullptr;
  // every exit after the first allocation frees the working buffers
  auto check = [&](cudaError_t e, const char* what) {
    if (rc == HW_OK && e != cudaSuccess) rc = afail(HW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  auto alloc = [&](void** p, size_t bytes, const char* what) {
    if (rc != HW_OK) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = afail(HW_ERR_NOMEM, std::string("hw_gauge_loss: allocation failed: ") + what);
    }
  };
  alloc((void**)&d_save, 9 * v.n * sizeof(double), "saved state");
  alloc((void**)&d_g, (size_t)nsteps * ngauge * sizeof(double), "gauge values");
  alloc((void**)&d_idx, ngauge * sizeof(int), "gauge indices");
  if (rc == HW_OK) {
    check(cudaMemcpyAsync(d_idx, gauge_idx, ngauge * sizeof(int), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    for (int q = 0; q < 9; ++q)
      check(cudaMemcpyAsync(d_save + (size_t)q * v.n, v.state[q], v.n * sizeof(double), cudaMemcpyDeviceToDevice, st),
            "cudaMemcpyAsync");
  }
  for (int j = 0; j < nsteps && rc == HW_OK; ++j) {
    rc = hw_rk3_step(s, dts[j]);
    hw::solver_view(s, &v);
    hw::k_gather_eta<<<(ngauge + 127) / 128, 128, 0, st>>>(v.state[0], d_idx, ngauge, d_g + (size_t)j * ngauge);
  }
  std::vector<double> g((size_t)nsteps * ngauge);
  if (rc == HW_OK) {
    check(cudaMemcpyAsync(g.data(), d_g, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    check(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  if (rc == HW_OK) {
    *loss_out = misfit_loss(g.data(), eta_obs, g.size());
    if (eta_gauges) std::copy(g.begin(), g.end(), eta_gauges);
    double* src[9];
    for (int q = 0; q < 9; ++q) src[q] = d_save + (size_t)q * v.n;
    rc = hw::solver_set_state_planes(s, src);
  }
  cudaStreamSynchronize(st);
  cudaFree(d_save);
  cudaFree(d_g);
  cudaFree(d_idx);
  return rc;
}

int hw_adjoint_run(hw_solver* s, int nsteps, const double* dts, const int* gauge_idx, int ngauge,
                   const double* eta_obs, int snapshots, double* loss_out, double* const* grad_state,
                   double* const* grad_static, long long* forward_steps_out) {
  hw::SolverView v;
  int rc = check_adjoint_solver(s, &v);
  if (rc) return rc;
  if (nsteps < 1 || !dts || !gauge_idx || ngauge < 1 || !eta_obs || !grad_state || !grad_static ||
      (snapshots < 0 && snapshots != HW_ADJ_TAPE && snapshots != HW_ADJ_AUTO))
    return afail(HW_ERR_ARG, "hw_adjoint_run: bad argument");
  for (int g = 0; g < ngauge; ++g)
    if (gauge_idx[g] < 0 || (size_t)gauge_idx[g] >= v.n) return afail(HW_ERR_ARG, "hw_adjoint_run: gauge out of range");
  for (int q = 0; q < 9; ++q)
    if (!grad_state[q]) return afail(HW_ERR_ARG, "hw_adjoint_run: null gradient plane");
  for (int q = 0; q < 3; ++q)
    if (!grad_static[q]) return afail(HW_ERR_ARG, "hw_adjoint_run: null gradient plane");
  AdjBuffers* B = nullptr;
  if ((rc = get_buffers(s, v, &B))) return rc;
  cudaStream_t st = v.stream;

  // storage mode: a whole-run tape, or binomial checkpointing with S snapshots besides the start
  const RunTape layout(v, nsteps);
  bool use_tape = false;
  int S = 0;
  if (snapshots == HW_ADJ_TAPE || snapshots == HW_ADJ_AUTO) {
    size_t free_b = 0, total_b = 0;
    ACUDA(cudaMemGetInfo(&free_b, &total_b));
    const double budget = 0.9 * (double)free_b;
    if ((double)layout.bytes() <= budget) {
      use_tape = true;
    } else if (snapshots == HW_ADJ_TAPE) {
      return afail(HW_ERR_NOMEM, "hw_adjoint_run: the whole-run tape does not fit in free device memory");
    } else {
      const double per = 9.0 * (double)v.n * sizeof(double);
      S = (int)std::max(0.0, std::min((double)(nsteps - 1), std::floor(budget / per) - 1.0));
    }
  } else {
    S = std::min(snapshots, std::max(nsteps - 1, 0));
  }

  RunCtx R;
  R.s = s; R.v = v; R.B = B; R.dts = dts; R.ng = ngauge; R.cur = 0; R.fwd_steps = 0;
  R.d_gvals = nullptr;
  double* d_obs = nullptr;
  int* d_idx = nullptr;
  double* tape = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (double* p : R.slots) if (p) cudaFree(p);
    cudaFree(tape);
    cudaFree(R.d_gvals);
    cudaFree(d_obs);
    cudaFree(d_idx);
    if (forward_steps_out) *forward_steps_out = R.fwd_steps;
  };
  auto alloc = [&](void** p, size_t bytes, const char* what) {
    if (rc != HW_OK) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = afail(HW_ERR_NOMEM, std::string("hw_adjoint_run: allocation failed: ") + what);
    }
  };
  alloc((void**)&R.d_gvals, (size_t)nsteps * ngauge * sizeof(double), "gauge values");
  alloc((void**)&d_obs, (size_t)nsteps * ngauge * sizeof(double), "observations");
  alloc((void**)&d_idx, ngauge * sizeof(int), "gauge indices");
  if (use_tape) alloc((void**)&tape, layout.bytes(), "tape");
  R.slots.assign(use_tape ? 0 : S + 1, nullptr);
  for (size_t k = 0; k < R.slots.size(); ++k) alloc((void**)&R.slots[k], 9 * v.n * sizeof(double), "snapshot");
  R.d_obs = d_obs;
  R.d_idx = d_idx;
  auto check = [&](cudaError_t e, const char* what) {
    if (rc == HW_OK && e != cudaSuccess) rc = afail(HW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  if (rc == HW_OK) {
    check(cudaMemcpyAsync(d_obs, eta_obs, (size_t)nsteps * ngauge * sizeof(double), cudaMemcpyHostToDevice, st),
          "hw_adjoint_run: copy of observations");
    check(cudaMemcpyAsync(d_idx, gauge_idx, ngauge * sizeof(int), cudaMemcpyHostToDevice, st),
          "hw_adjoint_run: copy of gauge indices");
  }
  // forward pass: loss and gauge values (recording the tape, or from the solver with a snapshot at 0)
  if (rc == HW_OK && use_tape) {
    const StepTape T0 = layout.step(tape, 0);
    for (int q = 0; q < 9 && rc == HW_OK; ++q)
      check(cudaMemcpyAsync(T0.in[0][q], v.state[q], v.n * sizeof(double), cudaMemcpyDeviceToDevice, st),
            "hw_adjoint_run: copy of the initial state");
    for (int j = 0; j < nsteps && rc == HW_OK; ++j) {
      const StepTape T = layout.step(tape, j);
      rc = forward_record(v, B, T, dts[j]);
      ++R.fwd_steps;
      hw::k_gather_eta<<<(ngauge + 127) / 128, 128, 0, st>>>(T.out[0], d_idx, ngauge, R.d_gvals + (size_t)j * ngauge);
    }
  } else if (rc == HW_OK) {
    rc = save_slot(R, 0);
    for (int j = 0; j < nsteps && rc == HW_OK; ++j) {
      rc = hw_rk3_step(s, dts[j]);
      hw::solver_view(s, &R.v);
      ++R.fwd_steps;
      hw::k_gather_eta<<<(ngauge + 127) / 128, 128, 0, st>>>(R.v.state[0], d_idx, ngauge,
                                                             R.d_gvals + (size_t)j * ngauge);
    }
  }
  if (rc == HW_OK) check(cudaGetLastError(), "hw_adjoint_run: forward pass");
  if (rc == HW_OK && loss_out) {
    std::vector<double> g((size_t)nsteps * ngauge);
    check(cudaMemcpyAsync(g.data(), R.d_gvals, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
          "hw_adjoint_run: copy of gauge values");
    check(cudaStreamSynchronize(st), "hw_adjoint_run: forward pass");
    *loss_out = misfit_loss(g.data(), eta_obs, g.size());
  }
  // reverse pass
  if (rc == HW_OK) rc = zero_planes(B->lam[0], 9, v.n, st);
  if (rc == HW_OK && use_tape) {
    for (int j = nsteps - 1; j >= 0 && rc == HW_OK; --j) {
      hw::k_loss_seed<<<(ngauge + 127) / 128, 128, 0, st>>>(R.d_gvals + (size_t)j * ngauge,
                                                           d_obs + (size_t)j * ngauge, d_idx, ngauge,
                                                           B->lam[R.cur][0]);
      rc = reverse_recorded(v, B, layout.step(tape, j), dts[j], &R.cur);
    }
  } else if (rc == HW_OK) {
    Schedule P(nsteps, S);
    rc = reverse_range(R, P, 0, nsteps, S, 0);
  }
  if (rc == HW_OK) {
    hw::solver_view(s, &R.v);
    const int blocks = std::min((int)((v.n + 255) / 256), 152 * 8);
    hw::Ptr9 src{}, dst{};
    for (int q = 0; q < 9; ++q) { src.p[q] = B->lam[R.cur][q]; dst.p[q] = grad_state[q]; }
    hw::k_adj_convert<<<blocks, 256, 0, st>>>((int)v.n, v.d2->dx, v.d2->dy, src, dst, 0);
    rc = zero_planes(grad_static, 3, v.n, st);
    if (rc == HW_OK) rc = finish_static(R.v, B, grad_static);
  }
  if (rc == HW_OK && !use_tape) rc = load_slot(R, 0);  // leave the solver at the initial state
  cleanup();
  return rc;
}

}  // extern "C"

// =============================================================================================
// The adjoint of a run of a block decomposition (hw_dd_*): every block reverses its own stages on its
// extended grid; between stages the transpose of the halo exchange adds the adjoints that landed on a
// block's ring to the nodes the ring was copied from (and clears the ring); the alpha adjoint is summed
// over the blocks and applied once, by the block owning the undecomposed grid's first maximising node.
// =============================================================================================
namespace {

// state planes (eta, m, w, H1, M1, W1, H2, M2, W2) odd across x- and y-walls; static (b, b_x, b_y)
constexpr unsigned kStateOddX = (1u << 1) | (1u << 3) | (1u << 5) | (1u << 7);
constexpr unsigned kStateOddY = (1u << 2) | (1u << 5) | (1u << 6) | (1u << 7);
constexpr unsigned kStatOddX = 1u << 1;
constexpr unsigned kStatOddY = 1u << 2;

struct DDBlock {
  hw_solver* s = nullptr;
  hw_part_info info{};
  hw::SolverView v{};
  AdjBuffers* B = nullptr;
  double* tape = nullptr;
  int* d_map = nullptr;  // [2][ng_p]: local extended node, global gauge slot
  int ng = 0;
};

}  // namespace

namespace {
int dd_adjoint_impl(hw_dd* dd, int nsteps, const double* dts, const int* gauge_idx, int ngauge, const double* eta_obs,
                    double* loss_out, double* const* grad_state, double* const* grad_static) {
  int np = 0;
  hw_solver* const* parts = nullptr;
  const hw_part_info* infos = nullptr;
  cudaStream_t st = nullptr;
  const hw_grid* grid = nullptr;
  int rc = hw::dd_blocks(dd, &np, &parts, &infos, &st, &grid);
  if (rc) return rc;
  if (nsteps < 1 || !dts || !gauge_idx || ngauge < 1 || !eta_obs || !grad_state || !grad_static)
    return afail(HW_ERR_ARG, "hw_dd_adjoint_run: bad argument");
  const int gnx = grid->nx, gny = grid->ny;
  for (int g = 0; g < ngauge; ++g)
    if (gauge_idx[g] < 0 || gauge_idx[g] >= gnx * gny) return afail(HW_ERR_ARG, "hw_dd_adjoint_run: gauge out of range");
  for (int q = 0; q < 9; ++q)
    if (!grad_state[q]) return afail(HW_ERR_ARG, "hw_dd_adjoint_run: null gradient plane");
  for (int q = 0; q < 3; ++q)
    if (!grad_static[q]) return afail(HW_ERR_ARG, "hw_dd_adjoint_run: null gradient plane");
  std::vector<DDBlock> bl(np);
  for (int p = 0; p < np; ++p) {
    bl[p].s = parts[p];
    bl[p].info = infos[p];
    if ((rc = check_adjoint_solver(parts[p], &bl[p].v))) return rc;
    if ((rc = get_buffers(parts[p], bl[p].v, &bl[p].B))) return rc;
  }
  ACUDA(cudaFuncSetAttribute(hw::k_adj_sweep_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hw::AY_SMEM));
  std::vector<RunTape> layout;
  for (int p = 0; p < np; ++p) layout.emplace_back(bl[p].v, nsteps);
  // gauges by owner block: local extended node and global slot
  std::vector<std::vector<int>> loc(np), slot(np);
  for (int g = 0; g < ngauge; ++g) {
    const int gi = gauge_idx[g] % gnx, gj = gauge_idx[g] / gnx;
    for (int p = 0; p < np; ++p) {
      const hw_part_info& I = infos[p];
      if (gi >= I.i0 && gi < I.i0 + I.nx && gj >= I.j0 && gj < I.j0 + I.ny) {
        loc[p].push_back((gj - I.j0 + 2) * (I.nx + 4) + (gi - I.i0 + 2));
        slot[p].push_back(g);
        break;
      }
    }
  }
  double *d_gvals = nullptr, *d_obs = nullptr, *lal = nullptr, *tmp = nullptr;
  unsigned long long* keys = nullptr;
  size_t max_ext = 0;
  for (int p = 0; p < np; ++p) max_ext = std::max(max_ext, bl[p].v.n);
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (DDBlock& b : bl) { cudaFree(b.tape); cudaFree(b.d_map); }
    cudaFree(d_gvals); cudaFree(d_obs); cudaFree(lal); cudaFree(keys); cudaFree(tmp);
  };
  auto alloc = [&](void** q, size_t bytes, const char* what) {
    if (rc != HW_OK) return;
    if (cudaMalloc(q, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = afail(HW_ERR_NOMEM, std::string("hw_dd_adjoint_run: allocation failed: ") + what);
    }
  };
  alloc((void**)&d_gvals, (size_t)nsteps * ngauge * sizeof(double), "gauge values");
  alloc((void**)&d_obs, (size_t)nsteps * ngauge * sizeof(double), "observations");
  alloc((void**)&lal, 4 * sizeof(double), "alpha adjoint");  // [0..1] alpha adjoint, [2] first maximising nodes
  alloc((void**)&keys, (2 * (size_t)np + 2) * sizeof(unsigned long long), "alpha keys");
  alloc((void**)&tmp, 12 * max_ext * sizeof(double), "gradient scratch");
  for (int p = 0; p < np; ++p) {
    alloc((void**)&bl[p].tape, layout[p].bytes(), "tape");
    bl[p].ng = (int)loc[p].size();
    if (bl[p].ng) alloc((void**)&bl[p].d_map, 2 * bl[p].ng * sizeof(int), "gauge map");
  }
  auto check = [&](cudaError_t e, const char* what) {
    if (rc == HW_OK && e != cudaSuccess) rc = afail(HW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  if (rc == HW_OK) {
    check(cudaMemcpyAsync(d_obs, eta_obs, (size_t)nsteps * ngauge * sizeof(double), cudaMemcpyHostToDevice, st),
          "hw_dd_adjoint_run: copy of observations");
    for (int p = 0; p < np && rc == HW_OK; ++p) {
      if (!bl[p].ng) continue;
      std::vector<int> m(loc[p]);
      m.insert(m.end(), slot[p].begin(), slot[p].end());
      check(cudaMemcpyAsync(bl[p].d_map, m.data(), m.size() * sizeof(int), cudaMemcpyHostToDevice, st),
            "hw_dd_adjoint_run: copy of the gauge map");
      check(cudaStreamSynchronize(st), "hw_dd_adjoint_run: copy of the gauge map");
    }
    for (int p = 0; p < np && rc == HW_OK; ++p) {
      const StepTape T0 = layout[p].step(bl[p].tape, 0);
      for (int q = 0; q < 9 && rc == HW_OK; ++q)
        check(cudaMemcpyAsync(T0.in[0][q], bl[p].v.state[q], bl[p].v.n * sizeof(double), cudaMemcpyDeviceToDevice, st),
              "hw_dd_adjoint_run: copy of the initial state");
    }
  }
  // forward pass, recorded: per stage the exchange, the blocks' alpha keys and their maximum, then the
  // blocks' sweeps and node update into the tape
  std::vector<double*> pl(9 * (size_t)np);
  std::vector<double* const*> plp(np);
  for (int p = 0; p < np; ++p) plp[p] = pl.data() + 9 * (size_t)p;
  for (int j = 0; j < nsteps && rc == HW_OK; ++j) {
    for (int p = 0; p < np && rc == HW_OK; ++p)
      check(cudaMemcpyAsync(bl[p].v.dt, &dts[j], sizeof(double), cudaMemcpyHostToDevice, st), "hw_dd_adjoint_run: dt");
    for (int k = 1; k <= 3 && rc == HW_OK; ++k) {
      for (int p = 0; p < np; ++p) {
        const StepTape T = layout[p].step(bl[p].tape, j);
        for (int q = 0; q < 9; ++q) pl[9 * (size_t)p + q] = T.in[k - 1][q];
      }
      if ((rc = hw::dd_exchange_planes(dd, plp.data(), 9, kStateOddX, kStateOddY, st))) break;
      if ((rc = hw::dd_fork_blocks(dd, st))) break;
      for (int p = 0; p < np; ++p) {
        const StepTape T = layout[p].step(bl[p].tape, j);
        hw::Dev2D d = *bl[p].v.d2;
        for (int q = 0; q < 9; ++q) d.S[q] = T.in[k - 1][q];
        hw::launch_alpha2d(d, bl[p].B->amax, (int*)(bl[p].B->lalpha + 2), bl[p].v.stream);
        check(cudaMemcpyAsync(keys + 2 * p, bl[p].B->amax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                              bl[p].v.stream),
              "hw_dd_adjoint_run: alpha keys");
      }
      if ((rc = hw::dd_join_blocks(dd, st))) break;
      hw::k_keys_max<<<1, 32, 0, st>>>(keys, np, keys + 2 * np);
      if ((rc = hw::dd_fork_blocks(dd, st))) break;
      for (int p = 0; p < np; ++p) {
        const StepTape T = layout[p].step(bl[p].tape, j);
        hw::Dev2D d = *bl[p].v.d2;
        for (int q = 0; q < 9; ++q) d.S[q] = T.in[k - 1][q];
        for (int c = 0; c < 3; ++c) { d.X[3 + c] = T.dbx[k - 1][c]; d.Y[3 + c] = T.dby[k - 1][c]; }
        d.X[0] = T.fx[k - 1];
        d.Y[0] = T.fy[k - 1];
        const cudaStream_t bs = bl[p].v.stream;
        hw::launch_finish_alpha2d(d, keys + 2 * np, T.alpha + 2 * (k - 1), nullptr, bl[p].v.params->cfl, nullptr, -1.0,
                                  bs);
        hw::launch_sweep_x2d(d, T.alpha + 2 * (k - 1), false, true, bs);
        hw::launch_sweep_y2d(d, T.alpha + 2 * (k - 1), false, true, bs);
        hw::StageArgs sa{};
        sa.k = k;
        sa.limiter = bl[p].v.params->limiter;
        sa.dt = bl[p].v.dt;
        for (int q = 0; q < 9; ++q) {
          sa.out[q] = k < 3 ? T.in[k][q] : T.out[q];
          sa.base[q] = bl[p].v.base[q];
        }
        hw::launch_node2d(d, sa, hw::MODE_STAGE, false, true, bs);
      }
      if ((rc = hw::dd_join_blocks(dd, st))) break;
    }
    for (int p = 0; p < np && rc == HW_OK; ++p)
      if (bl[p].ng) {
        const StepTape T = layout[p].step(bl[p].tape, j);
        hw::k_gather_eta_map<<<(bl[p].ng + 127) / 128, 128, 0, st>>>(T.out[0], bl[p].d_map, bl[p].d_map + bl[p].ng,
                                                                    bl[p].ng, d_gvals + (size_t)j * ngauge);
      }
  }
  if (rc == HW_OK) check(cudaGetLastError(), "hw_dd_adjoint_run: forward pass");
  if (rc == HW_OK && loss_out) {
    std::vector<double> g((size_t)nsteps * ngauge);
    check(cudaMemcpyAsync(g.data(), d_gvals, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
          "hw_dd_adjoint_run: copy of gauge values");
    check(cudaStreamSynchronize(st), "hw_dd_adjoint_run: forward pass");
    *loss_out = misfit_loss(g.data(), eta_obs, g.size());
  }
  // reverse pass
  int cur = 0;
  for (int p = 0; p < np && rc == HW_OK; ++p) rc = zero_planes(bl[p].B->lam[0], 9, bl[p].v.n, st);
  for (int j = nsteps - 1; j >= 0 && rc == HW_OK; --j) {
    for (int p = 0; p < np && rc == HW_OK; ++p) {
      if (bl[p].ng)
        hw::k_loss_seed_map<<<(bl[p].ng + 127) / 128, 128, 0, st>>>(d_gvals + (size_t)j * ngauge,
                                                                   d_obs + (size_t)j * ngauge, bl[p].d_map,
                                                                   bl[p].d_map + bl[p].ng, bl[p].ng,
                                                                   bl[p].B->lam[cur][0]);
      rc = zero_planes(bl[p].B->lbase, 9, bl[p].v.n, st);
    }
    for (int k = 3; k >= 1 && rc == HW_OK; --k) {
      check(cudaMemsetAsync(lal, 0, 2 * sizeof(double), st), "hw_dd_adjoint_run: alpha adjoint");
      check(cudaMemsetAsync(lal + 2, 0x7f, 2 * sizeof(int), st), "hw_dd_adjoint_run: alpha node");
      std::vector<hw::AdjDev> A(np);
      if (rc == HW_OK) rc = hw::dd_fork_blocks(dd, st);
      for (int p = 0; p < np && rc == HW_OK; ++p) {
        A[p] = stage_args(bl[p].v, bl[p].B, layout[p].step(bl[p].tape, j), dts[j], k, cur);
        A[p].lalpha = lal;
        A[p].argmax = (int*)(lal + 2);
        rc = reverse_stage_body(bl[p].v, bl[p].B, A[p]);  // on the block's stream
      }
      if (rc == HW_OK) rc = hw::dd_join_blocks(dd, st);
      for (int p = 0; p < np && rc == HW_OK; ++p) {
        const hw_part_info& I = bl[p].info;
        hw::k_adj_alpha_find_block<<<std::min((I.nx * I.ny + 255) / 256, 152 * 8), 256, 0, st>>>(A[p], I.nx, I.ny, I.i0,
                                                                                              I.j0, gnx);
      }
      for (int p = 0; p < np && rc == HW_OK; ++p) {
        const hw_part_info& I = bl[p].info;
        hw::k_adj_alpha_apply_block<<<1, 1, 0, st>>>(A[p], I.nx, I.ny, I.i0, I.j0, gnx);
      }
      if (rc == HW_OK) check(cudaGetLastError(), "hw_dd_adjoint_run: reverse stage");
      for (int p = 0; p < np; ++p)
        for (int q = 0; q < 9; ++q) pl[9 * (size_t)p + q] = bl[p].B->lam[cur ^ 1][q];
      if (rc == HW_OK) rc = hw::dd_exchange_adjoint(dd, plp.data(), 9, kStateOddX, kStateOddY, st);
      cur ^= 1;
    }
  }
  // gradients: the state's in physical units, the static ones with their rings moved to the owners; the
  // blocks' own nodes copied into the global planes (device)
  for (int p = 0; p < np && rc == HW_OK; ++p) {
    const hw_part_info& I = bl[p].info;
    const int nxe = I.nx + 4;
    const size_t n = bl[p].v.n;
    const int blocks = std::min((int)((n + 255) / 256), 152 * 8);
    hw::Ptr9 src{}, dst{};
    for (int q = 0; q < 9; ++q) { src.p[q] = bl[p].B->lam[cur][q]; dst.p[q] = tmp + q * max_ext; }
    hw::k_adj_convert<<<blocks, 256, 0, st>>>((int)n, bl[p].v.d2->dx, bl[p].v.d2->dy, src, dst, 0);
    for (int q = 0; q < 9 && rc == HW_OK; ++q)
      check(cudaMemcpy2DAsync(grad_state[q] + (size_t)I.j0 * gnx + I.i0, gnx * sizeof(double),
                              tmp + q * max_ext + 2 * (size_t)nxe + 2, nxe * sizeof(double), I.nx * sizeof(double), I.ny,
                              cudaMemcpyDeviceToDevice, st),
            "hw_dd_adjoint_run: state gradient");
  }
  std::vector<double*> stat_planes(3 * (size_t)np);
  std::vector<double* const*> sp(np);
  if (rc == HW_OK) rc = hw::dd_fork_blocks(dd, st);
  for (int p = 0; p < np && rc == HW_OK; ++p) {
    for (int q = 0; q < 3; ++q) stat_planes[3 * (size_t)p + q] = bl[p].B->lstatic_phys[q];
    sp[p] = stat_planes.data() + 3 * (size_t)p;
    rc = zero_planes(bl[p].B->lstatic_phys, 3, bl[p].v.n, bl[p].v.stream);
    if (rc == HW_OK) rc = finish_static(bl[p].v, bl[p].B, bl[p].B->lstatic_phys);
  }
  if (rc == HW_OK) rc = hw::dd_join_blocks(dd, st);
  if (rc == HW_OK) rc = hw::dd_exchange_adjoint(dd, sp.data(), 3, kStatOddX, kStatOddY, st);
  for (int p = 0; p < np && rc == HW_OK; ++p) {
    const hw_part_info& I = bl[p].info;
    const int nxe = I.nx + 4;
    for (int q = 0; q < 3 && rc == HW_OK; ++q)
      check(cudaMemcpy2DAsync(grad_static[q] + (size_t)I.j0 * gnx + I.i0, gnx * sizeof(double),
                              bl[p].B->lstatic_phys[q] + 2 * (size_t)nxe + 2, nxe * sizeof(double), I.nx * sizeof(double),
                              I.ny, cudaMemcpyDeviceToDevice, st),
            "hw_dd_adjoint_run: static gradient");
  }
  if (rc == HW_OK) check(cudaStreamSynchronize(st), "hw_dd_adjoint_run");
  cleanup();
  return rc;
}
}  // namespace

// The main stream orders the run: the exchanges, the alpha reductions and the gauges run on it, each
// block's stages on the block's own stream between a fork and a join.
extern "C" int hw_dd_adjoint_run(hw_dd* dd, int nsteps, const double* dts, const int* gauge_idx, int ngauge,
                                 const double* eta_obs, double* loss_out, double* const* grad_state,
                                 double* const* grad_static) {
  int np = 0;
  hw_solver* const* parts = nullptr;
  const hw_part_info* infos = nullptr;
  cudaStream_t st = nullptr;
  const hw_grid* grid = nullptr;
  int rc = hw::dd_blocks(dd, &np, &parts, &infos, &st, &grid);
  if (rc) return rc;
  ACUDA(cudaStreamSynchronize(st));
  for (int p = 0; p < np; ++p) ACUDA(cudaStreamSynchronize(hw::solver_stream(parts[p])));
  rc = dd_adjoint_impl(dd, nsteps, dts, gauge_idx, ngauge, eta_obs, loss_out, grad_state, grad_static);
  cudaStreamSynchronize(st);
  for (int p = 0; p < np; ++p) cudaStreamSynchronize(hw::solver_stream(parts[p]));
  return rc;
}

// =============================================================================================
// Per-block adjoint (hw_part_adj_*): the steps of dd_adjoint_impl for one block solver, so that blocks
// owned by different processes run the same adjoint with the exchanges, the alpha keys, the gauge values
// and the alpha adjoint carried between them by the caller (paper_2208_01260_gb300/decomp.py).
// =============================================================================================
struct hw_part_adj {
  hw_solver* s = nullptr;
  hw_part_info info{};
  hw::SolverView v{};
  AdjBuffers* B = nullptr;
  RunTape* layout = nullptr;
  double* tape = nullptr;
  int nsteps = 0, ngauge = 0, nloc = 0, gnx = 0;
  int* d_map = nullptr;     // [2][nloc]: local extended node, global gauge slot
  double* d_gvals = nullptr;  // [nsteps][ngauge]: this block's gauges (zeros elsewhere)
  double* d_gall = nullptr;   // [nsteps][ngauge]: all gauges (set_misfit)
  double* d_obs = nullptr;
  double* lal = nullptr;      // [2] alpha adjoint, then [2] ints: first maximising node
  double* tmp = nullptr;      // 9 planes: state gradient in physical units
  double* keys = nullptr;     // the alpha reduction's keys and scratch (kAlpha2dScratch slots)
  int cur = 0;
  bool reverse = false;
  hw::AdjDev last{};
  bool have_last = false;
};

namespace {
int pa_check(hw_part_adj* a, const char* fn) {
  if (!a || !a->s) return afail(HW_ERR_ARG, std::string(fn) + ": null context");
  return HW_OK;
}
int pa_stage(hw_part_adj* a, int j, int k, const char* fn) {
  int rc = pa_check(a, fn);
  if (rc) return rc;
  if (j < 0 || j >= a->nsteps || k < 1 || k > 3) return afail(HW_ERR_ARG, std::string(fn) + ": step or stage out of range");
  return HW_OK;
}
int pa_face(int face, const char* fn) {
  if (face < HW_FACE_W || face > HW_FACE_N) return afail(HW_ERR_ARG, std::string(fn) + ": bad face");
  return HW_OK;
}
__global__ void k_set_int2(int* p, int a, int b) {
  p[0] = a;
  p[1] = b;
}
void pa_free(hw_part_adj* a) {
  if (a->v.stream) cudaStreamSynchronize(a->v.stream);
  cudaFree(a->tape); cudaFree(a->d_map); cudaFree(a->d_gvals); cudaFree(a->d_gall); cudaFree(a->d_obs);
  cudaFree(a->lal); cudaFree(a->tmp); cudaFree(a->keys);
  delete a->layout;
  delete a;
}
}  // namespace

extern "C" {

int hw_part_adj_create(hw_solver* s, int nsteps, int ngauge, int nloc, const int* gauge_slot, const int* gauge_node,
                       int global_nx, hw_part_adj** out) {
  if (!out) return afail(HW_ERR_ARG, "hw_part_adj_create: null output");
  *out = nullptr;
  const hw_part_info* I = hw::part_info(s);
  if (!I) return afail(HW_ERR_ARG, "hw_part_adj_create: not a block solver");
  if (nsteps < 1 || ngauge < 1 || nloc < 0 || nloc > ngauge || (nloc > 0 && (!gauge_slot || !gauge_node)) || global_nx < 1)
    return afail(HW_ERR_ARG, "hw_part_adj_create: bad argument");
  hw_part_adj* a = new hw_part_adj();
  a->s = s;
  a->info = *I;
  int rc = check_adjoint_solver(s, &a->v);
  if (rc == HW_OK) rc = get_buffers(s, a->v, &a->B);
  if (rc) { delete a; return rc; }
  a->nsteps = nsteps; a->ngauge = ngauge; a->nloc = nloc; a->gnx = global_nx;
  std::vector<int> map(2 * (size_t)nloc);
  for (int g = 0; g < nloc; ++g) {
    const int gi = gauge_node[g] % global_nx - I->i0, gj = gauge_node[g] / global_nx - I->j0;
    if (gauge_node[g] < 0 || gi < 0 || gi >= I->nx || gj < 0 || gj >= I->ny || gauge_slot[g] < 0 || gauge_slot[g] >= ngauge) {
      delete a;
      return afail(HW_ERR_ARG, "hw_part_adj_create: gauge not on the block's own nodes, or slot out of range");
    }
    map[g] = (gj + 2) * (I->nx + 4) + (gi + 2);
    map[nloc + g] = gauge_slot[g];
  }
  a->layout = new RunTape(a->v, nsteps);
  auto alloc = [&](void** q, size_t bytes) {
    if (rc != HW_OK) return;
    if (cudaMalloc(q, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = afail(HW_ERR_NOMEM, "hw_part_adj_create: allocation failed");
    }
  };
  alloc((void**)&a->tape, a->layout->bytes());
  if (nloc) alloc((void**)&a->d_map, map.size() * sizeof(int));
  const size_t gb = (size_t)nsteps * ngauge * sizeof(double);
  alloc((void**)&a->d_gvals, gb);
  alloc((void**)&a->d_gall, gb);
  alloc((void**)&a->d_obs, gb);
  alloc((void**)&a->lal, 4 * sizeof(double));
  alloc((void**)&a->tmp, 9 * a->v.n * sizeof(double));
  alloc((void**)&a->keys, hw::kAlpha2dScratch * sizeof(double));
  if (rc) { pa_free(a); return rc; }
  cudaStream_t st = a->v.stream;
  cudaError_t e = cudaFuncSetAttribute(hw::k_adj_sweep_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hw::AY_SMEM);
  if (e == cudaSuccess && nloc) e = cudaMemcpyAsync(a->d_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a->d_gvals, 0, gb, st);
  const StepTape T0 = a->layout->step(a->tape, 0);
  for (int q = 0; q < 9 && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(T0.in[0][q], a->v.state[q], a->v.n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { pa_free(a); return afail(HW_ERR_CUDA, std::string("hw_part_adj_create: ") + cudaGetErrorString(e)); }
  *out = a;
  return HW_OK;
}

int hw_part_adj_destroy(hw_part_adj* a) {
  if (a) pa_free(a);
  return HW_OK;
}

int hw_part_adj_strip_size(hw_part_adj* a, int what, int face, long long* count) {
  int rc = pa_check(a, "hw_part_adj_strip_size");
  if (!rc) rc = pa_face(face, "hw_part_adj_strip_size");
  if (rc) return rc;
  if ((what != 0 && what != 1) || !count) return afail(HW_ERR_ARG, "hw_part_adj_strip_size: bad argument");
  const long long len = face < 2 ? a->info.ny : a->info.nx + 4;
  *count = (what == 0 ? 9 : 3) * 2 * len;
  return HW_OK;
}

int hw_part_adj_pack(hw_part_adj* a, int j, int k, int face, double* strip) {
  int rc = pa_stage(a, j, k, "hw_part_adj_pack");
  if (!rc) rc = pa_face(face, "hw_part_adj_pack");
  if (rc) return rc;
  if (!strip) return afail(HW_ERR_ARG, "hw_part_adj_pack: null strip");
  const StepTape T = a->layout->step(a->tape, j);
  return hw::halo_pack_planes(T.in[k - 1], 9, a->info.nx + 4, a->info.ny + 4, face, strip, a->v.stream);
}

int hw_part_adj_unpack(hw_part_adj* a, int j, int k, int face, int mode, const double* strip) {
  int rc = pa_stage(a, j, k, "hw_part_adj_unpack");
  if (!rc) rc = pa_face(face, "hw_part_adj_unpack");
  if (rc) return rc;
  if (!strip || mode < HW_HALO_NEIGHBOR || mode > HW_HALO_REPLICATE) return afail(HW_ERR_ARG, "hw_part_adj_unpack: bad argument");
  const StepTape T = a->layout->step(a->tape, j);
  return hw::halo_unpack_planes(T.in[k - 1], 9, a->info.nx + 4, a->info.ny + 4, face, mode,
                                face < 2 ? kStateOddX : kStateOddY, strip, a->v.stream);
}

int hw_part_adj_alpha_keys(hw_part_adj* a, int j, int k, unsigned long long* keys) {
  int rc = pa_stage(a, j, k, "hw_part_adj_alpha_keys");
  if (rc) return rc;
  if (!keys) return afail(HW_ERR_ARG, "hw_part_adj_alpha_keys: null keys");
  const StepTape T = a->layout->step(a->tape, j);
  hw::Dev2D d = *a->v.d2;
  for (int q = 0; q < 9; ++q) d.S[q] = T.in[k - 1][q];
  hw::launch_alpha2d(d, (unsigned long long*)a->keys, (int*)(a->B->lalpha + 2), a->v.stream);
  ACUDA(cudaMemcpyAsync(keys, a->keys, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, a->v.stream));
  return HW_OK;
}

int hw_part_adj_forward_stage(hw_part_adj* a, int j, int k, double dt, const unsigned long long* keys) {
  int rc = pa_stage(a, j, k, "hw_part_adj_forward_stage");
  if (rc) return rc;
  if (!keys || !(dt >= 0.0) || !(dt < 1e300)) return afail(HW_ERR_ARG, "hw_part_adj_forward_stage: bad argument");
  const hw::SolverView& v = a->v;
  cudaStream_t st = v.stream;
  const StepTape T = a->layout->step(a->tape, j);
  if (k == 1) ACUDA(cudaMemcpyAsync(v.dt, &dt, sizeof(double), cudaMemcpyHostToDevice, st));
  hw::Dev2D d = *v.d2;
  for (int q = 0; q < 9; ++q) d.S[q] = T.in[k - 1][q];
  for (int c = 0; c < 3; ++c) { d.X[3 + c] = T.dbx[k - 1][c]; d.Y[3 + c] = T.dby[k - 1][c]; }
  d.X[0] = T.fx[k - 1];
  d.Y[0] = T.fy[k - 1];
  hw::launch_finish_alpha2d(d, keys, T.alpha + 2 * (k - 1), nullptr, v.params->cfl, nullptr, -1.0, st);
  hw::launch_sweep_x2d(d, T.alpha + 2 * (k - 1), false, true, st);
  hw::launch_sweep_y2d(d, T.alpha + 2 * (k - 1), false, true, st);
  hw::StageArgs sa{};
  sa.k = k;
  sa.limiter = v.params->limiter;
  sa.dt = v.dt;
  for (int q = 0; q < 9; ++q) {
    sa.out[q] = k < 3 ? T.in[k][q] : T.out[q];
    sa.base[q] = v.base[q];
  }
  hw::launch_node2d(d, sa, hw::MODE_STAGE, false, true, st);
  if (k == 3 && a->nloc)
    hw::k_gather_eta_map<<<(a->nloc + 127) / 128, 128, 0, st>>>(T.out[0], a->d_map, a->d_map + a->nloc, a->nloc,
                                                              a->d_gvals + (size_t)j * a->ngauge);
  ACUDA(cudaGetLastError());
  return HW_OK;
}

int hw_part_adj_gauges(hw_part_adj* a, double* gvals) {
  int rc = pa_check(a, "hw_part_adj_gauges");
  if (rc) return rc;
  if (!gvals) return afail(HW_ERR_ARG, "hw_part_adj_gauges: null output");
  ACUDA(cudaMemcpyAsync(gvals, a->d_gvals, (size_t)a->nsteps * a->ngauge * sizeof(double), cudaMemcpyDeviceToHost,
                        a->v.stream));
  ACUDA(cudaStreamSynchronize(a->v.stream));
  return HW_OK;
}

int hw_part_adj_set_misfit(hw_part_adj* a, const double* gvals, const double* eta_obs, double* loss_out) {
  int rc = pa_check(a, "hw_part_adj_set_misfit");
  if (rc) return rc;
  if (!gvals || !eta_obs) return afail(HW_ERR_ARG, "hw_part_adj_set_misfit: null argument");
  if (loss_out) *loss_out = misfit_loss(gvals, eta_obs, (size_t)a->nsteps * a->ngauge);
  const size_t gb = (size_t)a->nsteps * a->ngauge * sizeof(double);
  cudaStream_t st = a->v.stream;
  ACUDA(cudaMemcpyAsync(a->d_gall, gvals, gb, cudaMemcpyHostToDevice, st));
  ACUDA(cudaMemcpyAsync(a->d_obs, eta_obs, gb, cudaMemcpyHostToDevice, st));
  ACUDA(cudaStreamSynchronize(st));
  a->cur = 0;
  rc = zero_planes(a->B->lam[0], 9, a->v.n, st);
  a->reverse = rc == HW_OK;
  a->have_last = false;
  return rc;
}

int hw_part_adj_reverse_stage(hw_part_adj* a, int j, int k, double dt, double* lalpha, int* argmax) {
  int rc = pa_stage(a, j, k, "hw_part_adj_reverse_stage");
  if (rc) return rc;
  if (!a->reverse) return afail(HW_ERR_STATE, "hw_part_adj_reverse_stage: call hw_part_adj_set_misfit first");
  if (!lalpha || !argmax) return afail(HW_ERR_ARG, "hw_part_adj_reverse_stage: null output");
  const hw::SolverView& v = a->v;
  cudaStream_t st = v.stream;
  if (k == 3) {  // the step's misfit seeds the adjoint of its output; the base adjoint starts at zero
    if (a->nloc)
      hw::k_loss_seed_map<<<(a->nloc + 127) / 128, 128, 0, st>>>(a->d_gall + (size_t)j * a->ngauge,
                                                                 a->d_obs + (size_t)j * a->ngauge, a->d_map,
                                                                 a->d_map + a->nloc, a->nloc, a->B->lam[a->cur][0]);
    if ((rc = zero_planes(a->B->lbase, 9, v.n, st))) return rc;
  }
  hw::AdjDev A = stage_args(v, a->B, a->layout->step(a->tape, j), dt, k, a->cur);
  A.lalpha = a->lal;
  A.argmax = (int*)(a->lal + 2);
  ACUDA(cudaMemsetAsync(a->lal, 0, 2 * sizeof(double), st));
  k_set_int2<<<1, 1, 0, st>>>(A.argmax, INT_MAX, INT_MAX);
  if ((rc = reverse_stage_body(v, a->B, A))) return rc;
  const hw_part_info& I = a->info;
  hw::k_adj_alpha_find_block<<<std::min((I.nx * I.ny + 255) / 256, 152 * 8), 256, 0, st>>>(A, I.nx, I.ny, I.i0, I.j0,
                                                                                        a->gnx);
  ACUDA(cudaGetLastError());
  double h[4];
  ACUDA(cudaMemcpyAsync(h, a->lal, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  ACUDA(cudaStreamSynchronize(st));
  lalpha[0] = h[0];
  lalpha[1] = h[1];
  std::memcpy(argmax, h + 2, 2 * sizeof(int));
  a->last = A;
  a->have_last = true;
  return HW_OK;
}

int hw_part_adj_alpha_apply(hw_part_adj* a, const double* lalpha, const int* argmax) {
  int rc = pa_check(a, "hw_part_adj_alpha_apply");
  if (rc) return rc;
  if (!a->have_last) return afail(HW_ERR_STATE, "hw_part_adj_alpha_apply: no reverse stage to complete");
  if (!lalpha || !argmax) return afail(HW_ERR_ARG, "hw_part_adj_alpha_apply: null argument");
  cudaStream_t st = a->v.stream;
  double h[4] = {lalpha[0], lalpha[1], 0.0, 0.0};
  std::memcpy(h + 2, argmax, 2 * sizeof(int));
  ACUDA(cudaMemcpyAsync(a->lal, h, 4 * sizeof(double), cudaMemcpyHostToDevice, st));
  const hw_part_info& I = a->info;
  hw::k_adj_alpha_apply_block<<<1, 1, 0, st>>>(a->last, I.nx, I.ny, I.i0, I.j0, a->gnx);
  ACUDA(cudaGetLastError());
  ACUDA(cudaStreamSynchronize(st));  // h is read by the copy
  a->cur ^= 1;  // the adjoint of the stage's input is now current
  a->have_last = false;
  return HW_OK;
}

int hw_part_adj_rpack(hw_part_adj* a, int what, int face, double* strip) {
  int rc = pa_check(a, "hw_part_adj_rpack");
  if (!rc) rc = pa_face(face, "hw_part_adj_rpack");
  if (rc) return rc;
  if ((what != 0 && what != 1) || !strip) return afail(HW_ERR_ARG, "hw_part_adj_rpack: bad argument");
  double* const* planes = what == 0 ? a->B->lam[a->cur] : a->B->lstatic_phys;
  return hw::halo_adj_pack_planes(planes, what == 0 ? 9 : 3, a->info.nx + 4, a->info.ny + 4, face, strip, a->v.stream);
}

int hw_part_adj_radd(hw_part_adj* a, int what, int face, int mode, const double* strip) {
  int rc = pa_check(a, "hw_part_adj_radd");
  if (!rc) rc = pa_face(face, "hw_part_adj_radd");
  if (rc) return rc;
  if ((what != 0 && what != 1) || !strip || mode < HW_HALO_NEIGHBOR || mode > HW_HALO_REPLICATE)
    return afail(HW_ERR_ARG, "hw_part_adj_radd: bad argument");
  double* const* planes = what == 0 ? a->B->lam[a->cur] : a->B->lstatic_phys;
  const unsigned odd = what == 0 ? (face < 2 ? kStateOddX : kStateOddY) : (face < 2 ? kStatOddX : kStatOddY);
  return hw::halo_adj_add_planes(planes, what == 0 ? 9 : 3, a->info.nx + 4, a->info.ny + 4, face, mode, odd, strip,
                                 a->v.stream);
}

int hw_part_adj_finish_static(hw_part_adj* a) {
  int rc = pa_check(a, "hw_part_adj_finish_static");
  if (rc) return rc;
  if ((rc = zero_planes(a->B->lstatic_phys, 3, a->v.n, a->v.stream))) return rc;
  return finish_static(a->v, a->B, a->B->lstatic_phys);
}

int hw_part_adj_gradients(hw_part_adj* a, double* const* grad_state, double* const* grad_static, int ld, int ptr_kind) {
  int rc = pa_check(a, "hw_part_adj_gradients");
  if (rc) return rc;
  if (!grad_state || !grad_static || ld < a->info.nx || (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE))
    return afail(HW_ERR_ARG, "hw_part_adj_gradients: bad argument");
  for (int q = 0; q < 9; ++q)
    if (!grad_state[q]) return afail(HW_ERR_ARG, "hw_part_adj_gradients: null plane");
  for (int q = 0; q < 3; ++q)
    if (!grad_static[q]) return afail(HW_ERR_ARG, "hw_part_adj_gradients: null plane");
  const hw::SolverView& v = a->v;
  cudaStream_t st = v.stream;
  const size_t n = v.n;
  const int nxe = a->info.nx + 4;
  hw::Ptr9 src{}, dst{};
  for (int q = 0; q < 9; ++q) { src.p[q] = a->B->lam[a->cur][q]; dst.p[q] = a->tmp + q * n; }
  hw::k_adj_convert<<<std::min((int)((n + 255) / 256), 152 * 8), 256, 0, st>>>((int)n, v.d2->dx, v.d2->dy, src, dst, 0);
  ACUDA(cudaGetLastError());
  const cudaMemcpyKind kind = ptr_kind == HW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int q = 0; q < 12; ++q) {
    const double* from = (q < 9 ? a->tmp + q * n : a->B->lstatic_phys[q - 9]) + 2 * (size_t)nxe + 2;
    double* to = q < 9 ? grad_state[q] : grad_static[q - 9];
    ACUDA(cudaMemcpy2DAsync(to, ld * sizeof(double), from, nxe * sizeof(double), a->info.nx * sizeof(double),
                            a->info.ny, kind, st));
  }
  ACUDA(cudaStreamSynchronize(st));
  return HW_OK;
}

}  // extern "C"
