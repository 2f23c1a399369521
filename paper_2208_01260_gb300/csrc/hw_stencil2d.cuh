// Stencil building blocks of the 2D scheme shared by the single-grid kernels (hw_kernels2d.cu) and
// the batched kernels (hw_batch.cu): boundary-mapped node loads, per-node flux records, one interface
// of a sweep (Sec. 2.1 Steps 1-2 along x or y, eq. mixed), the limiter along one direction (Sec. 2.2)
// and the node update (eq. swe-form-2d-dis, limiter, eq. RK). See hw_device.cuh for the conventions.
#pragma once
#include "hw_device.cuh"
#include "hw_internal.h"

namespace hw {

// ---------------------------------------------------------------------------------------------
// Loading a node with boundary mapping
// ---------------------------------------------------------------------------------------------
template <class R>
struct Node12T {
  R v[12];  // eta m w H1' M1' W1' H2' M2' W2' b bxs bys
};
using Node12 = Node12T<double>;

// Load of a plane that changes between launches. COH = false: through the read-only data path (valid
// while no block of the running kernel writes the plane). COH = true: an ordinary global load, for a
// kernel whose later phases read what its earlier phases wrote (a persistent kernel with grid
// barriers); the read-only path is not kept coherent with such writes.
template <bool COH, class T>
__device__ __forceinline__ T ldp(const T* p) {
  if constexpr (COH) return *p;
  else return __ldg(p);
}

// base: offset of the grid's first node in the node planes (0 unless the planes pool several grids).
template <bool COH = false, class R>
__device__ __forceinline__ void load_node(const Dev2DT<R>& d, int i, int j, Node12T<R>& n, size_t base = 0) {
  bool fx, fy;
  const int ii = map_index(i, d.nx, d.bc_x, fx);
  const int jj = map_index(j, d.ny, d.bc_y, fy);
  const size_t o = base + (size_t)jj * d.nx + ii;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    R x = ldp<COH>(d.S[q] + o);
    if (fx) x *= R(par_x2d(q));
    if (fy) x *= R(par_y2d(q));
    n.v[q] = x;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    R x = __ldg(d.stat[q] + o);
    if (fx) x *= R(par_x2d(9 + q));
    if (fy) x *= R(par_y2d(9 + q));
    n.v[9 + q] = x;
  }
}

// Per-node record a sweep keeps for its stencil (18 doubles).
enum { R_FP = 0, R_FM = 3, R_GP = 6, R_GM = 9, R_MIX = 12, R_H = 15, R_M = 16, R_W = 17, NREC = 18 };

// Pointwise fluxes of eq. (swe-form-2d-e) and their chain-rule derivatives of eq. (swe-form-2d-h),
// split with the global alpha (Sec. R(2.1) Step 1, without the factor 1/2). DIR = 0: x-sweep record
// (F1, d_x F1 for the split, d_y F1 for the mixed term); DIR = 1: y-sweep record (F2, d_y F2, d_x F2).
template <int DIR, class R, class M>
__device__ __forceinline__ void node_record_m(const Node12T<R>& n, R g, R alpha, R rec[NREC], M& mul) {
  const R eta = n.v[0], m = n.v[1], w = n.v[2], b = n.v[9];
  const R h = eta - b;
  const R rh = fast_rcp(h);
  const R u = mul(m, rh), v = mul(w, rh);
  const R gh = mul(g, h), ge = mul(g, eta);
  const R pres = mul(ge, fma(R(0.5), eta, -b));  // g/2 (eta^2 - 2 eta b)
  const R uv = mul(u, v);
  // derivative data along the sweep (split) and across it (mixed)
  const int qs = DIR == 0 ? 3 : 6, qm = DIR == 0 ? 6 : 3;
  const R Hs = n.v[qs], Ms = n.v[qs + 1], Ws = n.v[qs + 2], Bs = n.v[DIR == 0 ? 10 : 11];
  const R Hm = n.v[qm], Mm = n.v[qm + 1], Wm = n.v[qm + 2], Bm = n.v[DIR == 0 ? 11 : 10];
  R F[3], Gs[3], Gm[3];
  const R mv = mul(m, v);
  if (DIR == 0) {
    const R uu = mul(u, u), a1 = gh - uu, a2 = uu - ge, u2 = u + u;
    F[0] = m; F[1] = fma(m, u, pres); F[2] = mv;
    Gs[0] = Ms;
    Gs[1] = fma(u2, Ms, fma(a1, Hs, mul(a2, Bs)));
    Gs[2] = fma(uv, Bs - Hs, fma(v, Ms, mul(u, Ws)));
    Gm[0] = Mm;
    Gm[1] = fma(u2, Mm, fma(a1, Hm, mul(a2, Bm)));
    Gm[2] = fma(uv, Bm - Hm, fma(v, Mm, mul(u, Wm)));
  } else {
    const R vv = mul(v, v), a1 = gh - vv, a2 = vv - ge, v2 = v + v;
    F[0] = w; F[1] = mv; F[2] = fma(w, v, pres);
    Gs[0] = Ws;
    Gs[1] = fma(uv, Bs - Hs, fma(v, Ms, mul(u, Ws)));
    Gs[2] = fma(v2, Ws, fma(a1, Hs, mul(a2, Bs)));
    Gm[0] = Wm;
    Gm[1] = fma(uv, Bm - Hm, fma(v, Mm, mul(u, Wm)));
    Gm[2] = fma(v2, Wm, fma(a1, Hm, mul(a2, Bm)));
  }
  const R U[3] = {eta, m, w}, D[3] = {Hs, Ms, Ws};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    rec[R_FP + c] = fma(alpha, U[c], F[c]);
    rec[R_FM + c] = fma(-alpha, U[c], F[c]);
    rec[R_GP + c] = fma(alpha, D[c], Gs[c]);
    rec[R_GM + c] = fma(-alpha, D[c], Gs[c]);
    rec[R_MIX + c] = Gm[c];
  }
  rec[R_H] = h;
  rec[R_M] = m;
  rec[R_W] = w;
}

// The record on the FP64 pipe (moving its products to the integer pipes measured slower).
template <int DIR, class R>
__device__ __forceinline__ void node_record(const Node12T<R>& n, R g, R alpha, R rec[NREC]) {
  MulFP64 mf;
  node_record_m<DIR>(n, g, alpha, rec, mf);
}

// ---------------------------------------------------------------------------------------------
// One interface from the four stencil records (nodes i-1, i, i+1, i+2 along the sweep).
// Outputs (12): 2 Fhat, 2 bhat, 24 dS Ghat (derivative-equation flux), 12 dT Mhat (mixed term),
// where dS is the spacing along the sweep and dT the spacing across it.
// qb[6] = source candidates q_1..q_3 of (b, dS b_s) for the '+' side then the mirrored '-' side.
// ---------------------------------------------------------------------------------------------
// `mul` forms the products and reciprocals (MulFP64 or MulIntT, see hw_device.cuh).
template <int DIR, bool LINEAR, bool CHAR, class R, class M>
__device__ __forceinline__ void interface_values_m(const R* r0, const R* r1, const R* r2,
                                                   const R* r3, int stride, const R qb[6], R g,
                                                   R eps_w, R out[12], M& mul) {
#define RV(r, f) (r)[(f) * stride]
  // interface state: h = (h_i + h_{i+1})/2, u = (m_i + m_{i+1})/(h_i + h_{i+1}), v likewise
  const R hs = RV(r1, R_H) + RV(r2, R_H);
  const R rhs = mul.rcp(hs);
  const R ub = mul(RV(r1, R_M) + RV(r2, R_M), rhs);
  const R vb = mul(RV(r1, R_W) + RV(r2, R_W), rhs);
  const R gh = mul(mul.k(R(0.5), g), hs);
  const R rs = fast_rsqrt(gh);
  const R ic2 = mul.k(R(0.5), rs);  // 1/(2c)
  // normal / tangential velocity of this sweep
  const R un = DIR == 0 ? ub : vb, ut = DIR == 0 ? vb : ub;
  // un +- c with c = gh / sqrt(gh): fmas (a product on the integer pipes would leave the adds)
  const R upc = fma(gh, rs, un), umc = fma(-gh, rs, un);
  // component indices: normal momentum and tangential momentum
  const int cn = DIR == 0 ? 1 : 2, ct = DIR == 0 ? 2 : 1;
  // scaled epsilon: fields 1, 3 carry s = 4c, field 2 carries s = 2 (both 2 without projection)
  const R eps2 = mul.k(R(4.0), eps_w);
  const R eps13 = CHAR ? mul(mul(mul.k(R(8.0), g), eps_w), hs) : eps2;

  R G[3], GB1 = R(0.0), GB3 = R(0.0);  // per-field sums over both sides; source fields 1 and 3
  const R* rp[4] = {r0, r1, r2, r3};
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    // '+' uses nodes 0,1,2 of (F+, G+); '-' uses nodes 3,2,1 of (F-, G-) with the derivative negated.
    const int o0 = side == 0 ? 0 : 3, o1 = side == 0 ? 1 : 2, o2 = side == 0 ? 2 : 1;
    const int fo = side == 0 ? R_FP : R_FM, go = side == 0 ? R_GP : R_GM;
    const R sg = side == 0 ? R(1.0) : -R(1.0);
    R f[3][3], p[3][3];  // [field][stencil point]
    const int os[3] = {o0, o1, o2};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const R* r = rp[os[t]];
      const R F0 = RV(r, fo), Fn = RV(r, fo + cn), Ft = RV(r, fo + ct);
      const R G0 = sg * RV(r, go), Gn = sg * RV(r, go + cn), Gt = sg * RV(r, go + ct);
      if (CHAR) {
        // rows of L without 1/(2c): (un+c, -1, 0), (-ut, 0, 1), (-(un-c), 1, 0) on (rho, normal, tangential)
        f[0][t] = fma(upc, F0, -Fn);
        f[1][t] = fma(-ut, F0, Ft);
        f[2][t] = fma(-umc, F0, Fn);
        p[0][t] = fma(upc, G0, -Gn);
        p[1][t] = fma(-ut, G0, Gt);
        p[2][t] = fma(-umc, G0, Gn);
      } else {
        f[0][t] = F0; f[1][t] = Fn; f[2][t] = Ft;
        p[0][t] = G0; p[1][t] = Gn; p[2][t] = Gt;
      }
    }
    const R* qbs = qb + 3 * side;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      WeightsT<R> W;
      const R e = (k == 1) ? eps2 : eps13;
      const R v = hweno_side_m<LINEAR>(f[k][0], f[k][1], f[k][2], p[k][0], p[k][1], p[k][2], e, W, mul);
      G[k] = side == 0 ? v : G[k] + v;
      if (CHAR) {
        // source data per field: (-b, 0, +b) (row entries of the normal-momentum column)
        if (k == 0) GB1 -= weighted_m(W, qbs[0], qbs[1], qbs[2], mul);
        if (k == 2) GB3 += weighted_m(W, qbs[0], qbs[1], qbs[2], mul);
      } else {
        if (k == 1) GB1 += weighted_m(W, qbs[0], qbs[1], qbs[2], mul);  // the normal-momentum component itself
      }
    }
  }
  // back to physical components: 2 Fhat = R diag(1/s) G * 2
  R F2[3], B2[3];
  if (CHAR) {
    const R A = mul(G[0] + G[2], ic2);
    F2[0] = A;
    F2[cn] = fma(un, A, mul.k(R(0.5), G[2] - G[0]));
    F2[ct] = fma(ut, A, G[1]);
    const R Bs = mul(GB1 + GB3, ic2);
    B2[0] = Bs;
    B2[cn] = fma(un, Bs, mul.k(R(0.5), GB3 - GB1));
    B2[ct] = mul(ut, Bs);
  } else {
    F2[0] = G[0]; F2[cn] = G[1]; F2[ct] = G[2];
    B2[0] = R(0.0); B2[cn] = GB1; B2[ct] = R(0.0);
  }
  // derivative-equation flux (eq. Rec-phi, component-wise): 24 dS Ghat = 3 fpart + gpart
  // mixed term (eq. mixed): 12 dT Mhat = 7 (X_i + X_{i+1}) - (X_{i-1} + X_{i+2})
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R fpart =
        fma(R(7.0), RV(r2, R_FP + c) - RV(r1, R_FM + c),
            fma(R(8.0), RV(r2, R_FM + c) - RV(r1, R_FP + c), RV(r0, R_FP + c) - RV(r3, R_FM + c)));
    const R gpart = fma(-R(5.0), RV(r2, R_GP + c) + RV(r1, R_GM + c),
                             fma(-R(2.0), RV(r1, R_GP + c) + RV(r2, R_GM + c), RV(r0, R_GP + c) + RV(r3, R_GM + c)));
    out[c] = F2[c];
    out[3 + c] = B2[c];
    out[6 + c] = fma(R(3.0), fpart, gpart);
    out[9 + c] = fma(R(7.0), RV(r1, R_MIX + c) + RV(r2, R_MIX + c), -(RV(r0, R_MIX + c) + RV(r3, R_MIX + c)));
  }
#undef RV
}

// One interface. IMUL: the products run on the integer pipes (hw_fp64_int.h: each product is
// bit-identical to DMUL, but rounded on its own where the FP64 form may fuse it with an add into an fma,
// so the results differ from the FP64-pipe form by rounding; the reciprocals stay on the FP64 pipe:
// moving them raised spills); if any of them leaves the integer fast path (subnormal, infinite or NaN
// data), the interface is recomputed on the FP64 pipe from the same records.
template <int DIR, bool LINEAR, bool CHAR, bool IMUL = false, class R>
__device__ __forceinline__ void interface_values(const R* r0, const R* r1, const R* r2,
                                                 const R* r3, int stride, const R qb[6], R g,
                                                 R eps_w, R out[12]) {
  if constexpr (IMUL && !LINEAR && std::is_same<R, double>::value) {
    MulIntT<false> mi;
    interface_values_m<DIR, LINEAR, CHAR>(r0, r1, r2, r3, stride, qb, g, eps_w, out, mi);
    if (mi.bad) {
      MulFP64 mf;
      interface_values_m<DIR, LINEAR, CHAR>(r0, r1, r2, r3, stride, qb, g, eps_w, out, mf);
    }
  } else {
    MulFP64 mf;
    interface_values_m<DIR, LINEAR, CHAR>(r0, r1, r2, r3, stride, qb, g, eps_w, out, mf);
  }
}

// ---------------------------------------------------------------------------------------------
// alpha_x, alpha_y = max over nodes of |u| + c, |v| + c (exact max via ordered 64-bit keys) in two
// passes that keep the FP64 pipe out of most nodes: a coarse pass evaluates |u| + c in float (from the
// depth formed in double, converted by integer operations) and reduces the float maxima M; an exact pass
// re-evaluates every node in float and computes the double value only where the float one is within a
// relative 1e-5 of M (or cannot be trusted: values outside float's range, NaN, infinity). The float
// values are within about 1e-6 of the double ones, so the node attaining the double maximum is always
// re-evaluated and the result is the exact double maximum (a re-evaluated node contributes to both
// directions, which is harmless: no node's value exceeds a direction's maximum).
// ---------------------------------------------------------------------------------------------
// double -> float by truncation with integer operations (the FP64 pipe stays free): relative error
// below 2^-23 for values in float's normal range. Values below it become 0 (tiny is true); values
// above it, infinities and NaN set huge.
__device__ __forceinline__ float d2f_trunc(double x, bool& tiny, bool& huge) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  tiny = e <= 1023 - 127;
  huge = e >= 1023 + 128;
  const unsigned int sign = (unsigned int)((unsigned long long)b >> 32) & 0x80000000u;
  const unsigned int f = sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)((b >> 29) & 0x7fffff);
  return tiny ? 0.0f : __uint_as_float(f);
}

// Float estimates of |u| + c and |v| + c at node o from the depth formed in double. exact: the node
// needs the double evaluation regardless (a depth or momentum outside float's range, NaN, infinity);
// neg: the depth is negative.
template <bool COH = false>
__device__ __forceinline__ void alpha_coarse(const Dev2D& d, size_t o, float& ax, float& ay, bool& exact,
                                             bool& neg) {
  const double hd = ldp<COH>(d.S[0] + o) - __ldg(d.stat[0] + o);
  bool t0, h0, t1, h1, t2, h2;
  const float h = d2f_trunc(hd, t0, h0);
  const float m = d2f_trunc(ldp<COH>(d.S[1] + o), t1, h1);
  const float w = d2f_trunc(ldp<COH>(d.S[2] + o), t2, h2);
  exact = t0 || h0 || h1 || h2;
  neg = h < 0.0f;
  const float rh = fast_rcp(h);
  const float gh = (float)d.g * h;
  const float c = gh * fast_rsqrt(gh);
  ax = fabsf(m) * rh + c;
  ay = fabsf(w) * rh + c;
}

// The exact pass over nodes o = begin, begin + step, ... < end, with the coarse maxima m32[0..1]: keys of
// the double maxima into kx, ky and status flags into bad.
// The double evaluation of the exact pass at node o: keys of |u| + c and |v| + c into kx, ky (maxima),
// status flags into bad.
template <bool COH = false>
__device__ __forceinline__ void alpha_exact_node(const Dev2D& d, size_t o, unsigned long long& kx,
                                                 unsigned long long& ky, int& bad) {
  const double hd = ldp<COH>(d.S[0] + o) - __ldg(d.stat[0] + o);
  if (!(hd > 0.0) || !(hd < 1e300)) {
    bad |= hd == hd ? HW_STATUS_DEPTH : HW_STATUS_NONFINITE;
    return;
  }
  const double rh = fast_rcp(hd);
  const double gh = d.g * hd;
  const double c = gh * fast_rsqrt(gh);
  const double ax = dabs(ldp<COH>(d.S[1] + o) * rh) + c, ay = dabs(ldp<COH>(d.S[2] + o) * rh) + c;
  if (!(ax < 1e300) || !(ay < 1e300)) {
    bad |= HW_STATUS_NONFINITE;
    return;
  }
  kx = max(kx, dkey(ax));
  ky = max(ky, dkey(ay));
}

// Whether the exact pass evaluates a node, from its coarse estimates and the thresholds tx, ty (the coarse
// maxima lowered by the estimates' error bound).
__device__ __forceinline__ bool alpha_needs_exact(float fx, float fy, bool exact, bool neg, float tx, float ty) {
  return exact || (!neg && !(fx < tx && fy < ty));
}

template <bool COH = false>
__device__ __forceinline__ void alpha_exact_range(const Dev2D& d, const unsigned int* m32, size_t begin, size_t end,
                                                  size_t step, unsigned long long& kx, unsigned long long& ky,
                                                  int& bad) {
  const float tx = __uint_as_float(m32[0]) * (1.0f - 1e-5f), ty = __uint_as_float(m32[1]) * (1.0f - 1e-5f);
  for (size_t o = begin; o < end; o += step) {
    float fx, fy;
    bool exact, neg;
    alpha_coarse<COH>(d, o, fx, fy, exact, neg);
    if (alpha_needs_exact(fx, fy, exact, neg, tx, ty)) alpha_exact_node<COH>(d, o, kx, ky, bad);
  }
}

// ---------------------------------------------------------------------------------------------
// Sweep tiles over flattened extended lines (shared by the single-grid and the batched kernels).
// x: extended node E = j (nx + 4) + e stands for node (e - 2, j), e = 0 .. nx + 3 (each row with two halo
// nodes on either side, rows one after the other); the x-interface k of row j (between nodes k - 1 and k,
// k = 0 .. nx) sits at E = j (nx + 4) + k and reads the records of E .. E + 3, all in its row.
// y: the same over groups of yc adjacent columns: extended row E = g (ny + 4) + e of group g stands for
// nodes (g yc + c, e - 2), c = 0 .. yc - 1.
// A tile of TILE_T threads forms the node records of TILE_T consecutive extended nodes (x; yc columns of
// TILE_T / yc extended rows in y), then, after one barrier, the interfaces whose four records lie in the
// tile: tiles run across line ends, so no grid size leaves a ragged tile. All TILE_T threads must call;
// sm holds NREC * TILE_T values. on / oi: offsets of the grid in pooled node / interface planes (the
// batched form keeps the planes' base pointers in the kernel parameters and adds these, so that no
// per-grid pointer occupies a register). COH: state loads as in ldp.
// ---------------------------------------------------------------------------------------------
constexpr int TILE_T = 192;

template <bool LINEAR, bool CHAR, bool IMUL, bool COH = false, class R>
__device__ __forceinline__ void sweep_x_tile(const Dev2DT<R>& d, R ax, unsigned E0, R* sm, size_t on = 0,
                                             size_t oi = 0) {
  const unsigned W = d.nx + 4, total = (unsigned)d.ny * W;
  const int t = threadIdx.x;
  {
    const unsigned E = E0 + t;
    if (E < total) {
      const unsigned j = E / W, e = E - j * W;
      Node12T<R> n;
      load_node<COH>(d, (int)e - 2, (int)j, n, on);
      R rec[NREC];
      node_record<0>(n, R(d.g), ax, rec);
#pragma unroll
      for (int f = 0; f < NREC; ++f) sm[f * TILE_T + t] = rec[f];
    }
  }
  __syncthreads();
  const unsigned E = E0 + t;
  if (t >= TILE_T - 3 || E >= total) return;
  const unsigned j = E / W, k = E - j * W;
  if (k > (unsigned)d.nx) return;
  const size_t o = oi + (size_t)j * (d.nx + 1) + k;
  R qb[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) qb[q] = __ldg(d.qbx[q] + o);
  R out[12];
  interface_values<0, LINEAR, CHAR, IMUL>(sm + t, sm + t + 1, sm + t + 2, sm + t + 3, TILE_T, qb, R(d.g), R(d.eps_w), out);
#pragma unroll
  for (int q = 0; q < 12; ++q) d.X[q][o] = out[q];
}

template <bool LINEAR, bool CHAR, bool IMUL, bool COH = false, class R>
__device__ __forceinline__ void sweep_y_tile(const Dev2DT<R>& d, R ay, unsigned E0, int yc, R* sm, size_t on = 0,
                                             size_t oi = 0) {
  const int rows = TILE_T / yc, ifs = rows - 3;
  const unsigned H = d.ny + 4, total = (unsigned)((d.nx + yc - 1) / yc) * H;
  const int t = threadIdx.x, c = t % yc, r = t / yc;
  {
    const unsigned E = E0 + r;
    if (r < rows && E < total) {
      const unsigned g = E / H, e = E - g * H;
      const int i = (int)g * yc + c;
      if (i < d.nx) {
        Node12T<R> n;
        load_node<COH>(d, i, (int)e - 2, n, on);
        R rec[NREC];
        node_record<1>(n, R(d.g), ay, rec);
#pragma unroll
        for (int f = 0; f < NREC; ++f) sm[f * TILE_T + t] = rec[f];
      }
    }
  }
  __syncthreads();
  const unsigned E = E0 + r;
  if (r >= ifs || E >= total) return;
  const unsigned g = E / H, k = E - g * H;
  const int i = (int)g * yc + c;
  if (k > (unsigned)d.ny || i >= d.nx) return;
  const size_t o = oi + (size_t)k * d.nx + i;
  R qb[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) qb[q] = __ldg(d.qby[q] + o);
  R out[12];
  const R* s0 = sm + t;
  interface_values<1, LINEAR, CHAR, IMUL>(s0, s0 + yc, s0 + 2 * yc, s0 + 3 * yc, TILE_T, qb, R(d.g), R(d.eps_w), out);
#pragma unroll
  for (int q = 0; q < 12; ++q) d.Y[q][o] = out[q];
}

// ---------------------------------------------------------------------------------------------
// Node kernel: RHS assembly, limiter, RK combination (or the bare RHS).
// ---------------------------------------------------------------------------------------------
// Limiter along one direction at one node (Sec. R(2.2)), scaled data. L-rows without 1/(2c):
// x: (u+c, -1, 0), (-v, 0, 1), (-(u-c), 1, 0); y: (v+c, 0, -1), (-u, 1, 0), (-(v-c), 0, 1).
template <int DIR, bool LINEAR, bool CHAR, class R, class M>
__device__ __forceinline__ void limit_dir(const R Um[3], const R U0[3], const R Up[3],
                                          const R Dm[3], const R Dp[3], R u, R v, R c,
                                          R ic2, R gh, R eps, R out[3], M& mul) {
  const int cn = DIR == 0 ? 1 : 2, ct = DIR == 0 ? 2 : 1;
  const R un = DIR == 0 ? u : v, ut = DIR == 0 ? v : u;
  const R upc = un + c, umc = un - c;
  auto proj = [&](const R* a, R o[3]) {
    if (CHAR) {
      o[0] = fma(upc, a[0], -a[cn]);
      o[1] = fma(-ut, a[0], a[ct]);
      o[2] = fma(-umc, a[0], a[cn]);
    } else {
      o[0] = a[0]; o[1] = a[cn]; o[2] = a[ct];
    }
  };
  R m0[3], m1[3], m2[3], nl[3], nr[3];
  proj(Um, m0); proj(U0, m1); proj(Up, m2); proj(Dm, nl); proj(Dp, nr);
  const R e13 = CHAR ? mul(mul.k(R(4.0), eps), gh) : eps;
  R nu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) nu[k] = limiter_field_m<LINEAR>(m0[k], m1[k], m2[k], nl[k], nr[k], k == 1 ? eps : e13, mul);
  if (CHAR) {
    const R A = mul(nu[0] + nu[2], ic2);
    out[0] = A;
    out[cn] = fma(un, A, mul.k(R(0.5), nu[2] - nu[0]));
    out[ct] = fma(ut, A, nu[1]);
  } else {
    out[0] = nu[0]; out[cn] = nu[1]; out[ct] = nu[2];
  }
}

// RHS assembly, limiter and RK combination (or the bare RHS) at node (i, j) of one grid, products
// formed by `mul`. With MulInt nothing is written when a product left the integer fast path
// (mul.bad); the caller then recomputes the node with MulFP64 from the same (unchanged) inputs.
// on, oxo, oyo: offsets of the grid in pooled node, x-interface and y-interface planes (0 for one grid).
// COH: loads of the state, interface and base planes as in ldp.
template <int MODE, bool LINEAR, bool CHAR, bool COH, class R, class M>
__device__ __forceinline__ void node_update_m(const Dev2DT<R>& d, const StageArgsT<R>& sa, int i, int j, M& mul,
                                              size_t on = 0, size_t oxo = 0, size_t oyo = 0) {
  const size_t o = on + (size_t)j * d.nx + i;
  const size_t ox = oxo + (size_t)j * (d.nx + 1) + i;  // left x-interface; right is ox + 1
  const size_t oy = oyo + (size_t)j * d.nx + i;        // lower y-interface; upper is oy + nx
  R cur[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) cur[q] = ldp<COH>(d.S[q] + o);
  if (MODE == MODE_STAGE && !(*sa.dt > 0.0)) {
    // a step of size 0 (e.g. clipped at the end time) leaves the state unchanged
#pragma unroll
    for (int q = 0; q < 9; ++q) sa.out[q][o] = cur[q];
    return;
  }
  const R eta = cur[0], H1 = cur[3], H2 = cur[6];
  const R g = R(d.g);
  // grid constants in the working precision
  const R c_bx = R(d.c_bx), c_by = R(d.c_by), c_gx = R(d.c_gx), c_gy = R(d.c_gy), c_mx = R(d.c_mx),
          c_my = R(d.c_my);
  const R ge = mul(g, eta);
  // ---- RHS (eq. swe-form-2d-dis) in scaled units: R_U, dx R_V, dy R_Q ----
  R Rv[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R dFx = ldp<COH>(d.X[c] + ox + 1) - ldp<COH>(d.X[c] + ox);
    const R dFy = ldp<COH>(d.Y[c] + oy + d.nx) - ldp<COH>(d.Y[c] + oy);
    const R dbx = ldp<COH>(d.X[3 + c] + ox + 1) - ldp<COH>(d.X[3 + c] + ox);
    const R dby = ldp<COH>(d.Y[3 + c] + oy + d.nx) - ldp<COH>(d.Y[3 + c] + oy);
    const R dGx = ldp<COH>(d.X[6 + c] + ox + 1) - ldp<COH>(d.X[6 + c] + ox);
    const R dGy = ldp<COH>(d.Y[6 + c] + oy + d.nx) - ldp<COH>(d.Y[6 + c] + oy);
    const R dMx = ldp<COH>(d.X[9 + c] + ox + 1) - ldp<COH>(d.X[9 + c] + ox);
    const R dMy = ldp<COH>(d.Y[9 + c] + oy + d.nx) - ldp<COH>(d.Y[9 + c] + oy);
    const R db = fma(c_bx, dbx, mul(c_by, dby));  // [b~]_x/dx + [b-]_y/dy
    Rv[c] = fma(-ge, db, fma(-c_bx, dFx, -mul(c_by, dFy)));
    R rv = fma(-c_gx, dGx, -mul(c_my, dMy));
    R rq = fma(-c_mx, dMx, -mul(c_gy, dGy));
    if (c > 0) {
      rv = fma(-ge, __ldg(d.sv[c - 1] + o), rv);
      rq = fma(-ge, __ldg(d.sq[c - 1] + o), rq);
    }
    Rv[3 + c] = fma(-mul(g, H1), db, rv);
    Rv[6 + c] = fma(-mul(g, H2), db, rq);
  }
  if (MODE == MODE_RHS) {
    if (mul.bad) return;
    // physical units: R_V = (dx R_V)/dx, R_Q = (dy R_Q)/dy
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const R s = q < 3 ? R(1.0) : R(q < 6 ? d.inv_dx : d.inv_dy);
      sa.rhs_out[q][o] = mul(Rv[q], s);
    }
    return;
  }
  // ---- limiter (Sec. R(2.2), dimension by dimension) ----
  R mod[6];
  if (sa.limiter) {
    const R b0 = __ldg(d.stat[0] + o);
    const R h = eta - b0;
    const R gh = mul(g, h);
    const R rh = mul.rcp(h);
    const R u = mul(cur[1], rh), v = mul(cur[2], rh);
    const R rs = fast_rsqrt(gh);
    const R c = mul(gh, rs), ic2 = mul.k(R(0.5), rs);
    Node12T<R> nm, np;
    // x neighbours
    load_node<COH>(d, i - 1, j, nm, on);
    load_node<COH>(d, i + 1, j, np, on);
    limit_dir<0, LINEAR, CHAR>(nm.v, cur, np.v, nm.v + 3, np.v + 3, u, v, c, ic2, gh, R(d.eps_lim), mod, mul);
    load_node<COH>(d, i, j - 1, nm, on);
    load_node<COH>(d, i, j + 1, np, on);
    limit_dir<1, LINEAR, CHAR>(nm.v, cur, np.v, nm.v + 6, np.v + 6, u, v, c, ic2, gh, R(d.eps_lim), mod + 3, mul);
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) mod[q] = cur[3 + q];
  }
  // ---- SSP-RK3 combination (eq. RK) ----
  const R dt = R(*sa.dt);
  if (sa.k == 1) {
    if (mul.bad) return;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const R cq = q < 3 ? cur[q] : mod[q - 3];
      if (sa.base) sa.base[q][o] = cq;
      sa.out[q][o] = fma(dt, Rv[q], cq);
    }
  } else {
    const R a = sa.k == 2 ? R(0.75) : R(1.0) / R(3.0);
    const R b = sa.k == 2 ? R(0.25) : R(2.0) / R(3.0);
    R res[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const R cq = q < 3 ? cur[q] : mod[q - 3];
      res[q] = fma(a, ldp<COH>(sa.base[q] + o), mul(b, fma(dt, Rv[q], cq)));
    }
    if (mul.bad) return;
#pragma unroll
    for (int q = 0; q < 9; ++q) sa.out[q][o] = res[q];
  }
}

// The node update. IMUL: products on the integer pipes (each bit-identical to DMUL; results differ from
// the fma-contracted FP64-pipe form by rounding); if any leaves the integer fast path, the node is
// recomputed on the FP64 pipe, so an interface or node on that fallback rounds differently from its
// neighbours, within the same tolerances (int_mul_fallback parity case).
template <int MODE, bool LINEAR, bool CHAR, bool IMUL = false, bool COH = false, class R>
__device__ __forceinline__ void node_update(const Dev2DT<R>& d, const StageArgsT<R>& sa, int i, int j, size_t on = 0,
                                            size_t oxo = 0, size_t oyo = 0) {
  if constexpr (IMUL && !LINEAR && std::is_same<R, double>::value) {
    MulInt mi;
    node_update_m<MODE, LINEAR, CHAR, COH>(d, sa, i, j, mi, on, oxo, oyo);
    if (mi.bad) {
      MulFP64 mf;
      node_update_m<MODE, LINEAR, CHAR, COH>(d, sa, i, j, mf, on, oxo, oyo);
    }
  } else {
    MulFP64 mf;
    node_update_m<MODE, LINEAR, CHAR, COH>(d, sa, i, j, mf, on, oxo, oyo);
  }
}

}  // namespace hw
