// Hand-written reverse (adjoint) of the stencil building blocks in hw_device.cuh and hw_stencil2d.cuh,
// for the nonlinear, characteristic-projected scheme. Each function recomputes the forward values it
// needs from the same inputs and propagates adjoints through every operation in reverse order. The
// refined reciprocal and reciprocal square root are differentiated as the exact functions (their
// results are accurate to a few ulp).
#pragma once
#include "hw_stencil2d.cuh"

namespace hw {

// Reverse of hweno_side<false> (Sec. 2.1 eqs. HWEp1, GHYZZ, Rec-f). Inputs: forward data f, p, eps;
// the adjoint lv of the weighted value. With SRC, the same weights also reconstruct a source from the
// candidates qbs[3] (Sec. 2.1 Step 2) whose value has adjoint lw: its adjoint reaches the weight
// numerators and normaliser here and the candidates through lqbs (added). Outputs: adjoints of f, p
// (added); returns the adjoint of eps.
template <bool SRC>
__device__ __forceinline__ double hweno_side_rev(const double f[3], const double p[3], double eps, double lv,
                                                 const double* qbs, double lw, double* lqbs, double lf[3],
                                                 double lp[3]) {
  // forward
  const double d1 = f[0] - f[1], d2 = f[1] - f[2];
  const double B1 = fma(2.0, d1, p[0] + p[1]);
  const double A1 = B1 + (d1 + p[1]);
  const double B2 = fma(2.0, d2, p[1] + p[2]);
  const double A2 = B2 + (d2 + p[1]);
  const double P = fma(0.5, p[1], f[1]);
  const double e = fma(-2.0, f[1], f[0] + f[2]);
  const double q1 = fma(1.0 / 6.0, A1, P);
  const double q2 = fma(-1.0 / 6.0, A2, P);
  const double q3 = fma(1.0 / 12.0, e, P);
  const double g3 = fma(2.0, p[1], f[0] - f[2]);
  const double pp = p[1] * p[1];
  const double b1 = fma((781.0 / 20.0) * B1, B1, fma((13.0 / 3.0) * A1, A1, pp));
  const double b2 = fma((781.0 / 20.0) * B2, B2, fma((13.0 / 3.0) * A2, A2, pp));
  const double b3 = fma((781.0 / 80.0) * g3, g3, fma((13.0 / 12.0) * e, e, pp));
  const double t1 = b1 + eps, t2 = b2 + eps, t3 = b3 + eps;
  const double s1 = t1 * t1, s2 = t2 * t2, s3 = t3 * t3;
  const double n1 = s2 * s3, n2 = s1 * s3, n3 = (4.0 / 3.0) * (s1 * s2);
  const double r = fast_rcp(n1 + n2 + n3);
  const double num = fma(n1, q1, fma(n2, q2, n3 * q3));
  // reverse: source value S r with S = n1 qb1 + n2 qb2 + n3 qb3
  double ln1 = 0.0, ln2 = 0.0, ln3 = 0.0, lr = 0.0;
  if (SRC) {
    const double rw = r * lw;
    ln1 = qbs[0] * rw;
    ln2 = qbs[1] * rw;
    ln3 = qbs[2] * rw;
    lr = fma(n1, qbs[0], fma(n2, qbs[1], n3 * qbs[2])) * lw;
    lqbs[0] += n1 * rw;
    lqbs[1] += n2 * rw;
    lqbs[2] += n3 * rw;
  }
  // reverse of the weighted value
  const double lnum = r * lv;
  const double lrt = fma(num, lv, lr);
  const double lden = -r * r * lrt;
  const double ln1t = fma(q1, lnum, ln1 + lden);
  const double ln2t = fma(q2, lnum, ln2 + lden);
  const double ln3t = fma(q3, lnum, ln3 + lden);
  const double lq1 = n1 * lnum, lq2 = n2 * lnum, lq3 = n3 * lnum;
  const double ls1 = fma(s3, ln2t, (4.0 / 3.0) * s2 * ln3t);
  const double ls2 = fma(s3, ln1t, (4.0 / 3.0) * s1 * ln3t);
  const double ls3 = fma(s2, ln1t, s1 * ln2t);
  const double lb1 = 2.0 * t1 * ls1, lb2 = 2.0 * t2 * ls2, lb3 = 2.0 * t3 * ls3;
  const double leps = lb1 + lb2 + lb3;
  double lB1 = 2.0 * (781.0 / 20.0) * B1 * lb1;
  double lA1 = 2.0 * (13.0 / 3.0) * A1 * lb1;
  double lB2 = 2.0 * (781.0 / 20.0) * B2 * lb2;
  double lA2 = 2.0 * (13.0 / 3.0) * A2 * lb2;
  const double lg3 = 2.0 * (781.0 / 80.0) * g3 * lb3;
  double le = 2.0 * (13.0 / 12.0) * e * lb3;
  const double lpp = lb1 + lb2 + lb3;
  double lp1 = 2.0 * p[1] * lpp + 2.0 * lg3;
  double lf0 = lg3, lf2 = -lg3, lf1 = 0.0;
  le = fma(1.0 / 12.0, lq3, le);
  const double lP = lq1 + lq2 + lq3;
  lA2 = fma(-1.0 / 6.0, lq2, lA2);
  lA1 = fma(1.0 / 6.0, lq1, lA1);
  lf0 += le;
  lf2 += le;
  lf1 -= 2.0 * le;
  lf1 += lP;
  lp1 += 0.5 * lP;
  // A2 = B2 + d2 + p1; B2 = 2 d2 + p1 + p2
  lB2 += lA2;
  double ld2 = lA2;
  lp1 += lA2;
  ld2 += 2.0 * lB2;
  lp1 += lB2;
  const double lp2 = lB2;
  // A1 = B1 + d1 + p1; B1 = 2 d1 + p0 + p1
  lB1 += lA1;
  double ld1 = lA1;
  lp1 += lA1;
  ld1 += 2.0 * lB1;
  const double lp0 = lB1;
  lp1 += lB1;
  lf1 += ld2;
  lf2 -= ld2;
  lf0 += ld1;
  lf1 -= ld1;
  lf[0] += lf0; lf[1] += lf1; lf[2] += lf2;
  lp[0] += lp0; lp[1] += lp1; lp[2] += lp2;
  return leps;
}

// Reverse of limiter_field<false> (eqs. step1-dxi, limiter-1d). Returns adjoint of eps.
__device__ __forceinline__ double limiter_field_rev(double m0, double m1, double m2, double nl, double nr, double eps,
                                                    double lnu, double& lm0, double& lm1, double& lm2, double& lnl,
                                                    double& lnr) {
  const double dl = m1 - m0, dr = m2 - m1;
  const double pl = fma(2.0, dl, -nl), pr = fma(2.0, dr, -nr);
  const double pc2 = dl + dr;
  const double al = dl - nl, ar = dr - nr, ac = dr - dl;
  const double b1 = fma((13.0 / 3.0) * al, al, pl * pl);
  const double b2 = fma((13.0 / 3.0) * ar, ar, pr * pr);
  const double b3 = fma((13.0 / 12.0) * ac, ac, (0.25 * pc2) * pc2);
  const double t1 = b1 + eps, t2 = b2 + eps, t3 = b3 + eps;
  const double s1 = t1 * t1, s2 = t2 * t2, s3 = t3 * t3;
  const double n1 = s2 * s3, n2 = s1 * s3, n3 = s1 * s2;
  const double den = fma(2.0, n3, n1 + n2);
  const double num = fma(n1, pl, fma(n2, pr, n3 * pc2));
  const double r = fast_rcp(den);
  const double lnum = r * lnu;
  const double lden = -num * r * r * lnu;
  const double ln1 = fma(pl, lnum, lden), ln2 = fma(pr, lnum, lden), ln3 = fma(pc2, lnum, 2.0 * lden);
  double lpl = n1 * lnum, lpr = n2 * lnum, lpc2 = n3 * lnum;
  const double ls1 = fma(s3, ln2, s2 * ln3), ls2 = fma(s3, ln1, s1 * ln3), ls3 = fma(s2, ln1, s1 * ln2);
  const double lb1 = 2.0 * t1 * ls1, lb2 = 2.0 * t2 * ls2, lb3 = 2.0 * t3 * ls3;
  const double leps = lb1 + lb2 + lb3;
  const double lal = 2.0 * (13.0 / 3.0) * al * lb1;
  lpl += 2.0 * pl * lb1;
  const double lar = 2.0 * (13.0 / 3.0) * ar * lb2;
  lpr += 2.0 * pr * lb2;
  const double lac = 2.0 * (13.0 / 12.0) * ac * lb3;
  lpc2 += 0.5 * pc2 * lb3;
  double ldr = lac + lar + lpc2 + 2.0 * lpr;
  double ldl = -lac + lal + lpc2 + 2.0 * lpl;
  lnr += -lar - lpr;
  lnl += -lal - lpl;
  lm2 += ldr;
  lm1 += -ldr + ldl;
  lm0 += -ldl;
  return leps;
}

// Reverse of node_record<DIR> (pointwise fluxes, chain-rule derivative fluxes, split). lrec: adjoint of
// the 18 record entries; adds to ln (12 node entries) and returns the adjoint of alpha.
template <int DIR>
__device__ __forceinline__ double node_record_rev(const Node12& n, double g, double alpha, const double lrec[NREC],
                                                  double ln[12]) {
  const double eta = n.v[0], m = n.v[1], w = n.v[2], b = n.v[9];
  const double h = eta - b;
  const double rh = fast_rcp(h);
  const double u = m * rh, v = w * rh;
  const double gh = g * h, ge = g * eta;
  const double cpres = fma(0.5, eta, -b);
  const double uv = u * v;
  const int qs = DIR == 0 ? 3 : 6, qm = DIR == 0 ? 6 : 3;
  const int bs = DIR == 0 ? 10 : 11, bm = DIR == 0 ? 11 : 10;
  const double Hs = n.v[qs], Ms = n.v[qs + 1], Ws = n.v[qs + 2], Bs = n.v[bs];
  const double Hm = n.v[qm], Mm = n.v[qm + 1], Wm = n.v[qm + 2], Bm = n.v[bm];
  const double U[3] = {eta, m, w}, D[3] = {Hs, Ms, Ws};
  double lF[3], lGs[3], lGm[3];
  double lalpha = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double lp = lrec[R_FP + c], lm = lrec[R_FM + c];
    const double lgp = lrec[R_GP + c], lgm = lrec[R_GM + c];
    lF[c] = lp + lm;
    lGs[c] = lgp + lgm;
    lGm[c] = lrec[R_MIX + c];
    lalpha = fma(U[c], lp - lm, fma(D[c], lgp - lgm, lalpha));
    ln[c] += alpha * (lp - lm);       // U
    ln[qs + c] += alpha * (lgp - lgm);  // D
  }
  double leta = 0.0, lm_ = lrec[R_M], lw = lrec[R_W], lh = lrec[R_H], lb = 0.0;
  double lu = 0.0, lv = 0.0, luv = 0.0, lgh = 0.0, lge = 0.0, lpres = 0.0;
  double lHs = 0.0, lMs = 0.0, lWs = 0.0, lBs = 0.0, lHm = 0.0, lMm = 0.0, lWm = 0.0, lBm = 0.0;
  if (DIR == 0) {
    const double uu = u * u, a1 = gh - uu, a2 = uu - ge, u2 = u + u;
    // F = (m, m u + pres, m v)
    lm_ += lF[0] + u * lF[1] + v * lF[2];
    lu += m * lF[1];
    lpres += lF[1];
    lv += m * lF[2];
    // Gs = (Ms, u2 Ms + a1 Hs + a2 Bs, uv (Bs - Hs) + v Ms + u Ws); Gm likewise
    double lu2 = Ms * lGs[1] + Mm * lGm[1];
    double la1 = Hs * lGs[1] + Hm * lGm[1];
    double la2 = Bs * lGs[1] + Bm * lGm[1];
    lMs += lGs[0] + u2 * lGs[1] + v * lGs[2];
    lHs += a1 * lGs[1] - uv * lGs[2];
    lBs += a2 * lGs[1] + uv * lGs[2];
    lWs += u * lGs[2];
    lMm += lGm[0] + u2 * lGm[1] + v * lGm[2];
    lHm += a1 * lGm[1] - uv * lGm[2];
    lBm += a2 * lGm[1] + uv * lGm[2];
    lWm += u * lGm[2];
    luv += (Bs - Hs) * lGs[2] + (Bm - Hm) * lGm[2];
    lv += Ms * lGs[2] + Mm * lGm[2];
    lu += Ws * lGs[2] + Wm * lGm[2];
    lu += 2.0 * lu2;
    lgh += la1;
    double luu = la2 - la1;
    lge -= la2;
    lu += 2.0 * u * luu;
  } else {
    const double vv = v * v, a1 = gh - vv, a2 = vv - ge, v2 = v + v;
    // F = (w, m v, w v + pres)
    lw += lF[0] + v * lF[2];
    lm_ += v * lF[1];
    lv += m * lF[1] + w * lF[2];
    lpres += lF[2];
    // Gs = (Ws, uv (Bs - Hs) + v Ms + u Ws, v2 Ws + a1 Hs + a2 Bs); Gm likewise
    double lv2 = Ws * lGs[2] + Wm * lGm[2];
    double la1 = Hs * lGs[2] + Hm * lGm[2];
    double la2 = Bs * lGs[2] + Bm * lGm[2];
    lWs += lGs[0] + v2 * lGs[2] + u * lGs[1];
    lHs += a1 * lGs[2] - uv * lGs[1];
    lBs += a2 * lGs[2] + uv * lGs[1];
    lMs += v * lGs[1];
    lWm += lGm[0] + v2 * lGm[2] + u * lGm[1];
    lHm += a1 * lGm[2] - uv * lGm[1];
    lBm += a2 * lGm[2] + uv * lGm[1];
    lMm += v * lGm[1];
    luv += (Bs - Hs) * lGs[1] + (Bm - Hm) * lGm[1];
    lv += Ms * lGs[1] + Mm * lGm[1];
    lu += Ws * lGs[1] + Wm * lGm[1];
    lv += 2.0 * lv2;
    lgh += la1;
    double lvv = la2 - la1;
    lge -= la2;
    lv += 2.0 * v * lvv;
  }
  lu += v * luv;
  lv += u * luv;
  // pres = ge (eta/2 - b)
  lge += cpres * lpres;
  leta += 0.5 * ge * lpres;
  lb -= ge * lpres;
  leta += g * lge;
  lh += g * lgh;
  // u = m rh, v = w rh, rh = 1/h
  lm_ += rh * lu;
  lw += rh * lv;
  const double lrh = m * lu + w * lv;
  lh -= rh * rh * lrh;
  leta += lh;
  lb -= lh;
  ln[0] += leta;
  ln[1] += lm_;
  ln[2] += lw;
  ln[qs] += lHs; ln[qs + 1] += lMs; ln[qs + 2] += lWs; ln[bs] += lBs;
  ln[qm] += lHm; ln[qm + 1] += lMm; ln[qm + 2] += lWm; ln[bm] += lBm;
  ln[9] += lb;
  return lalpha;
}

// Record adjoints of the four nodes of an interface, kept in shared memory: entry (s, f) of thread t at
// p[(s * NREC + f) * stride] (stride = threads of the block, t already added to p).
struct SlabAcc {
  double* p;
  int stride;
  __device__ __forceinline__ double& operator()(int s, int f) const { return p[(s * NREC + f) * stride]; }
};

// Reverse of interface_values<DIR, false, true>. lout: adjoint of the 12 outputs. Writes the adjoints of
// the four nodes' records to lr(s, f) (every entry exactly once) and adds those of the source
// candidates to lqb[6]; the interface values do not depend on alpha directly. The forward weighted
// values enter only through the outputs' first components A and Bsum (read back from the forward
// sweep), so the reverse recomputes each side's projections and weights just once, inside the
// reverse of each reconstruction, with one side's data live at a time.
template <int DIR, class Acc>
__device__ __forceinline__ void interface_values_rev(const double* r0, int sstep, int stride, const double qb[6],
                                                     double A, double Bsum, double g, double eps_w,
                                                     const double lout[12], const Acc& lr, double lqb[6]) {
  // node s = 0..3 of the stencil: field f at r0[s * sstep + f * stride]
#define RV(r, f) (r)[(f) * stride]
  const double* r1 = r0 + sstep;
  const double* r2 = r0 + 2 * sstep;
  // ---- forward: interface state and eigenvectors ----
  const double hs = RV(r1, R_H) + RV(r2, R_H);
  const double rhs = fast_rcp(hs);
  const double smM = RV(r1, R_M) + RV(r2, R_M), smW = RV(r1, R_W) + RV(r2, R_W);
  const double ub = smM * rhs, vb = smW * rhs;
  const double gh = (0.5 * g) * hs;
  const double rs = fast_rsqrt(gh);
  const double cb = gh * rs, ic2 = 0.5 * rs;
  const double un = DIR == 0 ? ub : vb, ut = DIR == 0 ? vb : ub;
  const double upc = un + cb, umc = un - cb;
  const int cn = DIR == 0 ? 1 : 2, ct = DIR == 0 ? 2 : 1;
  const double eps13 = (8.0 * g * eps_w) * hs, eps2 = 4.0 * eps_w;
  // characteristic projections of one side's three nodes (rows of the left eigenvectors; side 1
  // reads the nodes mirrored and its derivative records negated)
  auto project = [&](int side, double f[3][3], double p[3][3]) {
    const int fo = side == 0 ? R_FP : R_FM, go = side == 0 ? R_GP : R_GM;
    const double sg = side == 0 ? 1.0 : -1.0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const double* r = r0 + (side == 0 ? t : 3 - t) * sstep;
      const double F0 = RV(r, fo), Fn = RV(r, fo + cn), Ft = RV(r, fo + ct);
      const double G0 = sg * RV(r, go), Gn = sg * RV(r, go + cn), Gt = sg * RV(r, go + ct);
      f[0][t] = fma(upc, F0, -Fn);
      f[1][t] = fma(-ut, F0, Ft);
      f[2][t] = fma(-umc, F0, Fn);
      p[0][t] = fma(upc, G0, -Gn);
      p[1][t] = fma(-ut, G0, Gt);
      p[2][t] = fma(-umc, G0, Gn);
    }
  };
  // A = (G_1 + G_3) ic2 and Bsum = (GB_1 + GB_3) ic2 are the first components of the forward outputs
  // 2 Fhat and 2 bhat, passed in; 1 / ic2 = 2 c.
  // ---- reverse ----
  // back-projection
  double lun = 0.0, lut = 0.0, lic2 = 0.0;
  const double lA = lout[0] + un * lout[cn] + ut * lout[ct];
  lun += A * lout[cn];
  lut += A * lout[ct];
  double lG[3];
  lG[0] = -0.5 * lout[cn] + ic2 * lA;
  lG[2] = 0.5 * lout[cn] + ic2 * lA;
  lG[1] = lout[ct];
  lic2 += 2.0 * cb * A * lA;
  const double lBs = lout[3] + un * lout[3 + cn] + ut * lout[3 + ct];
  lun += Bsum * lout[3 + cn];
  lut += Bsum * lout[3 + ct];
  const double lGB1 = -0.5 * lout[3 + cn] + ic2 * lBs;
  const double lGB3 = 0.5 * lout[3 + cn] + ic2 * lBs;
  lic2 += 2.0 * cb * Bsum * lBs;
  // per side and field: weighted values and the source with the same weights (projections recomputed)
  double lupc = 0.0, lumc = 0.0, leps13 = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int fo = side == 0 ? R_FP : R_FM, go = side == 0 ? R_GP : R_GM;
    const double sg = side == 0 ? 1.0 : -1.0;
    double f[3][3], p[3][3];
    project(side, f, p);
    double lf[3][3] = {}, lp[3][3] = {};
    // source: GB1 -= weighted(W0), GB3 += weighted(W2)
    leps13 += hweno_side_rev<true>(f[0], p[0], eps13, lG[0], qb + 3 * side, -lGB1, lqb + 3 * side, lf[0], lp[0]);
    (void)hweno_side_rev<false>(f[1], p[1], eps2, lG[1], nullptr, 0.0, nullptr, lf[1], lp[1]);
    leps13 += hweno_side_rev<true>(f[2], p[2], eps13, lG[2], qb + 3 * side, lGB3, lqb + 3 * side, lf[2], lp[2]);
    // projections f = (upc F0 - Fn, -ut F0 + Ft, -umc F0 + Fn), p likewise with sg G
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int sl = side == 0 ? t : 3 - t;
      const double* r = r0 + sl * sstep;
      const double F0 = RV(r, fo), G0 = sg * RV(r, go);
      lupc += F0 * lf[0][t] + G0 * lp[0][t];
      lut -= F0 * lf[1][t] + G0 * lp[1][t];
      lumc -= F0 * lf[2][t] + G0 * lp[2][t];
      // plus the derivative flux, linear in the records: 24 dx Ghat = 3 F+_{i-1} - 24 F+_i + 21 F+_{i+1}
      // + G+_{i-1} - 2 G+_i - 5 G+_{i+1} from the left, mirrored from the right (per component)
      const double kf = side == 0 ? (sl == 0 ? 3.0 : sl == 1 ? -24.0 : 21.0) : (sl == 3 ? -3.0 : sl == 2 ? 24.0 : -21.0);
      const double kg = side == 0 ? (sl == 0 ? 1.0 : sl == 1 ? -2.0 : -5.0) : (sl == 3 ? 1.0 : sl == 2 ? -2.0 : -5.0);
      lr(sl, fo) = fma(kf, lout[6], upc * lf[0][t] - ut * lf[1][t] - umc * lf[2][t]);
      lr(sl, fo + cn) = fma(kf, lout[6 + cn], -lf[0][t] + lf[2][t]);
      lr(sl, fo + ct) = fma(kf, lout[6 + ct], lf[1][t]);
      lr(sl, go) = fma(kg, lout[6], sg * (upc * lp[0][t] - ut * lp[1][t] - umc * lp[2][t]));
      lr(sl, go + cn) = fma(kg, lout[6 + cn], sg * (-lp[0][t] + lp[2][t]));
      lr(sl, go + ct) = fma(kg, lout[6 + ct], sg * lp[1][t]);
    }
    asm volatile("" ::: "memory");  // keep the two sides apart in the schedule (register pressure)
  }
  // eigen quantities
  lun += lupc + lumc;
  const double lcb = lupc - lumc;
  const double lub = DIR == 0 ? lun : lut, lvb = DIR == 0 ? lut : lun;
  double lrs = 0.5 * lic2 + gh * lcb;
  double lgh = rs * lcb;
  lgh += -0.5 * rs * rs * rs * lrs;
  double lhs = (8.0 * g * eps_w) * leps13 + (0.5 * g) * lgh;
  const double lrhs = smM * lub + smW * lvb;
  lhs -= rhs * rhs * lrhs;
  lr(1, R_H) = lhs;
  lr(2, R_H) = lhs;
  lr(1, R_M) = rhs * lub;
  lr(2, R_M) = rhs * lub;
  lr(1, R_W) = rhs * lvb;
  lr(2, R_W) = rhs * lvb;
  // the remaining entries: mixed term 24 (Phi hat) = -M_{i-1} + 7 M_i + 7 M_{i+1} - M_{i+2}, and
  // records that reach this interface through neither side
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double l9 = lout[9 + c];
    lr(0, R_MIX + c) = -l9;
    lr(1, R_MIX + c) = 7.0 * l9;
    lr(2, R_MIX + c) = 7.0 * l9;
    lr(3, R_MIX + c) = -l9;
    lr(3, R_FP + c) = 0.0;
    lr(3, R_GP + c) = 0.0;
    lr(0, R_FM + c) = 0.0;
    lr(0, R_GM + c) = 0.0;
  }
#pragma unroll
  for (int f = R_H; f <= R_W; ++f) {
    lr(0, f) = 0.0;
    lr(3, f) = 0.0;
  }
#undef RV
}

// Reverse of limit_dir<DIR, false, true>: lout (3) -> adjoints of Um, U0, Up, Dm, Dp and of the node's
// u, v, c (through ic2 and the projection rows) and of gh (through epsilon). Adds into the arrays.
template <int DIR>
__device__ __forceinline__ void limit_dir_rev(const double Um[3], const double U0[3], const double Up[3],
                                              const double Dm[3], const double Dp[3], double u, double v, double c,
                                              double ic2, double gh, double eps, const double lout[3], double lUm[3],
                                              double lU0[3], double lUp[3], double lDm[3], double lDp[3], double& lu,
                                              double& lv, double& lc, double& lic2, double& lgh) {
  const int cn = DIR == 0 ? 1 : 2, ct = DIR == 0 ? 2 : 1;
  const double un = DIR == 0 ? u : v, ut = DIR == 0 ? v : u;
  const double upc = un + c, umc = un - c;
  const double* src[5] = {Um, U0, Up, Dm, Dp};
  double* lsrc[5] = {lUm, lU0, lUp, lDm, lDp};
  double pr[5][3];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const double* a = src[s];
    pr[s][0] = fma(upc, a[0], -a[cn]);
    pr[s][1] = fma(-ut, a[0], a[ct]);
    pr[s][2] = fma(-umc, a[0], a[cn]);
  }
  const double e13 = (4.0 * eps) * gh;
  double nu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    nu[k] = limiter_field<false>(pr[0][k], pr[1][k], pr[2][k], pr[3][k], pr[4][k], k == 1 ? eps : e13);
  const double A = (nu[0] + nu[2]) * ic2;
  // reverse of the back-projection (A, un A + (nu2 - nu0)/2, ut A + nu1)
  const double lA = lout[0] + un * lout[cn] + ut * lout[ct];
  double lun = A * lout[cn], lut = A * lout[ct];
  double lnu[3];
  lnu[0] = -0.5 * lout[cn] + ic2 * lA;
  lnu[2] = 0.5 * lout[cn] + ic2 * lA;
  lnu[1] = lout[ct];
  lic2 += (nu[0] + nu[2]) * lA;
  double lpr[5][3] = {};
  double le13 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double le = limiter_field_rev(pr[0][k], pr[1][k], pr[2][k], pr[3][k], pr[4][k], k == 1 ? eps : e13, lnu[k],
                                        lpr[0][k], lpr[1][k], lpr[2][k], lpr[3][k], lpr[4][k]);
    if (k != 1) le13 += le;
  }
  lgh += (4.0 * eps) * le13;
  double lupc = 0.0, lumc = 0.0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const double* a = src[s];
    double* l = lsrc[s];
    lupc += a[0] * lpr[s][0];
    lut -= a[0] * lpr[s][1];
    lumc -= a[0] * lpr[s][2];
    l[0] += upc * lpr[s][0] - ut * lpr[s][1] - umc * lpr[s][2];
    l[cn] += -lpr[s][0] + lpr[s][2];
    l[ct] += lpr[s][1];
  }
  lun += lupc + lumc;
  lc += lupc - lumc;
  if (DIR == 0) { lu += lun; lv += lut; }
  else { lv += lun; lu += lut; }
}

}  // namespace hw
