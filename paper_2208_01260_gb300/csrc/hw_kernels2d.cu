// 2D kernels of the well-balanced fifth-order FD HWENO scheme (Zhao & Zhang, arXiv:2208.01260,
// Sec. 3) for sm_103a. One RK stage is four launches on the solver's stream:
//   k_alpha2d_* global Lax-Friedrichs constants alpha_x = max(|u|+c), alpha_y = max(|v|+c)
//   k_sweep_x   x-interfaces: Sec. 2.1 Steps 1-2 along x for (F1, Phi1, tilde-b, tilde-B1) and the
//               mixed term Psi1 of eq. (mixed)
//   k_sweep_y   y-interfaces: Steps 1-2 along y for (F2, Psi2, bar-b, bar-B2) and the mixed Phi2
//   k_node2d    eq. (swe-form-2d-dis) (source signs read as '-'), the HWENO limiter of Sec. 2.2
//               applied dimension by dimension, and the SSP-RK3 combination of eq. (RK)
// Interface values go through global memory: the FP64 pipe, not memory, bounds this scheme on
// GB300, so each interface is computed exactly once. Every kernel is instantiated for double and for
// the single-precision variant (float planes and constants).
#include "hw_stencil2d.cuh"

namespace hw {

// ---------------------------------------------------------------------------------------------
// Sweeps: one tile of TILE_T threads per block over the flattened extended lines (hw_stencil2d.cuh),
// TILE_T - 3 x-interfaces, or YS_C (TILE_T / YS_C - 3) y-interfaces, per block.
// ---------------------------------------------------------------------------------------------
constexpr int YS_C = 2;  // columns per y-tile group of the double y-sweep (measured: 2 beats 1 and 4)

// The double kernels form their products (and the node kernel also its reciprocals) on the integer
// pipes (hw_fp64_int.h: each product bit-identical to DMUL): the FP64 pipe is their bound, the integer
// pipes idle. The node records stay on the FP64 pipe (moving them measured slower).
template <class R>
constexpr bool kIntMul = std::is_same<R, double>::value;
// Blocks per SM the sweeps and the node kernel are compiled for: the double kernels carry the
// integer-pipe products in registers (168 per thread in the sweeps); the float kernels are bound by
// memory and issue and want occupancy.
template <class R>
constexpr int kXsBlocks = std::is_same<R, double>::value ? 2 : 5;
template <class R>
constexpr int kNodeBlocks = std::is_same<R, double>::value ? 3 : 5;

template <bool LINEAR, bool CHAR, class R>
__global__ void __launch_bounds__(TILE_T, kXsBlocks<R>) k_sweep_x(Dev2DT<R> d, const R* __restrict__ alpha) {
  __shared__ R sm[NREC * TILE_T];
  sweep_x_tile<LINEAR, CHAR, kIntMul<R>>(d, alpha[0], blockIdx.x * (TILE_T - 3), sm);
}

template <bool LINEAR, bool CHAR, class R>
__global__ void __launch_bounds__(TILE_T, kXsBlocks<R>) k_sweep_y(Dev2DT<R> d, const R* __restrict__ alpha) {
  __shared__ R sm[NREC * TILE_T];
  sweep_y_tile<LINEAR, CHAR, kIntMul<R>>(d, alpha[1], blockIdx.x * (TILE_T / YS_C - 3), YS_C, sm);
}

// Single-precision y-sweep: bound by memory rather than arithmetic, it keeps the column march, whose
// loads are 32 consecutive nodes of a row: each thread owns one column and marches down `seg`
// interfaces with the last four node records in a private shared-memory ring (no block barrier and
// only 3 extra records per segment). Measured at 2048^2: 0.139 ms against 0.164 ms for the best tile.
constexpr int YS_W = 32;

template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(YS_W, 32) k_sweep_y_col(Dev2DT<float> d, const float* __restrict__ alpha, int seg) {
  __shared__ float ring[4 * NREC * YS_W];
  const int i = blockIdx.x * YS_W + threadIdx.x;
  if (i >= d.nx) return;
  const int k0 = blockIdx.y * seg;
  const float ay = alpha[1];
  const int rend = min(k0 + seg, d.ny + 1);
  for (int r = k0 - 2; r <= rend; ++r) {
    Node12T<float> n;
    load_node(d, i, r, n);
    float rec[NREC];
    node_record<1>(n, d.g, ay, rec);
    float* slot = ring + (size_t)(r & 3) * NREC * YS_W + threadIdx.x;
#pragma unroll
    for (int f = 0; f < NREC; ++f) slot[f * YS_W] = rec[f];
    const int k = r - 1;
    if (k >= k0 && k < k0 + seg && k <= d.ny) {
      const float* s0 = ring + (size_t)((k - 2) & 3) * NREC * YS_W + threadIdx.x;
      const float* s1 = ring + (size_t)((k - 1) & 3) * NREC * YS_W + threadIdx.x;
      const float* s2 = ring + (size_t)((k) & 3) * NREC * YS_W + threadIdx.x;
      const float* s3 = ring + (size_t)((k + 1) & 3) * NREC * YS_W + threadIdx.x;
      const size_t o = (size_t)k * d.nx + i;
      float qb[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) qb[q] = __ldg(d.qby[q] + o);
      float out[12];
      interface_values<1, LINEAR, CHAR, false>(s0, s1, s2, s3, YS_W, qb, d.g, d.eps_w, out);
#pragma unroll
      for (int q = 0; q < 12; ++q) d.Y[q][o] = out[q];
    }
  }
}

template <int MODE, bool LINEAR, bool CHAR, class R>
__global__ void __launch_bounds__(256, kNodeBlocks<R>) k_node2d(Dev2DT<R> d, StageArgsT<R> sa) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  if (i >= d.nx || j >= d.ny) return;
  node_update<MODE, LINEAR, CHAR, kIntMul<R>>(d, sa, i, j);
}

// ---------------------------------------------------------------------------------------------
// alpha_x, alpha_y = max over nodes of |u| + c, |v| + c, plus a status flag for non-finite or
// non-positive depth: in double the two passes of hw_stencil2d.cuh (coarse float maxima, then the exact
// double maximum near them), in single precision one pass.
// ---------------------------------------------------------------------------------------------
// Each block reduces one contiguous tile of nodes; each thread keeps kAlphaU nodes' loads in flight. The
// coarse pass records every tile's float maxima (bit 31 set when a node of the tile needs the exact
// evaluation regardless), so the exact pass skips the tiles that cannot hold a maximum: it evaluates the
// same nodes, by the same rule, as a pass over all nodes would.
constexpr int kAlphaU = 4;
constexpr unsigned kTileExact = 0x80000000u;

__device__ __forceinline__ void alpha_tile(size_t n, size_t& begin, size_t& end) {
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  begin = min(n, (size_t)blockIdx.x * per);
  end = min(n, begin + per);
}

__global__ void __launch_bounds__(256) k_alpha2d_coarse(Dev2D d, unsigned long long* amax, int* status) {
  __shared__ float s_m[2][8];
  __shared__ int s_ex[8];
  size_t begin, end;
  alpha_tile((size_t)d.nx * d.ny, begin, end);
  float mx = 0.0f, my = 0.0f;
  int bad = 0, ex = 0;
  for (size_t o0 = begin + threadIdx.x; o0 < end; o0 += kAlphaU * blockDim.x) {
    float ax[kAlphaU], ay[kAlphaU];
    bool exact[kAlphaU], neg[kAlphaU];
#pragma unroll
    for (int u = 0; u < kAlphaU; ++u) {
      exact[u] = false;
      neg[u] = true;  // past the end: skipped
      if (o0 + u * blockDim.x < end) alpha_coarse(d, o0 + u * blockDim.x, ax[u], ay[u], exact[u], neg[u]);
    }
#pragma unroll
    for (int u = 0; u < kAlphaU; ++u) {
      if (o0 + u * blockDim.x >= end) continue;
      if (exact[u]) { ex = 1; continue; }  // the exact pass evaluates (and, if need be, flags) this node
      if (neg[u]) { bad |= HW_STATUS_DEPTH; continue; }
      mx = fmaxf(mx, ax[u]);
      my = fmaxf(my, ay[u]);
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, s));
  }
  ex = __any_sync(0xffffffffu, ex);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_m[0][w] = mx; s_m[1][w] = my; s_ex[w] = ex; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      mx = fmaxf(mx, s_m[0][k]);
      my = fmaxf(my, s_m[1][k]);
      ex |= s_ex[k];
    }
    // non-negative floats order as their bit patterns; both maxima share the third 64-bit slot
    unsigned int* m32 = reinterpret_cast<unsigned int*>(amax + 2);
    atomicMax(m32, __float_as_uint(mx));
    atomicMax(m32 + 1, __float_as_uint(my));
    const unsigned f = ex ? kTileExact : 0u;
    reinterpret_cast<uint2*>(amax + 3)[blockIdx.x] = make_uint2(__float_as_uint(mx) | f, __float_as_uint(my) | f);
  }
  if (bad) atomicOr(status, bad);
}

// The nodes alpha_exact_range would evaluate, in the tiles whose coarse maxima reach the thresholds.
__global__ void __launch_bounds__(256) k_alpha2d_exact(Dev2D d, unsigned long long* amax, int* status) {
  const unsigned int* m32 = reinterpret_cast<const unsigned int*>(amax + 2);
  const float tx = __uint_as_float(m32[0]) * (1.0f - 1e-5f), ty = __uint_as_float(m32[1]) * (1.0f - 1e-5f);
  const uint2 tile = reinterpret_cast<const uint2*>(amax + 3)[blockIdx.x];
  if (!((tile.x | tile.y) & kTileExact) && __uint_as_float(tile.x) < tx && __uint_as_float(tile.y) < ty) return;
  size_t begin, end;
  alpha_tile((size_t)d.nx * d.ny, begin, end);
  unsigned long long kx = 0, ky = 0;
  int bad = 0;
  for (size_t o0 = begin + threadIdx.x; o0 < end; o0 += kAlphaU * blockDim.x) {
    float fx[kAlphaU], fy[kAlphaU];
    bool exact[kAlphaU], neg[kAlphaU], in[kAlphaU];
#pragma unroll
    for (int u = 0; u < kAlphaU; ++u) {
      in[u] = o0 + u * blockDim.x < end;
      if (in[u]) alpha_coarse(d, o0 + u * blockDim.x, fx[u], fy[u], exact[u], neg[u]);
    }
#pragma unroll
    for (int u = 0; u < kAlphaU; ++u)
      if (in[u] && alpha_needs_exact(fx[u], fy[u], exact[u], neg[u], tx, ty))
        alpha_exact_node(d, o0 + u * blockDim.x, kx, ky, bad);
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    kx = max(kx, __shfl_xor_sync(0xffffffffu, kx, s));
    ky = max(ky, __shfl_xor_sync(0xffffffffu, ky, s));
  }
  if ((threadIdx.x & 31) == 0) {
    if (kx) atomicMax(amax, kx);
    if (ky) atomicMax(amax + 1, ky);
  }
  if (bad) atomicOr(status, bad);
}

// Single precision: the maximum in float, widened to a double key once per warp. Each thread keeps the
// loads of kAlphaU nodes in flight (the pass is bound by memory latency otherwise).
__global__ void __launch_bounds__(256) k_alpha2d_f32(Dev2DT<float> d, unsigned long long* amax, int* status) {
  int bad = 0;
  const size_t n = (size_t)d.nx * d.ny, step = (size_t)gridDim.x * blockDim.x;
  float mx = 0.0f, my = 0.0f;
  for (size_t o0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o0 < n; o0 += kAlphaU * step) {
    float hn[kAlphaU], mn[kAlphaU], wn[kAlphaU];
#pragma unroll
    for (int q = 0; q < kAlphaU; ++q) {
      const size_t o = o0 + q * step;
      hn[q] = 1.0f;
      mn[q] = wn[q] = 0.0f;
      if (o < n) {
        hn[q] = __ldg(d.S[0] + o) - __ldg(d.stat[0] + o);
        mn[q] = __ldg(d.S[1] + o);
        wn[q] = __ldg(d.S[2] + o);
      }
    }
#pragma unroll
    for (int q = 0; q < kAlphaU; ++q) {
      if (o0 + q * step >= n) continue;
      const float h = hn[q];
      if (!(h > 0.0f) || !(h < 3e38f)) { bad |= h == h ? HW_STATUS_DEPTH : HW_STATUS_NONFINITE; continue; }
      const float rh = fast_rcp(h);
      const float gh = d.g * h;
      const float c = gh * fast_rsqrt(gh);
      const float u = mn[q] * rh, v = wn[q] * rh;
      const float ax = fabsf(u) + c, ay = fabsf(v) + c;
      if (!(ax < 3e38f) || !(ay < 3e38f)) { bad |= HW_STATUS_NONFINITE; continue; }
      mx = fmaxf(mx, ax);
      my = fmaxf(my, ay);
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, s));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(amax, dkey((double)mx));
    atomicMax(amax + 1, dkey((double)my));
  }
  if (bad) atomicOr(status, bad);
}

// alpha keys -> doubles; dt = cfl / (alpha_x/dx + alpha_y/dy), optionally clipped to t_end - t.
__global__ void k_finish_alpha2d(const unsigned long long* amax, double* alpha, double* dt_out, double cfl,
                                 double inv_dx, double inv_dy, const double* t_now, double t_end) {
  const double ax = __longlong_as_double((long long)amax[0]);
  const double ay = __longlong_as_double((long long)amax[1]);
  alpha[0] = ax;
  alpha[1] = ay;
  if (dt_out) {
    double dt = cfl / fma(ax, inv_dx, ay * inv_dy);
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

// ---------------------------------------------------------------------------------------------
// Initialisation and conversion kernels
// ---------------------------------------------------------------------------------------------
// physical (h, hu, hv, b, h_x, hu_x, hv_x, h_y, hu_y, hv_y, b_x, b_y) -> equilibrium state with
// scaled derivatives (eta = h + b, H = h_x + b_x; Sec. 3) and static (b, dx b_x, dy b_y).
__global__ void k_init2d(Dev2D d, PhysIn in, int* status) {
  const size_t n = (size_t)d.nx * d.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double h = in.p[0][o], b = in.p[3][o], bx = in.p[10][o], by = in.p[11][o];
    if (!(h > 0.0) || !(h < 1e300)) atomicOr(status, h == h ? HW_STATUS_DEPTH : HW_STATUS_NONFINITE);
    d.S[0][o] = h + b;
    d.S[1][o] = in.p[1][o];
    d.S[2][o] = in.p[2][o];
    d.S[3][o] = d.dx * (in.p[4][o] + bx);
    d.S[4][o] = d.dx * in.p[5][o];
    d.S[5][o] = d.dx * in.p[6][o];
    d.S[6][o] = d.dy * (in.p[7][o] + by);
    d.S[7][o] = d.dy * in.p[8][o];
    d.S[8][o] = d.dy * in.p[9][o];
    d.stat[0][o] = b;
    d.stat[1][o] = d.dx * bx;
    d.stat[2][o] = d.dy * by;
    d.bxy[0][o] = bx;
    d.bxy[1][o] = by;
  }
}

// state <-> user planes. layout 0: physical (h, hu, hv, h_x, hu_x, hv_x, h_y, hu_y, hv_y);
// layout 1: equilibrium (eta, m, w, eta_x, m_x, w_x, eta_y, m_y, w_y). dir 0: export, 1: import.
__global__ void k_convert2d(Dev2D d, Ptr9 src9, Ptr9 dst9, int layout, int dir) {
  double* const* S = d.S;
  const size_t n = (size_t)d.nx * d.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double b = d.stat[0][o], bx = d.bxy[0][o], by = d.bxy[1][o];
    if (dir == 0) {
      double x[9];
      for (int q = 0; q < 9; ++q) x[q] = S[q][o];
      dst9.p[0][o] = layout == 0 ? x[0] - b : x[0];
      dst9.p[1][o] = x[1];
      dst9.p[2][o] = x[2];
      dst9.p[3][o] = layout == 0 ? x[3] * d.inv_dx - bx : x[3] * d.inv_dx;
      dst9.p[4][o] = x[4] * d.inv_dx;
      dst9.p[5][o] = x[5] * d.inv_dx;
      dst9.p[6][o] = layout == 0 ? x[6] * d.inv_dy - by : x[6] * d.inv_dy;
      dst9.p[7][o] = x[7] * d.inv_dy;
      dst9.p[8][o] = x[8] * d.inv_dy;
    } else {
      double x[9];
      for (int q = 0; q < 9; ++q) x[q] = src9.p[q][o];
      S[0][o] = layout == 0 ? x[0] + b : x[0];
      S[1][o] = x[1];
      S[2][o] = x[2];
      S[3][o] = d.dx * (layout == 0 ? x[3] + bx : x[3]);
      S[4][o] = d.dx * x[4];
      S[5][o] = d.dx * x[5];
      S[6][o] = d.dy * (layout == 0 ? x[6] + by : x[6]);
      S[7][o] = d.dy * x[7];
      S[8][o] = d.dy * x[8];
    }
  }
}

// Static parts of the source terms that depend on b only (Sec. 2.1 Step 2 and eq. mixed):
//   qbx/qby: Hermite candidates q_1..q_3 of (b, dS b_s) per interface and side (the nonlinear
//            weights are applied per stage),
//   sv, sq : dx [tilde-B1^]_x/dx + dx [bar-B1^]_y/dy and dy [tilde-B2^]_x/dx + dy [bar-B2^]_y/dy
//            (normal-momentum and tangential-momentum components; the first component is zero).
__device__ __forceinline__ double bval(const Dev2D& d, int q, int i, int j) {
  // q: 0 b, 1 b_x, 2 b_y (physical); parities: b even; b_x odd across x-walls; b_y odd across y-walls
  bool fx, fy;
  const int ii = map_index(i, d.nx, d.bc_x, fx);
  const int jj = map_index(j, d.ny, d.bc_y, fy);
  const size_t o = (size_t)jj * d.nx + ii;
  double x = q == 0 ? d.stat[0][o] : d.bxy[q - 1][o];
  if (fx && q == 1) x = -x;
  if (fy && q == 2) x = -x;
  return x;
}

__device__ __forceinline__ void cands(double f0, double f1, double f2, double p0, double p1, double p2, double q[3]) {
  q[0] = 0.5 * (f0 + f1) + (p0 + 5.0 * p1) / 6.0;
  q[1] = 0.5 * (f1 + f2) + (p1 - p2) / 6.0;
  q[2] = (f0 + 10.0 * f1 + f2) / 12.0 + 0.5 * p1;
}

// Derivative of the quintic at the interface, both sides summed, on (b/2, b_s/2) (eq. Rec-phi).
__device__ __forceinline__ double qprime_sum(double b0, double b1, double b2, double b3, double s0, double s1,
                                             double s2, double s3, double del) {
  const double qp = (b0 - 8.0 * b1 + 7.0 * b2) / (4.0 * del) + (s0 - 2.0 * s1 - 5.0 * s2) / 12.0;
  const double qm = (-7.0 * b1 + 8.0 * b2 - b3) / (4.0 * del) + (-5.0 * s1 - 2.0 * s2 + s3) / 12.0;
  return 0.5 * (qp + qm);
}

__device__ __forceinline__ double mixed4(double a, double b, double c, double e) {
  return (-a + 7.0 * b + 7.0 * c - e) / 12.0;
}

__global__ void k_static2d(Dev2D d) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  // x-interfaces k = i (0..nx) of row j; y-interfaces k = j (0..ny) of column i
  if (j < d.ny && i <= d.nx) {
    double b[4], s[4];
    for (int t = 0; t < 4; ++t) {
      b[t] = bval(d, 0, i - 2 + t, j);
      s[t] = d.dx * bval(d, 1, i - 2 + t, j);
    }
    double qp[3], qm[3];
    cands(b[0], b[1], b[2], s[0], s[1], s[2], qp);
    cands(b[3], b[2], b[1], -s[3], -s[2], -s[1], qm);
    const size_t o = (size_t)j * (d.nx + 1) + i;
    for (int q = 0; q < 3; ++q) { d.qbx[q][o] = qp[q]; d.qbx[3 + q][o] = qm[q]; }
  }
  if (i < d.nx && j <= d.ny) {
    double b[4], s[4];
    for (int t = 0; t < 4; ++t) {
      b[t] = bval(d, 0, i, j - 2 + t);
      s[t] = d.dy * bval(d, 2, i, j - 2 + t);
    }
    double qp[3], qm[3];
    cands(b[0], b[1], b[2], s[0], s[1], s[2], qp);
    cands(b[3], b[2], b[1], -s[3], -s[2], -s[1], qm);
    const size_t o = (size_t)j * d.nx + i;
    for (int q = 0; q < 3; ++q) { d.qby[q][o] = qp[q]; d.qby[3 + q][o] = qm[q]; }
  }
  if (i < d.nx && j < d.ny) {
    // x-interfaces i-1/2 (left, stencil i-2..i+1) and i+1/2 (right, i-1..i+2)
    auto B1x = [&](int k) {  // tilde-B1 hat (normal-momentum component) at x-interface k-1/2
      return qprime_sum(bval(d, 0, k - 2, j), bval(d, 0, k - 1, j), bval(d, 0, k, j), bval(d, 0, k + 1, j),
                        bval(d, 1, k - 2, j), bval(d, 1, k - 1, j), bval(d, 1, k, j), bval(d, 1, k + 1, j), d.dx);
    };
    auto B2x = [&](int k) {  // tilde-B2 hat = mixed(b_y) at x-interface k-1/2
      return mixed4(bval(d, 2, k - 2, j), bval(d, 2, k - 1, j), bval(d, 2, k, j), bval(d, 2, k + 1, j));
    };
    auto B1y = [&](int k) {  // bar-B1 hat = mixed(b_x) at y-interface k-1/2
      return mixed4(bval(d, 1, i, k - 2), bval(d, 1, i, k - 1), bval(d, 1, i, k), bval(d, 1, i, k + 1));
    };
    auto B2y = [&](int k) {  // bar-B2 hat (tangential = y-momentum component) at y-interface k-1/2
      return qprime_sum(bval(d, 0, i, k - 2), bval(d, 0, i, k - 1), bval(d, 0, i, k), bval(d, 0, i, k + 1),
                        bval(d, 2, i, k - 2), bval(d, 2, i, k - 1), bval(d, 2, i, k), bval(d, 2, i, k + 1), d.dy);
    };
    const size_t o = (size_t)j * d.nx + i;
    // dx * (tilde-B1 hat)_x / dx = difference; dx * (bar-B1 hat)_y / dy
    d.sv[0][o] = B1x(i + 1) - B1x(i);
    d.sv[1][o] = d.dx * (B1y(j + 1) - B1y(j)) * d.inv_dy;
    // dy * (tilde-B2 hat)_x / dx; dy * (bar-B2 hat)_y / dy = difference
    d.sq[0][o] = d.dy * (B2x(i + 1) - B2x(i)) * d.inv_dx;
    d.sq[1][o] = B2y(j + 1) - B2y(j);
  }
}

// ---------------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------------
template <bool L, bool C, class R>
static void launch_sx(const Dev2DT<R>& d, const R* alpha, cudaStream_t st) {
  const unsigned long long total = (unsigned long long)d.ny * (d.nx + 4);
  k_sweep_x<L, C, R><<<(unsigned)((total + TILE_T - 4) / (TILE_T - 3)), TILE_T, 0, st>>>(d, alpha);
}

// Segment length of the float column march: one balanced wave of resident blocks when the grid allows
// it (the blocks of a column segment all do the same work), at least 8 interfaces per segment.
static int sweep_y_segment(int nx, int ny, int blocks_per_sm) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int cols = (nx + YS_W - 1) / YS_W;
  const long resident = (long)sms * std::max(blocks_per_sm, 1);
  long segs = std::max(1L, resident / cols);
  int seg = (int)((ny + 1 + segs - 1) / segs);
  return std::max(seg, std::min(8, ny + 1));
}

template <bool L, bool C, class R>
static void launch_sy(const Dev2DT<R>& d, const R* alpha, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value) {
    static int bps = -1;
    if (bps < 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_sweep_y_col<L, C>, YS_W, 0) != cudaSuccess)
      bps = 1;
    const int seg = sweep_y_segment(d.nx, d.ny, bps);
    dim3 gy((d.nx + YS_W - 1) / YS_W, (d.ny + 1 + seg - 1) / seg);
    k_sweep_y_col<L, C><<<gy, YS_W, 0, st>>>(d, alpha, seg);
  } else {
    constexpr int IFS = TILE_T / YS_C - 3;
    const unsigned long long total = (unsigned long long)((d.nx + YS_C - 1) / YS_C) * (d.ny + 4);
    k_sweep_y<L, C, R><<<(unsigned)((total + IFS - 1) / IFS), TILE_T, 0, st>>>(d, alpha);
  }
}

template <int MODE, bool L, bool C, class R>
static void launch_node(const Dev2DT<R>& d, const StageArgsT<R>& sa, cudaStream_t st) {
  dim3 g((d.nx + 31) / 32, (d.ny + 7) / 8);
  k_node2d<MODE, L, C, R><<<g, dim3(32, 8), 0, st>>>(d, sa);
}

int set_kernel_attributes2d() { return 0; }

void launch_alpha2d(const Dev2D& d, unsigned long long* amax, int* status, cudaStream_t st) {
  cudaMemsetAsync(amax, 0, 3 * sizeof(unsigned long long), st);
  const size_t n = (size_t)d.nx * d.ny;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)kAlpha2dTiles);  // tiles: amax[3 ..]
  k_alpha2d_coarse<<<blocks, 256, 0, st>>>(d, amax, status);
  k_alpha2d_exact<<<blocks, 256, 0, st>>>(d, amax, status);
}
void launch_alpha2d(const Dev2DT<float>& d, unsigned long long* amax, int* status, cudaStream_t st) {
  cudaMemsetAsync(amax, 0, 3 * sizeof(unsigned long long), st);
  const size_t n = (size_t)d.nx * d.ny;
  int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)152 * 8);
  k_alpha2d_f32<<<blocks, 256, 0, st>>>(d, amax, status);
}

void launch_finish_alpha2d(const Dev2D& d, const unsigned long long* amax, double* alpha, double* dt_out,
                           double cfl, const double* t_now, double t_end, cudaStream_t st) {
  k_finish_alpha2d<<<1, 1, 0, st>>>(amax, alpha, dt_out, cfl, d.inv_dx, d.inv_dy, t_now, t_end);
}

template <class R>
static void sweep_x_impl(const Dev2DT<R>& d, const R* alpha, bool linear, bool chr, cudaStream_t st) {
  if (linear) { if (chr) launch_sx<true, true>(d, alpha, st); else launch_sx<true, false>(d, alpha, st); }
  else        { if (chr) launch_sx<false, true>(d, alpha, st); else launch_sx<false, false>(d, alpha, st); }
}
template <class R>
static void sweep_y_impl(const Dev2DT<R>& d, const R* alpha, bool linear, bool chr, cudaStream_t st) {
  if (linear) { if (chr) launch_sy<true, true>(d, alpha, st); else launch_sy<true, false>(d, alpha, st); }
  else        { if (chr) launch_sy<false, true>(d, alpha, st); else launch_sy<false, false>(d, alpha, st); }
}
template <class R>
static void node_impl(const Dev2DT<R>& d, const StageArgsT<R>& sa, int mode, bool linear, bool chr, cudaStream_t st) {
  if (mode == MODE_RHS) {
    if (linear) { if (chr) launch_node<MODE_RHS, true, true>(d, sa, st); else launch_node<MODE_RHS, true, false>(d, sa, st); }
    else        { if (chr) launch_node<MODE_RHS, false, true>(d, sa, st); else launch_node<MODE_RHS, false, false>(d, sa, st); }
  } else {
    if (linear) { if (chr) launch_node<MODE_STAGE, true, true>(d, sa, st); else launch_node<MODE_STAGE, true, false>(d, sa, st); }
    else        { if (chr) launch_node<MODE_STAGE, false, true>(d, sa, st); else launch_node<MODE_STAGE, false, false>(d, sa, st); }
  }
}

void launch_sweep_x2d(const Dev2D& d, const double* alpha, bool linear, bool chr, cudaStream_t st) {
  sweep_x_impl(d, alpha, linear, chr, st);
}
void launch_sweep_y2d(const Dev2D& d, const double* alpha, bool linear, bool chr, cudaStream_t st) {
  sweep_y_impl(d, alpha, linear, chr, st);
}
void launch_node2d(const Dev2D& d, const StageArgs& sa, int mode, bool linear, bool chr, cudaStream_t st) {
  node_impl(d, sa, mode, linear, chr, st);
}
void launch_sweep_x2d(const Dev2DT<float>& d, const float* alpha, bool linear, bool chr, cudaStream_t st) {
  sweep_x_impl(d, alpha, linear, chr, st);
}
void launch_sweep_y2d(const Dev2DT<float>& d, const float* alpha, bool linear, bool chr, cudaStream_t st) {
  sweep_y_impl(d, alpha, linear, chr, st);
}
void launch_node2d(const Dev2DT<float>& d, const StageArgsT<float>& sa, int mode, bool linear, bool chr,
                   cudaStream_t st) {
  node_impl(d, sa, mode, linear, chr, st);
}

// Plane conversion between precisions (the single-precision variant keeps double copies for the
// initialisation and the exchange with the caller).
__global__ void k_cast_planes(int nplanes, size_t n, Ptr12 src, Ptr12 dst, int to_float) {
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    for (int q = 0; q < nplanes; ++q) {
      if (to_float) ((float*)dst.p[q])[o] = (float)((const double*)src.p[q])[o];
      else ((double*)dst.p[q])[o] = (double)((const float*)src.p[q])[o];
    }
}

__global__ void k_scalars_to_float(const double* alpha, const double* dt, float* out) {
  out[0] = (float)alpha[0];
  out[1] = (float)alpha[1];
  out[2] = (float)*dt;
}

void launch_scalars_to_float(const double* alpha, const double* dt, float* out, cudaStream_t st) {
  k_scalars_to_float<<<1, 1, 0, st>>>(alpha, dt, out);
}

void launch_cast_planes(int nplanes, size_t n, const Ptr12& src, const Ptr12& dst, int to_float, cudaStream_t st) {
  int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)152 * 16);
  k_cast_planes<<<blocks, 256, 0, st>>>(nplanes, n, src, dst, to_float);
}

void launch_init2d(const Dev2D& d, const PhysIn& in, int* status, cudaStream_t st) {
  const size_t n = (size_t)d.nx * d.ny;
  int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)152 * 16);
  k_init2d<<<blocks, 256, 0, st>>>(d, in, status);
  dim3 g((d.nx + 1 + 31) / 32, (d.ny + 1 + 7) / 8);
  k_static2d<<<g, dim3(32, 8), 0, st>>>(d);
}

void launch_static2d(const Dev2D& d, cudaStream_t st) {
  dim3 g((d.nx + 1 + 31) / 32, (d.ny + 1 + 7) / 8);
  k_static2d<<<g, dim3(32, 8), 0, st>>>(d);
}

void launch_convert2d(const Dev2D& d, const Ptr9& src, const Ptr9& dst, int layout, int dir, cudaStream_t st) {
  const size_t n = (size_t)d.nx * d.ny;
  int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)152 * 16);
  k_convert2d<<<blocks, 256, 0, st>>>(d, src, dst, layout, dir);
}

}  // namespace hw
