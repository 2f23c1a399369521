// Batched form: many independent 2D grids of uneven sizes advance together, each with its own CFL
// time step. All instances share pooled planes; every phase of an RK stage (alpha reduction, x-sweep,
// y-sweep, node update) is ONE launch whose persistent blocks loop over a flattened list of tiles of
// every instance, so the launch count per step does not depend on the number of instances and small
// grids no longer leave the GPU idle. Two steps are captured in a CUDA graph. Tile shapes (interfaces
// per x-tile, interfaces per y-segment) are per instance, chosen by the autotuner. The arithmetic is
// the single-grid kernels' (hw_stencil2d.cuh), so each instance's result equals a single-grid
// solver's to rounding (the compiler may contract multiply-adds differently in the two kernels),
// with the same share of products on the integer pipes (bit-identical binary64, hw_fp64_int.h).
// No block ever waits on another block.
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/hwswe.h"
#include "hw_stencil2d.cuh"

namespace hw {

struct BInst {
  int nx, ny, bc_x, bc_y;
  double dx, dy, inv_dx, inv_dy, c_bx, c_by, c_gx, c_gy, c_mx, c_my;
  long long off_n, off_x, off_y;  // offsets of this grid in the pooled node / x-interface / y-interface planes
  int tx, seg;                     // x-tile row width (32, 64 or 128 threads = tx - 3 interfaces and their
                                   // tx node records; 128/tx rows per block), y segment
};

struct BatchDev {
  double g, eps_w, eps_lim, cfl;
  int limiter, k;
  const BInst* inst;
  double* S[9];
  double* stat[3];
  double* bxy[2];
  double* X[12];
  double* Y[12];
  double* qbx[6];
  double* qby[6];
  double* sv[2];
  double* sq[2];
  double* out[9];
  double* base[9];
  unsigned long long* amax;  // 2 per instance
  double* alpha;             // 2 per instance
  double* dt;                // 2 per instance: step, time after the step
  double* t;                 // 1 per instance
  unsigned long long* nsteps;
  int* status;
};

__device__ __forceinline__ void make_dev(const BatchDev& B, const BInst& I, Dev2D& d) {
  d.nx = I.nx; d.ny = I.ny; d.bc_x = I.bc_x; d.bc_y = I.bc_y;
  d.dx = I.dx; d.dy = I.dy; d.inv_dx = I.inv_dx; d.inv_dy = I.inv_dy;
  d.g = B.g; d.eps_w = B.eps_w; d.eps_lim = B.eps_lim;
  d.c_bx = I.c_bx; d.c_by = I.c_by; d.c_gx = I.c_gx; d.c_gy = I.c_gy; d.c_mx = I.c_mx; d.c_my = I.c_my;
#pragma unroll
  for (int q = 0; q < 9; ++q) d.S[q] = B.S[q] + I.off_n;
#pragma unroll
  for (int q = 0; q < 3; ++q) d.stat[q] = B.stat[q] + I.off_n;
#pragma unroll
  for (int q = 0; q < 2; ++q) d.bxy[q] = B.bxy[q] + I.off_n;
#pragma unroll
  for (int q = 0; q < 12; ++q) { d.X[q] = B.X[q] + I.off_x; d.Y[q] = B.Y[q] + I.off_y; }
#pragma unroll
  for (int q = 0; q < 6; ++q) { d.qbx[q] = B.qbx[q] + I.off_x; d.qby[q] = B.qby[q] + I.off_y; }
#pragma unroll
  for (int q = 0; q < 2; ++q) { d.sv[q] = B.sv[q] + I.off_n; d.sq[q] = B.sq[q] + I.off_n; }
}

constexpr int BX_THREADS = 128;
constexpr int BX_MAXN = BX_THREADS;     // node records per block: one per thread
constexpr int BY_W = 32;

// ---- alpha per instance: items (inst, first node, count) ----
__global__ void __launch_bounds__(256) k_balpha(BatchDev B, const int4* __restrict__ items, int nitems) {
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];
    const BInst& I = B.inst[it.x];
    const double* eta = B.S[0] + I.off_n;
    const double* m = B.S[1] + I.off_n;
    const double* wv = B.S[2] + I.off_n;
    const double* b = B.stat[0] + I.off_n;
    unsigned long long kx = 0, ky = 0;
    int bad = 0;
    for (int o = it.y + threadIdx.x; o < it.y + it.z; o += blockDim.x) {
      const double h = __ldg(eta + o) - __ldg(b + o);
      if (!(h > 0.0) || !(h < 1e300)) { bad = 1; continue; }
      const double rh = fast_rcp(h);
      const double gh = B.g * h;
      const double c = gh * fast_rsqrt(gh);
      const double ax = dabs(__ldg(m + o) * rh) + c, ay = dabs(__ldg(wv + o) * rh) + c;
      if (!(ax < 1e300) || !(ay < 1e300)) { bad = 1; continue; }
      kx = max(kx, dkey(ax));
      ky = max(ky, dkey(ay));
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      kx = max(kx, __shfl_xor_sync(0xffffffffu, kx, s));
      ky = max(ky, __shfl_xor_sync(0xffffffffu, ky, s));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(B.amax + 2 * it.x, kx);
      atomicMax(B.amax + 2 * it.x + 1, ky);
    }
    if (bad) atomicOr(B.status, HW_STATUS_DEPTH);
  }
}

// ---- per instance: alpha from the keys; at a step's start dt = cfl / (ax/dx + ay/dy) ----
__global__ void k_bfinish(BatchDev B, int n, int with_dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ax = __longlong_as_double((long long)B.amax[2 * i]);
  const double ay = __longlong_as_double((long long)B.amax[2 * i + 1]);
  B.alpha[2 * i] = ax;
  B.alpha[2 * i + 1] = ay;
  if (with_dt) {
    const BInst& I = B.inst[i];
    const double dt = B.cfl / fma(ax, I.inv_dx, ay * I.inv_dy);
    B.dt[2 * i] = dt;
    B.dt[2 * i + 1] = B.t[i] + dt;
  }
}

__global__ void k_btime(BatchDev B, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  B.t[i] = B.dt[2 * i + 1];
  if (B.dt[2 * i] > 0.0) ++B.nsteps[i];
}

// ---- x-sweep: items (inst, first row, first interface) ----
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(BX_THREADS, 3) k_bsweep_x(BatchDev B, const int4* __restrict__ items, int nitems) {
  __shared__ double sm[NREC * BX_MAXN];
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];
    const BInst I = B.inst[it.x];
    Dev2D d;
    make_dev(B, I, d);
    const int tx = I.tx, R = BX_THREADS / tx, NN = tx, stride = R * NN;  // tx - 3 interfaces per row
    const int j0 = it.y, k0 = it.z;
    const double ax = B.alpha[2 * it.x];
    for (int t = threadIdx.x; t < stride; t += BX_THREADS) {
      const int r = t / NN, c = t - r * NN;
      const int j = j0 + r, i = k0 - 2 + c;
      if (j >= d.ny || i > d.nx + 1) continue;
      Node12 n;
      load_node(d, i, j, n);
      double rec[NREC];
      node_record<0>(n, d.g, ax, rec);
#pragma unroll
      for (int f = 0; f < NREC; ++f) sm[f * stride + t] = rec[f];
    }
    __syncthreads();
    const int r = threadIdx.x / tx, c = threadIdx.x - r * tx;
    const int j = j0 + r, k = k0 + c;
    if (c < tx - 3 && j < d.ny && k <= d.nx) {
      const int t0 = r * NN + c;
      const size_t o = (size_t)j * (d.nx + 1) + k;
      double qb[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) qb[q] = __ldg(d.qbx[q] + o);
      double out[12];
      interface_values<0, LINEAR, CHAR, true>(sm + t0, sm + t0 + 1, sm + t0 + 2, sm + t0 + 3, stride, qb, d.g, d.eps_w, out);
#pragma unroll
      for (int q = 0; q < 12; ++q) d.X[q][o] = out[q];
    }
    __syncthreads();
  }
}

// ---- y-sweep: items (inst, first column, first interface); each thread marches its column ----
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(BY_W, 12) k_bsweep_y(BatchDev B, const int4* __restrict__ items, int nitems) {
  extern __shared__ double ring[];  // [4][NREC][BY_W]
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];
    const BInst I = B.inst[it.x];
    Dev2D d;
    make_dev(B, I, d);
    const int i = it.y + threadIdx.x;
    if (i >= d.nx) continue;
    const int k0 = it.z, seg = I.seg;
    const double ay = B.alpha[2 * it.x + 1];
    const int rend = min(k0 + seg, d.ny + 1);
    for (int r = k0 - 2; r <= rend; ++r) {
      Node12 n;
      load_node(d, i, r, n);
      double rec[NREC];
      node_record<1>(n, d.g, ay, rec);
      double* slot = ring + (size_t)(r & 3) * NREC * BY_W + threadIdx.x;
#pragma unroll
      for (int f = 0; f < NREC; ++f) slot[f * BY_W] = rec[f];
      const int k = r - 1;
      if (k >= k0 && k < k0 + seg && k <= d.ny) {
        const double* s0 = ring + (size_t)((k - 2) & 3) * NREC * BY_W + threadIdx.x;
        const double* s1 = ring + (size_t)((k - 1) & 3) * NREC * BY_W + threadIdx.x;
        const double* s2 = ring + (size_t)((k) & 3) * NREC * BY_W + threadIdx.x;
        const double* s3 = ring + (size_t)((k + 1) & 3) * NREC * BY_W + threadIdx.x;
        const size_t o = (size_t)k * d.nx + i;
        double qb[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) qb[q] = __ldg(d.qby[q] + o);
        double out[12];
        interface_values<1, LINEAR, CHAR, true>(s0, s1, s2, s3, BY_W, qb, d.g, d.eps_w, out);
#pragma unroll
        for (int q = 0; q < 12; ++q) d.Y[q][o] = out[q];
      }
    }
  }
}

// ---- node update: items (inst, first column, first row) of 32 x 8 tiles ----
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(256, 2) k_bnode(BatchDev B, const int4* __restrict__ items, int nitems) {
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];
    const BInst I = B.inst[it.x];
    const int i = it.y + threadIdx.x, j = it.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) continue;
    Dev2D d;
    make_dev(B, I, d);
    StageArgs sa;
    sa.k = B.k;
    sa.limiter = B.limiter;
    sa.dt = B.dt + 2 * it.x;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      sa.out[q] = B.out[q] + I.off_n;
      sa.base[q] = B.base[q] + I.off_n;
      sa.rhs_out[q] = nullptr;
    }
    node_update<MODE_STAGE, LINEAR, CHAR, true>(d, sa, i, j);
  }
}

}  // namespace hw

// =============================================================================================
// Host side
// =============================================================================================
namespace {
int bfail(int code, const std::string& m) { return hw::set_last_error(code, m.c_str()); }
#define BCUDA(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return bfail(HW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
}  // namespace

struct hw_batch {
  int n = 0;
  hw_params params{};
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::vector<hw_grid> grids;
  std::vector<hw::BInst> inst;  // host copy
  hw::BInst* d_inst = nullptr;
  size_t tot_n = 0, tot_x = 0, tot_y = 0;
  std::vector<void*> allocs;
  double* SA[9] = {};
  double* SB[9] = {};
  int cur = 0;
  double* staging[12] = {};  // sized for the largest instance
  size_t max_n = 0;
  hw::BatchDev B{};
  // work lists
  int4* d_items[4] = {};  // alpha, x, y, node
  int nitems[4] = {};
  int nb[4] = {1, 1, 1, 1};  // persistent grid size per phase (resident blocks on the device)
  std::vector<bool> inited;
  bool dirty = false;  // tile shapes changed since the work lists were built
  cudaGraphExec_t graph = nullptr;
};

namespace {
int balloc(hw_batch* b, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return bfail(HW_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  b->allocs.push_back(*p);
  return HW_OK;
}

// Per-instance Dev2D for the single-grid launchers (init, static terms, conversions).
hw::Dev2D dev_of(hw_batch* b, int i, double** S) {
  const hw::BInst& I = b->inst[i];
  hw::Dev2D d{};
  d.nx = I.nx; d.ny = I.ny; d.bc_x = I.bc_x; d.bc_y = I.bc_y;
  d.dx = I.dx; d.dy = I.dy; d.inv_dx = I.inv_dx; d.inv_dy = I.inv_dy;
  d.g = b->params.g; d.eps_w = b->params.eps_w; d.eps_lim = b->params.eps_lim;
  d.c_bx = I.c_bx; d.c_by = I.c_by; d.c_gx = I.c_gx; d.c_gy = I.c_gy; d.c_mx = I.c_mx; d.c_my = I.c_my;
  for (int q = 0; q < 9; ++q) d.S[q] = S[q] + I.off_n;
  for (int q = 0; q < 3; ++q) d.stat[q] = b->B.stat[q] + I.off_n;
  for (int q = 0; q < 2; ++q) d.bxy[q] = b->B.bxy[q] + I.off_n;
  for (int q = 0; q < 12; ++q) { d.X[q] = b->B.X[q] + I.off_x; d.Y[q] = b->B.Y[q] + I.off_y; }
  for (int q = 0; q < 6; ++q) { d.qbx[q] = b->B.qbx[q] + I.off_x; d.qby[q] = b->B.qby[q] + I.off_y; }
  for (int q = 0; q < 2; ++q) { d.sv[q] = b->B.sv[q] + I.off_n; d.sq[q] = b->B.sq[q] + I.off_n; }
  return d;
}

int default_tx(int nx) { return nx + 1 > 96 ? 128 : (nx + 1 > 48 ? 64 : 32); }

// Work lists for a subset of instances with their current tile shapes.
void build_items(const std::vector<hw::BInst>& inst, const std::vector<int>& ids, std::vector<int4> out[4]) {
  for (int p = 0; p < 4; ++p) out[p].clear();
  for (int i : ids) {
    const hw::BInst& I = inst[i];
    const int n = I.nx * I.ny;
    for (int o = 0; o < n; o += 4096) out[0].push_back(make_int4(i, o, std::min(4096, n - o), 0));
    const int R = hw::BX_THREADS / I.tx;
    for (int j = 0; j < I.ny; j += R)
      for (int k = 0; k <= I.nx; k += I.tx - 3) out[1].push_back(make_int4(i, j, k, 0));
    for (int c = 0; c < I.nx; c += hw::BY_W)
      for (int k = 0; k <= I.ny; k += I.seg) out[2].push_back(make_int4(i, c, k, 0));
    for (int j = 0; j < I.ny; j += 8)
      for (int c = 0; c < I.nx; c += 32) out[3].push_back(make_int4(i, c, j, 0));
  }
}

int upload_items(hw_batch* b, std::vector<int4> lists[4], int4** dst, int* counts) {
  for (int p = 0; p < 4; ++p) {
    if (dst[p]) { cudaFree(dst[p]); dst[p] = nullptr; }
    counts[p] = (int)lists[p].size();
    if (counts[p] == 0) continue;
    BCUDA(cudaMalloc(&dst[p], lists[p].size() * sizeof(int4)));
    BCUDA(cudaMemcpyAsync(dst[p], lists[p].data(), lists[p].size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  }
  BCUDA(cudaStreamSynchronize(b->stream));
  return HW_OK;
}

int persistent_blocks(const void* fn, int threads, size_t smem) {
  int dev = 0, sms = 1, bps = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem) != cudaSuccess || bps < 1) bps = 1;
  return sms * bps;
}

const size_t kRingBytes = (size_t)4 * hw::NREC * hw::BY_W * sizeof(double);

template <bool L, bool C>
void launch_phases(hw_batch* b, int which, int4* const* items, const int* counts, cudaStream_t st) {
  // which: bit 0 x-sweep, bit 1 y-sweep, bit 2 node
  if ((which & 1) && counts[1])
    hw::k_bsweep_x<L, C><<<std::min(b->nb[1], counts[1]), hw::BX_THREADS, 0, st>>>(b->B, items[1], counts[1]);
  if ((which & 2) && counts[2])
    hw::k_bsweep_y<L, C><<<std::min(b->nb[2], counts[2]), hw::BY_W, kRingBytes, st>>>(b->B, items[2], counts[2]);
  if ((which & 4) && counts[3])
    hw::k_bnode<L, C><<<std::min(b->nb[3], counts[3]), dim3(32, 8), 0, st>>>(b->B, items[3], counts[3]);
}

template <bool L, bool C>
int prime_blocks(hw_batch* b) {
  if (cudaFuncSetAttribute(hw::k_bsweep_y<L, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes) != cudaSuccess)
    return -1;
  b->nb[0] = persistent_blocks((const void*)hw::k_balpha, 256, 0);
  b->nb[1] = persistent_blocks((const void*)hw::k_bsweep_x<L, C>, hw::BX_THREADS, 0);
  b->nb[2] = persistent_blocks((const void*)hw::k_bsweep_y<L, C>, hw::BY_W, kRingBytes);
  b->nb[3] = persistent_blocks((const void*)hw::k_bnode<L, C>, 256, 0);
  return 0;
}

void enqueue_phases(hw_batch* b, int which, int4* const* items, const int* counts, cudaStream_t st) {
  const bool lin = b->params.linear_weights != 0, chr = b->params.char_decomp != 0;
  if (lin) { if (chr) launch_phases<true, true>(b, which, items, counts, st); else launch_phases<true, false>(b, which, items, counts, st); }
  else     { if (chr) launch_phases<false, true>(b, which, items, counts, st); else launch_phases<false, false>(b, which, items, counts, st); }
}

void bind(hw_batch* b) {
  double** in = b->cur == 0 ? b->SA : b->SB;
  double** out = b->cur == 0 ? b->SB : b->SA;
  for (int q = 0; q < 9; ++q) { b->B.S[q] = in[q]; b->B.out[q] = out[q]; }
}

void enqueue_alpha(hw_batch* b, int with_dt, cudaStream_t st) {
  bind(b);
  cudaMemsetAsync(b->B.amax, 0, 2 * sizeof(unsigned long long) * b->n, st);
  hw::k_balpha<<<std::min(b->nb[0], b->nitems[0]), 256, 0, st>>>(b->B, b->d_items[0], b->nitems[0]);
  hw::k_bfinish<<<(b->n + 127) / 128, 128, 0, st>>>(b->B, b->n, with_dt);
}

void enqueue_step(hw_batch* b, cudaStream_t st) {
  for (int k = 1; k <= 3; ++k) {
    enqueue_alpha(b, k == 1, st);
    b->B.k = k;
    bind(b);
    enqueue_phases(b, 7, b->d_items, b->nitems, st);
    b->cur ^= 1;
  }
  hw::k_btime<<<(b->n + 127) / 128, 128, 0, st>>>(b->B, b->n);
}

int rebuild(hw_batch* b) {
  std::vector<int> ids(b->n);
  for (int i = 0; i < b->n; ++i) ids[i] = i;
  std::vector<int4> lists[4];
  build_items(b->inst, ids, lists);
  BCUDA(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(hw::BInst) * b->n, cudaMemcpyHostToDevice, b->stream));
  int rc = upload_items(b, lists, b->d_items, b->nitems);
  if (rc) return rc;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return HW_OK;
}
}  // namespace

extern "C" {

int hw_batch_create(int n, const hw_grid* grids, const hw_params* params, void* cuda_stream, hw_batch** out) {
  if (!grids || !params || !out || n < 1) return bfail(HW_ERR_ARG, "hw_batch_create: bad argument");
  *out = nullptr;
  if (params->precision != HW_FP64) return bfail(HW_ERR_ARG, "hw_batch_create: the batched form is HW_FP64 only");
  if (!(params->g > 0) || !(params->eps_w > 0) || !(params->eps_lim > 0) || !(params->cfl > 0))
    return bfail(HW_ERR_ARG, "hw_batch_create: g, cfl, eps_w and eps_lim must be positive");
  hw_batch* b = new hw_batch();
  b->n = n;
  b->params = *params;
  b->stream = (cudaStream_t)cuda_stream;
  b->grids.assign(grids, grids + n);
  b->inst.resize(n);
  b->inited.assign(n, false);
  for (int i = 0; i < n; ++i) {
    const hw_grid& g = grids[i];
    if (g.dim != 2 || g.nx < 2 || g.ny < 2 || g.bc_x < 0 || g.bc_x > 2 || g.bc_y < 0 || g.bc_y > 2 ||
        !(g.x1 > g.x0) || !(g.y1 > g.y0) || (size_t)g.nx * g.ny > ((size_t)1 << 30)) {
      delete b;
      return bfail(HW_ERR_ARG, "hw_batch_create: every grid must be 2D with nx, ny >= 2 and a valid domain");
    }
    hw::BInst& I = b->inst[i];
    I.nx = g.nx; I.ny = g.ny; I.bc_x = g.bc_x; I.bc_y = g.bc_y;
    I.dx = (g.x1 - g.x0) / g.nx; I.dy = (g.y1 - g.y0) / g.ny;
    I.inv_dx = 1.0 / I.dx; I.inv_dy = 1.0 / I.dy;
    I.c_bx = 0.5 / I.dx; I.c_by = 0.5 / I.dy; I.c_gx = 1.0 / (24.0 * I.dx); I.c_gy = 1.0 / (24.0 * I.dy);
    I.c_mx = 1.0 / (12.0 * I.dx); I.c_my = 1.0 / (12.0 * I.dy);
    I.off_n = (long long)b->tot_n; I.off_x = (long long)b->tot_x; I.off_y = (long long)b->tot_y;
    I.tx = default_tx(g.nx);
    I.seg = 64;
    b->tot_n += (size_t)g.nx * g.ny;
    b->tot_x += (size_t)(g.nx + 1) * g.ny;
    b->tot_y += (size_t)g.nx * (g.ny + 1);
    b->max_n = std::max(b->max_n, (size_t)g.nx * g.ny);
  }
  int rc = HW_OK;
  auto A = [&](double** p, size_t cnt) {
    if (rc == HW_OK) rc = balloc(b, (void**)p, cnt * sizeof(double));
  };
  for (int q = 0; q < 9; ++q) { A(&b->SA[q], b->tot_n); A(&b->SB[q], b->tot_n); A(&b->B.base[q], b->tot_n); }
  for (int q = 0; q < 3; ++q) A(&b->B.stat[q], b->tot_n);
  for (int q = 0; q < 2; ++q) A(&b->B.bxy[q], b->tot_n);
  for (int q = 0; q < 12; ++q) { A(&b->B.X[q], b->tot_x); A(&b->B.Y[q], b->tot_y); }
  for (int q = 0; q < 6; ++q) { A(&b->B.qbx[q], b->tot_x); A(&b->B.qby[q], b->tot_y); }
  for (int q = 0; q < 2; ++q) { A(&b->B.sv[q], b->tot_n); A(&b->B.sq[q], b->tot_n); }
  for (int q = 0; q < 12; ++q) A(&b->staging[q], b->max_n);
  double* misc = nullptr;
  A(&misc, (size_t)8 * n + 8);
  if (rc == HW_OK) rc = balloc(b, (void**)&b->d_inst, sizeof(hw::BInst) * n);
  if (rc != HW_OK) { hw_batch_destroy(b); return rc; }
  b->B.amax = (unsigned long long*)misc;
  b->B.alpha = misc + 2 * n;
  b->B.dt = misc + 4 * n;
  b->B.t = misc + 6 * n;
  b->B.nsteps = (unsigned long long*)(misc + 7 * n);
  b->B.status = (int*)(misc + 8 * n);
  b->B.g = params->g; b->B.eps_w = params->eps_w; b->B.eps_lim = params->eps_lim; b->B.cfl = params->cfl;
  b->B.limiter = params->limiter;
  b->B.inst = b->d_inst;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { b->cap_stream = nullptr; hw_batch_destroy(b); return bfail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  e = cudaMemsetAsync(misc, 0, ((size_t)8 * n + 8) * sizeof(double), b->stream);
  if (e != cudaSuccess) { hw_batch_destroy(b); return bfail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  {
    const bool lin = params->linear_weights != 0, chr = params->char_decomp != 0;
    const int pr = lin ? (chr ? prime_blocks<true, true>(b) : prime_blocks<true, false>(b))
                       : (chr ? prime_blocks<false, true>(b) : prime_blocks<false, false>(b));
    if (pr != 0) { hw_batch_destroy(b); return bfail(HW_ERR_CUDA, "hw_batch_create: kernel attributes"); }
  }
  rc = rebuild(b);
  if (rc != HW_OK) { hw_batch_destroy(b); return rc; }
  *out = b;
  return HW_OK;
}

int hw_batch_destroy(hw_batch* b) {
  if (!b) return HW_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (int p = 0; p < 4; ++p)
    if (b->d_items[p]) cudaFree(b->d_items[p]);
  for (void* p : b->allocs) cudaFree(p);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  return HW_OK;
}

int hw_batch_init(hw_batch* b, int i, const double* h, const double* hu, const double* hv, const double* bb,
                  const double* const* deriv, int ptr_kind) {
  if (!b || i < 0 || i >= b->n || !h || !hu || !hv || !bb || !deriv) return bfail(HW_ERR_ARG, "hw_batch_init: bad argument");
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return bfail(HW_ERR_ARG, "hw_batch_init: bad ptr_kind");
  const hw::BInst& I = b->inst[i];
  const size_t n = (size_t)I.nx * I.ny;
  const double* in[12] = {h, hu, hv, bb, deriv[0], deriv[1], deriv[2], deriv[3], deriv[4], deriv[5], deriv[6], deriv[7]};
  hw::PhysIn pin;
  for (int q = 0; q < 12; ++q) {
    if (!in[q]) return bfail(HW_ERR_ARG, "hw_batch_init: null plane");
    if (ptr_kind == HW_DEVICE) {
      pin.p[q] = in[q];
    } else {
      BCUDA(cudaMemcpyAsync(b->staging[q], in[q], n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
      pin.p[q] = b->staging[q];
    }
  }
  hw::Dev2D d = dev_of(b, i, b->cur == 0 ? b->SA : b->SB);
  hw::launch_init2d(d, pin, b->B.status, b->stream);
  BCUDA(cudaGetLastError());
  BCUDA(cudaMemsetAsync(b->B.t + i, 0, sizeof(double), b->stream));
  BCUDA(cudaMemsetAsync(b->B.nsteps + i, 0, sizeof(unsigned long long), b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  int st = 0;
  BCUDA(cudaMemcpy(&st, b->B.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    BCUDA(cudaMemset(b->B.status, 0, sizeof(int)));
    return bfail(HW_ERR_DEPTH, "hw_batch_init: non-positive or non-finite depth");
  }
  b->inited[i] = true;
  return HW_OK;
}

int hw_batch_run(hw_batch* b, int nsteps, int use_graph) {
  if (!b || nsteps < 0) return bfail(HW_ERR_ARG, "hw_batch_run: bad argument");
  for (int i = 0; i < b->n; ++i)
    if (!b->inited[i]) return bfail(HW_ERR_STATE, "hw_batch_run: every instance must be initialised");
  if (b->dirty) {
    int rc = rebuild(b);
    if (rc != HW_OK) return rc;
    b->dirty = false;
  }
  if (use_graph && (!b->graph || b->cur != 0) && b->cur == 0) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    BCUDA(cudaStreamSynchronize(b->stream));
    cudaGraph_t g = nullptr;
    BCUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step(b, b->cap_stream);
    enqueue_step(b, b->cap_stream);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    b->cur = 0;
    if (e != cudaSuccess) return bfail(HW_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return bfail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  }
  int done = 0;
  while (done < nsteps) {
    if (use_graph && b->graph && b->cur == 0 && nsteps - done >= 2) {
      BCUDA(cudaGraphLaunch(b->graph, b->stream));
      done += 2;
    } else {
      enqueue_step(b, b->stream);
      done += 1;
    }
  }
  BCUDA(cudaGetLastError());
  BCUDA(cudaStreamSynchronize(b->stream));
  int st = 0;
  BCUDA(cudaMemcpy(&st, b->B.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    BCUDA(cudaMemset(b->B.status, 0, sizeof(int)));
    return bfail(HW_ERR_DEPTH, "hw_batch_run: non-positive or non-finite depth in some instance");
  }
  return HW_OK;
}

int hw_batch_get_state(hw_batch* b, int i, double* const* out, int layout, int ptr_kind) {
  if (!b || i < 0 || i >= b->n || !out) return bfail(HW_ERR_ARG, "hw_batch_get_state: bad argument");
  if (layout != HW_LAYOUT_PHYSICAL && layout != HW_LAYOUT_EQUILIBRIUM) return bfail(HW_ERR_ARG, "bad layout");
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return bfail(HW_ERR_ARG, "bad ptr_kind");
  const hw::BInst& I = b->inst[i];
  const size_t n = (size_t)I.nx * I.ny;
  hw::Ptr9 src{}, dst{};
  for (int q = 0; q < 9; ++q) {
    if (!out[q]) return bfail(HW_ERR_ARG, "null output plane");
    dst.p[q] = ptr_kind == HW_DEVICE ? out[q] : b->staging[q];
  }
  hw::Dev2D d = dev_of(b, i, b->cur == 0 ? b->SA : b->SB);
  hw::launch_convert2d(d, src, dst, layout, 0, b->stream);
  BCUDA(cudaGetLastError());
  if (ptr_kind == HW_HOST)
    for (int q = 0; q < 9; ++q)
      BCUDA(cudaMemcpyAsync(out[q], dst.p[q], n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  return HW_OK;
}

int hw_batch_get_time(hw_batch* b, double* t, int* steps) {
  if (!b) return bfail(HW_ERR_ARG, "hw_batch_get_time: null batch");
  std::vector<double> tt(b->n);
  std::vector<unsigned long long> ns(b->n);
  BCUDA(cudaMemcpyAsync(tt.data(), b->B.t, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaMemcpyAsync(ns.data(), b->B.nsteps, sizeof(unsigned long long) * b->n, cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->n; ++i) {
    if (t) t[i] = tt[i];
    if (steps) steps[i] = (int)ns[i];
  }
  return HW_OK;
}

int hw_batch_set_tiles(hw_batch* b, int i, int tx, int seg) {
  if (!b || i < 0 || i >= b->n) return bfail(HW_ERR_ARG, "hw_batch_set_tiles: bad instance");
  if (tx != 32 && tx != 64 && tx != 128) return bfail(HW_ERR_ARG, "hw_batch_set_tiles: tx must be 32, 64 or 128");
  if (seg < 1) return bfail(HW_ERR_ARG, "hw_batch_set_tiles: seg must be >= 1");
  b->inst[i].tx = tx;
  b->inst[i].seg = std::min(seg, b->inst[i].ny + 1);
  b->dirty = true;  // work lists are rebuilt by the next run
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return HW_OK;
}

int hw_batch_get_tiles(hw_batch* b, int i, int* tx, int* seg) {
  if (!b || i < 0 || i >= b->n || !tx || !seg) return bfail(HW_ERR_ARG, "hw_batch_get_tiles: bad argument");
  *tx = b->inst[i].tx;
  *seg = b->inst[i].seg;
  return HW_OK;
}

// Time the x- and y-sweeps of one stage over a subset of instances with trial tile shapes (the
// autotuner's measurement). Writes only interface planes, which every stage recomputes.
int hw_batch_time_tiles(hw_batch* b, int nids, const int* ids, int tx, int seg, int reps, double* ms_x, double* ms_y) {
  if (!b || nids < 1 || !ids || reps < 1) return bfail(HW_ERR_ARG, "hw_batch_time_tiles: bad argument");
  if (tx != 32 && tx != 64 && tx != 128) return bfail(HW_ERR_ARG, "hw_batch_time_tiles: tx must be 32, 64 or 128");
  std::vector<hw::BInst> trial = b->inst;
  std::vector<int> sub(ids, ids + nids);
  for (int i : sub) {
    if (i < 0 || i >= b->n) return bfail(HW_ERR_ARG, "hw_batch_time_tiles: bad instance id");
    trial[i].tx = tx;
    trial[i].seg = std::max(1, std::min(seg, trial[i].ny + 1));
  }
  std::vector<int4> lists[4];
  build_items(trial, sub, lists);
  int4* items[4] = {};
  int counts[4] = {};
  BCUDA(cudaMemcpyAsync(b->d_inst, trial.data(), sizeof(hw::BInst) * b->n, cudaMemcpyHostToDevice, b->stream));
  int rc = upload_items(b, lists, items, counts);
  if (rc) return rc;
  bind(b);
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
  enqueue_phases(b, 3, items, counts, b->stream);  // warm-up
  float tx_ms = 0.f, ty_ms = 0.f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, b->stream);
    enqueue_phases(b, 1, items, counts, b->stream);
    cudaEventRecord(e1, b->stream);
    enqueue_phases(b, 2, items, counts, b->stream);
    cudaEventRecord(e2, b->stream);
    cudaEventSynchronize(e2);
    float a = 0.f, c = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&c, e1, e2);
    tx_ms += a;
    ty_ms += c;
  }
  cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
  for (int p = 0; p < 4; ++p)
    if (items[p]) cudaFree(items[p]);
  BCUDA(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(hw::BInst) * b->n, cudaMemcpyHostToDevice, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  if (ms_x) *ms_x = tx_ms / reps;
  if (ms_y) *ms_y = ty_ms / reps;
  return HW_OK;
}

}  // extern "C"
