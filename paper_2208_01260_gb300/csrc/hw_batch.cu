// Batched form: many independent 2D grids of uneven sizes advance together, each with its own CFL
// time step. All instances share pooled planes; every phase of an RK stage (alpha reduction, x-sweep,
// y-sweep, node update) is ONE launch over a flattened list of work items of every instance (one block
// per item; the alpha passes loop over theirs), so the launch count per step does not depend on the
// number of instances and small grids no longer leave the GPU idle. Two steps are captured in a CUDA
// graph. The sweeps use the single-grid tiles over flattened extended lines (hw_stencil2d.cuh), so no
// grid size leaves a ragged tile; the y-tile width is per instance, chosen by the autotuner. The
// arithmetic is the single-grid kernels', so each instance's result equals a single-grid solver's to
// rounding (the compiler may contract multiply-adds differently in the two kernels), with the same
// share of products on the integer pipes (each bit-identical to DMUL, hw_fp64_int.h). The kernels read
// the pooled planes through the parameters' base pointers plus the instance's offsets, so that no
// per-instance pointer takes a register. No block ever waits on another block. hw_batch_set_persistent
// switches a batch to one cooperative launch per step instead (hw_bstep.cu).
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/hwswe.h"
#include "hw_batch.cuh"

namespace hw {

constexpr int BN_T = 256;  // nodes per node-kernel item

// ---- alpha per instance in two passes, as the single-grid reduction (a float estimate of every node,
// the double value only near the float maximum): items (inst, first node, count) ----
__global__ void __launch_bounds__(256) k_balpha_coarse(BatchDev B, const int4* __restrict__ items, int nitems) {
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];
    const BInst& I = B.inst[it.x];
    Dev2D d;
    make_dev(B, I, d);
    float mx = 0.0f, my = 0.0f;
    int bad = 0;
    const size_t base = (size_t)I.off_n;
    for (int o = it.y + threadIdx.x; o < it.y + it.z; o += blockDim.x) {
      float ax, ay;
      bool exact, neg;
      alpha_coarse(d, base + o, ax, ay, exact, neg);
      if (exact) continue;
      if (neg) { bad |= HW_STATUS_DEPTH; continue; }
      mx = fmaxf(mx, ax);
      my = fmaxf(my, ay);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
      my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, s));
    }
    unsigned int* m32 = reinterpret_cast<unsigned int*>(B.amax + 3 * it.x + 2);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(m32, __float_as_uint(mx));
      atomicMax(m32 + 1, __float_as_uint(my));
    }
    if (bad) atomicOr(B.status, bad);
  }
}

__global__ void __launch_bounds__(256) k_balpha_exact(BatchDev B, const int4* __restrict__ items, int nitems) {
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];
    const BInst& I = B.inst[it.x];
    Dev2D d;
    make_dev(B, I, d);
    const unsigned int* m32 = reinterpret_cast<const unsigned int*>(B.amax + 3 * it.x + 2);
    unsigned long long kx = 0, ky = 0;
    int bad = 0;
    const size_t base = (size_t)I.off_n;
    alpha_exact_range(d, m32, base + it.y + threadIdx.x, base + it.y + it.z, blockDim.x, kx, ky, bad);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      kx = max(kx, __shfl_xor_sync(0xffffffffu, kx, s));
      ky = max(ky, __shfl_xor_sync(0xffffffffu, ky, s));
    }
    if ((threadIdx.x & 31) == 0) {
      if (kx) atomicMax(B.amax + 3 * it.x, kx);
      if (ky) atomicMax(B.amax + 3 * it.x + 1, ky);
    }
    if (bad) atomicOr(B.status, bad);
  }
}

// ---- per instance: alpha from the keys; at a step's start dt = cfl / (ax/dx + ay/dy) ----
__global__ void k_bfinish(BatchDev B, int n, int with_dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ax = __longlong_as_double((long long)B.amax[3 * i]);
  const double ay = __longlong_as_double((long long)B.amax[3 * i + 1]);
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

// ---- x-sweep: items (inst, first extended node of the tile) over the flattened extended rows ----
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(TILE_T, 2) k_bsweep_x(BatchDev B, const int4* __restrict__ items, int nitems) {
  __shared__ double sm[NREC * TILE_T];
  {
    const int4 it = items[blockIdx.x];
    const BInst& I = B.inst[it.x];
    Dev2D d;
    make_dev(B, I, d);
    sweep_x_tile<LINEAR, CHAR, true>(d, B.alpha[2 * it.x], (unsigned)it.y, sm, (size_t)I.off_n, (size_t)I.off_x);
  }
}

// ---- y-sweep: items (inst, first extended row of the tile) over the flattened column groups ----
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(TILE_T, 2) k_bsweep_y(BatchDev B, const int4* __restrict__ items, int nitems) {
  __shared__ double sm[NREC * TILE_T];
  {
    const int4 it = items[blockIdx.x];
    const BInst& I = B.inst[it.x];
    Dev2D d;
    make_dev(B, I, d);
    sweep_y_tile<LINEAR, CHAR, true>(d, B.alpha[2 * it.x + 1], (unsigned)it.y, I.yc, sm, (size_t)I.off_n,
                                     (size_t)I.off_y);
  }
}

// ---- node update: items (inst, first node) of BN_T consecutive nodes of one grid ----
// Two blocks per SM: the instance's grid constants come from global memory and take registers that the
// single-grid kernel keeps in its parameters (measured: 3 blocks per SM spill 0.75 KB per thread and run
// no faster).
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(BN_T, 2) k_bnode(BatchDev B, const int4* __restrict__ items, int nitems) {
  {
    const int4 it = items[blockIdx.x];
    const BInst& I = B.inst[it.x];
    const int o = it.y + threadIdx.x;
    if (o >= I.nx * I.ny) return;
    const int j = o / I.nx, i = o - j * I.nx;
    Dev2D d;
    make_dev(B, I, d);
    StageArgs sa;
    sa.k = B.k;
    sa.limiter = B.limiter;
    sa.dt = B.dt + 2 * it.x;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      sa.out[q] = B.out[q];
      sa.base[q] = B.base[q];
      sa.rhs_out[q] = nullptr;
    }
    node_update<MODE_STAGE, LINEAR, CHAR, true>(d, sa, i, j, (size_t)I.off_n, (size_t)I.off_x, (size_t)I.off_y);
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
  int4* d_items[5] = {};  // alpha, x, y, node (BN_T nodes), node (TILE_T nodes, persistent step)
  int nitems[5] = {};
  // persistent step: one cooperative launch per step over bstep_blocks resident blocks
  bool persistent = false;
  int bstep_blocks = 0;
  hw::StepSync* d_sync = nullptr;
  int nb[1] = {1};  // blocks of the alpha passes (resident blocks on the device; they loop over items)
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

// Work lists of a subset of instances: alpha (inst, first node, count), x-sweep tiles (inst, first
// extended node), y-sweep tiles (inst, first extended row of a column group), node items (inst, first node)
// of BN_T nodes for the node kernel and of TILE_T nodes for the persistent step.
void build_items(const std::vector<hw::BInst>& inst, const std::vector<int>& ids, std::vector<int4> out[5]) {
  for (int p = 0; p < 5; ++p) out[p].clear();
  for (int i : ids) {
    const hw::BInst& I = inst[i];
    const int n = I.nx * I.ny;
    for (int o = 0; o < n; o += 4096) out[0].push_back(make_int4(i, o, std::min(4096, n - o), 0));
    const long long tx = (long long)I.ny * (I.nx + 4);
    for (long long e = 0; e < tx; e += hw::TILE_T - 3) out[1].push_back(make_int4(i, (int)e, 0, 0));
    const int ifs = hw::TILE_T / I.yc - 3;
    const long long ty = (long long)((I.nx + I.yc - 1) / I.yc) * (I.ny + 4);
    for (long long e = 0; e < ty; e += ifs) out[2].push_back(make_int4(i, (int)e, 0, 0));
    for (int o = 0; o < n; o += hw::BN_T) out[3].push_back(make_int4(i, o, 0, 0));
    for (int o = 0; o < n; o += hw::TILE_T) out[4].push_back(make_int4(i, o, 0, 0));
  }
}

int upload_items(hw_batch* b, std::vector<int4> lists[5], int4** dst, int* counts) {
  for (int p = 0; p < 5; ++p) {
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

template <bool L, bool C>
void launch_phases(hw_batch* b, int which, int4* const* items, const int* counts, cudaStream_t st) {
  // which: bit 0 x-sweep, bit 1 y-sweep, bit 2 node; one block per work item
  if ((which & 1) && counts[1]) hw::k_bsweep_x<L, C><<<counts[1], hw::TILE_T, 0, st>>>(b->B, items[1], counts[1]);
  if ((which & 2) && counts[2]) hw::k_bsweep_y<L, C><<<counts[2], hw::TILE_T, 0, st>>>(b->B, items[2], counts[2]);
  if ((which & 4) && counts[3]) hw::k_bnode<L, C><<<counts[3], hw::BN_T, 0, st>>>(b->B, items[3], counts[3]);
}

template <bool L, bool C>
int prime_blocks(hw_batch* b) {
  b->nb[0] = persistent_blocks((const void*)hw::k_balpha_exact, 256, 0);
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
  cudaMemsetAsync(b->B.amax, 0, 3 * sizeof(unsigned long long) * b->n, st);
  const int na = std::min(b->nb[0], b->nitems[0]);
  hw::k_balpha_coarse<<<na, 256, 0, st>>>(b->B, b->d_items[0], b->nitems[0]);
  hw::k_balpha_exact<<<na, 256, 0, st>>>(b->B, b->d_items[0], b->nitems[0]);
  hw::k_bfinish<<<(b->n + 127) / 128, 128, 0, st>>>(b->B, b->n, with_dt);
}

// The persistent step: the keys and the barrier counters start at zero, then one cooperative launch.
// drop_block >= 0 only in the test of the bounded barrier wait (that block leaves at once; short limits).
void enqueue_bstep(hw_batch* b, cudaStream_t st, int drop_block = -1) {
  hw::BatchDev B = b->B;
  for (int q = 0; q < 9; ++q) {
    B.S[q] = b->SA[q];
    B.out[q] = b->SB[q];
  }
  hw::StepItems P{};
  P.alpha = b->d_items[0]; P.n_alpha = b->nitems[0];
  P.x = b->d_items[1]; P.n_x = b->nitems[1];
  P.y = b->d_items[2]; P.n_y = b->nitems[2];
  P.node = b->d_items[4]; P.n_node = b->nitems[4];
  P.n_inst = b->n;
  P.sync = b->d_sync;
  P.limit_ns = drop_block < 0 ? hw::BSTEP_LIMIT_NS : 2000000ull;  // 2 ms in the test
  P.limit_polls = drop_block < 0 ? hw::BSTEP_LIMIT_POLLS : (1u << 16);
  P.drop_block = drop_block;
  cudaMemsetAsync(b->B.amax, 0, 3 * sizeof(unsigned long long) * b->n, st);
  cudaMemsetAsync(b->d_sync, 0, sizeof(hw::StepSync), st);
  hw::launch_bstep(B, P, b->cur, b->bstep_blocks, b->params.linear_weights != 0, b->params.char_decomp != 0, st);
  if (drop_block < 0) b->cur ^= 1;  // three stages: the step's result is in the other plane set
}

void enqueue_step(hw_batch* b, cudaStream_t st) {
  if (b->persistent) {
    enqueue_bstep(b, st);
    return;
  }
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
  std::vector<int4> lists[5];
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
    I.yc = 2;
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
  A(&misc, (size_t)9 * n + 8);
  if (rc == HW_OK) rc = balloc(b, (void**)&b->d_inst, sizeof(hw::BInst) * n);
  if (rc == HW_OK) rc = balloc(b, (void**)&b->d_sync, sizeof(hw::StepSync));
  if (rc != HW_OK) { hw_batch_destroy(b); return rc; }
  b->B.amax = (unsigned long long*)misc;
  b->B.alpha = misc + 3 * n;
  b->B.dt = misc + 5 * n;
  b->B.t = misc + 7 * n;
  b->B.nsteps = (unsigned long long*)(misc + 8 * n);
  b->B.status = (int*)(misc + 9 * n);
  b->B.g = params->g; b->B.eps_w = params->eps_w; b->B.eps_lim = params->eps_lim; b->B.cfl = params->cfl;
  b->B.limiter = params->limiter;
  b->B.inst = b->d_inst;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { b->cap_stream = nullptr; hw_batch_destroy(b); return bfail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  e = cudaMemsetAsync(misc, 0, ((size_t)9 * n + 8) * sizeof(double), b->stream);
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
  for (int p = 0; p < 5; ++p)
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
    if (st & hw::HW_STATUS_TIMEOUT)
      return bfail(HW_ERR_TIMEOUT, "hw_batch_run: a grid barrier of the persistent step timed out");
    return bfail(HW_ERR_DEPTH, "hw_batch_run: non-positive or non-finite depth in some instance");
  }
  return HW_OK;
}

int hw_batch_set_persistent(hw_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return bfail(HW_ERR_ARG, "hw_batch_set_persistent: bad argument");
  if (on && b->bstep_blocks == 0) {
    b->bstep_blocks = hw::bstep_grid(b->params.linear_weights != 0, b->params.char_decomp != 0);
    if (b->bstep_blocks == 0)
      return bfail(HW_ERR_CUDA, "hw_batch_set_persistent: the device cannot launch the step kernel cooperatively");
  }
  if ((bool)on != b->persistent && b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->persistent = on != 0;
  return HW_OK;
}

// One step launch with block 0 leaving before the first grid barrier: the other blocks' waits run out
// after 2 ms (or 2^16 polls) and every block leaves. The keys are the only memory written.
int hw_batch_test_barrier_timeout(hw_batch* b) {
  if (!b) return bfail(HW_ERR_ARG, "hw_batch_test_barrier_timeout: null batch");
  if (b->bstep_blocks < 2) return bfail(HW_ERR_STATE, "hw_batch_test_barrier_timeout: call hw_batch_set_persistent(b, 1) first");
  for (int i = 0; i < b->n; ++i)
    if (!b->inited[i]) return bfail(HW_ERR_STATE, "hw_batch_test_barrier_timeout: every instance must be initialised");
  if (b->dirty) {
    int rc = rebuild(b);
    if (rc != HW_OK) return rc;
    b->dirty = false;
  }
  enqueue_bstep(b, b->stream, 0);
  BCUDA(cudaGetLastError());
  BCUDA(cudaStreamSynchronize(b->stream));
  int st = 0;
  BCUDA(cudaMemcpy(&st, b->B.status, sizeof(int), cudaMemcpyDeviceToHost));
  BCUDA(cudaMemset(b->B.status, 0, sizeof(int)));
  if (st & hw::HW_STATUS_TIMEOUT) return bfail(HW_ERR_TIMEOUT, "hw_batch_test_barrier_timeout: the barrier wait ran out");
  return HW_OK;
}

int hw_batch_get_phase_times(hw_batch* b, double* ms) {
  if (!b || !ms) return bfail(HW_ERR_ARG, "hw_batch_get_phase_times: bad argument");
  if (!b->persistent) return bfail(HW_ERR_STATE, "hw_batch_get_phase_times: the batch is not in the persistent form");
  hw::StepSync s{};
  BCUDA(cudaStreamSynchronize(b->stream));
  BCUDA(cudaMemcpy(&s, b->d_sync, sizeof(s), cudaMemcpyDeviceToHost));
  for (int p = 0; p < hw::BSTEP_PHASES; ++p)
    ms[p] = (s.t[p + 1] >= s.t[p] && s.t[p] != 0) ? (double)(s.t[p + 1] - s.t[p]) * 1e-6 : -1.0;
  return HW_OK;
}

int hw_batch_get_persistent(hw_batch* b, int* on, int* blocks) {
  if (!b) return bfail(HW_ERR_ARG, "hw_batch_get_persistent: null batch");
  if (on) *on = b->persistent ? 1 : 0;
  if (blocks) *blocks = b->bstep_blocks;
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

int hw_batch_set_tiles(hw_batch* b, int i, int yc) {
  if (!b || i < 0 || i >= b->n) return bfail(HW_ERR_ARG, "hw_batch_set_tiles: bad instance");
  if (yc != 1 && yc != 2 && yc != 4) return bfail(HW_ERR_ARG, "hw_batch_set_tiles: yc must be 1, 2 or 4");
  b->inst[i].yc = yc;
  b->dirty = true;  // work lists are rebuilt by the next run
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return HW_OK;
}

int hw_batch_get_tiles(hw_batch* b, int i, int* yc) {
  if (!b || i < 0 || i >= b->n || !yc) return bfail(HW_ERR_ARG, "hw_batch_get_tiles: bad argument");
  *yc = b->inst[i].yc;
  return HW_OK;
}

// Time the x- and y-sweeps of one stage over a subset of instances with a trial y-tile shape (the
// autotuner's measurement). Writes only interface planes, which every stage recomputes.
int hw_batch_time_tiles(hw_batch* b, int nids, const int* ids, int yc, int reps, double* ms_x, double* ms_y) {
  if (!b || nids < 1 || !ids || reps < 1) return bfail(HW_ERR_ARG, "hw_batch_time_tiles: bad argument");
  if (yc != 1 && yc != 2 && yc != 4) return bfail(HW_ERR_ARG, "hw_batch_time_tiles: yc must be 1, 2 or 4");
  std::vector<hw::BInst> trial = b->inst;
  std::vector<int> sub(ids, ids + nids);
  for (int i : sub) {
    if (i < 0 || i >= b->n) return bfail(HW_ERR_ARG, "hw_batch_time_tiles: bad instance id");
    trial[i].yc = yc;
  }
  std::vector<int4> lists[5];
  build_items(trial, sub, lists);
  int4* items[5] = {};
  int counts[5] = {};
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
  for (int p = 0; p < 5; ++p)
    if (items[p]) cudaFree(items[p]);
  BCUDA(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(hw::BInst) * b->n, cudaMemcpyHostToDevice, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  if (ms_x) *ms_x = tx_ms / reps;
  if (ms_y) *ms_y = ty_ms / reps;
  return HW_OK;
}

}  // extern "C"
