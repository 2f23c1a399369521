// C ABI of the GB300 HWENO shallow-water solver (declared in include/hwswe.h).
// Owns the device buffers, sequences the kernels of one RK stage on the caller's stream, and
// captures whole steps in a CUDA graph for hw_advance.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hwswe.h"
#include "hw_internal.h"

namespace hw {
// 1D alpha's reduction with its finish in one launch (hw_kernels1d.cu): slot[0..1] are zero between
// launches (cleared by each launch's last block); same alpha and step as the separate launches.
void launch_alpha_finish1d(const Dev1D& d, unsigned long long* slot, int* status, double* alpha, double* dt_out,
                           double cfl, const double* t_now, double t_end, cudaStream_t st);
}  // namespace hw

namespace {

// NVTX range for the duration of one API call (a no-op unless a profiler is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_OK(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(HW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

__global__ void k_set_scalar(double* p, double v) { *p = v; }
// t <- t + dt, or the end time recorded next to dt by the CFL kernel (dt[1]) when dt came from it;
// counts the steps that advanced (dt > 0).
__global__ void k_add_time(double* t, const double* dt, int snapped, unsigned long long* nsteps) {
  *t = snapped ? dt[1] : *t + *dt;
  if (*dt > 0.0) ++*nsteps;
}

}  // namespace

namespace hw {
int set_last_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace hw

struct hw_solver {
  int dev = 0;
  hw_grid grid{};
  hw_params params{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture (the caller's may be the legacy one)
  bool inited = false;
  size_t n = 0;          // nodes
  int nstate = 0;        // 9 (2D) or 4 (1D)
  std::vector<void*> allocs;
  double* SA[9] = {};    // ping-pong state buffers
  double* SB[9] = {};
  double* base[9] = {};
  double* stage_in[9] = {};  // pointers of the state before the current stage
  int cur = 0;           // 0: SA holds the state, 1: SB
  double* staging[12] = {};  // device staging for host transfers
  unsigned long long* amax = nullptr;
  double* alpha = nullptr;   // [2]
  double* dt = nullptr;      // device dt
  double* t = nullptr;       // device simulated time
  int* status = nullptr;
  unsigned long long* nsteps = nullptr;  // steps that advanced (dt > 0)
  hw::Dev2D d2{};
  hw::Dev1D d1{};
  // single precision (params.precision == HW_FP32, 2D): the state, base and interface planes in float;
  // the double planes above then serve the initialisation and the exchange with the caller
  bool fp32 = false;
  float* FA[9] = {};
  float* FB[9] = {};
  float* fbase[9] = {};
  float* fsc = nullptr;  // alpha_x, alpha_y, dt rounded to float (refreshed before every stage)
  hw::Dev2DT<float> f2{};
  cudaGraphExec_t graph = nullptr;
  double graph_t_end = -1.0;
  // sub-domain of a block decomposition (hw_part_create): the grid above is the block extended by a
  // ring of 2 halo nodes, the spacing is the global grid's, and part_info places the block
  bool is_part = false;
  hw_part_info part_info{};
  // profiling: event pairs recorded around launches, resolved in hw_get_profile
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int cls, kernels; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  size_t ev_used = 0;

  double** state() { return cur == 0 ? SA : SB; }
  double** other() { return cur == 0 ? SB : SA; }
  float** fstate() { return cur == 0 ? FA : FB; }
  float** fother() { return cur == 0 ? FB : FA; }
  bool is2d() const { return grid.dim == 2; }
};

// Grid spacings and the assembly constants derived from them (a sub-domain takes the global grid's).
static void set_spacing2d(hw::Dev2D& d, double dx, double dy) {
  d.dx = dx; d.dy = dy; d.inv_dx = 1.0 / dx; d.inv_dy = 1.0 / dy;
  d.c_bx = 0.5 / dx; d.c_by = 0.5 / dy; d.c_gx = 1.0 / (24.0 * dx); d.c_gy = 1.0 / (24.0 * dy);
  d.c_mx = 1.0 / (12.0 * dx); d.c_my = 1.0 / (12.0 * dy);
}

// Bracket the launches enqueued by fn() (kernels of them) with a pair of events when profiling.
template <class Fn>
static void timed(hw_solver* s, int cls, Fn&& fn, int kernels = 1) {
  if (!s->profiling) { fn(); return; }
  while (s->ev_pool.size() < s->ev_used + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    s->ev_pool.push_back(e);
  }
  cudaEvent_t a = s->ev_pool[s->ev_used++], b = s->ev_pool[s->ev_used++];
  cudaEventRecord(a, s->stream);
  fn();
  cudaEventRecord(b, s->stream);
  s->recs.push_back({cls, kernels, a, b});
}

static int dalloc(hw_solver* s, double** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(double));
  if (e != cudaSuccess) return fail(HW_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->allocs.push_back(q);
  *p = (double*)q;
  return HW_OK;
}

static int falloc(hw_solver* s, float** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(float));
  if (e != cudaSuccess) return fail(HW_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->allocs.push_back(q);
  *p = (float*)q;
  return HW_OK;
}

static void bind_state(hw_solver* s, double** S) {
  for (int q = 0; q < s->nstate; ++q) {
    if (s->is2d()) s->d2.S[q] = S[q];
    else s->d1.S[q] = S[q];
  }
  if (s->fp32)
    for (int q = 0; q < 9; ++q) s->f2.S[q] = s->fstate()[q];
}

// Cast count planes of n values between the double and float buffers of a single-precision solver.
static void cast_planes(hw_solver* s, void* const* src, void* const* dst, int count, int to_float, size_t n) {
  hw::Ptr12 a{}, b{};
  for (int q = 0; q < count; ++q) { a.p[q] = src[q]; b.p[q] = dst[q]; }
  hw::launch_cast_planes(count, n, a, b, to_float, s->stream);
}

extern "C" {

const char* hw_last_error(void) { return g_err.c_str(); }
const char* hw_version(void) { return "hwswe-gb300 0.2 (sm_103a, FP64; FP32 variant)"; }

int hw_create(const hw_grid* grid, const hw_params* params, void* cuda_stream, hw_solver** out) {
  if (!grid || !params || !out) return fail(HW_ERR_ARG, "hw_create: null argument");
  *out = nullptr;
  if (grid->dim != 1 && grid->dim != 2) return fail(HW_ERR_ARG, "hw_create: dim must be 1 or 2");
  if (grid->nx < 2 || (grid->dim == 2 && grid->ny < 2) || (grid->dim == 1 && grid->ny != 1))
    return fail(HW_ERR_ARG, "hw_create: need nx >= 2 (and ny >= 2 in 2D, ny == 1 in 1D)");
  if (grid->bc_x < 0 || grid->bc_x > 2 || grid->bc_y < 0 || grid->bc_y > 2)
    return fail(HW_ERR_ARG, "hw_create: bad boundary condition");
  if (!(grid->x1 > grid->x0) || (grid->dim == 2 && !(grid->y1 > grid->y0)))
    return fail(HW_ERR_ARG, "hw_create: empty domain");
  if ((size_t)grid->nx * (size_t)grid->ny > ((size_t)1 << 31))
    return fail(HW_ERR_ARG, "hw_create: grid too large (more than 2^31 nodes)");
  // the sweeps index their flattened extended lines, ny (nx + 4) and (nx / 2 + 1) (ny + 4) nodes, in 32 bits
  if (grid->dim == 2 && ((size_t)grid->ny * ((size_t)grid->nx + 4) >= ((size_t)1 << 32) ||
                         ((size_t)grid->nx / 2 + 1) * ((size_t)grid->ny + 4) >= ((size_t)1 << 32)))
    return fail(HW_ERR_ARG, "hw_create: grid too elongated for the sweeps' 32-bit line indices");
  if (!(params->g > 0) || !(params->eps_w > 0) || !(params->eps_lim > 0) || !(params->cfl > 0))
    return fail(HW_ERR_ARG, "hw_create: g, cfl, eps_w and eps_lim must be positive");
  if (params->precision != HW_FP64 && params->precision != HW_FP32)
    return fail(HW_ERR_ARG, "hw_create: precision must be HW_FP64 or HW_FP32");
  if (params->precision == HW_FP32 && grid->dim != 2)
    return fail(HW_ERR_ARG, "hw_create: HW_FP32 is available for 2D grids only");

  hw_solver* s = new hw_solver();
  s->grid = *grid;
  s->params = *params;
  s->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&s->dev);
  const int nx = grid->nx, ny = grid->dim == 2 ? grid->ny : 1;
  s->n = (size_t)nx * ny;
  s->nstate = grid->dim == 2 ? 9 : 4;
  int rc = HW_OK;
  auto A = [&](double** p, size_t cnt) { if (rc == HW_OK) rc = dalloc(s, p, cnt); };
  for (int q = 0; q < s->nstate; ++q) { A(&s->SA[q], s->n); A(&s->SB[q], s->n); A(&s->base[q], s->n); }
  for (int q = 0; q < 12; ++q) A(&s->staging[q], s->n);
  double* misc = nullptr;
  A(&misc, 16);
  // the alpha reduction's keys and scratch (launch_alpha2d: kAlpha2dScratch 8-byte slots)
  A(reinterpret_cast<double**>(&s->amax), hw::kAlpha2dScratch);
  if (rc != HW_OK) { hw_destroy(s); return rc; }
  s->alpha = misc + 3;
  s->dt = misc + 5;  // dt[0] = step, dt[1] = time after the step (written by the CFL kernel)
  s->t = misc + 7;
  s->status = (int*)(misc + 8);
  s->nsteps = (unsigned long long*)(misc + 9);

  const double dx = (grid->x1 - grid->x0) / nx;
  if (grid->dim == 2) {
    hw::Dev2D& d = s->d2;
    const double dy = (grid->y1 - grid->y0) / ny;
    d.nx = nx; d.ny = ny; d.bc_x = grid->bc_x; d.bc_y = grid->bc_y;
    set_spacing2d(d, dx, dy);
    d.g = params->g; d.eps_w = params->eps_w; d.eps_lim = params->eps_lim;
    for (int q = 0; q < 3; ++q) A(&d.stat[q], s->n);
    for (int q = 0; q < 2; ++q) A(&d.bxy[q], s->n);
    for (int q = 0; q < 12; ++q) { A(&d.X[q], (size_t)(nx + 1) * ny); A(&d.Y[q], (size_t)nx * (ny + 1)); }
    for (int q = 0; q < 6; ++q) { A(&d.qbx[q], (size_t)(nx + 1) * ny); A(&d.qby[q], (size_t)nx * (ny + 1)); }
    for (int q = 0; q < 2; ++q) { A(&d.sv[q], s->n); A(&d.sq[q], s->n); }
    if (rc == HW_OK && hw::set_kernel_attributes2d() != 0) rc = fail(HW_ERR_CUDA, "hw_create: kernel attributes");
    if (params->precision == HW_FP32) {
      s->fp32 = true;
      hw::Dev2DT<float>& f = s->f2;
      auto F = [&](float** p, size_t cnt) { if (rc == HW_OK) rc = falloc(s, p, cnt); };
      for (int q = 0; q < 9; ++q) { F(&s->FA[q], s->n); F(&s->FB[q], s->n); F(&s->fbase[q], s->n); }
      f.nx = d.nx; f.ny = d.ny; f.bc_x = d.bc_x; f.bc_y = d.bc_y;
      f.dx = (float)d.dx; f.dy = (float)d.dy; f.inv_dx = (float)d.inv_dx; f.inv_dy = (float)d.inv_dy;
      f.g = (float)d.g; f.eps_w = (float)d.eps_w; f.eps_lim = (float)d.eps_lim;
      f.c_bx = (float)d.c_bx; f.c_by = (float)d.c_by; f.c_gx = (float)d.c_gx; f.c_gy = (float)d.c_gy;
      f.c_mx = (float)d.c_mx; f.c_my = (float)d.c_my;
      F(&s->fsc, 4);
      for (int q = 0; q < 3; ++q) F(&f.stat[q], s->n);
      for (int q = 0; q < 2; ++q) F(&f.bxy[q], s->n);
      for (int q = 0; q < 12; ++q) { F(&f.X[q], (size_t)(nx + 1) * ny); F(&f.Y[q], (size_t)nx * (ny + 1)); }
      for (int q = 0; q < 6; ++q) { F(&f.qbx[q], (size_t)(nx + 1) * ny); F(&f.qby[q], (size_t)nx * (ny + 1)); }
      for (int q = 0; q < 2; ++q) { F(&f.sv[q], s->n); F(&f.sq[q], s->n); }
    }
  } else {
    hw::Dev1D& d = s->d1;
    d.nx = nx; d.bc = grid->bc_x; d.dx = dx; d.inv_dx = 1.0 / dx;
    d.g = params->g; d.eps_w = params->eps_w; d.eps_lim = params->eps_lim;
    d.c_b = 0.5 / dx; d.c_g = 1.0 / (24.0 * dx);
    for (int q = 0; q < 2; ++q) A(&d.stat[q], s->n);
    A(&d.bx, s->n);
    for (int q = 0; q < 6; ++q) A(&d.X[q], (size_t)nx + 1);
    for (int q = 6; q < 9; ++q) d.X[q] = nullptr;
    for (int q = 0; q < 6; ++q) A(&d.qb[q], (size_t)nx + 1);
    A(&d.sv, s->n);
  }
  if (rc != HW_OK) { hw_destroy(s); return rc; }
  cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { s->cap_stream = nullptr; hw_destroy(s); return fail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  e = cudaMemsetAsync(misc, 0, 16 * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->amax + 2, 0, 2 * sizeof(unsigned long long), s->stream);  // 1D alpha slots
  if (e != cudaSuccess) { hw_destroy(s); return fail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  bind_state(s, s->SA);
  *out = s;
  return HW_OK;
}

int hw_destroy(hw_solver* s) {
  if (!s) return HW_OK;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->stream) cudaStreamSynchronize(s->stream);
  else cudaDeviceSynchronize();
  hw::adjoint_release(s);
  for (void* p : s->allocs) cudaFree(p);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  delete s;
  return HW_OK;
}

// Copy caller planes into device memory (host -> staging) or pass device pointers through.
static int stage_inputs(hw_solver* s, const double* const* in, int count, int ptr_kind, const double** dev) {
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return fail(HW_ERR_ARG, "bad ptr_kind");
  for (int q = 0; q < count; ++q) {
    if (!in[q]) return fail(HW_ERR_ARG, "null input plane");
    if (ptr_kind == HW_DEVICE) {
      dev[q] = in[q];
    } else {
      CUDA_OK(cudaMemcpyAsync(s->staging[q], in[q], s->n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      dev[q] = s->staging[q];
    }
  }
  return HW_OK;
}

static int read_status(hw_solver* s) {
  int st = 0;
  CUDA_OK(cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CUDA_OK(cudaStreamSynchronize(s->stream));
  if (st) {
    CUDA_OK(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream));
    if (st & hw::HW_STATUS_TIMEOUT) return fail(HW_ERR_TIMEOUT, "device wait timed out");
    if (st & hw::HW_STATUS_DEPTH) return fail(HW_ERR_DEPTH, "non-positive depth in the state");
    return fail(HW_ERR_NONFINITE, "non-finite value");
  }
  return HW_OK;
}

int hw_init(hw_solver* s, const double* h, const double* hu, const double* hv, const double* b,
            const double* const* deriv, int ptr_kind) {
  Range nvtx_range("hw_init");
  if (!s || !h || !hu || !b || !deriv) return fail(HW_ERR_ARG, "hw_init: null argument");
  if (s->is2d()) {
    if (!hv) return fail(HW_ERR_ARG, "hw_init: hv required in 2D");
    const double* in[12] = {h, hu, hv, b, deriv[0], deriv[1], deriv[2], deriv[3], deriv[4], deriv[5],
                            deriv[6], deriv[7]};
    hw::PhysIn pin;
    int rc = stage_inputs(s, in, 12, ptr_kind, pin.p);
    if (rc) return rc;
    s->cur = 0;
    bind_state(s, s->SA);
    hw::launch_init2d(s->d2, pin, s->status, s->stream);
    if (s->fp32) {
      // the state and the b-only terms of the double initialisation, rounded to float
      const hw::Dev2D& d = s->d2;
      hw::Dev2DT<float>& f = s->f2;
      void* src[12];
      void* dst[12];
      for (int q = 0; q < 9; ++q) { src[q] = s->SA[q]; dst[q] = s->FA[q]; }
      for (int q = 0; q < 3; ++q) { src[9 + q] = d.stat[q]; dst[9 + q] = f.stat[q]; }
      cast_planes(s, src, dst, 12, 1, s->n);
      for (int q = 0; q < 2; ++q) { src[q] = d.bxy[q]; dst[q] = f.bxy[q]; src[2 + q] = d.sv[q]; dst[2 + q] = f.sv[q];
                                    src[4 + q] = d.sq[q]; dst[4 + q] = f.sq[q]; }
      cast_planes(s, src, dst, 6, 1, s->n);
      for (int q = 0; q < 6; ++q) { src[q] = d.qbx[q]; dst[q] = f.qbx[q]; }
      cast_planes(s, src, dst, 6, 1, (size_t)(d.nx + 1) * d.ny);
      for (int q = 0; q < 6; ++q) { src[q] = d.qby[q]; dst[q] = f.qby[q]; }
      cast_planes(s, src, dst, 6, 1, (size_t)d.nx * (d.ny + 1));
      bind_state(s, s->SA);
    }
  } else {
    const double* in[6] = {h, hu, b, deriv[0], deriv[1], deriv[2]};
    hw::PhysIn1D pin;
    int rc = stage_inputs(s, in, 6, ptr_kind, pin.p);
    if (rc) return rc;
    s->cur = 0;
    bind_state(s, s->SA);
    hw::launch_init1d(s->d1, pin, s->status, s->stream);
  }
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaMemsetAsync(s->t, 0, sizeof(double), s->stream));
  s->inited = true;
  return read_status(s);
}

// alpha of the current state into s->alpha (and dt if dt_out).
static void enqueue_alpha(hw_solver* s, bool with_dt, double t_end) {
  bind_state(s, s->state());
  timed(s, HW_PROF_ALPHA, [&] {
    if (s->fp32) {
      hw::launch_alpha2d(s->f2, s->amax, s->status, s->stream);
      hw::launch_finish_alpha2d(s->d2, s->amax, s->alpha, with_dt ? s->dt : nullptr, s->params.cfl,
                                with_dt ? s->t : nullptr, t_end, s->stream);
    } else if (s->is2d()) {
      hw::launch_alpha2d(s->d2, s->amax, s->status, s->stream);
      hw::launch_finish_alpha2d(s->d2, s->amax, s->alpha, with_dt ? s->dt : nullptr, s->params.cfl,
                                with_dt ? s->t : nullptr, t_end, s->stream);
    } else {
      hw::launch_alpha_finish1d(s->d1, s->amax + 2, s->status, s->alpha, with_dt ? s->dt : nullptr, s->params.cfl,
                                with_dt ? s->t : nullptr, t_end, s->stream);
    }
  }, s->is2d() ? (s->fp32 ? 2 : 3) : 1);  // reduction (two passes in 2D double) and finish; one launch in 1D
}

// One stage: sweeps on the current state (alpha already in s->alpha), node kernel into the other
// buffer, then swap.
static void enqueue_stage(hw_solver* s, int k) {
  static const char* kNames[4] = {"", "stage 1", "stage 2", "stage 3"};
  Range nvtx_range(kNames[k]);
  double** in = s->state();
  double** out = s->other();
  bind_state(s, in);
  const bool lin = s->params.linear_weights != 0, chr = s->params.char_decomp != 0;
  if (s->fp32) {
    float** fout = s->fother();
    timed(s, HW_PROF_OTHER, [&] { hw::launch_scalars_to_float(s->alpha, s->dt, s->fsc, s->stream); });
    timed(s, HW_PROF_SWEEP_X, [&] { hw::launch_sweep_x2d(s->f2, s->fsc, lin, chr, s->stream); });
    timed(s, HW_PROF_SWEEP_Y, [&] { hw::launch_sweep_y2d(s->f2, s->fsc, lin, chr, s->stream); });
    hw::StageArgsT<float> sa{};
    sa.k = k; sa.limiter = s->params.limiter; sa.dt = s->fsc + 2;
    for (int q = 0; q < 9; ++q) { sa.out[q] = fout[q]; sa.base[q] = s->fbase[q]; }
    timed(s, HW_PROF_NODE, [&] { hw::launch_node2d(s->f2, sa, hw::MODE_STAGE, lin, chr, s->stream); });
  } else if (s->is2d()) {
    timed(s, HW_PROF_SWEEP_X, [&] { hw::launch_sweep_x2d(s->d2, s->alpha, lin, chr, s->stream); });
    timed(s, HW_PROF_SWEEP_Y, [&] { hw::launch_sweep_y2d(s->d2, s->alpha, lin, chr, s->stream); });
    hw::StageArgs sa{};
    sa.k = k; sa.limiter = s->params.limiter; sa.dt = s->dt;
    for (int q = 0; q < 9; ++q) { sa.out[q] = out[q]; sa.base[q] = s->base[q]; }
    timed(s, HW_PROF_NODE, [&] { hw::launch_node2d(s->d2, sa, hw::MODE_STAGE, lin, chr, s->stream); });
  } else {
    timed(s, HW_PROF_SWEEP_X, [&] { hw::launch_sweep1d(s->d1, s->alpha, lin, chr, s->stream); });
    hw::StageArgs1D sa{};
    sa.k = k; sa.limiter = s->params.limiter; sa.dt = s->dt;
    for (int q = 0; q < 4; ++q) { sa.out[q] = out[q]; sa.base[q] = s->base[q]; }
    timed(s, HW_PROF_NODE, [&] { hw::launch_node1d(s->d1, sa, hw::MODE_STAGE, lin, chr, s->stream); });
  }
  s->cur ^= 1;
}

int hw_rk3_stage(hw_solver* s, int k, double dt) {
  Range nvtx_range("hw_rk3_stage");
  if (!s) return fail(HW_ERR_ARG, "hw_rk3_stage: null solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_rk3_stage: call hw_init first");
  if (k < 1 || k > 3) return fail(HW_ERR_ARG, "hw_rk3_stage: k must be 1, 2 or 3");
  if (!(dt >= 0) || !(dt < 1e300)) return fail(HW_ERR_ARG, "hw_rk3_stage: dt must be finite and >= 0");
  k_set_scalar<<<1, 1, 0, s->stream>>>(s->dt, dt);
  enqueue_alpha(s, false, -1.0);
  enqueue_stage(s, k);
  CUDA_OK(cudaGetLastError());
  return HW_OK;
}

int hw_rk3_step(hw_solver* s, double dt) {
  Range nvtx_range("hw_rk3_step");
  if (!s) return fail(HW_ERR_ARG, "hw_rk3_step: null solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_rk3_step: call hw_init first");
  if (!(dt >= 0) || !(dt < 1e300)) return fail(HW_ERR_ARG, "hw_rk3_step: dt must be finite and >= 0");
  timed(s, HW_PROF_OTHER, [&] { k_set_scalar<<<1, 1, 0, s->stream>>>(s->dt, dt); });
  for (int k = 1; k <= 3; ++k) {
    enqueue_alpha(s, false, -1.0);
    enqueue_stage(s, k);
  }
  timed(s, HW_PROF_OTHER, [&] { k_add_time<<<1, 1, 0, s->stream>>>(s->t, s->dt, 0, s->nsteps); });
  CUDA_OK(cudaGetLastError());
  return HW_OK;
}

// One step with dt computed on the device from U^n (clipped to t_end when t_end > 0).
static void enqueue_cfl_step(hw_solver* s, double t_end) {
  enqueue_alpha(s, true, t_end);
  enqueue_stage(s, 1);
  for (int k = 2; k <= 3; ++k) {
    enqueue_alpha(s, false, -1.0);
    enqueue_stage(s, k);
  }
  timed(s, HW_PROF_OTHER, [&] { k_add_time<<<1, 1, 0, s->stream>>>(s->t, s->dt, 1, s->nsteps); });
}

int hw_advance(hw_solver* s, int nsteps, double t_end, int use_graph, double* t_out, int* steps_out) {
  Range nvtx_range("hw_advance");
  if (!s) return fail(HW_ERR_ARG, "hw_advance: null solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_advance: call hw_init first");
  if (nsteps < 0) return fail(HW_ERR_ARG, "hw_advance: nsteps < 0");
  double t0 = 0.0;
  unsigned long long n0 = 0, n1 = 0;
  CUDA_OK(cudaMemcpyAsync(&t0, s->t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CUDA_OK(cudaMemcpyAsync(&n0, s->nsteps, sizeof(n0), cudaMemcpyDeviceToHost, s->stream));
  CUDA_OK(cudaStreamSynchronize(s->stream));
  int done = 0;
  const bool has_end = t_end > 0.0;
  // A captured graph holds two steps (an even number of stages returns to the same buffer).
  if (s->profiling) use_graph = 0;
  if (use_graph && (!s->graph || s->graph_t_end != t_end || s->cur != 0)) {
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    if (s->cur == 0) {
      // capture on the private stream (capturing the legacy default stream is not permitted), after
      // the caller's stream has drained; the graph is launched on the caller's stream
      CUDA_OK(cudaStreamSynchronize(s->stream));
      cudaGraph_t g = nullptr;
      cudaStream_t user = s->stream;
      s->stream = s->cap_stream;
      cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { s->stream = user; return fail(HW_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e)); }
      enqueue_cfl_step(s, t_end);
      enqueue_cfl_step(s, t_end);
      e = cudaStreamEndCapture(s->stream, &g);
      s->stream = user;
      s->cur = 0;  // capture enqueued six stage swaps (even): the state buffer is unchanged until launch
      if (e != cudaSuccess) return fail(HW_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&s->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { s->graph = nullptr; return fail(HW_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
      s->graph_t_end = t_end;
    }
  }
  // With an end time the host reads the time back between chunks of steps: two steps at first, then half
  // the steps the last step size leaves to t_end (a step past t_end has size 0 and changes nothing), so a
  // run of n steps waits O(log n) times instead of n/2.
  int chunk = has_end ? 2 : 1 << 30;
  double t = t0;
  while (done < nsteps) {
    if (has_end && t >= t_end) break;
    int todo = std::min(nsteps - done, chunk);
    while (todo > 0) {
      if (use_graph && s->graph && s->cur == 0 && todo >= 2) {
        CUDA_OK(cudaGraphLaunch(s->graph, s->stream));
        todo -= 2;
        done += 2;
      } else {
        enqueue_cfl_step(s, t_end);
        todo -= 1;
        done += 1;
      }
    }
    CUDA_OK(cudaGetLastError());
    if (has_end) {
      double dt_t[3];  // dt[0] (the last step), dt[1], t: adjacent device scalars (s->t == s->dt + 2)
      CUDA_OK(cudaMemcpyAsync(dt_t, s->dt, sizeof(dt_t), cudaMemcpyDeviceToHost, s->stream));
      CUDA_OK(cudaStreamSynchronize(s->stream));
      t = dt_t[2];
      const double left = dt_t[0] > 0.0 ? (t_end - t) / dt_t[0] : 0.0;
      chunk = 2 * std::max(1, (int)std::min(0.25 * left, 1e6));
    }
  }
  CUDA_OK(cudaMemcpyAsync(&t, s->t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CUDA_OK(cudaMemcpyAsync(&n1, s->nsteps, sizeof(n1), cudaMemcpyDeviceToHost, s->stream));
  int rc = read_status(s);
  if (t_out) *t_out = t - t0;
  if (steps_out) *steps_out = (int)(n1 - n0);  // steps of size 0 after t_end (inside a graph) do not count
  return rc;
}

int hw_alpha(hw_solver* s, double* alpha) {
  if (!s || !alpha) return fail(HW_ERR_ARG, "hw_alpha: null argument");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_alpha: call hw_init first");
  enqueue_alpha(s, false, -1.0);
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaMemcpyAsync(alpha, s->alpha, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return read_status(s);
}

int hw_cfl_dt(hw_solver* s, double* dt_out) {
  Range nvtx_range("hw_cfl_dt");
  if (!s || !dt_out) return fail(HW_ERR_ARG, "hw_cfl_dt: null argument");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_cfl_dt: call hw_init first");
  enqueue_alpha(s, true, -1.0);
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaMemcpyAsync(dt_out, s->dt, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return read_status(s);
}

int hw_rhs(hw_solver* s, double* const* out, int ptr_kind) {
  Range nvtx_range("hw_rhs");
  if (!s || !out) return fail(HW_ERR_ARG, "hw_rhs: null argument");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_rhs: call hw_init first");
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return fail(HW_ERR_ARG, "hw_rhs: bad ptr_kind");
  for (int q = 0; q < s->nstate; ++q)
    if (!out[q]) return fail(HW_ERR_ARG, "hw_rhs: null output plane");
  enqueue_alpha(s, false, -1.0);
  double* dst[9];
  for (int q = 0; q < s->nstate; ++q) dst[q] = ptr_kind == HW_DEVICE ? out[q] : s->staging[q];
  const bool lin = s->params.linear_weights != 0, chr = s->params.char_decomp != 0;
  bind_state(s, s->state());
  if (s->fp32) {
    // float right-hand side into the spare state buffer, then widened into the output planes
    float** scratch = s->fother();
    hw::launch_scalars_to_float(s->alpha, s->dt, s->fsc, s->stream);
    hw::launch_sweep_x2d(s->f2, s->fsc, lin, chr, s->stream);
    hw::launch_sweep_y2d(s->f2, s->fsc, lin, chr, s->stream);
    hw::StageArgsT<float> sa{};
    for (int q = 0; q < 9; ++q) sa.rhs_out[q] = scratch[q];
    hw::launch_node2d(s->f2, sa, hw::MODE_RHS, lin, chr, s->stream);
    void* src[9];
    void* dd[9];
    for (int q = 0; q < 9; ++q) { src[q] = scratch[q]; dd[q] = dst[q]; }
    cast_planes(s, src, dd, 9, 0, s->n);
  } else if (s->is2d()) {
    hw::launch_sweep_x2d(s->d2, s->alpha, lin, chr, s->stream);
    hw::launch_sweep_y2d(s->d2, s->alpha, lin, chr, s->stream);
    hw::StageArgs sa{};
    for (int q = 0; q < 9; ++q) sa.rhs_out[q] = dst[q];
    hw::launch_node2d(s->d2, sa, hw::MODE_RHS, lin, chr, s->stream);
  } else {
    hw::launch_sweep1d(s->d1, s->alpha, lin, chr, s->stream);
    hw::StageArgs1D sa{};
    for (int q = 0; q < 4; ++q) sa.rhs_out[q] = dst[q];
    hw::launch_node1d(s->d1, sa, hw::MODE_RHS, lin, chr, s->stream);
  }
  CUDA_OK(cudaGetLastError());
  if (ptr_kind == HW_HOST)
    for (int q = 0; q < s->nstate; ++q)
      CUDA_OK(cudaMemcpyAsync(out[q], dst[q], s->n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return ptr_kind == HW_HOST ? read_status(s) : HW_OK;
}

// src_state: double planes, or (single precision) float planes fsrc widened first into the double
// buffer SB, which a single-precision solver uses only as scratch.
static int export_planes(hw_solver* s, double** src_state, double* const* out, int layout, int ptr_kind,
                         float** fsrc = nullptr) {
  if (!out) return fail(HW_ERR_ARG, "null output");
  if (layout != HW_LAYOUT_PHYSICAL && layout != HW_LAYOUT_EQUILIBRIUM) return fail(HW_ERR_ARG, "bad layout");
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return fail(HW_ERR_ARG, "bad ptr_kind");
  hw::Ptr9 src{}, dst{};
  for (int q = 0; q < s->nstate; ++q) {
    if (!out[q]) return fail(HW_ERR_ARG, "null output plane");
    dst.p[q] = ptr_kind == HW_DEVICE ? out[q] : s->staging[q];
  }
  if (fsrc) {
    void* a[9];
    void* b[9];
    for (int q = 0; q < 9; ++q) { a[q] = fsrc[q]; b[q] = s->SB[q]; }
    cast_planes(s, a, b, 9, 0, s->n);
    src_state = s->SB;
  }
  bind_state(s, src_state);
  if (s->is2d()) hw::launch_convert2d(s->d2, src, dst, layout, 0, s->stream);
  else hw::launch_convert1d(s->d1, src, dst, layout, 0, s->stream);
  bind_state(s, s->state());
  CUDA_OK(cudaGetLastError());
  if (ptr_kind == HW_HOST) {
    for (int q = 0; q < s->nstate; ++q)
      CUDA_OK(cudaMemcpyAsync(out[q], dst.p[q], s->n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CUDA_OK(cudaStreamSynchronize(s->stream));
  }
  return HW_OK;
}

int hw_get_state(hw_solver* s, double* const* out, int layout, int ptr_kind) {
  Range nvtx_range("hw_get_state");
  if (!s) return fail(HW_ERR_ARG, "hw_get_state: null solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_get_state: call hw_init first");
  if (s->fp32) return export_planes(s, nullptr, out, layout, ptr_kind, s->fstate());
  return export_planes(s, s->state(), out, layout, ptr_kind);
}

int hw_get_base(hw_solver* s, double* const* out, int ptr_kind) {
  if (!s) return fail(HW_ERR_ARG, "hw_get_base: null solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_get_base: call hw_init first");
  if (s->fp32) return export_planes(s, nullptr, out, HW_LAYOUT_EQUILIBRIUM, ptr_kind, s->fbase);
  return export_planes(s, s->base, out, HW_LAYOUT_EQUILIBRIUM, ptr_kind);
}

int hw_set_state(hw_solver* s, const double* const* in, int layout, int ptr_kind) {
  Range nvtx_range("hw_set_state");
  if (!s || !in) return fail(HW_ERR_ARG, "hw_set_state: null argument");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_set_state: call hw_init first (it loads b)");
  if (layout != HW_LAYOUT_PHYSICAL && layout != HW_LAYOUT_EQUILIBRIUM) return fail(HW_ERR_ARG, "bad layout");
  const double* dev[12];
  int rc = stage_inputs(s, in, s->nstate, ptr_kind, dev);
  if (rc) return rc;
  hw::Ptr9 src{}, dst{};
  for (int q = 0; q < s->nstate; ++q) src.p[q] = (double*)dev[q];
  bind_state(s, s->fp32 ? s->SB : s->state());
  if (s->is2d()) hw::launch_convert2d(s->d2, src, dst, layout, 1, s->stream);
  else hw::launch_convert1d(s->d1, src, dst, layout, 1, s->stream);
  if (s->fp32) {
    // converted in double into the scratch buffer, then rounded into the float state
    void* a[9];
    void* b[9];
    for (int q = 0; q < 9; ++q) { a[q] = s->SB[q]; b[q] = s->fstate()[q]; }
    cast_planes(s, a, b, 9, 1, s->n);
    bind_state(s, s->state());
  }
  CUDA_OK(cudaGetLastError());
  if (ptr_kind == HW_HOST) CUDA_OK(cudaStreamSynchronize(s->stream));
  return HW_OK;
}

}  // extern "C"

namespace hw {
int part_planes(hw_solver* s, int set, double** planes, int* nplanes) {
  double** S = s->state();
  for (int q = 0; q < 9; ++q) planes[q] = S[q];
  if (set == 1) {
    for (int q = 0; q < 3; ++q) planes[9 + q] = s->d2.stat[q];
    for (int q = 0; q < 2; ++q) planes[12 + q] = s->d2.bxy[q];
  }
  *nplanes = set == 1 ? 14 : 9;
  return HW_OK;
}
const Dev2D* part_dev(hw_solver* s) { return &s->d2; }
cudaStream_t solver_swap_stream(hw_solver* s, cudaStream_t st) {
  cudaStream_t old = s->stream;
  s->stream = st;
  return old;
}
int solver_cur(hw_solver* s) { return s->cur; }
cudaStream_t solver_stream(hw_solver* s) { return s->stream; }
const hw_part_info* part_info(hw_solver* s) { return s && s->is_part ? &s->part_info : nullptr; }

int solver_view(hw_solver* s, SolverView* v) {
  if (!s) return fail(HW_ERR_ARG, "null solver");
  if (!s->inited) return fail(HW_ERR_STATE, "call hw_init first");
  if (s->fp32) return fail(HW_ERR_ARG, "the adjoint needs an HW_FP64 solver");
  v->stream = s->stream;
  v->d2 = s->is2d() ? &s->d2 : nullptr;
  v->state = s->state();
  for (int q = 0; q < 9; ++q) v->base[q] = q < s->nstate ? s->base[q] : nullptr;
  v->alpha = s->alpha;
  v->dt = s->dt;
  v->params = &s->params;
  v->n = s->n;
  bind_state(s, s->state());
  return HW_OK;
}

int solver_set_state_planes(hw_solver* s, double* const* src) {
  double** S = s->state();
  for (int q = 0; q < s->nstate; ++q)
    CUDA_OK(cudaMemcpyAsync(S[q], src[q], s->n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  return HW_OK;
}
}  // namespace hw

extern "C" {

// ---- one block of a block decomposition (declared in hwswe.h; the exchange is in hw_dd.cu) ----
int hw_part_create(const hw_grid* grid, const hw_params* params, int px, int py, int part, void* cuda_stream,
                   hw_solver** out) {
  if (!grid || !params || !out) return fail(HW_ERR_ARG, "hw_part_create: null argument");
  *out = nullptr;
  if (params->precision != HW_FP64) return fail(HW_ERR_ARG, "hw_part_create: HW_FP64 only");
  hw_part_info info{};
  int rc = hw_dd_partition(grid, px, py, part, &info);
  if (rc != HW_OK) return rc;
  const double dx = (grid->x1 - grid->x0) / grid->nx, dy = (grid->y1 - grid->y0) / grid->ny;
  hw_grid ext = *grid;
  ext.nx = info.nx + 4;
  ext.ny = info.ny + 4;
  ext.x0 = grid->x0 + (info.i0 - 2) * dx;
  ext.x1 = ext.x0 + ext.nx * dx;
  ext.y0 = grid->y0 + (info.j0 - 2) * dy;
  ext.y1 = ext.y0 + ext.ny * dy;
  // the extended grid's own boundary only feeds ring nodes, which every exchange overwrites
  ext.bc_x = ext.bc_y = HW_BC_OUTFLOW;
  hw_solver* s = nullptr;
  rc = hw_create(&ext, params, cuda_stream, &s);
  if (rc != HW_OK) return rc;
  set_spacing2d(s->d2, dx, dy);  // the global spacings exactly (ext.x1 - ext.x0 may round)
  s->is_part = true;
  s->part_info = info;
  *out = s;
  return HW_OK;
}

int hw_part_init(hw_solver* s, const double* const* planes12, long long ld, int ptr_kind) {
  Range nvtx_range("hw_part_init");
  if (!s || !s->is_part || !planes12) return fail(HW_ERR_ARG, "hw_part_init: null argument or not a block solver");
  const hw_part_info& pi = s->part_info;
  if (ld < pi.nx) return fail(HW_ERR_ARG, "hw_part_init: ld below the block's nx");
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return fail(HW_ERR_ARG, "hw_part_init: bad ptr_kind");
  const int nxe = s->grid.nx;
  const cudaMemcpyKind kind = ptr_kind == HW_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  hw::PhysIn pin;
  for (int q = 0; q < 12; ++q) {
    if (!planes12[q]) return fail(HW_ERR_ARG, "hw_part_init: null plane");
    CUDA_OK(cudaMemcpy2DAsync(s->staging[q] + 2 * (size_t)nxe + 2, nxe * sizeof(double), planes12[q],
                              (size_t)ld * sizeof(double), pi.nx * sizeof(double), pi.ny, kind, s->stream));
    pin.p[q] = s->staging[q];
  }
  hw::launch_fill_ring(s->staging, nxe, s->grid.ny, s->stream);
  s->cur = 0;
  bind_state(s, s->SA);
  hw::launch_init2d(s->d2, pin, s->status, s->stream);
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaMemsetAsync(s->t, 0, sizeof(double), s->stream));
  s->inited = true;
  return read_status(s);
}

int hw_part_finish_init(hw_solver* s) {
  if (!s || !s->is_part || !s->inited) return fail(HW_ERR_ARG, "hw_part_finish_init: not an initialised block solver");
  hw::launch_static2d(s->d2, s->stream);
  CUDA_OK(cudaGetLastError());
  return read_status(s);
}

int hw_part_alpha_keys(hw_solver* s, unsigned long long* keys) {
  if (!s || !s->is_part || !keys) return fail(HW_ERR_ARG, "hw_part_alpha_keys: null argument or not a block solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_part_alpha_keys: call hw_part_init first");
  bind_state(s, s->state());
  hw::launch_alpha2d(s->d2, s->amax, s->status, s->stream);
  CUDA_OK(cudaMemcpyAsync(keys, s->amax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s->stream));
  return HW_OK;
}

int hw_part_stage(hw_solver* s, int k, const unsigned long long* keys, double t_end) {
  if (!s || !s->is_part || !keys) return fail(HW_ERR_ARG, "hw_part_stage: null argument or not a block solver");
  if (!s->inited) return fail(HW_ERR_STATE, "hw_part_stage: call hw_part_init first");
  if (k < 1 || k > 3) return fail(HW_ERR_ARG, "hw_part_stage: k must be 1, 2 or 3");
  bind_state(s, s->state());
  hw::launch_finish_alpha2d(s->d2, keys, s->alpha, k == 1 ? s->dt : nullptr, s->params.cfl, k == 1 ? s->t : nullptr,
                            t_end, s->stream);
  enqueue_stage(s, k);
  if (k == 3) k_add_time<<<1, 1, 0, s->stream>>>(s->t, s->dt, 1, s->nsteps);
  CUDA_OK(cudaGetLastError());
  return HW_OK;
}

int hw_set_profiling(hw_solver* s, int on) {
  if (!s) return fail(HW_ERR_ARG, "hw_set_profiling: null solver");
  s->profiling = on != 0;
  return HW_OK;
}

int hw_get_profile(hw_solver* s, double* ms, int* launches) {
  if (!s || !ms || !launches) return fail(HW_ERR_ARG, "hw_get_profile: null argument");
  CUDA_OK(cudaStreamSynchronize(s->stream));
  for (int c = 0; c < HW_PROF_N; ++c) { ms[c] = 0.0; launches[c] = 0; }
  for (auto& r : s->recs) {
    float t = 0.f;
    CUDA_OK(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.cls] += t;
    launches[r.cls] += r.kernels;
  }
  s->recs.clear();
  s->ev_used = 0;
  return HW_OK;
}

int hw_get_time(hw_solver* s, double* t, long long* steps) {
  if (!s || !t || !steps) return fail(HW_ERR_ARG, "hw_get_time: null argument");
  unsigned long long n = 0;
  CUDA_OK(cudaMemcpyAsync(t, s->t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CUDA_OK(cudaMemcpyAsync(&n, s->nsteps, sizeof(n), cudaMemcpyDeviceToHost, s->stream));
  CUDA_OK(cudaStreamSynchronize(s->stream));
  *steps = (long long)n;
  return HW_OK;
}

int hw_set_time(hw_solver* s, double t, long long steps) {
  if (!s) return fail(HW_ERR_ARG, "hw_set_time: null solver");
  if (!(t >= 0.0) || !(t < 1e300) || steps < 0) return fail(HW_ERR_ARG, "hw_set_time: bad time or step count");
  const unsigned long long n = (unsigned long long)steps;
  CUDA_OK(cudaMemcpyAsync(s->t, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream));
  CUDA_OK(cudaMemcpyAsync(s->nsteps, &n, sizeof(n), cudaMemcpyHostToDevice, s->stream));
  CUDA_OK(cudaStreamSynchronize(s->stream));
  return HW_OK;
}

int hw_sync(hw_solver* s) {
  if (!s) return fail(HW_ERR_ARG, "hw_sync: null solver");
  CUDA_OK(cudaGetLastError());
  return read_status(s);
}

}  // extern "C"
