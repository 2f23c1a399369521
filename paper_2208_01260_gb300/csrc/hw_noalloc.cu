// hw_rhs1d_noalloc: the 1D right-hand side without any device allocation.
//
// The regular path (hw_create + hw_init + hw_rhs) keeps the equilibrium state, the b-only source
// terms, the interface values and the alpha accumulator in buffers that hw_create obtains with
// cudaMalloc. This entry point places all of that working memory in one file-scope __device__
// array instead, so a caller who must not allocate device memory can still evaluate the operator:
// the caller passes its own input and output buffers, and this file allocates nothing.
//
// Limits and sharing (also stated in include/hwswe.h):
//   * at most HW_NOALLOC_MAX_NX nodes; larger grids are rejected with HW_ERR_ARG;
//   * the array lives as long as the library is loaded, on every GPU that loads it;
//   * every call reuses the same array and leaves its contents behind, so calls that overlap on the
//     GPU (different streams, or different host threads without ordering) race;
//   * the first call on a device looks up the array's device address with cudaGetSymbolAddress
//     while that device is current; make that first call before any stream capture;
//   * the kernels flag a non-positive or non-finite depth in a status word inside the array; each
//     call clears it first and reads it back at the end (a 4-byte copy and a wait for the stream), so
//     bad input is reported by the call that received it and never leaks into a later call.
#include <mutex>
#include <string>

#include "../../include/hwswe.h"
#include "hw_internal.h"

namespace {

constexpr int kMaxNx = HW_NOALLOC_MAX_NX;
// planes of nx doubles: state 4, static 2, b_x 1, source term 1; planes of nx+1: interface 6, candidates 6
constexpr size_t kPlane = (size_t)kMaxNx + 1;
constexpr size_t kScratchDoubles = 20 * kPlane + 16;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};  // device address of the array, per device ordinal

int noalloc_fail(int code, const char* msg) { return hw::set_last_error(code, msg); }

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return noalloc_fail(HW_ERR_CUDA, "hw_rhs1d_noalloc: no usable current device");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(HW_ERR_CUDA, (std::string("hw_rhs1d_noalloc: cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e)).c_str());
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return HW_OK;
}

}  // namespace

extern "C" int hw_rhs1d_noalloc(const hw_grid* grid, const hw_params* params, const double* h, const double* hu,
                                const double* b, const double* const* deriv, double* const* out,
                                void* cuda_stream) {
  if (!grid || !params || !h || !hu || !b || !deriv || !out)
    return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: null argument");
  if (grid->dim != 1 || grid->ny != 1) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: needs a 1D grid");
  if (grid->nx < 2) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: need nx >= 2");
  if (grid->nx > kMaxNx)
    return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: nx exceeds HW_NOALLOC_MAX_NX (16384); use hw_create/hw_rhs");
  if (grid->bc_x < 0 || grid->bc_x > 2) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: bad boundary condition");
  if (!(grid->x1 > grid->x0)) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: empty domain");
  if (params->precision != HW_FP64) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: HW_FP64 only");
  if (!(params->g > 0) || !(params->eps_w > 0))
    return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: g and eps_w must be positive");
  for (int q = 0; q < 3; ++q)
    if (!deriv[q]) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: null derivative plane");
  for (int q = 0; q < 4; ++q)
    if (!out[q]) return noalloc_fail(HW_ERR_ARG, "hw_rhs1d_noalloc: null output plane");

  double* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != HW_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  const int nx = grid->nx;
  const double dx = (grid->x1 - grid->x0) / nx;
  hw::Dev1D d{};
  d.nx = nx;
  d.bc = grid->bc_x;
  d.dx = dx;
  d.inv_dx = 1.0 / dx;
  d.g = params->g;
  d.eps_w = params->eps_w;
  d.eps_lim = params->eps_lim;
  d.c_b = 0.5 / dx;
  d.c_g = 1.0 / (24.0 * dx);
  double* p = base;
  for (int q = 0; q < 4; ++q, p += kPlane) d.S[q] = p;
  for (int q = 0; q < 2; ++q, p += kPlane) d.stat[q] = p;
  d.bx = p; p += kPlane;
  d.sv = p; p += kPlane;
  for (int q = 0; q < 6; ++q, p += kPlane) d.X[q] = p;
  for (int q = 6; q < 9; ++q) d.X[q] = nullptr;
  for (int q = 0; q < 6; ++q, p += kPlane) d.qb[q] = p;
  unsigned long long* amax = (unsigned long long*)p;  // 2 slots, cleared by launch_alpha1d
  double* alpha = p + 2;                               // 2 slots
  int* status = (int*)(p + 4);                         // depth flag written by the kernels

  // the status word keeps whatever the previous call left: clear it before this call's kernels
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess)
    return noalloc_fail(HW_ERR_CUDA, (std::string("hw_rhs1d_noalloc: clearing the status failed: ") +
                                      cudaGetErrorString(e)).c_str());

  hw::PhysIn1D in{};
  in.p[0] = h; in.p[1] = hu; in.p[2] = b;
  in.p[3] = deriv[0]; in.p[4] = deriv[1]; in.p[5] = deriv[2];
  // conversion to the equilibrium variables and the b-only source terms (overwrites every slot read)
  hw::launch_init1d(d, in, status, st);
  hw::launch_alpha1d(d, amax, status, st);
  hw::launch_finish_alpha1d(d, amax, alpha, nullptr, params->cfl, nullptr, -1.0, st);
  const bool lin = params->linear_weights != 0, chr = params->char_decomp != 0;
  hw::launch_sweep1d(d, alpha, lin, chr, st);
  hw::StageArgs1D sa{};
  for (int q = 0; q < 4; ++q) sa.rhs_out[q] = out[q];
  hw::launch_node1d(d, sa, hw::MODE_RHS, lin, chr, st);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(HW_ERR_CUDA, (std::string("hw_rhs1d_noalloc: launch failed: ") + cudaGetErrorString(e)).c_str());
  // the depth check of the initialisation and of the alpha reduction: read the flag back
  int flags = 0;
  e = cudaMemcpyAsync(&flags, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return noalloc_fail(HW_ERR_CUDA, (std::string("hw_rhs1d_noalloc: reading the status failed: ") +
                                      cudaGetErrorString(e)).c_str());
  if (flags & hw::HW_STATUS_DEPTH) return noalloc_fail(HW_ERR_DEPTH, "hw_rhs1d_noalloc: non-positive depth in the input");
  if (flags) return noalloc_fail(HW_ERR_NONFINITE, "hw_rhs1d_noalloc: non-finite depth or velocity in the input");
  return HW_OK;
}
