// Internal structures shared by the kernels and the C-ABI layer (not part of the public header).
#pragma once
#include <algorithm>
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/hwswe.h"

namespace hw {

enum { MODE_STAGE = 0, MODE_RHS = 1 };
enum { HW_STATUS_DEPTH = 1, HW_STATUS_NONFINITE = 2, HW_STATUS_TIMEOUT = 4, HW_STATUS_BOUNDS = 8 };

// Everything a 2D kernel needs, passed by value. R is the working precision (double for the scheme,
// float for the single-precision variant) of the planes and of the grid constants.
template <class R>
struct Dev2DT {
  int nx, ny, bc_x, bc_y;
  R dx, dy, inv_dx, inv_dy, g, eps_w, eps_lim;
  // assembly constants: 1/(2dx), 1/(2dy), 1/(24dx), 1/(24dy), 1/(12dx), 1/(12dy)
  R c_bx, c_by, c_gx, c_gy, c_mx, c_my;
  R* S[9];      // current state (eta, m, w, dx V, dy Q)
  R* stat[3];   // b, dx b_x, dy b_y
  R* bxy[2];    // b_x, b_y (physical, for conversions and static terms)
  R* X[12];     // x-interface values, pitch nx+1
  R* Y[12];     // y-interface values, pitch nx, ny+1 rows
  R* qbx[6];    // source candidates at x-interfaces ('+' q1..q3, '-' q1..q3)
  R* qby[6];
  R* sv[2];     // static derivative-source terms of the V equations (m, w components)
  R* sq[2];     // ... of the Q equations
};
using Dev2D = Dev2DT<double>;

template <class R>
struct StageArgsT {
  int k;             // RK stage 1..3
  int limiter;
  const R* dt;       // device scalar
  R* out[9];
  R* base[9];
  R* rhs_out[9];
};
using StageArgs = StageArgsT<double>;

struct Ptr9 {
  double* p[9];
};

struct Ptr12 {
  void* p[12];  // planes of either precision
};

struct PhysIn {
  const double* p[12];  // h, hu, hv, b, h_x, hu_x, hv_x, h_y, hu_y, hv_y, b_x, b_y
};

// 1D
struct Dev1D {
  int nx, bc;
  double dx, inv_dx, g, eps_w, eps_lim;
  double c_b, c_g;   // 1/(2dx), 1/(24dx)
  double* S[4];      // eta, m, dx H, dx M
  double* stat[2];   // b, dx b_x
  double* bx;        // b_x
  double* X[9];      // interface values: 2Fhat (2), 2bhat (2), 24dx Ghat (2), + 3 spare
  double* qb[6];
  double* sv;        // dx [B^]_x / dx (m component)
};

struct StageArgs1D {
  int k, limiter;
  const double* dt;
  double* out[4];
  double* base[4];
  double* rhs_out[4];
};

struct PhysIn1D {
  const double* p[6];  // h, hu, b, h_x, hu_x, b_x
};

// launchers (hw_kernels2d.cu)
int set_kernel_attributes2d();
// amax (double grids): kAlpha2dScratch device slots: the alpha_x and alpha_y keys, then scratch of the
// reduction (its float maxima, then one slot per tile); the first three are cleared here. The float
// variant's reduction uses the first three.
constexpr int kAlpha2dTiles = 152 * 8;
constexpr int kAlpha2dScratch = 3 + kAlpha2dTiles;
void launch_alpha2d(const Dev2D& d, unsigned long long* amax, int* status, cudaStream_t st);
void launch_finish_alpha2d(const Dev2D& d, const unsigned long long* amax, double* alpha, double* dt_out,
                           double cfl, const double* t_now, double t_end, cudaStream_t st);
void launch_sweep_x2d(const Dev2D& d, const double* alpha, bool linear, bool chr, cudaStream_t st);
void launch_sweep_y2d(const Dev2D& d, const double* alpha, bool linear, bool chr, cudaStream_t st);
void launch_node2d(const Dev2D& d, const StageArgs& sa, int mode, bool linear, bool chr, cudaStream_t st);
void launch_init2d(const Dev2D& d, const PhysIn& in, int* status, cudaStream_t st);
// the b-only source terms alone (launch_init2d runs them after the conversion)
void launch_static2d(const Dev2D& d, cudaStream_t st);
void launch_convert2d(const Dev2D& d, const Ptr9& src, const Ptr9& dst, int layout, int dir, cudaStream_t st);
// single-precision variant of the stage kernels, and plane casts between precisions
void launch_alpha2d(const Dev2DT<float>& d, unsigned long long* amax, int* status, cudaStream_t st);
void launch_sweep_x2d(const Dev2DT<float>& d, const float* alpha, bool linear, bool chr, cudaStream_t st);
void launch_sweep_y2d(const Dev2DT<float>& d, const float* alpha, bool linear, bool chr, cudaStream_t st);
// alpha[2] and dt of the double scalars, rounded into out[0..2] (once per stage of the float variant)
void launch_scalars_to_float(const double* alpha, const double* dt, float* out, cudaStream_t st);
void launch_node2d(const Dev2DT<float>& d, const StageArgsT<float>& sa, int mode, bool linear, bool chr,
                   cudaStream_t st);
void launch_cast_planes(int nplanes, size_t n, const Ptr12& src, const Ptr12& dst, int to_float, cudaStream_t st);

// record an error message for hw_last_error (hw_api.cu); returns code
int set_last_error(int code, const char* msg);

// launchers (hw_kernels1d.cu)
void launch_alpha1d(const Dev1D& d, unsigned long long* amax, int* status, cudaStream_t st);
void launch_finish_alpha1d(const Dev1D& d, const unsigned long long* amax, double* alpha, double* dt_out,
                           double cfl, const double* t_now, double t_end, cudaStream_t st);
void launch_sweep1d(const Dev1D& d, const double* alpha, bool linear, bool chr, cudaStream_t st);
void launch_node1d(const Dev1D& d, const StageArgs1D& sa, int mode, bool linear, bool chr, cudaStream_t st);
void launch_init1d(const Dev1D& d, const PhysIn1D& in, int* status, cudaStream_t st);
void launch_convert1d(const Dev1D& d, const Ptr9& src, const Ptr9& dst, int layout, int dir, cudaStream_t st);



// Solver internals used by the adjoint (hw_adjoint.cu); defined in hw_api.cu.
struct SolverView {
  cudaStream_t stream;
  Dev2D* d2;            // null for 1D solvers
  double** state;       // current state planes (9)
  double* base[9];
  double* alpha;
  double* dt;
  const hw_params* params;
  size_t n;
};
int solver_view(hw_solver* s, SolverView* v);
// Sub-domain solvers (hw_dd.cu): the planes a halo exchange moves (set 0: the 9 state planes of the current
// state; set 1: those and the static planes b, dx b_x, dy b_y, b_x, b_y), the extended grid's Dev2D, and
// the stream the solver launches on (swapped for graph capture; returns the previous one).
int part_planes(hw_solver* s, int set, double** planes, int* nplanes);
const Dev2D* part_dev(hw_solver* s);
cudaStream_t solver_swap_stream(hw_solver* s, cudaStream_t st);
int solver_cur(hw_solver* s);                  // which of the two state buffers holds the state
cudaStream_t solver_stream(hw_solver* s);
const hw_part_info* part_info(hw_solver* s);   // null unless a block solver
// still water (h = 1, everything else 0) on the 2-node ring of 12 extended input planes (hw_dd.cu)
void launch_fill_ring(double* const* planes12, int nxe, int nye, cudaStream_t st);
// The blocks of a single-GPU block decomposition (hw_dd.cu), and its halo exchange on any set of
// nplanes planes per block (planes[p][q], extended grids; oddx / oddy: bit q set for planes that change
// sign across x- / y-walls), and the transpose of that exchange (for adjoints: the ring's values are
// added to the nodes they were copied from and the ring is cleared). Stream-ordered on st.
int dd_blocks(hw_dd* d, int* np, hw_solver* const** parts, const hw_part_info** info, cudaStream_t* st,
              const hw_grid** grid);
int dd_exchange_planes(hw_dd* d, double* const* const* planes, int nplanes, unsigned oddx, unsigned oddy,
                       cudaStream_t st);
int dd_exchange_adjoint(hw_dd* d, double* const* const* planes, int nplanes, unsigned oddx, unsigned oddy,
                        cudaStream_t st);
// every block's stream waits for st (fork); st waits for every block's stream (join)
int dd_fork_blocks(hw_dd* d, cudaStream_t st);
int dd_join_blocks(hw_dd* d, cudaStream_t st);
int solver_set_state_planes(hw_solver* s, double* const* src);  // device copy into the current state
void adjoint_release(hw_solver* s);  // frees a solver's adjoint working buffers; hw_destroy calls it

}  // namespace hw
