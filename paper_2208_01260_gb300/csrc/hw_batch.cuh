// Device-side layout of the batched form (hw_batch.cu: one launch per phase; hw_bstep.cu: one persistent
// launch per step): per-instance grid constants, the pooled planes' base pointers, and the instance view
// the stencil functions take.
#pragma once
#include "hw_stencil2d.cuh"

namespace hw {

struct BInst {
  int nx, ny, bc_x, bc_y;
  double dx, dy, inv_dx, inv_dy, c_bx, c_by, c_gx, c_gy, c_mx, c_my;
  long long off_n, off_x, off_y;  // offsets of this grid in the pooled node / x-interface / y-interface planes
  int yc;                          // columns per y-tile group (1, 2 or 4; TILE_T / yc extended rows per tile)
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
  unsigned long long* amax;  // 3 per instance: alpha_x, alpha_y keys, the coarse pass's float maxima
  double* alpha;             // 2 per instance
  double* dt;                // 2 per instance: step, time after the step
  double* t;                 // 1 per instance
  unsigned long long* nsteps;
  int* status;
};

// The instance's grid constants with the pooled planes' base pointers (they stay in the kernel parameters;
// the kernels add the instance's offsets I.off_n, I.off_x, I.off_y to their indices).
__device__ __forceinline__ void make_dev(const BatchDev& B, const BInst& I, Dev2D& d) {
  d.nx = I.nx; d.ny = I.ny; d.bc_x = I.bc_x; d.bc_y = I.bc_y;
  d.dx = I.dx; d.dy = I.dy; d.inv_dx = I.inv_dx; d.inv_dy = I.inv_dy;
  d.g = B.g; d.eps_w = B.eps_w; d.eps_lim = B.eps_lim;
  d.c_bx = I.c_bx; d.c_by = I.c_by; d.c_gx = I.c_gx; d.c_gy = I.c_gy; d.c_mx = I.c_mx; d.c_my = I.c_my;
#pragma unroll
  for (int q = 0; q < 9; ++q) d.S[q] = B.S[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) d.stat[q] = B.stat[q];
#pragma unroll
  for (int q = 0; q < 2; ++q) d.bxy[q] = B.bxy[q];
#pragma unroll
  for (int q = 0; q < 12; ++q) { d.X[q] = B.X[q]; d.Y[q] = B.Y[q]; }
#pragma unroll
  for (int q = 0; q < 6; ++q) { d.qbx[q] = B.qbx[q]; d.qby[q] = B.qby[q]; }
#pragma unroll
  for (int q = 0; q < 2; ++q) { d.sv[q] = B.sv[q]; d.sq[q] = B.sq[q]; }
}

// Barrier and work counters of one persistent step launch (zeroed before the launch).
struct StepSync {
  unsigned int arrive;   // grid-barrier arrivals, monotonic within the launch
  unsigned int abort;    // set by a block whose barrier wait ran out; every block then leaves
  unsigned int next[6];  // work counters: per RK stage, the sweep phase and the node phase
  // global timer (ns): [0] block 0's start, [1 + p] block 0's exit from barrier p + 1 (p < 14), [15] the
  // last block's end; the 15 differences are the phases' durations (3 stages x 5 phases)
  unsigned long long t[16];
};
constexpr int BSTEP_PHASES = 15;

// Work lists of a persistent step: alpha items (inst, first node, count), x-sweep tiles (inst, first
// extended node), y-sweep tiles (inst, first extended row of a column group), node items (inst, first
// node) of TILE_T nodes.
struct StepItems {
  const int4* alpha;
  const int4* x;
  const int4* y;
  const int4* node;
  int n_alpha, n_x, n_y, n_node, n_inst;
  StepSync* sync;
  unsigned long long limit_ns;  // bound of one barrier wait on the global timer
  unsigned int limit_polls;     // and in polls
  int drop_block;               // -1; a block index only in the test of the bounded wait
};

constexpr unsigned long long BSTEP_LIMIT_NS = 10ull * 1000ull * 1000ull * 1000ull;  // 10 s
constexpr unsigned int BSTEP_LIMIT_POLLS = 1u << 26;

// One SSP-RK3 step of every instance in one cooperative launch of `grid` blocks of TILE_T threads (grid
// at most the co-resident blocks of k_bstep). B.S and B.out are the two plane sets; the step reads B.S
// when cur is 0, B.out when cur is 1. Returns the launch's cudaError_t.
int launch_bstep(const BatchDev& B, const StepItems& P, int cur, int grid, bool linear, bool chr, cudaStream_t st);
// Co-resident blocks of the persistent step kernel on the current device (0 if it cannot be launched
// cooperatively).
int bstep_grid(bool linear, bool chr);

}  // namespace hw
