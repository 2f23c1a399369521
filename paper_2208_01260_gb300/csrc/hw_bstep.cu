// Batched form, persistent: one cooperative launch advances every instance of a batch by one SSP-RK3
// step (Sec. 2.2 eq. RK; each stage the 2D operator of Sec. 3 with the alpha of Sec. 2.1 Step 1 taken
// per instance). The launch has as many blocks as can be resident at once; its phases are separated by
// grid-wide barriers:
//   per stage k = 1, 2, 3:
//     alpha, coarse pass  | alpha, exact pass  | per instance: alpha from the keys (stage 1 also the
//     step's dt, stage 3 the time update), keys cleared for the next stage  | x- and y-sweep tiles of
//     all instances  | node updates of all instances
// Alpha passes stride over their items; sweep tiles and node items are taken by blocks one at a time from
// counters, so a phase ends within one item of its last block; consecutive sweep tiles alternate between
// two shared-memory buffers, so a tile costs one block barrier as in the per-phase kernels. The tile and
// node code is the per-phase kernels' (hw_batch.cu) with state, interface and base planes read by
// ordinary loads (they are written by earlier phases of the same launch). Results equal the per-phase
// form's bit for bit in every case tested (the same source; the compiler could in principle contract
// multiply-adds differently in the two kernels).
//
// Every barrier wait is bounded: a block whose wait runs out (P.limit_ns on the global timer, or
// P.limit_polls polls) sets HW_STATUS_TIMEOUT and the abort flag; every other block leaves at its next
// barrier, so a launch always ends. The cooperative launch guarantees that all blocks are resident.
#include "../../include/hwswe.h"
#include "hw_batch.cuh"

namespace hw {

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier number ++phase (all threads of every block call it). Arrival is a release add by one
// thread after the block's barrier, the wait an acquire load followed by the block's barrier, so every
// write made by any block before the grid barrier is visible to every thread after it. Returns false if
// the block must leave the kernel (its own wait ran out, or another block's did).
__device__ __forceinline__ bool grid_barrier(const StepItems& P, unsigned int& phase, int* status, int* s_flag) {
  StepSync* const s = P.sync;
  ++phase;
  const unsigned int target = phase * gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_add_release_gpu(&s->arrive, 1u);
    const unsigned long long t0 = global_ns();
    for (unsigned int poll = 0;; ++poll) {
      if (ld_acquire_gpu(&s->arrive) >= target) break;
      if (ld_acquire_gpu(&s->abort)) {
        ok = 0;
        break;
      }
      if (poll >= P.limit_polls || global_ns() - t0 > P.limit_ns) {
        atomicOr(status, HW_STATUS_TIMEOUT);
        atomicExch(&s->abort, 1u);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    *s_flag = ok;
    if (blockIdx.x == 0 && phase < 15) s->t[phase] = global_ns();
  }
  __syncthreads();
  return *s_flag != 0;
}

// The instance view of stage input planes: B.S (sel = false) or B.out (sel = true).
__device__ __forceinline__ void make_dev_in(const BatchDev& B, const BInst& I, bool sel, Dev2D& d) {
  make_dev(B, I, d);
  if (sel) {
#pragma unroll
    for (int q = 0; q < 9; ++q) d.S[q] = B.out[q];
  }
}

// Shared memory of a block: two sweep tiles (consecutive tiles alternate, so one barrier per tile
// suffices) and the block-uniform values the phases pass around.
struct BStepSmem {
  double tile[2][NREC * TILE_T];
  int item[2];     // the next sweep tile, written by thread 0 during the current one
  int node_item;   // the block's current node item
  int flag;        // grid barrier: 1 = continue
};

// Next node item for the whole block (all threads call; the value is block-uniform).
__device__ __forceinline__ int next_node_item(unsigned int* counter, BStepSmem& sh) {
  __syncthreads();  // every thread has read the previous value
  if (threadIdx.x == 0) sh.node_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return sh.node_item;
}

// One RK stage k of every instance: it reads B.S and writes B.out, or the reverse if sel.
template <bool LINEAR, bool CHAR>
__device__ __forceinline__ bool bstep_stage(const BatchDev& B, const StepItems& P, int k, bool sel, BStepSmem& sh,
                                            unsigned int& phase) {
  StepSync* const S = P.sync;
  // ---- alpha, coarse pass (float estimates of |u| + c, |v| + c per node; maxima per instance) ----
  for (int w = blockIdx.x; w < P.n_alpha; w += gridDim.x) {
    const int4 it = P.alpha[w];
    const BInst& I = B.inst[it.x];
    Dev2D d;
    make_dev_in(B, I, sel, d);
    float mx = 0.0f, my = 0.0f;
    int bad = 0;
    const size_t base = (size_t)I.off_n;
    for (int o = it.y + threadIdx.x; o < it.y + it.z; o += blockDim.x) {
      float ax, ay;
      bool exact, neg;
      alpha_coarse<true>(d, base + o, ax, ay, exact, neg);
      if (exact) continue;
      if (neg) {
        bad |= HW_STATUS_DEPTH;
        continue;
      }
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
  if (!grid_barrier(P, phase, B.status, &sh.flag)) return false;
  // ---- alpha, exact pass (double values of the nodes near the float maxima, as ordered keys) ----
  for (int w = blockIdx.x; w < P.n_alpha; w += gridDim.x) {
    const int4 it = P.alpha[w];
    const BInst& I = B.inst[it.x];
    Dev2D d;
    make_dev_in(B, I, sel, d);
    const unsigned int* m32 = reinterpret_cast<const unsigned int*>(B.amax + 3 * it.x + 2);
    unsigned long long kx = 0, ky = 0;
    int bad = 0;
    const size_t base = (size_t)I.off_n;
    alpha_exact_range<true>(d, m32, base + it.y + threadIdx.x, base + it.y + it.z, blockDim.x, kx, ky, bad);
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
  if (!grid_barrier(P, phase, B.status, &sh.flag)) return false;
  // ---- per instance: alpha; the step's dt at stage 1 (dt = cfl / (ax/dx + ay/dy)), its time at stage 3 ----
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n_inst; i += gridDim.x * blockDim.x) {
    const double ax = __longlong_as_double((long long)B.amax[3 * i]);
    const double ay = __longlong_as_double((long long)B.amax[3 * i + 1]);
    B.alpha[2 * i] = ax;
    B.alpha[2 * i + 1] = ay;
    if (k == 1) {
      const BInst& I = B.inst[i];
      const double dt = B.cfl / fma(ax, I.inv_dx, ay * I.inv_dy);
      B.dt[2 * i] = dt;
      B.dt[2 * i + 1] = B.t[i] + dt;
    } else if (k == 3) {
      B.t[i] = B.dt[2 * i + 1];
      if (B.dt[2 * i] > 0.0) ++B.nsteps[i];
    }
    B.amax[3 * i] = 0ull;
    B.amax[3 * i + 1] = 0ull;
    B.amax[3 * i + 2] = 0ull;
  }
  // ---- x- and y-sweep tiles of every instance, taken from a counter one tile ahead ----
  unsigned int* const sweep_ctr = &S->next[2 * (k - 1)];
  if (threadIdx.x == 0) sh.item[0] = (int)atomicAdd(sweep_ctr, 1u);
  if (!grid_barrier(P, phase, B.status, &sh.flag)) return false;  // (its block barrier publishes item[0])
  const int n_sweep = P.n_x + P.n_y;
  // Tile i uses tile[i & 1] and item[i & 1]. Thread 0 writes item[(i + 1) & 1] before tile i's internal
  // barrier, and every thread reads it after that barrier; both buffers of parity i & 1 were last read
  // before tile i - 1's internal barrier, which every thread has passed when tile i starts writing them.
  for (int i = 0;; ++i) {
    const int w = sh.item[i & 1];
    if (w >= n_sweep) break;
    if (threadIdx.x == 0) sh.item[(i + 1) & 1] = (int)atomicAdd(sweep_ctr, 1u);
    double* sm = sh.tile[i & 1];
    if (w < P.n_x) {
      const int4 it = P.x[w];
      const BInst& I = B.inst[it.x];
      Dev2D d;
      make_dev_in(B, I, sel, d);
      sweep_x_tile<LINEAR, CHAR, true, true>(d, B.alpha[2 * it.x], (unsigned)it.y, sm, (size_t)I.off_n,
                                             (size_t)I.off_x);
    } else {
      const int4 it = P.y[w - P.n_x];
      const BInst& I = B.inst[it.x];
      Dev2D d;
      make_dev_in(B, I, sel, d);
      sweep_y_tile<LINEAR, CHAR, true, true>(d, B.alpha[2 * it.x + 1], (unsigned)it.y, I.yc, sm,
                                             (size_t)I.off_n, (size_t)I.off_y);
    }
  }
  if (!grid_barrier(P, phase, B.status, &sh.flag)) return false;
  // ---- node updates (RHS assembly, limiter, RK combination), TILE_T consecutive nodes of one grid per
  // block item (measured: warp-sized items taken by each warp from the counter ran slower) ----
  {
    unsigned int* const node_ctr = &S->next[2 * (k - 1) + 1];
    for (;;) {
      const int w = next_node_item(node_ctr, sh);
      if (w >= P.n_node) break;
      const int4 it = P.node[w];
      const BInst& I = B.inst[it.x];
      const int o = it.y + threadIdx.x;
      if (o < I.nx * I.ny) {
        const int j = o / I.nx, ii = o - j * I.nx;
        Dev2D d;
        make_dev_in(B, I, sel, d);
        StageArgs sa;
        sa.k = k;
        sa.limiter = B.limiter;
        sa.dt = B.dt + 2 * it.x;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          sa.out[q] = sel ? B.S[q] : B.out[q];
          sa.base[q] = B.base[q];
          sa.rhs_out[q] = nullptr;
        }
        node_update<MODE_STAGE, LINEAR, CHAR, true, true>(d, sa, ii, j, (size_t)I.off_n, (size_t)I.off_x,
                                                          (size_t)I.off_y);
      }
    }
  }
  if (k < 3 && !grid_barrier(P, phase, B.status, &sh.flag)) return false;
  return true;
}

// B.S and B.out are the two plane sets; the step's input is B.S when cur is 0, and the stages alternate.
// (One copy of the stage code selects the input pointers: two inlined copies, one per direction, spill
// several times more.) Dynamic shared memory: one BStepSmem.
template <bool LINEAR, bool CHAR>
__global__ void __launch_bounds__(TILE_T, 2) k_bstep(const BatchDev B, const StepItems P, int cur) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BStepSmem& sh = *reinterpret_cast<BStepSmem*>(smem_raw);
  if ((int)blockIdx.x == P.drop_block) return;  // test of the bounded wait: this block never arrives
  if (blockIdx.x == 0 && threadIdx.x == 0) P.sync->t[0] = global_ns();
  unsigned int phase = 0;
  for (int k = 1; k <= 3; ++k)
    if (!bstep_stage<LINEAR, CHAR>(B, P, k, ((cur + k - 1) & 1) != 0, sh, phase)) return;
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&P.sync->t[15], global_ns());
}

template <bool L, bool C>
int launch_bstep_t(const BatchDev& B, const StepItems& P, int cur, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TILE_T);
  cfg.dynamicSmemBytes = sizeof(BStepSmem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_bstep<L, C>, B, P, cur);
}

int launch_bstep(const BatchDev& B, const StepItems& P, int cur, int grid, bool linear, bool chr, cudaStream_t st) {
  if (linear) return chr ? launch_bstep_t<true, true>(B, P, cur, grid, st) : launch_bstep_t<true, false>(B, P, cur, grid, st);
  return chr ? launch_bstep_t<false, true>(B, P, cur, grid, st) : launch_bstep_t<false, false>(B, P, cur, grid, st);
}

template <bool L, bool C>
int bstep_grid_t() {
  int dev = 0, sms = 0, coop = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_bstep<L, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BStepSmem)) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_bstep<L, C>, TILE_T, sizeof(BStepSmem)) != cudaSuccess)
    return 0;
  return sms * bps;
}

int bstep_grid(bool linear, bool chr) {
  if (linear) return chr ? bstep_grid_t<true, true>() : bstep_grid_t<true, false>();
  return chr ? bstep_grid_t<false, true>() : bstep_grid_t<false, false>();
}

}  // namespace hw
