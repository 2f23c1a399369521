/*
 * hwswe.h — C ABI of the GB300 (sm_103a) implementation of the well-balanced fifth-order
 * finite-difference Hermite WENO scheme for the shallow water equations in pre-balanced form
 * (Zhao & Zhang, arXiv:2208.01260).
 *
 * The problem statement the calls follow: the pre-balanced system in the equilibrium variables
 * U = (eta = h + b, m = hu[, w = hv]) with the bottom b and its derivatives (Sec. 2 eq. swe-form-1d-e,
 * Sec. 3 eq. swe-form-2d-e), evolved together with the first derivatives V = U_x (and Q = U_y in 2D)
 * (eqs. swe-form-1d-h, swe-form-2d-h), gravity g, a CFL number (Sec. 4: 0.6, g = 9.812), and
 * boundary conditions per direction.
 *
 * Conventions for every call:
 *   - Return value: HW_OK (0) or a negative HW_ERR_* code; hw_last_error() gives a message for the
 *     calling thread. No exception crosses the ABI.
 *   - Arrays are FP64, row-major [ny][nx] with x fastest (1D: [nx]).
 *   - ptr_kind HW_HOST: pageable or pinned host memory; the call copies synchronously on the solver's
 *     stream. HW_DEVICE: device memory of the solver's GPU; the call is stream-ordered.
 *   - The library owns every device buffer it allocates (hw_create) and frees them (hw_destroy).
 *     Caller arrays are only read (inputs) or written (outputs) during the call, never retained.
 *   - One solver is bound to one CUDA stream; a solver is not thread-safe.
 *   - Node layout: periodic directions place nodes at x0 + i dx, reflective and transmissive
 *     directions at cell centres x0 + (i + 1/2) dx with the boundaries at x0 and x1; dx = (x1 - x0) / nx.
 *     Transmissive boundaries (the paper's Ex. 4.4-4.5 name none; this reading extrapolates at order
 *     zero): each ghost node copies the nearest boundary node, values and derivatives alike.
 */
#ifndef HWSWE_H
#define HWSWE_H

#ifdef __cplusplus
extern "C" {
#endif

#define HW_OK 0
#define HW_ERR_ARG (-1)       /* invalid argument, size or pointer kind                          */
#define HW_ERR_DEPTH (-2)     /* h <= 0 in the state (the scheme has no wet/dry treatment)        */
#define HW_ERR_NONFINITE (-3) /* NaN or Inf in the state (depth or velocities)                    */
#define HW_ERR_CUDA (-4)      /* a CUDA runtime call failed (message in hw_last_error)            */
#define HW_ERR_TIMEOUT (-5)   /* a bounded device wait gave up                                    */
#define HW_ERR_STATE (-6)     /* call out of order (e.g. rk3_step before init)                    */
#define HW_ERR_NOMEM (-7)     /* device allocation failed                                         */

#define HW_BC_PERIODIC 0
#define HW_BC_REFLECTIVE 1
#define HW_BC_OUTFLOW 2 /* transmissive: each ghost node copies the nearest boundary node (all variables) */

#define HW_HOST 0
#define HW_DEVICE 1

#define HW_LAYOUT_PHYSICAL 0    /* h, hu[, hv], h_x, hu_x[, hv_x][, h_y, hu_y, hv_y]                  */
#define HW_LAYOUT_EQUILIBRIUM 1 /* eta, m[, w], eta_x, m_x[, w_x][, eta_y, m_y, w_y] (the scheme's U, V, Q) */

/* Grid: dim 1 (ny must be 1) or 2; nx, ny >= 2 (2D) or nx >= 2 (1D); bc_* are HW_BC_*. */
typedef struct {
  int dim;
  int nx, ny;
  double x0, x1, y0, y1;
  int bc_x, bc_y;
} hw_grid;

/* Parameters (Sec. 2.1 eq. GHYZZ: eps = 1e-6, 1e-10 for tiny perturbations per Ex. 4.3; Sec. 4: CFL
 * 0.6, g = 9.812). eps_lim is the epsilon of the limiter weights (Sec. 2.2). char_decomp = 1 projects
 * on characteristic fields (Sec. 2.1); limiter = 1 applies the HWENO limiter (Sec. 2.2);
 * linear_weights = 1 replaces the nonlinear weights by the linear ones (accuracy tests only).
 * precision: HW_FP64 (the scheme) or HW_FP32, the single-precision runs of Sec. 4 (Tables 1-3): the
 * state, the interface values and the stage arithmetic in float, 2D single-grid solvers only (not the
 * batched form, the adjoint or the 1D scheme). The initialisation, the b-only source terms, alpha's
 * reduction keys, dt and time stay double, and every call still takes and returns double planes. */
#define HW_FP64 0
#define HW_FP32 1
typedef struct {
  double g, cfl, eps_w, eps_lim;
  int char_decomp, limiter, linear_weights;
  int precision;
} hw_params;

typedef struct hw_solver hw_solver;

/* Create a solver on the current CUDA device, bound to cuda_stream (a cudaStream_t; NULL = legacy
 * default stream). Allocates all device buffers. *out is set on success. */
int hw_create(const hw_grid* grid, const hw_params* params, void* cuda_stream, hw_solver** out);

/* Free all device buffers of the solver and the solver itself. Safe on NULL. */
int hw_destroy(hw_solver* s);

/* Load the initial state from physical variables (Sec. 2: eta = h + b; V = (h_x + b_x, hu_x)).
 *   2D: h, hu, hv, b: nx*ny each; deriv[8] = h_x, hu_x, hv_x, h_y, hu_y, hv_y, b_x, b_y.
 *   1D: h, hu, b: nx each (hv ignored, may be NULL); deriv[3] = h_x, hu_x, b_x.
 * Precomputes the parts of the source terms that depend on b only. Returns HW_ERR_DEPTH if any
 * h <= 0 and HW_ERR_NONFINITE if any h is NaN or infinite (the state is still loaded). Synchronises the
 * stream. */
int hw_init(hw_solver* s, const double* h, const double* hu, const double* hv, const double* b,
            const double* const* deriv, int ptr_kind);

/* Right-hand side of the semi-discrete scheme at the current state, without limiter (Sec. 2.1
 * eq. swe-form-1d-semi; Sec. 3 eq. swe-form-2d-dis with the source terms read with '-'), using
 * alpha = max(|u|+c) per direction over the current state (Sec. 2.1 Step 1).
 * out: 2D 9 planes d/dt (eta, m, w, eta_x, m_x, w_x, eta_y, m_y, w_y); 1D 4 planes d/dt (eta, m, eta_x,
 * m_x). Stream-ordered for HW_DEVICE, synchronous for HW_HOST. */
int hw_rhs(hw_solver* s, double* const* out, int ptr_kind);

/* Lax-Friedrichs constants of the current state: alpha[0] = max(|u|+c), alpha[1] = max(|v|+c) (2D;
 * 0 in 1D). Synchronises the stream. HW_ERR_DEPTH if the state has h <= 0, HW_ERR_NONFINITE if it
 * holds a NaN or an infinite depth or velocity. */
int hw_alpha(hw_solver* s, double* alpha);

/* CFL time step of the current state (Sec. 4, CFL from params): 2D dt = cfl / (alpha_x/dx +
 * alpha_y/dy), 1D dt = cfl dx / alpha. Synchronises the stream. */
int hw_cfl_dt(hw_solver* s, double* dt_out);

/* One SSP-RK3 step (Sec. 2.2 eq. RK, applied to eq. swe-form-2d-dis in 2D): the right-hand side is
 * evaluated on the unmodified stage states, the combination uses the limited derivatives, alpha is
 * recomputed at every stage, and the new derivatives are stored unlimited. Asynchronous on the
 * stream; errors from the device are reported by the next synchronising call. */
int hw_rk3_step(hw_solver* s, double dt);

/* One stage k = 1, 2, 3 of the step above (per-stage testing). Stage 1 stores the step's base U^n and
 * the limited V^{n,mod}, Q^{n,mod}; stages 2, 3 use them. */
int hw_rk3_stage(hw_solver* s, int k, double dt);

/* nsteps RK3 steps with dt = CFL step computed on the device at the start of each step, clipped so
 * that the last step ends at t_end if t_end > 0 (stops early once t_end is reached: the host reads the
 * time back after chunks of about half the steps left, and steps launched past t_end have size 0 and
 * leave the state unchanged). The steps run from a captured CUDA graph when use_graph != 0. On return
 * *t_out (may be NULL) holds the simulated time advanced and *steps_out (may be NULL) the steps taken
 * (those of size 0 not counted); synchronises the stream. */
int hw_advance(hw_solver* s, int nsteps, double t_end, int use_graph, double* t_out, int* steps_out);

/* Read / write the state (the variables of Sec. 2 / Sec. 3: the physical layout h, hu, hv and their
 * derivatives, or the equilibrium layout eta = h + b, m, w and theirs). layout is HW_LAYOUT_*; out/in
 * hold 9 (2D) or 4 (1D) caller-owned planes of nx*ny doubles, host or device per ptr_kind; the
 * solver's buffers are written by a set. Synchronous for HW_HOST. HW_ERR_ARG on null planes or a bad
 * layout, HW_ERR_STATE before hw_init. */
int hw_get_state(hw_solver* s, double* const* out, int layout, int ptr_kind);
int hw_set_state(hw_solver* s, const double* const* in, int layout, int ptr_kind);

/* Read the base of the current step stored by stage 1 (U^n, V^{n,mod}, Q^{n,mod}) in the
 * equilibrium layout; out holds 9 (2D) or 4 (1D) planes. */
int hw_get_base(hw_solver* s, double* const* out, int ptr_kind);

/* Per-kernel timing of the hot path (no counterpart in the paper). While profiling is on, every kernel the solver launches is
 * bracketed by CUDA events on the solver's stream and hw_advance runs without a CUDA graph.
 * hw_get_profile waits for the stream, returns per kernel class the accumulated device time in ms and
 * the launch count, then clears them. Classes (HW_PROF_*): alpha reduction, x-sweep, y-sweep, node
 * (assembly + limiter + RK), other (scalars, conversions). ms and launches hold HW_PROF_N entries. */
#define HW_PROF_ALPHA 0
#define HW_PROF_SWEEP_X 1
#define HW_PROF_SWEEP_Y 2
#define HW_PROF_NODE 3
#define HW_PROF_OTHER 4
#define HW_PROF_N 5
int hw_set_profiling(hw_solver* s, int on);
int hw_get_profile(hw_solver* s, double* ms, int* launches);

/* Simulated time and the number of steps that advanced it (dt > 0), kept on the device by hw_rk3_step
 * and hw_advance (no counterpart in the paper; t is the time of the run of Sec. 4's examples). Together with hw_get_state / hw_set_state they checkpoint and resume a run: a
 * solver restored with hw_init (for b), hw_set_state and hw_set_time continues exactly as the
 * original would (bitwise with the equilibrium layout when the grid spacings are powers of two, so
 * that the derivative scalings are exact). hw_get_time synchronises the stream. */
int hw_get_time(hw_solver* s, double* t, long long* steps);
int hw_set_time(hw_solver* s, double t, long long steps);

/* ---------------------------------------------------------------------------------------------
 * Batched form (no counterpart in the paper, which runs one grid at a time): n independent 2D grids of
 * uneven sizes (all HW_BC_* allowed, shared parameters, HW_FP64), each advanced by the scheme of Sec. 3
 * with SSP-RK3 (Sec. 2.2 eq. RK), together, each with its own CFL time step computed on the device
 * (Sec. 4: dt from the CFL number and alpha of that grid). Each phase of an RK stage is one launch over the tiles of all grids,
 * and two steps run from one CUDA graph. Every grid's result equals a single-grid solver's
 * (hw_create + hw_advance) to rounding; tile shapes do not change it at all.
 * ------------------------------------------------------------------------------------------- */
typedef struct hw_batch hw_batch;

/* grids[n]: 2D grids (nx, ny >= 2). Allocates pooled device buffers. */
int hw_batch_create(int n, const hw_grid* grids, const hw_params* params, void* cuda_stream, hw_batch** out);
int hw_batch_destroy(hw_batch* b);
/* Initial state of grid i, as hw_init (2D): h, hu, hv, b and deriv[8]. Synchronises the stream. */
int hw_batch_init(hw_batch* b, int i, const double* h, const double* hu, const double* hv, const double* bb,
                  const double* const* deriv, int ptr_kind);
/* nsteps SSP-RK3 steps of every grid at its own CFL dt; synchronises and reports HW_ERR_DEPTH if any
 * grid produced a non-positive or non-finite depth. */
int hw_batch_run(hw_batch* b, int nsteps, int use_graph);
/* State of grid i (9 planes, layout HW_LAYOUT_*). */
int hw_batch_get_state(hw_batch* b, int i, double* const* out, int layout, int ptr_kind);
/* Simulated time and step count of every grid (t[n], steps[n]; either may be NULL). */
int hw_batch_get_time(hw_batch* b, double* t, int* steps);
/* Tile shape of grid i. The sweeps run over flattened extended lines (each row, or each group of yc
 * columns, with its 2 halo nodes on either side, one after the other): a tile of 192 threads forms 192
 * node records and the interfaces whose stencils lie among them, so tiles run across line ends and no
 * grid size leaves a ragged tile. An x-tile covers 192 consecutive extended nodes of the rows (189
 * interfaces); a y-tile yc = 1, 2 or 4 adjacent columns of 192 / yc extended rows (yc (192 / yc - 3)
 * interfaces). Chosen by the autotuner; arithmetic is unaffected. */
int hw_batch_set_tiles(hw_batch* b, int i, int yc);
int hw_batch_get_tiles(hw_batch* b, int i, int* yc);
/* Autotuner measurement: average ms of the batched x-sweep and y-sweep over the grids ids[nids] with
 * the trial y-tile width yc, over reps repetitions. Changes no state (interface planes are scratch). */
int hw_batch_time_tiles(hw_batch* b, int nids, const int* ids, int yc, int reps, double* ms_x, double* ms_y);
/* Launch form of hw_batch_run (no counterpart in the paper). on = 0 (default): each phase of an RK stage
 * is one launch over all grids (12 launches and 3 small key resets per step). on = 1: each step is ONE
 * cooperative launch of as many blocks as the device holds at once (two small resets before it); its
 * phases (the two alpha passes, the per-grid alpha and dt, both sweeps, the node update; three times) are
 * separated by grid-wide barriers, and sweep tiles and node items are taken from counters. Each barrier
 * wait is bounded (about 10 s): if one runs out, every block leaves the launch and hw_batch_run returns
 * HW_ERR_TIMEOUT (the state is then undefined). The results equal the default form's to rounding.
 * hw_batch_set_persistent returns HW_ERR_CUDA if the device cannot launch the step kernel cooperatively,
 * HW_ERR_ARG for on other than 0 or 1; a switch drops the captured graph. hw_batch_get_persistent
 * gives the form and the step kernel's block count (0 before the first switch to on = 1). */
int hw_batch_set_persistent(hw_batch* b, int on);
int hw_batch_get_persistent(hw_batch* b, int* on, int* blocks);
/* Test of the persistent step's bounded barrier wait (after hw_batch_set_persistent(b, 1)): one launch in
 * which block 0 leaves before the first grid barrier, with a 2 ms bound; the other blocks' waits run out
 * and every block leaves. Returns HW_ERR_TIMEOUT when the bound worked (HW_OK would mean a barrier
 * passed without block 0). The state, times and the context stay usable: the alpha keys, which every
 * step resets, are the only memory written. HW_ERR_STATE before hw_batch_set_persistent(b, 1). */
int hw_batch_test_barrier_timeout(hw_batch* b);
/* Phase durations of the last persistent step launch, ms[15] in ms: for each RK stage the alpha coarse
 * pass, the alpha exact pass, the per-grid alpha and dt, both sweeps, the node update (from the device's
 * global timer read by block 0 as it leaves each grid barrier; the last phase ends with the last block).
 * -1 for a phase the launch did not reach. Synchronises the stream. HW_ERR_STATE unless the batch is in
 * the persistent form. */
int hw_batch_get_phase_times(hw_batch* b, double* ms);

/* ---------------------------------------------------------------------------------------------
 * Discrete adjoint (2D, nonlinear weights and characteristic projection; limiter on or off).
 * The paper has no adjoint: these calls reverse the discrete map it defines, i.e. one SSP-RK3 step
 * (Sec. 2.2 eq. RK) of the 2D semi-discrete scheme (Sec. 3 eq. swe-form-2d-dis, with the reconstruction
 * and source balance of Sec. 2.1 and the limiter of Sec. 2.2 applied per direction).
 * Gradients are with respect to the equilibrium state planes (eta, m, w, eta_x, m_x, w_x, eta_y, m_y,
 * w_y) and the static planes (b, b_x, b_y) taken as independent arrays (eta held fixed when b moves).
 * The time steps are given explicitly, so the adjoint differentiates the map the caller evaluates.
 * alpha = max(|u|+c) is differentiated through the first node attaining the maximum, with d|x| = dx at
 * x = 0 (max is not differentiable where several nodes tie).
 * All planes are caller-owned device arrays of nx*ny doubles, row-major [ny][nx], on the solver's
 * device; the calls run on the solver's stream and return once the work is queued (hw_adjoint_run
 * synchronises the stream). Errors: HW_ERR_ARG (null pointer, 1D solver, linear weights or no
 * characteristic projection, gauge index outside the grid, grid above about 2^30 nodes), HW_ERR_STATE
 * (before hw_init), HW_ERR_NOMEM (working buffers, snapshots or tape), HW_ERR_CUDA.
 * Working buffers (about 180 planes of nx*ny doubles) are allocated at the first call and freed by
 * hw_destroy.
 * ------------------------------------------------------------------------------------------- */
/* Reverse of one hw_rk3_step(dt) taken from the solver's current state: lam_state (9 device planes,
 * equilibrium layout) holds the adjoint of the step's output on entry and of its input on return;
 * lam_static (3 device planes: b, b_x, b_y) is incremented. The solver's state is unchanged. */
int hw_adjoint_step(hw_solver* s, double dt, double* const* lam_state, double* const* lam_static);

/* Gauge misfit L = sum_{n=1..nsteps} sum_g (eta^n[gauge_idx[g]] - eta_obs[(n-1)*ngauge + g])^2 of the run
 * from the current state with time steps dts[nsteps] (host arrays; gauge_idx are node indices j*nx+i).
 * eta_gauges (host, may be NULL) receives the model's gauge values. The solver returns to the initial
 * state. */
int hw_gauge_loss(hw_solver* s, int nsteps, const double* dts, const int* gauge_idx, int ngauge,
                  const double* eta_obs, double* loss_out, double* eta_gauges);

/* The same loss and its gradient (grad_state: 9 device planes, grad_static: 3 device planes, both
 * overwritten) by the adjoint. `snapshots` selects the storage of the forward run:
 *   >= 0          binomial checkpointing: at most `snapshots` intermediate states are held and the
 *                 schedule minimising the recomputed forward steps is found by dynamic programming over
 *                 (steps left, snapshots left); each reversed step is first recomputed from its state;
 *   HW_ADJ_TAPE   every stage input, stage alpha and source interface value of every step is kept in
 *                 device memory (about 51 planes of nx*ny doubles per step), so nothing is recomputed;
 *                 HW_ERR_NOMEM when that exceeds 90% of the free device memory;
 *   HW_ADJ_AUTO   HW_ADJ_TAPE when it fits, else checkpointing with as many snapshots as fit.
 * *forward_steps_out (may be NULL) receives the forward steps taken (loss pass plus recomputation). The
 * solver returns to the initial state. */
#define HW_ADJ_TAPE (-1)
#define HW_ADJ_AUTO (-2)
int hw_adjoint_run(hw_solver* s, int nsteps, const double* dts, const int* gauge_idx, int ngauge,
                   const double* eta_obs, int snapshots, double* loss_out, double* const* grad_state,
                   double* const* grad_static, long long* forward_steps_out);

/* ---------------------------------------------------------------------------------------------
 * Block decomposition of one 2D grid (no counterpart in the paper, which runs one grid at a time). The
 * nx x ny grid is split into px x py blocks, each advanced by its own solver on its own nodes plus a ring
 * of 2 halo nodes on every side: an interface's stencil spans nodes i-1..i+2 (Sec. 2.1 Step 1) and the
 * limiter's i-1..i+1 (Sec. 2.2). Before every RK stage the ring is refreshed from the neighbouring blocks
 * (on the grid's own boundary: from the block itself, by the boundary condition), and alpha, global per
 * direction and stage (Sec. 2.1 Step 1), is the maximum over the blocks' maxima. Every node of every
 * block then computes from the same values as on the undecomposed grid: the result is hw_advance's, bit
 * for bit. HW_FP64 only. The blocks may live in one process (hw_dd_*) or in one process per GPU, whose
 * halo strips and alpha keys the caller moves (hw_part_*, hw_halo_*).
 * ------------------------------------------------------------------------------------------- */
#define HW_FACE_W 0 /* x lower */
#define HW_FACE_E 1 /* x upper */
#define HW_FACE_S 2 /* y lower */
#define HW_FACE_N 3 /* y upper */
#define HW_HALO_NEIGHBOR 0  /* the neighbouring block's 2 nodes next to the shared face (periodic: across the wrap) */
#define HW_HALO_MIRROR 1    /* reflective wall: the block's own 2 nodes mirrored, signs by the parity table */
#define HW_HALO_REPLICATE 2 /* transmissive boundary: the block's boundary node, twice */
typedef struct {
  int i0, j0, nx, ny; /* the block's nodes: [i0, i0 + nx) x [j0, j0 + ny) of the global grid */
  int nbr[4];         /* per face (HW_FACE_*): the block across it for HW_HALO_NEIGHBOR, else the block itself */
  int mode[4];        /* per face: HW_HALO_* */
} hw_part_info;

/* Host only (no CUDA call). Block `part` (= bx + px * by) of the grid split into px x py blocks of nearly
 * equal size (the first nx % px block columns and ny % py block rows one node larger). HW_ERR_ARG unless
 * the grid is 2D, 1 <= px, 1 <= py, 0 <= part < px * py and every block has at least 2 x 2 nodes. */
int hw_dd_partition(const hw_grid* grid, int px, int py, int part, hw_part_info* out);

/* The solver of one block (HW_FP64): a grid of (nx + 4) x (ny + 4) nodes, the block at offset (2, 2) of
 * it, with the global grid's spacings exactly. Its own calls (hw_get_state, hw_destroy, ...) see the
 * extended grid. */
int hw_part_create(const hw_grid* grid, const hw_params* params, int px, int py, int part, void* cuda_stream,
                   hw_solver** out);
/* Initial data of the block's own nodes: 12 planes as hw_init (h, hu, hv, b, h_x, hu_x, hv_x, h_y, hu_y,
 * hv_y, b_x, b_y), each pointing at the block's first node, rows ld >= the block's nx doubles apart. The
 * ring holds still water until the set-1 exchange fills it; hw_part_finish_init then forms the b-only
 * source terms. Both synchronise the stream; HW_ERR_DEPTH / HW_ERR_NONFINITE as hw_init. */
int hw_part_init(hw_solver* s, const double* const* planes12, long long ld, int ptr_kind);
int hw_part_finish_init(hw_solver* s);
/* Halo strips (device arrays of doubles). Set 0: the 9 state planes (before every stage); set 1: those and
 * the static planes b, dx b_x, dy b_y, b_x, b_y (once, between hw_part_init and hw_part_finish_init). The
 * strip of a face holds, per plane, the 2 node rows (y faces) or columns (x faces) of the block next to
 * that face, in increasing coordinate: x faces over the block's ny rows, y faces over the full extended
 * width nx + 4, so that the y exchange, run after the x exchange, also fills the ring's corners.
 * hw_halo_strip_size: *count = doubles per strip. hw_halo_pack: the block's strip of a face into `strip`.
 * hw_halo_unpack: the ring on a face from `strip`, which is the neighbour's strip of the opposite face
 * (HW_HALO_NEIGHBOR) or the block's own strip of this face (HW_HALO_MIRROR, HW_HALO_REPLICATE).
 * Stream-ordered on the solver's stream. */
int hw_halo_strip_size(hw_solver* s, int set, int face, long long* count);
int hw_halo_pack(hw_solver* s, int set, int face, double* strip);
int hw_halo_unpack(hw_solver* s, int set, int face, int mode, const double* strip);
/* alpha keys of the block (device, 2 x 64-bit): max(|u|+c) and max(|v|+c) over its nodes and ring as the
 * bit patterns of the non-negative doubles, so that the integer maximum over all blocks (an all-reduce
 * with MAX) is the global alpha of Sec. 2.1 Step 1. Stream-ordered. */
int hw_part_alpha_keys(hw_solver* s, unsigned long long* keys);
/* RK stage k = 1, 2, 3 of the block (Sec. 2.2 eq. RK) with alpha from the global keys (device, 2): stage 1
 * takes dt = the CFL step of that alpha (Sec. 4; clipped to end at t_end if t_end > 0), stage 3 advances
 * the block's time. The ring must hold the stage's input. Stream-ordered. */
int hw_part_stage(hw_solver* s, int k, const unsigned long long* keys, double t_end);
/* out[0..1] = the maxima over n rows of keys (device, n x 2 keys as above; out device, 2): the alpha of
 * several blocks held by one process, before the maximum over processes. Stream-ordered on cuda_stream. */
int hw_dd_max_keys(const unsigned long long* keys, int n, unsigned long long* out, void* cuda_stream);

/* All px x py blocks of one grid on the current GPU, the exchange as device copies between them: create,
 * initialise from the global arrays (as hw_init), advance (as hw_advance, the same result bit for bit;
 * with use_graph two steps of all blocks run from one CUDA graph), read the global state (as
 * hw_get_state), destroy. */
typedef struct hw_dd hw_dd;
int hw_dd_create(const hw_grid* grid, const hw_params* params, int px, int py, void* cuda_stream, hw_dd** out);
int hw_dd_init(hw_dd* d, const double* h, const double* hu, const double* hv, const double* b,
               const double* const* deriv, int ptr_kind);
int hw_dd_advance(hw_dd* d, int nsteps, double t_end, int use_graph, double* t_out, int* steps_out);
int hw_dd_get_state(hw_dd* d, double* const* out, int layout, int ptr_kind);
int hw_dd_destroy(hw_dd* d);

/* Gauge misfit and its gradient for a run of the blocks (as hw_adjoint_run with HW_ADJ_TAPE, on the
 * block decomposition's current state, with every stage of every step of every block kept in device
 * memory): gauge_idx are nodes of the global grid (j nx + i); grad_state (9) and grad_static (3) are
 * device planes of the global grid (overwritten). Each block reverses its own stages; between stages the
 * transpose of the halo exchange adds the adjoints that reach a block's ring to the nodes the ring was
 * copied from; the alpha adjoint (Sec. 2.1 Step 1) is summed over the blocks and applied once, at the
 * global grid's first node attaining alpha. The loss equals hw_adjoint_run's bit for bit and the gradient
 * to rounding (sums in another order). The blocks' states are unchanged. Synchronises the stream;
 * HW_ERR_ARG, HW_ERR_NOMEM, HW_ERR_CUDA as hw_adjoint_run. */
int hw_dd_adjoint_run(hw_dd* d, int nsteps, const double* dts, const int* gauge_idx, int ngauge,
                      const double* eta_obs, double* loss_out, double* const* grad_state, double* const* grad_static);

/* The same adjoint one block at a time, for blocks owned by different processes (no counterpart in the
 * paper): the caller carries the exchanges, alpha keys, gauge values and the alpha adjoint between the
 * blocks (paper_2208_01260_gb300/decomp.py, adjoint_run). On block solver s (hw_part_create, initialised,
 * nonlinear weights and characteristic projection), in order:
 *   forward, for each step j = 0 .. nsteps-1 and stage k = 1, 2, 3: the exchange of the stage input
 *     (hw_part_adj_pack / _unpack, with the same modes, pairing and order as hw_halo_pack / _unpack),
 *     hw_part_adj_alpha_keys, the maximum of all blocks' keys, hw_part_adj_forward_stage with it;
 *   hw_part_adj_gauges, summed over all blocks (each slot holds one block's value, zeros elsewhere),
 *     and hw_part_adj_set_misfit with the full arrays (it also gives the loss);
 *   reverse, for j = nsteps-1 .. 0 and k = 3, 2, 1: hw_part_adj_reverse_stage, the sum over all blocks
 *     of their alpha adjoints and the minimum of their nodes, hw_part_adj_alpha_apply with those, then
 *     the transposed exchange of what = 0 (y faces first, then x faces): every block's ring strip of each
 *     face by hw_part_adj_rpack (which clears the ring), added by hw_part_adj_radd on the block it was
 *     copied from: the NEIGHBOR's opposite face, or the block's own face for MIRROR / REPLICATE;
 *   hw_part_adj_finish_static, the transposed exchange of what = 1, hw_part_adj_gradients.
 * Everything runs on the block solver's stream. Memory: the block's whole-run tape (every stage of every
 * step), as hw_dd_adjoint_run. Errors: HW_ERR_ARG (bad step, stage, face, mode or pointer; gauge not on
 * the block's own nodes), HW_ERR_STATE (reverse before set_misfit, apply without a reverse stage),
 * HW_ERR_NOMEM, HW_ERR_CUDA. */
typedef struct hw_part_adj hw_part_adj;
/* nloc of the ngauge gauges lie on the block's own nodes: gauge_node their global nodes (j global_nx + i),
 * gauge_slot their positions in the global list. The tape starts from the block's current state. */
int hw_part_adj_create(hw_solver* s, int nsteps, int ngauge, int nloc, const int* gauge_slot, const int* gauge_node,
                       int global_nx, hw_part_adj** out);
int hw_part_adj_destroy(hw_part_adj* a);
/* doubles of a strip of face: what = 0, the 9 state planes (stage input or its adjoint); 1, the 3 static */
int hw_part_adj_strip_size(hw_part_adj* a, int what, int face, long long* count);
int hw_part_adj_pack(hw_part_adj* a, int j, int k, int face, double* strip);                  /* device strip */
int hw_part_adj_unpack(hw_part_adj* a, int j, int k, int face, int mode, const double* strip);
int hw_part_adj_alpha_keys(hw_part_adj* a, int j, int k, unsigned long long* keys);           /* device keys[2] */
int hw_part_adj_forward_stage(hw_part_adj* a, int j, int k, double dt, const unsigned long long* keys);
int hw_part_adj_gauges(hw_part_adj* a, double* gvals);                  /* host [nsteps][ngauge]; syncs */
/* host, full arrays; loss_out (optional): the misfit, summed as hw_adjoint_run and hw_dd_adjoint_run do */
int hw_part_adj_set_misfit(hw_part_adj* a, const double* gvals, const double* eta_obs, double* loss_out);
/* lalpha[2] (host): the block's share of the alpha adjoint; argmax[2] (host): its first node (global
 * index) attaining each alpha, INT_MAX if none. Stage 3 first adds the step's misfit. Syncs. */
int hw_part_adj_reverse_stage(hw_part_adj* a, int j, int k, double dt, double* lalpha, int* argmax);
int hw_part_adj_alpha_apply(hw_part_adj* a, const double* lalpha, const int* argmax);        /* host */
int hw_part_adj_rpack(hw_part_adj* a, int what, int face, double* strip);                     /* device */
int hw_part_adj_radd(hw_part_adj* a, int what, int face, int mode, const double* strip);
int hw_part_adj_finish_static(hw_part_adj* a);
/* The block's own nodes of the state gradient (9, physical units as hw_adjoint_run) and the static one
 * (3), rows ld apart, HW_HOST or HW_DEVICE; syncs. */
int hw_part_adj_gradients(hw_part_adj* a, double* const* grad_state, double* const* grad_static, int ld, int ptr_kind);

/* Allocation-free variant of the 1D right-hand side: the same numbers as hw_create + hw_init + hw_rhs on
 * a 1D grid (out: 4 planes d/dt (eta, m, eta_x, m_x)), with every array pointer on the device. The paper
 * has no counterpart; this call exists for callers that must not allocate device memory, such as code
 * inside a framework whose memory pool owns the GPU's memory (a separate cudaMalloc could fail or escape
 * the pool's accounting) and time-critical loops that cannot pay for cudaMalloc's implicit
 * synchronisation and unpredictable latency. The caller passes inputs (h, hu, b: nx each; deriv[3] =
 * h_x, hu_x, b_x) and outputs; the working memory (state, b-only source terms, interface values, the
 * alpha accumulator) is a file-scope device array sized for HW_NOALLOC_MAX_NX nodes, which every GPU
 * that loads the library holds until the process exits. Larger grids return HW_ERR_ARG.
 *   - The call allocates nothing. Its kernels run on cuda_stream (NULL = legacy default stream); it
 *     then waits for that stream and returns HW_ERR_DEPTH if any h <= 0 and HW_ERR_NONFINITE if any
 *     depth or velocity is NaN or infinite (the output planes then hold no usable values).
 *   - Every call reuses the same array and leaves its contents behind (it clears what must start at
 *     zero), so calls that may overlap on the GPU (other streams or unordered host threads) race.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current; make that first call before any stream capture. */
#define HW_NOALLOC_MAX_NX 16384
int hw_rhs1d_noalloc(const hw_grid* grid, const hw_params* params, const double* h, const double* hu,
                     const double* b, const double* const* deriv, double* const* out, void* cuda_stream);

/* Self-check of the integer-pipe FP64 arithmetic that the 2D double kernels use for part of their
 * products and reciprocals (no counterpart in the paper; an implementation device of this library).
 * On the current device, n seeded pseudo-random operands go through the integer path and the FP64 pipe.
 * op 0, products against DMUL (operand mix: the scheme's range, short significands, near-squares,
 * signed zeros, the edges of the normal range, subnormal, infinite and NaN operands); op 1, reciprocals
 * against the correctly rounded __drcp_rn (significands near 1 and 2, every exponent); op 2, products
 * by the literal constants the kernels multiply by (the constant-folded form), against DMUL. counts
 * (host, 3 entries): results the integer fast path accepted; accepted results that differ from the
 * FP64 pipe's in any bit (ops 0, 2) or by more than one ulp (op 1); operands the fast path must take
 * but rejected (normal operands with a normal result; not counted for op 2). The last two must be 0.
 * Synchronous on the legacy default stream; allocates and frees 24 bytes. HW_ERR_ARG for another op,
 * n < 1 or counts == NULL, HW_ERR_CUDA on a CUDA failure. */
int hw_selftest_fp64_int(int op, long long n, unsigned long long seed, long long* counts);

/* FP64 throughput of the current GPU (no counterpart in the paper; the denominator of the FP64 roofline
 * that bounds this scheme's kernels on GB300, whose FP64 pipe is narrow). A kernel of independent fused
 * multiply-add chains (eight per thread, eight blocks of 256 threads on every SM) runs once to warm up
 * and then `reps` times (1..1000), each launch timed with CUDA events. out (host, 3 entries): the best
 * rate in FP64 fma per second (thread operations; one fma = 2 flops), the median rate, and the best
 * launch time in ms. Synchronous on a private stream; allocates and frees a small result buffer.
 * HW_ERR_ARG for bad arguments, HW_ERR_CUDA on a CUDA failure. */
int hw_measure_fp64_peak(int reps, double* out);

/* Wait for the stream and return the device status as an HW_ERR_* code (HW_OK if clean). */
int hw_sync(hw_solver* s);

/* Message of the last error on the calling thread ("" if none). Valid until the next call. */
const char* hw_last_error(void);

/* Library version string. */
const char* hw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HWSWE_H */
