// Block decomposition of one 2D grid (hwswe.h: hw_dd_partition, hw_halo_*, hw_dd_*).
//
// Each block is a solver on its own nodes plus a ring of 2 halo nodes (hw_part_create in hw_api.cu).
// The scheme's stencils reach 2 nodes beyond an interface or a node (Sec. 2.1 Step 1: nodes i-1..i+2 of
// the interface i+1/2; Sec. 2.2: nodes i-1..i+1 of the limiter), so once the ring holds the values the
// undecomposed grid has there, every interior interface and node of a block is computed from the same
// values in the same arithmetic, and the decomposed run equals the undecomposed one bit for bit:
//   * inside the grid the ring is a copy of the neighbouring block's nodes;
//   * on the grid's boundary it is what the undecomposed solver's index mapping reads there: the block's
//     own nodes mirrored with the parity signs (reflective walls), the boundary node (transmissive), or
//     the block across the wrap (periodic);
//   * the x faces are exchanged first over the block's rows, then the y faces over the full extended
//     width, so the ring's corners receive the diagonal neighbour's values (or their mirror images);
//   * alpha (Sec. 2.1 Step 1, global per direction and stage) is the maximum over the blocks' maxima:
//     ring nodes are copies (or mirror images, with the same |u| + c) of grid nodes, so no block's
//     maximum exceeds the global one and the block holding the maximising node attains it.
// A halo strip holds, per plane, the 2 node columns (x faces) or rows (y faces) next to a face; packing
// and unpacking are the same kernels whether the strip then moves between blocks on one GPU (hw_dd_*) or
// between processes (the caller's transport).
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/hwswe.h"
#include "hw_halo.h"
#include "hw_internal.h"

namespace hw {
namespace {

struct PlaneSet {
  double* p[14];
};

// Planes odd across x-walls and across y-walls (the parity table of the reflective boundary): state
// (eta, m, w, dx H1, dx M1, dx W1, dy H2, dy M2, dy W2), then b, dx b_x, dy b_y, b_x, b_y.
constexpr unsigned kOddX = (1u << 1) | (1u << 3) | (1u << 5) | (1u << 7) | (1u << 10) | (1u << 12);
constexpr unsigned kOddY = (1u << 2) | (1u << 5) | (1u << 6) | (1u << 7) | (1u << 11) | (1u << 13);

// Strip layout: [plane q][offset c = 0, 1 in increasing coordinate][position r along the face].
// x faces: r over the block's rows (len = nye - 4); y faces: r over the full extended width (len = nxe).
__device__ __forceinline__ void strip_coords(int face, int nxe, int nye, int c, int r, int& i, int& j) {
  const int nxl = nxe - 4, nyl = nye - 4;
  if (face == HW_FACE_W) { i = 2 + c; j = 2 + r; }
  else if (face == HW_FACE_E) { i = nxl + c; j = 2 + r; }
  else if (face == HW_FACE_S) { i = r; j = 2 + c; }
  else { i = r; j = nyl + c; }
}
__device__ __forceinline__ void ring_coords(int face, int nxe, int nye, int c, int r, int& i, int& j) {
  const int nxl = nxe - 4, nyl = nye - 4;
  if (face == HW_FACE_W) { i = c; j = 2 + r; }
  else if (face == HW_FACE_E) { i = nxl + 2 + c; j = 2 + r; }
  else if (face == HW_FACE_S) { i = r; j = c; }
  else { i = r; j = nyl + 2 + c; }
}

__global__ void k_halo_pack(PlaneSet ps, int np, int nxe, int nye, int face, double* __restrict__ strip) {
  const int len = face < 2 ? nye - 4 : nxe;
  const long long total = (long long)np * 2 * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % len), c = (int)((t / len) & 1), q = (int)(t / (2 * len));
    int i, j;
    strip_coords(face, nxe, nye, c, r, i, j);
    strip[t] = ps.p[q][(size_t)j * nxe + i];
  }
}

// The strip offset a ring offset c reads: NEIGHBOR c (the neighbour's nodes in increasing coordinate);
// MIRROR 1 - c (the ring node at distance d outside the wall is the node at distance d - 1 inside it,
// negated for planes odd across this wall); REPLICATE the boundary node.
__device__ __forceinline__ int ring_source(int face, int mode, int c) {
  if (mode == HW_HALO_MIRROR) return 1 - c;
  if (mode == HW_HALO_REPLICATE) return (face == HW_FACE_W || face == HW_FACE_S) ? 0 : 1;
  return c;
}

__global__ void k_halo_unpack(PlaneSet ps, int np, int nxe, int nye, int face, int mode, unsigned odd,
                              const double* __restrict__ strip) {
  const int len = face < 2 ? nye - 4 : nxe;
  const long long total = (long long)np * 2 * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % len), c = (int)((t / len) & 1), q = (int)(t / (2 * len));
    double v = strip[((long long)q * 2 + ring_source(face, mode, c)) * len + r];
    if (mode == HW_HALO_MIRROR && ((odd >> q) & 1u)) v = -v;
    int i, j;
    ring_coords(face, nxe, nye, c, r, i, j);
    ps.p[q][(size_t)j * nxe + i] = v;
  }
}

// Transpose of the exchange, for adjoints: the ring's values of a face (the adjoints of copies) move into
// a strip in ring order and the ring is cleared ...
__global__ void k_halo_adj_pack(PlaneSet ps, int np, int nxe, int nye, int face, double* __restrict__ strip) {
  const int len = face < 2 ? nye - 4 : nxe;
  const long long total = (long long)np * 2 * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % len), c = (int)((t / len) & 1), q = (int)(t / (2 * len));
    int i, j;
    ring_coords(face, nxe, nye, c, r, i, j);
    double* x = ps.p[q] + (size_t)j * nxe + i;
    strip[t] = *x;
    *x = 0.0;
  }
}

// ... and are added to the nodes they were copied from: the neighbour's nodes next to the opposite face
// (NEIGHBOR: called on the neighbour with that face), or the block's own nodes next to this face with the
// mirror's signs (MIRROR) or summed into the boundary node (REPLICATE). One thread per strip position
// and plane adds both ring offsets that read it, so no two threads write one node.
__global__ void k_halo_adj_add(PlaneSet ps, int np, int nxe, int nye, int face, int mode, unsigned odd,
                               const double* __restrict__ strip) {
  const int len = face < 2 ? nye - 4 : nxe;
  const long long total = (long long)np * 2 * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % len), sc = (int)((t / len) & 1), q = (int)(t / (2 * len));
    double v = 0.0;
    for (int c = 0; c < 2; ++c)
      if (ring_source(face, mode, c) == sc) v += strip[((long long)q * 2 + c) * len + r];
    if (v == 0.0) continue;
    if (mode == HW_HALO_MIRROR && ((odd >> q) & 1u)) v = -v;
    int i, j;
    strip_coords(face, nxe, nye, sc, r, i, j);
    ps.p[q][(size_t)j * nxe + i] += v;
  }
}

struct Planes12 {
  double* p[12];
};

// still water on the ring of the 12 extended input planes (interior untouched)
__global__ void k_fill_ring(Planes12 in, int nxe, int nye) {
  const long long n = (long long)nxe * nye;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % nxe), j = (int)(o / nxe);
    if (i >= 2 && i < nxe - 2 && j >= 2 && j < nye - 2) continue;
    for (int q = 0; q < 12; ++q) in.p[q][o] = q == 0 ? 1.0 : 0.0;
  }
}

// alpha keys: out[d] = maximum over the np rows keys[2 p + d] (out may follow the rows in one buffer)
__global__ void k_max_keys(const unsigned long long* keys, int np, unsigned long long* out) {
  const int d = threadIdx.x;
  if (d >= 2) return;
  unsigned long long m = 0;
  for (int p = 0; p < np; ++p) m = max(m, keys[2 * p + d]);
  out[d] = m;
}

int blocks_for(long long work) { return (int)std::max(1LL, std::min((work + 255) / 256, 152LL * 8)); }

int check_halo_args(hw_solver* s, int set, int face, const char* who) {
  if (!s || !part_info(s)) return set_last_error(HW_ERR_ARG, (std::string(who) + ": not a block solver").c_str());
  if (set != 0 && set != 1) return set_last_error(HW_ERR_ARG, (std::string(who) + ": set must be 0 or 1").c_str());
  if (face < 0 || face > 3) return set_last_error(HW_ERR_ARG, (std::string(who) + ": bad face").c_str());
  return HW_OK;
}

}  // namespace

void launch_fill_ring(double* const* planes12, int nxe, int nye, cudaStream_t st) {
  Planes12 in;
  for (int q = 0; q < 12; ++q) in.p[q] = planes12[q];
  k_fill_ring<<<blocks_for((long long)nxe * nye), 256, 0, st>>>(in, nxe, nye);
}

}  // namespace hw

extern "C" {

int hw_dd_partition(const hw_grid* g, int px, int py, int part, hw_part_info* out) {
  if (!g || !out) return hw::set_last_error(HW_ERR_ARG, "hw_dd_partition: null argument");
  if (g->dim != 2) return hw::set_last_error(HW_ERR_ARG, "hw_dd_partition: 2D grids only");
  if (px < 1 || py < 1 || part < 0 || part >= px * py)
    return hw::set_last_error(HW_ERR_ARG, "hw_dd_partition: need px, py >= 1 and 0 <= part < px * py");
  if (g->nx < 2 * px || g->ny < 2 * py)
    return hw::set_last_error(HW_ERR_ARG, "hw_dd_partition: every block needs at least 2 x 2 nodes");
  if (g->bc_x < 0 || g->bc_x > 2 || g->bc_y < 0 || g->bc_y > 2)
    return hw::set_last_error(HW_ERR_ARG, "hw_dd_partition: bad boundary condition");
  const int bx = part % px, by = part / px;
  auto split = [](int n, int p, int b, int& start, int& len) {
    const int q = n / p, r = n % p;
    len = q + (b < r ? 1 : 0);
    start = b * q + std::min(b, r);
  };
  hw_part_info& o = *out;
  split(g->nx, px, bx, o.i0, o.nx);
  split(g->ny, py, by, o.j0, o.ny);
  const int bcs[4] = {g->bc_x, g->bc_x, g->bc_y, g->bc_y};
  const bool edge[4] = {bx == 0, bx == px - 1, by == 0, by == py - 1};
  const int nb[4] = {((bx + px - 1) % px) + px * by, ((bx + 1) % px) + px * by, bx + px * ((by + py - 1) % py),
                     bx + px * ((by + 1) % py)};
  for (int f = 0; f < 4; ++f) {
    if (!edge[f] || bcs[f] == HW_BC_PERIODIC) {
      o.mode[f] = HW_HALO_NEIGHBOR;
      o.nbr[f] = nb[f];
    } else {
      o.mode[f] = bcs[f] == HW_BC_REFLECTIVE ? HW_HALO_MIRROR : HW_HALO_REPLICATE;
      o.nbr[f] = part;
    }
  }
  return HW_OK;
}

int hw_dd_max_keys(const unsigned long long* keys, int n, unsigned long long* out, void* cuda_stream) {
  if (!keys || !out || n < 1) return hw::set_last_error(HW_ERR_ARG, "hw_dd_max_keys: null pointer or n < 1");
  hw::k_max_keys<<<1, 32, 0, (cudaStream_t)cuda_stream>>>(keys, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hw::set_last_error(HW_ERR_CUDA, cudaGetErrorString(e));
  return HW_OK;
}

int hw_halo_strip_size(hw_solver* s, int set, int face, long long* count) {
  int rc = hw::check_halo_args(s, set, face, "hw_halo_strip_size");
  if (rc != HW_OK) return rc;
  if (!count) return hw::set_last_error(HW_ERR_ARG, "hw_halo_strip_size: null count");
  const hw::Dev2D* d = hw::part_dev(s);
  const long long len = face < 2 ? d->ny - 4 : d->nx;
  *count = (set == 1 ? 14 : 9) * 2 * len;
  return HW_OK;
}

int hw_halo_pack(hw_solver* s, int set, int face, double* strip) {
  int rc = hw::check_halo_args(s, set, face, "hw_halo_pack");
  if (rc != HW_OK) return rc;
  if (!strip) return hw::set_last_error(HW_ERR_ARG, "hw_halo_pack: null strip");
  hw::PlaneSet ps{};
  int np = 0;
  hw::part_planes(s, set, ps.p, &np);
  const hw::Dev2D* d = hw::part_dev(s);
  cudaStream_t st = hw::solver_stream(s);
  const long long len = face < 2 ? d->ny - 4 : d->nx;
  hw::k_halo_pack<<<hw::blocks_for(np * 2 * len), 256, 0, st>>>(ps, np, d->nx, d->ny, face, strip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hw::set_last_error(HW_ERR_CUDA, cudaGetErrorString(e));
  return HW_OK;
}

int hw_halo_unpack(hw_solver* s, int set, int face, int mode, const double* strip) {
  int rc = hw::check_halo_args(s, set, face, "hw_halo_unpack");
  if (rc != HW_OK) return rc;
  if (!strip) return hw::set_last_error(HW_ERR_ARG, "hw_halo_unpack: null strip");
  if (mode < HW_HALO_NEIGHBOR || mode > HW_HALO_REPLICATE) return hw::set_last_error(HW_ERR_ARG, "hw_halo_unpack: bad mode");
  hw::PlaneSet ps{};
  int np = 0;
  hw::part_planes(s, set, ps.p, &np);
  const hw::Dev2D* d = hw::part_dev(s);
  cudaStream_t st = hw::solver_stream(s);
  const long long len = face < 2 ? d->ny - 4 : d->nx;
  const unsigned odd = face < 2 ? hw::kOddX : hw::kOddY;
  hw::k_halo_unpack<<<hw::blocks_for(np * 2 * len), 256, 0, st>>>(ps, np, d->nx, d->ny, face, mode, odd, strip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hw::set_last_error(HW_ERR_CUDA, cudaGetErrorString(e));
  return HW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// All blocks on one GPU
// ---------------------------------------------------------------------------------------------
struct hw_dd {
  hw_grid grid{};
  hw_params params{};
  int px = 0, py = 0, np = 0;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::vector<hw_solver*> parts;
  std::vector<hw_part_info> info;
  std::vector<double*> strips;  // [part][face], sized for set 1
  unsigned long long* keys = nullptr;  // [np][2] block keys, then the 2 global keys
  double* tmp[9] = {};                 // export scratch of one extended block
  std::vector<void*> allocs;
  bool inited = false;
  cudaGraphExec_t graph = nullptr;
  double graph_t_end = -1.0;
  // every block launches on its own stream, forked from and joined back to the main stream around the
  // blocks' alpha and stage phases, so the blocks' kernels overlap (in a captured graph: parallel branches)
  std::vector<cudaStream_t> pstream;
  std::vector<cudaEvent_t> pevent;
  cudaEvent_t fork_ev = nullptr;
};

namespace {

int dd_fail(int code, const std::string& msg) { return hw::set_last_error(code, msg.c_str()); }

#define DD_OK(call)                                                            \
  do {                                                                         \
    int rc_ = (call);                                                          \
    if (rc_ != HW_OK) return rc_;                                              \
  } while (0)
#define DD_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return dd_fail(HW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int dd_alloc(hw_dd* d, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return dd_fail(HW_ERR_NOMEM, std::string("hw_dd: cudaMalloc: ") + cudaGetErrorString(e));
  d->allocs.push_back(*p);
  return HW_OK;
}

hw::PlaneSet plane_set(double* const* planes, int nplanes) {
  hw::PlaneSet ps{};
  for (int q = 0; q < nplanes; ++q) ps.p[q] = planes[q];
  return ps;
}

int dd_exchange(hw_dd* d, int set, cudaStream_t st);

// The blocks' streams wait for the main stream ...
int dd_fork(hw_dd* d, cudaStream_t st) {
  DD_CUDA(cudaEventRecord(d->fork_ev, st));
  for (cudaStream_t ps : d->pstream) DD_CUDA(cudaStreamWaitEvent(ps, d->fork_ev, 0));
  return HW_OK;
}
// ... and the main stream for every block's stream.
int dd_join(hw_dd* d, cudaStream_t st) {
  for (int p = 0; p < d->np; ++p) {
    DD_CUDA(cudaEventRecord(d->pevent[p], d->pstream[p]));
    DD_CUDA(cudaStreamWaitEvent(st, d->pevent[p], 0));
  }
  return HW_OK;
}

// One SSP-RK3 step of every block (dt from the CFL step at the step's start, clipped to t_end): per stage
// the exchange on the main stream, the blocks' alpha keys on their streams, the maximum on the main
// stream, the blocks' stages on their streams. On entry and on return every block's work is ordered
// before the main stream's.
int dd_step(hw_dd* d, cudaStream_t st, double t_end) {
  for (int k = 1; k <= 3; ++k) {
    DD_OK(dd_exchange(d, 0, st));
    DD_OK(dd_fork(d, st));
    for (int p = 0; p < d->np; ++p) DD_OK(hw_part_alpha_keys(d->parts[p], d->keys + 2 * p));
    DD_OK(dd_join(d, st));
    hw::k_max_keys<<<1, 32, 0, st>>>(d->keys, d->np, d->keys + 2 * d->np);
    DD_OK(dd_fork(d, st));
    for (int p = 0; p < d->np; ++p) DD_OK(hw_part_stage(d->parts[p], k, d->keys + 2 * d->np, t_end));
    DD_OK(dd_join(d, st));
  }
  DD_CUDA(cudaGetLastError());
  return HW_OK;
}

// every block's stream drained after the main stream (before host reads through a block's stream)
int dd_drain(hw_dd* d) {
  DD_CUDA(cudaStreamSynchronize(d->stream));
  for (cudaStream_t ps : d->pstream) DD_CUDA(cudaStreamSynchronize(ps));
  return HW_OK;
}

}  // namespace

namespace hw {

int dd_fork_blocks(hw_dd* d, cudaStream_t st) { return dd_fork(d, st); }
int dd_join_blocks(hw_dd* d, cudaStream_t st) { return dd_join(d, st); }

int dd_blocks(hw_dd* d, int* np, hw_solver* const** parts, const hw_part_info** info, cudaStream_t* st,
              const hw_grid** grid) {
  if (!d) return set_last_error(HW_ERR_ARG, "null block decomposition");
  *np = d->np;
  *parts = d->parts.data();
  *info = d->info.data();
  *st = d->stream;
  *grid = &d->grid;
  return HW_OK;
}

int dd_exchange_planes(hw_dd* d, double* const* const* planes, int nplanes, unsigned oddx, unsigned oddy,
                       cudaStream_t st) {
  if (nplanes < 1 || nplanes > 14) return set_last_error(HW_ERR_ARG, "dd_exchange_planes: 1..14 planes");
  for (int phase = 0; phase < 2; ++phase) {
    for (int p = 0; p < d->np; ++p) {
      const int nxe = d->info[p].nx + 4, nye = d->info[p].ny + 4;
      for (int f = 2 * phase; f < 2 * phase + 2; ++f) {
        const long long len = f < 2 ? nye - 4 : nxe;
        k_halo_pack<<<blocks_for(nplanes * 2 * len), 256, 0, st>>>(plane_set(planes[p], nplanes), nplanes, nxe, nye,
                                                                    f, d->strips[4 * p + f]);
      }
    }
    for (int p = 0; p < d->np; ++p) {
      const int nxe = d->info[p].nx + 4, nye = d->info[p].ny + 4;
      for (int f = 2 * phase; f < 2 * phase + 2; ++f) {
        const int mode = d->info[p].mode[f];
        const int src = mode == HW_HALO_NEIGHBOR ? 4 * d->info[p].nbr[f] + (f ^ 1) : 4 * p + f;
        const long long len = f < 2 ? nye - 4 : nxe;
        k_halo_unpack<<<blocks_for(nplanes * 2 * len), 256, 0, st>>>(plane_set(planes[p], nplanes), nplanes, nxe, nye,
                                                                      f, mode, f < 2 ? oddx : oddy, d->strips[src]);
      }
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HW_OK : set_last_error(HW_ERR_CUDA, cudaGetErrorString(e));
}

int dd_exchange_adjoint(hw_dd* d, double* const* const* planes, int nplanes, unsigned oddx, unsigned oddy,
                        cudaStream_t st) {
  if (nplanes < 1 || nplanes > 14) return set_last_error(HW_ERR_ARG, "dd_exchange_adjoint: 1..14 planes");
  for (int phase = 1; phase >= 0; --phase) {  // the reverse order of the exchange: y faces, then x faces
    for (int p = 0; p < d->np; ++p) {
      const int nxe = d->info[p].nx + 4, nye = d->info[p].ny + 4;
      for (int f = 2 * phase; f < 2 * phase + 2; ++f) {
        const long long len = f < 2 ? nye - 4 : nxe;
        k_halo_adj_pack<<<blocks_for(nplanes * 2 * len), 256, 0, st>>>(plane_set(planes[p], nplanes), nplanes, nxe,
                                                                        nye, f, d->strips[4 * p + f]);
      }
    }
    for (int p = 0; p < d->np; ++p)
      for (int f = 2 * phase; f < 2 * phase + 2; ++f) {
        const int mode = d->info[p].mode[f];
        // the ring of face f of block p was read from block q's nodes next to face g
        const int q = mode == HW_HALO_NEIGHBOR ? d->info[p].nbr[f] : p;
        const int g = mode == HW_HALO_NEIGHBOR ? (f ^ 1) : f;
        const int nxe = d->info[q].nx + 4, nye = d->info[q].ny + 4;
        const long long len = g < 2 ? nye - 4 : nxe;
        k_halo_adj_add<<<blocks_for(nplanes * 2 * len), 256, 0, st>>>(plane_set(planes[q], nplanes), nplanes, nxe, nye,
                                                                       g, mode, g < 2 ? oddx : oddy,
                                                                       d->strips[4 * p + f]);
      }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HW_OK : set_last_error(HW_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace hw

namespace hw {
static int halo_launch_done() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HW_OK : set_last_error(HW_ERR_CUDA, cudaGetErrorString(e));
}
int halo_pack_planes(double* const* planes, int np, int nxe, int nye, int face, double* strip, cudaStream_t st) {
  const long long len = face < 2 ? nye - 4 : nxe;
  k_halo_pack<<<blocks_for(np * 2 * len), 256, 0, st>>>(plane_set(planes, np), np, nxe, nye, face, strip);
  return halo_launch_done();
}
int halo_unpack_planes(double* const* planes, int np, int nxe, int nye, int face, int mode, unsigned odd,
                       const double* strip, cudaStream_t st) {
  const long long len = face < 2 ? nye - 4 : nxe;
  k_halo_unpack<<<blocks_for(np * 2 * len), 256, 0, st>>>(plane_set(planes, np), np, nxe, nye, face, mode, odd, strip);
  return halo_launch_done();
}
int halo_adj_pack_planes(double* const* planes, int np, int nxe, int nye, int face, double* strip, cudaStream_t st) {
  const long long len = face < 2 ? nye - 4 : nxe;
  k_halo_adj_pack<<<blocks_for(np * 2 * len), 256, 0, st>>>(plane_set(planes, np), np, nxe, nye, face, strip);
  return halo_launch_done();
}
int halo_adj_add_planes(double* const* planes, int np, int nxe, int nye, int face, int mode, unsigned odd,
                        const double* strip, cudaStream_t st) {
  const long long len = face < 2 ? nye - 4 : nxe;
  k_halo_adj_add<<<blocks_for(np * 2 * len), 256, 0, st>>>(plane_set(planes, np), np, nxe, nye, face, mode, odd, strip);
  return halo_launch_done();
}
}  // namespace hw

namespace {
// One exchange of plane set 0 (state) or 1 (state and static planes) on the main stream.
int dd_exchange(hw_dd* d, int set, cudaStream_t st) {
  std::vector<double*> pl(14 * (size_t)d->np);
  std::vector<double* const*> pp(d->np);
  int nplanes = 0;
  for (int p = 0; p < d->np; ++p) {
    hw::part_planes(d->parts[p], set, pl.data() + 14 * (size_t)p, &nplanes);
    pp[p] = pl.data() + 14 * (size_t)p;
  }
  return hw::dd_exchange_planes(d, pp.data(), nplanes, hw::kOddX, hw::kOddY, st);
}
}  // namespace

extern "C" {

int hw_dd_destroy(hw_dd* d) {
  if (!d) return HW_OK;
  if (d->graph) cudaGraphExecDestroy(d->graph);
  if (d->stream) cudaStreamSynchronize(d->stream);
  else cudaDeviceSynchronize();
  for (hw_solver* s : d->parts) hw_destroy(s);
  for (void* p : d->allocs) cudaFree(p);
  for (cudaStream_t ps : d->pstream) cudaStreamDestroy(ps);
  for (cudaEvent_t e : d->pevent) cudaEventDestroy(e);
  if (d->fork_ev) cudaEventDestroy(d->fork_ev);
  if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
  delete d;
  return HW_OK;
}

int hw_dd_create(const hw_grid* grid, const hw_params* params, int px, int py, void* cuda_stream, hw_dd** out) {
  if (!grid || !params || !out) return dd_fail(HW_ERR_ARG, "hw_dd_create: null argument");
  *out = nullptr;
  hw_part_info probe{};
  DD_OK(hw_dd_partition(grid, px, py, 0, &probe));
  hw_dd* d = new hw_dd();
  d->grid = *grid;
  d->params = *params;
  d->px = px;
  d->py = py;
  d->np = px * py;
  d->stream = (cudaStream_t)cuda_stream;
  int rc = HW_OK;
  size_t max_ext = 0;
  for (int p = 0; p < d->np && rc == HW_OK; ++p) {
    cudaStream_t ps = nullptr;
    cudaEvent_t pe = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) d->pstream.push_back(ps);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pe, cudaEventDisableTiming);
    if (e == cudaSuccess) d->pevent.push_back(pe);
    if (e != cudaSuccess) { rc = dd_fail(HW_ERR_CUDA, cudaGetErrorString(e)); break; }
    hw_solver* s = nullptr;
    rc = hw_part_create(grid, params, px, py, p, ps, &s);
    if (rc != HW_OK) break;
    d->parts.push_back(s);
    d->info.push_back(*hw::part_info(s));
    const hw_part_info& pi = d->info.back();
    max_ext = std::max(max_ext, (size_t)(pi.nx + 4) * (pi.ny + 4));
    for (int f = 0; f < 4 && rc == HW_OK; ++f) {
      long long cnt = 0;
      rc = hw_halo_strip_size(s, 1, f, &cnt);
      void* q = nullptr;
      if (rc == HW_OK) rc = dd_alloc(d, &q, cnt * sizeof(double));
      d->strips.push_back((double*)q);
    }
  }
  void* q = nullptr;
  if (rc == HW_OK) rc = dd_alloc(d, &q, (2 * d->np + 2) * sizeof(unsigned long long));
  d->keys = (unsigned long long*)q;
  for (int c = 0; c < 9 && rc == HW_OK; ++c) {
    rc = dd_alloc(d, &q, max_ext * sizeof(double));
    d->tmp[c] = (double*)q;
  }
  if (rc == HW_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { d->cap_stream = nullptr; rc = dd_fail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  }
  if (rc == HW_OK) {
    cudaError_t e = cudaEventCreateWithFlags(&d->fork_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { d->fork_ev = nullptr; rc = dd_fail(HW_ERR_CUDA, cudaGetErrorString(e)); }
  }
  if (rc != HW_OK) {
    hw_dd_destroy(d);
    return rc;
  }
  *out = d;
  return HW_OK;
}

int hw_dd_init(hw_dd* d, const double* h, const double* hu, const double* hv, const double* b,
               const double* const* deriv, int ptr_kind) {
  if (!d || !h || !hu || !hv || !b || !deriv) return dd_fail(HW_ERR_ARG, "hw_dd_init: null argument");
  const double* in[12] = {h, hu, hv, b, deriv[0], deriv[1], deriv[2], deriv[3], deriv[4], deriv[5], deriv[6], deriv[7]};
  for (int q = 0; q < 12; ++q)
    if (!in[q]) return dd_fail(HW_ERR_ARG, "hw_dd_init: null plane");
  int first_err = HW_OK;
  for (int p = 0; p < d->np; ++p) {
    const hw_part_info& pi = d->info[p];
    const double* win[12];
    for (int q = 0; q < 12; ++q) win[q] = in[q] + (size_t)pi.j0 * d->grid.nx + pi.i0;
    int rc = hw_part_init(d->parts[p], win, d->grid.nx, ptr_kind);
    if (rc == HW_ERR_DEPTH || rc == HW_ERR_NONFINITE) { if (first_err == HW_OK) first_err = rc; }
    else if (rc != HW_OK) return rc;
  }
  DD_OK(dd_exchange(d, 1, d->stream));
  DD_CUDA(cudaStreamSynchronize(d->stream));
  for (int p = 0; p < d->np; ++p) DD_OK(hw_part_finish_init(d->parts[p]));
  d->inited = true;
  if (first_err != HW_OK) return dd_fail(first_err, "hw_dd_init: non-positive or non-finite depth in the input");
  return HW_OK;
}

int hw_dd_advance(hw_dd* d, int nsteps, double t_end, int use_graph, double* t_out, int* steps_out) {
  if (!d) return dd_fail(HW_ERR_ARG, "hw_dd_advance: null argument");
  if (!d->inited) return dd_fail(HW_ERR_STATE, "hw_dd_advance: call hw_dd_init first");
  if (nsteps < 0) return dd_fail(HW_ERR_ARG, "hw_dd_advance: nsteps < 0");
  double t0 = 0.0, t = 0.0;
  long long n0 = 0, n1 = 0;
  DD_OK(dd_drain(d));
  DD_OK(hw_get_time(d->parts[0], &t0, &n0));
  const bool has_end = t_end > 0.0;
  // a graph holds two steps (six stages: every block's state buffer returns to where it was)
  if (use_graph && (!d->graph || d->graph_t_end != t_end) && hw::solver_cur(d->parts[0]) == 0) {
    if (d->graph) { cudaGraphExecDestroy(d->graph); d->graph = nullptr; }
    DD_OK(dd_drain(d));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = HW_OK;
    if (e == cudaSuccess) {
      rc = dd_step(d, d->cap_stream, t_end);
      if (rc == HW_OK) rc = dd_step(d, d->cap_stream, t_end);
      e = cudaStreamEndCapture(d->cap_stream, &g);
    }
    if (rc != HW_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return dd_fail(HW_ERR_CUDA, std::string("hw_dd_advance: capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&d->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { d->graph = nullptr; return dd_fail(HW_ERR_CUDA, std::string("hw_dd_advance: instantiate: ") + cudaGetErrorString(e)); }
    d->graph_t_end = t_end;
  }
  const int chunk = has_end ? 2 : 1 << 30;
  int done = 0;
  t = t0;
  while (done < nsteps) {
    if (has_end && t >= t_end) break;
    int todo = std::min(nsteps - done, chunk);
    while (todo > 0) {
      if (use_graph && d->graph && hw::solver_cur(d->parts[0]) == 0 && todo >= 2) {
        DD_CUDA(cudaGraphLaunch(d->graph, d->stream));
        todo -= 2;
        done += 2;
      } else {
        DD_OK(dd_step(d, d->stream, t_end));
        todo -= 1;
        done += 1;
      }
    }
    if (has_end) {
      DD_OK(dd_drain(d));
      DD_OK(hw_get_time(d->parts[0], &t, &n1));
    }
  }
  DD_OK(dd_drain(d));
  int rc = HW_OK;
  for (hw_solver* s : d->parts) {
    int r = hw_sync(s);
    if (r != HW_OK && rc == HW_OK) rc = r;
  }
  DD_OK(hw_get_time(d->parts[0], &t, &n1));
  if (t_out) *t_out = t - t0;
  if (steps_out) *steps_out = (int)(n1 - n0);
  return rc;
}

int hw_dd_get_state(hw_dd* d, double* const* out, int layout, int ptr_kind) {
  if (!d || !out) return dd_fail(HW_ERR_ARG, "hw_dd_get_state: null argument");
  if (!d->inited) return dd_fail(HW_ERR_STATE, "hw_dd_get_state: call hw_dd_init first");
  if (ptr_kind != HW_HOST && ptr_kind != HW_DEVICE) return dd_fail(HW_ERR_ARG, "hw_dd_get_state: bad ptr_kind");
  for (int q = 0; q < 9; ++q)
    if (!out[q]) return dd_fail(HW_ERR_ARG, "hw_dd_get_state: null plane");
  const cudaMemcpyKind kind = ptr_kind == HW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  DD_OK(dd_drain(d));
  for (int p = 0; p < d->np; ++p) {
    const hw_part_info& pi = d->info[p];
    DD_OK(hw_get_state(d->parts[p], d->tmp, layout, HW_DEVICE));  // on the block's stream
    const int nxe = pi.nx + 4;
    for (int q = 0; q < 9; ++q)
      DD_CUDA(cudaMemcpy2DAsync(out[q] + (size_t)pi.j0 * d->grid.nx + pi.i0, d->grid.nx * sizeof(double),
                                d->tmp[q] + 2 * (size_t)nxe + 2, nxe * sizeof(double), pi.nx * sizeof(double), pi.ny,
                                kind, d->pstream[p]));
    DD_CUDA(cudaStreamSynchronize(d->pstream[p]));  // d->tmp is reused by the next block
  }
  return HW_OK;
}

}  // extern "C"
