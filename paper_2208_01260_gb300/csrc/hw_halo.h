// Halo strips of explicit plane sets of one block (extended size nxe x nye; the strip layout of
// hw_halo_pack: [plane][ring offset 0, 1][position along the face]): the forward copy and its transpose,
// for the per-block adjoint of the multi-process decomposition (hw_adjoint.cu). Kernels in hw_dd.cu.
#pragma once
#include <cuda_runtime.h>

namespace hw {
int halo_pack_planes(double* const* planes, int np, int nxe, int nye, int face, double* strip, cudaStream_t st);
int halo_unpack_planes(double* const* planes, int np, int nxe, int nye, int face, int mode, unsigned odd,
                       const double* strip, cudaStream_t st);
// the ring's values of a face into the strip, the ring cleared
int halo_adj_pack_planes(double* const* planes, int np, int nxe, int nye, int face, double* strip, cudaStream_t st);
// a strip added to the nodes its ring was copied from (the strip of the opposite face of a NEIGHBOR, or the
// block's own face for MIRROR / REPLICATE)
int halo_adj_add_planes(double* const* planes, int np, int nxe, int nye, int face, int mode, unsigned odd,
                        const double* strip, cudaStream_t st);
}  // namespace hw
