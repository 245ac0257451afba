// mdf_step_tile16.cu -- the tile kernel (mdf_tile.cuh) with the 16-bit
// deviation storage modes: each node is u, v, P in FP32 and the
// non-equilibrium parts n_1..n_4 as FP16 or BF16 pairs; phase A rebuilds
// fhat = feq(u, v, P) + n, phase C stores the moments and n of the output
// (the arithmetic is FP32 throughout).
#include "mdf_tile.cuh"

namespace mdf {

MDF_TILE_DEFINE(STORAGE_FP16)
MDF_TILE_DEFINE(STORAGE_BF16)

}  // namespace mdf
