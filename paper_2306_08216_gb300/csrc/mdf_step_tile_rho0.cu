// mdf_step_tile_rho0.cu -- the tile kernel (mdf_tile.cuh) with the alpha = 0
// distribution of Eq. 2.1.2 evolved beside alpha = 1, 2 (FP32 storage, 15
// planes): phase A relaxes fhat_{j,0} with the node's u, v and rates, phase B
// streams and recovers it with the u, v of the alpha = 1, 2 fbar (source
// h w_j R) and sets its wall nodes by NEE with the neighbour's rho_0, phase C
// streams it at dt (source dt w_j R) and writes planes 10..14.
#include "mdf_tile.cuh"

namespace mdf {

cudaError_t tile_occupancy_rho0(int metric, int power_law, int walls, int *occ, int *smem) {
    MDF_TILE_DISPATCH_RHO0(tile_occupancy_t, occ, smem)
}

cudaError_t tile_launch_rho0(const StepArgs &args, int metric, const StepPlan &plan, cudaStream_t stream) {
    const int power_law = args.power_law;
    const int walls = (args.xwall || args.ywall) ? 1 : 0;
    MDF_TILE_DISPATCH_RHO0(tile_launch_t, args, plan, stream)
}

}  // namespace mdf
