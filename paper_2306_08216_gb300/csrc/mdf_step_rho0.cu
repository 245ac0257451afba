// mdf_step_rho0.cu -- the fused step with the alpha = 0 distribution of
// Eq. 2.1.2 (ubar_0 = rho_0, E_0 = 0, source w_j R) evolved beside
// alpha = 1, 2: the shared-ring march of mdf_march.cuh with its scalar lane
// enabled, for every grid kind, wall type and fluid model (periodic
// Newtonian problems on uniform and separable grids also have the
// register-window march of mdf_step_fast.cu with the lane).  The lane reads
// the velocity of the alpha = 1, 2 moments of the same stage and writes
// planes 10..14; nothing flows back (Remark 1), so the alpha = 1, 2 results
// are those of the step without it.
#include "mdf_march.cuh"

namespace mdf {

cudaError_t rho0_occupancy(int metric, int power_law, int walls, int *occ, int *smem) {
    MDF_MARCH_DISPATCH(true, occupancy_t, occ, smem)
}

cudaError_t rho0_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                        cudaStream_t stream) {
    const int power_law = args.power_law;
    const int walls = (args.xwall || args.ywall) ? 1 : 0;
    MDF_MARCH_DISPATCH(true, launch_t, tmap, args, plan, stream)
}

}  // namespace mdf
