// mdf_step_walls16.cu -- the batched wall and power-law march
// (mdf_walls.cuh) with 16-bit storage: FP32 u, v, P plus FP16 or BF16
// non-equilibrium pairs, FP32 arithmetic, rolled form.
#include "mdf_walls.cuh"

namespace mdf {

cudaError_t walls_batch_occupancy16(int metric, int power_law, int storage, int *occ, int *smem) {
    if (storage == STORAGE_BF16) {
        MDF_WALLS_DISPATCH_ST(kWallsBatchNT, STORAGE_BF16, batch_occupancy_t, occ, smem)
    }
    MDF_WALLS_DISPATCH_ST(kWallsBatchNT, STORAGE_FP16, batch_occupancy_t, occ, smem)
}

cudaError_t walls_batch_launch16(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps,
                                 int metric, int power_law, int grid, int forced, int roll, int storage,
                                 cudaStream_t stream) {
    if (storage == STORAGE_BF16) {
        MDF_WALLS_DISPATCH_ST(kWallsBatchNT, STORAGE_BF16, batch_launch_t, items, nitems, args, maps, grid, forced,
                              roll, stream)
    }
    MDF_WALLS_DISPATCH_ST(kWallsBatchNT, STORAGE_FP16, batch_launch_t, items, nitems, args, maps, grid, forced, roll,
                          stream)
}

}  // namespace mdf
