// mdf_step_walls.cu -- the wall and power-law march (mdf_walls.cuh) with
// FP32 storage, and the entry points that pick the storage mode's batched
// instantiation (16-bit ones in mdf_step_walls16.cu).
#include "mdf_walls.cuh"

namespace mdf {

bool walls_path_applies(int metric, int power_law, int walls, int storage) {
    return metric != METRIC_CURVILINEAR && storage == STORAGE_FP32 && (power_law || walls);
}

cudaError_t walls_occupancy(int metric, int power_law, int nt, int *occ, int *smem) {
    if (nt == 256) {
        MDF_WALLS_DISPATCH(256, occupancy_t, occ, smem)
    }
    MDF_WALLS_DISPATCH(128, occupancy_t, occ, smem)
}

cudaError_t walls_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                         cudaStream_t stream) {
    if (plan.NT == 256) return launch_nt<256>(tmap, args, metric, plan, stream);
    return launch_nt<128>(tmap, args, metric, plan, stream);
}

cudaError_t walls_batch_occupancy(int metric, int power_law, int storage, int *nt, int *occ, int *smem) {
    *nt = kWallsBatchNT;
    if (storage != STORAGE_FP32) return walls_batch_occupancy16(metric, power_law, storage, occ, smem);
    MDF_WALLS_DISPATCH_ST(kWallsBatchNT, STORAGE_FP32, batch_occupancy_t, occ, smem)
}

cudaError_t walls_batch_launch(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps,
                               int metric, int power_law, int grid, int forced, int roll, int storage,
                               cudaStream_t stream) {
    if (storage != STORAGE_FP32)
        return walls_batch_launch16(items, nitems, args, maps, metric, power_law, grid, forced, roll, storage, stream);
    MDF_WALLS_DISPATCH_ST(kWallsBatchNT, STORAGE_FP32, batch_launch_t, items, nitems, args, maps, grid, forced, roll,
                          stream)
}

}  // namespace mdf
