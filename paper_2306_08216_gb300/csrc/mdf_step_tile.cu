// mdf_step_tile.cu -- the tile kernel (mdf_tile.cuh) with FP32 storage, and
// the entry points that pick the storage mode's instantiation.
#include "mdf_tile.cuh"

namespace mdf {

MDF_TILE_DEFINE(STORAGE_FP32)

// Every storage mode; the alpha = 0 distribution with FP32 storage.
bool tile_path_applies(int storage, int rho0) { return !rho0 || storage == STORAGE_FP32; }

cudaError_t tile_occupancy(int metric, int power_law, int walls, int storage, int rho0, int *tx, int *ty, int *occ,
                           int *smem) {
    *tx = kTX;
    *ty = kTY;
    if (rho0) return tile_occupancy_rho0(metric, power_law, walls, occ, smem);
    switch (storage) {
        case STORAGE_FP16: return tile_occupancy_st<STORAGE_FP16>(metric, power_law, walls, occ, smem);
        case STORAGE_BF16: return tile_occupancy_st<STORAGE_BF16>(metric, power_law, walls, occ, smem);
        default: return tile_occupancy_st<STORAGE_FP32>(metric, power_law, walls, occ, smem);
    }
}

cudaError_t tile_launch(const StepArgs &args, int metric, const StepPlan &plan, cudaStream_t stream) {
    if (args.rho0) return tile_launch_rho0(args, metric, plan, stream);
    switch (args.storage) {
        case STORAGE_FP16: return tile_launch_st<STORAGE_FP16>(args, metric, plan, stream);
        case STORAGE_BF16: return tile_launch_st<STORAGE_BF16>(args, metric, plan, stream);
        default: return tile_launch_st<STORAGE_FP32>(args, metric, plan, stream);
    }
}

cudaError_t tile_batch_occupancy(int metric, int power_law, int walls, int storage, int *occ, int *smem) {
    switch (storage) {
        case STORAGE_FP16: return tile_batch_occupancy_st<STORAGE_FP16>(metric, power_law, walls, occ, smem);
        case STORAGE_BF16: return tile_batch_occupancy_st<STORAGE_BF16>(metric, power_law, walls, occ, smem);
        default: return tile_batch_occupancy_st<STORAGE_FP32>(metric, power_law, walls, occ, smem);
    }
}

cudaError_t tile_batch_launch(const BatchItem *items, int nitems, const StepArgs *args, int metric, int power_law,
                              int walls, int storage, int grid, cudaStream_t stream) {
    switch (storage) {
        case STORAGE_FP16:
            return tile_batch_launch_st<STORAGE_FP16>(items, nitems, args, metric, power_law, walls, grid, stream);
        case STORAGE_BF16:
            return tile_batch_launch_st<STORAGE_BF16>(items, nitems, args, metric, power_law, walls, grid, stream);
        default:
            return tile_batch_launch_st<STORAGE_FP32>(items, nitems, args, metric, power_law, walls, grid, stream);
    }
}

}  // namespace mdf
