// mdf_internal.cuh -- declarations shared by the translation units of
// libmdf.so (the fused MDF-FDLBM step, its auxiliary kernels and the host
// runtime).  Nothing here is part of the public C ABI (include/mdf.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace mdf {

// Storage: each of the 10 planes fhat_{alpha,j} (plane k = 5 alpha + j) is
// ny rows of `pitch` floats; node (x, y) lives at column GHOST + x.  The
// GHOST columns on each side hold periodic images on a periodic x axis
// (written by the step that produces the plane) and are unused otherwise.
constexpr int GHOST = 4;
constexpr int NPLANES = 10;
constexpr int RHO0_PLANES = 15;  // with the alpha = 0 distribution: planes 10..14 = fhat_{j,0}

enum MetricKind { METRIC_UNIFORM = 0, METRIC_SEPARABLE = 1, METRIC_CURVILINEAR = 2 };

// State storage.  STORAGE_FP32: 10 FP32 planes fhat_{alpha,j}.  The 16-bit
// modes keep the macroscopic fields exact and round only the small
// non-equilibrium part n = fhat - feq(u, v, P): 7 planes of 32-bit words,
// u, v, P in FP32 followed by, for j = 1..4, the pair word of S n_{u,j}
// (low half) and S n_{v,j} (high half) in FP16 or BF16;
// n_{alpha,0} = -(n_1 + n_2 + n_3 + n_4).  The scale S = 2^(12 - floor(log2
// c)) is a power of two (exact both ways) that lifts n, a few orders of
// magnitude below c, out of the FP16 subnormal range while keeping
// |S n| < 65504 for |n| up to about 16 c.
enum StorageKind { STORAGE_FP32 = 0, STORAGE_FP16 = 1, STORAGE_BF16 = 2 };
constexpr int DEV_FPLANES = 3;  // u, v, P
constexpr int DEV_PLANES = 7;   // plus 4 pair planes
constexpr int NSCALE_EXP = 12;

// 32-bit planes of one state buffer (FP32 storage with the alpha = 0
// distribution: 15 planes).
__host__ __device__ inline int state_planes(int storage, int rho0 = 0) {
    return storage == STORAGE_FP32 ? (rho0 ? RHO0_PLANES : NPLANES) : DEV_PLANES;
}
inline size_t state_buffer_bytes(int storage, long long plane, int rho0 = 0) {
    return (size_t)state_planes(storage, rho0) * plane * 4;
}

// One-time per-kernel launch setup (the dynamic shared-memory attribute) is
// a property of each device: a launcher keeps a bitmask of the devices
// (0..63) it has set up and redoes the setup on a device it has not seen.
// The mask is atomic, so contexts on different host threads may launch
// concurrently; two threads may both set a kernel up, which is harmless.
inline bool needs_device_setup(const std::atomic<unsigned long long> &mask) {
    int d = 0;
    cudaGetDevice(&d);
    return d >= 64 || !((mask.load(std::memory_order_acquire) >> d) & 1ull);
}
inline void mark_device_setup(std::atomic<unsigned long long> &mask) {
    int d = 0;
    cudaGetDevice(&d);
    if (d < 64) mask.fetch_or(1ull << d, std::memory_order_release);
}

// Error codes the kernels raise in StepArgs::err (first one wins):
// a bounded TMA wait that gave up, or (debug build, -DMDF_DEBUG) a global
// access outside its buffer, which is skipped instead of made.
enum DeviceError { DEVERR_NONE = 0, DEVERR_TMA_TIMEOUT = 1, DEVERR_INDEX = 2 };

struct StepArgs {
    float *fout;            // output state (same layout as the input)
    const float *fin;       // input state (the tile kernel reads it with plain loads; the marches use TMA)
    int storage;            // StorageKind of both state buffers
    int rho0;               // the buffers also hold the alpha = 0 distribution
    float nscale, ninv;     // 16-bit storage: S and 1/S
    int nx, ny, pitch;      // nodes, row pitch in floats
    long long plane;        // floats per plane (pitch * ny)
    int W, H;               // output columns / rows per block
    int xwall, ywall;       // 1: NEE walls on that axis, 0: periodic
    float c, inv2c;         // lattice speed, 1/(2c)
    float dt, h;            // time step and half step
    // mixed-scheme weights (Eqs. 2.2.12-2.2.13) on unit spacing, for a
    // population moving in +chi: a1 Pi(+1) + a0 Pi(0) + am1 Pi(-1) + am2 Pi(-2)
    float a1, a0, am1, am2;
    // uniform grid: c/dx and c/dy
    float kx, ky;
    // separable grid: c xi_x per column (padded layout) and c eta_y per row
    const float *kxv, *kyv;
    // curvilinear grid: c xi_x, c xi_y, c eta_x, c eta_y planes (padded layout)
    const float *mxx, *mxy, *mex, *mey;
    // Newtonian rates: eigenvalues (free, first-moment) of
    // I - Lambda (fhat^+), I - 3 Lambda/4 (fbar^+), (I + h/2 Lt)^-1 (recovery)
    float rpp, rp, rbp, rb, rkp, rk;
    // power-law fluid
    int power_law;
    float K, n_index, nu_min, nu_max, cs2, s_ratio, a_pl;  // a_pl = cs2 dt / 2
    float lnK, ln_nu_min, ln_nu_max, inv_n;                  // ln K, ln nu_min, ln nu_max, 1/n
    // body force: F for the h step (Eq. 2.3.25); F + dt/2 dF/dt for the dt
    // step (Eq. 2.3.24), mode 0 none, 1 constant, 2 padded field
    int force_mode;
    float Fx, Fy;
    const float *Fxp, *Fyp;  // padded layout
    int force_mode_d;
    float Fxd, Fyd;
    const float *Fxdp, *Fydp;
    // source R of Eq. 2.1.1 (mode 0 none, 1 constant Rc, 2 padded field Rp)
    // and its pressure factors (Eq. 2.3.23) for fhat and fbar
    int r_mode;
    float Rc, rk_hat, rk_bar;
    const float *Rp;
    // wall velocities (west, east, south, north)
    float uw[4], vw[4];
    int *err;
    // Packed (x, x) pairs of the constants above for the f32x2 fast path:
    // difference weights -h k a and -dt k a of each axis (uniform grids),
    // the relaxation increments -(1 - A') and (A - A')/2 of the three maps,
    // and the source factors h/5, dt/5.
    unsigned long long pwxh[3], pwxd[3], pwyh[3], pwyd[3];
    unsigned long long pmKp, pDp, pmKb, pDb, pmKk, pDk, phw, pdw;
};

// Pair (x, x) as the 64-bit pattern the f32x2 instructions read.
inline unsigned long long pack_pair(float x) {
    union {
        float f[2];
        unsigned long long u;
    } v;
    v.f[0] = x;
    v.f[1] = x;
    return v.u;
}

// Fused step kernel launcher (mdf_step.cu).
struct StepPlan {
    int kind;     // PLAN_MARCH or PLAN_TILE
    int NT;       // threads per block
    int W, H;     // output columns / rows per block
    int gx, gy;   // grid
    int smem;     // dynamic shared memory bytes
    int occ;      // resident blocks per SM
};

enum PlanKind { PLAN_MARCH = 0, PLAN_TILE = 1 };
constexpr int TILE_X = 16, TILE_Y = 16;  // output tile of the tile kernel (halo of 4 on each side)

// Candidate launch plans of the fused step (the first one is the default);
// returns how many were written to out[0..max).
int step_candidates(int metric, int power_law, int walls, int storage, int rho0, int nx, int ny, int num_sms,
                    StepPlan *out, int max, cudaError_t *err);
cudaError_t step_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                        cudaStream_t stream);
int step_pitch(int nx, int W);

// Batched step: one work item = one block's march (strip bx, band by) of one
// problem of the batch (mdf_step.cu).
struct BatchItem {
    int problem, bx, by, pad;
};
// storage: the batch's storage mode (16-bit: uniform and separable grids
// only, rolled form).  roll: the rolled form of the register-window march
// (uniform and separable grids; ignored on curvilinear grids).
cudaError_t batch_occupancy(int metric, int power_law, int walls, int storage, int *nt, int *occ, int *smem);
cudaError_t batch_launch(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps, int metric,
                         int power_law, int walls, int grid, int forced, int roll, int storage, cudaStream_t stream);

// Walls and/or power law on uniform/separable grids, FP32 storage, in the
// register-window form of the fast path (mdf_step_walls.cu).
bool walls_path_applies(int metric, int power_law, int walls, int storage);
cudaError_t walls_occupancy(int metric, int power_law, int nt, int *occ, int *smem);
cudaError_t walls_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                         cudaStream_t stream);
cudaError_t walls_batch_occupancy(int metric, int power_law, int storage, int *nt, int *occ, int *smem);
cudaError_t walls_batch_launch(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps,
                               int metric, int power_law, int grid, int forced, int roll, int storage,
                               cudaStream_t stream);
// The 16-bit batched wall march (FP16/BF16 storage, rolled form only).
cudaError_t walls_batch_occupancy16(int metric, int power_law, int storage, int *occ, int *smem);
cudaError_t walls_batch_launch16(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps,
                                 int metric, int power_law, int grid, int forced, int roll, int storage,
                                 cudaStream_t stream);

// The shared-ring march with the alpha = 0 distribution (planes 10..14) on
// every grid kind, FP32 storage (mdf_step_rho0.cu).
cudaError_t rho0_occupancy(int metric, int power_law, int walls, int *occ, int *smem);
cudaError_t rho0_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                        cudaStream_t stream);

// One block per 2-D tile of output nodes, three phases per step, for grids
// too small for marching bands (mdf_step_tile.cu, mdf_step_tile16.cu,
// mdf_step_tile_rho0.cu); every storage mode, and the alpha = 0
// distribution with FP32 storage.  It is also the only kernel for 16-bit
// storage outside the periodic fast path.
bool tile_path_applies(int storage, int rho0);
cudaError_t tile_occupancy(int metric, int power_law, int walls, int storage, int rho0, int *tx, int *ty, int *occ,
                           int *smem);
cudaError_t tile_launch(const StepArgs &args, int metric, const StepPlan &plan, cudaStream_t stream);
// The same kernel over the work items (problem, tile x, tile y) of a batch.
cudaError_t tile_batch_occupancy(int metric, int power_law, int walls, int storage, int *occ, int *smem);
cudaError_t tile_batch_launch(const BatchItem *items, int nitems, const StepArgs *args, int metric, int power_law,
                              int walls, int storage, int grid, cudaStream_t stream);

// Periodic Newtonian fast path on uniform/separable grids (mdf_step_fast.cu).
bool fast_path_applies(int metric, int power_law, int walls);
cudaError_t fast_occupancy(int metric, int storage, int rho0, int nt, int *occ, int *smem);
cudaError_t fast_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                        cudaStream_t stream);

}  // namespace mdf
