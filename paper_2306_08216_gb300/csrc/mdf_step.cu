// mdf_step.cu -- the fused MDF-FDLBM time step for sm_103a.
//
// One launch performs one time step of Sec. 2.2, Steps (1)-(4), of
// arXiv:2306.08216 with the simplified evolution equations of Remark 2:
//   Step 1  fhat^+ = feq + (I - Lambda)(fhat - feq)             (Eq. 2.2.14)
//           fbar^+ = feq + (I - 3 Lambda/4)(fhat - feq)         (Eq. 2.2.15)
//   Step 2  fbar(t+h) = fbar^+ - h c_j.grad fbar^+ + h w_j F     (Eq. 2.3.25 / 2.2.11)
//   Step 3  f(t+h) = feq + (I + h/2 Lt)^-1 (fbar - feq)          (Eq. 2.2.16)
//   Step 4  fhat(t+dt) = fhat^+ - dt c_j.grad f(t+h)
//                        + dt w_j (F + dt/2 dF/dt)                (Eq. 2.3.24)
// This file instantiates the shared-ring march (mdf_march.cuh) for
// curvilinear grids and holds the launch planning and dispatch.  Uniform
// and separable grids run the register-window marches of mdf_step_fast.cu
// (periodic, Newtonian; also with the alpha = 0 distribution) and
// mdf_step_walls.cu (walls and/or power law); with the alpha = 0
// distribution every other grid runs mdf_step_rho0.cu.  The
// tile kernel (mdf_tile.cuh) is a candidate plan on every grid and the only
// one for 16-bit storage off the periodic fast path; the autotuner of
// mdf_create chooses between the families by timing.
// The MRT matrix of Eq. 2.2.4 with s0 = s3 = s4 = s' and s1 = s2 = s equals
// s' I + (s - s') P_c, P_c the projector on the first moments, so every
// function of it acts on a distribution through its zeroth and first moments
// only; with the D2Q5 lattice (Eq. 3.1.0) and the linear equilibrium
// (Eq. 2.2.5) each of the three local maps costs a handful of FMAs per
// population and no 5x5 product appears (cf. the 2x5x5 loop count of Sec. 4.2).
//
// The shared-ring march itself (arithmetic layout, work decomposition,
// walls) is in mdf_march.cuh.
#include "mdf_march.cuh"

namespace mdf {

namespace {

using namespace dev;

cudaError_t occupancy(int metric, int power_law, int walls, int *occ, int *smem) {
    MDF_MARCH_DISPATCH(false, occupancy_t, occ, smem)
}

}  // namespace

int step_pitch(int nx, int W) {
    const int strips = (nx + W - 1) / W;
    const int cols = strips * W + 2 * GHOST;
    return ((cols + 31) / 32) * 32;
}

// Launch geometry for block size nt and `waves` blocks per resident slot:
// a strip of nt - 8 output columns per block, bands sized so the grid fills
// every SM at the measured occupancy.  A band of H rows costs H + 9 row
// iterations (halo), and a row iteration is latency-bound, so on a grid too
// small to fill the GPU many short bands (down to 2 rows) finish sooner
// than fewer long ones (257^2 cavity: 10.7 us per step with 2-row bands,
// 15.1 us with 8-row bands).
static void fill_plan(int nt, int occ, int smem, int waves, int nx, int ny, int num_sms, StepPlan *plan) {
    plan->kind = PLAN_MARCH;
    plan->NT = nt;
    plan->W = nt - 8;
    plan->occ = occ;
    plan->smem = smem;
    plan->gx = (nx + plan->W - 1) / plan->W;
    const int slots = waves * (occ > 0 ? occ : 1) * (num_sms > 0 ? num_sms : 1);
    int bands = slots / plan->gx;
    if (bands < 1) bands = 1;
    int H = (ny + bands - 1) / bands;
    if (H < 2) H = 2;
    plan->H = H;
    plan->gy = (ny + H - 1) / H;
}

int step_candidates(int metric, int power_law, int walls, int storage, int rho0, int nx, int ny, int num_sms,
                    StepPlan *out, int max, cudaError_t *err) {
    int n = 0;
    *err = cudaSuccess;
    const bool fast = fast_path_applies(metric, power_law, walls);
    const bool wpath = !rho0 && !fast && walls_path_applies(metric, power_law, walls, storage);
    // the shared-ring march keeps FP32 storage; 16-bit storage off the fast
    // path has the tile kernel only
    const bool march = fast || wpath || storage == STORAGE_FP32;
    const int nts[2] = {128, 256};
    for (int i = 0; march && i < (fast || wpath ? 2 : 1); ++i) {
        int occ = 0, smem = 0;
        cudaError_t e = fast    ? fast_occupancy(metric, storage, rho0, nts[i], &occ, &smem)
                        : wpath ? walls_occupancy(metric, power_law, nts[i], &occ, &smem)
                        : rho0  ? rho0_occupancy(metric, power_law, walls, &occ, &smem)
                                : occupancy(metric, power_law, walls, &occ, &smem);
        if (e != cudaSuccess) {
            *err = e;
            return n;
        }
        if (occ < 1) continue;
        for (int waves = 1; waves <= 2 && n < max; ++waves) fill_plan(nts[i], occ, smem, waves, nx, ny, num_sms, &out[n++]);
    }
    // the tile kernel, last: the marches stay the default
    if (tile_path_applies(storage, rho0) && n < max) {
        int tx = 0, ty = 0, occ = 0, smem = 0;
        const cudaError_t e = tile_occupancy(metric, power_law, walls, storage, rho0, &tx, &ty, &occ, &smem);
        if (e != cudaSuccess) {
            *err = e;
            return n;
        }
        if (occ >= 1) {
            StepPlan &p = out[n++];
            p.kind = PLAN_TILE;
            p.NT = tx * ty;
            p.W = tx;
            p.H = ty;
            p.gx = (nx + tx - 1) / tx;
            p.gy = (ny + ty - 1) / ty;
            p.smem = smem;
            p.occ = occ;
        }
    }
    return n;
}

cudaError_t batch_occupancy(int metric, int power_law, int walls, int storage, int *nt, int *occ, int *smem) {
    if (metric != METRIC_CURVILINEAR) return walls_batch_occupancy(metric, power_law, storage, nt, occ, smem);
    *nt = kMarchNT;
    MDF_CURVI_DISPATCH(batch_occupancy_t, occ, smem)
}

cudaError_t batch_launch(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps, int metric,
                         int power_law, int walls, int grid, int forced, int roll, int storage, cudaStream_t stream) {
    if (metric != METRIC_CURVILINEAR)
        return walls_batch_launch(items, nitems, args, maps, metric, power_law, grid, forced, roll, storage, stream);
    MDF_CURVI_DISPATCH(batch_launch_t, items, nitems, args, maps, grid, stream)
}

cudaError_t step_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                        cudaStream_t stream) {
    const int power_law = args.power_law;
    const int walls = (args.xwall || args.ywall) ? 1 : 0;
    if (plan.kind == PLAN_TILE) return tile_launch(args, metric, plan, stream);
    if (fast_path_applies(metric, power_law, walls)) return fast_launch(tmap, args, metric, plan, stream);
    if (args.rho0) return rho0_launch(tmap, args, metric, plan, stream);
    if (walls_path_applies(metric, power_law, walls, args.storage))
        return walls_launch(tmap, args, metric, plan, stream);
    MDF_MARCH_DISPATCH(false, launch_t, tmap, args, plan, stream)
}

}  // namespace mdf
