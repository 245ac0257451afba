// mdf_ctx.cuh -- the context behind the opaque mdf_ctx handle of the C ABI,
// shared by the single-problem runtime (mdf_api.cu) and the batch runtime
// (mdf_batch.cu).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "../../include/mdf.h"
#include "mdf_aux.cuh"
#include "mdf_internal.cuh"

// NVTX range around a host call (a no-op unless a profiler is attached).
struct MdfRange {
    explicit MdfRange(const char *name) { nvtxRangePushA(name); }
    ~MdfRange() { nvtxRangePop(); }
    MdfRange(const MdfRange &) = delete;
    MdfRange &operator=(const MdfRange &) = delete;
};

struct mdf_ctx {
    // the members are documented where they are set (mdf_create)
    int dev = 0, num_sms = 0;
    int nx = 0, ny = 0, kind = 0, xwall = 0, ywall = 0;
    double lx = 0, ly = 0;
    mdf_fluid fluid{};
    mdf_bc bc{};
    mdf_params prm{};
    double cs2 = 0, dt = 0, dxmin = 0;
    int pitch = 0;
    long long plane = 0;
    float *buf[2] = {nullptr, nullptr};
    int cur = 0;
    float *kxv = nullptr, *kyv = nullptr;
    float *mxx = nullptr, *mxy = nullptr, *mex = nullptr, *mey = nullptr;
    float *Fxp = nullptr, *Fyp = nullptr;
    int force_mode = 0;
    // dF/dt (mode 0 none, 1 constant, 2 field) and the dt step's force planes
    int rate_mode = 0;
    double drx = 0, dry = 0;
    float *dFxp = nullptr, *dFyp = nullptr, *Fxdp = nullptr, *Fydp = nullptr;
    // source R of Eq. 2.1.1
    float *Rp = nullptr;
    double fx = 0, fy = 0;
    float *snap_u = nullptr, *snap_v = nullptr;
    long long snap_step = 0;
    // h_result: pinned, 8 doubles: [0..4] the residual sums, [6] holds the
    // copy of the device error word that every host wait brings back
    double *partials = nullptr, *result = nullptr, *h_result = nullptr;
    int *err = nullptr;
    cudaEvent_t ev_wait = nullptr;  // recorded by every host wait on `stream`
    // a residual enqueued by mdf_residual_start and not yet collected
    cudaEvent_t ev_res = nullptr;
    bool res_pending = false;
    long long res_window = 0;
    float *scratch = nullptr;  // dense staging for host transfers
    size_t scratch_bytes = 0;
    CUtensorMap tmap[2];
    static constexpr int kMaxCandidates = 8;
    mdf::StepPlan cand[kMaxCandidates];
    int ncand = 0;
    mdf::StepPlan plan{};
    mdf::StepArgs args{};
    mdf::AuxArgs aux{};
    cudaStream_t stream = nullptr;
    // captured graphs of kGraphSteps launches from buffer 0 / 1 (mdf_step),
    // valid while args_version and the plan are unchanged
    static constexpr int kGraphSteps = 16;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_version[2] = {-1, -1};
    long long steps = 0;
    int args_version = 0;  // bumped whenever args change after creation (forcing)
    char last_error[256] = {0};
};


namespace mdf {
// Shared helpers of the host runtime (mdf_api.cu).
mdf_status ctx_fail(mdf_ctx *c, mdf_status st, const char *msg);
mdf_status ctx_encode_maps(mdf_ctx *c, int box_nt, CUtensorMap maps[2]);
mdf_status ctx_create_untuned(const mdf_grid *grid, const mdf_fluid *fluid, const mdf_bc *bc,
                              const mdf_params *params, mdf_ctx **out);
mdf_status ctx_wait(mdf_ctx *c, double timeout_s);
}  // namespace mdf
