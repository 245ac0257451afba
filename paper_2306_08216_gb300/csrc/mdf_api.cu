// mdf_api.cu -- host runtime behind the C ABI of include/mdf.h.
//
// Owns the device state (two buffers of padded 32-bit planes: 10 FP32
// distributions, or u, v, P and 4 planes of 16-bit pairs), the TMA
// descriptors of both buffers, the launch plan of the fused step, the grid
// metrics and force planes, and the FP64 residual machinery.  Argument
// validation happens before any CUDA call, so MDF_E_INVALID never touches
// the GPU.
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <chrono>
#include <new>
#include <thread>

#include "mdf_ctx.cuh"

using namespace mdf;

static thread_local char g_create_error[256] = {0};

static mdf_status fail(mdf_ctx *c, mdf_status st, const char *fmt, ...) {
    char *dst = c ? c->last_error : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

#define CK(ctx, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MDF_E_NOMEM : MDF_E_CUDA,       \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

static bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// Host-side fault injection for the creation path: with MDF_FAIL_ALLOC=k in
// the environment, the k-th device (or pinned host) allocation made while a
// context is created fails as if memory had run out, so that every error
// path of mdf_create can be exercised without touching the GPU's state.
// The count restarts with every mdf_create; 0 or unset disables it.  The
// counter belongs to the creating thread.
static thread_local int g_fail_alloc = 0;

static cudaError_t dev_malloc(void **p, size_t bytes) {
    if (g_fail_alloc > 0 && --g_fail_alloc == 0) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}
template <typename T>
static cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
static cudaError_t host_malloc(void **p, size_t bytes) {
    if (g_fail_alloc > 0 && --g_fail_alloc == 0) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, bytes);
}

static void free_ctx(mdf_ctx *c) {
    if (!c) return;
    float *fp[] = {c->buf[0], c->buf[1], c->kxv, c->kyv, c->mxx, c->mxy, c->mex, c->mey, c->Fxp, c->Fyp,
                   c->dFxp, c->dFyp, c->Fxdp, c->Fydp, c->Rp, c->snap_u, c->snap_v, c->scratch};
    for (float *p : fp)
        if (p) cudaFree(p);
    if (c->partials) cudaFree(c->partials);
    if (c->result) cudaFree(c->result);
    if (c->err) cudaFree(c->err);
    if (c->h_result) cudaFreeHost(c->h_result);
    for (int p = 0; p < 2; ++p)
        if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
    if (c->ev_wait) cudaEventDestroy(c->ev_wait);
    if (c->ev_res) cudaEventDestroy(c->ev_res);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    delete c;
}

static mdf_status encode_maps_box(mdf_ctx *c, int box_nt, CUtensorMap maps[2]);

// Row boxes of the marches for the current plan (a tile plan does not use
// them, so any valid box will do).
static mdf_status encode_maps(mdf_ctx *c) {
    return encode_maps_box(c, c->plan.kind == PLAN_TILE ? 128 : c->plan.NT, c->tmap);
}

// Tensor maps of both state buffers for boxes of box_nt columns x 1 row x
// all planes (32-bit elements; the 16-bit pair words move as opaque 32-bit
// values).
static mdf_status encode_maps_box(mdf_ctx *c, int box_nt, CUtensorMap maps[2]) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        CK(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn)
            return fail(c, MDF_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int planes = state_planes(c->prm.storage, c->prm.rho0);
    for (int b = 0; b < 2; ++b) {
        cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->ny, (cuuint64_t)planes};
        cuuint64_t strides[2] = {(cuuint64_t)c->pitch * 4, (cuuint64_t)c->plane * 4};
        cuuint32_t box[3] = {(cuuint32_t)box_nt, 1, (cuuint32_t)planes};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = encode(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->buf[b], dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(c, MDF_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return MDF_OK;
}

static void fill_rates(mdf_ctx *c) {
    const double s = c->cs2 / c->fluid.nu, sp = c->prm.s_ratio * s, dt = c->dt;
    auto rho = [&](double l) { return (1.0 - 0.5 * dt * l) / (1.0 + 0.5 * dt * l); };
    auto kap = [&](double l) { return 1.0 / (1.0 + 0.25 * dt * l); };
    StepArgs &a = c->args;
    a.rpp = (float)rho(sp);
    a.rp = (float)rho(s);
    a.rbp = (float)(0.25 * (1.0 + 3.0 * rho(sp)));
    a.rb = (float)(0.25 * (1.0 + 3.0 * rho(s)));
    a.rkp = (float)kap(sp);
    a.rk = (float)kap(s);
}

static mdf_status ensure_scratch(mdf_ctx *c, size_t bytes) {
    if (c->scratch_bytes >= bytes) return MDF_OK;
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    CK(c, dev_malloc(&c->scratch, bytes));
    c->scratch_bytes = bytes;
    return MDF_OK;
}

// Bounded host wait for an event recorded on the context's stream.  Polls
// without sleeping for the first 2 ms (the work behind a residual check of
// a small grid ends within microseconds, and a sleeping thread wakes tens of
// microseconds late), then every 20 us up to the limit.
static mdf_status wait_event(mdf_ctx *c, cudaEvent_t ev, double timeout_s) {
    if (timeout_s <= 0) timeout_s = 60.0;
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return MDF_OK;
        if (e != cudaErrorNotReady) return fail(c, MDF_E_CUDA, "stream work failed: %s", cudaGetErrorString(e));
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(c, MDF_E_TIMEOUT, "stream did not finish within %.1f s", timeout_s);
        if (el > 2e-3) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// The device error word comes back in the same ordered stream as the work,
// into pinned memory (h_result[6]), so a wait is the only round trip.
static int *pinned_err(mdf_ctx *c) { return reinterpret_cast<int *>(c->h_result + 6); }

static mdf_status check_device_error(mdf_ctx *c) {
    const int herr = *pinned_err(c);
    if (herr == DEVERR_INDEX)
        return fail(c, MDF_E_CUDA, "the debug build's index check skipped a global access outside its buffer");
    if (herr != 0) return fail(c, MDF_E_TIMEOUT, "a bounded device wait gave up (code %d)", herr);
    return MDF_OK;
}

static mdf_status wait_stream(mdf_ctx *c, double timeout_s) {
    if (!c->ev_wait || !c->h_result || !c->err) {  // part-built context
        CK(c, cudaStreamSynchronize(c->stream));
        return MDF_OK;
    }
    CK(c, cudaMemcpyAsync(pinned_err(c), c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaEventRecord(c->ev_wait, c->stream));
    const mdf_status st = wait_event(c, c->ev_wait, timeout_s);
    if (st != MDF_OK) return st;
    return check_device_error(c);
}

// Launch-plan autotuner: time every candidate plan (march block size and
// band height, or the tile kernel) for a few steps from the initial state
// in buffer 0 (which keeps its contents; the output goes to buffer 1) and
// keep the fastest.  March plans compute the same values whatever the band
// split; the tile kernel is taken only when it beats the best march by more
// than 10 %, so that timing noise near the crossover cannot flip the kernel
// (and the last bits of the results) from one run to the next.
static mdf_status autotune(mdf_ctx *c) {
    if (c->ncand > 1) {
        cudaEvent_t e0, e1;
        CK(c, cudaEventCreate(&e0));
        CK(c, cudaEventCreate(&e1));
        float best = 1e30f, best_tile = 1e30f;
        int best_i = 0, tile_i = -1;
        // two passes over the candidates, 8 timed launches each; keep the
        // fastest time seen per candidate
        for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < c->ncand; ++i) {
            c->plan = c->cand[i];
            mdf_status s = encode_maps(c);
            if (s != MDF_OK) return s;
            StepArgs a = c->args;
            a.W = c->plan.W;
            a.H = c->plan.H;
            a.fout = c->buf[1];
            a.fin = c->buf[0];
            CK(c, step_launch(&c->tmap[0], a, c->kind, c->plan, 0));
            CK(c, cudaEventRecord(e0, 0));
            for (int r = 0; r < 8; ++r) CK(c, step_launch(&c->tmap[0], a, c->kind, c->plan, 0));
            CK(c, cudaEventRecord(e1, 0));
            CK(c, cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(c, cudaEventElapsedTime(&ms, e0, e1));
            if (c->plan.kind == PLAN_TILE) {
                if (ms < best_tile) {
                    best_tile = ms;
                    tile_i = i;
                }
            } else if (ms < best) {
                best = ms;
                best_i = i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->plan = c->cand[(tile_i >= 0 && best_tile < 0.9f * best) ? tile_i : best_i];
    }
    c->args.W = c->plan.W;
    c->args.H = c->plan.H;
    return encode_maps(c);
}

namespace mdf {
mdf_status ctx_fail(mdf_ctx *c, mdf_status st, const char *msg) { return fail(c, st, "%s", msg); }
mdf_status ctx_encode_maps(mdf_ctx *c, int box_nt, CUtensorMap maps[2]) { return encode_maps_box(c, box_nt, maps); }
mdf_status ctx_wait(mdf_ctx *c, double timeout_s) { return wait_stream(c, timeout_s); }
}  // namespace mdf

static mdf_status create_ctx(const mdf_grid *grid, const mdf_fluid *fluid, const mdf_bc *bc,
                             const mdf_params *params, int tune, mdf_ctx **out);

namespace mdf {
// Contexts that only serve as problems of a batch step with the batch's own
// launch plan: the single-problem autotuner is skipped.
mdf_status ctx_create_untuned(const mdf_grid *grid, const mdf_fluid *fluid, const mdf_bc *bc,
                              const mdf_params *params, mdf_ctx **out) {
    const mdf_status s = create_ctx(grid, fluid, bc, params, 0, out);
    g_fail_alloc = 0;
    return s;
}
}  // namespace mdf

extern "C" {

mdf_status mdf_create(const mdf_grid *grid, const mdf_fluid *fluid, const mdf_bc *bc, const mdf_params *params,
                      mdf_ctx **out) {
    MdfRange r("mdf_create");
    const mdf_status s = create_ctx(grid, fluid, bc, params, 1, out);
    g_fail_alloc = 0;
    return s;
}

}  // extern "C"

static mdf_status create_ctx(const mdf_grid *grid, const mdf_fluid *fluid, const mdf_bc *bc,
                             const mdf_params *params, int tune, mdf_ctx **out) {
    if (!out) return fail(nullptr, MDF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!grid || !fluid || !bc) return fail(nullptr, MDF_E_INVALID, "grid, fluid and bc are required");
    if (grid->nx < 5 || grid->ny < 5) return fail(nullptr, MDF_E_INVALID, "nx, ny must be >= 5");
    if ((long long)grid->nx * grid->ny > (1ll << 31))
        return fail(nullptr, MDF_E_INVALID, "grid too large (nx*ny > 2^31)");
    if (grid->kind < 0 || grid->kind > 2) return fail(nullptr, MDF_E_INVALID, "unknown grid kind %d", grid->kind);
    for (int s = 0; s < 4; ++s)
        if (bc->type[s] != MDF_BC_PERIODIC && bc->type[s] != MDF_BC_WALL)
            return fail(nullptr, MDF_E_INVALID, "unknown boundary type on side %d", s);
    if (bc->type[0] != bc->type[1] || bc->type[2] != bc->type[3])
        return fail(nullptr, MDF_E_INVALID, "both sides of an axis need the same boundary type");
    const int xwall = bc->type[0] == MDF_BC_WALL, ywall = bc->type[2] == MDF_BC_WALL;
    if (grid->kind == MDF_GRID_UNIFORM && (!finite_pos(grid->lx) || !finite_pos(grid->ly)))
        return fail(nullptr, MDF_E_INVALID, "uniform grid needs lx, ly > 0");
    if (grid->kind != MDF_GRID_UNIFORM) {
        if (!grid->x || !grid->y) return fail(nullptr, MDF_E_INVALID, "grid coordinates are required");
        if ((!xwall && !finite_pos(grid->lx)) || (!ywall && !finite_pos(grid->ly)))
            return fail(nullptr, MDF_E_INVALID, "periodic axes of a coordinate grid need their period");
    }
    if (!finite_pos(fluid->nu)) return fail(nullptr, MDF_E_INVALID, "nu must be > 0");
    if (fluid->power_law) {
        if (!finite_pos(fluid->K) || !finite_pos(fluid->n) || !finite_pos(fluid->nu_min) ||
            !finite_pos(fluid->nu_max) || fluid->nu_min > fluid->nu_max)
            return fail(nullptr, MDF_E_INVALID, "power law needs K, n > 0 and 0 < nu_min <= nu_max");
    }
    mdf_params prm = params ? *params : mdf_params{1.0, 0.5, 0.8, 1.5, MDF_STORAGE_FP32, 0};
    if (!finite_pos(prm.c)) return fail(nullptr, MDF_E_INVALID, "c must be > 0");
    if (!(prm.cfl > 0 && prm.cfl < 1)) return fail(nullptr, MDF_E_INVALID, "cfl must be in (0, 1)");
    if (!(prm.eta >= 0 && prm.eta <= 1)) return fail(nullptr, MDF_E_INVALID, "eta must be in [0, 1]");
    if (!finite_pos(prm.s_ratio)) return fail(nullptr, MDF_E_INVALID, "s_ratio must be > 0");
    for (int s = 0; s < 4; ++s)
        if (!isfinite(bc->u_wall[s]) || !isfinite(bc->v_wall[s]))
            return fail(nullptr, MDF_E_INVALID, "wall velocities must be finite");
    if (prm.storage < MDF_STORAGE_FP32 || prm.storage > MDF_STORAGE_BF16)
        return fail(nullptr, MDF_E_INVALID, "unknown storage mode %d", prm.storage);
    if (prm.rho0 && prm.storage != MDF_STORAGE_FP32)
        return fail(nullptr, MDF_E_INVALID, "the alpha = 0 distribution needs FP32 storage");
    prm.rho0 = prm.rho0 ? 1 : 0;

    {
        const char *fa = getenv("MDF_FAIL_ALLOC");
        g_fail_alloc = fa ? atoi(fa) : 0;
    }
    // host allocations never throw across the C ABI
    mdf_ctx *c = new (std::nothrow) mdf_ctx();
    if (!c) return fail(nullptr, MDF_E_NOMEM, "host allocation of the context failed");
    c->nx = grid->nx;
    c->ny = grid->ny;
    c->kind = grid->kind;
    c->xwall = xwall;
    c->ywall = ywall;
    c->lx = grid->lx;
    c->ly = grid->ly;
    c->fluid = *fluid;
    c->bc = *bc;
    c->prm = prm;
    c->cs2 = 0.4 * prm.c * prm.c;  // second moment of the D2Q5 weights (Eq. 2.3.4)

#define CKC(call)                                          \
    do {                                                   \
        mdf_status s_ = (call);                            \
        if (s_ != MDF_OK) {                                \
            strncpy(g_create_error, c->last_error, 255);   \
            free_ctx(c);                                   \
            return s_;                                     \
        }                                                  \
    } while (0)
#define CKE(call) CKC(([&]() -> mdf_status { CK(c, call); return MDF_OK; })())

    CKE(cudaGetDevice(&c->dev));
    CKE(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
    const int metric = grid->kind;
    {
        cudaError_t pe = cudaSuccess;
        c->ncand = step_candidates(metric, fluid->power_law ? 1 : 0, (xwall || ywall) ? 1 : 0, prm.storage, prm.rho0,
                                   c->nx, c->ny, c->num_sms, c->cand, mdf_ctx::kMaxCandidates, &pe);
        CKE(pe);
        if (c->ncand < 1) CKE(cudaErrorInvalidConfiguration);
    }
    c->plan = c->cand[0];
    c->pitch = 0;
    for (int i = 0; i < c->ncand; ++i) {
        const int pt = step_pitch(c->nx, c->cand[i].W);
        if (pt > c->pitch) c->pitch = pt;
    }
    c->plane = (long long)c->pitch * c->ny;
    const size_t state_bytes = state_buffer_bytes(prm.storage, c->plane, prm.rho0);
    for (int b = 0; b < 2; ++b) {
        CKE(dev_malloc(&c->buf[b], state_bytes));
        CKE(cudaMemset(c->buf[b], 0, state_bytes));
    }
    const size_t N = (size_t)c->nx * c->ny;
    CKE(dev_malloc(&c->snap_u, N * sizeof(float)));
    CKE(dev_malloc(&c->snap_v, N * sizeof(float)));
    CKE(dev_malloc(&c->err, sizeof(int)));
    CKE(cudaMemset(c->err, 0, sizeof(int)));
    CKE(dev_malloc(&c->result, 8 * sizeof(double)));
    CKE(host_malloc(reinterpret_cast<void **>(&c->h_result), 8 * sizeof(double)));
    CKE(cudaEventCreateWithFlags(&c->ev_wait, cudaEventDisableTiming));
    CKE(cudaEventCreateWithFlags(&c->ev_res, cudaEventDisableTiming));

    AuxArgs &x = c->aux;
    x.nx = c->nx; x.ny = c->ny; x.pitch = c->pitch; x.plane = c->plane;
    x.xwall = xwall; x.ywall = ywall; x.lx = grid->lx; x.ly = grid->ly;
    x.c = (float)prm.c; x.inv2c = (float)(0.5 / prm.c);
    for (int s = 0; s < 4; ++s) { x.uw[s] = (float)bc->u_wall[s]; x.vw[s] = (float)bc->v_wall[s]; }
    x.power_law = fluid->power_law ? 1 : 0;
    x.nu = (float)fluid->nu; x.K = (float)fluid->K; x.n_index = (float)fluid->n;
    x.nu_min = (float)fluid->nu_min; x.nu_max = (float)fluid->nu_max;
    x.storage = prm.storage;
    x.rho0 = prm.rho0;
    x.nscale = (float)ldexp(1.0, NSCALE_EXP - ilogb(prm.c));
    x.ninv = (float)ldexp(1.0, ilogb(prm.c) - NSCALE_EXP);
    CKE(dev_malloc(&c->partials, (size_t)aux_residual_blocks(x) * 5 * sizeof(double)));

    // Grid metrics (FP64 on the GPU) and the time step of Eq. 3.1.
    if (grid->kind == MDF_GRID_UNIFORM) {
        const double dx = xwall ? grid->lx / (c->nx - 1) : grid->lx / c->nx;
        const double dy = ywall ? grid->ly / (c->ny - 1) : grid->ly / c->ny;
        c->dxmin = fmin(dx, dy);
        c->args.kx = (float)(prm.c / dx);
        c->args.ky = (float)(prm.c / dy);
    } else {
        const size_t ncoord = grid->kind == MDF_GRID_SEPARABLE ? (size_t)(c->nx + c->ny) : 2 * N;
        double *dcoord = nullptr, *dedge = nullptr;
        CKE(dev_malloc(&dcoord, ncoord * sizeof(double)));
        const size_t nedge = grid->kind == MDF_GRID_SEPARABLE ? (size_t)(c->nx + c->ny) : N;
        mdf_status st = MDF_OK;
        do {
            cudaError_t e = dev_malloc(&dedge, nedge * sizeof(double));
            if (e != cudaSuccess) { st = fail(c, MDF_E_NOMEM, "metric scratch"); break; }
            double *hedge = (double *)malloc(nedge * sizeof(double));
            if (!hedge) { st = fail(c, MDF_E_NOMEM, "host metric scratch"); break; }
            if (grid->kind == MDF_GRID_SEPARABLE) {
                e = cudaMemcpy(dcoord, grid->x, c->nx * sizeof(double), cudaMemcpyHostToDevice);
                if (e == cudaSuccess)
                    e = cudaMemcpy(dcoord + c->nx, grid->y, c->ny * sizeof(double), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = dev_malloc(&c->kxv, c->pitch * sizeof(float));
                if (e == cudaSuccess) e = dev_malloc(&c->kyv, c->ny * sizeof(float));
                if (e == cudaSuccess)
                    e = aux_metrics1d(x, dcoord, dcoord + c->nx, prm.c, c->kxv, c->kyv, dedge, 0);
            } else {
                e = cudaMemcpy(dcoord, grid->x, N * sizeof(double), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = cudaMemcpy(dcoord + N, grid->y, N * sizeof(double), cudaMemcpyHostToDevice);
                const size_t mp = (size_t)c->pitch * c->ny * sizeof(float);
                if (e == cudaSuccess) e = dev_malloc(&c->mxx, mp);
                if (e == cudaSuccess) e = dev_malloc(&c->mxy, mp);
                if (e == cudaSuccess) e = dev_malloc(&c->mex, mp);
                if (e == cudaSuccess) e = dev_malloc(&c->mey, mp);
                if (e == cudaSuccess)
                    e = aux_metrics2d(x, dcoord, dcoord + N, prm.c, c->mxx, c->mxy, c->mex, c->mey, dedge, 0);
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e == cudaSuccess) e = cudaMemcpy(hedge, dedge, nedge * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                free(hedge);
                st = fail(c, e == cudaErrorMemoryAllocation ? MDF_E_NOMEM : MDF_E_CUDA, "metric setup: %s",
                          cudaGetErrorString(e));
                break;
            }
            double m = INFINITY;
            for (size_t i = 0; i < nedge; ++i) m = fmin(m, hedge[i]);
            free(hedge);
            if (!(m > 0 && isfinite(m))) { st = fail(c, MDF_E_INVALID, "degenerate grid (min edge %g)", m); break; }
            c->dxmin = m;
        } while (0);
        cudaFree(dcoord);
        if (dedge) cudaFree(dedge);
        CKC(st);
    }
    c->dt = prm.cfl * c->dxmin / prm.c;  // Eq. 3.1

    StepArgs &a = c->args;
    a.storage = prm.storage;
    a.rho0 = prm.rho0;
    a.nscale = x.nscale;
    a.ninv = x.ninv;
    a.nx = c->nx; a.ny = c->ny; a.pitch = c->pitch; a.plane = c->plane;
    a.W = c->plan.W; a.H = c->plan.H;
    a.xwall = xwall; a.ywall = ywall;
    a.c = (float)prm.c; a.inv2c = (float)(0.5 / prm.c);
    a.dt = (float)c->dt; a.h = (float)(0.5 * c->dt);
    const double eta = prm.eta;
    a.a1 = (float)(0.5 * eta);
    a.a0 = (float)(1.5 * (1.0 - eta));
    a.am1 = (float)(-0.5 * (4.0 - 3.0 * eta));
    a.am2 = (float)(0.5 * (1.0 - eta));
    a.kxv = c->kxv; a.kyv = c->kyv;
    a.mxx = c->mxx; a.mxy = c->mxy; a.mex = c->mex; a.mey = c->mey;
    fill_rates(c);
    a.power_law = fluid->power_law ? 1 : 0;
    a.K = (float)fluid->K; a.n_index = (float)fluid->n; a.nu_min = (float)fluid->nu_min;
    a.nu_max = (float)fluid->nu_max; a.cs2 = (float)c->cs2; a.s_ratio = (float)prm.s_ratio;
    a.a_pl = (float)(0.5 * c->cs2 * c->dt);
    if (fluid->power_law) {
        a.lnK = (float)log(fluid->K);
        a.ln_nu_min = (float)log(fluid->nu_min);
        a.ln_nu_max = (float)log(fluid->nu_max);
        a.inv_n = (float)(1.0 / fluid->n);
    }
    a.force_mode = 0;
    for (int s = 0; s < 4; ++s) { a.uw[s] = x.uw[s]; a.vw[s] = x.vw[s]; }
    a.err = c->err;
    x.a_pl = a.a_pl;
    if (grid->kind == MDF_GRID_UNIFORM) {
        const float kxs = a.kx, kys = a.ky;
        const float w[3] = {a.a1, a.a0, a.am2};
        for (int i = 0; i < 3; ++i) {
            a.pwxh[i] = pack_pair(-a.h * kxs * w[i]);
            a.pwxd[i] = pack_pair(-a.dt * kxs * w[i]);
            a.pwyh[i] = pack_pair(-a.h * kys * w[i]);
            a.pwyd[i] = pack_pair(-a.dt * kys * w[i]);
        }
    }
    a.rk_hat = (float)(0.5 * (fluid->nu + c->cs2 * c->dt / 2.0));  // Eq. 2.3.23 from fhat
    a.rk_bar = (float)(0.5 * (fluid->nu + c->cs2 * c->dt / 4.0));  // ... from fbar (h = dt/2)
    x.rk_hat = a.rk_hat;
    a.pmKp = pack_pair(-(1.0f - a.rpp));
    a.pDp = pack_pair(0.5f * (a.rp - a.rpp));
    a.pmKb = pack_pair(-(1.0f - a.rbp));
    a.pDb = pack_pair(0.5f * (a.rb - a.rbp));
    a.pmKk = pack_pair(-(1.0f - a.rkp));
    a.pDk = pack_pair(0.5f * (a.rk - a.rkp));
    a.phw = pack_pair(a.h * 0.2f);
    a.pdw = pack_pair(a.dt * 0.2f);
    CKC(encode_maps(c));

    // Rest state.
    CKE(ensure_scratch(c, 3 * N * sizeof(float)) == MDF_OK ? cudaSuccess : cudaErrorMemoryAllocation);
    CKE(cudaMemset(c->scratch, 0, 3 * N * sizeof(float)));
    CKE(aux_init(x, c->scratch, c->scratch + N, c->scratch + 2 * N, c->buf[0], 0));
    CKE(aux_snapshot(x, c->buf[0], c->snap_u, c->snap_v, 0));
    CKE(cudaDeviceSynchronize());
    if (tune) CKC(autotune(c));
    else {
        c->args.W = c->plan.W;
        c->args.H = c->plan.H;
        CKC(encode_maps(c));
    }
    c->cur = 0;
    *out = c;
    return MDF_OK;
#undef CKE
#undef CKC
}

extern "C" {

void mdf_destroy(mdf_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

mdf_status mdf_set_stream(mdf_ctx *c, void *stream) {
    if (!c) return MDF_E_INVALID;
    c->stream = (cudaStream_t)stream;
    return MDF_OK;
}

// Copy caller arrays (host or device) into the dense staging buffer.
static mdf_status stage_in(mdf_ctx *c, const float *const *src, int count, int on_device) {
    const size_t N = (size_t)c->nx * c->ny;
    mdf_status s = ensure_scratch(c, (size_t)count * N * sizeof(float));
    if (s != MDF_OK) return s;
    for (int i = 0; i < count; ++i)
        CK(c, cudaMemcpyAsync(c->scratch + i * N, src[i], N * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    return MDF_OK;
}

// The dt step's force F + dt/2 dF/dt (Eq. 2.3.24) from the force and its rate.
static mdf_status update_force_d(mdf_ctx *c) {
    StepArgs &a = c->args;
    const double k = 0.5 * c->dt;
    if (c->rate_mode == 0) {
        a.force_mode_d = a.force_mode;
        a.Fxd = a.Fx;
        a.Fyd = a.Fy;
        a.Fxdp = a.Fxp;
        a.Fydp = a.Fyp;
    } else if (c->rate_mode == 1 && c->force_mode != MDF_FORCE_FIELD) {
        const double fx = c->force_mode ? c->fx : 0.0, fy = c->force_mode ? c->fy : 0.0;
        a.force_mode_d = 1;
        a.Fxd = (float)(fx + k * c->drx);
        a.Fyd = (float)(fy + k * c->dry);
    } else {
        const size_t pb = (size_t)c->pitch * c->ny * sizeof(float);
        if (!c->Fxdp) CK(c, cudaMalloc(&c->Fxdp, pb));
        if (!c->Fydp) CK(c, cudaMalloc(&c->Fydp, pb));
        const bool ff = c->force_mode == MDF_FORCE_FIELD, rf = c->rate_mode == MDF_FORCE_FIELD;
        const float fx = c->force_mode == MDF_FORCE_CONSTANT ? (float)c->fx : 0.0f;
        const float fy = c->force_mode == MDF_FORCE_CONSTANT ? (float)c->fy : 0.0f;
        CK(c, aux_axpy_field(c->aux, ff ? c->Fxp : nullptr, fx, rf ? c->dFxp : nullptr, (float)c->drx, (float)k,
                             c->Fxdp, c->stream));
        CK(c, aux_axpy_field(c->aux, ff ? c->Fyp : nullptr, fy, rf ? c->dFyp : nullptr, (float)c->dry, (float)k,
                             c->Fydp, c->stream));
        a.force_mode_d = 2;
        a.Fxdp = c->Fxdp;
        a.Fydp = c->Fydp;
    }
    ++c->args_version;
    return MDF_OK;
}

mdf_status mdf_set_force(mdf_ctx *c, int mode, double fx, double fy, const float *Fx, const float *Fy,
                         int on_device) {
    if (!c) return MDF_E_INVALID;
    if (mode < MDF_FORCE_NONE || mode > MDF_FORCE_FIELD) return fail(c, MDF_E_INVALID, "unknown force mode");
    if (mode == MDF_FORCE_CONSTANT && (!isfinite(fx) || !isfinite(fy)))
        return fail(c, MDF_E_INVALID, "force must be finite");
    if (mode == MDF_FORCE_FIELD) {
        if (!Fx || !Fy) return fail(c, MDF_E_INVALID, "force field arrays are required");
        const size_t pb = (size_t)c->pitch * c->ny * sizeof(float);
        if (!c->Fxp) CK(c, cudaMalloc(&c->Fxp, pb));
        if (!c->Fyp) CK(c, cudaMalloc(&c->Fyp, pb));
        const float *src[2] = {Fx, Fy};
        mdf_status s = stage_in(c, src, 2, on_device);
        if (s != MDF_OK) return s;
        const size_t N = (size_t)c->nx * c->ny;
        CK(c, aux_pad_field(c->aux, c->scratch, c->Fxp, c->stream));
        CK(c, aux_pad_field(c->aux, c->scratch + N, c->Fyp, c->stream));
    }
    c->force_mode = mode;
    c->fx = fx;
    c->fy = fy;
    ++c->args_version;
    c->args.force_mode = mode;
    c->args.Fx = (float)fx;
    c->args.Fy = (float)fy;
    c->args.Fxp = c->Fxp;
    c->args.Fyp = c->Fyp;
    return update_force_d(c);
}

mdf_status mdf_set_force_rate(mdf_ctx *c, int mode, double dfx, double dfy, const float *dFx, const float *dFy,
                              int on_device) {
    if (!c) return MDF_E_INVALID;
    if (mode < MDF_FORCE_NONE || mode > MDF_FORCE_FIELD) return fail(c, MDF_E_INVALID, "unknown force-rate mode");
    if (mode == MDF_FORCE_CONSTANT && (!isfinite(dfx) || !isfinite(dfy)))
        return fail(c, MDF_E_INVALID, "force rate must be finite");
    if (mode == MDF_FORCE_FIELD) {
        if (!dFx || !dFy) return fail(c, MDF_E_INVALID, "force-rate field arrays are required");
        const size_t pb = (size_t)c->pitch * c->ny * sizeof(float);
        if (!c->dFxp) CK(c, cudaMalloc(&c->dFxp, pb));
        if (!c->dFyp) CK(c, cudaMalloc(&c->dFyp, pb));
        const float *src[2] = {dFx, dFy};
        mdf_status s = stage_in(c, src, 2, on_device);
        if (s != MDF_OK) return s;
        const size_t N = (size_t)c->nx * c->ny;
        CK(c, aux_pad_field(c->aux, c->scratch, c->dFxp, c->stream));
        CK(c, aux_pad_field(c->aux, c->scratch + N, c->dFyp, c->stream));
    }
    c->rate_mode = mode;
    c->drx = mode == MDF_FORCE_CONSTANT ? dfx : 0.0;
    c->dry = mode == MDF_FORCE_CONSTANT ? dfy : 0.0;
    return update_force_d(c);
}

mdf_status mdf_set_source(mdf_ctx *c, int mode, double r, const float *R, int on_device) {
    if (!c) return MDF_E_INVALID;
    if (mode < MDF_FORCE_NONE || mode > MDF_FORCE_FIELD) return fail(c, MDF_E_INVALID, "unknown source mode");
    if (mode != MDF_FORCE_NONE && c->fluid.power_law)
        return fail(c, MDF_E_INVALID, "the source term needs a Newtonian fluid");
    if (mode != MDF_FORCE_NONE && c->prm.storage != MDF_STORAGE_FP32)
        return fail(c, MDF_E_INVALID, "the source term needs FP32 storage");
    if (mode == MDF_FORCE_CONSTANT && !isfinite(r)) return fail(c, MDF_E_INVALID, "source must be finite");
    if (mode == MDF_FORCE_FIELD) {
        if (!R) return fail(c, MDF_E_INVALID, "source field array is required");
        if (!c->Rp) CK(c, cudaMalloc(&c->Rp, (size_t)c->pitch * c->ny * sizeof(float)));
        const float *src[1] = {R};
        mdf_status s = stage_in(c, src, 1, on_device);
        if (s != MDF_OK) return s;
        CK(c, aux_pad_field(c->aux, c->scratch, c->Rp, c->stream));
    }
    StepArgs &a = c->args;
    a.r_mode = mode;
    a.Rc = mode == MDF_FORCE_CONSTANT ? (float)r : 0.0f;
    a.Rp = c->Rp;
    c->aux.r_mode = a.r_mode;
    c->aux.Rc = a.Rc;
    c->aux.Rp = a.Rp;
    ++c->args_version;
    return MDF_OK;
}

mdf_status mdf_set_metrics(mdf_ctx *c, const double *xi_x, const double *xi_y, const double *eta_x,
                           const double *eta_y, int on_device) {
    if (!c) return MDF_E_INVALID;
    if (c->kind != MDF_GRID_CURVILINEAR) return fail(c, MDF_E_INVALID, "given metrics need a curvilinear grid");
    if (!xi_x || !xi_y || !eta_x || !eta_y) return fail(c, MDF_E_INVALID, "xi_x, xi_y, eta_x, eta_y are required");
    const size_t N = (size_t)c->nx * c->ny;
    const double *in[4] = {xi_x, xi_y, eta_x, eta_y};
    if (!on_device) {
        for (int k = 0; k < 4; ++k)
            for (size_t i = 0; i < N; ++i)
                if (!isfinite(in[k][i])) return fail(c, MDF_E_INVALID, "metric coefficients must be finite");
    }
    double *d = nullptr;
    const double *m[4] = {xi_x, xi_y, eta_x, eta_y};
    if (!on_device) {
        CK(c, cudaMalloc(&d, 4 * N * sizeof(double)));
        for (int k = 0; k < 4; ++k) {
            const cudaError_t e = cudaMemcpyAsync(d + k * N, in[k], N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) {
                cudaFree(d);
                return fail(c, MDF_E_CUDA, "metric upload: %s", cudaGetErrorString(e));
            }
            m[k] = d + k * N;
        }
    }
    cudaError_t e = aux_metrics_given(c->aux, m, c->prm.c, c->mxx, c->mxy, c->mex, c->mey, c->stream);
    mdf_status st = MDF_OK;
    if (e != cudaSuccess) st = fail(c, MDF_E_CUDA, "metric kernel: %s", cudaGetErrorString(e));
    else if (!on_device) st = wait_stream(c, 0);  // the host copies and the scratch are released below
    if (d) cudaFree(d);
    return st;
}

mdf_status mdf_init_fields(mdf_ctx *c, const float *u, const float *v, const float *p, int on_device) {
    if (!c) return MDF_E_INVALID;
    if (!u || !v || !p) return fail(c, MDF_E_INVALID, "u, v, p are required");
    const float *src[3] = {u, v, p};
    mdf_status s = stage_in(c, src, 3, on_device);
    if (s != MDF_OK) return s;
    const size_t N = (size_t)c->nx * c->ny;
    c->cur = 0;
    CK(c, aux_init(c->aux, c->scratch, c->scratch + N, c->scratch + 2 * N, c->buf[0], c->stream));
    CK(c, aux_snapshot(c->aux, c->buf[0], c->snap_u, c->snap_v, c->stream));
    c->steps = 0;
    c->snap_step = 0;
    if (!on_device) return wait_stream(c, 0);
    return MDF_OK;
}

static void drop_graphs(mdf_ctx *c) {
    for (int p = 0; p < 2; ++p) {
        if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
        c->graph[p] = nullptr;
        c->graph_version[p] = -1;
    }
}

// Capture kGraphSteps launches starting from buffer `parity` on the capture
// stream (the kernel arguments, buffer pointers and tensor maps are baked in).
static mdf_status build_step_graph(mdf_ctx *c, int parity) {
    if (!c->cstream) {
        CK(c, cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
        CK(c, cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    }
    if (c->graph[parity]) cudaGraphExecDestroy(c->graph[parity]);
    c->graph[parity] = nullptr;
    CK(c, cudaStreamBeginCapture(c->cstream, cudaStreamCaptureModeThreadLocal));
    StepArgs a = c->args;
    int cur = parity;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < mdf_ctx::kGraphSteps && e == cudaSuccess; ++i) {
        a.fout = c->buf[1 - cur];
        a.fin = c->buf[cur];
        e = step_launch(&c->tmap[cur], a, c->kind, c->plan, c->cstream);
        cur = 1 - cur;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->cstream, &g);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    CK(c, e);
    c->graph_version[parity] = c->args_version;
    return MDF_OK;
}

mdf_status mdf_step(mdf_ctx *c, int n) {
    if (!c) return MDF_E_INVALID;
    MdfRange r("mdf_step");
    if (n < 0) return fail(c, MDF_E_INVALID, "n must be >= 0");
    int done = 0;
    const int reps = n / mdf_ctx::kGraphSteps;
    if (reps >= 2) {
        // replay a captured graph on the capture stream, ordered after and
        // before the context's stream by events; an even number of steps
        // leaves the buffer parity unchanged
        if (!c->graph[c->cur] || c->graph_version[c->cur] != c->args_version) {
            mdf_status s = build_step_graph(c, c->cur);
            if (s != MDF_OK) return s;
        }
        CK(c, cudaEventRecord(c->ev_in, c->stream));
        CK(c, cudaStreamWaitEvent(c->cstream, c->ev_in, 0));
        for (int r = 0; r < reps; ++r) CK(c, cudaGraphLaunch(c->graph[c->cur], c->cstream));
        CK(c, cudaEventRecord(c->ev_out, c->cstream));
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_out, 0));
        done = reps * mdf_ctx::kGraphSteps;
        c->steps += done;
    }
    for (int i = done; i < n; ++i) {
        c->args.fout = c->buf[1 - c->cur];
        c->args.fin = c->buf[c->cur];
        CK(c, step_launch(&c->tmap[c->cur], c->args, c->kind, c->plan, c->stream));
        c->cur = 1 - c->cur;
        ++c->steps;
    }
    return MDF_OK;
}

mdf_status mdf_fields(mdf_ctx *c, unsigned mask, float *const *out, int on_device) {
    if (!c) return MDF_E_INVALID;
    MdfRange r("mdf_fields");
    if (mask >> 17) return fail(c, MDF_E_INVALID, "unknown field bits in mask");
    if (mask && !out) return fail(c, MDF_E_INVALID, "out is NULL");
    const size_t N = (size_t)c->nx * c->ny;
    int count = 0;
    for (int q = 0; q < 17; ++q)
        if (mask & (1u << q)) {
            if (!out[count]) return fail(c, MDF_E_INVALID, "output %d is NULL", count);
            ++count;
        }
    if (!count) return MDF_OK;
    FieldPtrs dst;
    if (!on_device) {
        mdf_status s = ensure_scratch(c, (size_t)count * N * sizeof(float));
        if (s != MDF_OK) return s;
    }
    int k = 0;
    for (int q = 0; q < 17; ++q) {
        dst.p[q] = nullptr;
        if (mask & (1u << q)) {
            dst.p[q] = on_device ? out[k] : c->scratch + (size_t)k * N;
            ++k;
        }
    }
    CK(c, aux_fields(c->aux, c->buf[c->cur], dst, c->stream));
    if (!on_device) {
        for (int i = 0; i < count; ++i)
            CK(c, cudaMemcpyAsync(out[i], c->scratch + (size_t)i * N, N * sizeof(float), cudaMemcpyDeviceToHost,
                                  c->stream));
        return wait_stream(c, 0);
    }
    return MDF_OK;
}

mdf_status mdf_residual_start(mdf_ctx *c) {
    if (!c) return MDF_E_INVALID;
    if (c->res_pending) return fail(c, MDF_E_STATE, "a residual is already pending (mdf_residual_finish)");
    MdfRange rr("mdf_residual_start");
    CK(c, aux_residual(c->aux, c->buf[c->cur], c->snap_u, c->snap_v, c->partials, c->result, c->stream));
    CK(c, cudaMemcpyAsync(c->h_result, c->result, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(pinned_err(c), c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaEventRecord(c->ev_res, c->stream));
    c->res_window = c->steps - c->snap_step;
    c->snap_step = c->steps;
    c->res_pending = true;
    return MDF_OK;
}

mdf_status mdf_residual_finish(mdf_ctx *c, double *residual, double drift[2]) {
    if (!c) return MDF_E_INVALID;
    if (!c->res_pending) return fail(c, MDF_E_STATE, "no residual pending (mdf_residual_start)");
    MdfRange rr("mdf_residual_finish");
    mdf_status s = wait_event(c, c->ev_res, 0);
    c->res_pending = false;
    if (s != MDF_OK) return s;
    s = check_device_error(c);
    if (s != MDF_OK) return s;
    const double *r = c->h_result;
    const long long window = c->res_window;
    const double val = window > 0 ? sqrt(r[0]) / ((double)window * sqrt(r[1])) : NAN;
    if (residual) *residual = val;
    if (drift) { drift[0] = r[2]; drift[1] = r[3]; }
    if (r[4] > 0 || !isfinite(r[2]) || !isfinite(r[3]))
        return fail(c, MDF_E_DIVERGED, "non-finite velocity at %.0f nodes", r[4]);
    if (window <= 0) return fail(c, MDF_E_STATE, "no step since the previous residual");
    return MDF_OK;
}

mdf_status mdf_residual(mdf_ctx *c, double *residual, double drift[2]) {
    if (!c) return MDF_E_INVALID;
    MdfRange rr("mdf_residual");
    const mdf_status s = mdf_residual_start(c);
    if (s != MDF_OK) return s;
    return mdf_residual_finish(c, residual, drift);
}

mdf_status mdf_get_distributions(mdf_ctx *c, float *out, int on_device) {
    if (!c || !out) return c ? fail(c, MDF_E_INVALID, "out is NULL") : MDF_E_INVALID;
    const size_t n = (size_t)NPLANES * c->nx * c->ny;
    if (on_device) {
        CK(c, aux_pack(c->aux, c->buf[c->cur], out, c->stream));
        return MDF_OK;
    }
    mdf_status s = ensure_scratch(c, n * sizeof(float));
    if (s != MDF_OK) return s;
    CK(c, aux_pack(c->aux, c->buf[c->cur], c->scratch, c->stream));
    CK(c, cudaMemcpyAsync(out, c->scratch, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c, 0);
}

mdf_status mdf_set_distributions(mdf_ctx *c, const float *in, int on_device) {
    if (!c || !in) return c ? fail(c, MDF_E_INVALID, "in is NULL") : MDF_E_INVALID;
    const size_t n = (size_t)NPLANES * c->nx * c->ny;
    const float *src = in;
    if (!on_device) {
        mdf_status s = ensure_scratch(c, n * sizeof(float));
        if (s != MDF_OK) return s;
        CK(c, cudaMemcpyAsync(c->scratch, in, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        src = c->scratch;
    }
    CK(c, aux_unpack(c->aux, src, c->buf[c->cur], c->stream));
    CK(c, aux_snapshot(c->aux, c->buf[c->cur], c->snap_u, c->snap_v, c->stream));
    c->snap_step = c->steps;
    if (!on_device) return wait_stream(c, 0);
    return MDF_OK;
}

static mdf_status need_rho0(mdf_ctx *c) {
    return c->prm.rho0 ? MDF_OK : fail(c, MDF_E_INVALID, "this context does not evolve rho_0 (params->rho0 = 0)");
}

mdf_status mdf_init_rho0(mdf_ctx *c, const float *rho0, int on_device) {
    if (!c) return MDF_E_INVALID;
    mdf_status s = need_rho0(c);
    if (s != MDF_OK) return s;
    if (!rho0) return fail(c, MDF_E_INVALID, "rho0 is NULL");
    const float *src[1] = {rho0};
    s = stage_in(c, src, 1, on_device);
    if (s != MDF_OK) return s;
    CK(c, aux_init_rho0(c->aux, c->scratch, c->buf[c->cur], c->stream));
    if (!on_device) return wait_stream(c, 0);
    return MDF_OK;
}

mdf_status mdf_get_rho0(mdf_ctx *c, float *out, int on_device) {
    if (!c) return MDF_E_INVALID;
    mdf_status s = need_rho0(c);
    if (s != MDF_OK) return s;
    if (!out) return fail(c, MDF_E_INVALID, "out is NULL");
    const size_t N = (size_t)c->nx * c->ny;
    if (on_device) {
        CK(c, aux_rho0_field(c->aux, c->buf[c->cur], out, c->stream));
        return MDF_OK;
    }
    s = ensure_scratch(c, N * sizeof(float));
    if (s != MDF_OK) return s;
    CK(c, aux_rho0_field(c->aux, c->buf[c->cur], c->scratch, c->stream));
    CK(c, cudaMemcpyAsync(out, c->scratch, N * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c, 0);
}

mdf_status mdf_get_rho0_distributions(mdf_ctx *c, float *out, int on_device) {
    if (!c) return MDF_E_INVALID;
    mdf_status s = need_rho0(c);
    if (s != MDF_OK) return s;
    if (!out) return fail(c, MDF_E_INVALID, "out is NULL");
    const size_t n = (size_t)5 * c->nx * c->ny;
    if (on_device) {
        CK(c, aux_pack_rho0(c->aux, c->buf[c->cur], out, c->stream));
        return MDF_OK;
    }
    s = ensure_scratch(c, n * sizeof(float));
    if (s != MDF_OK) return s;
    CK(c, aux_pack_rho0(c->aux, c->buf[c->cur], c->scratch, c->stream));
    CK(c, cudaMemcpyAsync(out, c->scratch, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c, 0);
}

mdf_status mdf_set_rho0_distributions(mdf_ctx *c, const float *in, int on_device) {
    if (!c) return MDF_E_INVALID;
    mdf_status s = need_rho0(c);
    if (s != MDF_OK) return s;
    if (!in) return fail(c, MDF_E_INVALID, "in is NULL");
    const size_t n = (size_t)5 * c->nx * c->ny;
    const float *src = in;
    if (!on_device) {
        s = ensure_scratch(c, n * sizeof(float));
        if (s != MDF_OK) return s;
        CK(c, cudaMemcpyAsync(c->scratch, in, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        src = c->scratch;
    }
    CK(c, aux_unpack_rho0(c->aux, src, c->buf[c->cur], c->stream));
    if (!on_device) return wait_stream(c, 0);
    return MDF_OK;
}

mdf_status mdf_synchronize(mdf_ctx *c, double timeout_s) {
    if (!c) return MDF_E_INVALID;
    return wait_stream(c, timeout_s);
}

// 16-bit storage: the checkpoint holds the raw device buffer (padded planes
// u, v, P and the 16-bit non-equilibrium planes), so a restart is bitwise.
static mdf_status save_raw(mdf_ctx *c, const char *path) {
    const size_t bytes = state_buffer_bytes(c->prm.storage, c->plane);
    unsigned char *h = (unsigned char *)malloc(bytes);
    if (!h) return fail(c, MDF_E_NOMEM, "host buffer");
    CK(c, cudaMemcpyAsync(h, c->buf[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream));
    mdf_status s = wait_stream(c, 0);
    if (s != MDF_OK) { free(h); return s; }
    FILE *fp = fopen(path, "wb");
    if (!fp) { free(h); return fail(c, MDF_E_INVALID, "cannot open %s", path); }
    char hdr[256];
    memset(hdr, 0, sizeof(hdr));
    snprintf(hdr, sizeof(hdr), "MDFCKPT1 nx=%d ny=%d steps=%lld dt=%.17g planes=%d storage=%d pitch=%d\n", c->nx,
             c->ny, c->steps, c->dt, DEV_PLANES, c->prm.storage, c->pitch);
    const bool ok = fwrite(hdr, 1, sizeof(hdr), fp) == sizeof(hdr) && fwrite(h, 1, bytes, fp) == bytes;
    fclose(fp);
    free(h);
    return ok ? MDF_OK : fail(c, MDF_E_INVALID, "short write to %s", path);
}

mdf_status mdf_save(mdf_ctx *c, const char *path) {
    if (!c || !path) return c ? fail(c, MDF_E_INVALID, "path is NULL") : MDF_E_INVALID;
    MdfRange r("mdf_save");
    if (c->prm.storage != MDF_STORAGE_FP32) return save_raw(c, path);
    const int planes = state_planes(c->prm.storage, c->prm.rho0);
    const size_t N = (size_t)c->nx * c->ny, n = (size_t)planes * N;
    float *h = (float *)malloc(n * sizeof(float));
    if (!h) return fail(c, MDF_E_NOMEM, "host buffer");
    mdf_status s = mdf_get_distributions(c, h, 0);
    if (s == MDF_OK && c->prm.rho0) s = mdf_get_rho0_distributions(c, h + NPLANES * N, 0);
    if (s != MDF_OK) { free(h); return s; }
    FILE *fp = fopen(path, "wb");
    if (!fp) { free(h); return fail(c, MDF_E_INVALID, "cannot open %s", path); }
    char hdr[256];
    memset(hdr, 0, sizeof(hdr));
    snprintf(hdr, sizeof(hdr), "MDFCKPT1 nx=%d ny=%d steps=%lld dt=%.17g planes=%d\n", c->nx, c->ny, c->steps, c->dt,
             planes);
    const bool ok = fwrite(hdr, 1, sizeof(hdr), fp) == sizeof(hdr) && fwrite(h, sizeof(float), n, fp) == n;
    fclose(fp);
    free(h);
    return ok ? MDF_OK : fail(c, MDF_E_INVALID, "short write to %s", path);
}

mdf_status mdf_load(mdf_ctx *c, const char *path) {
    if (!c || !path) return c ? fail(c, MDF_E_INVALID, "path is NULL") : MDF_E_INVALID;
    MdfRange r("mdf_load");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(c, MDF_E_INVALID, "cannot open %s", path);
    char hdr[256];
    if (fread(hdr, 1, sizeof(hdr), fp) != sizeof(hdr)) { fclose(fp); return fail(c, MDF_E_INVALID, "bad header"); }
    hdr[255] = 0;
    int nx = 0, ny = 0, planes = 0, storage = 0, pitch = 0;
    long long steps = 0;
    double dt = 0;
    const int got = sscanf(hdr, "MDFCKPT1 nx=%d ny=%d steps=%lld dt=%lg planes=%d storage=%d pitch=%d", &nx, &ny,
                           &steps, &dt, &planes, &storage, &pitch);
    if (got < 5 || nx != c->nx || ny != c->ny) {
        fclose(fp);
        return fail(c, MDF_E_INVALID, "checkpoint does not match this grid");
    }
    if (c->prm.storage != MDF_STORAGE_FP32 || got == 7) {
        // raw 16-bit checkpoint: same storage mode and padded layout only
        if (got != 7 || storage != c->prm.storage || pitch != c->pitch || planes != DEV_PLANES) {
            fclose(fp);
            return fail(c, MDF_E_INVALID, "checkpoint storage mode or layout does not match this solver");
        }
        const size_t bytes = state_buffer_bytes(storage, c->plane);
        unsigned char *h = (unsigned char *)malloc(bytes);
        if (!h) { fclose(fp); return fail(c, MDF_E_NOMEM, "host buffer"); }
        const bool ok = fread(h, 1, bytes, fp) == bytes;
        fclose(fp);
        if (!ok) { free(h); return fail(c, MDF_E_INVALID, "short read from %s", path); }
        cudaError_t e = cudaMemcpyAsync(c->buf[c->cur], h, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = aux_snapshot(c->aux, c->buf[c->cur], c->snap_u, c->snap_v, c->stream);
        mdf_status s = e == cudaSuccess ? wait_stream(c, 0)
                                         : fail(c, MDF_E_CUDA, "checkpoint upload: %s", cudaGetErrorString(e));
        free(h);
        if (s == MDF_OK) { c->steps = steps; c->snap_step = steps; }
        return s;
    }
    if (planes != state_planes(c->prm.storage, c->prm.rho0)) {
        fclose(fp);
        return fail(c, MDF_E_INVALID, "checkpoint plane count %d does not match this solver", planes);
    }
    const size_t N = (size_t)c->nx * c->ny, n = (size_t)planes * N;
    float *h = (float *)malloc(n * sizeof(float));
    if (!h) { fclose(fp); return fail(c, MDF_E_NOMEM, "host buffer"); }
    const bool ok = fread(h, sizeof(float), n, fp) == n;
    fclose(fp);
    if (!ok) { free(h); return fail(c, MDF_E_INVALID, "short read from %s", path); }
    mdf_status s = mdf_set_distributions(c, h, 0);
    if (s == MDF_OK && c->prm.rho0) s = mdf_set_rho0_distributions(c, h + NPLANES * N, 0);
    free(h);
    if (s == MDF_OK) { c->steps = steps; c->snap_step = steps; }
    return s;
}

double mdf_dt(const mdf_ctx *c) { return c ? c->dt : NAN; }
long long mdf_steps_done(const mdf_ctx *c) { return c ? c->steps : -1; }
const char *mdf_last_error(const mdf_ctx *c) { return c ? c->last_error : g_create_error; }

mdf_status mdf_launch_info(const mdf_ctx *c, int info[8]) {
    if (!c || !info) return MDF_E_INVALID;
    info[0] = c->plan.NT;
    info[1] = c->plan.W;
    info[2] = c->plan.H;
    info[3] = c->plan.gx;
    info[4] = c->plan.gy;
    info[5] = c->plan.smem;
    info[6] = c->plan.occ;
    info[7] = c->pitch;
    return MDF_OK;
}

mdf_status mdf_set_launch(mdf_ctx *c, int threads, int rows_per_block) {
    if (!c) return MDF_E_INVALID;
    int found = -1;
    for (int i = 0; i < c->ncand; ++i) {
        const bool tile = c->cand[i].kind == PLAN_TILE;
        if (threads == 0 ? tile : (!tile && c->cand[i].NT == threads)) { found = i; break; }
    }
    if (found < 0) return fail(c, MDF_E_INVALID, "no launch plan with %d threads for this problem", threads);
    if (threads != 0 && rows_per_block < 1) return fail(c, MDF_E_INVALID, "rows_per_block must be >= 1");
    StepPlan p = c->cand[found];
    if (threads != 0) {
        p.H = rows_per_block;
        p.gy = (c->ny + p.H - 1) / p.H;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->cstream) CK(c, cudaStreamSynchronize(c->cstream));
    c->plan = p;
    c->args.W = p.W;
    c->args.H = p.H;
    drop_graphs(c);
    return encode_maps(c);
}

int mdf_launch_kind(const mdf_ctx *c) { return c ? c->plan.kind : -1; }

mdf_status mdf_debug_poison(mdf_ctx *c) {
    if (!c) return MDF_E_INVALID;
    for (int b = 0; b < 2; ++b)
        CK(c, aux_poison(c->aux, c->buf[b], state_planes(c->prm.storage, c->prm.rho0), c->stream));
    return wait_stream(c, 0);
}

double mdf_bytes_per_node(const mdf_ctx *c) {
    if (!c) return NAN;
    double b = 2.0 * 4.0 * state_planes(c->prm.storage, c->prm.rho0);
    if (c->force_mode == MDF_FORCE_FIELD) b += 8.0;
    if (c->args.force_mode_d == MDF_FORCE_FIELD && c->args.Fxdp != c->args.Fxp) b += 8.0;
    if (c->args.r_mode == MDF_FORCE_FIELD) b += 4.0;
    if (c->kind == MDF_GRID_CURVILINEAR) b += 16.0;
    return b;
}

}  // extern "C"
