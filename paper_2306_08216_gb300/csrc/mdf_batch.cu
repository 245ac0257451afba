// mdf_batch.cu -- many MDF-FDLBM problems stepped by one persistent launch.
//
// Each problem of a batch is an ordinary context (mdf_create: its own state
// buffers, metrics, forcing and residual snapshot), so every single-problem
// call (mdf_fields, mdf_get_distributions, mdf_residual, ...) works on it.
// mdf_batch_step advances all of them together: one launch per time step of
// a persistent kernel whose blocks walk a table of work items ordered
// largest problem first, with the problems' arguments (and TMA descriptors)
// in global memory: either marches (problem, strip, band: walls_batch_kernel
// or batch_kernel) or tiles (problem, tile x, tile y: tile_batch_kernel).
// The batch times both at creation and keeps the faster.  Repeated steps are
// replayed from captured CUDA graphs of kGraphSteps launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mdf_ctx.cuh"

using namespace mdf;

namespace {
constexpr int kBandRows = 128;    // longest band (rows per work item)
constexpr int kGraphSteps = 16;   // launches per captured graph (even: parity returns)
}  // namespace

struct mdf_batch {
    int count = 0;
    std::vector<mdf_ctx *> ctx;
    int metric = 0, power_law = 0, walls = 0;
    StepArgs *d_args[2] = {nullptr, nullptr};      // per parity: fout = the other buffer
    CUtensorMap *d_maps[2] = {nullptr, nullptr};   // per parity: maps of the input buffer
    BatchItem *d_items = nullptr;
    int nt = 0;                                    // block size of the march kernel (strips of nt - 8 columns)
    int nitems = 0, grid = 0, occ = 0, smem = 0;
    int tile = 0, occ_tile = 0, smem_tile = 0;     // tile mode: one work item per 16 x 16 tile
    int roll = 0;                                  // march mode: the rolled register-window march
    int pinned = 0;                                // mode set by mdf_batch_set_launch (no re-timing)
    int storage = 0;                               // StorageKind of every problem (16-bit: tile mode only)
    int forced = 0;                                // some problem has a force, force rate or source
    int cur = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cstream = nullptr;                // capture / replay stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double *h_res = nullptr;                       // pinned, 5 doubles per problem
    std::vector<int> H;                            // rows per work item of each problem
    std::vector<int> seen_version;                 // args_version of each context last uploaded
    std::vector<char> active;                      // problems that step (mdf_batch_set_active)
    std::vector<CUtensorMap> h_maps[2];            // host copies of d_maps
    int num_sms = 0, items_cap = 0;
    long long steps = 0;
    long long nodes = 0;
    char last_error[256] = {0};
};

static thread_local char g_batch_error[256] = {0};

static mdf_status bfail(mdf_batch *b, mdf_status st, const char *fmt, ...) {
    char *dst = b ? b->last_error : g_batch_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

#define BCK(b, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? MDF_E_NOMEM : MDF_E_CUDA,       \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

static void free_batch(mdf_batch *b) {
    if (!b) return;
    for (int p = 0; p < 2; ++p) {
        if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
        if (b->d_args[p]) cudaFree(b->d_args[p]);
        if (b->d_maps[p]) cudaFree(b->d_maps[p]);
    }
    if (b->d_items) cudaFree(b->d_items);
    if (b->h_res) cudaFreeHost(b->h_res);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->cstream) cudaStreamDestroy(b->cstream);
    for (mdf_ctx *c : b->ctx) mdf_destroy(c);
    delete b;
}

// Upload the per-problem argument tables (both parities) from the contexts.
static mdf_status upload_args(mdf_batch *b) {
    std::vector<StepArgs> args;
    try {
        args.resize(b->count);
    } catch (const std::bad_alloc &) {
        return bfail(b, MDF_E_NOMEM, "host allocation of the argument table failed");
    }
    for (int p = 0; p < 2; ++p) {
        for (int i = 0; i < b->count; ++i) {
            mdf_ctx *c = b->ctx[i];
            StepArgs a = c->args;
            a.W = b->nt - 8;
            a.H = b->H[i];
            a.fout = c->buf[1 - p];
            a.fin = c->buf[p];
            a.err = b->ctx[0]->err;  // one fault word for the whole batch
            args[i] = a;
        }
        BCK(b, cudaMemcpy(b->d_args[p], args.data(), b->count * sizeof(StepArgs), cudaMemcpyHostToDevice));
    }
    for (int i = 0; i < b->count; ++i) b->seen_version[i] = b->ctx[i]->args_version;
    int forced = 0;
    for (int i = 0; i < b->count; ++i) {
        const StepArgs &a = b->ctx[i]->args;
        forced |= (a.force_mode || a.force_mode_d || a.r_mode) ? 1 : 0;
    }
    if (forced != b->forced) {
        // the captured graphs launch the other kernel variant
        for (int p = 0; p < 2; ++p) {
            if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
            b->graph[p] = nullptr;
        }
        b->forced = forced;
    }
    return MDF_OK;
}

static cudaError_t launch_one(mdf_batch *b, int parity, cudaStream_t st) {
    if (b->tile)
        return tile_batch_launch(b->d_items, b->nitems, b->d_args[parity], b->metric, b->power_law, b->walls,
                                 b->storage, b->grid, st);
    return batch_launch(b->d_items, b->nitems, b->d_args[parity], b->d_maps[parity], b->metric, b->power_law,
                        b->walls, b->grid, b->forced, b->roll, b->storage, st);
}

static mdf_status launch_steps(mdf_batch *b, cudaStream_t st, int n) {
    for (int i = 0; i < n; ++i) {
        BCK(b, launch_one(b, b->cur, st));
        b->cur ^= 1;
    }
    return MDF_OK;
}

static mdf_status build_graph(mdf_batch *b, int parity) {
    const int saved = b->cur;
    b->cur = parity;
    BCK(b, cudaStreamBeginCapture(b->cstream, cudaStreamCaptureModeThreadLocal));
    mdf_status s = launch_steps(b, b->cstream, kGraphSteps);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cstream, &g);
    b->cur = saved;
    if (s != MDF_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return bfail(b, MDF_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, MDF_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MDF_OK;
}

// Work items of the active problems, largest problems first, with band
// heights sized to the active work: a band of H rows costs H + 9 row
// iterations (halo), so long bands are cheapest when there is enough work to
// fill every resident block; a small batch instead gets bands short enough
// that its items cover the grid (one item per block, at least 2 rows).
static mdf_status build_items(mdf_batch *b) {
    const int count = b->count;
    const int W = b->nt - 8;
    long long strip_rows = 0;
    for (int i = 0; i < count; ++i)
        if (b->active[i]) strip_rows += (long long)((b->ctx[i]->nx + W - 1) / W) * b->ctx[i]->ny;
    const long long slots = (long long)std::max(1, b->occ) * b->num_sms;
    const int band_target = (int)std::max(2ll, std::min((long long)kBandRows, (strip_rows + slots - 1) / slots));
    for (int i = 0; i < count; ++i) {
        const int ny = b->ctx[i]->ny;
        const int bands = (ny + band_target - 1) / band_target;
        int H = (ny + bands - 1) / bands;
        if (H < 2) H = 2;
        b->H[i] = H;
    }
    std::vector<int> order;
    std::vector<BatchItem> items;
    try {
        for (int i = 0; i < count; ++i)
            if (b->active[i]) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (long long)b->ctx[x]->nx * b->ctx[x]->ny > (long long)b->ctx[y]->nx * b->ctx[y]->ny;
        });
        for (int i : order) {
            mdf_ctx *c = b->ctx[i];
            const int tw = b->tile ? TILE_X : W, th = b->tile ? TILE_Y : b->H[i];
            const int gx = (c->nx + tw - 1) / tw;
            const int gy = (c->ny + th - 1) / th;
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) items.push_back(BatchItem{i, bx, by, 0});
        }
    } catch (const std::bad_alloc &) {
        return bfail(b, MDF_E_NOMEM, "host allocation of the work items failed");
    }
    b->nitems = (int)items.size();
    b->grid = std::min(b->nitems, std::max(1, b->tile ? b->occ_tile : b->occ) * b->num_sms);
    if (b->nitems > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        BCK(b, cudaMalloc(&b->d_items, items.size() * sizeof(BatchItem)));
        b->items_cap = b->nitems;
    }
    if (b->nitems)
        BCK(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    for (int p = 0; p < 2; ++p) {
        if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
        b->graph[p] = nullptr;
    }
    return MDF_OK;
}

// Time a few steps of each kernel over the active problems (their current
// buffers are read and the other ones written, so the states are unchanged;
// the batch's streams must be idle): the register-window march unrolled or
// rolled (the same values; the faster is kept: the rolled one wins on a
// full GPU, where the unrolled body misses the instruction cache, the
// unrolled one on a few small problems, where row latency decides), and
// the tile kernel, kept only when more than 10 % faster than the better
// march (its last bits differ).  Run at creation and whenever the active
// set changes: a batch whose remaining problems are few and small steps
// faster by tiles than by the long serial bands of a march.
static mdf_status choose_kernel(mdf_batch *b) {
    struct Mode {
        int tile, roll;
    };
    Mode modes[3];
    int nm = 0;
    if (b->storage == MDF_STORAGE_FP32) modes[nm++] = Mode{0, 0};
    if (b->metric != METRIC_CURVILINEAR) modes[nm++] = Mode{0, 1};
    if (b->occ_tile >= 1) modes[nm++] = Mode{1, 0};
    if (nm == 0) return bfail(b, MDF_E_INVALID, "no batch kernel serves this problem set");
    if (nm == 1) {
        b->tile = modes[0].tile;
        b->roll = modes[0].roll;
        return build_items(b);
    }
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    float best[3] = {1e30f, 1e30f, 1e30f};
    const int parity = b->cur;
    for (int pass = 0; pass < 2; ++pass)
        for (int m = 0; m < nm; ++m) {
            b->tile = modes[m].tile;
            b->roll = modes[m].roll;
            mdf_status s = build_items(b);
            if (s != MDF_OK) return s;
            BCK(b, launch_one(b, parity, b->stream));
            BCK(b, cudaEventRecord(e0, b->stream));
            for (int r = 0; r < 4; ++r) BCK(b, launch_one(b, parity, b->stream));
            BCK(b, cudaEventRecord(e1, b->stream));
            BCK(b, cudaEventSynchronize(e1));
            float ms = 0.0f;
            BCK(b, cudaEventElapsedTime(&ms, e0, e1));
            best[m] = std::min(best[m], ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the better march, then the tiles if more than 10 % faster than it (or
    // the tiles alone)
    int pick = -1;
    for (int m = 0; m < nm; ++m)
        if (!modes[m].tile && (pick < 0 || best[m] < best[pick])) pick = m;
    for (int m = 0; m < nm; ++m)
        if (modes[m].tile && (pick < 0 || best[m] < 0.9f * best[pick])) pick = m;
    b->tile = modes[pick].tile;
    b->roll = modes[pick].roll;
    return build_items(b);
}

extern "C" {

mdf_status mdf_batch_create(int count, const mdf_grid *grids, const mdf_fluid *fluids, const mdf_bc *bcs,
                            const mdf_params *params, mdf_batch **out) {
    if (!out) return bfail(nullptr, MDF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (count < 1 || !grids || !fluids || !bcs) return bfail(nullptr, MDF_E_INVALID, "count >= 1 and arrays required");
    // one kernel variant serves the whole batch
    const int metric = grids[0].kind;
    const int power_law = fluids[0].power_law ? 1 : 0;
    const int walls = (bcs[0].type[0] == MDF_BC_WALL || bcs[0].type[2] == MDF_BC_WALL) ? 1 : 0;
    const int storage = params ? params[0].storage : MDF_STORAGE_FP32;
    for (int i = 0; i < count && params; ++i) {
        if (params[i].storage != storage)
            return bfail(nullptr, MDF_E_INVALID, "problem %d: every problem of a batch has the same storage mode", i);
        if (params[i].rho0) return bfail(nullptr, MDF_E_INVALID, "problem %d: batches do not evolve rho_0", i);
    }
    for (int i = 1; i < count; ++i) {
        const int w = (bcs[i].type[0] == MDF_BC_WALL || bcs[i].type[2] == MDF_BC_WALL) ? 1 : 0;
        if (grids[i].kind != metric || (fluids[i].power_law ? 1 : 0) != power_law || w != walls)
            return bfail(nullptr, MDF_E_INVALID,
                         "problem %d differs from problem 0 in grid kind, fluid model or wall/periodic type", i);
    }
    // host allocations never throw across the C ABI
    mdf_batch *b = new (std::nothrow) mdf_batch();
    if (!b) return bfail(nullptr, MDF_E_NOMEM, "host allocation of the batch failed");
    b->count = count;
    b->metric = metric;
    b->power_law = power_law;
    b->walls = walls;
    b->storage = storage;
#define BCKC(call)                                          \
    do {                                                    \
        mdf_status s_ = (call);                             \
        if (s_ != MDF_OK) {                                 \
            strncpy(g_batch_error, b->last_error, 255);     \
            free_batch(b);                                  \
            return s_;                                      \
        }                                                   \
    } while (0)
#define BCKE(call) BCKC(([&]() -> mdf_status { BCK(b, call); return MDF_OK; })())
    try {
        b->ctx.reserve(count);
        b->H.resize(count);
        b->seen_version.resize(count);
        b->active.assign(count, 1);
        for (int p = 0; p < 2; ++p) b->h_maps[p].resize(count);
    } catch (const std::bad_alloc &) {
        bfail(b, MDF_E_NOMEM, "host allocation of the batch tables failed");
        BCKC(MDF_E_NOMEM);
    }
    for (int i = 0; i < count; ++i) {
        mdf_ctx *c = nullptr;
        mdf_status s = ctx_create_untuned(&grids[i], &fluids[i], &bcs[i], params ? &params[i] : nullptr, &c);
        if (s != MDF_OK) {
            bfail(b, s, "problem %d: %s", i, mdf_last_error(nullptr));
            BCKC(s);
        }
        b->ctx.push_back(c);
        b->nodes += (long long)c->nx * c->ny;
    }
    int num_sms = 0, dev = 0;
    BCKE(batch_occupancy(metric, power_law, walls, storage, &b->nt, &b->occ, &b->smem));
    BCKE(cudaGetDevice(&dev));
    BCKE(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    b->num_sms = num_sms;
    for (int i = 0; i < count; ++i) {
        CUtensorMap m[2];
        BCKC(ctx_encode_maps(b->ctx[i], b->nt, m));
        for (int p = 0; p < 2; ++p) b->h_maps[p][i] = m[p];
    }
    BCKC(build_items(b));
    for (int p = 0; p < 2; ++p) {
        BCKE(cudaMalloc(&b->d_args[p], count * sizeof(StepArgs)));
        BCKE(cudaMalloc(&b->d_maps[p], count * sizeof(CUtensorMap)));
        BCKE(cudaMemcpy(b->d_maps[p], b->h_maps[p].data(), count * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    }
    BCKC(upload_args(b));
    BCKE(tile_batch_occupancy(metric, power_law, walls, storage, &b->occ_tile, &b->smem_tile));
    if (storage != MDF_STORAGE_FP32 && metric == METRIC_CURVILINEAR) {
        // the curvilinear march keeps FP32 storage
        if (b->occ_tile < 1) BCKC(bfail(b, MDF_E_INVALID, "the tile kernel does not fit"));
        b->tile = 1;
        BCKC(build_items(b));
    } else {
        BCKC(choose_kernel(b));
    }
    BCKE(cudaMallocHost(&b->h_res, (size_t)count * 5 * sizeof(double)));
    BCKE(cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking));
    BCKE(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    BCKE(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    *out = b;
    return MDF_OK;
#undef BCKE
#undef BCKC
}

void mdf_batch_destroy(mdf_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    cudaStreamSynchronize(b->cstream);
    free_batch(b);
}

mdf_status mdf_batch_set_stream(mdf_batch *b, void *stream) {
    if (!b) return MDF_E_INVALID;
    b->stream = (cudaStream_t)stream;
    for (mdf_ctx *c : b->ctx) c->stream = b->stream;
    return MDF_OK;
}

mdf_status mdf_batch_problem(mdf_batch *b, int index, mdf_ctx **ctx) {
    if (!b || !ctx || index < 0 || index >= b->count) return b ? bfail(b, MDF_E_INVALID, "bad index") : MDF_E_INVALID;
    *ctx = b->ctx[index];
    return MDF_OK;
}

mdf_status mdf_batch_init_fields(mdf_batch *b, int index, const float *u, const float *v, const float *p,
                                 int on_device) {
    if (!b || index < 0 || index >= b->count) return b ? bfail(b, MDF_E_INVALID, "bad index") : MDF_E_INVALID;
    if (b->steps != 0 || b->cur != 0)
        return bfail(b, MDF_E_STATE, "initial fields are set before the batch takes its first step");
    mdf_status s = mdf_init_fields(b->ctx[index], u, v, p, on_device);
    if (s != MDF_OK) bfail(b, s, "problem %d: %s", index, mdf_last_error(b->ctx[index]));
    return s;
}

mdf_status mdf_batch_step(mdf_batch *b, int n) {
    if (!b) return MDF_E_INVALID;
    MdfRange r("mdf_batch_step");
    if (n < 0) return bfail(b, MDF_E_INVALID, "n must be >= 0");
    // arguments changed since the last upload (forcing set on a problem)?
    for (int i = 0; i < b->count; ++i)
        if (b->seen_version[i] != b->ctx[i]->args_version) {
            BCK(b, cudaStreamSynchronize(b->stream));
            BCK(b, cudaStreamSynchronize(b->cstream));
            mdf_status s = upload_args(b);
            if (s != MDF_OK) return s;
            break;
        }
    if (b->nitems == 0) return MDF_OK;  // every problem retired
    int done = 0;
    const int reps = n / kGraphSteps;
    if (reps >= 2) {
        // replay captured graphs on the capture stream, ordered after and
        // before the batch stream by events
        if (!b->graph[b->cur]) {
            mdf_status s = build_graph(b, b->cur);
            if (s != MDF_OK) return s;
        }
        BCK(b, cudaEventRecord(b->ev_in, b->stream));
        BCK(b, cudaStreamWaitEvent(b->cstream, b->ev_in, 0));
        for (int r = 0; r < reps; ++r) BCK(b, cudaGraphLaunch(b->graph[b->cur], b->cstream));
        BCK(b, cudaEventRecord(b->ev_out, b->cstream));
        BCK(b, cudaStreamWaitEvent(b->stream, b->ev_out, 0));
        done = reps * kGraphSteps;  // even: the parity is unchanged
    }
    mdf_status s = launch_steps(b, b->stream, n - done);
    if (s != MDF_OK) return s;
    b->steps += n;
    for (int i = 0; i < b->count; ++i)
        if (b->active[i]) {
            b->ctx[i]->cur = b->cur;
            b->ctx[i]->steps += n;
        }
    return MDF_OK;
}

mdf_status mdf_batch_set_active(mdf_batch *b, int index, int active) {
    if (!b || index < 0 || index >= b->count) return b ? bfail(b, MDF_E_INVALID, "bad index") : MDF_E_INVALID;
    active = active ? 1 : 0;
    if (b->active[index] == active) return MDF_OK;
    BCK(b, cudaStreamSynchronize(b->stream));
    BCK(b, cudaStreamSynchronize(b->cstream));
    mdf_ctx *c = b->ctx[index];
    if (active && c->cur != b->cur) {
        // the batch reads buffer `cur` of every problem: give this problem's
        // current state that role by exchanging its two buffers
        std::swap(c->buf[0], c->buf[1]);
        std::swap(c->tmap[0], c->tmap[1]);
        std::swap(b->h_maps[0][index], b->h_maps[1][index]);
        c->cur = b->cur;
        for (int p = 0; p < 2; ++p)
            BCK(b, cudaMemcpy(b->d_maps[p] + index, &b->h_maps[p][index], sizeof(CUtensorMap),
                              cudaMemcpyHostToDevice));
    }
    b->active[index] = (char)active;
    mdf_status s = build_items(b);
    if (s != MDF_OK) return s;
    s = upload_args(b);
    if (s != MDF_OK) return s;
    if (!b->pinned && (b->storage == MDF_STORAGE_FP32 || b->metric != METRIC_CURVILINEAR) && b->nitems > 0)
        s = choose_kernel(b);
    return s;
}

mdf_status mdf_batch_residual(mdf_batch *b, double *residual, int *status) {
    if (!b || !residual) return b ? bfail(b, MDF_E_INVALID, "residual is NULL") : MDF_E_INVALID;
    MdfRange rr("mdf_batch_residual");
    for (int i = 0; i < b->count; ++i) {
        if (!b->active[i]) continue;
        mdf_ctx *c = b->ctx[i];
        BCK(b, aux_residual(c->aux, c->buf[c->cur], c->snap_u, c->snap_v, c->partials, c->result, b->stream));
        BCK(b, cudaMemcpyAsync(b->h_res + 5 * i, c->result, 5 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    }
    mdf_status s = ctx_wait(b->ctx[0], 0);
    if (s != MDF_OK) return bfail(b, s, "%s", mdf_last_error(b->ctx[0]));
    int any_diverged = 0;
    for (int i = 0; i < b->count; ++i) {
        if (!b->active[i]) {
            residual[i] = NAN;
            if (status) status[i] = MDF_E_STATE;
            continue;
        }
        mdf_ctx *c = b->ctx[i];
        const double *r = b->h_res + 5 * i;
        const long long window = c->steps - c->snap_step;
        c->snap_step = c->steps;
        residual[i] = window > 0 ? sqrt(r[0]) / ((double)window * sqrt(r[1])) : NAN;
        int st = MDF_OK;
        if (r[4] > 0 || !isfinite(r[2]) || !isfinite(r[3])) st = MDF_E_DIVERGED;
        else if (window <= 0) st = MDF_E_STATE;
        if (status) status[i] = st;
        any_diverged |= st == MDF_E_DIVERGED;
    }
    return any_diverged ? bfail(b, MDF_E_DIVERGED, "at least one problem diverged") : MDF_OK;
}

mdf_status mdf_batch_info(const mdf_batch *b, long long info[6]) {
    if (!b || !info) return MDF_E_INVALID;
    info[0] = b->count;
    info[1] = b->nitems;
    info[2] = b->grid;
    info[3] = b->occ;
    info[4] = b->nodes;
    info[5] = b->steps;
    return MDF_OK;
}

mdf_status mdf_batch_set_launch(mdf_batch *b, int kind) {
    if (!b) return MDF_E_INVALID;
    if (kind < 0 || kind > 2)
        return bfail(b, MDF_E_INVALID, "kind must be 0 (march), 1 (tile) or 2 (rolled march)");
    if (kind == 1 && b->occ_tile < 1) return bfail(b, MDF_E_INVALID, "the tile kernel does not fit");
    if (kind == 0 && b->storage != MDF_STORAGE_FP32)
        return bfail(b, MDF_E_INVALID, "with 16-bit storage the march of a batch runs in rolled form (kind 2)");
    if (kind == 2 && b->metric == METRIC_CURVILINEAR)
        return bfail(b, MDF_E_INVALID, "the rolled march serves uniform and separable grids");
    BCK(b, cudaStreamSynchronize(b->stream));
    BCK(b, cudaStreamSynchronize(b->cstream));
    b->tile = kind == 1 ? 1 : 0;
    b->roll = kind == 2 ? 1 : 0;
    b->pinned = 1;
    return build_items(b);
}

int mdf_batch_launch_kind(const mdf_batch *b) { return b ? (b->tile ? 1 : (b->roll ? 2 : 0)) : -1; }

const char *mdf_batch_last_error(const mdf_batch *b) { return b ? b->last_error : g_batch_error; }

}  // extern "C"
