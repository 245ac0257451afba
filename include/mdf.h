/*
 * mdf.h -- C ABI of the GB300 MDF-FDLBM library (libmdf.so).
 *
 * The library advances the multiple-distribution-function finite-difference
 * lattice Boltzmann method (MDF-FDLBM) of Chen, Chai, Zhao and Shi
 * (arXiv:2306.08216) for the 2-D incompressible Navier-Stokes equations
 * written as convection-diffusion equations (Sec. 2.1, Eq. 2.1.2), on one GPU.
 * One time step is Steps (1)-(4) of Sec. 2.2 with the simplified evolution
 * equations of Remark 2 (Eqs. 2.3.24-2.3.25), the D2Q5 lattice of Sec. 3.1
 * (Eq. 3.1.0), the MRT collision of Eq. 2.2.4 with s0 = s3 = s4 = s',
 * s1 = s2 = s (Sec. 3.1), the linear equilibrium of Eq. 2.2.5, the mixed
 * central/upwind differences of Eqs. 2.2.12-2.2.13 and the time step of
 * Eq. 3.1.  The state is the two distributions fhat_{j,alpha}, alpha = u, v;
 * the alpha = 0 distribution (rho_0, Eq. 2.1.2), which feeds back into
 * neither u nor P (Remark 1), is evolved beside them when
 * mdf_params.rho0 is set.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an mdf_status; the library never aborts, exits or
 *    traps on the device.  mdf_last_error() gives a one-line reason.
 *  - Input arrays are copied; the caller keeps ownership.  Output arrays are
 *    owned by the caller.  `on_device` = 1 means the pointer is CUDA device
 *    memory of the current device, 0 means host memory.
 *  - Field arrays are FP32, row-major [ny][nx] (x fastest), unless stated.
 *  - Device work is enqueued on the stream set by mdf_set_stream (default:
 *    the legacy default stream) and is asynchronous unless stated.
 *  - A context belongs to the device that was current at mdf_create; calls
 *    must be made with that device current.  A context (or batch) is not
 *    thread-safe: use it from one host thread at a time.  Different contexts
 *    may be created and stepped from different threads at once.
 */
#ifndef MDF_H
#define MDF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdf_ctx mdf_ctx; /* opaque, library-owned */

typedef enum {
    MDF_OK = 0,
    MDF_E_INVALID = 1,  /* bad argument; nothing was changed */
    MDF_E_CUDA = 2,     /* a CUDA runtime/driver call failed */
    MDF_E_NOMEM = 3,    /* device or host allocation failed */
    MDF_E_DIVERGED = 4, /* NaN/Inf found in the velocity field */
    MDF_E_TIMEOUT = 5,  /* a host wait or a bounded device wait ran out */
    MDF_E_STATE = 6     /* call not valid in the current state */
} mdf_status;

enum { MDF_GRID_UNIFORM = 0, MDF_GRID_SEPARABLE = 1, MDF_GRID_CURVILINEAR = 2 };
enum { MDF_BC_PERIODIC = 0, MDF_BC_WALL = 1 };
enum { MDF_FORCE_NONE = 0, MDF_FORCE_CONSTANT = 1, MDF_FORCE_FIELD = 2 };

/* Grid (Eq. 2.2.13 spacings; Sec. 4.2 anisotropic grids; coordinate
 * transformation for the keyword of the abstract).
 *  nx, ny  nodes per axis (>= 5: the stencil reaches two nodes each way).
 *  kind    MDF_GRID_UNIFORM: spacing lx/nx on a periodic axis, lx/(nx-1) on
 *          a walled axis (walls sit on the first and last node);
 *          MDF_GRID_SEPARABLE: node coordinates x[nx], y[ny] (FP64);
 *          MDF_GRID_CURVILINEAR: node coordinates x[ny*nx], y[ny*nx] (FP64,
 *          row-major) of a body-fitted grid; the library forms the metric
 *          coefficients xi_x, xi_y, eta_x, eta_y in FP64 on the GPU from
 *          second-order differences of the coordinates.
 *  lx, ly  extent (uniform) or period of a periodic axis (other kinds). */
typedef struct {
    int nx, ny;
    int kind;
    double lx, ly;
    const double *x, *y;
} mdf_grid;

/* Fluid (Eq. 2.1.1).  Newtonian: nu > 0, relaxation rate s = cs^2/nu
 * (Sec. 2.3).  power_law != 0: nu = K gdot^(n-1), gdot = sqrt(2 S:S) with S
 * from the non-equilibrium first moment (Eqs. 2.4.1, 2.4.3), solved per node
 * every step and clamped to [nu_min, nu_max]; `nu` must still be > 0 and
 * is then unused. */
typedef struct {
    double nu;
    int power_law;
    double K, n;
    double nu_min, nu_max;
} mdf_fluid;

/* Boundaries, sides ordered west, east, south, north.  type: MDF_BC_PERIODIC
 * or MDF_BC_WALL (non-equilibrium extrapolation velocity wall, Secs. 4.3-4.4);
 * both sides of an axis must have the same type.  Corner nodes take the
 * west/east wall velocity. */
typedef struct {
    int type[4];
    double u_wall[4], v_wall[4];
} mdf_bc;

/* Scheme parameters: lattice speed c (= |c_j|, Eq. 3.1.0), CFL number
 * (Eq. 3.1, 0 < cfl < 1), mixed-scheme weight eta (Eq. 2.2.12, 0..1) and the
 * ratio s'/s of the free rates (Sec. 4 uses 1.5).  A NULL params pointer
 * selects c = 1, cfl = 0.5, eta = 0.8, s_ratio = 1.5, FP32 storage and no
 * alpha = 0 distribution.
 *
 * storage selects how the state is kept in device memory between steps (the
 * arithmetic is FP32 in every mode; the paper stores fhat in full
 * precision, the 16-bit modes have no counterpart there):
 *   MDF_STORAGE_FP32  the 10 distributions fhat_{alpha,j} in FP32 (40 B/node)
 *   MDF_STORAGE_FP16  u, v, P (Eqs. 2.3.5-2.3.7) in FP32 and the
 *   MDF_STORAGE_BF16  non-equilibrium parts fhat_{alpha,j} - feq_{alpha,j}
 *                     of j = 1..4 in FP16 / BF16 (j = 0 follows, since the
 *                     non-equilibrium part carries no zeroth moment),
 *                     scaled by the power of two 2^(12 - floor(log2 c)):
 *                     28 B/node.  Periodic Newtonian problems on uniform or
 *                     separable grids step on the fast path; every other
 *                     problem (walls, power law, curvilinear grids) on the
 *                     tile kernel (see mdf_set_launch), also in batches;
 *                     not with the alpha = 0 distribution.  Rounding
 *                     the non-equilibrium part perturbs each step by at most
 *                     2^-11 (FP16) or 2^-8 (BF16) of |fhat - feq|; in FP16
 *                     a non-equilibrium part above about 16 c overflows and
 *                     the next residual reports MDF_E_DIVERGED.
 * The distribution and field calls convert, so their layouts do not depend
 * on the storage mode; checkpoints of the 16-bit modes hold the raw device
 * buffer (see mdf_save). */
enum { MDF_STORAGE_FP32 = 0, MDF_STORAGE_FP16 = 1, MDF_STORAGE_BF16 = 2 };
/*
 * rho0 != 0 also evolves the alpha = 0 distribution of Eq. 2.1.2
 * (ubar_0 = rho_0, E_0 = 0, so feq_{j,0} = w_j (rho_0 + c_j.(rho_0 u)/cs^2),
 * source F_{j,0} = w_j R) with the same Steps (1)-(4), rates and stencils,
 * u taken from the alpha = 1, 2 moments of the same stage.  Remark 1: it
 * feeds back into neither u nor P, so the alpha = 1, 2 results do not change.
 * Walls: non-equilibrium extrapolation with the wall's rho_0 equal to the
 * interior neighbour's (the paper leaves the alpha = 0 wall condition open).
 * The state grows to 15 FP32 planes (60 B/node); every grid kind has a
 * kernel with the lane (periodic Newtonian problems the register-window
 * march, the others the shared-ring march, all of them the tile kernel).
 * FP32 storage only, and batches reject it (MDF_E_INVALID).
 * mdf_init_fields starts it at rho_0 = 1. */
typedef struct {
    double c, cfl, eta, s_ratio;
    int storage;
    int rho0;
} mdf_params;

/* Create a solver: validates the arguments (MDF_E_INVALID before any CUDA
 * call), allocates two state buffers (layout chosen by params->storage) on
 * the current device, forms the grid metrics and dt = cfl * dx_min / c (Eq. 3.1), and
 * sets the state to rest (u = v = p = 0).  *out receives the context. */
mdf_status mdf_create(const mdf_grid *grid, const mdf_fluid *fluid, const mdf_bc *bc,
                      const mdf_params *params, mdf_ctx **out);

/* Fault injection (host side, for tests of the error paths): with the
 * environment variable MDF_FAIL_ALLOC=k, the k-th device or pinned-host
 * allocation made while mdf_create (or mdf_batch_create, per problem) builds
 * a context fails as out of memory: the call returns MDF_E_NOMEM and frees
 * what it had allocated.  Read at every creation; unset or 0 disables it. */

/* Release every resource of the context (waits for its stream first). */
void mdf_destroy(mdf_ctx *ctx);

/* Stream for all later device work (a cudaStream_t; NULL = legacy stream). */
mdf_status mdf_set_stream(mdf_ctx *ctx, void *cuda_stream);

/* Body force F_alpha of Eq. 2.2.6 (F_{j,alpha} = w_j F_alpha).  mode:
 * MDF_FORCE_NONE, MDF_FORCE_CONSTANT (fx, fy) or MDF_FORCE_FIELD (arrays
 * Fx, Fy of nx*ny FP32, copied).  May change between steps (a time-dependent
 * force is set before every step); its time derivative is given by
 * mdf_set_force_rate. */
mdf_status mdf_set_force(mdf_ctx *ctx, int mode, double fx, double fy,
                         const float *Fx, const float *Fy, int on_device);

/* Time derivative dF_alpha/dt of the body force (same modes and layouts as
 * mdf_set_force; MDF_FORCE_NONE = 0, the default).  It enters the fhat
 * update as dt^2/2 w_j dF/dt (Eq. 2.2.1 with G dropped, Eq. 2.3.24); the
 * h^2/2 term of the fbar update is dropped (Remark 2).  The dt step then
 * reads F + dt/2 dF/dt (one extra pair of planes when either is a field). */
mdf_status mdf_set_force_rate(mdf_ctx *ctx, int mode, double dfx, double dfy,
                              const float *dFx, const float *dFy, int on_device);

/* Source R of the continuity equation div u = R (Eq. 2.1.1): mode
 * MDF_FORCE_NONE (R = 0, the default), MDF_FORCE_CONSTANT (r) or
 * MDF_FORCE_FIELD (array R of nx*ny FP32, copied).  R enters the pressure of
 * Eq. 2.3.23, P = (sum c f + (cs^2/s) R - |u|^2)/2, which is stated for f;
 * computed from fhat (Step 1) and fbar (Step 3), whose non-equilibrium
 * first moments are (1 + dt s/2) and (1 + h s/2) times that of f
 * (Eqs. 2.2.2, 2.2.16), the term becomes (nu + cs^2 dt/2) R / 2 and
 * (nu + cs^2 h/2) R / 2.  Newtonian fluids and FP32 storage only
 * (MDF_E_INVALID otherwise).  With params->rho0 set, R is also the source
 * w_j R of the alpha = 0 distribution (Eq. 2.1.2), added in Steps (2) and
 * (4) like the body force. */
mdf_status mdf_set_source(mdf_ctx *ctx, int mode, double r, const float *R, int on_device);

/* Metric coefficients of a curvilinear grid given by the caller, in place
 * of those mdf_create forms from second-order differences of the node
 * coordinates (the coordinate transformation of the body-fitted path; the
 * paper leaves open how the coefficients are obtained, so exact derivatives
 * of an analytic mapping may be passed).  xi_x, xi_y, eta_x, eta_y: FP64,
 * row-major [ny][nx], derivatives of the computational coordinates per unit
 * node index (xi = i, eta = j) with respect to x and y; copied.  The time
 * step keeps the value Eq. 3.1 gave from the node coordinates.  Enqueued on
 * the context's stream: steps enqueued later use the new coefficients
 * (synchronise a batch that holds the context first).  Host input is
 * checked for finite values and the call waits for the upload; device
 * input (on_device = 1) is read on the stream, so it must stay valid until
 * the stream has passed this call.  Errors:
 * MDF_E_INVALID (not a curvilinear grid, NULL arrays, non-finite values),
 * MDF_E_NOMEM, MDF_E_CUDA. */
mdf_status mdf_set_metrics(mdf_ctx *ctx, const double *xi_x, const double *xi_y, const double *eta_x,
                           const double *eta_y, int on_device);

/* Initial state fhat = feq(u, v, p) (Sec. 4: distributions start at
 * equilibrium); wall nodes take the wall velocity.  Resets the step count
 * and the residual snapshot.  With params->rho0 set, the alpha = 0
 * distribution starts at feq_{j,0}(1, u). */
mdf_status mdf_init_fields(mdf_ctx *ctx, const float *u, const float *v, const float *p,
                           int on_device);

/* The alpha = 0 distribution (contexts created with params->rho0 != 0;
 * MDF_E_INVALID otherwise).  mdf_init_rho0 sets fhat_{j,0} =
 * feq_{j,0}(rho0, u) (Eq. 2.2.5 with ubar_0 = rho_0, E_0 = 0) with rho0 an
 * nx*ny FP32 array (row-major [y][x]) and u the velocity of the current
 * state; the step count is kept.  mdf_get_rho0 writes rho_0 = sum_j
 * fhat_{j,0} (nx*ny).  mdf_get/set_rho0_distributions copy the 5 planes
 * [j][ny][nx] of fhat_{j,0}.  Host outputs are complete on return. */
mdf_status mdf_init_rho0(mdf_ctx *ctx, const float *rho0, int on_device);
mdf_status mdf_get_rho0(mdf_ctx *ctx, float *out, int on_device);
mdf_status mdf_get_rho0_distributions(mdf_ctx *ctx, float *out, int on_device);
mdf_status mdf_set_rho0_distributions(mdf_ctx *ctx, const float *in, int on_device);

/* Enqueue n time steps (Sec. 2.2 Steps (1)-(4)); one fused kernel launch per
 * step.  Asynchronous. */
mdf_status mdf_step(mdf_ctx *ctx, int n);

/* Derived fields from the current state (Sec. 2.4).  mask selects fields by
 * bit, out[] holds one nx*ny FP32 array per set bit in increasing bit order.
 * Host outputs (on_device = 0) are complete on return; each is one
 * device-to-host copy into the caller's array, at full link speed when the
 * caller's memory is pinned (page-locked), staged by the driver otherwise.
 * The same holds for the host inputs of mdf_init_fields. */
enum {
    MDF_FIELD_U = 1u << 0, MDF_FIELD_V = 1u << 1, MDF_FIELD_P = 1u << 2,        /* Eq. 2.3.23 */
    MDF_FIELD_DUDX = 1u << 3, MDF_FIELD_DUDY = 1u << 4,                          /* Eq. 2.4.1 */
    MDF_FIELD_DVDX = 1u << 5, MDF_FIELD_DVDY = 1u << 6,
    MDF_FIELD_DIV = 1u << 7,                                                     /* Eq. 2.4.2 */
    MDF_FIELD_SXX = 1u << 8, MDF_FIELD_SXY = 1u << 9, MDF_FIELD_SYY = 1u << 10,  /* Eq. 2.4.3 */
    MDF_FIELD_SIGXX = 1u << 11, MDF_FIELD_SIGXY = 1u << 12, MDF_FIELD_SIGYY = 1u << 13, /* Eq. 2.4.4 */
    MDF_FIELD_OMEGA = 1u << 14,                                                  /* Eq. 2.4.5, Omega_xy */
    MDF_FIELD_VORT = 1u << 15,                                                   /* dv/dx - du/dy */
    MDF_FIELD_NU = 1u << 16                                                      /* local viscosity */
};
mdf_status mdf_fields(mdf_ctx *ctx, unsigned mask, float *const *out, int on_device);

/* Windowed residual r = ||U^n - U^m||_2 / ((n - m) ||U^n||_2), U = (u, v) over
 * all nodes, accumulated in FP64, where m is the step of the previous call
 * (or of mdf_init_fields); then U^m := U^n.  drift[0..1] = sum of u and of v
 * over all nodes.  Synchronises the stream (bounded wait).  Returns
 * MDF_E_DIVERGED if U holds NaN/Inf, MDF_E_STATE if no step was taken since
 * the previous snapshot (r is then set to NaN). */
mdf_status mdf_residual(mdf_ctx *ctx, double *residual, double drift[2]);

/* mdf_residual in two halves, so that a march can enqueue its next steps
 * before it reads the last check: mdf_residual_start enqueues the reductions
 * of the current state against the snapshot (and takes the new snapshot) on
 * the context's stream and returns; mdf_residual_finish waits (bounded) for
 * exactly that work, not for steps enqueued after it, and returns what
 * mdf_residual would have returned at the start.  One residual may be
 * pending at a time: a second start, or a finish with none pending, is
 * MDF_E_STATE. */
mdf_status mdf_residual_start(mdf_ctx *ctx);
mdf_status mdf_residual_finish(mdf_ctx *ctx, double *residual, double drift[2]);

/* Copy of the state fhat as FP32 [2][5][ny][nx] (alpha, j, y, x). */
mdf_status mdf_get_distributions(mdf_ctx *ctx, float *out, int on_device);
/* Replace the state by `in` (same layout). */
mdf_status mdf_set_distributions(mdf_ctx *ctx, const float *in, int on_device);

/* Wait for all enqueued work, at most timeout_s seconds (<= 0: 60 s).
 * Returns MDF_E_TIMEOUT if the wait ran out or a bounded device wait gave up. */
mdf_status mdf_synchronize(mdf_ctx *ctx, double timeout_s);

/* Checkpoint: a 256-byte text header (grid size, step count, dt, plane
 * count) followed by the state.  FP32 storage: the 10 planes of
 * mdf_get_distributions, little-endian FP32, then (rho0 contexts, 15 planes)
 * the 5 of mdf_get_rho0_distributions; mdf_load requires a context of the
 * same grid size and plane count.  16-bit storage: the raw padded device buffer (header
 * adds the storage mode and row pitch), so a restart continues bitwise;
 * mdf_load then requires a context with the same grid, storage mode and
 * pitch, else MDF_E_INVALID. */
mdf_status mdf_save(mdf_ctx *ctx, const char *path);
mdf_status mdf_load(mdf_ctx *ctx, const char *path);

double mdf_dt(const mdf_ctx *ctx);                 /* time step of Eq. 3.1 */
long long mdf_steps_done(const mdf_ctx *ctx);
/* The reason for the context's last failed call; with ctx NULL, the reason
 * the calling thread's last mdf_create failed.  Valid until the next call on
 * the same context (or thread). */
const char *mdf_last_error(const mdf_ctx *ctx);

/* Launch geometry of the fused step kernel: info[0] threads per block,
 * info[1] output columns per block, info[2] rows per block, info[3] blocks in
 * x, info[4] blocks in y, info[5] dynamic shared memory bytes,
 * info[6] blocks resident per SM (occupancy query; 0 without a GPU). */
mdf_status mdf_launch_info(const mdf_ctx *ctx, int info[8]);

/* Override the launch plan the library chose (tile-shape tuning).  The step
 * has two kernel families: marches, where a block of `threads` (128, or 256
 * on uniform/separable grids) sweeps a strip of threads - 8 columns down a
 * band of `rows_per_block` (>= 1) rows, and the tile kernel (threads = 0;
 * rows_per_block is ignored), where a block of 16 x 16 threads computes one
 * 16 x 16 tile in three phases with a recomputed halo of 4 nodes: on grids
 * too small to fill the GPU with long bands it avoids the serial march
 * (every storage mode, not with the alpha = 0 distribution; the only plan
 * for 16-bit storage off the periodic fast path).  mdf_create times every
 * candidate plan for a few steps and keeps the fastest (the tile kernel only
 * if it beats the best march by more than 10 %); this call replaces that
 * choice.  Waits for the context's stream; MDF_E_INVALID for an unsupported
 * block size. */
mdf_status mdf_set_launch(mdf_ctx *ctx, int threads, int rows_per_block);

/* Kernel family of the current launch plan: 0 march, 1 tile (-1 for NULL). */
int mdf_launch_kind(const mdf_ctx *ctx);

/* Debug aid standing in for a memory checker: writes NaN (the 32-bit
 * pattern 0x7fc07fc0, NaN as FP32 and as each 16-bit half) into every
 * storage element of both state buffers, all planes, that no valid result
 * may read -- the row padding past the last ghost column and, on an x axis
 * with walls, the ghost columns (on a periodic axis they hold periodic
 * images and stay).  Steps taken afterwards must give the same results,
 * bit for bit, as without it; a result that changes or turns NaN read
 * outside its stencil.  Synchronises. */
mdf_status mdf_debug_poison(mdf_ctx *ctx);

/* Algorithmic bytes moved per node update by the fused step (state read and
 * written once, plus force/metric planes read once). */
double mdf_bytes_per_node(const mdf_ctx *ctx);

/* ---- Batches: many problems, one persistent launch per time step ----------
 *
 * A batch holds `count` independent problems (each an ordinary context with
 * its own grid, fluid, walls and scheme parameters) and advances them
 * together: each time step is ONE launch whose blocks walk a table of work
 * items (problem, strip, band), largest problems first, reading each
 * problem's arguments and TMA descriptor from device memory; repeated steps
 * are replayed from captured CUDA graphs.  All problems must share the grid
 * kind, the fluid model (Newtonian or power law) and the wall/periodic type
 * (one kernel variant); sizes, viscosities, power-law indices, wall
 * velocities and forcing may differ (mdf_set_force on a problem's context
 * takes effect at the next mdf_batch_step).  The paper itself has no
 * counterpart: it solves one problem at a time. */
typedef struct mdf_batch mdf_batch;

/* grids/fluids/bcs: `count` entries each; params: NULL or `count` entries.
 * Each problem starts at rest.  MDF_E_INVALID if the problems cannot share
 * one kernel variant, any problem is invalid (see mdf_create), the storage
 * modes differ or a problem asks for the alpha = 0 distribution.  A batch in
 * 16-bit storage steps with the rolled march or the tile kernel on uniform
 * and separable grids, with the tile kernel on curvilinear ones (see
 * mdf_batch_set_launch). */
mdf_status mdf_batch_create(int count, const mdf_grid *grids, const mdf_fluid *fluids, const mdf_bc *bcs,
                            const mdf_params *params, mdf_batch **out);
void mdf_batch_destroy(mdf_batch *batch);
mdf_status mdf_batch_set_stream(mdf_batch *batch, void *cuda_stream);
/* Initial fields of problem `index` (as mdf_init_fields); only before the
 * first batch step. */
mdf_status mdf_batch_init_fields(mdf_batch *batch, int index, const float *u, const float *v, const float *p,
                                 int on_device);
/* n time steps of every problem (asynchronous). */
mdf_status mdf_batch_step(mdf_batch *batch, int n);
/* Per-problem windowed residuals (definition of mdf_residual) into
 * residual[count] and per-problem status into status[count] (may be NULL):
 * MDF_OK, MDF_E_DIVERGED or MDF_E_STATE.  Synchronises; returns
 * MDF_E_DIVERGED if any problem diverged (the others keep running). */
mdf_status mdf_batch_residual(mdf_batch *batch, double *residual, int *status);
/* Retire (active = 0) or re-admit (active = 1) problem `index`: a retired
 * problem keeps its state and step count, takes no work in later batch
 * steps and reports MDF_E_STATE with a NaN residual from
 * mdf_batch_residual; the work items (and band heights) are rebuilt over the
 * remaining problems.  Lets a sweep stop paying for problems that have
 * converged or diverged.  Waits for the batch's streams. */
mdf_status mdf_batch_set_active(mdf_batch *batch, int index, int active);
/* The context of problem `index` (owned by the batch): use it with
 * mdf_fields, mdf_get_distributions, mdf_dt, ...; do not step or destroy it. */
mdf_status mdf_batch_problem(mdf_batch *batch, int index, mdf_ctx **ctx);
/* info[0] problems, [1] work items, [2] blocks per launch, [3] blocks per
 * SM, [4] nodes in all problems, [5] steps taken. */
mdf_status mdf_batch_info(const mdf_batch *batch, long long info[6]);
/* Kernel of the batch step: 0 marches (work items are strips x bands of
 * each problem), 1 tiles (work items are the 16 x 16 tiles of each
 * problem, the tile kernel of mdf_set_launch), 2 marches in rolled form
 * (uniform and separable grids: the same values as 0 from a body a fifth
 * the size, faster on a full GPU, slower on a few small problems; the only
 * march form with 16-bit storage).
 * mdf_batch_create times them and keeps the faster march unless the tiles
 * are more than 10 % faster, and mdf_batch_set_active times them again over
 * the problems that remain (FP32 batches); mdf_batch_set_launch fixes the
 * choice for good (waits for the batch's streams; MDF_E_INVALID for another
 * kind, a kind that does not fit or does not apply).
 * mdf_batch_launch_kind returns the current one (-1 for NULL). */
mdf_status mdf_batch_set_launch(mdf_batch *batch, int kind);
int mdf_batch_launch_kind(const mdf_batch *batch);
const char *mdf_batch_last_error(const mdf_batch *batch); /* NULL: this thread's last failed create */

/* Residual and drift with no allocation at all (the paper has no
 * counterpart; this is a service for callers that may not allocate device
 * memory -- under an allocator that owns all device memory and forbids side
 * allocations, or in a loop that must not risk an allocation failure or the
 * implicit device synchronisation of cudaMalloc/cudaFree).
 *   fhat            device, FP32 [2][5][ny][nx] (the layout of
 *                   mdf_get_distributions with on_device = 1)
 *   u_prev, v_prev  device, FP32 [ny][nx], velocity `window` steps earlier
 *                   (e.g. from mdf_fields with on_device = 1); not modified
 *   window          steps between u_prev/v_prev and fhat (>= 1)
 *   cuda_stream     stream of the current device to enqueue on (NULL =
 *                   legacy stream); asynchronous
 *   out             device, 4 doubles: residual as defined for mdf_residual,
 *                   sum of u, sum of v, count of non-finite nodes, where u, v
 *                   are the FP32 sums of the five fhat of each distribution.
 *                   For a context with FP32 storage that is the velocity
 *                   mdf_residual uses.  With FP16/BF16 storage mdf_residual
 *                   reads the stored FP32 u, v, while the fhat that
 *                   mdf_get_distributions rebuilds (feq + non-equilibrium
 *                   part) sum to them only up to FP32 rounding (a few ulp of
 *                   |u|), so the two residuals differ by about that rounding
 *                   divided by window * |U| and this one levels off near
 *                   1e-7 / window instead of falling to zero at a steady
 *                   state.
 * The only scratch is a fixed array of 160 KiB of device memory that the
 * library holds on every GPU that loads it, so nx * ny may not exceed
 * 16,777,216 (4096 x 4096): larger fields, NULL pointers or window < 1
 * return MDF_E_INVALID before anything is enqueued.  The first call on a
 * device looks up that array's device address (once per device, with that
 * device current) and keeps it; make that first call before any stream
 * capture, and make no call on a device after cudaDeviceReset of it (the
 * kept address is no longer valid).  All calls share the one array, which
 * keeps the last call's partial sums (every call overwrites the slots it
 * reads), so calls that may run at the same time on the GPU (other streams,
 * other host threads) race; serialise them.  Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call on any path. */
mdf_status mdf_residual_noalloc(const float *fhat, const float *u_prev, const float *v_prev, int nx, int ny,
                                long long window, void *cuda_stream, double *out);

#ifdef __cplusplus
}
#endif
#endif /* MDF_H */
