/*
 * mdf_oracle.c -- FP64 CPU oracle of the MDF-FDLBM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against
 * which the CUDA path is checked.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and neither includes the
 * other.
 *
 * Method: Chen, Chai, Zhao, Shi, "Multiple-distribution-function
 * finite-difference lattice Boltzmann method for incompressible
 * Navier-Stokes equation", arXiv:2306.08216.
 *
 * The step follows Sec. 2.2, Steps (1)-(4), in the paper's order and
 * notation, with the simplified evolution equations of Remark 2
 * (Eqs. 2.3.24-2.3.25):
 *   Step 1  f^+ = (I - Lambda) fhat + Lambda feq                 (Eq. 2.2.14)
 *           fbar^+ = (I - 3 Lambda/4) fhat + (3 Lambda/4) feq     (Eq. 2.2.15)
 *   Step 2  fbar(x,t+h) = fbar^+ - h c_j.grad fbar^+ + h F_j      (Eqs. 2.2.11, 2.3.25)
 *   Step 3  f(x,t+h) = (I + h/2 Lt)^-1 (fbar + h/2 Lt feq)         (Eq. 2.2.16)
 *   Step 4  fhat(t+dt) = f^+ - dt c_j.grad f(t+h) + dt F_j         (Eq. 2.3.24)
 * with Lt the MRT collision matrix (Eqs. 2.2.4, 3.1.0; rates of Sec. 3.1),
 * Lambda = I - (I - dt/2 Lt)(I + dt/2 Lt)^-1, the linear equilibrium of
 * Eq. 2.2.5, the mixed central/upwind gradient of Eqs. 2.2.12-2.2.13, the
 * pressure of Eq. 2.3.23 and the local derived quantities of
 * Eqs. 2.4.1-2.4.5.  Every matrix is formed and inverted explicitly; no
 * closed form of the collision operator is used here.
 *
 * Readings where the paper is silent (the same list is kept with the
 * design notes of the repository):
 *   - c_s^2 is the second moment of the D2Q5 weights, 2c^2/5 (Eq. 2.3.4).
 *   - MRT moment basis: e, c_x, c_y, (-4,1,1,1,1), (0,1,-1,1,-1), with
 *     s0=s3=s4=s' and s1=s2=s (Sec. 3.1).
 *   - Upwind branch for c<0 uses Pi(chi+2 dchi) as third point (typo in
 *     Eq. 2.2.13b); central part weighted by eta as in Eq. 2.2.12.
 *   - Walls: non-equilibrium extrapolation (Sec. 4.3/4.4, named only):
 *     wall value = feq(u_wall, P_nb) + (g_nb - feq(u_nb, P_nb)), with the
 *     wall-normal interior neighbour (diagonal one at corners), applied to
 *     f(t+h) after Step 3 and to fhat(t+dt) after Step 4.  Ghost values
 *     beyond a wall are linearly extrapolated, Pi(-1) = 2 Pi(0) - Pi(1).
 *     Corner nodes take the velocity of the west/east wall.
 *   - Coordinate transformation (keyword only in the paper): c.grad =
 *     ct_xi d/dxi + ct_eta d/deta on a unit computational grid, metrics from
 *     second-order differences of node coordinates, upwind by sign of ct.
 *   - Power-law fluid (keyword only): nu = K gdot^(n-1) with
 *     gdot = sqrt(2 S:S), S from the non-equilibrium first moment
 *     (Eqs. 2.4.1, 2.4.3), solved per node from fhat(t) and clamped to
 *     [nu_min, nu_max]; the rates so found serve the whole step at that node.
 *   - Source R of the continuity equation (Eq. 2.1.1) enters the
 *     pressure, P = (sum c f + (cs^2/s_1) R - |u|^2)/d (Eq. 2.3.23), with
 *     s_1 = s = cs^2/nu.  Eq. 2.3.23 is stated for f; computed from fhat or
 *     fbar, whose non-equilibrium first moments are (1 + dt s/2) and
 *     (1 + h s/2) times that of f, the R term takes the same factor
 *     (see moments_rk).  Newtonian fluids only (with a power-law viscosity
 *     nu would depend on P through the trace of the non-equilibrium moment).
 *     The G source is dropped (Remark 2).
 *   - The alpha = 0 equation (ubar_0 = rho_0, E_0 = 0, source R; Eq. 2.1.2)
 *     is evolved on request (rho0 != 0) with the same steps, rates and
 *     stencils: feq_{j,0} = w_j (rho_0 + c_j.(rho_0 u)/cs^2) with u taken
 *     from the alpha = 1, 2 moments of the same stage, source w_j R.  It
 *     feeds back into nothing (Remark 1).  Walls: non-equilibrium
 *     extrapolation with the wall's rho_0 taken equal to the neighbour's.
 *   - dF/dt enters Step 4 as dt^2/2 w_j dF/dt (Eq. 2.3.24); the h^2/2 term
 *     of the fbar update is dropped (Remark 2).  R, F and dF/dt are set by
 *     the caller (constants or fields) and may change between steps.
 * The curvilinear path is pinned on a doubly periodic non-affine map by the
 * steady periodic flow of Sec. 4.2 (second-order convergence to the closed
 * form); the differenced metrics, one-sided ones at walls included, equal
 * the analytic ones on the bilinear trapezoid and on a biquadratic map
 * (both differences are exact there).  The wall reading is pinned by plane
 * Couette flow against each of the four walls, uniform flow through a box
 * of moving walls (corners between two moving walls), mirror equivariance
 * and the wall-node identities the reading implies.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 5   /* D2Q5 (Eq. 3.1.0) */
#define NA 2  /* alpha = 1..d, d = 2; alpha = 0 is ignorable (Remark 1) */

typedef struct {
    int nx, ny;
    int grid_kind;        /* 0 uniform, 1 separable coordinates, 2 curvilinear */
    double lx, ly;        /* uniform: extent; periodic axes of kinds 1-2: period */
    const double *xc, *yc;/* kind 1: xc[nx], yc[ny]; kind 2: xc[ny*nx], yc[ny*nx] */
    double nu;
    int power_law;
    double K, n_index, nu_min, nu_max;
    int bc[4];            /* west, east, south, north: 0 periodic, 1 NEE wall */
    double u_wall[4], v_wall[4];
    double c, cfl, eta, s_ratio;
    int force_mode;       /* 0 none, 1 constant, 2 field */
    double fx, fy;
    const double *force_x, *force_y;
    int threads;
    int rho0;             /* evolve the alpha = 0 distribution */
} orc_params;

typedef struct {
    orc_params p;
    int nx, ny;
    long N;
    double cx[Q], cy[Q], w[Q], cs2;
    double dx, dy;        /* uniform spacings (kind 0) */
    double dt, h;
    double *X, *Y;        /* node coordinates (kinds 1-2) */
    double *xi_x, *xi_y, *eta_x, *eta_y;
    double *Fx, *Fy;      /* body force per node */
    double *dFx, *dFy;    /* its time derivative per node */
    double *Rs;           /* source R of Eq. 2.1.1 per node */
    double *fh, *fhp, *fbp, *fb, *f, *fn;  /* 10 planes each */
    double *s_node;       /* per-node first-moment rate s */
    double *r_fh, *r_fhp, *r_fbp, *r_fb, *r_f, *r_fn;  /* alpha = 0: Q planes each (rho0 != 0) */
    double Minv[Q][Q], M[Q][Q];
    /* constant-rate matrices (Newtonian) */
    double A[Q][Q], Ab[Q][Q], L[Q][Q], L34[Q][Q], Rinv[Q][Q], RL[Q][Q];
    long steps;
} orc_ctx;

static int g_last_status = 0;

/* ---- small dense linear algebra ------------------------------------- */

static int mat_inv(double a_in[Q][Q], double out[Q][Q]) {
    /* Gauss-Jordan elimination with partial pivoting. */
    double a[Q][2 * Q];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < 2 * Q; ++j)
            a[i][j] = j < Q ? a_in[i][j] : (j - Q == i ? 1.0 : 0.0);
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < 2 * Q; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[col][col];
        for (int j = 0; j < 2 * Q; ++j) a[col][j] /= d;
        for (int r = 0; r < Q; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m != 0.0)
                for (int j = 0; j < 2 * Q; ++j) a[r][j] -= m * a[col][j];
        }
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) out[i][j] = a[i][j + Q];
    return 0;
}

static void mat_mul(double a[Q][Q], double b[Q][Q], double out[Q][Q]) {
    double t[Q][Q];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double s = 0.0;
            for (int k = 0; k < Q; ++k) s += a[i][k] * b[k][j];
            t[i][j] = s;
        }
    memcpy(out, t, sizeof(t));
}

static void mat_vec(double a[Q][Q], const double *x, double *y) {
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += a[i][k] * x[k];
        y[i] = s;
    }
}

/* ---- MRT collision matrix (Eq. 2.2.4, Sec. 3.1 rates) ---------------- */

static void mrt_basis(orc_ctx *o) {
    /* Rows: e, c_x/c, c_y/c and two higher-order moments, mutually orthogonal. */
    static const double M[Q][Q] = {
        { 1, 1, 1, 1, 1 },
        { 0, 1, 0, -1, 0 },
        { 0, 0, 1, 0, -1 },
        { -4, 1, 1, 1, 1 },
        { 0, 1, -1, 1, -1 },
    };
    memcpy(o->M, M, sizeof(M));
    double Mc[Q][Q];
    memcpy(Mc, M, sizeof(M));
    mat_inv(Mc, o->Minv);
}

/* Lt = M^-1 S M with S = diag(s', s, s, s', s'), s' = s_ratio * s. */
static void collision_matrix(const orc_ctx *o, double s, double Lt[Q][Q]) {
    double sp = o->p.s_ratio * s;
    double S[Q] = { sp, s, s, sp, sp };
    double SM[Q][Q];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) SM[i][j] = S[i] * o->M[i][j];
    double Minv[Q][Q];
    memcpy(Minv, o->Minv, sizeof(Minv));
    mat_mul(Minv, SM, Lt);
}

/* The matrices every step needs for a given rate s:
 *   A  = I - Lambda,            L   = Lambda        (Eq. 2.2.14)
 *   Ab = I - 3 Lambda / 4,      L34 = 3 Lambda / 4  (Eq. 2.2.15)
 *   Rinv = (I + h/2 Lt)^-1,     RL  = Rinv h/2 Lt   (Eq. 2.2.16)
 * with Lambda = I - (I - dt/2 Lt)(I + dt/2 Lt)^-1 (below Eq. 2.2.14). */
static void step_matrices(const orc_ctx *o, double s,
                          double A[Q][Q], double Ab[Q][Q], double L[Q][Q],
                          double L34[Q][Q], double Rinv[Q][Q], double RL[Q][Q]) {
    double Lt[Q][Q], Ip[Q][Q], Im[Q][Q], Ipinv[Q][Q], T[Q][Q];
    collision_matrix(o, s, Lt);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double d = (i == j) ? 1.0 : 0.0;
            Ip[i][j] = d + 0.5 * o->dt * Lt[i][j];
            Im[i][j] = d - 0.5 * o->dt * Lt[i][j];
        }
    mat_inv(Ip, Ipinv);
    mat_mul(Im, Ipinv, T);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double d = (i == j) ? 1.0 : 0.0;
            L[i][j] = d - T[i][j];
            A[i][j] = d - L[i][j];
            L34[i][j] = 0.75 * L[i][j];
            Ab[i][j] = d - L34[i][j];
        }
    double Ih[Q][Q], hLt[Q][Q];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double d = (i == j) ? 1.0 : 0.0;
            hLt[i][j] = 0.5 * o->h * Lt[i][j];
            Ih[i][j] = d + hLt[i][j];
        }
    mat_inv(Ih, Rinv);
    mat_mul(Rinv, hLt, RL);
}

/* ---- moments and equilibrium --------------------------------------- */

static inline long idx(const orc_ctx *o, int a, int j, int x, int y) {
    return ((long)(a * Q + j) * o->ny + y) * o->nx + x;
}

/* Zeroth moments ubar_alpha and pressure P of Eq. 2.3.23 from a
 * distribution g.  Eq. 2.3.23 holds for f, whose non-equilibrium first
 * moment has trace -(cs^2/s) R (Eq. 2.3.22).  fhat and fbar carry that
 * moment scaled by 1 + dt s/2 and 1 + h s/2 (Eqs. 2.2.2 and 2.2.16: Lt acts
 * on the first moments with rate s), so the R term takes the same factor:
 * rk = (cs^2/s)(1 + k s/2) = nu + cs^2 k/2 with k = dt (fhat), h (fbar) or
 * 0 (f). */
static void moments_rk(const orc_ctx *o, const double *g, int x, int y, double rk,
                       double *u, double *v, double *P) {
    double ub[NA] = { 0, 0 };
    double first = 0.0;  /* sum_alpha sum_i c_{i,alpha} g_{i,alpha} */
    for (int a = 0; a < NA; ++a)
        for (int j = 0; j < Q; ++j) {
            double gj = g[idx(o, a, j, x, y)];
            ub[a] += gj;
            first += (a == 0 ? o->cx[j] : o->cy[j]) * gj;
        }
    *u = ub[0];
    *v = ub[1];
    *P = (first + rk * o->Rs[(long)y * o->nx + x] - ub[0] * ub[0] - ub[1] * ub[1]) / 2.0;  /* d = 2 */
}

/* Moments of fhat (the stored state). */
static void moments(const orc_ctx *o, const double *g, int x, int y, double *u, double *v, double *P) {
    moments_rk(o, g, x, y, o->p.nu + o->cs2 * o->dt / 2.0, u, v, P);
}

/* Eq. 2.2.5: feq_{j,alpha} = w_j [ubar_alpha + c_j.(ubar_alpha u + P E_alpha)/cs2]. */
static void equilibrium(const orc_ctx *o, double u, double v, double P,
                        double feq[NA][Q]) {
    double ub[NA] = { u, v };
    for (int a = 0; a < NA; ++a) {
        double flx = ub[a] * u + (a == 0 ? P : 0.0);
        double fly = ub[a] * v + (a == 1 ? P : 0.0);
        for (int j = 0; j < Q; ++j)
            feq[a][j] = o->w[j] * (ub[a] + (o->cx[j] * flx + o->cy[j] * fly) / o->cs2);
    }
}

/* ---- boundaries ---------------------------------------------------- */

static inline int xwall(const orc_ctx *o) { return o->p.bc[0] == 1; }
static inline int ywall(const orc_ctx *o) { return o->p.bc[2] == 1; }

static inline int is_wall(const orc_ctx *o, int x, int y) {
    if (xwall(o) && (x == 0 || x == o->nx - 1)) return 1;
    if (ywall(o) && (y == 0 || y == o->ny - 1)) return 1;
    return 0;
}

/* Non-equilibrium extrapolation at wall node (x,y) of distribution g:
 * g_w = feq(u_w, P_nb) + (g_nb - feq(u_nb, P_nb)). */
static void nee_node(const orc_ctx *o, double *g, int x, int y) {
    int nxn = x, nyn = y;
    double uw = 0.0, vw = 0.0;
    int onx = 0;
    if (xwall(o) && x == 0) { nxn = 1; uw = o->p.u_wall[0]; vw = o->p.v_wall[0]; onx = 1; }
    if (xwall(o) && x == o->nx - 1) { nxn = o->nx - 2; uw = o->p.u_wall[1]; vw = o->p.v_wall[1]; onx = 1; }
    if (ywall(o) && y == 0) {
        nyn = 1;
        if (!onx) { uw = o->p.u_wall[2]; vw = o->p.v_wall[2]; }
    }
    if (ywall(o) && y == o->ny - 1) {
        nyn = o->ny - 2;
        if (!onx) { uw = o->p.u_wall[3]; vw = o->p.v_wall[3]; }
    }
    double un, vn, Pn;
    moments(o, g, nxn, nyn, &un, &vn, &Pn);
    double feq_w[NA][Q], feq_n[NA][Q];
    equilibrium(o, uw, vw, Pn, feq_w);
    equilibrium(o, un, vn, Pn, feq_n);
    for (int a = 0; a < NA; ++a)
        for (int j = 0; j < Q; ++j)
            g[idx(o, a, j, x, y)] = feq_w[a][j] + (g[idx(o, a, j, nxn, nyn)] - feq_n[a][j]);
}

/* Eq. 2.2.5 for alpha = 0: ubar_0 = rho_0, E_0 = 0. */
static void equilibrium0(const orc_ctx *o, double rho, double u, double v, double feq[Q]) {
    for (int j = 0; j < Q; ++j) feq[j] = o->w[j] * (rho + (o->cx[j] * rho * u + o->cy[j] * rho * v) / o->cs2);
}

static double rho0_at(const orc_ctx *o, const double *r, long n) {
    double s = 0.0;
    for (int j = 0; j < Q; ++j) s += r[(long)j * o->N + n];
    return s;
}

/* Non-equilibrium extrapolation of the alpha = 0 distribution r at wall
 * node (x,y): the wall's rho_0 is the neighbour's, the velocities are the
 * wall's and the neighbour's (from the alpha = 1, 2 distribution g). */
static void nee_node0(const orc_ctx *o, double *r, const double *g, int x, int y) {
    int nxn = x, nyn = y;
    double uw = 0.0, vw = 0.0;
    int onx = 0;
    if (xwall(o) && x == 0) { nxn = 1; uw = o->p.u_wall[0]; vw = o->p.v_wall[0]; onx = 1; }
    if (xwall(o) && x == o->nx - 1) { nxn = o->nx - 2; uw = o->p.u_wall[1]; vw = o->p.v_wall[1]; onx = 1; }
    if (ywall(o) && y == 0) { nyn = 1; if (!onx) { uw = o->p.u_wall[2]; vw = o->p.v_wall[2]; } }
    if (ywall(o) && y == o->ny - 1) { nyn = o->ny - 2; if (!onx) { uw = o->p.u_wall[3]; vw = o->p.v_wall[3]; } }
    double un, vn, Pn;
    moments(o, g, nxn, nyn, &un, &vn, &Pn);
    const long nb = (long)nyn * o->nx + nxn, n = (long)y * o->nx + x;
    const double rho = rho0_at(o, r, nb);
    double fw[Q], fn[Q];
    equilibrium0(o, rho, uw, vw, fw);
    equilibrium0(o, rho, un, vn, fn);
    for (int j = 0; j < Q; ++j) r[(long)j * o->N + n] = fw[j] + (r[(long)j * o->N + nb] - fn[j]);
}

static void apply_nee0(const orc_ctx *o, double *r, const double *g) {
    if (xwall(o))
        for (int y = 0; y < o->ny; ++y) { nee_node0(o, r, g, 0, y); nee_node0(o, r, g, o->nx - 1, y); }
    if (ywall(o))
        for (int x = 0; x < o->nx; ++x) { nee_node0(o, r, g, x, 0); nee_node0(o, r, g, x, o->ny - 1); }
}

static void apply_nee(const orc_ctx *o, double *g) {
    if (xwall(o))
        for (int y = 0; y < o->ny; ++y) { nee_node(o, g, 0, y); nee_node(o, g, o->nx - 1, y); }
    if (ywall(o))
        for (int x = 0; x < o->nx; ++x) { nee_node(o, g, x, 0); nee_node(o, g, x, o->ny - 1); }
}

/* ---- mixed difference scheme (Eqs. 2.2.12-2.2.13) -------------------- */

/* Value of plane `g` (already offset to plane a,j) at index k along an axis
 * of n nodes; periodic wrap or linear extrapolation beyond a wall. */
static inline double fetch_x(const orc_ctx *o, const double *g, int k, int y) {
    int n = o->nx;
    if (!xwall(o)) { k %= n; if (k < 0) k += n; return g[(long)y * n + k]; }
    if (k < 0) return 2.0 * g[(long)y * n + 0] - g[(long)y * n + 1];
    if (k > n - 1) return 2.0 * g[(long)y * n + n - 1] - g[(long)y * n + n - 2];
    return g[(long)y * n + k];
}

static inline double fetch_y(const orc_ctx *o, const double *g, int x, int k) {
    int n = o->ny, nx = o->nx;
    if (!ywall(o)) { k %= n; if (k < 0) k += n; return g[(long)k * nx + x]; }
    if (k < 0) return 2.0 * g[(long)0 * nx + x] - g[(long)1 * nx + x];
    if (k > n - 1) return 2.0 * g[(long)(n - 1) * nx + x] - g[(long)(n - 2) * nx + x];
    return g[(long)k * nx + x];
}

/* d Pi / d chi by the mixed scheme with spacing d, upwind side chosen by the
 * sign of the advecting speed (>= 0: backward), given the five values
 * Pi(chi-2d) .. Pi(chi+2d). */
static inline double mixed_derivative(double eta, double d, double sgn_speed,
                                      const double P[5]) {
    double central = (P[3] - P[1]) / (2.0 * d);                       /* Eq. 2.2.13a */
    double upwind;
    if (sgn_speed >= 0.0)
        upwind = (3.0 * P[2] - 4.0 * P[1] + P[0]) / (2.0 * d);         /* Eq. 2.2.13b, c >= 0 */
    else
        upwind = -(3.0 * P[2] - 4.0 * P[3] + P[4]) / (2.0 * d);        /* Eq. 2.2.13b, c < 0  */
    return eta * central + (1.0 - eta) * upwind;                        /* Eq. 2.2.12 */
}

/* c_j . grad Pi at node (x,y) for plane g of population j. */
static double c_dot_grad(const orc_ctx *o, const double *g, int j, int x, int y) {
    double P[5];
    double eta = o->p.eta;
    if (o->p.grid_kind == 0) {
        double r = 0.0;
        if (o->cx[j] != 0.0) {
            for (int k = -2; k <= 2; ++k) P[k + 2] = fetch_x(o, g, x + k, y);
            r += o->cx[j] * mixed_derivative(eta, o->dx, o->cx[j], P);
        }
        if (o->cy[j] != 0.0) {
            for (int k = -2; k <= 2; ++k) P[k + 2] = fetch_y(o, g, x, y + k);
            r += o->cy[j] * mixed_derivative(eta, o->dy, o->cy[j], P);
        }
        return r;
    }
    /* Coordinate transformation: c.grad = ct_xi d/dxi + ct_eta d/deta. */
    long n = (long)y * o->nx + x;
    double ct_xi = o->cx[j] * o->xi_x[n] + o->cy[j] * o->xi_y[n];
    double ct_eta = o->cx[j] * o->eta_x[n] + o->cy[j] * o->eta_y[n];
    double r = 0.0;
    if (ct_xi != 0.0) {
        for (int k = -2; k <= 2; ++k) P[k + 2] = fetch_x(o, g, x + k, y);
        r += ct_xi * mixed_derivative(eta, 1.0, ct_xi, P);
    }
    if (ct_eta != 0.0) {
        for (int k = -2; k <= 2; ++k) P[k + 2] = fetch_y(o, g, x, y + k);
        r += ct_eta * mixed_derivative(eta, 1.0, ct_eta, P);
    }
    return r;
}

/* ---- power-law viscosity (reading of the keyword "power-law fluid") -- */

/* Solve nu = K gdot^(n-1), gdot = g / (nu + cs2 dt / 2), by Newton's method
 * on phi(nu) = nu - K (g/(nu+a))^(n-1), then clamp to [nu_min, nu_max]. */
static double power_law_nu(const orc_ctx *o, double g) {
    double K = o->p.K, n = o->p.n_index;
    double a = o->cs2 * o->dt / 2.0;
    if (n == 1.0) return fmin(fmax(K, o->p.nu_min), o->p.nu_max);
    if (g <= 0.0) return n < 1.0 ? o->p.nu_max : o->p.nu_min;
    /* Bracket [lo, hi] with phi(lo) <= 0 <= phi(hi), then safeguarded Newton. */
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 2000; ++it) {
        double phi = hi - K * pow(g / (hi + a), n - 1.0);
        if (phi >= 0.0) break;
        lo = hi; hi *= 2.0;
    }
    double nu = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double rhs = K * pow(g / (nu + a), n - 1.0);
        double phi = nu - rhs;
        if (phi > 0.0) hi = nu; else lo = nu;
        double dphi = 1.0 + (n - 1.0) * rhs / (nu + a);
        double nn = nu - phi / dphi;
        if (!(nn > lo && nn < hi)) nn = 0.5 * (lo + hi);
        if (fabs(nn - nu) <= 1e-14 * nu) { nu = nn; break; }
        nu = nn;
    }
    return fmin(fmax(nu, o->p.nu_min), o->p.nu_max);
}

/* Relaxation rate s at node (x,y) from fhat(t): Newtonian s = cs2/nu
 * (Sec. 2.3); power-law: local nu from the non-equilibrium first moment. */
static double node_rate(const orc_ctx *o, int x, int y) {
    if (!o->p.power_law) return o->cs2 / o->p.nu;
    double u, v, P, feq[NA][Q];
    moments(o, o->fh, x, y, &u, &v, &P);
    equilibrium(o, u, v, P, feq);
    double G[2][2];  /* G[beta][alpha] = sum_i c_{i,beta} (fhat - feq)_{i,alpha} */
    for (int a = 0; a < NA; ++a) {
        double gx = 0.0, gy = 0.0;
        for (int j = 0; j < Q; ++j) {
            double ne = o->fh[idx(o, a, j, x, y)] - feq[a][j];
            gx += o->cx[j] * ne;
            gy += o->cy[j] * ne;
        }
        G[0][a] = gx;
        G[1][a] = gy;
    }
    /* grad_beta u_alpha = -G[beta][alpha] / (nu + cs2 dt/2)  (Eq. 2.4.1);
     * S = sym(grad u) (Eq. 2.4.3), gdot = sqrt(2 S:S) = g / (nu + cs2 dt/2). */
    double sxx = G[0][0], syy = G[1][1], sxy = 0.5 * (G[1][0] + G[0][1]);
    double g = sqrt(2.0 * (sxx * sxx + syy * syy + 2.0 * sxy * sxy));
    return o->cs2 / power_law_nu(o, g);
}

/* ---- creation ------------------------------------------------------- */

static double *alloc0(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

/* Periodic continuation of node coordinates (kinds 1-2): crossing a periodic
 * x boundary shifts x by the period lx, crossing a periodic y boundary shifts
 * y by ly.  Walled axes are never indexed outside [0, n). */
static double coord_x(const orc_ctx *o, int i, int j) {
    int nx = o->nx, ny = o->ny;
    double off = 0.0;
    while (i < 0) { i += nx; off -= o->p.lx; }
    while (i >= nx) { i -= nx; off += o->p.lx; }
    while (j < 0) j += ny;
    while (j >= ny) j -= ny;
    return o->X[(long)j * nx + i] + off;
}
static double coord_y(const orc_ctx *o, int i, int j) {
    int nx = o->nx, ny = o->ny;
    double off = 0.0;
    while (j < 0) { j += ny; off -= o->p.ly; }
    while (j >= ny) { j -= ny; off += o->p.ly; }
    while (i < 0) i += nx;
    while (i >= nx) i -= nx;
    return o->Y[(long)j * nx + i] + off;
}

/* d/dxi (dir 0) or d/deta (dir 1) of a coordinate field by second-order
 * central differences, one-sided second order at walls. */
static double coord_deriv(const orc_ctx *o, double (*cf)(const orc_ctx *, int, int),
                          int dir, int i, int j) {
    int n = dir == 0 ? o->nx : o->ny;
    int k = dir == 0 ? i : j;
    int wall = dir == 0 ? xwall(o) : ywall(o);
#define CF(dk) (dir == 0 ? cf(o, i + (dk), j) : cf(o, i, j + (dk)))
    if (wall && k == 0) return (-3.0 * CF(0) + 4.0 * CF(1) - CF(2)) / 2.0;
    if (wall && k == n - 1) return (3.0 * CF(0) - 4.0 * CF(-1) + CF(-2)) / 2.0;
    return (CF(1) - CF(-1)) / 2.0;
#undef CF
}

orc_ctx *orc_create(const orc_params *p) {
    g_last_status = 0;
    if (!p || p->nx < 5 || p->ny < 5 || !(p->nu > 0.0) || !(p->cfl > 0.0) ||
        !(p->cfl < 1.0) || p->eta < 0.0 || p->eta > 1.0 || !(p->c > 0.0) ||
        p->bc[0] != p->bc[1] || p->bc[2] != p->bc[3]) {
        g_last_status = 1;
        return NULL;
    }
    orc_ctx *o = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    o->p = *p;
    o->nx = p->nx;
    o->ny = p->ny;
    o->N = (long)p->nx * p->ny;
    double c = p->c;
    const double ex[Q] = { 0, 1, 0, -1, 0 }, ey[Q] = { 0, 0, 1, 0, -1 };
    o->cs2 = 0.0;
    for (int j = 0; j < Q; ++j) {
        o->cx[j] = ex[j] * c;
        o->cy[j] = ey[j] * c;
        o->w[j] = 1.0 / 5.0;
        o->cs2 += o->w[j] * o->cx[j] * o->cx[j];
    }
    mrt_basis(o);

    long N = o->N;
    double dxmin;
    if (p->grid_kind == 0) {
        o->dx = xwall(o) ? p->lx / (p->nx - 1) : p->lx / p->nx;
        o->dy = ywall(o) ? p->ly / (p->ny - 1) : p->ly / p->ny;
        dxmin = fmin(o->dx, o->dy);
    } else {
        o->X = alloc0(N);
        o->Y = alloc0(N);
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                long n = (long)j * o->nx + i;
                if (p->grid_kind == 1) { o->X[n] = p->xc[i]; o->Y[n] = p->yc[j]; }
                else { o->X[n] = p->xc[n]; o->Y[n] = p->yc[n]; }
            }
        o->xi_x = alloc0(N); o->xi_y = alloc0(N); o->eta_x = alloc0(N); o->eta_y = alloc0(N);
        dxmin = INFINITY;
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                long n = (long)j * o->nx + i;
                double x_xi = coord_deriv(o, coord_x, 0, i, j);
                double x_eta = coord_deriv(o, coord_x, 1, i, j);
                double y_xi = coord_deriv(o, coord_y, 0, i, j);
                double y_eta = coord_deriv(o, coord_y, 1, i, j);
                double J = x_xi * y_eta - x_eta * y_xi;
                o->xi_x[n] = y_eta / J;
                o->xi_y[n] = -x_eta / J;
                o->eta_x[n] = -y_xi / J;
                o->eta_y[n] = x_xi / J;
                /* minimum physical edge length (Eq. 3.1: minimum grid scale) */
                if (i + 1 < o->nx || !xwall(o)) {
                    double ddx = coord_x(o, i + 1, j) - coord_x(o, i, j);
                    double ddy = coord_y(o, i + 1, j) - coord_y(o, i, j);
                    dxmin = fmin(dxmin, sqrt(ddx * ddx + ddy * ddy));
                }
                if (j + 1 < o->ny || !ywall(o)) {
                    double ddx = coord_x(o, i, j + 1) - coord_x(o, i, j);
                    double ddy = coord_y(o, i, j + 1) - coord_y(o, i, j);
                    dxmin = fmin(dxmin, sqrt(ddx * ddx + ddy * ddy));
                }
            }
    }
    o->dt = p->cfl * dxmin / c;  /* Eq. 3.1 */
    o->h = o->dt / 2.0;

    o->Fx = alloc0(N);
    o->Fy = alloc0(N);
    o->dFx = alloc0(N);
    o->dFy = alloc0(N);
    o->Rs = alloc0(N);
    for (long n = 0; n < N; ++n) {
        if (p->force_mode == 1) { o->Fx[n] = p->fx; o->Fy[n] = p->fy; }
        else if (p->force_mode == 2) { o->Fx[n] = p->force_x[n]; o->Fy[n] = p->force_y[n]; }
    }
    long NF = (long)NA * Q * N;
    o->fh = alloc0(NF); o->fhp = alloc0(NF); o->fbp = alloc0(NF);
    o->fb = alloc0(NF); o->f = alloc0(NF); o->fn = alloc0(NF);
    o->s_node = alloc0(N);
    if (p->rho0) {
        o->r_fh = alloc0(Q * N); o->r_fhp = alloc0(Q * N); o->r_fbp = alloc0(Q * N);
        o->r_fb = alloc0(Q * N); o->r_f = alloc0(Q * N); o->r_fn = alloc0(Q * N);
    }
    step_matrices(o, o->cs2 / p->nu, o->A, o->Ab, o->L, o->L34, o->Rinv, o->RL);
    return o;
}

void orc_destroy(orc_ctx *o) {
    if (!o) return;
    free(o->X); free(o->Y); free(o->xi_x); free(o->xi_y); free(o->eta_x); free(o->eta_y);
    free(o->Fx); free(o->Fy); free(o->dFx); free(o->dFy); free(o->Rs);
    free(o->fh); free(o->fhp); free(o->fbp); free(o->fb); free(o->f); free(o->fn);
    free(o->s_node);
    free(o->r_fh); free(o->r_fhp); free(o->r_fbp); free(o->r_fb); free(o->r_f); free(o->r_fn);
    free(o);
}

/* Body force (mode 0 none, 1 constant, 2 field), its time derivative, and
 * the source R (Newtonian only: returns -1 for a power-law fluid). */
static void fill_pair(const orc_ctx *o, int mode, double cx, double cy, const double *Fx, const double *Fy,
                      double *outx, double *outy) {
    for (long n = 0; n < o->N; ++n) {
        outx[n] = mode == 1 ? cx : mode == 2 ? Fx[n] : 0.0;
        outy[n] = mode == 1 ? cy : mode == 2 ? Fy[n] : 0.0;
    }
}
void orc_set_force(orc_ctx *o, int mode, double fx, double fy, const double *Fx, const double *Fy) {
    fill_pair(o, mode, fx, fy, Fx, Fy, o->Fx, o->Fy);
}
void orc_set_force_rate(orc_ctx *o, int mode, double dfx, double dfy, const double *dFx, const double *dFy) {
    fill_pair(o, mode, dfx, dfy, dFx, dFy, o->dFx, o->dFy);
}
int orc_set_source(orc_ctx *o, int mode, double r, const double *R) {
    if (o->p.power_law && mode != 0) return -1;
    for (long n = 0; n < o->N; ++n) o->Rs[n] = mode == 1 ? r : mode == 2 ? R[n] : 0.0;
    return 0;
}

/* Metric coefficients xi_x, xi_y, eta_x, eta_y given by the caller (for
 * instance the exact derivatives of an analytic mapping) instead of the
 * second-order differences of the node coordinates; curvilinear grids only.
 * The time step keeps the value Eq. 3.1 gave from the node coordinates. */
int orc_set_metrics(orc_ctx *o, const double *xi_x, const double *xi_y, const double *eta_x, const double *eta_y) {
    if (!o->xi_x || o->p.grid_kind != 2) return -1;
    for (long n = 0; n < o->N; ++n) {
        o->xi_x[n] = xi_x[n];
        o->xi_y[n] = xi_y[n];
        o->eta_x[n] = eta_x[n];
        o->eta_y[n] = eta_y[n];
    }
    return 0;
}

/* Copies of the metric coefficients the step uses (curvilinear grids): the
 * differenced ones of orc_create or those given by orc_set_metrics. */
int orc_get_metrics(const orc_ctx *o, double *xi_x, double *xi_y, double *eta_x, double *eta_y) {
    if (!o->xi_x || o->p.grid_kind != 2) return -1;
    for (long n = 0; n < o->N; ++n) {
        xi_x[n] = o->xi_x[n];
        xi_y[n] = o->xi_y[n];
        eta_x[n] = o->eta_x[n];
        eta_y[n] = o->eta_y[n];
    }
    return 0;
}

int orc_last_status(void) { return g_last_status; }
double orc_dt(const orc_ctx *o) { return o->dt; }
double orc_cs2(const orc_ctx *o) { return o->cs2; }
long orc_steps(const orc_ctx *o) { return o->steps; }

/* Copies of the matrices for tests (row-major 5x5). */
void orc_collision_matrix(const orc_ctx *o, double s, double *out) {
    double Lt[Q][Q];
    collision_matrix(o, s, Lt);
    memcpy(out, Lt, sizeof(Lt));
}
void orc_lambda_matrix(const orc_ctx *o, double *out) { memcpy(out, o->L, sizeof(o->L)); }

/* Initial state fhat = feq(u, v, p) (Sec. 4: "initialized by the
 * equilibrium distribution function"); wall nodes take the wall velocity. */
void orc_init(orc_ctx *o, const double *u, const double *v, const double *p) {
    for (int y = 0; y < o->ny; ++y)
        for (int x = 0; x < o->nx; ++x) {
            long n = (long)y * o->nx + x;
            double uu = u[n], vv = v[n];
            if (is_wall(o, x, y)) {
                int side;
                if (xwall(o) && (x == 0 || x == o->nx - 1)) side = x == 0 ? 0 : 1;
                else side = y == 0 ? 2 : 3;
                uu = o->p.u_wall[side];
                vv = o->p.v_wall[side];
            }
            double feq[NA][Q];
            equilibrium(o, uu, vv, p[n], feq);
            for (int a = 0; a < NA; ++a)
                for (int j = 0; j < Q; ++j) o->fh[idx(o, a, j, x, y)] = feq[a][j];
            if (o->r_fh) {  /* rho_0 = 1 */
                double f0[Q];
                equilibrium0(o, 1.0, uu, vv, f0);
                for (int j = 0; j < Q; ++j) o->r_fh[(long)j * o->N + n] = f0[j];
            }
        }
    o->steps = 0;
}

/* alpha = 0 state: fhat_{j,0} = feq_{j,0}(rho0, u) with u from the current
 * alpha = 1, 2 state; rho0[ny*nx].  Returns -1 if rho0 is not evolved. */
int orc_init_rho0(orc_ctx *o, const double *rho0) {
    if (!o->r_fh) return -1;
    for (int y = 0; y < o->ny; ++y)
        for (int x = 0; x < o->nx; ++x) {
            const long n = (long)y * o->nx + x;
            double u, v, P, f0[Q];
            moments(o, o->fh, x, y, &u, &v, &P);
            equilibrium0(o, rho0[n], u, v, f0);
            for (int j = 0; j < Q; ++j) o->r_fh[(long)j * o->N + n] = f0[j];
        }
    return 0;
}
/* rho0 = sum_j fhat_{j,0} per node; Q planes of the alpha = 0 state. */
int orc_rho0(const orc_ctx *o, double *out) {
    if (!o->r_fh) return -1;
    for (long n = 0; n < o->N; ++n) out[n] = rho0_at(o, o->r_fh, n);
    return 0;
}
int orc_get_rho0_state(const orc_ctx *o, double *out) {
    if (!o->r_fh) return -1;
    memcpy(out, o->r_fh, sizeof(double) * (size_t)Q * o->N);
    return 0;
}
int orc_set_rho0_state(orc_ctx *o, const double *in) {
    if (!o->r_fh) return -1;
    memcpy(o->r_fh, in, sizeof(double) * (size_t)Q * o->N);
    return 0;
}

void orc_set_state(orc_ctx *o, const double *fh) {
    memcpy(o->fh, fh, sizeof(double) * (size_t)NA * Q * o->N);
}
void orc_get_state(const orc_ctx *o, double *fh) {
    memcpy(fh, o->fh, sizeof(double) * (size_t)NA * Q * o->N);
}

/* ---- one time step: Steps (1)-(4) of Sec. 2.2 ----------------------- */

static void one_step(orc_ctx *o) {
    const int nx = o->nx, ny = o->ny;
    const long N = o->N;
    const double dt = o->dt, h = o->h;
    const int pl = o->p.power_law;

    /* Relaxation rate per node, from fhat(t). */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) o->s_node[(long)y * nx + x] = node_rate(o, x, y);

    /* Step 1 (Eqs. 2.2.14-2.2.15), at every node. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double A[Q][Q], Ab[Q][Q], L[Q][Q], L34[Q][Q], Ri[Q][Q], RL[Q][Q];
            if (pl) step_matrices(o, o->s_node[(long)y * nx + x], A, Ab, L, L34, Ri, RL);
            else {
                memcpy(A, o->A, sizeof(A)); memcpy(Ab, o->Ab, sizeof(Ab));
                memcpy(L, o->L, sizeof(L)); memcpy(L34, o->L34, sizeof(L34));
            }
            double u, v, P, feq[NA][Q];
            moments(o, o->fh, x, y, &u, &v, &P);
            equilibrium(o, u, v, P, feq);
            for (int a = 0; a < NA; ++a) {
                double g[Q], t1[Q], t2[Q], t3[Q], t4[Q];
                for (int j = 0; j < Q; ++j) g[j] = o->fh[idx(o, a, j, x, y)];
                mat_vec(A, g, t1);
                mat_vec(L, feq[a], t2);
                mat_vec(Ab, g, t3);
                mat_vec(L34, feq[a], t4);
                for (int j = 0; j < Q; ++j) {
                    o->fhp[idx(o, a, j, x, y)] = t1[j] + t2[j];
                    o->fbp[idx(o, a, j, x, y)] = t3[j] + t4[j];
                }
            }
            if (o->r_fh) {  /* alpha = 0 */
                const long n = (long)y * nx + x;
                double g[Q], f0[Q], t1[Q], t2[Q], t3[Q], t4[Q];
                for (int j = 0; j < Q; ++j) g[j] = o->r_fh[(long)j * N + n];
                equilibrium0(o, rho0_at(o, o->r_fh, n), u, v, f0);
                mat_vec(A, g, t1);
                mat_vec(L, f0, t2);
                mat_vec(Ab, g, t3);
                mat_vec(L34, f0, t4);
                for (int j = 0; j < Q; ++j) {
                    o->r_fhp[(long)j * N + n] = t1[j] + t2[j];
                    o->r_fbp[(long)j * N + n] = t3[j] + t4[j];
                }
            }
        }

    /* Step 2 (Eq. 2.3.25 via Eq. 2.2.11) and Step 3 (Eq. 2.2.16), at nodes
     * that are not walls. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_wall(o, x, y)) continue;
            long n = (long)y * nx + x;
            double Fa[NA] = { o->Fx[n], o->Fy[n] };
            for (int a = 0; a < NA; ++a)
                for (int j = 0; j < Q; ++j) {
                    const double *plane = o->fbp + (long)(a * Q + j) * N;
                    double cg = (j == 0) ? 0.0 : c_dot_grad(o, plane, j, x, y);
                    o->fb[idx(o, a, j, x, y)] = plane[n] - h * cg + h * o->w[j] * Fa[a];
                }
            double Ri[Q][Q], RL[Q][Q];
            if (pl) {
                double A[Q][Q], Ab[Q][Q], L[Q][Q], L34[Q][Q];
                step_matrices(o, o->s_node[n], A, Ab, L, L34, Ri, RL);
            } else { memcpy(Ri, o->Rinv, sizeof(Ri)); memcpy(RL, o->RL, sizeof(RL)); }
            double u, v, P, feq[NA][Q];
            moments_rk(o, o->fb, x, y, o->p.nu + o->cs2 * h / 2.0, &u, &v, &P);
            equilibrium(o, u, v, P, feq);
            for (int a = 0; a < NA; ++a) {
                double g[Q], t1[Q], t2[Q];
                for (int j = 0; j < Q; ++j) g[j] = o->fb[idx(o, a, j, x, y)];
                mat_vec(Ri, g, t1);
                mat_vec(RL, feq[a], t2);
                for (int j = 0; j < Q; ++j) o->f[idx(o, a, j, x, y)] = t1[j] + t2[j];
            }
            if (o->r_fh) {  /* alpha = 0: source F_{j,0} = w_j R */
                double g[Q], f0[Q], t1[Q], t2[Q];
                for (int j = 0; j < Q; ++j) {
                    const double *plane = o->r_fbp + (long)j * N;
                    double cg = (j == 0) ? 0.0 : c_dot_grad(o, plane, j, x, y);
                    o->r_fb[(long)j * N + n] = plane[n] - h * cg + h * o->w[j] * o->Rs[n];
                }
                for (int j = 0; j < Q; ++j) g[j] = o->r_fb[(long)j * N + n];
                equilibrium0(o, rho0_at(o, o->r_fb, n), u, v, f0);
                mat_vec(Ri, g, t1);
                mat_vec(RL, f0, t2);
                for (int j = 0; j < Q; ++j) o->r_f[(long)j * N + n] = t1[j] + t2[j];
            }
        }
    apply_nee(o, o->f);
    if (o->r_fh) apply_nee0(o, o->r_f, o->f);

    /* Step 4 (Eq. 2.3.24), at nodes that are not walls. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_wall(o, x, y)) continue;
            long n = (long)y * nx + x;
            double Fa[NA] = { o->Fx[n], o->Fy[n] };
            double dFa[NA] = { o->dFx[n], o->dFy[n] };
            for (int a = 0; a < NA; ++a)
                for (int j = 0; j < Q; ++j) {
                    const double *plane = o->f + (long)(a * Q + j) * N;
                    double cg = (j == 0) ? 0.0 : c_dot_grad(o, plane, j, x, y);
                    o->fn[idx(o, a, j, x, y)] = o->fhp[idx(o, a, j, x, y)] - dt * cg + dt * o->w[j] * Fa[a] +
                                                0.5 * dt * dt * o->w[j] * dFa[a];
                }
            if (o->r_fh)
                for (int j = 0; j < Q; ++j) {
                    const double *plane = o->r_f + (long)j * N;
                    double cg = (j == 0) ? 0.0 : c_dot_grad(o, plane, j, x, y);
                    o->r_fn[(long)j * N + n] = o->r_fhp[(long)j * N + n] - dt * cg + dt * o->w[j] * o->Rs[n];
                }
        }
    apply_nee(o, o->fn);
    if (o->r_fh) {
        apply_nee0(o, o->r_fn, o->fn);
        double *rt = o->r_fh; o->r_fh = o->r_fn; o->r_fn = rt;
    }

    double *t = o->fh; o->fh = o->fn; o->fn = t;
    o->steps++;
}

void orc_step(orc_ctx *o, int nsteps) {
#ifdef _OPENMP
    if (o->p.threads > 0) omp_set_num_threads(o->p.threads);
#endif
    for (int k = 0; k < nsteps; ++k) one_step(o);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- derived quantities (Sec. 2.4) ----------------------------------- */

/* out: 17 planes of N doubles, in this order:
 *  0 u, 1 v, 2 P, 3 du/dx, 4 du/dy, 5 dv/dx, 6 dv/dy, 7 div u,
 *  8 S_xx, 9 S_xy, 10 S_yy, 11 sigma_xx, 12 sigma_xy, 13 sigma_yy,
 *  14 Omega_xy, 15 vorticity dv/dx - du/dy, 16 nu. */
void orc_fields(const orc_ctx *o, double *out) {
    const int nx = o->nx, ny = o->ny;
    const long N = o->N;
    const double rho0 = 1.0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long n = (long)y * nx + x;
            double s = node_rate(o, x, y);
            double u, v, P, feq[NA][Q];
            moments(o, o->fh, x, y, &u, &v, &P);
            equilibrium(o, u, v, P, feq);
            /* first moment of f^ne = f - feq: sum_i c_i (fhat - feq) / (1 + dt s/2),
             * since Lt acts on the first-moment subspace with rate s (Eq. 2.2.4). */
            double m[2][2];  /* m[beta][alpha] */
            for (int a = 0; a < NA; ++a) {
                double gx = 0.0, gy = 0.0;
                for (int j = 0; j < Q; ++j) {
                    double ne = o->fh[idx(o, a, j, x, y)] - feq[a][j];
                    gx += o->cx[j] * ne;
                    gy += o->cy[j] * ne;
                }
                m[0][a] = gx / (1.0 + o->dt * s / 2.0);
                m[1][a] = gy / (1.0 + o->dt * s / 2.0);
            }
            double k = -s / o->cs2;                 /* Eq. 2.4.1 */
            double dudx = k * m[0][0], dudy = k * m[1][0];
            double dvdx = k * m[0][1], dvdy = k * m[1][1];
            double nu = o->cs2 / s;
            out[0 * N + n] = u;
            out[1 * N + n] = v;
            out[2 * N + n] = P;
            out[3 * N + n] = dudx;
            out[4 * N + n] = dudy;
            out[5 * N + n] = dvdx;
            out[6 * N + n] = dvdy;
            out[7 * N + n] = dudx + dvdy;            /* Eq. 2.4.2 */
            double sxx = dudx, syy = dvdy, sxy = 0.5 * (dudy + dvdx);  /* Eq. 2.4.3 */
            out[8 * N + n] = sxx;
            out[9 * N + n] = sxy;
            out[10 * N + n] = syy;
            out[11 * N + n] = 2.0 * rho0 * nu * sxx; /* Eq. 2.4.4 */
            out[12 * N + n] = 2.0 * rho0 * nu * sxy;
            out[13 * N + n] = 2.0 * rho0 * nu * syy;
            out[14 * N + n] = 0.5 * (dudy - dvdx);   /* Eq. 2.4.5, Omega_xy */
            out[15 * N + n] = dvdx - dudy;           /* vorticity, Eq. 4.1.3 */
            out[16 * N + n] = nu;
        }
}
