// mdf_aux.cu -- auxiliary kernels of libmdf.so: initial state (Sec. 4,
// fhat = feq), grid metrics in FP64 (coordinate transformation), derived
// fields (Sec. 2.4), the FP64 residual/drift reduction, and the packing
// between the padded plane layout and dense caller arrays.  Every kernel
// reads and writes both state layouts (10 FP32 planes, or u, v, P in FP32
// plus 8 16-bit non-equilibrium planes); with the alpha = 0 distribution
// the FP32 layout has 5 more planes, which the *_rho0 kernels initialise,
// sum and copy.
#include <math.h>

#include "mdf_aux.cuh"
#include "mdf_device.cuh"

namespace mdf {

namespace {

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Linear equilibrium of Eq. 2.2.5 on D2Q5 with w_j = 1/5 and cs^2 = 2c^2/5,
// so w_j c_j / cs^2 = e_j / (2c): with flux Phi = ub_alpha u + P E_alpha,
// feq_0 = ub/5, feq_{1,3} = ub/5 +- Phi_x/(2c), feq_{2,4} = ub/5 +- Phi_y/(2c).
__device__ __forceinline__ void equilibrium(float u, float v, float P, float inv2c, float out[10]) {
    const float u5 = 0.2f * u, v5 = 0.2f * v;
    const float F1x = (u * u + P) * inv2c, F1y = u * v * inv2c;
    const float F2y = (v * v + P) * inv2c;
    out[0] = u5; out[1] = u5 + F1x; out[3] = u5 - F1x; out[2] = u5 + F1y; out[4] = u5 - F1y;
    out[5] = v5; out[6] = v5 + F1y; out[8] = v5 - F1y; out[7] = v5 + F2y; out[9] = v5 - F2y;
}

// The alpha = 0 equilibrium (Eq. 2.2.5 with ubar_0 = rho_0, E_0 = 0):
// rho/5 for j = 0 (formed as rho - 4 rho/5, as the step does) and
// rho/5 +- rho u/(2c), rho/5 +- rho v/(2c) for j = 1, 3 and 2, 4.
__device__ __forceinline__ void equilibrium0(float rho, float u, float v, float inv2c, float out[5]) {
    const float r5 = 0.2f * rho, fx = rho * u * inv2c, fy = rho * v * inv2c;
    out[0] = fmaf(-4.0f, r5, rho);
    out[1] = r5 + fx;
    out[3] = r5 - fx;
    out[2] = r5 + fy;
    out[4] = r5 - fy;
}

// ---- access to one node of either state layout ------------------------------

// Non-equilibrium pair n_j = (n_{u,j}, n_{v,j}), j = 1..4, of a 16-bit
// layout at storage element s (unscaled).
__device__ __forceinline__ dev::F2 pair_at(const AuxArgs &a, const float *f, int j, long long s) {
    const unsigned w = reinterpret_cast<const unsigned *>(f)[(DEV_FPLANES + j - 1) * a.plane + s];
    const dev::F2 p = a.storage == STORAGE_FP16 ? dev::unpack16<STORAGE_FP16>(w) : dev::unpack16<STORAGE_BF16>(w);
    return p * dev::splat(a.ninv);
}

// Velocity (u, v) = sum_j fhat_{alpha,j} (Eq. 2.3.5) at storage element s.
__device__ __forceinline__ void node_uv(const AuxArgs &a, const float *f, long long s, float &u, float &v) {
    if (a.storage == STORAGE_FP32) {
        u = 0.0f;
        v = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            u += f[j * a.plane + s];
            v += f[(5 + j) * a.plane + s];
        }
    } else {
        u = f[s];
        v = f[a.plane + s];
    }
}

// The 10 distributions fhat_{alpha,j} (plane order k = 5 alpha + j).  In the
// 16-bit layouts fhat = feq(u, v, P) + n, formed exactly as the step does.
__device__ __forceinline__ void node_full(const AuxArgs &a, const float *f, long long s, float g[10]) {
    if (a.storage == STORAGE_FP32) {
#pragma unroll
        for (int k = 0; k < NPLANES; ++k) g[k] = f[k * a.plane + s];
        return;
    }
    dev::F2 nn[4], gp[5], np[5];
#pragma unroll
    for (int j = 1; j < 5; ++j) nn[j - 1] = pair_at(a, f, j, s);
    dev::dev_build(f[s], f[a.plane + s], f[2 * a.plane + s], nn, a.inv2c, gp, np);
#pragma unroll
    for (int j = 0; j < 5; ++j) dev::split2(gp[j], g[j], g[5 + j]);
}

// Write node (u, v, P, n_1..n_4) of a 16-bit layout at storage element s.
__device__ __forceinline__ void node_store16(const AuxArgs &a, float *f, long long s, float u, float v, float P,
                                             const dev::F2 n[4]) {
    f[s] = u;
    f[a.plane + s] = v;
    f[2 * a.plane + s] = P;
    unsigned *w = reinterpret_cast<unsigned *>(f);
    const dev::F2 S = dev::splat(a.nscale);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        w[(DEV_FPLANES + j) * a.plane + s] = a.storage == STORAGE_FP16 ? dev::pack16<STORAGE_FP16>(n[j] * S)
                                                                        : dev::pack16<STORAGE_BF16>(n[j] * S);
}

// Split 10 distributions into (u, v, P, n_1..n_4) with the moments and
// non-equilibrium part the step uses.
__device__ __forceinline__ void node_split(const AuxArgs &a, const float g[10], float &u, float &v, float &P,
                                           dev::F2 n[4]) {
    dev::F2 gp[5], np[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) gp[j] = dev::mk2(g[j], g[5 + j]);
    const dev::Mom2 m = dev::moments2(gp, a.c);
    dev::noneq2(gp, m, a.inv2c, np);
    u = m.u;
    v = m.v;
    P = m.P;
#pragma unroll
    for (int j = 1; j < 5; ++j) n[j - 1] = np[j];
}

}  // namespace

// One thread per stored column slot (including ghosts) and row.
__global__ void init_kernel(AuxArgs a, const float *u, const float *v, const float *p, float *f) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;  // storage column
    const int y = blockIdx.y;
    if (col >= a.pitch || y >= a.ny) return;
    const int X = col - GHOST;
    const long long s = (long long)y * a.pitch + col;
    const dev::F2 zero4[4] = {dev::splat(0.0f), dev::splat(0.0f), dev::splat(0.0f), dev::splat(0.0f)};
    int xs = X;
    if (!a.xwall) xs = wrapi(X, a.nx);
    else if (X < 0 || X >= a.nx) {
        if (a.storage != STORAGE_FP32) {
            node_store16(a, f, s, 0.0f, 0.0f, 0.0f, zero4);
            return;
        }
#pragma unroll
        for (int k = 0; k < NPLANES; ++k) f[k * a.plane + s] = 0.0f;
        if (a.rho0)
#pragma unroll
            for (int j = 0; j < 5; ++j) f[(NPLANES + j) * a.plane + s] = 0.0f;
        return;
    }
    const long long n = (long long)y * a.nx + xs;
    float uu = u[n], vv = v[n];
    if (a.xwall && (xs == 0 || xs == a.nx - 1)) {
        const int side = xs == 0 ? 0 : 1;
        uu = a.uw[side]; vv = a.vw[side];
    } else if (a.ywall && (y == 0 || y == a.ny - 1)) {
        const int side = y == 0 ? 2 : 3;
        uu = a.uw[side]; vv = a.vw[side];
    }
    if (a.storage != STORAGE_FP32) {  // fhat = feq: no non-equilibrium part
        node_store16(a, f, s, uu, vv, p[n], zero4);
        return;
    }
    float e[10];
    equilibrium(uu, vv, p[n], a.inv2c, e);
#pragma unroll
    for (int k = 0; k < NPLANES; ++k) f[k * a.plane + s] = e[k];
    if (a.rho0) {  // rho_0 = 1 at rest density
        float e0[5];
        equilibrium0(1.0f, uu, vv, a.inv2c, e0);
#pragma unroll
        for (int j = 0; j < 5; ++j) f[(NPLANES + j) * a.plane + s] = e0[j];
    }
}

// alpha = 0 distribution at equilibrium with the given rho_0 and the
// velocity of the current alpha = 1, 2 state (FP32 storage).
__global__ void init_rho0_kernel(AuxArgs a, const float *rho0, float *f) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (col >= a.pitch || y >= a.ny) return;
    const int X = col - GHOST;
    const long long s = (long long)y * a.pitch + col;
    int xs = X;
    if (!a.xwall) xs = wrapi(X, a.nx);
    else if (X < 0 || X >= a.nx) {
#pragma unroll
        for (int j = 0; j < 5; ++j) f[(NPLANES + j) * a.plane + s] = 0.0f;
        return;
    }
    float u, v, e0[5];
    node_uv(a, f, s, u, v);
    equilibrium0(rho0 ? rho0[(long long)y * a.nx + xs] : 1.0f, u, v, a.inv2c, e0);
#pragma unroll
    for (int j = 0; j < 5; ++j) f[(NPLANES + j) * a.plane + s] = e0[j];
}

// rho_0 = sum_j fhat_{j,0} per node, dense [ny][nx].
__global__ void rho0_field_kernel(AuxArgs a, const float *f, float *dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    const float *g = f + NPLANES * a.plane + (long long)y * a.pitch + GHOST + x;
    dense[(long long)y * a.nx + x] = (g[0] + g[a.plane]) + (g[2 * a.plane] + g[3 * a.plane]) + g[4 * a.plane];
}

// Dense [2][5][ny][nx] <-> padded planes.  On unpack, ghost columns of a
// periodic x axis receive the periodic image.
__global__ void pack_kernel(AuxArgs a, const float *f, float *dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int k = blockIdx.z;
    if (x >= a.nx) return;
    dense[((long long)k * a.ny + y) * a.nx + x] = f[k * a.plane + (long long)y * a.pitch + GHOST + x];
}

// 16-bit layouts: one thread per node and all planes.
__global__ void pack16_kernel(AuxArgs a, const float *f, float *dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    float g[10];
    node_full(a, f, (long long)y * a.pitch + GHOST + x, g);
#pragma unroll
    for (int k = 0; k < NPLANES; ++k) dense[((long long)k * a.ny + y) * a.nx + x] = g[k];
}

__global__ void unpack16_kernel(AuxArgs a, const float *dense, float *f) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (col >= a.pitch) return;
    const int X = col - GHOST;
    float g[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int xs = -1;
    if (!a.xwall) xs = wrapi(X, a.nx);
    else if (X >= 0 && X < a.nx) xs = X;
    if (xs >= 0)
#pragma unroll
        for (int k = 0; k < NPLANES; ++k) g[k] = dense[((long long)k * a.ny + y) * a.nx + xs];
    float u, v, P;
    dev::F2 nn[4];
    node_split(a, g, u, v, P, nn);
    node_store16(a, f, (long long)y * a.pitch + col, u, v, P, nn);
}

__global__ void unpack_kernel(AuxArgs a, const float *dense, float *f) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int k = blockIdx.z;
    if (col >= a.pitch) return;
    const int X = col - GHOST;
    float val = 0.0f;
    if (!a.xwall) val = dense[((long long)k * a.ny + y) * a.nx + wrapi(X, a.nx)];
    else if (X >= 0 && X < a.nx) val = dense[((long long)k * a.ny + y) * a.nx + X];
    f[k * a.plane + (long long)y * a.pitch + col] = val;
}

// Dense [ny][nx] field -> padded plane (periodic image in ghost columns).
__global__ void pad_field_kernel(AuxArgs a, const float *src, float *dst) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (col >= a.pitch) return;
    const int X = col - GHOST;
    float val = 0.0f;
    if (!a.xwall) val = src[(long long)y * a.nx + wrapi(X, a.nx)];
    else if (X >= 0 && X < a.nx) val = src[(long long)y * a.nx + X];
    dst[(long long)y * a.pitch + col] = val;
}

__global__ void axpy_field_kernel(AuxArgs a, const float *F, float f0, const float *dF, float d0, float k,
                                  float *dst) {
    const long long n = a.plane;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (F ? F[i] : f0) + k * (dF ? dF[i] : d0);
}

// ---- grid metrics (FP64) ----------------------------------------------

// Coordinates with periodic continuation: crossing a periodic boundary shifts
// the coordinate along that axis by the period.
struct Coords {
    const double *X, *Y;
    int nx, ny, xwall, ywall;
    double lx, ly;
    __device__ double x(int i, int j) const {
        double off = 0.0;
        while (i < 0) { i += nx; off -= lx; }
        while (i >= nx) { i -= nx; off += lx; }
        j = wrapi(j, ny);
        return X[(long long)j * nx + i] + off;
    }
    __device__ double y(int i, int j) const {
        double off = 0.0;
        while (j < 0) { j += ny; off -= ly; }
        while (j >= ny) { j -= ny; off += ly; }
        i = wrapi(i, nx);
        return Y[(long long)j * nx + i] + off;
    }
};

// Second-order central difference along dir (0: xi, 1: eta), one-sided
// second-order at a wall.
template <bool XC>
__device__ double dcoord(const Coords &c, int dir, int i, int j) {
    const int n = dir == 0 ? c.nx : c.ny;
    const int k = dir == 0 ? i : j;
    const bool wall = dir == 0 ? c.xwall : c.ywall;
    auto at = [&](int d) {
        const int ii = dir == 0 ? i + d : i, jj = dir == 0 ? j : j + d;
        return XC ? c.x(ii, jj) : c.y(ii, jj);
    };
    if (wall && k == 0) return (-3.0 * at(0) + 4.0 * at(1) - at(2)) / 2.0;
    if (wall && k == n - 1) return (3.0 * at(0) - 4.0 * at(-1) + at(-2)) / 2.0;
    return (at(1) - at(-1)) / 2.0;
}

// Metric planes c*xi_x, c*xi_y, c*eta_x, c*eta_y in the padded layout, and
// per-node minimum edge length (to the +x and +y neighbours) for Eq. 3.1.
__global__ void metric_kernel(AuxArgs a, Coords cd, double c, float *mxx, float *mxy, float *mex, float *mey,
                              double *edge_min) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (col >= a.pitch) return;
    const int X = col - GHOST;
    const long long o = (long long)j * a.pitch + col;
    if (a.xwall && (X < 0 || X >= a.nx)) {
        mxx[o] = mxy[o] = mex[o] = mey[o] = 0.0f;
        return;
    }
    const int i = a.xwall ? X : wrapi(X, a.nx);
    const double x_xi = dcoord<true>(cd, 0, i, j), x_eta = dcoord<true>(cd, 1, i, j);
    const double y_xi = dcoord<false>(cd, 0, i, j), y_eta = dcoord<false>(cd, 1, i, j);
    const double J = x_xi * y_eta - x_eta * y_xi;
    mxx[o] = (float)(c * y_eta / J);
    mxy[o] = (float)(-c * x_eta / J);
    mex[o] = (float)(-c * y_xi / J);
    mey[o] = (float)(c * x_xi / J);
    if (X >= 0 && X < a.nx) {
        double m = 1e300;
        if (i + 1 < a.nx || !a.xwall) {
            const double dx = cd.x(i + 1, j) - cd.x(i, j), dy = cd.y(i + 1, j) - cd.y(i, j);
            m = fmin(m, sqrt(dx * dx + dy * dy));
        }
        if (j + 1 < a.ny || !a.ywall) {
            const double dx = cd.x(i, j + 1) - cd.x(i, j), dy = cd.y(i, j + 1) - cd.y(i, j);
            m = fmin(m, sqrt(dx * dx + dy * dy));
        }
        edge_min[(long long)j * a.nx + i] = m;
    }
}

// Metric planes from coefficients given per node (FP64, [ny][nx], per unit
// node index), in the padded layout of metric_kernel: periodic images in the
// ghost columns of a periodic x axis, zeros beyond x walls.
__global__ void metric_given_kernel(AuxArgs a, const double *xix, const double *xiy, const double *etx,
                                    const double *ety, double c, float *mxx, float *mxy, float *mex, float *mey) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (col >= a.pitch) return;
    const int X = col - GHOST;
    const long long o = (long long)j * a.pitch + col;
    if (a.xwall && (X < 0 || X >= a.nx)) {
        mxx[o] = mxy[o] = mex[o] = mey[o] = 0.0f;
        return;
    }
    const long long n = (long long)j * a.nx + (a.xwall ? X : wrapi(X, a.nx));
    mxx[o] = (float)(c * xix[n]);
    mxy[o] = (float)(c * xiy[n]);
    mex[o] = (float)(c * etx[n]);
    mey[o] = (float)(c * ety[n]);
}

// Separable grid: c*xi_x per storage column, c*eta_y per row, and the
// spacing minima, from 1-D node coordinates (FP64).
__global__ void metric1d_kernel(AuxArgs a, const double *xc, const double *yc, double c, float *kxv, float *kyv,
                                double *edge_min) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    auto xat = [&](int i) {
        double off = 0.0;
        while (i < 0) { i += a.nx; off -= a.lx; }
        while (i >= a.nx) { i -= a.nx; off += a.lx; }
        return xc[i] + off;
    };
    auto yat = [&](int j) {
        double off = 0.0;
        while (j < 0) { j += a.ny; off -= a.ly; }
        while (j >= a.ny) { j -= a.ny; off += a.ly; }
        return yc[j] + off;
    };
    if (idx < a.pitch) {
        const int X = idx - GHOST;
        float val = 0.0f;
        if (!a.xwall || (X >= 0 && X < a.nx)) {
            const int i = a.xwall ? X : wrapi(X, a.nx);
            double d;
            if (a.xwall && i == 0) d = (-3.0 * xat(0) + 4.0 * xat(1) - xat(2)) / 2.0;
            else if (a.xwall && i == a.nx - 1) d = (3.0 * xat(i) - 4.0 * xat(i - 1) + xat(i - 2)) / 2.0;
            else d = (xat(i + 1) - xat(i - 1)) / 2.0;
            val = (float)(c / d);
        }
        kxv[idx] = val;
    }
    if (idx < a.ny) {
        const int j = idx;
        double d;
        if (a.ywall && j == 0) d = (-3.0 * yat(0) + 4.0 * yat(1) - yat(2)) / 2.0;
        else if (a.ywall && j == a.ny - 1) d = (3.0 * yat(j) - 4.0 * yat(j - 1) + yat(j - 2)) / 2.0;
        else d = (yat(j + 1) - yat(j - 1)) / 2.0;
        kyv[j] = (float)(c / d);
    }
    if (idx < a.nx) {
        double m = 1e300;
        if (idx + 1 < a.nx || !a.xwall) m = fmin(m, fabs(xat(idx + 1) - xat(idx)));
        edge_min[idx] = m;
    }
    if (idx < a.ny) {
        double m = 1e300;
        if (idx + 1 < a.ny || !a.ywall) m = fmin(m, fabs(yat(idx + 1) - yat(idx)));
        edge_min[a.nx + idx] = m;
    }
}

// ---- derived fields (Sec. 2.4) -------------------------------------------

__device__ float pl_nu(float g, const AuxArgs &a) {
    const float n = a.n_index;
    if (n == 1.0f) return fminf(fmaxf(a.K, a.nu_min), a.nu_max);
    if (!(g > 1e-30f)) return n < 1.0f ? a.nu_max : a.nu_min;
    const float lnK = logf(a.K), lng = logf(g);
    const float lmin = logf(a.nu_min), lmax = logf(a.nu_max);
    float l = (lnK + (n - 1.0f) * lng) / n;
    l = fminf(fmaxf(l, lmin), lmax);
    for (int it = 0; it < 8; ++it) {
        const float e = expf(l);
        const float F = l - lnK - (n - 1.0f) * (lng - logf(e + a.a_pl));
        const float dF = 1.0f + (n - 1.0f) * e / (e + a.a_pl);
        l = l - F / dF;
        l = fminf(fmaxf(l, lmin - 1.0f), lmax + 1.0f);
    }
    return fminf(fmaxf(expf(l), a.nu_min), a.nu_max);
}

// Field order: u, v, P, du/dx, du/dy, dv/dx, dv/dy, div u, Sxx, Sxy, Syy,
// sigma_xx, sigma_xy, sigma_yy, Omega_xy, vorticity, nu.  dst[k] is the
// output of field k (nullptr when not requested), dense [ny][nx].
__global__ void fields_kernel(AuxArgs a, const float *f, FieldPtrs dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    const long long s = (long long)y * a.pitch + GHOST + x;
    const float c = a.c;
    float u, v, P, gx1, gy1, gx2, gy2;
    if (a.storage == STORAGE_FP32) {
        float g[10];
#pragma unroll
        for (int k = 0; k < NPLANES; ++k) g[k] = f[k * a.plane + s];
        u = g[0] + g[1] + g[2] + g[3] + g[4];
        v = g[5] + g[6] + g[7] + g[8] + g[9];
        const float d1x = g[1] - g[3], d1y = g[2] - g[4], d2x = g[6] - g[8], d2y = g[7] - g[9];
        P = 0.5f * (c * (d1x + d2y) - u * u - v * v);  // Eq. 2.3.23
        if (a.r_mode) P += a.rk_hat * (a.r_mode == 1 ? a.Rc : a.Rp[s]);
        // first moment of fhat - feq (Eq. 2.2.5 fluxes ub u + P E)
        gx1 = c * d1x - (u * u + P);
        gy1 = c * d1y - u * v;
        gx2 = c * d2x - u * v;
        gy2 = c * d2y - (v * v + P);
    } else {
        // stored u, v, P; the first moment of fhat - feq is c (n_1 - n_3),
        // c (n_2 - n_4) per component
        u = f[s];
        v = f[a.plane + s];
        P = f[2 * a.plane + s];
        float n1u, n1v, n2u, n2v, n3u, n3v, n4u, n4v;
        dev::split2(pair_at(a, f, 1, s), n1u, n1v);
        dev::split2(pair_at(a, f, 2, s), n2u, n2v);
        dev::split2(pair_at(a, f, 3, s), n3u, n3v);
        dev::split2(pair_at(a, f, 4, s), n4u, n4v);
        gx1 = c * (n1u - n3u);
        gy1 = c * (n2u - n4u);
        gx2 = c * (n1v - n3v);
        gy2 = c * (n2v - n4v);
    }
    float nu = a.nu;
    if (a.power_law) {
        const float sxy = 0.5f * (gy1 + gx2);
        nu = pl_nu(sqrtf(2.0f * (gx1 * gx1 + gy2 * gy2 + 2.0f * sxy * sxy)), a);
    }
    // grad_beta u_alpha = -(s/cs2) sum_i c_beta f^ne = -G / (nu + cs2 dt/2)  (Eq. 2.4.1)
    const float k = -1.0f / (nu + a.a_pl);
    const float dudx = k * gx1, dudy = k * gy1, dvdx = k * gx2, dvdy = k * gy2;
    const float sxx = dudx, syy = dvdy, sxy = 0.5f * (dudy + dvdx);
    float val[17] = {u, v, P, dudx, dudy, dvdx, dvdy, dudx + dvdy, sxx, sxy, syy,
                     2.0f * nu * sxx, 2.0f * nu * sxy, 2.0f * nu * syy, 0.5f * (dudy - dvdx), dvdx - dudy, nu};
    const long long o = (long long)y * a.nx + x;
#pragma unroll
    for (int q = 0; q < 17; ++q)
        if (dst.p[q]) dst.p[q][o] = val[q];
}

// ---- residual / drift reduction (FP64) -------------------------------------

// Stage 1: per block, sums of |U - U_snap|^2, |U|^2, u, v and a non-finite
// count; the snapshot is replaced by U.  Partials: 5 doubles per block.
__global__ void residual_partial_kernel(AuxArgs a, const float *f, float *su, float *sv, double *partials) {
    __shared__ double red[5][32];
    const long long N = (long long)a.nx * a.ny;
    double d2 = 0.0, n2 = 0.0, su_ = 0.0, sv_ = 0.0, bad = 0.0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / a.nx), x = (int)(n % a.nx);
        const long long s = (long long)y * a.pitch + GHOST + x;
        float u, v;
        node_uv(a, f, s, u, v);
        if (!isfinite(u) || !isfinite(v)) bad += 1.0;
        const double du = (double)u - su[n], dv = (double)v - sv[n];
        d2 += du * du + dv * dv;
        n2 += (double)u * u + (double)v * v;
        su_ += u;
        sv_ += v;
        su[n] = u;
        sv[n] = v;
    }
    double vals[5] = {d2, n2, su_, sv_, bad};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double x = vals[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double x = lane < nw ? red[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) partials[(long long)blockIdx.x * 5 + q] = x;
        }
    }
}

// Stage 2: one block sums the partials in a fixed order (deterministic).
__global__ void residual_final_kernel(const double *partials, int nblocks, double *out) {
    __shared__ double red[5][32];
    double vals[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) vals[q] += partials[(long long)b * 5 + q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double x = vals[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double x = lane < nw ? red[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out[q] = x;
        }
    }
}

// Snapshot U := current velocity (after mdf_init_fields / mdf_set_distributions).
__global__ void snapshot_kernel(AuxArgs a, const float *f, float *su, float *sv) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    const long long s = (long long)y * a.pitch + GHOST + x;
    float u, v;
    node_uv(a, f, s, u, v);
    su[(long long)y * a.nx + x] = u;
    sv[(long long)y * a.nx + x] = v;
}


// ---- host-side launch wrappers --------------------------------------------

static inline dim3 rows_grid(int cols, int ny, int threads, int z = 1) {
    return dim3((cols + threads - 1) / threads, ny, z);
}

cudaError_t aux_init(const AuxArgs &a, const float *u, const float *v, const float *p, float *f, cudaStream_t st) {
    init_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, u, v, p, f);
    return cudaGetLastError();
}

cudaError_t aux_pack(const AuxArgs &a, const float *f, float *dense, cudaStream_t st) {
    if (a.storage != STORAGE_FP32) {
        pack16_kernel<<<rows_grid(a.nx, a.ny, 128), 128, 0, st>>>(a, f, dense);
        return cudaGetLastError();
    }
    pack_kernel<<<rows_grid(a.nx, a.ny, 128, NPLANES), 128, 0, st>>>(a, f, dense);
    return cudaGetLastError();
}

cudaError_t aux_unpack(const AuxArgs &a, const float *dense, float *f, cudaStream_t st) {
    if (a.storage != STORAGE_FP32) {
        unpack16_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, dense, f);
        return cudaGetLastError();
    }
    unpack_kernel<<<rows_grid(a.pitch, a.ny, 128, NPLANES), 128, 0, st>>>(a, dense, f);
    return cudaGetLastError();
}

cudaError_t aux_init_rho0(const AuxArgs &a, const float *rho0, float *f, cudaStream_t st) {
    init_rho0_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, rho0, f);
    return cudaGetLastError();
}

cudaError_t aux_rho0_field(const AuxArgs &a, const float *f, float *dense, cudaStream_t st) {
    rho0_field_kernel<<<rows_grid(a.nx, a.ny, 128), 128, 0, st>>>(a, f, dense);
    return cudaGetLastError();
}

cudaError_t aux_pack_rho0(const AuxArgs &a, const float *f, float *dense, cudaStream_t st) {
    pack_kernel<<<rows_grid(a.nx, a.ny, 128, 5), 128, 0, st>>>(a, f + NPLANES * a.plane, dense);
    return cudaGetLastError();
}

cudaError_t aux_unpack_rho0(const AuxArgs &a, const float *dense, float *f, cudaStream_t st) {
    unpack_kernel<<<rows_grid(a.pitch, a.ny, 128, 5), 128, 0, st>>>(a, dense, f + NPLANES * a.plane);
    return cudaGetLastError();
}

cudaError_t aux_pad_field(const AuxArgs &a, const float *src, float *dst, cudaStream_t st) {
    pad_field_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, src, dst);
    return cudaGetLastError();
}

cudaError_t aux_axpy_field(const AuxArgs &a, const float *F, float f0, const float *dF, float d0, float k, float *dst,
                           cudaStream_t st) {
    long long b = (a.plane + 255) / 256;
    if (b > 65535) b = 65535;
    axpy_field_kernel<<<(unsigned)b, 256, 0, st>>>(a, F, f0, dF, d0, k, dst);
    return cudaGetLastError();
}

cudaError_t aux_metrics2d(const AuxArgs &a, const double *X, const double *Y, double c, float *mxx, float *mxy,
                          float *mex, float *mey, double *edge_min, cudaStream_t st) {
    Coords cd{X, Y, a.nx, a.ny, a.xwall, a.ywall, a.lx, a.ly};
    metric_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, cd, c, mxx, mxy, mex, mey, edge_min);
    return cudaGetLastError();
}

cudaError_t aux_metrics_given(const AuxArgs &a, const double *const m[4], double c, float *mxx, float *mxy, float *mex,
                              float *mey, cudaStream_t st) {
    metric_given_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, m[0], m[1], m[2], m[3], c, mxx, mxy, mex,
                                                                       mey);
    return cudaGetLastError();
}

cudaError_t aux_metrics1d(const AuxArgs &a, const double *xc, const double *yc, double c, float *kxv, float *kyv,
                          double *edge_min, cudaStream_t st) {
    int n = a.pitch > a.ny ? a.pitch : a.ny;
    metric1d_kernel<<<(n + 127) / 128, 128, 0, st>>>(a, xc, yc, c, kxv, kyv, edge_min);
    return cudaGetLastError();
}

cudaError_t aux_fields(const AuxArgs &a, const float *f, const FieldPtrs &dst, cudaStream_t st) {
    fields_kernel<<<rows_grid(a.nx, a.ny, 128), 128, 0, st>>>(a, f, dst);
    return cudaGetLastError();
}

int aux_residual_blocks(const AuxArgs &a) {
    const long long N = (long long)a.nx * a.ny;
    long long b = (N + 255) / 256;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t aux_residual(const AuxArgs &a, const float *f, float *su, float *sv, double *partials, double *out,
                         cudaStream_t st) {
    const int nb = aux_residual_blocks(a);
    residual_partial_kernel<<<nb, 256, 0, st>>>(a, f, su, sv, partials);
    residual_final_kernel<<<1, 1024, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

__global__ void poison_kernel(AuxArgs a, float *f, int planes) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (col >= a.pitch) return;
    const bool pad = col >= a.nx + 2 * GHOST;
    const bool ghost = a.xwall && (col < GHOST || col >= a.nx + GHOST);
    if (!(pad || ghost)) return;
    unsigned *w = reinterpret_cast<unsigned *>(f);
    for (int k = 0; k < planes; ++k) w[k * a.plane + (long long)y * a.pitch + col] = 0x7fc07fc0u;
}

cudaError_t aux_poison(const AuxArgs &a, float *f, int planes, cudaStream_t st) {
    poison_kernel<<<rows_grid(a.pitch, a.ny, 128), 128, 0, st>>>(a, f, planes);
    return cudaGetLastError();
}

cudaError_t aux_snapshot(const AuxArgs &a, const float *f, float *su, float *sv, cudaStream_t st) {
    snapshot_kernel<<<rows_grid(a.nx, a.ny, 128), 128, 0, st>>>(a, f, su, sv);
    return cudaGetLastError();
}

}  // namespace mdf
