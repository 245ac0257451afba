// mdf_step.cu -- the fused MDF-FDLBM time step for sm_103a.
//
// One launch performs one time step of Sec. 2.2, Steps (1)-(4), of
// arXiv:2306.08216 with the simplified evolution equations of Remark 2:
//   Step 1  fhat^+ = feq + (I - Lambda)(fhat - feq)             (Eq. 2.2.14)
//           fbar^+ = feq + (I - 3 Lambda/4)(fhat - feq)         (Eq. 2.2.15)
//   Step 2  fbar(t+h) = fbar^+ - h c_j.grad fbar^+ + h w_j F     (Eq. 2.3.25 / 2.2.11)
//   Step 3  f(t+h) = feq + (I + h/2 Lt)^-1 (fbar - feq)          (Eq. 2.2.16)
//   Step 4  fhat(t+dt) = fhat^+ - dt c_j.grad f(t+h) + dt w_j F  (Eq. 2.3.24)
// The MRT matrix of Eq. 2.2.4 with s0 = s3 = s4 = s' and s1 = s2 = s equals
// s' I + (s - s') P_c, P_c the projector on the first moments, so every
// function of it acts on a distribution through its zeroth and first moments
// only; with the D2Q5 lattice (Eq. 3.1.0) and the linear equilibrium
// (Eq. 2.2.5) each of the three local maps costs a handful of FMAs per
// population and no 5x5 product appears (cf. the 2x5x5 loop count of Sec. 4.2).
//
// Work decomposition.  A block owns a strip of W output columns and marches
// down a band of H rows.  Thread t holds column x0 - 4 + t; the 8 extra
// columns are the halo the two chained stencils need (reach 2 + 2).  Each
// iteration of the march
//   A: takes row p of fhat from a TMA ring (cp.async.bulk.tensor, one 3-D box
//      of 10 planes x NT columns per row) and writes fhat^+ and fbar^+ of row
//      p to shared rings;
//   B: forms fbar and then f(t+h) of row q = p - 2 from the fbar^+ ring
//      (x stencils across threads, y stencils across ring rows);
//   C: forms fhat(t+dt) of row r = p - 4 from the f ring and stores it.
// Only the x halo is recomputed; rows are streamed once.  Walls use
// non-equilibrium extrapolation written by the interior neighbour's thread,
// and the one-sided second-order upwind point beyond a wall is replaced by
// its linear extrapolation (Pi(-1) = 2 Pi(0) - Pi(1)).
#include "mdf_internal.cuh"

namespace mdf {

namespace {

constexpr int TMA_SLOTS = 3;   // rows in flight
constexpr int RB = 5;          // fbar^+ ring rows (y stencil reach 2 + 2)
constexpr int RF = 5;          // f(t+h) ring rows
constexpr int RP = 6;          // fhat^+ ring rows (used 4 iterations later)
constexpr int RK = 5;          // power-law recovery rates ring

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^32 clock cycles (about two seconds).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > (1ll << 32)) return false;
    }
}

__device__ __forceinline__ void tma_load_row(const CUtensorMap *map, uint64_t *bar, float *dst, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// Moments of a node (10 values, plane order 5 alpha + j): u, v, the four odd
// differences and P of Eq. 2.3.23 (R = 0), which fhat, fbar and f share.
struct Mom {
    float u, v, d1x, d1y, d2x, d2y, P;
};

__device__ __forceinline__ Mom moments(const float g[10], float c) {
    Mom m;
    m.u = g[0] + g[1] + g[2] + g[3] + g[4];
    m.v = g[5] + g[6] + g[7] + g[8] + g[9];
    m.d1x = g[1] - g[3];
    m.d1y = g[2] - g[4];
    m.d2x = g[6] - g[8];
    m.d2y = g[7] - g[9];
    m.P = 0.5f * (c * (m.d1x + m.d2y) - m.u * m.u - m.v * m.v);
    return m;
}

// Non-equilibrium part n = g - feq of a node (Eq. 2.2.5 on D2Q5 with
// w_j = 1/5, cs^2 = 2c^2/5: feq_0 = ub/5, feq_{1,3} = ub/5 +- Phi_x/(2c),
// feq_{2,4} = ub/5 +- Phi_y/(2c), Phi = ub_alpha u + P E_alpha).  feq_0 is
// formed as ub - 4 ub/5 so that sum_j feq_j = ub carries no rounding bias of
// the constant 1/5; otherwise every step would scale the conserved zeroth
// moment by the same FP32 factor and the drift would grow linearly in time.
__device__ __forceinline__ void noneq(const float g[10], const Mom &m, float inv2c, float n[10]) {
    const float u5 = 0.2f * m.u, v5 = 0.2f * m.v;
    const float f1x = fmaf(m.u, m.u, m.P) * inv2c, uv = m.u * m.v * inv2c;
    const float f2y = fmaf(m.v, m.v, m.P) * inv2c;
    n[0] = g[0] - fmaf(-4.0f, u5, m.u);
    n[1] = g[1] - (u5 + f1x);
    n[3] = g[3] - (u5 - f1x);
    n[2] = g[2] - (u5 + uv);
    n[4] = g[4] - (u5 - uv);
    n[5] = g[5] - fmaf(-4.0f, v5, m.v);
    n[6] = g[6] - (v5 + uv);
    n[8] = g[8] - (v5 - uv);
    n[7] = g[7] - (v5 + f2y);
    n[9] = g[9] - (v5 - f2y);
}

// Local relaxation map shared by Steps 1 and 3, applied as an increment:
// out = g - (1 - Ap) n + (A - Ap) P_c n, which equals
// feq + Ap (g - feq) + (A - Ap) P_c (g - feq); Ap / A are the eigenvalues on
// the free / first-moment subspaces, (P_c n)_{1,3} = +-(n_1 - n_3)/2 and
// (P_c n)_{2,4} = +-(n_2 - n_4)/2.  Written this way the zeroth moment is
// kept up to unbiased per-node rounding.
__device__ __forceinline__ void relax10(const float g[10], const float n[10], float Ap, float A, float out[10]) {
    const float K = 1.0f - Ap, D = 0.5f * (A - Ap);
#pragma unroll
    for (int b = 0; b < 10; b += 5) {
        const float dx = D * (n[b + 1] - n[b + 3]);
        const float dy = D * (n[b + 2] - n[b + 4]);
        out[b + 0] = fmaf(-K, n[b + 0], g[b + 0]);
        out[b + 1] = fmaf(-K, n[b + 1], g[b + 1]) + dx;
        out[b + 3] = fmaf(-K, n[b + 3], g[b + 3]) - dx;
        out[b + 2] = fmaf(-K, n[b + 2], g[b + 2]) + dy;
        out[b + 4] = fmaf(-K, n[b + 4], g[b + 4]) - dy;
    }
}

// Non-equilibrium extrapolation: node value = g_nb + feq(u_w, P) - feq(u_nb, P)
// (the pressure cancels in the difference of the linear equilibria).
__device__ __forceinline__ void nee(const float g[10], float uw, float vw, float inv2c, float out[10]) {
    const float un = g[0] + g[1] + g[2] + g[3] + g[4];
    const float vn = g[5] + g[6] + g[7] + g[8] + g[9];
    const float du = 0.2f * (uw - un), dv = 0.2f * (vw - vn);
    const float uux = (uw * uw - un * un) * inv2c, uvy = (uw * vw - un * vn) * inv2c;
    const float vvy = (vw * vw - vn * vn) * inv2c;
    out[0] = g[0] + du;
    out[1] = g[1] + du + uux;
    out[3] = g[3] + du - uux;
    out[2] = g[2] + du + uvy;
    out[4] = g[4] + du - uvy;
    out[5] = g[5] + dv;
    out[6] = g[6] + dv + uvy;
    out[8] = g[8] + dv - uvy;
    out[7] = g[7] + dv + vvy;
    out[9] = g[9] + dv - vvy;
}

// Rates of the three local maps for first-moment rate s (s' = s_ratio s):
// rho(l) = (1 - dt l/2)/(1 + dt l/2) for I - Lambda, (1 + 3 rho)/4 for
// I - 3 Lambda/4, 1/(1 + h l/2) for (I + h/2 Lt)^-1.
struct Rates {
    float rpp, rp, rbp, rb, rkp, rk;
};

__device__ __forceinline__ Rates rates_for(float s, float s_ratio, float dt) {
    const float sp = s_ratio * s;
    Rates r;
    r.rpp = (1.0f - 0.5f * dt * sp) / (1.0f + 0.5f * dt * sp);
    r.rp = (1.0f - 0.5f * dt * s) / (1.0f + 0.5f * dt * s);
    r.rbp = 0.25f * (1.0f + 3.0f * r.rpp);
    r.rb = 0.25f * (1.0f + 3.0f * r.rp);
    r.rkp = 1.0f / (1.0f + 0.25f * dt * sp);
    r.rk = 1.0f / (1.0f + 0.25f * dt * s);
    return r;
}

// Power-law viscosity nu = K gdot^(n-1), gdot = g/(nu + a), solved by Newton
// iterations on l = ln nu (the residual l - ln K - (n-1)(ln g - ln(e^l + a))
// has a derivative in (min(1,n), max(1,n)), so the iteration is safe), then
// clamped to [nu_min, nu_max].
__device__ __forceinline__ float power_law_nu(float g, const StepArgs &a) {
    const float n = a.n_index;
    if (n == 1.0f) return fminf(fmaxf(a.K, a.nu_min), a.nu_max);
    if (!(g > 1e-30f)) return n < 1.0f ? a.nu_max : a.nu_min;
    const float lnK = __logf(a.K), lng = __logf(g);
    const float lmin = __logf(a.nu_min), lmax = __logf(a.nu_max);
    // start: solution without the a term, clamped
    float l = (lnK + (n - 1.0f) * lng) / n;
    l = fminf(fmaxf(l, lmin), lmax);
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const float e = __expf(l);
        const float F = l - lnK - (n - 1.0f) * (lng - __logf(e + a.a_pl));
        const float dF = 1.0f + (n - 1.0f) * e / (e + a.a_pl);
        l = l - F / dF;
        l = fminf(fmaxf(l, lmin - 1.0f), lmax + 1.0f);
    }
    return fminf(fmaxf(__expf(l), a.nu_min), a.nu_max);
}

// Streaming term along one axis, population moving towards +chi (sgn > 0) or
// -chi: a1 Pi(+-1) + a0 Pi(0) + am1 Pi(-+1) + am2 Pi(-+2), with the far
// upwind point replaced by 2 Pi(-+1) - Pi(0) next to a wall.
// Written in differences from Pi(-+1) (the weights sum to zero), so a
// uniform field gives exactly zero and the FP32 rounding of the weights puts
// no bias on conserved sums.
__device__ __forceinline__ float stencil(float pf, float p0, float pb1, float pb2, bool wall_adj, const StepArgs &a) {
    const float d0 = p0 - pb1;
    const float dfar = wall_adj ? -d0 : (pb2 - pb1);
    return fmaf(a.a1, pf - pb1, fmaf(a.a0, d0, a.am2 * dfar));
}

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Store one node of the output (10 planes), with its periodic image in the
// ghost columns when the x axis is periodic.
__device__ __forceinline__ void store_node(const StepArgs &a, int row, int X, const float v[10]) {
    const long long base = (long long)row * a.pitch + GHOST + X;
#pragma unroll
    for (int k = 0; k < NPLANES; ++k) a.fout[k * a.plane + base] = v[k];
    if (!a.xwall) {
        // a node can be the image of a ghost on both sides when nx < 2 GHOST
        if (X < GHOST) {
            const long long b2 = (long long)row * a.pitch + GHOST + X + a.nx;
#pragma unroll
            for (int k = 0; k < NPLANES; ++k) a.fout[k * a.plane + b2] = v[k];
        }
        if (X >= a.nx - GHOST) {
            const long long b2 = (long long)row * a.pitch + GHOST + X - a.nx;
#pragma unroll
            for (int k = 0; k < NPLANES; ++k) a.fout[k * a.plane + b2] = v[k];
        }
    }
}

template <int NT, int MK, bool PL>
__global__ void __launch_bounds__(NT) step_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int ROW = NPLANES * NT;
    float *tma = reinterpret_cast<float *>(smem_raw);
    float *rB = tma + TMA_SLOTS * ROW;
    float *rF = rB + RB * ROW;
    float *rP = rF + RF * ROW;
    float *rK = rP + RP * ROW;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(rK + (PL ? RK * 2 * NT : 0));
    __shared__ int s_abort;

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * a.W;
    const int X = x0 - 4 + t;
    const int y0 = blockIdx.y * a.H;
    const int y1 = min(y0 + a.H, a.ny);
    const int nIt = (y1 - y0) + 8;
    const int rowBase = y0 - 4;
    const float c = a.c, inv2c = a.inv2c;

    if (t == 0) {
        s_abort = 0;
        for (int i = 0; i < TMA_SLOTS; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto load_row = [&](int it) {
        const int p = rowBase + it;
        const int yy = a.ywall ? p : wrap(p, a.ny);
        const int slot = it % TMA_SLOTS;
        mbar_expect_tx(&mbar[slot], ROW * 4);
        tma_load_row(&tmap, &mbar[slot], tma + slot * ROW, x0, yy);
    };
    if (t == 0)
        for (int i = 0; i < TMA_SLOTS && i < nIt; ++i) load_row(i);

    // per-column constants
    const bool colx_wall = a.xwall && (X == 0 || X == a.nx - 1);
    const bool colx_out = a.xwall ? (X < 0 || X >= a.nx) : false;
    const bool xadj_plus = a.xwall && X == 1;            // +x population: far point beyond west wall
    const bool xadj_minus = a.xwall && X == a.nx - 2;    // -x population: far point beyond east wall
    float kxc = a.kx;
    if (MK == METRIC_SEPARABLE) kxc = a.kxv[GHOST + X];

    int issued = min(TMA_SLOTS, nIt);
    for (int it = 0; it < nIt; ++it) {
        const int p = rowBase + it;
        // ------------------------------------------------ Stage A: row p
        {
            const int slot = it % TMA_SLOTS;
            const bool ok = mbar_wait_bounded(&mbar[slot], (uint32_t)((it / TMA_SLOTS) & 1));
            if (!ok) atomicExch(&s_abort, 1);
            const float *src = tma + slot * ROW;
            float g[10];
#pragma unroll
            for (int k = 0; k < NPLANES; ++k) g[k] = src[k * NT + t];
            const Mom m = moments(g, c);
            Rates R;
            if (PL) {
                const float F1x = fmaf(m.u, m.u, m.P), F1y = m.u * m.v;
                const float F2y = fmaf(m.v, m.v, m.P);
                const float gx1 = c * m.d1x - F1x, gy1 = c * m.d1y - F1y;
                const float gx2 = c * m.d2x - F1y, gy2 = c * m.d2y - F2y;
                const float sxy = 0.5f * (gy1 + gx2);
                const float gg = sqrtf(2.0f * (gx1 * gx1 + gy2 * gy2 + 2.0f * sxy * sxy));
                const float nu = power_law_nu(gg, a);
                R = rates_for(a.cs2 / nu, a.s_ratio, a.dt);
                float *k = rK + (it % RK) * 2 * NT;
                k[t] = R.rkp;
                k[NT + t] = R.rk;
            } else {
                R.rpp = a.rpp; R.rp = a.rp; R.rbp = a.rbp; R.rb = a.rb;
            }
            float nq[10], o[10];
            noneq(g, m, inv2c, nq);
            relax10(g, nq, R.rpp, R.rp, o);
            float *dP = rP + (it % RP) * ROW;
#pragma unroll
            for (int k = 0; k < NPLANES; ++k) dP[k * NT + t] = o[k];
            relax10(g, nq, R.rbp, R.rb, o);
            float *dB = rB + (it % RB) * ROW;
#pragma unroll
            for (int k = 0; k < NPLANES; ++k) dB[k * NT + t] = o[k];
        }
        // all threads are done with TMA slot `it % TMA_SLOTS` and ring rows
        if (__syncthreads_or(s_abort)) break;
        if (t == 0 && issued < nIt) {
            fence_proxy_async();
            load_row(issued);
            ++issued;
        }
        // ------------------------------------------------ Stage B: row q = p - 2
        if (it >= 4 && t >= 2 && t < NT - 2) {
            const int q = p - 2;
            const bool qwall = a.ywall && (q == 0 || q == a.ny - 1);
            const bool qout = a.ywall && (q < 0 || q >= a.ny);
            const int qw = a.ywall ? q : wrap(q, a.ny);
            float *Fq = rF + ((it - 2) % RF) * ROW;
            if (!qout && !colx_out) {
                if (a.ywall && q == a.ny - 1) {
                    // north wall row: NEE from row ny-2 (this column, written last iteration)
                    if (!colx_wall) {
                        const float *Fn = rF + ((it - 3) % RF) * ROW;
                        float g[10], w[10];
#pragma unroll
                        for (int k = 0; k < NPLANES; ++k) g[k] = Fn[k * NT + t];
                        nee(g, a.uw[3], a.vw[3], inv2c, w);
#pragma unroll
                        for (int k = 0; k < NPLANES; ++k) Fq[k * NT + t] = w[k];
                        if (xadj_plus) {  // north-west corner from the diagonal node
                            nee(g, a.uw[0], a.vw[0], inv2c, w);
#pragma unroll
                            for (int k = 0; k < NPLANES; ++k) Fq[k * NT + t - 1] = w[k];
                        }
                        if (xadj_minus) {
                            nee(g, a.uw[1], a.vw[1], inv2c, w);
#pragma unroll
                            for (int k = 0; k < NPLANES; ++k) Fq[k * NT + t + 1] = w[k];
                        }
                    }
                } else if (!qwall && !colx_wall) {
                    // Step 2: fbar = fbar^+ - h c.grad fbar^+ + h w F
                    const float *Bq = rB + ((it - 2) % RB) * ROW;
                    const float *Bm2 = rB + ((it - 4) % RB) * ROW;
                    const float *Bm1 = rB + ((it - 3) % RB) * ROW;
                    const float *Bp1 = rB + ((it - 1) % RB) * ROW;
                    const float *Bp2 = rB + (it % RB) * ROW;
                    const bool yadj_plus = a.ywall && q == 1;
                    const bool yadj_minus = a.ywall && q == a.ny - 2;
                    float fx = 0.0f, fy = 0.0f;
                    if (a.force_mode == 1) { fx = a.Fx; fy = a.Fy; }
                    else if (a.force_mode == 2) {
                        const long long fi = (long long)qw * a.pitch + GHOST + X;
                        fx = a.Fxp[fi]; fy = a.Fyp[fi];
                    }
                    float fb[10];
#pragma unroll
                    for (int al = 0; al < 2; ++al) {
                        const int b = 5 * al;
                        const float hF = a.h * 0.2f * (al == 0 ? fx : fy);
                        fb[b] = Bq[b * NT + t] + hF;
                        // populations 1 (+x) and 3 (-x) along x
                        const float *P1 = Bq + (b + 1) * NT + t;
                        const float *P3 = Bq + (b + 3) * NT + t;
                        const float *P2c = Bq + (b + 2) * NT + t;
                        const float *P4c = Bq + (b + 4) * NT + t;
                        if (MK != METRIC_CURVILINEAR) {
                            const float kyq = (MK == METRIC_SEPARABLE) ? a.kyv[qw] : a.ky;
                            const float s1 = kxc * stencil(P1[1], P1[0], P1[-1], P1[-2], xadj_plus, a);
                            const float s3 = kxc * stencil(P3[-1], P3[0], P3[1], P3[2], xadj_minus, a);
                            const float s2 = kyq * stencil(Bp1[(b + 2) * NT + t], P2c[0], Bm1[(b + 2) * NT + t],
                                                           Bm2[(b + 2) * NT + t], yadj_plus, a);
                            const float s4 = kyq * stencil(Bm1[(b + 4) * NT + t], P4c[0], Bp1[(b + 4) * NT + t],
                                                           Bp2[(b + 4) * NT + t], yadj_minus, a);
                            fb[b + 1] = fmaf(-a.h, s1, P1[0]) + hF;
                            fb[b + 3] = fmaf(-a.h, s3, P3[0]) + hF;
                            fb[b + 2] = fmaf(-a.h, s2, P2c[0]) + hF;
                            fb[b + 4] = fmaf(-a.h, s4, P4c[0]) + hF;
                        } else {
                            const long long mi = (long long)qw * a.pitch + GHOST + X;
                            const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
#pragma unroll
                            for (int j = 1; j <= 4; ++j) {
                                const float sx = (j == 1) ? cxx : (j == 2) ? cxy : (j == 3) ? -cxx : -cxy;
                                const float se = (j == 1) ? cex : (j == 2) ? cey : (j == 3) ? -cex : -cey;
                                const float *Px = Bq + (b + j) * NT + t;
                                float acc = 0.0f;
                                if (sx != 0.0f) {
                                    const float st = sx > 0.0f ? stencil(Px[1], Px[0], Px[-1], Px[-2], xadj_plus, a)
                                                               : stencil(Px[-1], Px[0], Px[1], Px[2], xadj_minus, a);
                                    acc = fabsf(sx) * st;
                                }
                                if (se != 0.0f) {
                                    const float pm2 = Bm2[(b + j) * NT + t], pm1 = Bm1[(b + j) * NT + t];
                                    const float pp1 = Bp1[(b + j) * NT + t], pp2 = Bp2[(b + j) * NT + t];
                                    const float st = se > 0.0f ? stencil(pp1, Px[0], pm1, pm2, yadj_plus, a)
                                                               : stencil(pm1, Px[0], pp1, pp2, yadj_minus, a);
                                    acc = fmaf(fabsf(se), st, acc);
                                }
                                fb[b + j] = fmaf(-a.h, acc, Px[0]) + hF;
                            }
                        }
                    }
                    // Step 3: f = feq + (I + h/2 Lt)^-1 (fbar - feq)
                    float rkp = a.rkp, rk = a.rk;
                    if (PL) {
                        const float *k = rK + ((it - 2) % RK) * 2 * NT;
                        rkp = k[t];
                        rk = k[NT + t];
                    }
                    const Mom m = moments(fb, c);
                    float nq[10], f[10];
                    noneq(fb, m, inv2c, nq);
                    relax10(fb, nq, rkp, rk, f);
#pragma unroll
                    for (int k = 0; k < NPLANES; ++k) Fq[k * NT + t] = f[k];
                    float w[10];
                    if (xadj_plus) {  // west wall node of this row
                        nee(f, a.uw[0], a.vw[0], inv2c, w);
#pragma unroll
                        for (int k = 0; k < NPLANES; ++k) Fq[k * NT + t - 1] = w[k];
                    }
                    if (xadj_minus) {
                        nee(f, a.uw[1], a.vw[1], inv2c, w);
#pragma unroll
                        for (int k = 0; k < NPLANES; ++k) Fq[k * NT + t + 1] = w[k];
                    }
                    if (a.ywall && q == 1) {  // south wall row (and corners) from row 1
                        float *F0 = rF + ((it - 3) % RF) * ROW;
                        nee(f, a.uw[2], a.vw[2], inv2c, w);
#pragma unroll
                        for (int k = 0; k < NPLANES; ++k) F0[k * NT + t] = w[k];
                        if (xadj_plus) {
                            nee(f, a.uw[0], a.vw[0], inv2c, w);
#pragma unroll
                            for (int k = 0; k < NPLANES; ++k) F0[k * NT + t - 1] = w[k];
                        }
                        if (xadj_minus) {
                            nee(f, a.uw[1], a.vw[1], inv2c, w);
#pragma unroll
                            for (int k = 0; k < NPLANES; ++k) F0[k * NT + t + 1] = w[k];
                        }
                    }
                }
            }
        }
        __syncthreads();
        // ------------------------------------------------ Stage C: row r = p - 4
        if (it >= 8 && t >= 4 && t < NT - 4) {
            const int r = p - 4;
            const bool active = (X >= 0 && X < a.nx) && !colx_wall && !(a.ywall && (r == 0 || r == a.ny - 1));
            if (active) {
                const int rw = r;  // r is inside [0, ny) by construction
                const float *Pr = rP + ((it - 4) % RP) * ROW;
                const float *Fr = rF + ((it - 4) % RF) * ROW;
                const float *Fm2 = rF + ((it - 6) % RF) * ROW;
                const float *Fm1 = rF + ((it - 5) % RF) * ROW;
                const float *Fp1 = rF + ((it - 3) % RF) * ROW;
                const float *Fp2 = rF + ((it - 2) % RF) * ROW;
                const bool yadj_plus = a.ywall && r == 1;
                const bool yadj_minus = a.ywall && r == a.ny - 2;
                float fx = 0.0f, fy = 0.0f;
                if (a.force_mode == 1) { fx = a.Fx; fy = a.Fy; }
                else if (a.force_mode == 2) {
                    const long long fi = (long long)rw * a.pitch + GHOST + X;
                    fx = a.Fxp[fi]; fy = a.Fyp[fi];
                }
                float out[10];
#pragma unroll
                for (int al = 0; al < 2; ++al) {
                    const int b = 5 * al;
                    const float dF = a.dt * 0.2f * (al == 0 ? fx : fy);
                    out[b] = Pr[b * NT + t] + dF;
                    const float *P1 = Fr + (b + 1) * NT + t;
                    const float *P3 = Fr + (b + 3) * NT + t;
                    if (MK != METRIC_CURVILINEAR) {
                        const float kyr = (MK == METRIC_SEPARABLE) ? a.kyv[rw] : a.ky;
                        const float s1 = kxc * stencil(P1[1], P1[0], P1[-1], P1[-2], xadj_plus, a);
                        const float s3 = kxc * stencil(P3[-1], P3[0], P3[1], P3[2], xadj_minus, a);
                        const float s2 = kyr * stencil(Fp1[(b + 2) * NT + t], Fr[(b + 2) * NT + t],
                                                       Fm1[(b + 2) * NT + t], Fm2[(b + 2) * NT + t], yadj_plus, a);
                        const float s4 = kyr * stencil(Fm1[(b + 4) * NT + t], Fr[(b + 4) * NT + t],
                                                       Fp1[(b + 4) * NT + t], Fp2[(b + 4) * NT + t], yadj_minus, a);
                        out[b + 1] = fmaf(-a.dt, s1, Pr[(b + 1) * NT + t]) + dF;
                        out[b + 3] = fmaf(-a.dt, s3, Pr[(b + 3) * NT + t]) + dF;
                        out[b + 2] = fmaf(-a.dt, s2, Pr[(b + 2) * NT + t]) + dF;
                        out[b + 4] = fmaf(-a.dt, s4, Pr[(b + 4) * NT + t]) + dF;
                    } else {
                        const long long mi = (long long)rw * a.pitch + GHOST + X;
                        const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
#pragma unroll
                        for (int j = 1; j <= 4; ++j) {
                            const float sx = (j == 1) ? cxx : (j == 2) ? cxy : (j == 3) ? -cxx : -cxy;
                            const float se = (j == 1) ? cex : (j == 2) ? cey : (j == 3) ? -cex : -cey;
                            const float *Px = Fr + (b + j) * NT + t;
                            float acc = 0.0f;
                            if (sx != 0.0f) {
                                const float st = sx > 0.0f ? stencil(Px[1], Px[0], Px[-1], Px[-2], xadj_plus, a)
                                                           : stencil(Px[-1], Px[0], Px[1], Px[2], xadj_minus, a);
                                acc = fabsf(sx) * st;
                            }
                            if (se != 0.0f) {
                                const float pm2 = Fm2[(b + j) * NT + t], pm1 = Fm1[(b + j) * NT + t];
                                const float pp1 = Fp1[(b + j) * NT + t], pp2 = Fp2[(b + j) * NT + t];
                                const float st = se > 0.0f ? stencil(pp1, Px[0], pm1, pm2, yadj_plus, a)
                                                           : stencil(pm1, Px[0], pp1, pp2, yadj_minus, a);
                                acc = fmaf(fabsf(se), st, acc);
                            }
                            out[b + j] = fmaf(-a.dt, acc, Pr[(b + j) * NT + t]) + dF;
                        }
                    }
                }
                store_node(a, rw, X, out);
                // Walls after Step 4: NEE from this interior node.
                if (a.xwall || a.ywall) {
                    float w[10];
                    if (xadj_plus) { nee(out, a.uw[0], a.vw[0], inv2c, w); store_node(a, rw, 0, w); }
                    if (xadj_minus) { nee(out, a.uw[1], a.vw[1], inv2c, w); store_node(a, rw, a.nx - 1, w); }
                    if (a.ywall && (r == 1 || r == a.ny - 2)) {
                        const int rr = (r == 1) ? 0 : a.ny - 1;
                        const int side = (r == 1) ? 2 : 3;
                        nee(out, a.uw[side], a.vw[side], inv2c, w);
                        store_node(a, rr, X, w);
                        if (xadj_plus) { nee(out, a.uw[0], a.vw[0], inv2c, w); store_node(a, rr, 0, w); }
                        if (xadj_minus) { nee(out, a.uw[1], a.vw[1], inv2c, w); store_node(a, rr, a.nx - 1, w); }
                    }
                }
            }
        }
    }
    // On an aborted march, wait (bounded) for the row copies still in flight
    // before the block's shared memory is released, and report the fault.
    if (s_abort) {
        if (t == 0) {
            for (int it = issued - TMA_SLOTS; it < issued; ++it) {
                if (it < 0) continue;
                mbar_wait_bounded(&mbar[it % TMA_SLOTS], (uint32_t)((it / TMA_SLOTS) & 1));
            }
            atomicCAS(a.err, DEVERR_NONE, DEVERR_TMA_TIMEOUT);
        }
    }
}

template <int NT, int MK, bool PL>
int smem_bytes() {
    return (TMA_SLOTS + RB + RF + RP) * NPLANES * NT * 4 + (PL ? RK * 2 * NT * 4 : 0) + TMA_SLOTS * 8;
}

template <int NT, int MK, bool PL>
cudaError_t launch_t(const CUtensorMap *tmap, const StepArgs &args, const StepPlan &plan, cudaStream_t stream) {
    auto k = step_kernel<NT, MK, PL>;
    const int smem = smem_bytes<NT, MK, PL>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k<<<dim3(plan.gx, plan.gy), NT, smem, stream>>>(*tmap, args);
    return cudaGetLastError();
}

template <int NT, int MK, bool PL>
cudaError_t occupancy_t(int *occ) {
    auto k = step_kernel<NT, MK, PL>;
    const int smem = smem_bytes<NT, MK, PL>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, NT, smem);
}

constexpr int kNT = 128;

}  // namespace

int step_pitch(int nx, int W) {
    const int strips = (nx + W - 1) / W;
    const int cols = strips * W + 2 * GHOST;
    return ((cols + 31) / 32) * 32;
}

#define MDF_DISPATCH(FN, ...)                                                              \
    switch (metric * 2 + (power_law ? 1 : 0)) {                                             \
        case 0: return FN<kNT, METRIC_UNIFORM, false>(__VA_ARGS__);                         \
        case 1: return FN<kNT, METRIC_UNIFORM, true>(__VA_ARGS__);                          \
        case 2: return FN<kNT, METRIC_SEPARABLE, false>(__VA_ARGS__);                       \
        case 3: return FN<kNT, METRIC_SEPARABLE, true>(__VA_ARGS__);                        \
        case 4: return FN<kNT, METRIC_CURVILINEAR, false>(__VA_ARGS__);                     \
        default: return FN<kNT, METRIC_CURVILINEAR, true>(__VA_ARGS__);                     \
    }

static cudaError_t occupancy(int metric, int power_law, int *occ) { MDF_DISPATCH(occupancy_t, occ) }

cudaError_t step_plan(int metric, int power_law, int nx, int ny, int num_sms, StepPlan *plan) {
    plan->NT = kNT;
    plan->W = kNT - 8;
    int occ = 0;
    cudaError_t e = occupancy(metric, power_law, &occ);
    if (e != cudaSuccess) return e;
    plan->occ = occ;
    switch (metric * 2 + (power_law ? 1 : 0)) {
        case 0: plan->smem = smem_bytes<kNT, METRIC_UNIFORM, false>(); break;
        case 1: plan->smem = smem_bytes<kNT, METRIC_UNIFORM, true>(); break;
        case 2: plan->smem = smem_bytes<kNT, METRIC_SEPARABLE, false>(); break;
        case 3: plan->smem = smem_bytes<kNT, METRIC_SEPARABLE, true>(); break;
        case 4: plan->smem = smem_bytes<kNT, METRIC_CURVILINEAR, false>(); break;
        default: plan->smem = smem_bytes<kNT, METRIC_CURVILINEAR, true>(); break;
    }
    plan->gx = (nx + plan->W - 1) / plan->W;
    // Bands: enough blocks to fill every SM at the measured occupancy, but no
    // band shorter than 8 rows (the march recomputes 8 halo rows per band).
    const int slots = (occ > 0 ? occ : 1) * (num_sms > 0 ? num_sms : 1);
    int bands = slots / plan->gx;
    if (bands < 1) bands = 1;
    int H = (ny + bands - 1) / bands;
    if (H < 8) H = 8;
    plan->H = H;
    plan->gy = (ny + H - 1) / H;
    return cudaSuccess;
}

cudaError_t step_launch(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                        cudaStream_t stream) {
    const int power_law = args.power_law;
    MDF_DISPATCH(launch_t, tmap, args, plan, stream)
}

}  // namespace mdf
