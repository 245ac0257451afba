// mdf_device.cuh -- device helpers shared by the fused step kernels:
// packed f32x2 pairs, TMA/mbarrier primitives with bounded waits, and the
// local maps of the MDF-FDLBM step (moments, equilibrium, relaxation,
// non-equilibrium extrapolation, mixed-scheme streaming increment).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mdf_internal.cuh"

namespace mdf {
namespace dev {

constexpr int TMA_SLOTS = 3;  // rows of fhat in flight
constexpr int RING = 5;       // rows of every shared ring (stencil reach 2 + 2)

// ------------------------------------------------------------ f32x2 pairs

struct F2 {
    unsigned long long r;
};

__device__ __forceinline__ F2 mk2(float x, float y) {
    F2 a;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a.r) : "f"(x), "f"(y));
    return a;
}
__device__ __forceinline__ F2 splat(float x) { return mk2(x, x); }
__device__ __forceinline__ void split2(F2 a, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.r));
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}
__device__ __forceinline__ F2 sel2(bool p, F2 a, F2 b) {
    F2 d;
    d.r = p ? a.r : b.r;
    return d;
}
__device__ __forceinline__ F2 lds2(const unsigned char *base, int byte_off) {
    F2 a;
    a.r = *reinterpret_cast<const unsigned long long *>(base + byte_off);
    return a;
}
__device__ __forceinline__ void sts2(unsigned char *base, int byte_off, F2 a) {
    *reinterpret_cast<unsigned long long *>(base + byte_off) = a.r;
}
__device__ __forceinline__ float lds1(const unsigned char *base, int byte_off) {
    return *reinterpret_cast<const float *>(base + byte_off);
}
__device__ __forceinline__ void sts1(unsigned char *base, int byte_off, float v) {
    *reinterpret_cast<float *>(base + byte_off) = v;
}

// ------------------------------------------------- programmatic dependent launch

// A kernel launched with programmatic stream serialization may start while
// the previous kernel of its stream still runs.  grid_dependency_wait blocks
// (in hardware, no spin of ours) until that kernel has completed and its
// memory is visible; it must precede every global load of data the previous
// kernel writes and every global store to memory it reads.  Launched without
// the attribute it returns at once.  launch_dependents lets the next such
// kernel of the stream be scheduled; it changes no ordering of memory
// (the next kernel's own wait still covers the whole of this one).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------ TMA, mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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
__device__ __forceinline__ void tma_load_row(const CUtensorMap *map, uint64_t *bar, void *dst, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------ local maps

// Node in pair form: g[j] = (g_{j,u}, g_{j,v}), j = 0..4.
// Moments shared by fhat, fbar and f: (u, v) = sum_j g_j, the odd
// differences (g1 - g3), (g2 - g4) and P of Eq. 2.3.23 without the source
// term (moments2r adds it).
struct Mom2 {
    F2 uv, d13, d24;
    float u, v, P;
};

__device__ __forceinline__ Mom2 moments2(const F2 g[5], float c) {
    Mom2 m;
    m.uv = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
    m.d13 = g[1] - g[3];
    m.d24 = g[2] - g[4];
    float d1x, d2x, d1y, d2y;
    split2(m.d13, d1x, d2x);
    split2(m.d24, d1y, d2y);
    split2(m.uv, m.u, m.v);
    m.P = 0.5f * (c * (d1x + d2y) - m.u * m.u - m.v * m.v);
    return m;
}

// As moments2, with the source term of Eq. 2.3.23 added to P: pr =
// (cs^2/s)(1 + k s/2) R / 2 for a distribution whose non-equilibrium first
// moment carries the factor 1 + k s/2 (k = dt for fhat, h for fbar).
__device__ __forceinline__ Mom2 moments2r(const F2 g[5], float c, float pr) {
    Mom2 m = moments2(g, c);
    m.P += pr;
    return m;
}

// Index checks of the debug build (-DMDF_DEBUG): a global access outside
// its buffer is skipped and raises DEVERR_INDEX in the error word (no trap,
// the context stays usable); the release build compiles them out.
__device__ __forceinline__ bool index_ok(const StepArgs &a, long long e, long long limit) {
#ifdef MDF_DEBUG
    if (e >= 0 && e < limit) return true;
    atomicCAS(a.err, DEVERR_NONE, DEVERR_INDEX);
    return false;
#else
    (void)a;
    (void)e;
    (void)limit;
    return true;
#endif
}
// An element of the state buffer (every plane of the storage mode).
__device__ __forceinline__ bool state_index_ok(const StepArgs &a, long long e) {
    return index_ok(a, e, (long long)state_planes(a.storage, a.rho0) * a.plane);
}
// A pair of padded field planes (force, force rate) at element e.
__device__ __forceinline__ F2 field_pair(const StepArgs &a, const float *fx, const float *fy, long long e) {
    if (!index_ok(a, e, a.plane)) return splat(0.0f);
    return mk2(fx[e], fy[e]);
}

// Source R of Eq. 2.1.1 at storage element (row, X) (constant or padded field).
__device__ __forceinline__ float source_at(const StepArgs &a, int row, int X) {
    if (a.r_mode == 1) return a.Rc;
    const long long e = (long long)row * a.pitch + GHOST + X;
    return index_ok(a, e, a.plane) ? a.Rp[e] : 0.0f;
}

// Non-equilibrium part n = g - feq (Eq. 2.2.5 on D2Q5 with w_j = 1/5 and
// cs^2 = 2c^2/5: feq_0 = ub/5, feq_{1,3} = ub/5 +- Phi_x/(2c),
// feq_{2,4} = ub/5 +- Phi_y/(2c), Phi = ub_alpha u + P E_alpha).  feq_0 is
// formed as ub - 4 ub/5 so that sum_j feq_j = ub carries no rounding bias of
// the constant 1/5; otherwise every step would scale the conserved zeroth
// moments by the same FP32 factor and the drift would grow linearly in time.
__device__ __forceinline__ void noneq2(const F2 g[5], const Mom2 &m, float inv2c, F2 n[5]) {
    const F2 u5 = splat(0.2f) * m.uv;
    const float uu = fmaf(m.u, m.u, m.P) * inv2c, uv = m.u * m.v * inv2c, vv = fmaf(m.v, m.v, m.P) * inv2c;
    const F2 fx = mk2(uu, uv), fy = mk2(uv, vv);
    n[0] = g[0] - fma2(splat(-4.0f), u5, m.uv);
    n[1] = g[1] - (u5 + fx);
    n[3] = g[3] - (u5 - fx);
    n[2] = g[2] - (u5 + fy);
    n[4] = g[4] - (u5 - fy);
}

// Local relaxation shared by Steps 1 and 3, as an increment:
// out = g - (1 - Ap) n + (A - Ap) P_c n, which equals
// feq + Ap (g - feq) + (A - Ap) P_c (g - feq); Ap / A are the eigenvalues on
// the free / first-moment subspaces, (P_c n)_{1,3} = +-(n_1 - n_3)/2 and
// (P_c n)_{2,4} = +-(n_2 - n_4)/2.  The zeroth moment is kept up to unbiased
// per-node rounding.  n13 = n1 - n3, n24 = n2 - n4; mK = -(1 - Ap),
// D = (A - Ap)/2.
__device__ __forceinline__ void relax2(const F2 g[5], const F2 n[5], F2 n13, F2 n24, F2 mK, F2 D, F2 out[5]) {
    const F2 dx = D * n13, dy = D * n24;
    out[0] = fma2(mK, n[0], g[0]);
    out[1] = fma2(mK, n[1], g[1]) + dx;
    out[3] = fma2(mK, n[3], g[3]) - dx;
    out[2] = fma2(mK, n[2], g[2]) + dy;
    out[4] = fma2(mK, n[4], g[4]) - dy;
}

// Non-equilibrium extrapolation: node value = g_nb + feq(u_w, P) - feq(u_nb, P)
// (the pressure cancels in the difference of the linear equilibria).
__device__ __forceinline__ void nee2(const F2 g[5], float uw, float vw, float inv2c, F2 out[5]) {
    float un, vn;
    split2((g[0] + g[1]) + (g[2] + g[3]) + g[4], un, vn);
    const float du = 0.2f * (uw - un), dv = 0.2f * (vw - vn);
    const float uux = (uw * uw - un * un) * inv2c, uvy = (uw * vw - un * vn) * inv2c;
    const float vvy = (vw * vw - vn * vn) * inv2c;
    out[0] = g[0] + mk2(du, dv);
    out[1] = g[1] + mk2(du + uux, dv + uvy);
    out[3] = g[3] + mk2(du - uux, dv - uvy);
    out[2] = g[2] + mk2(du + uvy, dv + vvy);
    out[4] = g[4] + mk2(du - uvy, dv - vvy);
}

// Eigenvalues of the three local maps for first-moment rate s (s' = s_ratio s):
// rho(l) = (1 - dt l/2)/(1 + dt l/2) for I - Lambda, (1 + 3 rho)/4 for
// I - 3 Lambda/4, 1/(1 + h l/2) for (I + h/2 Lt)^-1.
struct Rates {
    float rpp, rp, rbp, rb, rkp, rk;
};
// Rates of the three local maps at a node of viscosity nu, with s = cs^2/nu
// and s' = s_ratio s: rho(l) = (1 - dt l/2)/(1 + dt l/2) (Eq. 2.2.14),
// 1/4 + 3/4 rho(l) (Eq. 2.2.15) and kappa(l) = 1/(1 + h l/2) (Eq. 2.2.16) for
// l = s, s', written in nu (c1 = cs^2 dt/2) so that the per-node power-law
// solve needs no quotient for s; the quotients take the fast reciprocal
// (2 ulp).
__device__ __forceinline__ Rates rates_nu(float nu, float s_ratio, float c1) {
    const float c1p = s_ratio * c1;
    Rates r;
    r.rpp = __fdividef(nu - c1p, nu + c1p);
    r.rp = __fdividef(nu - c1, nu + c1);
    r.rbp = 0.25f * (1.0f + 3.0f * r.rpp);
    r.rb = 0.25f * (1.0f + 3.0f * r.rp);
    r.rkp = __fdividef(nu, nu + 0.5f * c1p);
    r.rk = __fdividef(nu, nu + 0.5f * c1);
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
    const float lnK = a.lnK, lng = __logf(g);
    const float lmin = a.ln_nu_min, lmax = a.ln_nu_max;
    // the start is the root when cs^2 dt/2 << nu; Newton converges
    // quadratically from it, and its step only needs F (no division) to be
    // exact at the root, so the step may use the fast approximate quotient
    float l = (lnK + (n - 1.0f) * lng) * a.inv_n;
    l = fminf(fmaxf(l, lmin), lmax);
    // four steps: from this start (clamped to [nu_min, nu_max], where the
    // root lies too) three already reach the FP32 evaluation floor of the
    // residual (1.5e-6 relative) over n in [0.5, 1.5], Re in [100, 5000],
    // grids of 65-513 nodes and strain rates from 1e-12 to 1e6 of the
    // reference rate; kept rolled: the call sits in five-fold unrolled
    // marches, and unrolled copies cost instruction-cache misses
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
        const float e = __expf(l);
        const float F = l - lnK - (n - 1.0f) * (lng - __logf(e + a.a_pl));
        const float dF = 1.0f + (n - 1.0f) * __fdividef(e, e + a.a_pl);
        l = l - __fdividef(F, dF);
        l = fminf(fmaxf(l, lmin - 1.0f), lmax + 1.0f);
    }
    return fminf(fmaxf(__expf(l), a.nu_min), a.nu_max);
}

// Streaming increment along one axis for a population moving towards +chi
// (pf = Pi(+1), pb1 = Pi(-1), pb2 = Pi(-2)) or -chi (mirrored), added to
// `base`:  w1 (Pi(+1) - Pi(-1)) + w0 (Pi(0) - Pi(-1)) + w2 (Pi(-2) - Pi(-1)),
// the mixed scheme of Eqs. 2.2.12-2.2.13 written in differences (its weights
// sum to zero, so a uniform field gives exactly zero).  Next to a wall the
// far point is 2 Pi(-1) - Pi(0).  The weights carry -h c/dx (or -dt c/dx).
template <bool WALLS>
__device__ __forceinline__ F2 stream2(F2 base, F2 pf, F2 p0, F2 pb1, F2 pb2, bool wall_adj, F2 w1, F2 w0, F2 w2) {
    const F2 d0 = p0 - pb1;
    F2 dfar = pb2 - pb1;
    if (WALLS) dfar = sel2(wall_adj, splat(0.0f) - d0, dfar);
    return fma2(w1, pf - pb1, fma2(w0, d0, fma2(w2, dfar, base)));
}

// ---- the alpha = 0 (rho_0) lane: one scalar distribution of 5 populations
// with ubar_0 = rho_0 and E_0 = 0 (Eq. 2.1.2), feq_{j,0} = w_j (rho_0 +
// c_j.(rho_0 u)/cs^2): rho_0/5 for j = 0 (as rho_0 - 4 rho_0/5) and
// rho_0/5 +- rho_0 u/(2c), rho_0/5 +- rho_0 v/(2c) for j = 1,3 and 2,4.

// Non-equilibrium part n = g - feq_0(sum g, u, v).
__device__ __forceinline__ void noneq0(const float g[5], float u, float v, float inv2c, float n[5]) {
    const float rho = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
    const float r5 = 0.2f * rho;
    const float fx = rho * u * inv2c, fy = rho * v * inv2c;
    n[0] = g[0] - fmaf(-4.0f, r5, rho);
    n[1] = g[1] - (r5 + fx);
    n[3] = g[3] - (r5 - fx);
    n[2] = g[2] - (r5 + fy);
    n[4] = g[4] - (r5 - fy);
}

// The local maps of relax2 on the scalar lane.
__device__ __forceinline__ void relax0(const float g[5], const float n[5], float mK, float D, float out[5]) {
    const float dx = D * (n[1] - n[3]), dy = D * (n[2] - n[4]);
    out[0] = fmaf(mK, n[0], g[0]);
    out[1] = fmaf(mK, n[1], g[1]) + dx;
    out[3] = fmaf(mK, n[3], g[3]) - dx;
    out[2] = fmaf(mK, n[2], g[2]) + dy;
    out[4] = fmaf(mK, n[4], g[4]) - dy;
}

// Wall node of the rho_0 lane: g_nb + feq_0(rho_nb, u_w) - feq_0(rho_nb, u_nb)
// (the wall's rho_0 is the neighbour's; (un, vn) is the neighbour's velocity).
__device__ __forceinline__ void nee0(const float g[5], float uw, float vw, float un, float vn, float inv2c,
                                     float out[5]) {
    const float rho = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
    const float dx = rho * (uw - un) * inv2c, dy = rho * (vw - vn) * inv2c;
    out[0] = g[0];
    out[1] = g[1] + dx;
    out[3] = g[3] - dx;
    out[2] = g[2] + dy;
    out[4] = g[4] - dy;
}

// stream2 on the scalar lane.
template <bool WALLS>
__device__ __forceinline__ float stream1(float base, float pf, float p0, float pb1, float pb2, bool wall_adj, float w1,
                                         float w0, float w2) {
    const float d0 = p0 - pb1;
    float dfar = pb2 - pb1;
    if (WALLS && wall_adj) dfar = -d0;
    return fmaf(w1, pf - pb1, fmaf(w0, d0, fmaf(w2, dfar, base)));
}

// Rotate a register window by one row for a rolled march (the register-
// window marches that keep their loop rolled).  Its window slots follow the slot formula of the unrolled march with the slot of the
// newest row p fixed at 0: row p - a sits in slot (5 - a) mod 5 (row p - 1 in
// slot 4, ..., row p - 4 in slot 1, and slot 0 before the write of row p
// still holds row p - 5).  Advancing p moves every row to the slot below it
// (modulo 5): new[i] = old[(i + 1) mod 5].
template <typename T, int N>
__device__ __forceinline__ void rot5(T (&w)[5][N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const T w0 = w[0][i];
        w[0][i] = w[1][i];
        w[1][i] = w[2][i];
        w[2][i] = w[3][i];
        w[3][i] = w[4][i];
        w[4][i] = w0;
    }
}

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Store one node (5 pairs -> 10 planes), with its periodic image in the ghost
// columns when the x axis is periodic.
template <bool XPER>
__device__ __forceinline__ void store_node(const StepArgs &a, int row, int X, const F2 v[5]) {
    const long long base = (long long)row * a.pitch + GHOST + X;
    float lo[5], hi[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) split2(v[j], lo[j], hi[j]);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if (state_index_ok(a, j * a.plane + base)) a.fout[j * a.plane + base] = lo[j];
        if (state_index_ok(a, (5 + j) * a.plane + base)) a.fout[(5 + j) * a.plane + base] = hi[j];
    }
    if (XPER) {
        // a node can be the image of a ghost on both sides when nx < 2 GHOST
        if (X < GHOST) {
            const long long b2 = base + a.nx;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                if (state_index_ok(a, j * a.plane + b2)) a.fout[j * a.plane + b2] = lo[j];
                if (state_index_ok(a, (5 + j) * a.plane + b2)) a.fout[(5 + j) * a.plane + b2] = hi[j];
            }
        }
        if (X >= a.nx - GHOST) {
            const long long b2 = base - a.nx;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                if (state_index_ok(a, j * a.plane + b2)) a.fout[j * a.plane + b2] = lo[j];
                if (state_index_ok(a, (5 + j) * a.plane + b2)) a.fout[(5 + j) * a.plane + b2] = hi[j];
            }
        }
    }
}


// ------------------------------------------------------------ 16-bit storage

// 16-bit pair word (low half: alpha = u, high half: alpha = v) <-> pair.
// Store the rho_0 lane of one node (planes 10..14), with its periodic
// images in the ghost columns when the x axis is periodic.
template <bool XPER>
__device__ __forceinline__ void store_node0(const StepArgs &a, int row, int X, const float v[5]) {
    const long long base = (long long)row * a.pitch + GHOST + X;
#pragma unroll
    for (int j = 0; j < 5; ++j)
        if (state_index_ok(a, (NPLANES + j) * a.plane + base)) a.fout[(NPLANES + j) * a.plane + base] = v[j];
    if (XPER) {
        if (X < GHOST)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (state_index_ok(a, (NPLANES + j) * a.plane + base + a.nx))
                    a.fout[(NPLANES + j) * a.plane + base + a.nx] = v[j];
        if (X >= a.nx - GHOST)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (state_index_ok(a, (NPLANES + j) * a.plane + base - a.nx))
                    a.fout[(NPLANES + j) * a.plane + base - a.nx] = v[j];
    }
}

template <int ST>
__device__ __forceinline__ F2 unpack16(unsigned w) {
    float2 f;
    if (ST == STORAGE_FP16) {
        __half2 h;
        memcpy(&h, &w, 4);
        f = __half22float2(h);
    } else {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        f = __bfloat1622float2(h);
    }
    return mk2(f.x, f.y);
}
template <int ST>
__device__ __forceinline__ unsigned pack16(F2 a) {
    float x, y;
    split2(a, x, y);
    unsigned w;
    if (ST == STORAGE_FP16) {
        const __half2 h = __floats2half2_rn(x, y);
        memcpy(&w, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        memcpy(&w, &h, 4);
    }
    return w;
}

// Node of the 16-bit layouts: fhat = feq(u, v, P) + n with
// n_0 = -(n_1 + n_2 + n_3 + n_4); nn[j - 1] = n_j (j = 1..4, unscaled).
// Returns the pairs g = fhat and n.
__device__ __forceinline__ void dev_build(float u, float v, float P, const F2 nn[4], float inv2c, F2 g[5],
                                          F2 n[5]) {
#pragma unroll
    for (int j = 1; j < 5; ++j) n[j] = nn[j - 1];
    n[0] = splat(0.0f) - ((n[1] + n[2]) + (n[3] + n[4]));
    const F2 uv = mk2(u, v);
    const F2 u5 = splat(0.2f) * uv;
    const float uu = fmaf(u, u, P) * inv2c, uvv = u * v * inv2c, vv = fmaf(v, v, P) * inv2c;
    const F2 fx = mk2(uu, uvv), fy = mk2(uvv, vv);
    g[0] = fma2(splat(-4.0f), u5, uv) + n[0];
    g[1] = (u5 + fx) + n[1];
    g[3] = (u5 - fx) + n[3];
    g[2] = (u5 + fy) + n[2];
    g[4] = (u5 - fy) + n[4];
}

// Store one node in a 16-bit layout at element e of every plane.
__device__ __forceinline__ void dev_store_at(const StepArgs &a, long long e, float u, float v, float P,
                                             const unsigned w[4]) {
    float *fp = a.fout;
    unsigned *wp = reinterpret_cast<unsigned *>(fp);
    if (state_index_ok(a, e)) fp[e] = u;
    if (state_index_ok(a, a.plane + e)) fp[a.plane + e] = v;
    if (state_index_ok(a, 2 * a.plane + e)) fp[2 * a.plane + e] = P;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (state_index_ok(a, (DEV_FPLANES + j) * a.plane + e)) wp[(DEV_FPLANES + j) * a.plane + e] = w[j];
}

// Output of one node (5 pairs of fhat) in a 16-bit layout: moments and
// non-equilibrium part as the FP32 path forms them on load, n scaled by S
// and rounded to 16 bits.
template <int ST, bool XPER>
__device__ __forceinline__ void store_node_dev(const StepArgs &a, int row, int X, const F2 v[5]) {
    const Mom2 m = moments2(v, a.c);
    F2 n[5];
    noneq2(v, m, a.inv2c, n);
    const F2 S = splat(a.nscale);
    unsigned w[4];
#pragma unroll
    for (int j = 1; j < 5; ++j) w[j - 1] = pack16<ST>(n[j] * S);
    const long long base = (long long)row * a.pitch + GHOST + X;
    dev_store_at(a, base, m.u, m.v, m.P, w);
    if (XPER) {
        if (X < GHOST) dev_store_at(a, base + a.nx, m.u, m.v, m.P, w);
        if (X >= a.nx - GHOST) dev_store_at(a, base - a.nx, m.u, m.v, m.P, w);
    }
}

}  // namespace dev
}  // namespace mdf
