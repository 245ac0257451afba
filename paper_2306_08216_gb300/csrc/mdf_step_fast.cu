// mdf_step_fast.cu -- fused MDF-FDLBM step for periodic Newtonian problems on
// uniform or separable (stretched) grids.
//
// Same time step as mdf_step.cu (Sec. 2.2 Steps (1)-(4) of arXiv:2306.08216
// with Eqs. 2.3.24-2.3.25, f32x2 pairs for alpha = u, v), with less shared
// memory per column so that more warps fit on an SM:
//  * populations 2 and 4 stream along y only, which is the direction each
//    thread marches, so their five-row windows of fbar^+ (pass 1) and of
//    f(t+h) (pass 2) live in registers;
//  * populations 1 and 3 stream along x only: their x stencils run on the row
//    just formed, through one-row exchange buffers, and the results wait in
//    registers until the y part of their row is ready;
//  * fhat^+ waits five rows in a shared ring (it is needed when the output
//    row is formed).
// The march is unrolled by five so every window index is a compile-time
// constant.  Per row, with p the newest row:
//   S0: output fhat(t+dt) of row r = p-5 (fhat^+ ring, register windows);
//   S2: row p of fhat by TMA; fhat^+ -> ring, fbar^+ of pops 1,3 -> exchange
//       buffer, of pops 2,4 -> register window;
//   -- the one barrier of the row --
//   S1: pass 2 x increments of row p-3 from the previous row's f exchange;
//   S3: pass 1 x part of row p; pass 1 y part, fbar and f(t+h) of row q = p-2;
//       f of pops 1,3 -> exchange buffer, of pops 2,4 -> register window.
// The exchange buffers are double-buffered by row parity, which is what lets
// a single barrier per row order every shared-memory hand-off.
//
// The alpha = 0 distribution (template flag RHO0, FP32 storage, 128 threads)
// rides along as a scalar lane with the same stages, windows and exchange
// rows: relaxed in S2 with the node's u, v; streamed in S1/S3 and recovered
// in S3 with the u, v of the alpha = 1, 2 fbar of its node; streamed in S0;
// source w_j R in both streaming steps (Eq. 2.1.2 with ubar_0 = rho_0,
// E_0 = 0).  Nothing of it flows back into alpha = 1, 2 (Remark 1).
#include <type_traits>

#include "mdf_device.cuh"

namespace mdf {

namespace {

using namespace dev;

// Rows of fhat in flight: four slots still leave two blocks of 256 threads
// per SM and measured 0.4 % faster than three at 4096^2.  With the alpha = 0
// lane (15 planes per row) three slots keep three blocks of 128 per SM.
constexpr int FAST_SLOTS = 4;
constexpr int FAST_SLOTS_RHO0 = 3;
constexpr int RHO0_NT = 128;

template <bool RHO0>
__host__ __device__ constexpr int fast_slots() {
    return RHO0 ? FAST_SLOTS_RHO0 : FAST_SLOTS;
}

__device__ __forceinline__ F2 pair_of(unsigned long long bits) {
    F2 a;
    a.r = bits;
    return a;
}

struct W3 {
    F2 w1, w0, w2;
};
// The same weights for the scalar alpha = 0 lane.
struct W1 {
    float w1, w0, w2;
};
__device__ __forceinline__ float lo(F2 p) {
    float x, y;
    split2(p, x, y);
    return x;
}
__device__ __forceinline__ W1 lo(const W3 &w) { return W1{lo(w.w1), lo(w.w0), lo(w.w2)}; }

__device__ __forceinline__ W3 weights(float k, float step, const StepArgs &a) {
    W3 w;
    w.w1 = splat(-step * k * a.a1);
    w.w0 = splat(-step * k * a.a0);
    w.w2 = splat(-step * k * a.am2);
    return w;
}

// Force increment factor (step/5) (Fx, Fy) at a node, F_{j,alpha} = w_j F_alpha:
// the h step's F, and the dt step's F + dt/2 dF/dt (Eq. 2.3.24).
__device__ __forceinline__ F2 force_at(const StepArgs &a, int row, int X, F2 factor) {
    if (a.force_mode == 0) return splat(0.0f);
    if (a.force_mode == 1) return factor * mk2(a.Fx, a.Fy);
    const long long fi = (long long)row * a.pitch + GHOST + X;
    return factor * mk2(a.Fxp[fi], a.Fyp[fi]);
}
__device__ __forceinline__ F2 force_at_d(const StepArgs &a, int row, int X, F2 factor) {
    if (a.force_mode_d == 0) return splat(0.0f);
    if (a.force_mode_d == 1) return factor * mk2(a.Fxd, a.Fyd);
    const long long fi = (long long)row * a.pitch + GHOST + X;
    return factor * mk2(a.Fxdp[fi], a.Fydp[fi]);
}

template <int NT, int MK, bool FORCED, int ST, bool RHO0>
__global__ void __launch_bounds__(NT, RHO0 ? 3 : (NT <= 128 ? 4 : 2))
    fast_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs a) {
    constexpr int SLOTS = fast_slots<RHO0>();
    // one TMA row: 10 FP32 planes (15 with alpha = 0), or u, v, P and 4
    // planes of 16-bit pairs
    constexpr int TROW = (RHO0 ? RHO0_PLANES : ST == STORAGE_FP32 ? NPLANES : DEV_PLANES) * NT * 4;
    constexpr int PROW = 5 * NT * 8;             // one fhat^+ ring row: 5 pairs x NT
    constexpr int XROW = 2 * NT * 8;             // one exchange row: pops 1, 3 x NT
    constexpr int P0ROW = RHO0 ? 5 * NT * 4 : 0;  // the same two for alpha = 0 (scalars)
    constexpr int X0ROW = RHO0 ? 2 * NT * 4 : 0;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *tma = smem;
    unsigned char *ringP = tma + SLOTS * TROW;
    unsigned char *xB0 = ringP + RING * PROW;  // fbar^+ of pops 1, 3 of row p (two buffers)
    unsigned char *xF0 = xB0 + 2 * XROW;       // f(t+h) of pops 1, 3 of row q (two buffers)
    unsigned char *ringP0 = xF0 + 2 * XROW;    // alpha = 0: fhat^+ ring, exchange rows
    unsigned char *xB00 = ringP0 + RING * P0ROW;
    unsigned char *xF00 = xB00 + 2 * X0ROW;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(xF00 + 2 * X0ROW);
    __shared__ int s_abort;

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * a.W;
    const int X = x0 - 4 + t;
    const int y0 = blockIdx.y * a.H;
    const int y1 = min(y0 + a.H, a.ny);
    const int nIt = (y1 - y0) + 9;
    const int rowBase = y0 - 4;
    const float c = a.c, inv2c = a.inv2c;
    constexpr bool forced = FORCED;

    if (t == 0) {
        s_abort = 0;
        for (int i = 0; i < SLOTS; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto load_row = [&](int it, int slot) {
        mbar_expect_tx(&mbar[slot], TROW);
        tma_load_row(&tmap, &mbar[slot], tma + slot * TROW, x0, wrap(rowBase + it, a.ny));
    };
    int issued = min(SLOTS, nIt);
    if (t == 0)
        for (int i = 0; i < issued; ++i) load_row(i, i);

    W3 wxh, wxd;
    if (MK == METRIC_UNIFORM) {
        wxh = {pair_of(a.pwxh[0]), pair_of(a.pwxh[1]), pair_of(a.pwxh[2])};
        wxd = {pair_of(a.pwxd[0]), pair_of(a.pwxd[1]), pair_of(a.pwxd[2])};
    } else {
        const float kx = a.kxv[GHOST + X];
        wxh = weights(kx, a.h, a);
        wxd = weights(kx, a.dt, a);
    }
    const F2 zero = splat(0.0f);
    // alpha = 0: the x weights and the rates of the three local maps
    const W1 wxh1 = lo(wxh), wxd1 = lo(wxd);
    const float mKp0 = lo(pair_of(a.pmKp)), Dp0 = lo(pair_of(a.pDp));
    const float mKb0 = lo(pair_of(a.pmKb)), Db0 = lo(pair_of(a.pDb));
    const float mKk0 = lo(pair_of(a.pmKk)), Dk0 = lo(pair_of(a.pDk));
    const float hw0 = a.h * 0.2f, dw0 = a.dt * 0.2f;
    const bool calc = t >= 2 && t < NT - 2;   // forms fbar and f
    const bool outc = t >= 4 && t < NT - 4 && X < a.nx;  // forms outputs

    // register windows, slot = (row - rowBase) mod 5
    F2 BY[5][2];    // fbar^+ of pops 2, 4
    F2 D013[5][3];  // fbar of pops 0, 1, 3 (x part done)
    F2 FY[5][2];    // f(t+h) of pops 2, 4
    F2 XF[5][2];    // pass-2 x increments of pops 1, 3
    float BY0[5][2], D0[5][3], FY0[5][2], XF0[5][2];  // the same windows for alpha = 0
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        BY[s][0] = BY[s][1] = FY[s][0] = FY[s][1] = XF[s][0] = XF[s][1] = zero;
        D013[s][0] = D013[s][1] = D013[s][2] = zero;
        BY0[s][0] = BY0[s][1] = FY0[s][0] = FY0[s][1] = XF0[s][0] = XF0[s][1] = 0.0f;
        D0[s][0] = D0[s][1] = D0[s][2] = 0.0f;
    }

    int tslot = 0;
    bool aborted = false;
    // One row iteration: window slot k of row p (row p-5 shares it), slots
    // s1..s4 of rows p-1 .. p-4, row ps of the fhat^+ rings.  Returns false
    // when the block aborts.
    auto row = [&](const int it, auto kc, const int ps) -> bool {
        constexpr int k = decltype(kc)::value;
        constexpr int s1 = (k + 4) % 5, s2 = (k + 3) % 5, s3 = (k + 2) % 5, s4 = (k + 1) % 5;
        {
            const int p = rowBase + it;
            // exchange buffers of this iteration (fbar^+) and of the previous one (f)
            unsigned char *xB = xB0 + (it & 1) * XROW;
            const unsigned char *xFp = xF0 + ((it & 1) ^ 1) * XROW;
            unsigned char *xF = xF0 + (it & 1) * XROW;
            unsigned char *xB_0 = xB00 + (it & 1) * X0ROW;
            const unsigned char *xFp_0 = xF00 + ((it & 1) ^ 1) * X0ROW;
            unsigned char *xF_0 = xF00 + (it & 1) * X0ROW;
            // ---------------------------------------------- S0: output row r = p - 5
            if (it >= 9 && outc) {
                // slot k of every window and of the ring holds row r
                const int r = p - 5;
                const unsigned char *Pr = ringP + ps * PROW;
                F2 out[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) out[j] = lds2(Pr, (j * NT + t) * 8);
                if (forced) {
                    const F2 fF = force_at_d(a, r, X, pair_of(a.pdw));
#pragma unroll
                    for (int j = 0; j < 5; ++j) out[j] = out[j] + fF;
                }
                out[1] = out[1] + XF[k][0];
                out[3] = out[3] + XF[k][1];
                W3 wy;
                if (MK == METRIC_UNIFORM) wy = {pair_of(a.pwyd[0]), pair_of(a.pwyd[1]), pair_of(a.pwyd[2])};
                else wy = weights(a.kyv[r], a.dt, a);
                // rows r-2, r-1, r, r+1, r+2 -> slots s2, s1, k, s4, s3
                out[2] = stream2<false>(out[2], FY[s4][0], FY[k][0], FY[s1][0], FY[s2][0], false, wy.w1, wy.w0,
                                        wy.w2);
                out[4] = stream2<false>(out[4], FY[s1][1], FY[k][1], FY[s4][1], FY[s3][1], false, wy.w1, wy.w0,
                                        wy.w2);
                if (ST == STORAGE_FP32) store_node<true>(a, r, X, out);
                else store_node_dev<ST, true>(a, r, X, out);
                if (RHO0) {
                    // Step 4 on alpha = 0: fhat^+ - dt c.grad f + dt w_j R
                    const unsigned char *P0r = ringP0 + ps * P0ROW;
                    float out0[5];
#pragma unroll
                    for (int j = 0; j < 5; ++j) out0[j] = lds1(P0r, (j * NT + t) * 4);
                    if (forced && a.r_mode) {
                        const float sR = dw0 * source_at(a, r, X);
#pragma unroll
                        for (int j = 0; j < 5; ++j) out0[j] += sR;
                    }
                    out0[1] += XF0[k][0];
                    out0[3] += XF0[k][1];
                    const W1 wy1 = lo(wy);
                    out0[2] = stream1<false>(out0[2], FY0[s4][0], FY0[k][0], FY0[s1][0], FY0[s2][0], false, wy1.w1,
                                             wy1.w0, wy1.w2);
                    out0[4] = stream1<false>(out0[4], FY0[s1][1], FY0[k][1], FY0[s4][1], FY0[s3][1], false, wy1.w1,
                                             wy1.w0, wy1.w2);
                    store_node0<true>(a, r, X, out0);
                }
            }
            // ---------------------------------------------- S2: row p
            F2 own1, own3;
            float own01 = 0.0f, own03 = 0.0f;
            {
                const bool ok = mbar_wait_bounded(&mbar[tslot], (uint32_t)((it / SLOTS) & 1));
                if (!ok) atomicExch(&s_abort, 1);
                const float *src = reinterpret_cast<const float *>(tma + tslot * TROW);
                F2 g[5], n[5], o[5];
                if (ST == STORAGE_FP32) {
#pragma unroll
                    for (int j = 0; j < 5; ++j) g[j] = mk2(src[j * NT + t], src[(5 + j) * NT + t]);
                    const Mom2 m = (forced && a.r_mode)
                                       ? moments2r(g, c, a.rk_hat * source_at(a, wrap(p, a.ny), X))
                                       : moments2(g, c);
                    noneq2(g, m, inv2c, n);
                    if (RHO0) {
                        // Step 1 on alpha = 0 with u, v of this node and the same rates
                        float g0[5], n0[5], q0[5];
#pragma unroll
                        for (int j = 0; j < 5; ++j) g0[j] = src[(NPLANES + j) * NT + t];
                        noneq0(g0, m.u, m.v, inv2c, n0);
                        relax0(g0, n0, mKp0, Dp0, q0);
                        unsigned char *dP0 = ringP0 + ps * P0ROW;
#pragma unroll
                        for (int j = 0; j < 5; ++j) sts1(dP0, (j * NT + t) * 4, q0[j]);
                        relax0(g0, n0, mKb0, Db0, q0);
                        sts1(xB_0, t * 4, q0[1]);
                        sts1(xB_0, (NT + t) * 4, q0[3]);
                        own01 = q0[1];
                        own03 = q0[3];
                        BY0[k][0] = q0[2];
                        BY0[k][1] = q0[4];
                        D0[k][0] = q0[0];
                    }
                } else {
                    // fhat = feq(u, v, P) + n: the stored macroscopic fields
                    // give the equilibrium directly
                    const unsigned *w = reinterpret_cast<const unsigned *>(src + DEV_FPLANES * NT);
                    const F2 inv = splat(a.ninv);
                    F2 nn[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) nn[j] = unpack16<ST>(w[j * NT + t]) * inv;
                    dev_build(src[t], src[NT + t], src[2 * NT + t], nn, inv2c, g, n);
                }
                const F2 n13 = n[1] - n[3], n24 = n[2] - n[4];
                relax2(g, n, n13, n24, pair_of(a.pmKp), pair_of(a.pDp), o);
                unsigned char *dP = ringP + ps * PROW;
#pragma unroll
                for (int j = 0; j < 5; ++j) sts2(dP, (j * NT + t) * 8, o[j]);
                relax2(g, n, n13, n24, pair_of(a.pmKb), pair_of(a.pDb), o);
                sts2(xB, t * 8, o[1]);
                sts2(xB, (NT + t) * 8, o[3]);
                own1 = o[1];
                own3 = o[3];
                BY[k][0] = o[2];
                BY[k][1] = o[4];
                D013[k][0] = o[0];
            }
            // One barrier per row: the exchange rows are double-buffered, so
            // the buffers written before this barrier are read only after it,
            // and those read after it are rewritten only after the next one.
            if (__syncthreads_or(s_abort)) return false;
            if (t == 0 && issued < nIt) {
                fence_proxy_async();
                load_row(issued, tslot);
                ++issued;
            }
            tslot = (tslot == SLOTS - 1) ? 0 : tslot + 1;
            // ---------------------------------------------- S1: pass-2 x increments of row p-3
            if (it >= 5 && outc) {
                const F2 f1p1 = lds2(xFp, (t + 1) * 8), f1 = lds2(xFp, t * 8);
                const F2 f1m1 = lds2(xFp, (t - 1) * 8), f1m2 = lds2(xFp, (t - 2) * 8);
                const F2 f3m1 = lds2(xFp, (NT + t - 1) * 8), f3 = lds2(xFp, (NT + t) * 8);
                const F2 f3p1 = lds2(xFp, (NT + t + 1) * 8), f3p2 = lds2(xFp, (NT + t + 2) * 8);
                XF[s3][0] = stream2<false>(zero, f1p1, f1, f1m1, f1m2, false, wxd.w1, wxd.w0, wxd.w2);
                XF[s3][1] = stream2<false>(zero, f3m1, f3, f3p1, f3p2, false, wxd.w1, wxd.w0, wxd.w2);
                if (RHO0) {
                    XF0[s3][0] = stream1<false>(0.0f, lds1(xFp_0, (t + 1) * 4), lds1(xFp_0, t * 4),
                                                lds1(xFp_0, (t - 1) * 4), lds1(xFp_0, (t - 2) * 4), false, wxd1.w1,
                                                wxd1.w0, wxd1.w2);
                    XF0[s3][1] = stream1<false>(0.0f, lds1(xFp_0, (NT + t - 1) * 4), lds1(xFp_0, (NT + t) * 4),
                                                lds1(xFp_0, (NT + t + 1) * 4), lds1(xFp_0, (NT + t + 2) * 4), false,
                                                wxd1.w1, wxd1.w0, wxd1.w2);
                }
            }
            // ---------------------------------------------- S3
            if (calc) {
                // pass 1, x part of row p: fbar = fbar^+ - h c.grad fbar^+ + h w F
                F2 b1 = own1, b3 = own3;
                if (forced) {
                    const F2 hF = force_at(a, wrap(p, a.ny), X, pair_of(a.phw));
                    D013[k][0] = D013[k][0] + hF;
                    b1 = b1 + hF;
                    b3 = b3 + hF;
                }
                D013[k][1] = stream2<false>(b1, lds2(xB, (t + 1) * 8), own1, lds2(xB, (t - 1) * 8),
                                            lds2(xB, (t - 2) * 8), false, wxh.w1, wxh.w0, wxh.w2);
                D013[k][2] = stream2<false>(b3, lds2(xB, (NT + t - 1) * 8), own3, lds2(xB, (NT + t + 1) * 8),
                                            lds2(xB, (NT + t + 2) * 8), false, wxh.w1, wxh.w0, wxh.w2);
                if (RHO0) {
                    // the same on alpha = 0, with h w_j R
                    float b01 = own01, b03 = own03;
                    if (forced && a.r_mode) {
                        const float sR = hw0 * source_at(a, wrap(p, a.ny), X);
                        D0[k][0] += sR;
                        b01 += sR;
                        b03 += sR;
                    }
                    D0[k][1] = stream1<false>(b01, lds1(xB_0, (t + 1) * 4), own01, lds1(xB_0, (t - 1) * 4),
                                              lds1(xB_0, (t - 2) * 4), false, wxh1.w1, wxh1.w0, wxh1.w2);
                    D0[k][2] = stream1<false>(b03, lds1(xB_0, (NT + t - 1) * 4), own03, lds1(xB_0, (NT + t + 1) * 4),
                                              lds1(xB_0, (NT + t + 2) * 4), false, wxh1.w1, wxh1.w0, wxh1.w2);
                }
                if (it >= 4) {
                    // row q = p - 2 (slot s2); fbar^+ rows q-2..q+2 -> slots s4, s3, s2, s1, k
                    const int qw = wrap(p - 2, a.ny);
                    F2 by2 = BY[s2][0], by4 = BY[s2][1];
                    if (forced) {
                        const F2 hFq = force_at(a, qw, X, pair_of(a.phw));
                        by2 = by2 + hFq;
                        by4 = by4 + hFq;
                    }
                    W3 wy;
                    if (MK == METRIC_UNIFORM) wy = {pair_of(a.pwyh[0]), pair_of(a.pwyh[1]), pair_of(a.pwyh[2])};
                    else wy = weights(a.kyv[qw], a.h, a);
                    F2 fb[5];
                    fb[0] = D013[s2][0];
                    fb[1] = D013[s2][1];
                    fb[3] = D013[s2][2];
                    fb[2] = stream2<false>(by2, BY[s1][0], BY[s2][0], BY[s3][0], BY[s4][0], false, wy.w1, wy.w0, wy.w2);
                    fb[4] = stream2<false>(by4, BY[s3][1], BY[s2][1], BY[s1][1], BY[k][1], false, wy.w1, wy.w0, wy.w2);
                    // Step 3: f = feq + (I + h/2 Lt)^-1 (fbar - feq)
                    const Mom2 m = (forced && a.r_mode) ? moments2r(fb, c, a.rk_bar * source_at(a, qw, X))
                                                        : moments2(fb, c);
                    F2 n[5], f[5];
                    noneq2(fb, m, inv2c, n);
                    relax2(fb, n, n[1] - n[3], n[2] - n[4], pair_of(a.pmKk), pair_of(a.pDk), f);
                    sts2(xF, t * 8, f[1]);
                    sts2(xF, (NT + t) * 8, f[3]);
                    FY[s2][0] = f[2];
                    FY[s2][1] = f[4];
                    if (RHO0) {
                        // Steps 2-3 on alpha = 0, recovered with u, v of the alpha = 1, 2 fbar
                        float by02 = BY0[s2][0], by04 = BY0[s2][1];
                        if (forced && a.r_mode) {
                            const float sRq = hw0 * source_at(a, qw, X);
                            by02 += sRq;
                            by04 += sRq;
                        }
                        const W1 wy1 = lo(wy);
                        float fb0[5], n0[5], f0[5];
                        fb0[0] = D0[s2][0];
                        fb0[1] = D0[s2][1];
                        fb0[3] = D0[s2][2];
                        fb0[2] = stream1<false>(by02, BY0[s1][0], BY0[s2][0], BY0[s3][0], BY0[s4][0], false, wy1.w1,
                                                wy1.w0, wy1.w2);
                        fb0[4] = stream1<false>(by04, BY0[s3][1], BY0[s2][1], BY0[s1][1], BY0[k][1], false, wy1.w1,
                                                wy1.w0, wy1.w2);
                        noneq0(fb0, m.u, m.v, inv2c, n0);
                        relax0(fb0, n0, mKk0, Dk0, f0);
                        sts1(xF_0, t * 4, f0[1]);
                        sts1(xF_0, (NT + t) * 4, f0[3]);
                        FY0[s2][0] = f0[2];
                        FY0[s2][1] = f0[4];
                    }
                }
            }
        }
        return true;
    };
    // The march, unrolled by five so that every window slot is a
    // compile-time index.  (A rolled form whose windows rotate by one row,
    // as the batched wall march has, measured 3.5 % slower on the alpha = 0
    // variant at 4096^2.)
    using std::integral_constant;
    for (int it0 = 0; it0 < nIt && !aborted; it0 += 5) {
        if (!row(it0, integral_constant<int, 0>{}, 0)) { aborted = true; break; }
        if (it0 + 1 >= nIt) break;
        if (!row(it0 + 1, integral_constant<int, 1>{}, 1)) { aborted = true; break; }
        if (it0 + 2 >= nIt) break;
        if (!row(it0 + 2, integral_constant<int, 2>{}, 2)) { aborted = true; break; }
        if (it0 + 3 >= nIt) break;
        if (!row(it0 + 3, integral_constant<int, 3>{}, 3)) { aborted = true; break; }
        if (it0 + 4 >= nIt) break;
        if (!row(it0 + 4, integral_constant<int, 4>{}, 4)) { aborted = true; break; }
    }
    (void)aborted;
    if (s_abort) {
        if (t == 0) {
            for (int it = issued - SLOTS; it < issued; ++it) {
                if (it < 0) continue;
                mbar_wait_bounded(&mbar[it % SLOTS], (uint32_t)((it / SLOTS) & 1));
            }
            atomicCAS(a.err, DEVERR_NONE, DEVERR_TMA_TIMEOUT);
        }
    }
}

template <int NT, int ST, bool RHO0>
constexpr int fast_smem() {
    return fast_slots<RHO0>() * (RHO0 ? RHO0_PLANES : ST == STORAGE_FP32 ? NPLANES : DEV_PLANES) * NT * 4 +
           RING * 5 * NT * 8 + 4 * (2 * NT * 8) + (RHO0 ? RING * 5 * NT * 4 + 4 * (2 * NT * 4) : 0) +
           fast_slots<RHO0>() * 8;
}

template <int NT, int MK, bool FORCED, int ST, bool RHO0>
cudaError_t fast_launch_t(const CUtensorMap *tmap, const StepArgs &args,
                          const StepPlan &plan, cudaStream_t stream) {
    auto k = fast_kernel<NT, MK, FORCED, ST, RHO0>;
    constexpr int smem = fast_smem<NT, ST, RHO0>();
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    k<<<dim3(plan.gx, plan.gy), NT, smem, stream>>>(*tmap, args);
    return cudaGetLastError();
}

template <int NT, int MK, int ST, bool RHO0>
cudaError_t fast_occupancy_t(int *occ, int *smem) {
    // both force variants have the same shared memory; take the smaller occupancy
    int o1 = 0, o2 = 0;
    *smem = fast_smem<NT, ST, RHO0>();
    cudaError_t e = cudaFuncSetAttribute(fast_kernel<NT, MK, false, ST, RHO0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fast_kernel<NT, MK, true, ST, RHO0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 *smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, fast_kernel<NT, MK, false, ST, RHO0>, NT, *smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, fast_kernel<NT, MK, true, ST, RHO0>, NT, *smem);
    *occ = o1 < o2 ? o1 : o2;
    return e;
}

template <int NT, int MK, int ST, bool RHO0>
cudaError_t fast_launch_f(const CUtensorMap *tmap, const StepArgs &args,
                          const StepPlan &plan, cudaStream_t stream) {
    return (args.force_mode || args.force_mode_d || args.r_mode)
               ? fast_launch_t<NT, MK, true, ST, RHO0>(tmap, args, plan, stream)
               : fast_launch_t<NT, MK, false, ST, RHO0>(tmap, args, plan, stream);
}

template <int NT, int MK>
cudaError_t fast_occupancy_s(int storage, int *occ, int *smem) {
    switch (storage) {
        case STORAGE_FP16: return fast_occupancy_t<NT, MK, STORAGE_FP16, false>(occ, smem);
        case STORAGE_BF16: return fast_occupancy_t<NT, MK, STORAGE_BF16, false>(occ, smem);
        default: return fast_occupancy_t<NT, MK, STORAGE_FP32, false>(occ, smem);
    }
}

template <int NT, int MK>
cudaError_t fast_launch_s(const CUtensorMap *tmap, const StepArgs &args,
                          const StepPlan &plan, cudaStream_t stream) {
    switch (args.storage) {
        case STORAGE_FP16: return fast_launch_f<NT, MK, STORAGE_FP16, false>(tmap, args, plan, stream);
        case STORAGE_BF16: return fast_launch_f<NT, MK, STORAGE_BF16, false>(tmap, args, plan, stream);
        default: return fast_launch_f<NT, MK, STORAGE_FP32, false>(tmap, args, plan, stream);
    }
}

}  // namespace

bool fast_path_applies(int metric, int power_law, int walls) {
    return !walls && !power_law && (metric == METRIC_UNIFORM || metric == METRIC_SEPARABLE);
}

cudaError_t fast_occupancy(int metric, int storage, int rho0, int nt, int *occ, int *smem) {
    if (rho0) {
        // the alpha = 0 lane: FP32 storage, 128 threads only
        *occ = 0;
        *smem = 0;
        if (nt != RHO0_NT || storage != STORAGE_FP32) return cudaSuccess;
        return metric == METRIC_UNIFORM ? fast_occupancy_t<RHO0_NT, METRIC_UNIFORM, STORAGE_FP32, true>(occ, smem)
                                        : fast_occupancy_t<RHO0_NT, METRIC_SEPARABLE, STORAGE_FP32, true>(occ, smem);
    }
    if (nt == 256)
        return metric == METRIC_UNIFORM ? fast_occupancy_s<256, METRIC_UNIFORM>(storage, occ, smem)
                                        : fast_occupancy_s<256, METRIC_SEPARABLE>(storage, occ, smem);
    return metric == METRIC_UNIFORM ? fast_occupancy_s<128, METRIC_UNIFORM>(storage, occ, smem)
                                    : fast_occupancy_s<128, METRIC_SEPARABLE>(storage, occ, smem);
}

cudaError_t fast_launch(const CUtensorMap *tmap, const StepArgs &args, int metric,
                        const StepPlan &plan, cudaStream_t stream) {
    if (args.rho0) {
        if (plan.NT != RHO0_NT || args.storage != STORAGE_FP32) return cudaErrorInvalidConfiguration;
        return metric == METRIC_UNIFORM
                   ? fast_launch_f<RHO0_NT, METRIC_UNIFORM, STORAGE_FP32, true>(tmap, args, plan, stream)
                   : fast_launch_f<RHO0_NT, METRIC_SEPARABLE, STORAGE_FP32, true>(tmap, args, plan, stream);
    }
    if (plan.NT == 256)
        return metric == METRIC_UNIFORM ? fast_launch_s<256, METRIC_UNIFORM>(tmap, args, plan, stream)
                                        : fast_launch_s<256, METRIC_SEPARABLE>(tmap, args, plan, stream);
    return metric == METRIC_UNIFORM ? fast_launch_s<128, METRIC_UNIFORM>(tmap, args, plan, stream)
                                    : fast_launch_s<128, METRIC_SEPARABLE>(tmap, args, plan, stream);
}

}  // namespace mdf
