// mdf_march.cuh -- the shared-ring march of the fused step (curvilinear
// grids, and every grid when the alpha = 0 distribution is evolved): the
// device function, its kernels and their launch helpers, included by
// mdf_step.cu (alpha = 1, 2 only) and mdf_step_rho0.cu (with alpha = 0).
//
// Arithmetic layout.  The two distributions alpha = u, v (Eq. 2.1.2 with
// alpha = 1, 2) see the same collision rates and the same difference
// weights, so each population j is carried as one 64-bit pair
// (fhat_{j,u}, fhat_{j,v}) and processed with the packed FP32 instructions
// of sm_100-family GPUs (add/sub/mul/fma .f32x2); shared rings hold the
// pairs, so every ring access is one 64-bit load or store.
//
// Work decomposition.  A block owns a strip of W = NT - 8 output columns and
// marches down a band of H rows.  Thread t holds column x0 - 4 + t; the 8
// extra columns are the halo of the two chained stencils (reach 2 + 2).  Per
// row of the march, with p the newest row:
//   C: fhat(t+dt) of row r = p - 5 from the f ring and the fhat^+ ring -> HBM;
//   A: row p of fhat arrives by TMA (one 3-D box of 10 planes x NT columns);
//      fhat^+ and fbar^+ of row p go to their rings;
//   -- barrier --
//   B: fbar and f(t+h) of row q = p - 2 (x stencils across threads, y
//      stencils across ring rows) go to the f ring; walls by NEE;
//   -- barrier --
// All rings have five rows; slot offsets rotate by one each row.  Only the x
// halo (8 of NT columns) and 9 rows per band are recomputed; every row is
// read from HBM once.  Walls use non-equilibrium extrapolation written by the
// interior neighbour's thread, and the second-order upwind point beyond a
// wall is replaced by its linear extrapolation Pi(-1) = 2 Pi(0) - Pi(1).
//
// The alpha = 0 lane (template flag RHO0) carries fhat_{j,0} (planes
// 10..14) through the same stages as scalars, in three more rings of 5 x NT
// floats: relaxed in stage A with the node's u, v; streamed and recovered in
// stage B with the u, v of the alpha = 1, 2 fbar; streamed in stage C; walls
// by non-equilibrium extrapolation with the neighbour's rho_0.
#pragma once

#include "mdf_device.cuh"

namespace mdf {

namespace {

using namespace dev;

// Shared-memory layout of one ring row: 5 pairs x NT columns, 8 bytes each.
template <int NT>
struct Ring {
    static constexpr int ROW = 5 * NT * 8;  // bytes per ring row
    static __device__ __forceinline__ int at(int j, int t) { return (j * NT + t) * 8; }
};

// The alpha = 0 rings: 5 populations x NT columns, 4 bytes each (half a
// pair ring row, so a pair ring's byte offset halved addresses the same row).
template <int NT>
struct Ring0 {
    static constexpr int ROW = 5 * NT * 4;
    static __device__ __forceinline__ int at(int j, int t) { return (j * NT + t) * 4; }
};

// Difference weights of one axis for pass 1 (h) and pass 2 (dt):
// w = -step * k * (a1, a0, am2) with k = c/dx (or c times the metric).
struct AxisW {
    F2 h1, h0, h2, d1, d0, d2;
};
__device__ __forceinline__ AxisW axis_weights(float k, const StepArgs &a) {
    AxisW w;
    w.h1 = splat(-a.h * k * a.a1);
    w.h0 = splat(-a.h * k * a.a0);
    w.h2 = splat(-a.h * k * a.am2);
    w.d1 = splat(-a.dt * k * a.a1);
    w.d0 = splat(-a.dt * k * a.a0);
    w.d2 = splat(-a.dt * k * a.am2);
    return w;
}

// The same weights as scalars (the alpha = 0 lane).
struct AxisW1 {
    float h1, h0, h2, d1, d0, d2;
};
__device__ __forceinline__ AxisW1 axis_weights1(float k, const StepArgs &a) {
    return AxisW1{-a.h * k * a.a1, -a.h * k * a.a0, -a.h * k * a.am2, -a.dt * k * a.a1, -a.dt * k * a.a0,
                  -a.dt * k * a.am2};
}

// Streaming increment of population j (1..4) at a curvilinear node, added to
// base: -step (|ct_xi| D_xi + |ct_eta| D_eta), upwinded by the sign of ct.
// rows[0..4] are the ring rows of chi_eta - 2 .. chi_eta + 2.
template <int NT>
__device__ __forceinline__ F2 curvi_term(const unsigned char *const rows[5], int j, int t, float cxi, float ceta,
                                         bool xadj_p, bool xadj_m, bool yadj_p, bool yadj_m, float step,
                                         const StepArgs &a, F2 base) {
    using R = Ring<NT>;
    const unsigned char *mid = rows[2];
    const F2 p0 = lds2(mid, R::at(j, t));
    F2 acc = base;
    if (cxi != 0.0f) {
        const float k = -step * fabsf(cxi);
        const F2 w1 = splat(k * a.a1), w0 = splat(k * a.a0), w2 = splat(k * a.am2);
        if (cxi > 0.0f)
            acc = stream2<true>(acc, lds2(mid, R::at(j, t + 1)), p0, lds2(mid, R::at(j, t - 1)),
                                lds2(mid, R::at(j, t - 2)), xadj_p, w1, w0, w2);
        else
            acc = stream2<true>(acc, lds2(mid, R::at(j, t - 1)), p0, lds2(mid, R::at(j, t + 1)),
                                lds2(mid, R::at(j, t + 2)), xadj_m, w1, w0, w2);
    }
    if (ceta != 0.0f) {
        const float k = -step * fabsf(ceta);
        const F2 w1 = splat(k * a.a1), w0 = splat(k * a.a0), w2 = splat(k * a.am2);
        if (ceta > 0.0f)
            acc = stream2<true>(acc, lds2(rows[3], R::at(j, t)), p0, lds2(rows[1], R::at(j, t)),
                                lds2(rows[0], R::at(j, t)), yadj_p, w1, w0, w2);
        else
            acc = stream2<true>(acc, lds2(rows[1], R::at(j, t)), p0, lds2(rows[3], R::at(j, t)),
                                lds2(rows[4], R::at(j, t)), yadj_m, w1, w0, w2);
    }
    return acc;
}

// curvi_term on the alpha = 0 rings.
template <int NT>
__device__ __forceinline__ float curvi_term0(const unsigned char *const rows[5], int j, int t, float cxi, float ceta,
                                             bool xadj_p, bool xadj_m, bool yadj_p, bool yadj_m, float step,
                                             const StepArgs &a, float base) {
    using R = Ring0<NT>;
    const unsigned char *mid = rows[2];
    const float p0 = lds1(mid, R::at(j, t));
    float acc = base;
    if (cxi != 0.0f) {
        const float k = -step * fabsf(cxi);
        const float w1 = k * a.a1, w0 = k * a.a0, w2 = k * a.am2;
        if (cxi > 0.0f)
            acc = stream1<true>(acc, lds1(mid, R::at(j, t + 1)), p0, lds1(mid, R::at(j, t - 1)),
                                lds1(mid, R::at(j, t - 2)), xadj_p, w1, w0, w2);
        else
            acc = stream1<true>(acc, lds1(mid, R::at(j, t - 1)), p0, lds1(mid, R::at(j, t + 1)),
                                lds1(mid, R::at(j, t + 2)), xadj_m, w1, w0, w2);
    }
    if (ceta != 0.0f) {
        const float k = -step * fabsf(ceta);
        const float w1 = k * a.a1, w0 = k * a.a0, w2 = k * a.am2;
        if (ceta > 0.0f)
            acc = stream1<true>(acc, lds1(rows[3], R::at(j, t)), p0, lds1(rows[1], R::at(j, t)),
                                lds1(rows[0], R::at(j, t)), yadj_p, w1, w0, w2);
        else
            acc = stream1<true>(acc, lds1(rows[1], R::at(j, t)), p0, lds1(rows[3], R::at(j, t)),
                                lds1(rows[4], R::at(j, t)), yadj_m, w1, w0, w2);
    }
    return acc;
}

// Streaming of the alpha = 0 lane at one node: out[1..4] += the increments
// of pass `dt` (pass 2) or `h` (pass 1) from the ring rows
// rows[0..4] = chi - 2 .. chi + 2.
template <int NT, int MK, bool WALLS>
__device__ __forceinline__ void stream_lane0(const unsigned char *const rows[5], int t, const AxisW1 &wx,
                                             const AxisW1 &wy, bool pass2, bool xadj_p, bool xadj_m, bool yadj_p,
                                             bool yadj_m, const StepArgs &a, long long mi, float out[5]) {
    using R = Ring0<NT>;
    const unsigned char *C = rows[2];
    if (MK != METRIC_CURVILINEAR) {
        const float x1 = pass2 ? wx.d1 : wx.h1, x0 = pass2 ? wx.d0 : wx.h0, x2 = pass2 ? wx.d2 : wx.h2;
        const float y1 = pass2 ? wy.d1 : wy.h1, y0 = pass2 ? wy.d0 : wy.h0, y2 = pass2 ? wy.d2 : wy.h2;
        out[1] = stream1<WALLS>(out[1], lds1(C, R::at(1, t + 1)), lds1(C, R::at(1, t)), lds1(C, R::at(1, t - 1)),
                                lds1(C, R::at(1, t - 2)), xadj_p, x1, x0, x2);
        out[3] = stream1<WALLS>(out[3], lds1(C, R::at(3, t - 1)), lds1(C, R::at(3, t)), lds1(C, R::at(3, t + 1)),
                                lds1(C, R::at(3, t + 2)), xadj_m, x1, x0, x2);
        out[2] = stream1<WALLS>(out[2], lds1(rows[3], R::at(2, t)), lds1(C, R::at(2, t)),
                                lds1(rows[1], R::at(2, t)), lds1(rows[0], R::at(2, t)), yadj_p, y1, y0, y2);
        out[4] = stream1<WALLS>(out[4], lds1(rows[1], R::at(4, t)), lds1(C, R::at(4, t)),
                                lds1(rows[3], R::at(4, t)), lds1(rows[4], R::at(4, t)), yadj_m, y1, y0, y2);
    } else {
        const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
        const float step = pass2 ? a.dt : a.h;
        out[1] = curvi_term0<NT>(rows, 1, t, cxx, cex, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[1]);
        out[2] = curvi_term0<NT>(rows, 2, t, cxy, cey, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[2]);
        out[3] = curvi_term0<NT>(rows, 3, t, -cxx, -cex, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[3]);
        out[4] = curvi_term0<NT>(rows, 4, t, -cxy, -cey, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[4]);
    }
}

__device__ __forceinline__ void sum_uv(const F2 g[5], float &u, float &v) {
    split2((g[0] + g[1]) + (g[2] + g[3]) + g[4], u, v);
}

// One block's march over strip bx, band by of one problem.  `tmap` is the
// TMA descriptor of the input state, `a` the problem's arguments (kernel
// parameter space for a single problem, global memory for a batch).
template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
__device__ __forceinline__ void march(const CUtensorMap *tmap, const StepArgs &a, int bx, int by, unsigned char *smem,
                                      int *abort_flag) {
    using R = Ring<NT>;
    using R0 = Ring0<NT>;
    // bytes of one TMA row: 10 planes (15 with alpha = 0) x NT floats
    constexpr int TROW = (RHO0 ? RHO0_PLANES : NPLANES) * NT * 4;
    unsigned char *tma = smem;
    unsigned char *ringP = tma + TMA_SLOTS * TROW;   // fhat^+
    unsigned char *ringB = ringP + RING * R::ROW;    // fbar^+
    unsigned char *ringF = ringB + RING * R::ROW;    // f(t+h)
    float *ringK = reinterpret_cast<float *>(ringF + RING * R::ROW);  // power law: recovery rates
    // alpha = 0: fhat^+, fbar^+ and f rings, addressed with the pair offsets
    // halved; they take no shared memory without the lane
    constexpr int R0BYTES = RHO0 ? RING * R0::ROW : 0;
    unsigned char *ringP0 = reinterpret_cast<unsigned char *>(ringK + (PL ? RING * 2 * NT : 0));
    unsigned char *ringB0 = ringP0 + R0BYTES;
    unsigned char *ringF0 = ringB0 + R0BYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(ringF0 + R0BYTES);
    int &s_abort = *abort_flag;

    const int t = threadIdx.x;
    const int x0 = bx * a.W;
    const int X = x0 - 4 + t;
    const int y0 = by * a.H;
    const int y1 = min(y0 + a.H, a.ny);
    const int nIt = (y1 - y0) + 9;
    const int rowBase = y0 - 4;
    const float c = a.c, inv2c = a.inv2c;

    if (t == 0) {
        s_abort = 0;
        for (int i = 0; i < TMA_SLOTS; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto load_row = [&](int it, int slot) {
        const int p = rowBase + it;
        const int yy = (WALLS && a.ywall) ? p : wrap(p, a.ny);
        mbar_expect_tx(&mbar[slot], TROW);
        tma_load_row(tmap, &mbar[slot], tma + slot * TROW, x0, yy);
    };
    int issued = min(TMA_SLOTS, nIt);
    if (t == 0)
        for (int i = 0; i < issued; ++i) load_row(i, i);

    // per-column constants
    const bool xwall = WALLS && a.xwall;
    const bool ywall = WALLS && a.ywall;
    const bool colx_wall = xwall && (X == 0 || X == a.nx - 1);
    const bool colx_out = xwall && (X < 0 || X >= a.nx);
    const bool xadj_p = xwall && X == 1;
    const bool xadj_m = xwall && X == a.nx - 2;
    AxisW wx{}, wy{};
    if (MK == METRIC_UNIFORM) {
        wx = axis_weights(a.kx, a);
        wy = axis_weights(a.ky, a);
    } else if (MK == METRIC_SEPARABLE) {
        wx = axis_weights(a.kxv[GHOST + X], a);
    }
    AxisW1 wx1{}, wy1{};
    if (RHO0 && MK == METRIC_UNIFORM) {
        wx1 = axis_weights1(a.kx, a);
        wy1 = axis_weights1(a.ky, a);
    } else if (RHO0 && MK == METRIC_SEPARABLE) {
        wx1 = axis_weights1(a.kxv[GHOST + X], a);
    }
    const F2 hw = splat(a.h * 0.2f), dw = splat(a.dt * 0.2f);
    const F2 mKp = splat(-(1.0f - a.rpp)), Dp = splat(0.5f * (a.rp - a.rpp));
    const F2 mKb = splat(-(1.0f - a.rbp)), Db = splat(0.5f * (a.rb - a.rbp));
    const F2 mKk = splat(-(1.0f - a.rkp)), Dk = splat(0.5f * (a.rk - a.rkp));

    // Rotating slot offsets: o_k = byte offset of the ring row written k
    // iterations ago (every ring is indexed by iteration mod 5; o0 is the
    // slot written in the current iteration).
    int o0 = 0, o1 = 4 * R::ROW, o2 = 3 * R::ROW, o3 = 2 * R::ROW, o4 = 1 * R::ROW;
    int k0 = 0, k2 = 3 * 2 * NT;  // the same rotation for the power-law ring (floats)
    int tslot = 0;

    for (int it = 0; it < nIt; ++it) {
        const int p = rowBase + it;
        // ------------------------------------------------ Stage C: row r = p - 5
        if (it >= 9 && t >= 4 && t < NT - 4) {
            const int r = p - 5;
            bool active = (X >= 0 && X < a.nx);
            if (WALLS) active = active && !colx_wall && !(ywall && (r == 0 || r == a.ny - 1));
            if (active) {
                // F rows r-2..r+2 were written 5..1 iterations ago; fhat^+ of
                // row r 5 iterations ago (slot o0, rewritten by stage A below).
                const unsigned char *Fm2 = ringF + o0, *Fm1 = ringF + o4, *F0 = ringF + o3;
                const unsigned char *Fp1 = ringF + o2, *Fp2 = ringF + o1;
                const unsigned char *Pr = ringP + o0;
                const bool yadj_p = ywall && r == 1, yadj_m = ywall && r == a.ny - 2;
                F2 fF = splat(0.0f);
                if (a.force_mode_d == 1) fF = dw * mk2(a.Fxd, a.Fyd);
                else if (a.force_mode_d == 2) {
                    const long long fi = (long long)r * a.pitch + GHOST + X;
                    fF = dw * field_pair(a, a.Fxdp, a.Fydp, fi);
                }
                F2 out[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) out[j] = lds2(Pr, R::at(j, t)) + fF;
                if (MK != METRIC_CURVILINEAR) {
                    AxisW wyr = wy;
                    if (MK == METRIC_SEPARABLE) wyr = axis_weights(a.kyv[r], a);
                    out[1] = stream2<WALLS>(out[1], lds2(F0, R::at(1, t + 1)), lds2(F0, R::at(1, t)),
                                            lds2(F0, R::at(1, t - 1)), lds2(F0, R::at(1, t - 2)), xadj_p, wx.d1,
                                            wx.d0, wx.d2);
                    out[3] = stream2<WALLS>(out[3], lds2(F0, R::at(3, t - 1)), lds2(F0, R::at(3, t)),
                                            lds2(F0, R::at(3, t + 1)), lds2(F0, R::at(3, t + 2)), xadj_m, wx.d1,
                                            wx.d0, wx.d2);
                    out[2] = stream2<WALLS>(out[2], lds2(Fp1, R::at(2, t)), lds2(F0, R::at(2, t)),
                                            lds2(Fm1, R::at(2, t)), lds2(Fm2, R::at(2, t)), yadj_p, wyr.d1, wyr.d0,
                                            wyr.d2);
                    out[4] = stream2<WALLS>(out[4], lds2(Fm1, R::at(4, t)), lds2(F0, R::at(4, t)),
                                            lds2(Fp1, R::at(4, t)), lds2(Fp2, R::at(4, t)), yadj_m, wyr.d1, wyr.d0,
                                            wyr.d2);
                } else {
                    const long long mi = (long long)r * a.pitch + GHOST + X;
                    const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
                    const unsigned char *const rows[5] = {Fm2, Fm1, F0, Fp1, Fp2};
                    out[1] = curvi_term<NT>(rows, 1, t, cxx, cex, xadj_p, xadj_m, yadj_p, yadj_m, a.dt, a, out[1]);
                    out[2] = curvi_term<NT>(rows, 2, t, cxy, cey, xadj_p, xadj_m, yadj_p, yadj_m, a.dt, a, out[2]);
                    out[3] = curvi_term<NT>(rows, 3, t, -cxx, -cex, xadj_p, xadj_m, yadj_p, yadj_m, a.dt, a, out[3]);
                    out[4] = curvi_term<NT>(rows, 4, t, -cxy, -cey, xadj_p, xadj_m, yadj_p, yadj_m, a.dt, a, out[4]);
                }
                float out0[5];
                if (RHO0) {
                    // Step 4 on alpha = 0: fhat^+ - dt c.grad f + dt w_j R
                    const float sR = a.r_mode ? a.dt * 0.2f * source_at(a, r, X) : 0.0f;
                    const unsigned char *P0r = ringP0 + (o0 >> 1);
#pragma unroll
                    for (int j = 0; j < 5; ++j) out0[j] = lds1(P0r, R0::at(j, t)) + sR;
                    const unsigned char *const rows0[5] = {ringF0 + (o0 >> 1), ringF0 + (o4 >> 1), ringF0 + (o3 >> 1),
                                                           ringF0 + (o2 >> 1), ringF0 + (o1 >> 1)};
                    AxisW1 wyr1 = wy1;
                    if (MK == METRIC_SEPARABLE) wyr1 = axis_weights1(a.kyv[r], a);
                    stream_lane0<NT, MK, WALLS>(rows0, t, wx1, wyr1, true, xadj_p, xadj_m, yadj_p, yadj_m, a,
                                                (long long)r * a.pitch + GHOST + X, out0);
                }
                if (!WALLS) {
                    store_node<true>(a, r, X, out);
                    if (RHO0) store_node0<true>(a, r, X, out0);
                } else {
                    // the x axis of a walled kernel may still be periodic
                    if (xwall) store_node<false>(a, r, X, out);
                    else store_node<true>(a, r, X, out);
                    F2 w[5];
                    float w0[5], un = 0.0f, vn = 0.0f;
                    if (RHO0) {
                        if (xwall) store_node0<false>(a, r, X, out0);
                        else store_node0<true>(a, r, X, out0);
                        sum_uv(out, un, vn);
                    }
                    if (xadj_p) {
                        nee2(out, a.uw[0], a.vw[0], inv2c, w);
                        store_node<false>(a, r, 0, w);
                        if (RHO0) { nee0(out0, a.uw[0], a.vw[0], un, vn, inv2c, w0); store_node0<false>(a, r, 0, w0); }
                    }
                    if (xadj_m) {
                        nee2(out, a.uw[1], a.vw[1], inv2c, w);
                        store_node<false>(a, r, a.nx - 1, w);
                        if (RHO0) {
                            nee0(out0, a.uw[1], a.vw[1], un, vn, inv2c, w0);
                            store_node0<false>(a, r, a.nx - 1, w0);
                        }
                    }
                    if (ywall && (r == 1 || r == a.ny - 2)) {
                        const int rr = (r == 1) ? 0 : a.ny - 1;
                        const int side = (r == 1) ? 2 : 3;
                        nee2(out, a.uw[side], a.vw[side], inv2c, w);
                        if (xwall) store_node<false>(a, rr, X, w);
                        else store_node<true>(a, rr, X, w);
                        if (RHO0) {
                            nee0(out0, a.uw[side], a.vw[side], un, vn, inv2c, w0);
                            if (xwall) store_node0<false>(a, rr, X, w0);
                            else store_node0<true>(a, rr, X, w0);
                        }
                        if (xadj_p) {
                            nee2(out, a.uw[0], a.vw[0], inv2c, w);
                            store_node<false>(a, rr, 0, w);
                            if (RHO0) {
                                nee0(out0, a.uw[0], a.vw[0], un, vn, inv2c, w0);
                                store_node0<false>(a, rr, 0, w0);
                            }
                        }
                        if (xadj_m) {
                            nee2(out, a.uw[1], a.vw[1], inv2c, w);
                            store_node<false>(a, rr, a.nx - 1, w);
                            if (RHO0) {
                                nee0(out0, a.uw[1], a.vw[1], un, vn, inv2c, w0);
                                store_node0<false>(a, rr, a.nx - 1, w0);
                            }
                        }
                    }
                }
            }
        }
        // ------------------------------------------------ Stage A: row p
        {
            const bool ok = mbar_wait_bounded(&mbar[tslot], (uint32_t)((it / TMA_SLOTS) & 1));
            if (!ok) atomicExch(&s_abort, 1);
            const float *src = reinterpret_cast<const float *>(tma + tslot * TROW);
            F2 g[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) g[j] = mk2(src[j * NT + t], src[(5 + j) * NT + t]);
            const int pw = (WALLS && ywall) ? p : wrap(p, a.ny);
            const Mom2 m = a.r_mode && pw >= 0 && pw < a.ny && X >= -GHOST && X < a.nx + GHOST
                               ? moments2r(g, c, a.rk_hat * source_at(a, pw, X))
                               : moments2(g, c);
            F2 n[5];
            noneq2(g, m, inv2c, n);
            const F2 n13 = n[1] - n[3], n24 = n[2] - n[4];
            F2 mKp_ = mKp, Dp_ = Dp, mKb_ = mKb, Db_ = Db;
            float rpp = a.rpp, rp = a.rp, rbp = a.rbp, rb = a.rb;
            if (PL) {
                float gx1, gx2, gy1, gy2;
                split2(splat(c) * n13, gx1, gx2);
                split2(splat(c) * n24, gy1, gy2);
                const float sxy = 0.5f * (gy1 + gx2);
                const float gg = sqrtf(2.0f * (gx1 * gx1 + gy2 * gy2 + 2.0f * sxy * sxy));
                const Rates Rr = rates_nu(power_law_nu(gg, a), a.s_ratio, a.a_pl);
                mKp_ = splat(-(1.0f - Rr.rpp));
                Dp_ = splat(0.5f * (Rr.rp - Rr.rpp));
                mKb_ = splat(-(1.0f - Rr.rbp));
                Db_ = splat(0.5f * (Rr.rb - Rr.rbp));
                rpp = Rr.rpp; rp = Rr.rp; rbp = Rr.rbp; rb = Rr.rb;
                float *k = ringK + k0;
                k[t] = Rr.rkp;
                k[NT + t] = Rr.rk;
            }
            F2 o[5];
            relax2(g, n, n13, n24, mKp_, Dp_, o);
            unsigned char *dP = ringP + o0;
#pragma unroll
            for (int j = 0; j < 5; ++j) sts2(dP, R::at(j, t), o[j]);
            relax2(g, n, n13, n24, mKb_, Db_, o);
            unsigned char *dB = ringB + o0;
#pragma unroll
            for (int j = 0; j < 5; ++j) sts2(dB, R::at(j, t), o[j]);
            if (RHO0) {
                // Step 1 on alpha = 0 with u, v of this node and the same rates
                float g0[5], n0[5], q0[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) g0[j] = src[(NPLANES + j) * NT + t];
                noneq0(g0, m.u, m.v, inv2c, n0);
                relax0(g0, n0, -(1.0f - rpp), 0.5f * (rp - rpp), q0);
#pragma unroll
                for (int j = 0; j < 5; ++j) sts1(ringP0 + (o0 >> 1), R0::at(j, t), q0[j]);
                relax0(g0, n0, -(1.0f - rbp), 0.5f * (rb - rbp), q0);
#pragma unroll
                for (int j = 0; j < 5; ++j) sts1(ringB0 + (o0 >> 1), R0::at(j, t), q0[j]);
            }
        }
        // all threads are done with TMA slot `tslot`, with the rows stage C
        // read, and have written the ring rows of stage A
        if (__syncthreads_or(s_abort)) break;
        if (t == 0 && issued < nIt) {
            fence_proxy_async();
            load_row(issued, tslot);
            ++issued;
        }
        tslot = (tslot == TMA_SLOTS - 1) ? 0 : tslot + 1;
        // ------------------------------------------------ Stage B: row q = p - 2
        if (it >= 4 && t >= 2 && t < NT - 2) {
            const int q = p - 2;
            bool skip = false;
            if (WALLS) skip = colx_out || (ywall && (q < 0 || q >= a.ny));
            // the f row of q goes to slot o0 (the oldest f row, read by stage C above)
            unsigned char *Fq = ringF + o0;
            if (!skip) {
                if (WALLS && ywall && q == a.ny - 1) {
                    // north wall row: NEE from row ny-2 (this column, written last iteration)
                    if (!colx_wall) {
                        const unsigned char *Fn = ringF + o1;
                        F2 g[5], w[5];
#pragma unroll
                        for (int j = 0; j < 5; ++j) g[j] = lds2(Fn, R::at(j, t));
                        nee2(g, a.uw[3], a.vw[3], inv2c, w);
#pragma unroll
                        for (int j = 0; j < 5; ++j) sts2(Fq, R::at(j, t), w[j]);
                        float g0[5], w0[5], un = 0.0f, vn = 0.0f;
                        unsigned char *Fq0 = ringF0 + (o0 >> 1);
                        if (RHO0) {
#pragma unroll
                            for (int j = 0; j < 5; ++j) g0[j] = lds1(ringF0 + (o1 >> 1), R0::at(j, t));
                            sum_uv(g, un, vn);
                            nee0(g0, a.uw[3], a.vw[3], un, vn, inv2c, w0);
#pragma unroll
                            for (int j = 0; j < 5; ++j) sts1(Fq0, R0::at(j, t), w0[j]);
                        }
                        if (xadj_p) {
                            nee2(g, a.uw[0], a.vw[0], inv2c, w);
#pragma unroll
                            for (int j = 0; j < 5; ++j) sts2(Fq, R::at(j, t - 1), w[j]);
                            if (RHO0) {
                                nee0(g0, a.uw[0], a.vw[0], un, vn, inv2c, w0);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts1(Fq0, R0::at(j, t - 1), w0[j]);
                            }
                        }
                        if (xadj_m) {
                            nee2(g, a.uw[1], a.vw[1], inv2c, w);
#pragma unroll
                            for (int j = 0; j < 5; ++j) sts2(Fq, R::at(j, t + 1), w[j]);
                            if (RHO0) {
                                nee0(g0, a.uw[1], a.vw[1], un, vn, inv2c, w0);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts1(Fq0, R0::at(j, t + 1), w0[j]);
                            }
                        }
                    }
                } else if (!(WALLS && ((ywall && q == 0) || colx_wall))) {
                    // fbar^+ rows q-2..q+2 were written 4..0 iterations ago
                    const unsigned char *Bm2 = ringB + o4, *Bm1 = ringB + o3, *B0 = ringB + o2;
                    const unsigned char *Bp1 = ringB + o1, *Bp2 = ringB + o0;
                    const int qw = (WALLS && ywall) ? q : wrap(q, a.ny);
                    const bool yadj_p = ywall && q == 1, yadj_m = ywall && q == a.ny - 2;
                    F2 fF = splat(0.0f);
                    if (a.force_mode == 1) fF = hw * mk2(a.Fx, a.Fy);
                    else if (a.force_mode == 2) {
                        const long long fi = (long long)qw * a.pitch + GHOST + X;
                        fF = hw * field_pair(a, a.Fxp, a.Fyp, fi);
                    }
                    // Step 2 (pass 1): fbar = fbar^+ - h c.grad fbar^+ + h w F
                    F2 fb[5];
#pragma unroll
                    for (int j = 0; j < 5; ++j) fb[j] = lds2(B0, R::at(j, t)) + fF;
                    if (MK != METRIC_CURVILINEAR) {
                        AxisW wyq = wy;
                        if (MK == METRIC_SEPARABLE) wyq = axis_weights(a.kyv[qw], a);
                        fb[1] = stream2<WALLS>(fb[1], lds2(B0, R::at(1, t + 1)), lds2(B0, R::at(1, t)),
                                               lds2(B0, R::at(1, t - 1)), lds2(B0, R::at(1, t - 2)), xadj_p, wx.h1,
                                               wx.h0, wx.h2);
                        fb[3] = stream2<WALLS>(fb[3], lds2(B0, R::at(3, t - 1)), lds2(B0, R::at(3, t)),
                                               lds2(B0, R::at(3, t + 1)), lds2(B0, R::at(3, t + 2)), xadj_m, wx.h1,
                                               wx.h0, wx.h2);
                        fb[2] = stream2<WALLS>(fb[2], lds2(Bp1, R::at(2, t)), lds2(B0, R::at(2, t)),
                                               lds2(Bm1, R::at(2, t)), lds2(Bm2, R::at(2, t)), yadj_p, wyq.h1, wyq.h0,
                                               wyq.h2);
                        fb[4] = stream2<WALLS>(fb[4], lds2(Bm1, R::at(4, t)), lds2(B0, R::at(4, t)),
                                               lds2(Bp1, R::at(4, t)), lds2(Bp2, R::at(4, t)), yadj_m, wyq.h1, wyq.h0,
                                               wyq.h2);
                    } else {
                        const long long mi = (long long)qw * a.pitch + GHOST + X;
                        const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
                        const unsigned char *const rows[5] = {Bm2, Bm1, B0, Bp1, Bp2};
                        fb[1] = curvi_term<NT>(rows, 1, t, cxx, cex, xadj_p, xadj_m, yadj_p, yadj_m, a.h, a, fb[1]);
                        fb[2] = curvi_term<NT>(rows, 2, t, cxy, cey, xadj_p, xadj_m, yadj_p, yadj_m, a.h, a, fb[2]);
                        fb[3] = curvi_term<NT>(rows, 3, t, -cxx, -cex, xadj_p, xadj_m, yadj_p, yadj_m, a.h, a, fb[3]);
                        fb[4] = curvi_term<NT>(rows, 4, t, -cxy, -cey, xadj_p, xadj_m, yadj_p, yadj_m, a.h, a, fb[4]);
                    }
                    // Step 3: f = feq + (I + h/2 Lt)^-1 (fbar - feq)
                    F2 mKk_ = mKk, Dk_ = Dk;
                    if (PL) {
                        const float *k = ringK + k2;  // rates of row q, written 2 iterations ago
                        mKk_ = splat(-(1.0f - k[t]));
                        Dk_ = splat(0.5f * (k[NT + t] - k[t]));
                    }
                    const Mom2 m = a.r_mode ? moments2r(fb, c, a.rk_bar * source_at(a, qw, X)) : moments2(fb, c);
                    F2 n[5], f[5];
                    noneq2(fb, m, inv2c, n);
                    relax2(fb, n, n[1] - n[3], n[2] - n[4], mKk_, Dk_, f);
#pragma unroll
                    for (int j = 0; j < 5; ++j) sts2(Fq, R::at(j, t), f[j]);
                    float f0[5], w0[5], un = 0.0f, vn = 0.0f;
                    unsigned char *Fq0 = ringF0 + (o0 >> 1);
                    if (RHO0) {
                        // Steps 2-3 on alpha = 0: fbar = fbar^+ - h c.grad fbar^+ + h w_j R,
                        // recovered with u, v of the alpha = 1, 2 fbar and the same rates
                        float fb0[5], n0[5];
                        const float sR = a.r_mode ? a.h * 0.2f * source_at(a, qw, X) : 0.0f;
#pragma unroll
                        for (int j = 0; j < 5; ++j) fb0[j] = lds1(ringB0 + (o2 >> 1), R0::at(j, t)) + sR;
                        const unsigned char *const rows0[5] = {ringB0 + (o4 >> 1), ringB0 + (o3 >> 1),
                                                               ringB0 + (o2 >> 1), ringB0 + (o1 >> 1),
                                                               ringB0 + (o0 >> 1)};
                        AxisW1 wyq1 = wy1;
                        if (MK == METRIC_SEPARABLE) wyq1 = axis_weights1(a.kyv[qw], a);
                        stream_lane0<NT, MK, WALLS>(rows0, t, wx1, wyq1, false, xadj_p, xadj_m, yadj_p, yadj_m, a,
                                                    (long long)qw * a.pitch + GHOST + X, fb0);
                        float kp = a.rkp, kk = a.rk;
                        if (PL) {
                            const float *k = ringK + k2;
                            kp = k[t];
                            kk = k[NT + t];
                        }
                        noneq0(fb0, m.u, m.v, inv2c, n0);
                        relax0(fb0, n0, -(1.0f - kp), 0.5f * (kk - kp), f0);
#pragma unroll
                        for (int j = 0; j < 5; ++j) sts1(Fq0, R0::at(j, t), f0[j]);
                        sum_uv(f, un, vn);
                    }
                    if (WALLS) {
                        F2 w[5];
                        if (xadj_p) {  // west wall node of this row
                            nee2(f, a.uw[0], a.vw[0], inv2c, w);
#pragma unroll
                            for (int j = 0; j < 5; ++j) sts2(Fq, R::at(j, t - 1), w[j]);
                            if (RHO0) {
                                nee0(f0, a.uw[0], a.vw[0], un, vn, inv2c, w0);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts1(Fq0, R0::at(j, t - 1), w0[j]);
                            }
                        }
                        if (xadj_m) {
                            nee2(f, a.uw[1], a.vw[1], inv2c, w);
#pragma unroll
                            for (int j = 0; j < 5; ++j) sts2(Fq, R::at(j, t + 1), w[j]);
                            if (RHO0) {
                                nee0(f0, a.uw[1], a.vw[1], un, vn, inv2c, w0);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts1(Fq0, R0::at(j, t + 1), w0[j]);
                            }
                        }
                        if (ywall && q == 1) {  // south wall row (and corners) from row 1
                            unsigned char *F0r = ringF + o1;
                            unsigned char *F0r0 = ringF0 + (o1 >> 1);
                            nee2(f, a.uw[2], a.vw[2], inv2c, w);
#pragma unroll
                            for (int j = 0; j < 5; ++j) sts2(F0r, R::at(j, t), w[j]);
                            if (RHO0) {
                                nee0(f0, a.uw[2], a.vw[2], un, vn, inv2c, w0);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts1(F0r0, R0::at(j, t), w0[j]);
                            }
                            if (xadj_p) {
                                nee2(f, a.uw[0], a.vw[0], inv2c, w);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts2(F0r, R::at(j, t - 1), w[j]);
                                if (RHO0) {
                                    nee0(f0, a.uw[0], a.vw[0], un, vn, inv2c, w0);
#pragma unroll
                                    for (int j = 0; j < 5; ++j) sts1(F0r0, R0::at(j, t - 1), w0[j]);
                                }
                            }
                            if (xadj_m) {
                                nee2(f, a.uw[1], a.vw[1], inv2c, w);
#pragma unroll
                                for (int j = 0; j < 5; ++j) sts2(F0r, R::at(j, t + 1), w[j]);
                                if (RHO0) {
                                    nee0(f0, a.uw[1], a.vw[1], un, vn, inv2c, w0);
#pragma unroll
                                    for (int j = 0; j < 5; ++j) sts1(F0r0, R0::at(j, t + 1), w0[j]);
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // rotate: the slot written in this iteration becomes "1 iteration ago"
        {
            const int tmp = o4;
            o4 = o3; o3 = o2; o2 = o1; o1 = o0; o0 = tmp;
            if (PL) {
                k0 = (k0 == 4 * 2 * NT) ? 0 : k0 + 2 * NT;
                k2 = (k2 == 4 * 2 * NT) ? 0 : k2 + 2 * NT;
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
    // every copy was consumed: the barriers may be invalidated for reuse
    __syncthreads();
    if (t == 0)
        for (int i = 0; i < TMA_SLOTS; ++i) mbar_inval(&mbar[i]);
    __syncthreads();
}

template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
__global__ void __launch_bounds__(NT) step_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    march<NT, MK, PL, WALLS, RHO0>(&tmap, a, blockIdx.x, blockIdx.y, smem, &s_abort);
}

// Many problems in one persistent launch: block b takes work items
// b, b + gridDim.x, ... of the table (problem, strip, band), which lists the
// largest problems first.  Arguments and TMA descriptors live in global memory.
template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
__global__ void __launch_bounds__(NT) batch_kernel(const BatchItem *__restrict__ items, int nitems,
                                                   const StepArgs *__restrict__ args,
                                                   const CUtensorMap *__restrict__ maps) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const BatchItem item = items[w];
        march<NT, MK, PL, WALLS, RHO0>(&maps[item.problem], args[item.problem], item.bx, item.by, smem, &s_abort);
        if (s_abort) break;
    }
}

template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
int smem_bytes() {
    return TMA_SLOTS * (RHO0 ? RHO0_PLANES : NPLANES) * NT * 4 + 3 * RING * Ring<NT>::ROW +
           (PL ? RING * 2 * NT * 4 : 0) + (RHO0 ? 3 * RING * Ring0<NT>::ROW : 0) + TMA_SLOTS * 8;
}

template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
cudaError_t launch_t(const CUtensorMap *tmap, const StepArgs &args, const StepPlan &plan, cudaStream_t stream) {
    auto k = step_kernel<NT, MK, PL, WALLS, RHO0>;
    const int smem = smem_bytes<NT, MK, PL, WALLS, RHO0>();
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    k<<<dim3(plan.gx, plan.gy), NT, smem, stream>>>(*tmap, args);
    return cudaGetLastError();
}

template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
cudaError_t occupancy_t(int *occ, int *smem) {
    auto k = step_kernel<NT, MK, PL, WALLS, RHO0>;
    *smem = smem_bytes<NT, MK, PL, WALLS, RHO0>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, NT, *smem);
}

template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
cudaError_t batch_launch_t(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps,
                           int grid, cudaStream_t stream) {
    auto k = batch_kernel<NT, MK, PL, WALLS, RHO0>;
    const int smem = smem_bytes<NT, MK, PL, WALLS, RHO0>();
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    k<<<grid, NT, smem, stream>>>(items, nitems, args, maps);
    return cudaGetLastError();
}

template <int NT, int MK, bool PL, bool WALLS, bool RHO0>
cudaError_t batch_occupancy_t(int *occ, int *smem) {
    auto k = batch_kernel<NT, MK, PL, WALLS, RHO0>;
    *smem = smem_bytes<NT, MK, PL, WALLS, RHO0>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, NT, *smem);
}

constexpr int kMarchNT = 128;

// Instantiate FN for the grid kind, fluid model and wall variant at run time.
#define MDF_MARCH_DISPATCH(RHO0, FN, ...)                                              \
    switch (metric * 4 + (power_law ? 2 : 0) + (walls ? 1 : 0)) {                     \
        case 0: return FN<kMarchNT, METRIC_UNIFORM, false, false, RHO0>(__VA_ARGS__);     \
        case 1: return FN<kMarchNT, METRIC_UNIFORM, false, true, RHO0>(__VA_ARGS__);      \
        case 2: return FN<kMarchNT, METRIC_UNIFORM, true, false, RHO0>(__VA_ARGS__);      \
        case 3: return FN<kMarchNT, METRIC_UNIFORM, true, true, RHO0>(__VA_ARGS__);       \
        case 4: return FN<kMarchNT, METRIC_SEPARABLE, false, false, RHO0>(__VA_ARGS__);   \
        case 5: return FN<kMarchNT, METRIC_SEPARABLE, false, true, RHO0>(__VA_ARGS__);    \
        case 6: return FN<kMarchNT, METRIC_SEPARABLE, true, false, RHO0>(__VA_ARGS__);    \
        case 7: return FN<kMarchNT, METRIC_SEPARABLE, true, true, RHO0>(__VA_ARGS__);     \
        case 8: return FN<kMarchNT, METRIC_CURVILINEAR, false, false, RHO0>(__VA_ARGS__); \
        case 9: return FN<kMarchNT, METRIC_CURVILINEAR, false, true, RHO0>(__VA_ARGS__);  \
        case 10: return FN<kMarchNT, METRIC_CURVILINEAR, true, false, RHO0>(__VA_ARGS__); \
        default: return FN<kMarchNT, METRIC_CURVILINEAR, true, true, RHO0>(__VA_ARGS__);  \
    }

// Curvilinear grids only (the batched march; other grids batch in mdf_step_walls.cu).
#define MDF_CURVI_DISPATCH(FN, ...)                                                    \
    switch ((power_law ? 2 : 0) + (walls ? 1 : 0)) {                                   \
        case 0: return FN<kMarchNT, METRIC_CURVILINEAR, false, false, false>(__VA_ARGS__); \
        case 1: return FN<kMarchNT, METRIC_CURVILINEAR, false, true, false>(__VA_ARGS__);  \
        case 2: return FN<kMarchNT, METRIC_CURVILINEAR, true, false, false>(__VA_ARGS__);  \
        default: return FN<kMarchNT, METRIC_CURVILINEAR, true, true, false>(__VA_ARGS__);  \
    }

}  // namespace

}  // namespace mdf
