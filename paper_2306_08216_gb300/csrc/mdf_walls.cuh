// mdf_walls.cuh -- fused MDF-FDLBM step with non-equilibrium
// extrapolation walls and/or a power-law fluid, on uniform or separable
// grids, in the register-window form of the periodic fast path.
//
// The time step is that of mdf_step.cu (Sec. 2.2 Steps (1)-(4) of
// arXiv:2306.08216 with Eqs. 2.3.24-2.3.25, f32x2 pairs for alpha = u, v)
// with the same row march as mdf_step_fast.cu: populations 2 and 4 keep
// their five-row windows of fbar^+ and f(t+h) in registers, populations 1
// and 3 run their x stencils through double-buffered exchange rows, fhat^+
// waits in a shared ring, and one barrier orders each row.  On top of that:
//  * walls (Secs. 4.3-4.4): wall nodes take the non-equilibrium
//    extrapolation of their wall-normal interior neighbour (the diagonal one
//    at corners) for f(t+h) and for fhat(t+dt), written by the neighbour's
//    thread; next to a wall the second-order upwind point beyond it is
//    replaced by its linear extrapolation (stream2 with the wall flag);
//    rows beyond a y wall are not wrapped (TMA fills them with zeros, and
//    nothing reads them);
//  * power law: the relaxation rates of every node follow from its
//    non-equilibrium first moment in Step 1 and wait two rows in a register
//    window for the recovery of Step 3.
// f(t+h) of a wall node is needed only by the stencils of interior nodes:
// pops 1 and 3 of a wall column go to the exchange row (written by the
// thread of the adjacent interior column), pops 2 and 4 of a wall row to the
// register window of the same column (south: when row 1 is formed; north:
// from row ny-2 through a one-row shared buffer, one iteration later).
//
// This header holds the march and its kernel templates; mdf_step_walls.cu
// instantiates the FP32 kernels and the entry points, mdf_step_walls16.cu
// the batched kernels with 16-bit storage (FP32 u, v, P plus FP16/BF16
// non-equilibrium pairs, as on the periodic fast path).
#pragma once

#include <algorithm>
#include <type_traits>

#include "mdf_device.cuh"

namespace mdf {

namespace {

using namespace dev;

__device__ __forceinline__ F2 pair_of(unsigned long long bits) {
    F2 a;
    a.r = bits;
    return a;
}

struct W3 {
    F2 w1, w0, w2;
};

__device__ __forceinline__ W3 weights(float k, float step, const StepArgs &a) {
    W3 w;
    w.w1 = splat(-step * k * a.a1);
    w.w0 = splat(-step * k * a.a0);
    w.w2 = splat(-step * k * a.am2);
    return w;
}

__device__ __forceinline__ F2 force_h(const StepArgs &a, int row, int X, F2 factor) {
    if (a.force_mode == 0) return splat(0.0f);
    if (a.force_mode == 1) return factor * mk2(a.Fx, a.Fy);
    const long long fi = (long long)row * a.pitch + GHOST + X;
    return factor * field_pair(a, a.Fxp, a.Fyp, fi);
}
__device__ __forceinline__ F2 force_d(const StepArgs &a, int row, int X, F2 factor) {
    if (a.force_mode_d == 0) return splat(0.0f);
    if (a.force_mode_d == 1) return factor * mk2(a.Fxd, a.Fyd);
    const long long fi = (long long)row * a.pitch + GHOST + X;
    return factor * field_pair(a, a.Fxdp, a.Fydp, fi);
}

// One TMA row: 10 FP32 planes, or u, v, P and 4 planes of 16-bit pairs.
template <int ST>
constexpr int walls_row_planes() {
    return ST == STORAGE_FP32 ? NPLANES : DEV_PLANES;
}

template <int NT, int ST = STORAGE_FP32>
constexpr int walls_smem() {
    return TMA_SLOTS * walls_row_planes<ST>() * NT * 4 + RING * 5 * NT * 8 + 4 * (2 * NT * 8) + 2 * NT * 8 +
           TMA_SLOTS * 8;
}

// Store one node in the layout of the storage mode (with the periodic
// images of a periodic x axis when XPER).
template <int ST, bool XPER>
__device__ __forceinline__ void store_node_st(const StepArgs &a, int row, int X, const F2 v[5]) {
    if (ST == STORAGE_FP32) store_node<XPER>(a, row, X, v);
    else store_node_dev<ST, XPER>(a, row, X, v);
}

// One block's march over strip bx, band by.  FORCED: body force, force rate
// or source present (read at run time); otherwise those terms are compiled out.
// ROLL: the march loop is not unrolled and the register windows rotate by
// one row per iteration (rot5); otherwise it is unrolled by five and every
// window slot is a compile-time index.  The two compute the same values; the
// rolled body is a fifth of the size (fewer instruction-cache misses on a
// full GPU), the unrolled one has the shorter row latency (small batches).
// ST: the storage mode of the state (16-bit: fhat is rebuilt from the
// stored u, v, P and non-equilibrium pairs on load, and stored back in that
// form, as on the periodic fast path).
template <int NT, int MK, bool PL, bool FORCED, bool ROLL, int ST>
__device__ __forceinline__ void march_walls(const CUtensorMap *tmap, const StepArgs &a, int bx, int by,
                                            unsigned char *smem, int *abort_flag) {
    constexpr int TROW = walls_row_planes<ST>() * NT * 4;  // one TMA row
    constexpr int PROW = 5 * NT * 8;        // one fhat^+ ring row
    constexpr int XROW = 2 * NT * 8;        // one exchange row: pops 1, 3
    unsigned char *tma = smem;
    unsigned char *ringP = tma + TMA_SLOTS * TROW;
    unsigned char *xB0 = ringP + RING * PROW;  // fbar^+ of pops 1, 3 of row p (two buffers)
    unsigned char *xF0 = xB0 + 2 * XROW;       // f(t+h) of pops 1, 3 of row q (two buffers)
    unsigned char *nrow = xF0 + 2 * XROW;      // f(t+h) of pops 2, 4 of the north wall row
    uint64_t *mbar = reinterpret_cast<uint64_t *>(nrow + 2 * NT * 8);
    int &s_abort = *abort_flag;

    const int t = threadIdx.x;
    const int x0 = bx * a.W;
    const int X = x0 - 4 + t;
    const int y0 = by * a.H;
    const int y1 = min(y0 + a.H, a.ny);
    const int nIt = (y1 - y0) + 9;
    const int rowBase = y0 - 4;
    const float c = a.c, inv2c = a.inv2c;
    const bool xwall = a.xwall, ywall = a.ywall;
    const bool colx_wall = xwall && (X == 0 || X == a.nx - 1);
    const bool colx_out = xwall && (X < 0 || X >= a.nx);
    const bool xadj_p = xwall && X == 1, xadj_m = xwall && X == a.nx - 2;
    const bool col_in = X >= -GHOST && X < a.nx + GHOST;  // has a padded-field entry

    if (t == 0) {
        s_abort = 0;
        for (int i = 0; i < TMA_SLOTS; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto row_of = [&](int p) { return ywall ? p : wrap(p, a.ny); };
    auto load_row = [&](int it, int slot) {
        mbar_expect_tx(&mbar[slot], TROW);
        tma_load_row(tmap, &mbar[slot], tma + slot * TROW, x0, row_of(rowBase + it));
    };
    int issued = min(TMA_SLOTS, nIt);
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
    const bool calc = t >= 2 && t < NT - 2 && !colx_out && !colx_wall;          // forms fbar and f
    const bool outc = t >= 4 && t < NT - 4 && X >= 0 && X < a.nx && !colx_wall;  // forms outputs

    F2 BY[5][2];    // fbar^+ of pops 2, 4
    F2 D013[5][3];  // fbar of pops 0, 1, 3 (x part done)
    F2 FY[5][2];    // f(t+h) of pops 2, 4
    F2 XF[5][2];    // pass-2 x increments of pops 1, 3
    float RK[5][2]; // power law: recovery rates (rkp, rk) of the row
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        BY[s][0] = BY[s][1] = FY[s][0] = FY[s][1] = XF[s][0] = XF[s][1] = zero;
        D013[s][0] = D013[s][1] = D013[s][2] = zero;
        RK[s][0] = RK[s][1] = 0.0f;
    }

    int tslot = 0;
    bool aborted = false;
    // One row iteration: window slot K of row p (and of row p - 5 before its
    // write), slots s1..s4 of rows p-1..p-4, row ps of the fhat^+ ring.
    // Returns false when the block aborts.
    auto row = [&](const int it, auto kc, const int ps) -> bool {
        constexpr int k = decltype(kc)::value;
        constexpr int s1 = (k + 4) % 5, s2 = (k + 3) % 5, s3 = (k + 2) % 5, s4 = (k + 1) % 5;
        {
            const int p = rowBase + it;
            unsigned char *xB = xB0 + (it & 1) * XROW;
            const unsigned char *xFp = xF0 + ((it & 1) ^ 1) * XROW;
            unsigned char *xF = xF0 + (it & 1) * XROW;
            // ---------------------------------------------- S0: output row r = p - 5
            if (it >= 9 && outc) {
                const int r = p - 5;  // in [y0, y1): a row of the domain
                if (!(ywall && (r == 0 || r == a.ny - 1))) {
                    const unsigned char *Pr = ringP + ps * PROW;
                    F2 out[5];
#pragma unroll
                    for (int j = 0; j < 5; ++j) out[j] = lds2(Pr, (j * NT + t) * 8);
                    if (FORCED) {
                        const F2 fF = force_d(a, r, X, pair_of(a.pdw));
#pragma unroll
                        for (int j = 0; j < 5; ++j) out[j] = out[j] + fF;
                    }
                    out[1] = out[1] + XF[k][0];
                    out[3] = out[3] + XF[k][1];
                    W3 wy;
                    if (MK == METRIC_UNIFORM) wy = {pair_of(a.pwyd[0]), pair_of(a.pwyd[1]), pair_of(a.pwyd[2])};
                    else wy = weights(a.kyv[r], a.dt, a);
                    const bool yadj_p = ywall && r == 1, yadj_m = ywall && r == a.ny - 2;
                    out[2] = stream2<true>(out[2], FY[s4][0], FY[k][0], FY[s1][0], FY[s2][0], yadj_p, wy.w1, wy.w0,
                                           wy.w2);
                    out[4] = stream2<true>(out[4], FY[s1][1], FY[k][1], FY[s4][1], FY[s3][1], yadj_m, wy.w1, wy.w0,
                                           wy.w2);
                    if (xwall) store_node_st<ST, false>(a, r, X, out);
                    else store_node_st<ST, true>(a, r, X, out);
                    F2 w[5];
                    if (xadj_p) { nee2(out, a.uw[0], a.vw[0], inv2c, w); store_node_st<ST, false>(a, r, 0, w); }
                    if (xadj_m) { nee2(out, a.uw[1], a.vw[1], inv2c, w); store_node_st<ST, false>(a, r, a.nx - 1, w); }
                    if (yadj_p || yadj_m) {
                        const int rr = yadj_p ? 0 : a.ny - 1;
                        const int side = yadj_p ? 2 : 3;
                        nee2(out, a.uw[side], a.vw[side], inv2c, w);
                        if (xwall) store_node_st<ST, false>(a, rr, X, w);
                        else store_node_st<ST, true>(a, rr, X, w);
                        if (xadj_p) { nee2(out, a.uw[0], a.vw[0], inv2c, w); store_node_st<ST, false>(a, rr, 0, w); }
                        if (xadj_m) { nee2(out, a.uw[1], a.vw[1], inv2c, w); store_node_st<ST, false>(a, rr, a.nx - 1, w); }
                    }
                }
            }
            // ---------------------------------------------- S2: row p
            const bool p_in = !ywall || (p >= 0 && p < a.ny);
            F2 own1, own3;
            {
                const bool ok = mbar_wait_bounded(&mbar[tslot], (uint32_t)((it / TMA_SLOTS) & 1));
                if (!ok) atomicExch(&s_abort, 1);
                const float *src = reinterpret_cast<const float *>(tma + tslot * TROW);
                F2 g[5], n[5], o[5];
                if (ST == STORAGE_FP32) {
#pragma unroll
                    for (int j = 0; j < 5; ++j) g[j] = mk2(src[j * NT + t], src[(5 + j) * NT + t]);
                    const Mom2 m = (FORCED && a.r_mode && p_in && col_in)
                                       ? moments2r(g, c, a.rk_hat * source_at(a, row_of(p), X))
                                       : moments2(g, c);
                    noneq2(g, m, inv2c, n);
                } else {
                    // fhat = feq(u, v, P) + n from the stored fields (16-bit
                    // modes carry no source term)
                    const unsigned *w = reinterpret_cast<const unsigned *>(src + DEV_FPLANES * NT);
                    const F2 inv = splat(a.ninv);
                    F2 nn[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) nn[j] = unpack16<ST>(w[j * NT + t]) * inv;
                    dev_build(src[t], src[NT + t], src[2 * NT + t], nn, inv2c, g, n);
                }
                const F2 n13 = n[1] - n[3], n24 = n[2] - n[4];
                F2 mKp = pair_of(a.pmKp), Dp = pair_of(a.pDp), mKb = pair_of(a.pmKb), Db = pair_of(a.pDb);
                if (PL) {
                    float gx1, gx2, gy1, gy2;
                    split2(splat(c) * n13, gx1, gx2);
                    split2(splat(c) * n24, gy1, gy2);
                    const float sxy = 0.5f * (gy1 + gx2);
                    const float gg = sqrtf(2.0f * (gx1 * gx1 + gy2 * gy2 + 2.0f * sxy * sxy));
                    const Rates Rr = rates_nu(power_law_nu(gg, a), a.s_ratio, a.a_pl);
                    mKp = splat(-(1.0f - Rr.rpp));
                    Dp = splat(0.5f * (Rr.rp - Rr.rpp));
                    mKb = splat(-(1.0f - Rr.rbp));
                    Db = splat(0.5f * (Rr.rb - Rr.rbp));
                    RK[k][0] = Rr.rkp;
                    RK[k][1] = Rr.rk;
                }
                relax2(g, n, n13, n24, mKp, Dp, o);
                unsigned char *dP = ringP + ps * PROW;
#pragma unroll
                for (int j = 0; j < 5; ++j) sts2(dP, (j * NT + t) * 8, o[j]);
                relax2(g, n, n13, n24, mKb, Db, o);
                sts2(xB, t * 8, o[1]);
                sts2(xB, (NT + t) * 8, o[3]);
                own1 = o[1];
                own3 = o[3];
                BY[k][0] = o[2];
                BY[k][1] = o[4];
                D013[k][0] = o[0];
            }
            // one barrier per row (exchange rows double-buffered by row parity)
            if (__syncthreads_or(s_abort)) return false;
            if (t == 0 && issued < nIt) {
                fence_proxy_async();
                load_row(issued, tslot);
                ++issued;
            }
            tslot = (tslot == TMA_SLOTS - 1) ? 0 : tslot + 1;
            // ---------------------------------------------- S1: pass-2 x increments of row p-3
            if (it >= 5 && outc) {
                const F2 f1p1 = lds2(xFp, (t + 1) * 8), f1 = lds2(xFp, t * 8);
                const F2 f1m1 = lds2(xFp, (t - 1) * 8), f1m2 = lds2(xFp, (t - 2) * 8);
                const F2 f3m1 = lds2(xFp, (NT + t - 1) * 8), f3 = lds2(xFp, (NT + t) * 8);
                const F2 f3p1 = lds2(xFp, (NT + t + 1) * 8), f3p2 = lds2(xFp, (NT + t + 2) * 8);
                XF[s3][0] = stream2<true>(zero, f1p1, f1, f1m1, f1m2, xadj_p, wxd.w1, wxd.w0, wxd.w2);
                XF[s3][1] = stream2<true>(zero, f3m1, f3, f3p1, f3p2, xadj_m, wxd.w1, wxd.w0, wxd.w2);
            }
            // ---------------------------------------------- S3
            if (calc) {
                // pass 1, x part of row p
                F2 hF = zero;
                if (FORCED && p_in) hF = force_h(a, row_of(p), X, pair_of(a.phw));
                D013[k][0] = D013[k][0] + hF;
                D013[k][1] = stream2<true>(own1 + hF, lds2(xB, (t + 1) * 8), own1, lds2(xB, (t - 1) * 8),
                                           lds2(xB, (t - 2) * 8), xadj_p, wxh.w1, wxh.w0, wxh.w2);
                D013[k][2] = stream2<true>(own3 + hF, lds2(xB, (NT + t - 1) * 8), own3, lds2(xB, (NT + t + 1) * 8),
                                           lds2(xB, (NT + t + 2) * 8), xadj_m, wxh.w1, wxh.w0, wxh.w2);
                const int q = p - 2;
                if (it >= 4 && (!ywall || (q >= 0 && q < a.ny))) {
                    if (ywall && q == a.ny - 1) {
                        // north wall row: pops 2, 4 of its NEE value were formed with row ny-2
                        FY[s2][0] = lds2(nrow, t * 8);
                        FY[s2][1] = lds2(nrow, (NT + t) * 8);
                    } else if (!(ywall && q == 0)) {
                        const int qw = row_of(q);
                        F2 hFq = zero;
                        if (FORCED) hFq = force_h(a, qw, X, pair_of(a.phw));
                        W3 wy;
                        if (MK == METRIC_UNIFORM) wy = {pair_of(a.pwyh[0]), pair_of(a.pwyh[1]), pair_of(a.pwyh[2])};
                        else wy = weights(a.kyv[qw], a.h, a);
                        const bool yadj_p = ywall && q == 1, yadj_m = ywall && q == a.ny - 2;
                        F2 fb[5];
                        fb[0] = D013[s2][0];
                        fb[1] = D013[s2][1];
                        fb[3] = D013[s2][2];
                        fb[2] = stream2<true>(BY[s2][0] + hFq, BY[s1][0], BY[s2][0], BY[s3][0], BY[s4][0], yadj_p,
                                              wy.w1, wy.w0, wy.w2);
                        fb[4] = stream2<true>(BY[s2][1] + hFq, BY[s3][1], BY[s2][1], BY[s1][1], BY[k][1], yadj_m,
                                              wy.w1, wy.w0, wy.w2);
                        // Step 3: f = feq + (I + h/2 Lt)^-1 (fbar - feq)
                        F2 mKk = pair_of(a.pmKk), Dk = pair_of(a.pDk);
                        if (PL) {
                            mKk = splat(-(1.0f - RK[s2][0]));
                            Dk = splat(0.5f * (RK[s2][1] - RK[s2][0]));
                        }
                        const Mom2 m = (FORCED && a.r_mode) ? moments2r(fb, c, a.rk_bar * source_at(a, qw, X))
                                                            : moments2(fb, c);
                        F2 n[5], f[5];
                        noneq2(fb, m, inv2c, n);
                        relax2(fb, n, n[1] - n[3], n[2] - n[4], mKk, Dk, f);
                        sts2(xF, t * 8, f[1]);
                        sts2(xF, (NT + t) * 8, f[3]);
                        FY[s2][0] = f[2];
                        FY[s2][1] = f[4];
                        F2 w[5];
                        if (xadj_p) {  // west wall column of this row: pops 1, 3 for the x stencils
                            nee2(f, a.uw[0], a.vw[0], inv2c, w);
                            sts2(xF, (t - 1) * 8, w[1]);
                            sts2(xF, (NT + t - 1) * 8, w[3]);
                        }
                        if (xadj_m) {
                            nee2(f, a.uw[1], a.vw[1], inv2c, w);
                            sts2(xF, (t + 1) * 8, w[1]);
                            sts2(xF, (NT + t + 1) * 8, w[3]);
                        }
                        if (yadj_p) {  // south wall row (slot of row q - 1): pops 2, 4 for the y stencils
                            nee2(f, a.uw[2], a.vw[2], inv2c, w);
                            FY[s3][0] = w[2];
                            FY[s3][1] = w[4];
                        }
                        if (yadj_m) {  // north wall row, taken up next iteration
                            nee2(f, a.uw[3], a.vw[3], inv2c, w);
                            sts2(nrow, t * 8, w[2]);
                            sts2(nrow, (NT + t) * 8, w[4]);
                        }
                    }
                }
            }
        }
        return true;
    };
    using std::integral_constant;
    if (ROLL) {
        int pslot = 0;  // it mod 5
#pragma unroll 1
        for (int it = 0; it < nIt; ++it) {
            if (!row(it, integral_constant<int, 0>{}, pslot)) {
                aborted = true;
                break;
            }
            rot5(BY);
            rot5(D013);
            rot5(FY);
            rot5(XF);
            rot5(RK);
            pslot = pslot == 4 ? 0 : pslot + 1;
        }
    } else {
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
    }
    (void)aborted;
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

// Resident blocks the register budget is sized for: 4 x 96 or 3 x 128
// threads (up to 170 registers: the wall and power-law logic does not fit
// 128 without spilling), 2 x 256.
template <int NT>
constexpr int walls_min_blocks() {
    return NT <= 96 ? 4 : (NT <= 128 ? 3 : 2);
}

template <int NT, int MK, bool PL, bool FORCED>
__global__ void __launch_bounds__(NT, walls_min_blocks<NT>())
    walls_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    march_walls<NT, MK, PL, FORCED, false, STORAGE_FP32>(&tmap, a, blockIdx.x, blockIdx.y, smem, &s_abort);
}

// Persistent batch form: block b takes work items b, b + gridDim.x, ...
// FORCED if any problem of the batch has a force, force rate or source;
// ROLL selects the rolled march, ST the storage mode (see march_walls).
template <int NT, int MK, bool PL, bool FORCED, bool ROLL, int ST>
__global__ void __launch_bounds__(NT, walls_min_blocks<NT>())
    walls_batch_kernel(const BatchItem *__restrict__ items, int nitems, const StepArgs *__restrict__ args,
                       const CUtensorMap *__restrict__ maps) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const BatchItem item = items[w];
        march_walls<NT, MK, PL, FORCED, ROLL, ST>(&maps[item.problem], args[item.problem], item.bx, item.by, smem,
                                                  &s_abort);
        if (s_abort) break;
    }
}

template <int NT, int MK, bool PL, bool FORCED>
cudaError_t launch_t(const CUtensorMap *tmap, const StepArgs &args, const StepPlan &plan, cudaStream_t stream) {
    auto k = walls_kernel<NT, MK, PL, FORCED>;
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, walls_smem<NT>());
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    k<<<dim3(plan.gx, plan.gy), NT, walls_smem<NT>(), stream>>>(*tmap, args);
    return cudaGetLastError();
}

template <int NT, int MK, bool PL>
cudaError_t occupancy_t(int *occ, int *smem) {
    int o1 = 0, o2 = 0;
    *smem = walls_smem<NT>();
    cudaError_t e = cudaFuncSetAttribute(walls_kernel<NT, MK, PL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         *smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(walls_kernel<NT, MK, PL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, walls_kernel<NT, MK, PL, false>, NT, *smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, walls_kernel<NT, MK, PL, true>, NT, *smem);
    *occ = o1 < o2 ? o1 : o2;
    return e;
}

template <int NT, int MK, bool PL, bool FORCED, bool ROLL, int ST>
cudaError_t batch_launch_ft(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps,
                            int grid, cudaStream_t stream) {
    auto k = walls_batch_kernel<NT, MK, PL, FORCED, ROLL, ST>;
    constexpr int smem = walls_smem<NT, ST>();
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    k<<<grid, NT, smem, stream>>>(items, nitems, args, maps);
    return cudaGetLastError();
}

// The batch kernels of one storage mode: both march forms with FP32
// storage, the rolled form only with 16-bit storage (the form a full GPU
// keeps; small 16-bit batches have the tile kernel beside it).
template <int ST>
constexpr bool walls_unrolled_batch() {
    return ST == STORAGE_FP32;
}

template <int NT, int MK, bool PL, int ST>
cudaError_t batch_launch_t(const BatchItem *items, int nitems, const StepArgs *args, const CUtensorMap *maps, int grid,
                           int forced, int roll, cudaStream_t stream) {
    if constexpr (walls_unrolled_batch<ST>()) {
        if (!roll) {
            if (forced) return batch_launch_ft<NT, MK, PL, true, false, ST>(items, nitems, args, maps, grid, stream);
            return batch_launch_ft<NT, MK, PL, false, false, ST>(items, nitems, args, maps, grid, stream);
        }
    } else {
        if (!roll) return cudaErrorInvalidConfiguration;
    }
    if (forced) return batch_launch_ft<NT, MK, PL, true, true, ST>(items, nitems, args, maps, grid, stream);
    return batch_launch_ft<NT, MK, PL, false, true, ST>(items, nitems, args, maps, grid, stream);
}

// Occupancy of one batch kernel variant.
template <int NT, int MK, bool PL, bool FORCED, bool ROLL, int ST>
cudaError_t batch_occupancy_v(int smem, int *occ) {
    auto k = walls_batch_kernel<NT, MK, PL, FORCED, ROLL, ST>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, NT, smem);
    return e;
}

template <int NT, int MK, bool PL, int ST>
cudaError_t batch_occupancy_t(int *occ, int *smem) {
    // every variant of a storage mode has the same shared memory; take the
    // smallest occupancy
    int o[4] = {1 << 30, 1 << 30, 1 << 30, 1 << 30};
    *smem = walls_smem<NT, ST>();
    cudaError_t e = batch_occupancy_v<NT, MK, PL, false, true, ST>(*smem, &o[0]);
    if (e == cudaSuccess) e = batch_occupancy_v<NT, MK, PL, true, true, ST>(*smem, &o[1]);
    if constexpr (walls_unrolled_batch<ST>()) {
        if (e == cudaSuccess) e = batch_occupancy_v<NT, MK, PL, false, false, ST>(*smem, &o[2]);
        if (e == cudaSuccess) e = batch_occupancy_v<NT, MK, PL, true, false, ST>(*smem, &o[3]);
    }
    *occ = std::min(std::min(o[0], o[1]), std::min(o[2], o[3]));
    return e;
}

#define MDF_WALLS_DISPATCH(NTV, FN, ...)                                             \
    switch ((metric == METRIC_SEPARABLE ? 2 : 0) + (power_law ? 1 : 0)) {            \
        case 0: return FN<NTV, METRIC_UNIFORM, false>(__VA_ARGS__);                   \
        case 1: return FN<NTV, METRIC_UNIFORM, true>(__VA_ARGS__);                    \
        case 2: return FN<NTV, METRIC_SEPARABLE, false>(__VA_ARGS__);                 \
        default: return FN<NTV, METRIC_SEPARABLE, true>(__VA_ARGS__);                 \
    }

#define MDF_WALLS_DISPATCH_ST(NTV, STV, FN, ...)                                     \
    switch ((metric == METRIC_SEPARABLE ? 2 : 0) + (power_law ? 1 : 0)) {            \
        case 0: return FN<NTV, METRIC_UNIFORM, false, STV>(__VA_ARGS__);              \
        case 1: return FN<NTV, METRIC_UNIFORM, true, STV>(__VA_ARGS__);               \
        case 2: return FN<NTV, METRIC_SEPARABLE, false, STV>(__VA_ARGS__);            \
        default: return FN<NTV, METRIC_SEPARABLE, true, STV>(__VA_ARGS__);            \
    }

template <int NT, int MK, bool PL>
cudaError_t launch_f(const CUtensorMap *tmap, const StepArgs &args, const StepPlan &plan, cudaStream_t stream) {
    if (args.force_mode || args.force_mode_d || args.r_mode) return launch_t<NT, MK, PL, true>(tmap, args, plan, stream);
    return launch_t<NT, MK, PL, false>(tmap, args, plan, stream);
}

template <int NT>
cudaError_t launch_nt(const CUtensorMap *tmap, const StepArgs &args, int metric, const StepPlan &plan,
                      cudaStream_t stream) {
    const int power_law = args.power_law;
    MDF_WALLS_DISPATCH(NT, launch_f, tmap, args, plan, stream)
}

}  // namespace

// Batches use 96-thread blocks (strips of 88 columns): the 2^k + 1 node
// sides of a cavity sweep waste fewer thread columns than with 120-column
// strips (513 nodes: 6 x 96 = 576 threads against 5 x 128 = 640).
constexpr int kWallsBatchNT = 96;

}  // namespace mdf
