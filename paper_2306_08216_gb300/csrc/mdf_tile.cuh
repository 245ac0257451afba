// mdf_tile.cuh -- the fused MDF-FDLBM step on grids too small to keep the
// GPU busy with marching bands (kernels of mdf_step_tile.cu, FP32 storage,
// and mdf_step_tile16.cu, the 16-bit deviation storage modes).
//
// Same time step as the marches (Sec. 2.2 Steps (1)-(4) of arXiv:2306.08216
// with Eqs. 2.3.24-2.3.25, f32x2 pairs for alpha = u, v, every grid kind,
// walls by non-equilibrium extrapolation, power law), organised per 2-D
// tile instead of per band: a block of TX x TY threads owns a TX x TY tile
// of output nodes and performs the step in three phases separated by
// barriers:
//   A  fhat(t) of the tile plus a halo of 4 (read from L2/HBM with plain
//      loads) -> fbar^+ of every node of that region into shared memory;
//      fhat^+ of the thread's own node stays in registers (and, for a power
//      law, the recovery rates of the nodes of the inner region go to shared
//      memory);
//   B  fbar (pass 1, Eq. 2.3.25) and f(t+h) (Eq. 2.2.16) on the tile plus a
//      halo of 2 -> shared memory; then the wall nodes of that region by NEE
//      from their interior neighbour;
//   C  fhat(t+dt) (pass 2, Eq. 2.3.24) of the thread's own node -> HBM, and
//      the NEE value of an adjacent wall node.
// The halo is recomputed (a 16 x 16 tile computes fbar^+ on 24 x 24 nodes
// and f on 20 x 20), which the marches avoid; in exchange a step is three
// short phases per block instead of a march of H + 9 rows, and a 257^2 grid
// is 289 blocks of 8 warps instead of a few hundred 4-warp marches, so
// small grids are no longer bound by the length of a serial march.
#pragma once

#include "mdf_device.cuh"

namespace mdf {

namespace {

using namespace dev;

// Three 256-thread blocks per SM (at most 85 registers; a few variants spill
// 20-24 bytes): on the 513^2 trapezoid cavities 18 % faster than two.
constexpr int kTileMinBlocks = 3;

__device__ __forceinline__ F2 pair_of_bits(unsigned long long bits) {
    F2 p;
    p.r = bits;
    return p;
}

// Index of node i on an axis of n nodes: unchanged on a walled axis, else
// the periodic image.  Region nodes lie within a few tiles of the domain, so
// the integer modulo is needed only on grids smaller than the region.
__device__ __forceinline__ int axis_index(int i, int n, bool wall) {
    if (wall || (i >= 0 && i < n)) return i;
    if (i < 0 && i >= -n) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    return wrap(i, n);
}

template <int TX, int TY>
struct Tile {
    static constexpr int NT = TX * TY;
    static constexpr int X8 = TX + 8, Y8 = TY + 8, N8 = X8 * Y8;  // fbar^+ region: tile + 4
    static constexpr int X4 = TX + 4, Y4 = TY + 4, N4 = X4 * Y4;  // f region: tile + 2
    static constexpr int B_BYTES = 5 * N8 * 8;
    static constexpr int F_BYTES = 5 * N4 * 8;
    static constexpr int K_BYTES = 2 * N4 * 4;
    static constexpr int B0_BYTES = 5 * N8 * 4;  // the alpha = 0 lane: fbar^+ and f as floats
    static constexpr int F0_BYTES = 5 * N4 * 4;
};

// Difference weights of one axis (as the marches): w = -step k (a1, a0, am2).
struct TW {
    F2 w1, w0, w2;
};
__device__ __forceinline__ TW tweights(float k, float step, const StepArgs &a) {
    return TW{splat(-step * k * a.a1), splat(-step * k * a.a0), splat(-step * k * a.am2)};
}

// Streaming increment of population j at a curvilinear node n of the pair
// array A (row stride S), upwinded by the sign of each contravariant speed.
template <int NN>
__device__ __forceinline__ F2 curvi_tile(const unsigned char *A, int j, int n, int S, float cxi, float ceta,
                                         bool xadj_p, bool xadj_m, bool yadj_p, bool yadj_m, float step,
                                         const StepArgs &a, F2 acc) {
    auto at = [&](int m) { return lds2(A, (j * NN + m) * 8); };
    const F2 p0 = at(n);
    if (cxi != 0.0f) {
        const float k = -step * fabsf(cxi);
        const F2 w1 = splat(k * a.a1), w0 = splat(k * a.a0), w2 = splat(k * a.am2);
        if (cxi > 0.0f) acc = stream2<true>(acc, at(n + 1), p0, at(n - 1), at(n - 2), xadj_p, w1, w0, w2);
        else acc = stream2<true>(acc, at(n - 1), p0, at(n + 1), at(n + 2), xadj_m, w1, w0, w2);
    }
    if (ceta != 0.0f) {
        const float k = -step * fabsf(ceta);
        const F2 w1 = splat(k * a.a1), w0 = splat(k * a.a0), w2 = splat(k * a.am2);
        if (ceta > 0.0f) acc = stream2<true>(acc, at(n + S), p0, at(n - S), at(n - 2 * S), yadj_p, w1, w0, w2);
        else acc = stream2<true>(acc, at(n - S), p0, at(n + S), at(n + 2 * S), yadj_m, w1, w0, w2);
    }
    return acc;
}

// Streaming increments of populations 1..4 at node n of the pair array A
// (NN nodes per population, row stride S), added to out[1..4].  The grid
// coordinates (Xw, Yw) locate the metric coefficients.
template <int NN, int MK, bool WALLS>
__device__ __forceinline__ void stream_tile(const unsigned char *A, int n, int S, float step, int Xw, int Yw,
                                            bool xadj_p, bool xadj_m, bool yadj_p, bool yadj_m, const StepArgs &a,
                                            F2 out[5]) {
    auto at = [&](int j, int m) { return lds2(A, (j * NN + m) * 8); };
    if (MK != METRIC_CURVILINEAR) {
        TW wx, wy;
        if (MK == METRIC_UNIFORM) {
            wx = tweights(a.kx, step, a);
            wy = tweights(a.ky, step, a);
        } else {
            wx = tweights(a.kxv[GHOST + Xw], step, a);
            wy = tweights(a.kyv[Yw], step, a);
        }
        out[1] = stream2<WALLS>(out[1], at(1, n + 1), at(1, n), at(1, n - 1), at(1, n - 2), xadj_p, wx.w1, wx.w0,
                                wx.w2);
        out[3] = stream2<WALLS>(out[3], at(3, n - 1), at(3, n), at(3, n + 1), at(3, n + 2), xadj_m, wx.w1, wx.w0,
                                wx.w2);
        out[2] = stream2<WALLS>(out[2], at(2, n + S), at(2, n), at(2, n - S), at(2, n - 2 * S), yadj_p, wy.w1, wy.w0,
                                wy.w2);
        out[4] = stream2<WALLS>(out[4], at(4, n - S), at(4, n), at(4, n + S), at(4, n + 2 * S), yadj_m, wy.w1, wy.w0,
                                wy.w2);
    } else {
        const long long mi = (long long)Yw * a.pitch + GHOST + Xw;
        const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
        out[1] = curvi_tile<NN>(A, 1, n, S, cxx, cex, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[1]);
        out[2] = curvi_tile<NN>(A, 2, n, S, cxy, cey, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[2]);
        out[3] = curvi_tile<NN>(A, 3, n, S, -cxx, -cex, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[3]);
        out[4] = curvi_tile<NN>(A, 4, n, S, -cxy, -cey, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[4]);
    }
}

// The same two helpers on the scalar alpha = 0 lane (arrays of floats).
template <int NN>
__device__ __forceinline__ float curvi_tile0(const float *A, int j, int n, int S, float cxi, float ceta, bool xadj_p,
                                             bool xadj_m, bool yadj_p, bool yadj_m, float step, const StepArgs &a,
                                             float acc) {
    auto at = [&](int m) { return A[j * NN + m]; };
    const float p0 = at(n);
    if (cxi != 0.0f) {
        const float k = -step * fabsf(cxi);
        const float w1 = k * a.a1, w0 = k * a.a0, w2 = k * a.am2;
        if (cxi > 0.0f) acc = stream1<true>(acc, at(n + 1), p0, at(n - 1), at(n - 2), xadj_p, w1, w0, w2);
        else acc = stream1<true>(acc, at(n - 1), p0, at(n + 1), at(n + 2), xadj_m, w1, w0, w2);
    }
    if (ceta != 0.0f) {
        const float k = -step * fabsf(ceta);
        const float w1 = k * a.a1, w0 = k * a.a0, w2 = k * a.am2;
        if (ceta > 0.0f) acc = stream1<true>(acc, at(n + S), p0, at(n - S), at(n - 2 * S), yadj_p, w1, w0, w2);
        else acc = stream1<true>(acc, at(n - S), p0, at(n + S), at(n + 2 * S), yadj_m, w1, w0, w2);
    }
    return acc;
}

template <int NN, int MK, bool WALLS>
__device__ __forceinline__ void stream_tile0(const float *A, int n, int S, float step, int Xw, int Yw, bool xadj_p,
                                             bool xadj_m, bool yadj_p, bool yadj_m, const StepArgs &a,
                                             float out[5]) {
    auto at = [&](int j, int m) { return A[j * NN + m]; };
    if (MK != METRIC_CURVILINEAR) {
        float kx = a.kx, ky = a.ky;
        if (MK == METRIC_SEPARABLE) {
            kx = a.kxv[GHOST + Xw];
            ky = a.kyv[Yw];
        }
        const float x1 = -step * kx * a.a1, x0 = -step * kx * a.a0, x2 = -step * kx * a.am2;
        const float y1 = -step * ky * a.a1, y0 = -step * ky * a.a0, y2 = -step * ky * a.am2;
        out[1] = stream1<WALLS>(out[1], at(1, n + 1), at(1, n), at(1, n - 1), at(1, n - 2), xadj_p, x1, x0, x2);
        out[3] = stream1<WALLS>(out[3], at(3, n - 1), at(3, n), at(3, n + 1), at(3, n + 2), xadj_m, x1, x0, x2);
        out[2] = stream1<WALLS>(out[2], at(2, n + S), at(2, n), at(2, n - S), at(2, n - 2 * S), yadj_p, y1, y0, y2);
        out[4] = stream1<WALLS>(out[4], at(4, n - S), at(4, n), at(4, n + S), at(4, n + 2 * S), yadj_m, y1, y0, y2);
    } else {
        const long long mi = (long long)Yw * a.pitch + GHOST + Xw;
        const float cxx = a.mxx[mi], cxy = a.mxy[mi], cex = a.mex[mi], cey = a.mey[mi];
        out[1] = curvi_tile0<NN>(A, 1, n, S, cxx, cex, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[1]);
        out[2] = curvi_tile0<NN>(A, 2, n, S, cxy, cey, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[2]);
        out[3] = curvi_tile0<NN>(A, 3, n, S, -cxx, -cex, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[3]);
        out[4] = curvi_tile0<NN>(A, 4, n, S, -cxy, -cey, xadj_p, xadj_m, yadj_p, yadj_m, step, a, out[4]);
    }
}

template <int TX, int TY, int MK, bool WALLS, int ST, bool RHO0>
__device__ __forceinline__ void tile_output(const StepArgs &a, int X, int Y, int li, int lj, const unsigned char *Fs,
                                            const float *Fs0, const F2 hp[5], const float hp0[5]);

// One tile (bx, by) of one problem.  Every thread reaches every barrier
// (no early exit), so a block may step several tiles in a row: the barrier
// after phase A of the next tile orders its shared-memory writes after the
// reads of the previous tile.
template <int TX, int TY, int MK, bool PL, bool WALLS, int ST, bool RHO0>
__device__ __forceinline__ void tile_step(const StepArgs &a, int bx, int by, unsigned char *smem) {
    using T = Tile<TX, TY>;
    unsigned char *Bs = smem;                          // fbar^+ [5][N8] pairs
    unsigned char *Fs = smem + T::B_BYTES;             // f(t+h) [5][N4] pairs
    float *Ks = reinterpret_cast<float *>(Fs + T::F_BYTES);  // power law: rkp [N4], rk [N4]
    // the alpha = 0 lane (planes 10..14): fbar^+ [5][N8] and f [5][N4] floats
    float *Bs0 = Ks + (PL ? 2 * T::N4 : 0);
    float *Fs0 = Bs0 + (RHO0 ? 5 * T::N8 : 0);

    const int t = threadIdx.x;
    const int x0 = bx * TX, y0 = by * TY;
    const bool xwall = WALLS && a.xwall, ywall = WALLS && a.ywall;
    const float c = a.c, inv2c = a.inv2c;
    const F2 mKp = pair_of_bits(a.pmKp), Dp = pair_of_bits(a.pDp), mKb = pair_of_bits(a.pmKb), Db = pair_of_bits(a.pDb);

    // ------------------------------------------------ A: fbar^+ on tile + 4
    // The thread's nodes of the region: first its own output node, then
    // nodes of the halo ring (4 rows above, 4 below, 4 columns each side).
    // All their loads are issued before any arithmetic, so that the passes
    // share one memory latency.
    constexpr int PASSES = (T::N8 + T::NT - 1) / T::NT;
    auto region_node = [&](int i, int &lx, int &ly) {
        if (i < T::NT) {
            lx = 4 + i % TX;
            ly = 4 + i / TX;
            return;
        }
        int h = i - T::NT;
        if (h < 4 * T::X8) {
            ly = h / T::X8;
            lx = h % T::X8;
        } else if (h < 8 * T::X8) {
            h -= 4 * T::X8;
            ly = TY + 4 + h / T::X8;
            lx = h % T::X8;
        } else {
            h -= 8 * T::X8;
            ly = 4 + h / 8;
            const int cc = h % 8;
            lx = cc < 4 ? cc : TX + cc;
        }
    };
    // the planes of a node: 10 FP32 distributions, or u, v, P and four
    // 16-bit pair words (as 32-bit patterns)
    constexpr int NW = ST == STORAGE_FP32 ? (RHO0 ? RHO0_PLANES : NPLANES) : DEV_PLANES;
    float raw[PASSES][NW];
#pragma unroll
    for (int q = 0; q < PASSES; ++q) {
        const int i = t + q * T::NT;
#pragma unroll
        for (int k = 0; k < NW; ++k) raw[q][k] = 0.0f;
        if (i < T::N8) {
            int lx, ly;
            region_node(i, lx, ly);
            const int X = x0 - 4 + lx, Y = y0 - 4 + ly;
            const bool ok = (xwall ? (X >= 0 && X < a.nx) : true) && (ywall ? (Y >= 0 && Y < a.ny) : true);
            if (ok) {
                const long long s =
                    (long long)axis_index(Y, a.ny, ywall) * a.pitch + GHOST + axis_index(X, a.nx, xwall);
#pragma unroll
                for (int k = 0; k < NW; ++k)
                    if (state_index_ok(a, k * a.plane + s)) raw[q][k] = a.fin[k * a.plane + s];
            }
        }
    }
    F2 hp[5];      // fhat^+ of the thread's own node
    float hp0[5];  // ... and of its alpha = 0 populations
#pragma unroll
    for (int q = 0; q < PASSES; ++q) {
        const int i = t + q * T::NT;
        if (i >= T::N8) break;
        int lx, ly;
        region_node(i, lx, ly);
        const int X = x0 - 4 + lx, Y = y0 - 4 + ly;
        const bool okx = xwall ? (X >= 0 && X < a.nx) : true;
        const bool oky = ywall ? (Y >= 0 && Y < a.ny) : true;
        const int Xw = axis_index(X, a.nx, xwall), Yw = axis_index(Y, a.ny, ywall);
        F2 g[5], n[5];
        float uq = 0.0f, vq = 0.0f;  // velocity of the node (the alpha = 0 lane's equilibrium)
        if (ST == STORAGE_FP32) {
#pragma unroll
            for (int j = 0; j < 5; ++j) g[j] = mk2(raw[q][j], raw[q][5 + j]);
            const Mom2 m =
                (a.r_mode && okx && oky) ? moments2r(g, c, a.rk_hat * source_at(a, Yw, Xw)) : moments2(g, c);
            noneq2(g, m, inv2c, n);
            uq = m.u;
            vq = m.v;
        } else {
            // fhat = feq(u, v, P) + n straight from the stored fields (no source
            // term in the 16-bit modes)
            const F2 inv = splat(a.ninv);
            F2 nn[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) nn[j] = unpack16<ST>(__float_as_uint(raw[q][DEV_FPLANES + j])) * inv;
            dev_build(raw[q][0], raw[q][1], raw[q][2], nn, inv2c, g, n);
        }
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
            rpp = Rr.rpp;
            rp = Rr.rp;
            rbp = Rr.rbp;
            rb = Rr.rb;
            if (lx >= 2 && lx < T::X8 - 2 && ly >= 2 && ly < T::Y8 - 2) {
                const int n4 = (ly - 2) * T::X4 + (lx - 2);
                Ks[n4] = Rr.rkp;
                Ks[T::N4 + n4] = Rr.rk;
            }
        }
        F2 o[5];
        if (q == 0) relax2(g, n, n13, n24, mKp_, Dp_, hp);
        relax2(g, n, n13, n24, mKb_, Db_, o);
        const int n8 = ly * T::X8 + lx;
#pragma unroll
        for (int j = 0; j < 5; ++j) sts2(Bs, (j * T::N8 + n8) * 8, o[j]);
        if (RHO0) {
            // Step 1 on alpha = 0 with the node's u, v and the same rates
            float g0[5], n0[5], o0[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) g0[j] = raw[q][NPLANES + j];
            noneq0(g0, uq, vq, inv2c, n0);
            if (q == 0) relax0(g0, n0, -(1.0f - rpp), 0.5f * (rp - rpp), hp0);
            relax0(g0, n0, -(1.0f - rbp), 0.5f * (rb - rbp), o0);
#pragma unroll
            for (int j = 0; j < 5; ++j) Bs0[j * T::N8 + n8] = o0[j];
        }
    }
    __syncthreads();

    // ------------------------------------------------ B: f(t+h) on tile + 2
    const F2 hw = splat(a.h * 0.2f);
    const F2 mKk = pair_of_bits(a.pmKk), Dk = pair_of_bits(a.pDk);
#pragma unroll 1
    for (int i4 = t; i4 < T::N4; i4 += T::NT) {
        const int lx4 = i4 % T::X4, ly4 = i4 / T::X4;
        const int X = x0 - 2 + lx4, Y = y0 - 2 + ly4;
        if (WALLS) {
            const bool skip = (xwall && (X <= 0 || X >= a.nx - 1)) || (ywall && (Y <= 0 || Y >= a.ny - 1));
            if (skip) {  // beyond or on a wall: NEE below (the values beyond are never read)
#pragma unroll
                for (int j = 0; j < 5; ++j) sts2(Fs, (j * T::N4 + i4) * 8, splat(0.0f));
                if (RHO0)
#pragma unroll
                    for (int j = 0; j < 5; ++j) Fs0[j * T::N4 + i4] = 0.0f;
                continue;
            }
        }
        const int Xw = axis_index(X, a.nx, xwall), Yw = axis_index(Y, a.ny, ywall);
        const bool xadj_p = xwall && X == 1, xadj_m = xwall && X == a.nx - 2;
        const bool yadj_p = ywall && Y == 1, yadj_m = ywall && Y == a.ny - 2;
        const int n8 = (ly4 + 2) * T::X8 + lx4 + 2;
        F2 fF = splat(0.0f);
        if (a.force_mode == 1) fF = hw * mk2(a.Fx, a.Fy);
        else if (a.force_mode == 2) {
            const long long fi = (long long)Yw * a.pitch + GHOST + Xw;
            fF = hw * field_pair(a, a.Fxp, a.Fyp, fi);
        }
        // Step 2 (pass 1): fbar = fbar^+ - h c.grad fbar^+ + h w F
        F2 fb[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) fb[j] = lds2(Bs, (j * T::N8 + n8) * 8) + fF;
        stream_tile<T::N8, MK, WALLS>(Bs, n8, T::X8, a.h, Xw, Yw, xadj_p, xadj_m, yadj_p, yadj_m, a, fb);
        // Step 3: f = feq + (I + h/2 Lt)^-1 (fbar - feq)
        F2 mKk_ = mKk, Dk_ = Dk;
        if (PL) {
            const float kp = Ks[i4], kk = Ks[T::N4 + i4];
            mKk_ = splat(-(1.0f - kp));
            Dk_ = splat(0.5f * (kk - kp));
        }
        const Mom2 m = a.r_mode ? moments2r(fb, c, a.rk_bar * source_at(a, Yw, Xw)) : moments2(fb, c);
        F2 n[5], f[5];
        noneq2(fb, m, inv2c, n);
        relax2(fb, n, n[1] - n[3], n[2] - n[4], mKk_, Dk_, f);
#pragma unroll
        for (int j = 0; j < 5; ++j) sts2(Fs, (j * T::N4 + i4) * 8, f[j]);
        if (RHO0) {
            // Steps 2-3 on alpha = 0: source h w_j R, recovery with the u, v of
            // the alpha = 1, 2 fbar and the same rates
            const float sR = a.r_mode ? a.h * 0.2f * source_at(a, Yw, Xw) : 0.0f;
            float fb0[5], n0[5], f0[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) fb0[j] = Bs0[j * T::N8 + n8] + sR;
            stream_tile0<T::N8, MK, WALLS>(Bs0, n8, T::X8, a.h, Xw, Yw, xadj_p, xadj_m, yadj_p, yadj_m, a, fb0);
            float kp = a.rkp, kk = a.rk;
            if (PL) {
                kp = Ks[i4];
                kk = Ks[T::N4 + i4];
            }
            noneq0(fb0, m.u, m.v, inv2c, n0);
            relax0(fb0, n0, -(1.0f - kp), 0.5f * (kk - kp), f0);
#pragma unroll
            for (int j = 0; j < 5; ++j) Fs0[j * T::N4 + i4] = f0[j];
        }
    }
    __syncthreads();
    if (WALLS) {
        // wall nodes of the f region from their interior neighbour (corners:
        // the diagonal neighbour and the west/east wall velocity)
#pragma unroll 1
        for (int i4 = t; i4 < T::N4; i4 += T::NT) {
            const int lx4 = i4 % T::X4, ly4 = i4 / T::X4;
            const int X = x0 - 2 + lx4, Y = y0 - 2 + ly4;
            const bool inx = X >= 0 && X < a.nx, iny = Y >= 0 && Y < a.ny;
            const bool wx = xwall && (X == 0 || X == a.nx - 1) && iny;
            const bool wy = ywall && (Y == 0 || Y == a.ny - 1) && inx;
            if (!(wx || wy)) continue;
            const int dx = xwall ? (X == 0 ? 1 : (X == a.nx - 1 ? -1 : 0)) : 0;
            const int dy = ywall ? (Y == 0 ? 1 : (Y == a.ny - 1 ? -1 : 0)) : 0;
            const int side = (xwall && dx != 0) ? (X == 0 ? 0 : 1) : (Y == 0 ? 2 : 3);
            const int nb = i4 + dy * T::X4 + dx;
            F2 g[5], w[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) g[j] = lds2(Fs, (j * T::N4 + nb) * 8);
            nee2(g, a.uw[side], a.vw[side], inv2c, w);
#pragma unroll
            for (int j = 0; j < 5; ++j) sts2(Fs, (j * T::N4 + i4) * 8, w[j]);
            if (RHO0) {  // the wall's rho_0 is the neighbour's
                float un, vn, g0[5], w0[5];
                split2((g[0] + g[1]) + (g[2] + g[3]) + g[4], un, vn);
#pragma unroll
                for (int j = 0; j < 5; ++j) g0[j] = Fs0[j * T::N4 + nb];
                nee0(g0, a.uw[side], a.vw[side], un, vn, inv2c, w0);
#pragma unroll
                for (int j = 0; j < 5; ++j) Fs0[j * T::N4 + i4] = w0[j];
            }
        }
        __syncthreads();
    }

    // ------------------------------------------------ C: fhat(t+dt) of the own node
    const int li = t % TX, lj = t / TX;
    const int X = x0 + li, Y = y0 + lj;
    if (X >= a.nx || Y >= a.ny) return;
    if (WALLS && ((xwall && (X == 0 || X == a.nx - 1)) || (ywall && (Y == 0 || Y == a.ny - 1)))) return;
    tile_output<TX, TY, MK, WALLS, ST, RHO0>(a, X, Y, li, lj, Fs, Fs0, hp, hp0);
}

// Phase C of the own node (X, Y): pass 2 from the f region, the output and
// the NEE output of an adjacent wall node.
// Store one node in the layout of the storage mode (with the periodic
// images of a periodic x axis when XPER).
template <int ST, bool XPER>
__device__ __forceinline__ void tile_store(const StepArgs &a, int row, int X, const F2 v[5]) {
    if (ST == STORAGE_FP32) store_node<XPER>(a, row, X, v);
    else store_node_dev<ST, XPER>(a, row, X, v);
}

// Store the alpha = 0 populations of one node (planes 10..14).
template <bool RHO0, bool XPER>
__device__ __forceinline__ void tile_store0(const StepArgs &a, int row, int X, const float v[5]) {
    if (RHO0) store_node0<XPER>(a, row, X, v);
}

template <int TX, int TY, int MK, bool WALLS, int ST, bool RHO0>
__device__ __forceinline__ void tile_output(const StepArgs &a, int X, int Y, int li, int lj, const unsigned char *Fs,
                                            const float *Fs0, const F2 hp[5], const float hp0[5]) {
    using T = Tile<TX, TY>;
    const bool xwall = WALLS && a.xwall, ywall = WALLS && a.ywall;
    const float inv2c = a.inv2c;
    const bool xadj_p = xwall && X == 1, xadj_m = xwall && X == a.nx - 2;
    const bool yadj_p = ywall && Y == 1, yadj_m = ywall && Y == a.ny - 2;
    const int n4 = (lj + 2) * T::X4 + li + 2;
    F2 fF = splat(0.0f);
    const F2 dw = splat(a.dt * 0.2f);
    if (a.force_mode_d == 1) fF = dw * mk2(a.Fxd, a.Fyd);
    else if (a.force_mode_d == 2) {
        const long long fi = (long long)Y * a.pitch + GHOST + X;
        fF = dw * field_pair(a, a.Fxdp, a.Fydp, fi);
    }
    F2 out[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) out[j] = hp[j] + fF;
    stream_tile<T::N4, MK, WALLS>(Fs, n4, T::X4, a.dt, X, Y, xadj_p, xadj_m, yadj_p, yadj_m, a, out);
    float out0[5], un = 0.0f, vn = 0.0f;
    if (RHO0) {
        // Step 4 on alpha = 0: fhat^+ - dt c.grad f + dt w_j R
        const float sR = a.r_mode ? a.dt * 0.2f * source_at(a, Y, X) : 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j) out0[j] = hp0[j] + sR;
        stream_tile0<T::N4, MK, WALLS>(Fs0, n4, T::X4, a.dt, X, Y, xadj_p, xadj_m, yadj_p, yadj_m, a, out0);
        split2((out[0] + out[1]) + (out[2] + out[3]) + out[4], un, vn);
    }
    if (!WALLS) {
        tile_store<ST, true>(a, Y, X, out);
        tile_store0<RHO0, true>(a, Y, X, out0);
        return;
    }
    if (xwall) {
        tile_store<ST, false>(a, Y, X, out);
        tile_store0<RHO0, false>(a, Y, X, out0);
    } else {
        tile_store<ST, true>(a, Y, X, out);
        tile_store0<RHO0, true>(a, Y, X, out0);
    }
    F2 w[5];
    float w0[5];
    auto wall = [&](int side, int row, int col, bool xper) {
        nee2(out, a.uw[side], a.vw[side], inv2c, w);
        if (RHO0) nee0(out0, a.uw[side], a.vw[side], un, vn, inv2c, w0);
        if (xper) {
            tile_store<ST, true>(a, row, col, w);
            tile_store0<RHO0, true>(a, row, col, w0);
        } else {
            tile_store<ST, false>(a, row, col, w);
            tile_store0<RHO0, false>(a, row, col, w0);
        }
    };
    if (xadj_p) wall(0, Y, 0, false);
    if (xadj_m) wall(1, Y, a.nx - 1, false);
    if (ywall && (Y == 1 || Y == a.ny - 2)) {
        const int rr = (Y == 1) ? 0 : a.ny - 1;
        wall((Y == 1) ? 2 : 3, rr, X, !xwall);
        if (xadj_p) wall(0, rr, 0, false);
        if (xadj_m) wall(1, rr, a.nx - 1, false);
    }
}

template <int TX, int TY, int MK, bool PL, bool WALLS, int ST, bool RHO0>
__global__ void __launch_bounds__(TX *TY, kTileMinBlocks) tile_kernel(const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    // launched with programmatic stream serialization: the block touches
    // global memory only after the previous step has completed.  The next
    // step is released only as this one's blocks exit (no early trigger): a
    // grid of fewer blocks than resident slots would otherwise place the
    // next step's blocks on the SMs left free, up to three on one SM
    grid_dependency_wait();
    tile_step<TX, TY, MK, PL, WALLS, ST, RHO0>(a, blockIdx.x, blockIdx.y, smem);
}

// Many problems in one persistent launch: block b steps work items
// b, b + gridDim.x, ... (problem, tile x, tile y), largest problems first.
template <int TX, int TY, int MK, bool PL, bool WALLS, int ST>
__global__ void __launch_bounds__(TX *TY, kTileMinBlocks) tile_batch_kernel(const BatchItem *__restrict__ items, int nitems,
                                                               const StepArgs *__restrict__ args) {
    extern __shared__ __align__(128) unsigned char smem[];
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const BatchItem item = items[w];
        tile_step<TX, TY, MK, PL, WALLS, ST, false>(args[item.problem], item.bx, item.by, smem);
    }
}

constexpr int kTX = TILE_X, kTY = TILE_Y;

template <int MK, bool PL, bool WALLS, bool RHO0 = false>
constexpr int tile_smem() {
    using T = Tile<kTX, kTY>;
    return T::B_BYTES + T::F_BYTES + (PL ? T::K_BYTES : 0) + (RHO0 ? T::B0_BYTES + T::F0_BYTES : 0);
}

template <int MK, bool PL, bool WALLS, int ST, bool RHO0 = false>
cudaError_t tile_occupancy_t(int *occ, int *smem) {
    auto k = tile_kernel<kTX, kTY, MK, PL, WALLS, ST, RHO0>;
    *smem = tile_smem<MK, PL, WALLS, RHO0>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, kTX * kTY, *smem);
}

template <int MK, bool PL, bool WALLS, int ST, bool RHO0 = false>
cudaError_t tile_launch_t(const StepArgs &args, const StepPlan &plan, cudaStream_t stream) {
    auto k = tile_kernel<kTX, kTY, MK, PL, WALLS, ST, RHO0>;
    constexpr int smem = tile_smem<MK, PL, WALLS, RHO0>();
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    // programmatic stream serialization: the next step's blocks are
    // scheduled while this one drains (tile_kernel waits for it in hardware)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.gx, plan.gy);
    cfg.blockDim = dim3(kTX * kTY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, args);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int MK, bool PL, bool WALLS, int ST>
cudaError_t tile_batch_occupancy_t(int *occ, int *smem) {
    auto k = tile_batch_kernel<kTX, kTY, MK, PL, WALLS, ST>;
    *smem = tile_smem<MK, PL, WALLS>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, kTX * kTY, *smem);
}

template <int MK, bool PL, bool WALLS, int ST>
cudaError_t tile_batch_launch_t(const BatchItem *items, int nitems, const StepArgs *args, int grid,
                                cudaStream_t stream) {
    auto k = tile_batch_kernel<kTX, kTY, MK, PL, WALLS, ST>;
    static std::atomic<unsigned long long> configured{0};  // devices set up
    if (needs_device_setup(configured)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_smem<MK, PL, WALLS>());
        if (e != cudaSuccess) return e;
        mark_device_setup(configured);
    }
    k<<<grid, kTX * kTY, tile_smem<MK, PL, WALLS>(), stream>>>(items, nitems, args);
    return cudaGetLastError();
}

// Instantiate FN for the grid kind, fluid model and wall variant at run time.
#define MDF_TILE_DISPATCH(ST, FN, ...)                                             \
    switch (metric * 4 + (power_law ? 2 : 0) + (walls ? 1 : 0)) {                  \
        case 0: return FN<METRIC_UNIFORM, false, false, ST>(__VA_ARGS__);          \
        case 1: return FN<METRIC_UNIFORM, false, true, ST>(__VA_ARGS__);           \
        case 2: return FN<METRIC_UNIFORM, true, false, ST>(__VA_ARGS__);           \
        case 3: return FN<METRIC_UNIFORM, true, true, ST>(__VA_ARGS__);            \
        case 4: return FN<METRIC_SEPARABLE, false, false, ST>(__VA_ARGS__);        \
        case 5: return FN<METRIC_SEPARABLE, false, true, ST>(__VA_ARGS__);         \
        case 6: return FN<METRIC_SEPARABLE, true, false, ST>(__VA_ARGS__);         \
        case 7: return FN<METRIC_SEPARABLE, true, true, ST>(__VA_ARGS__);          \
        case 8: return FN<METRIC_CURVILINEAR, false, false, ST>(__VA_ARGS__);      \
        case 9: return FN<METRIC_CURVILINEAR, false, true, ST>(__VA_ARGS__);       \
        case 10: return FN<METRIC_CURVILINEAR, true, false, ST>(__VA_ARGS__);      \
        default: return FN<METRIC_CURVILINEAR, true, true, ST>(__VA_ARGS__);       \
    }

// FN with the alpha = 0 lane (FP32 storage).
#define MDF_TILE_DISPATCH_RHO0(FN, ...)                                                    \
    switch (metric * 4 + (power_law ? 2 : 0) + (walls ? 1 : 0)) {                          \
        case 0: return FN<METRIC_UNIFORM, false, false, STORAGE_FP32, true>(__VA_ARGS__);     \
        case 1: return FN<METRIC_UNIFORM, false, true, STORAGE_FP32, true>(__VA_ARGS__);      \
        case 2: return FN<METRIC_UNIFORM, true, false, STORAGE_FP32, true>(__VA_ARGS__);      \
        case 3: return FN<METRIC_UNIFORM, true, true, STORAGE_FP32, true>(__VA_ARGS__);       \
        case 4: return FN<METRIC_SEPARABLE, false, false, STORAGE_FP32, true>(__VA_ARGS__);   \
        case 5: return FN<METRIC_SEPARABLE, false, true, STORAGE_FP32, true>(__VA_ARGS__);    \
        case 6: return FN<METRIC_SEPARABLE, true, false, STORAGE_FP32, true>(__VA_ARGS__);    \
        case 7: return FN<METRIC_SEPARABLE, true, true, STORAGE_FP32, true>(__VA_ARGS__);     \
        case 8: return FN<METRIC_CURVILINEAR, false, false, STORAGE_FP32, true>(__VA_ARGS__); \
        case 9: return FN<METRIC_CURVILINEAR, false, true, STORAGE_FP32, true>(__VA_ARGS__);  \
        case 10: return FN<METRIC_CURVILINEAR, true, false, STORAGE_FP32, true>(__VA_ARGS__); \
        default: return FN<METRIC_CURVILINEAR, true, true, STORAGE_FP32, true>(__VA_ARGS__);  \
    }

}  // namespace

// The tile kernel with the alpha = 0 lane (mdf_step_tile_rho0.cu).
cudaError_t tile_occupancy_rho0(int metric, int power_law, int walls, int *occ, int *smem);
cudaError_t tile_launch_rho0(const StepArgs &args, int metric, const StepPlan &plan, cudaStream_t stream);

// The tile kernel's launch helpers for one storage mode ST (defined in
// mdf_step_tile.cu for FP32 and mdf_step_tile16.cu for FP16 and BF16).
template <int ST>
cudaError_t tile_occupancy_st(int metric, int power_law, int walls, int *occ, int *smem);
template <int ST>
cudaError_t tile_launch_st(const StepArgs &args, int metric, const StepPlan &plan, cudaStream_t stream);
template <int ST>
cudaError_t tile_batch_occupancy_st(int metric, int power_law, int walls, int *occ, int *smem);
template <int ST>
cudaError_t tile_batch_launch_st(const BatchItem *items, int nitems, const StepArgs *args, int metric, int power_law,
                                 int walls, int grid, cudaStream_t stream);

// Definitions of the four helpers for storage mode ST in the including file.
#define MDF_TILE_DEFINE(ST)                                                                                        \
    template <>                                                                                                    \
    cudaError_t tile_occupancy_st<ST>(int metric, int power_law, int walls, int *occ, int *smem) {                 \
        MDF_TILE_DISPATCH(ST, tile_occupancy_t, occ, smem)                                                         \
    }                                                                                                              \
    template <>                                                                                                    \
    cudaError_t tile_launch_st<ST>(const StepArgs &args, int metric, const StepPlan &plan, cudaStream_t stream) {  \
        const int power_law = args.power_law;                                                                      \
        const int walls = (args.xwall || args.ywall) ? 1 : 0;                                                      \
        MDF_TILE_DISPATCH(ST, tile_launch_t, args, plan, stream)                                                   \
    }                                                                                                              \
    template <>                                                                                                    \
    cudaError_t tile_batch_occupancy_st<ST>(int metric, int power_law, int walls, int *occ, int *smem) {           \
        MDF_TILE_DISPATCH(ST, tile_batch_occupancy_t, occ, smem)                                                   \
    }                                                                                                              \
    template <>                                                                                                    \
    cudaError_t tile_batch_launch_st<ST>(const BatchItem *items, int nitems, const StepArgs *args, int metric,     \
                                         int power_law, int walls, int grid, cudaStream_t stream) {               \
        MDF_TILE_DISPATCH(ST, tile_batch_launch_t, items, nitems, args, grid, stream)                              \
    }

}  // namespace mdf
