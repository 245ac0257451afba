// net_kernels.cu -- kernels of the warm-start network.
//
// The 3 x 3 convolutions are implicit GEMMs on the BF16 tensor cores
// (mma.sync m16n8k16, FP32 accumulation): a block computes a 128 x 64 tile of
// out[pixel][channel] with 8 warps of 32 x 32, gathering the input rows of
// one filter tap per 32-wide K step straight from the NHWC activations (zero
// outside the image) into double-buffered shared memory.  The weight
// gradient is the transposed product, split over pixels and reduced with
// FP32 atomics into the flat gradient vector.
#include <math.h>

#include "net_internal.cuh"

namespace mdfnet {

namespace {

constexpr int LDS = 40;  // shared row stride in BF16 (80 B: conflict-free fragment loads)

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 32-wide K step of a warp's 32 x 32 tile: A rows [arow, arow + 32),
// B rows [brow, brow + 32) of K-contiguous shared tiles.
__device__ __forceinline__ void warp_tile_k32(const bf16 *A, const bf16 *B, int arow, int brow, int lane,
                                              float acc[2][4][4]) {
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const bf16 *p = A + (arow + mi * 16 + g) * LDS + kk + 2 * c;
            af[mi][0] = ld32(p);
            af[mi][1] = ld32(p + 8 * LDS);
            af[mi][2] = ld32(p + 8);
            af[mi][3] = ld32(p + 8 * LDS + 8);
        }
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const bf16 *p = B + (brow + ni * 8 + g) * LDS + kk + 2 * c;
            bfr[ni][0] = ld32(p);
            bfr[ni][1] = ld32(p + 8);
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma16816(acc[mi][ni], af[mi], bfr[ni]);
    }
}

// ---------------------------------------------------------------- convolution

constexpr int CBM = 128, CBN = 64;

__global__ void __launch_bounds__(256) conv_kernel(ConvArgs a) {
    __shared__ __align__(16) bf16 As[2][CBM * LDS];
    __shared__ __align__(16) bf16 Bs[2][CBN * LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int RR = a.R * a.R;
    const long long M = (long long)a.B * RR;
    const long long m0 = (long long)blockIdx.x * CBM;
    const int n0 = blockIdx.y * CBN;
    const int K = 9 * a.Cx, KT = K / 32;
    const int q = tid & 3;

    // the two A rows and the B row this thread stages
    long long abase[2];
    int ay[2], ax[2];
    bool aval[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const long long m = m0 + (tid >> 2) + 64 * i;
        aval[i] = m < M;
        const long long img = aval[i] ? m / RR : 0;
        const int rem = aval[i] ? (int)(m - img * RR) : 0;
        abase[i] = img * RR;
        ay[i] = rem / a.R;
        ax[i] = rem - ay[i] * a.R;
    }
    const int bco = n0 + (tid >> 2);
    const uint4 zero = make_uint4(0, 0, 0, 0);
    uint4 ra[2], rb;

    auto load = [&](int kt) {
        const int k0 = kt * 32;
        const int tap = k0 / a.Cx, c0 = k0 - tap * a.Cx;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int yy = ay[i] + dy, xx = ax[i] + dx;
            ra[i] = (aval[i] && yy >= 0 && yy < a.R && xx >= 0 && xx < a.R)
                        ? *reinterpret_cast<const uint4 *>(a.X + (abase[i] + (long long)yy * a.R + xx) * a.Cx + c0 +
                                                           8 * q)
                        : zero;
        }
        rb = bco < a.N ? *reinterpret_cast<const uint4 *>(a.W + (long long)bco * K + k0 + 8 * q) : zero;
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 2; ++i) *reinterpret_cast<uint4 *>(&As[buf][((tid >> 2) + 64 * i) * LDS + 8 * q]) = ra[i];
        *reinterpret_cast<uint4 *>(&Bs[buf][(tid >> 2) * LDS + 8 * q]) = rb;
    };

    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.0f;

    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < KT; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < KT) load(kt + 1);
        warp_tile_k32(As[cur], Bs[cur], wm * 32, wn * 32, lane, acc);
        if (kt + 1 < KT) store(cur ^ 1);
        __syncthreads();
    }

    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int col = n0 + wn * 32 + ni * 8 + 2 * c;
            if (col >= a.N) continue;
            const float b0 = a.bias ? a.bias[col] : 0.0f, b1 = a.bias ? a.bias[col + 1] : 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long m = m0 + wm * 32 + mi * 16 + g + 8 * h;
                if (m >= M) continue;
                float v0 = acc[mi][ni][2 * h] + b0, v1 = acc[mi][ni][2 * h + 1] + b1;
                if (a.skip) {
                    const float2 s = __bfloat1622float2(
                        *reinterpret_cast<const __nv_bfloat162 *>(a.skip + m * a.N + col));
                    v0 += s.x;
                    v1 += s.y;
                }
                const __nv_bfloat162 zb = __floats2bfloat162_rn(v0, v1);
                if (a.out) *reinterpret_cast<__nv_bfloat162 *>(a.out + m * a.N + col) = zb;
                if (a.act)
                    *reinterpret_cast<__nv_bfloat162 *>(a.act + m * a.N + col) =
                        __halves2bfloat162(silu_bf16(__low2bfloat16(zb)), silu_bf16(__high2bfloat16(zb)));
                if (a.outf) {
                    if (col < a.nf) a.outf[m * a.nf + col] = v0;
                    if (col + 1 < a.nf) a.outf[m * a.nf + col + 1] = v1;
                }
            }
        }
}

// ------------------------------------------------------------ weight gradient

constexpr int WBM = 64, WBN = 128;

__global__ void __launch_bounds__(256) wgrad_kernel(WGradArgs a, int chunk) {
    __shared__ __align__(16) bf16 As[2][WBM * LDS];  // [co][pixel]
    __shared__ __align__(16) bf16 Bs[2][WBN * LDS];  // [(tap, ci)][pixel]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int RR = a.R * a.R;
    const long long P = (long long)a.B * RR;
    const int NC = 9 * a.Cin;
    const int co0 = blockIdx.y * WBM, n0 = blockIdx.x * WBN;
    const long long ktiles = (P + 31) / 32;
    const long long kt0 = (long long)blockIdx.z * chunk;
    const long long kt1 = kt0 + chunk < ktiles ? kt0 + chunk : ktiles;
    if (kt0 >= kt1) return;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    uint4 ra, rb[2];

    auto load = [&](long long kt) {
        const long long p = kt * 32 + lane;  // this lane's pixel
        const bool pv = p < P;
        const int co = co0 + 8 * warp;
        ra = (pv && co < a.Cout) ? *reinterpret_cast<const uint4 *>(a.dZ + p * a.Cout + co) : zero;
        const long long img = pv ? p / RR : 0;
        const int rem = pv ? (int)(p - img * RR) : 0;
        const int y = rem / a.R, x = rem - y * a.R;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int n = n0 + 8 * (warp + 8 * i);
            const int tap = n / a.Cin, ci = n - tap * a.Cin;
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            rb[i] = (pv && n < NC && yy >= 0 && yy < a.R && xx >= 0 && xx < a.R)
                        ? *reinterpret_cast<const uint4 *>(a.X + (img * RR + (long long)yy * a.R + xx) * a.Cin + ci)
                        : zero;
        }
    };
    auto store = [&](int buf) {
        const bf16 *e = reinterpret_cast<const bf16 *>(&ra);
#pragma unroll
        for (int k = 0; k < 8; ++k) As[buf][(8 * warp + k) * LDS + lane] = e[k];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const bf16 *f = reinterpret_cast<const bf16 *>(&rb[i]);
#pragma unroll
            for (int k = 0; k < 8; ++k) Bs[buf][(8 * (warp + 8 * i) + k) * LDS + lane] = f[k];
        }
    };

    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.0f;

    load(kt0);
    store(0);
    __syncthreads();
    for (long long kt = kt0; kt < kt1; ++kt) {
        const int cur = (int)((kt - kt0) & 1);
        if (kt + 1 < kt1) load(kt + 1);
        warp_tile_k32(As[cur], Bs[cur], wm * 32, wn * 32, lane, acc);
        if (kt + 1 < kt1) store(cur ^ 1);
        __syncthreads();
    }

    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = co0 + wm * 32 + mi * 16 + g + 8 * (e >> 1);
                const int n = n0 + wn * 32 + ni * 8 + 2 * c + (e & 1);
                if (co >= a.cout_real || n >= NC) continue;
                const int tap = n / a.Cin, ci = n - tap * a.Cin;
                if (ci >= a.cin_real) continue;
                atomicAdd(a.g + a.off + ((long long)co * 9 + tap) * a.cin_real + ci, acc[mi][ni][e]);
            }
}

// Bias gradient: sum over pixels of dZ[m][co], one block per pixel chunk.
__global__ void bias_grad_kernel(const bf16 *dZ, long long P, int Cout, int cout_real, long long chunk, float *g) {
    const long long p0 = (long long)blockIdx.x * chunk;
    const long long p1 = p0 + chunk < P ? p0 + chunk : P;
    for (int co = threadIdx.x; co < cout_real; co += blockDim.x) {
        float s = 0.0f;
        for (long long p = p0; p < p1; ++p) s += __bfloat162float(dZ[p * Cout + co]);
        atomicAdd(g + co, s);
    }
}

// ------------------------------------------------------------- elementwise

__device__ __forceinline__ float sigm(float z) { return net_sigmoid(z); }

__global__ void silu_fwd_kernel(const bf16 *z, bf16 *y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = silu_bf16(z[i]);
}

// The elementwise kernels below move 8 BF16 channels (16 bytes) per thread
// and step: C is a multiple of 32, so a group never straddles two pixels.
typedef uint4 bf16x8;

__device__ __forceinline__ void unpack8(const bf16x8 &w, float f[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float2 t = __bfloat1622float2(h[e]);
        f[2 * e] = t.x;
        f[2 * e + 1] = t.y;
    }
}
__device__ __forceinline__ bf16x8 pack8(const float f[8]) {
    bf16x8 w;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&w);
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
    return w;
}

// dz = dy silu'(z), silu'(z) = s (1 + z (1 - s)), s = sigmoid(z); n8 = n / 8
__global__ void silu_bwd_kernel(const bf16x8 *z, const bf16x8 *dy, bf16x8 *dz, long long n8) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x) {
        float a[8], b[8];
        unpack8(z[i], a);
        unpack8(dy[i], b);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float sg = sigm(a[e]);
            b[e] = b[e] * sg * (1.0f + a[e] * (1.0f - sg));
        }
        dz[i] = pack8(b);
    }
}

// x [B][R][R][C] -> y [B][R/2][R/2][C]; C8 = C / 8
__global__ void pool_fwd_kernel(const bf16x8 *x, bf16x8 *y, int B, int R, int C8) {
    const int h = R / 2;
    const long long n = (long long)B * h * h * C8;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8);
        long long t = i / C8;
        const int xo = (int)(t % h);
        t /= h;
        const int yo = (int)(t % h);
        const long long b = t / h;
        const long long base = ((b * R + 2 * yo) * R + 2 * xo) * C8 + c;
        float p[8], q[8], r[8], u[8];
        unpack8(x[base], p);
        unpack8(x[base + C8], q);
        unpack8(x[base + (long long)R * C8], r);
        unpack8(x[base + (long long)R * C8 + C8], u);
#pragma unroll
        for (int e = 0; e < 8; ++e) p[e] = 0.25f * (p[e] + q[e] + r[e] + u[e]);
        y[i] = pack8(p);
    }
}

// dy [B][R/2][R/2][C] -> dx [B][R][R][C] = dy / 4 on each 2 x 2 block
__global__ void pool_bwd_kernel(const bf16x8 *dy, bf16x8 *dx, int B, int R, int C8) {
    const long long n = (long long)B * R * R * C8;
    const int h = R / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8);
        long long t = i / C8;
        const int x = (int)(t % R);
        t /= R;
        const int y = (int)(t % R);
        const long long b = t / R;
        float f[8];
        unpack8(dy[((b * h + y / 2) * h + x / 2) * C8 + c], f);
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] *= 0.25f;
        dx[i] = pack8(f);
    }
}

// x [B][R][R][C] -> y [B][2R][2R][C] (nearest)
__global__ void up_fwd_kernel(const bf16x8 *x, bf16x8 *y, int B, int R, int C8) {
    const int R2 = 2 * R;
    const long long n = (long long)B * R2 * R2 * C8;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8);
        long long t = i / C8;
        const int xo = (int)(t % R2);
        t /= R2;
        const int yo = (int)(t % R2);
        const long long b = t / R2;
        y[i] = x[((b * R + yo / 2) * R + xo / 2) * C8 + c];
    }
}

// dy [B][2R][2R][C] -> dx [B][R][R][C] = sum of the four children
__global__ void up_bwd_kernel(const bf16x8 *dy, bf16x8 *dx, int B, int R, int C8) {
    const int R2 = 2 * R;
    const long long n = (long long)B * R * R * C8;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8);
        long long t = i / C8;
        const int x = (int)(t % R);
        t /= R;
        const int y = (int)(t % R);
        const long long b = t / R;
        const long long base = ((b * R2 + 2 * y) * R2 + 2 * x) * C8 + c;
        float p[8], q[8], r[8], u[8];
        unpack8(dy[base], p);
        unpack8(dy[base + C8], q);
        unpack8(dy[base + (long long)R2 * C8], r);
        unpack8(dy[base + (long long)R2 * C8 + C8], u);
#pragma unroll
        for (int e = 0; e < 8; ++e) p[e] = p[e] + q[e] + r[e] + u[e];
        dx[i] = pack8(p);
    }
}

__global__ void add_kernel(bf16x8 *dst, const bf16x8 *src, long long n8) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x) {
        float a[8], b[8];
        unpack8(dst[i], a);
        unpack8(src[i], b);
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] += b[e];
        dst[i] = pack8(a);
    }
}

__global__ void pack_input_kernel(const float *in, bf16 *x, int B, int R) {
    const long long P = (long long)B * R * R;
    const int RR = R * R;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const long long b = p / RR;
        const int s = (int)(p - b * RR);
        bf16 *o = x + p * 32;
#pragma unroll
        for (int c = 0; c < 32; ++c)
            o[c] = __float2bfloat16_rn(c < NET_IN_PLANES ? in[(b * NET_IN_PLANES + c) * RR + s] : 0.0f);
    }
}

__global__ void unpack_output_kernel(const float *o, float *out, int B, int R) {
    const long long P = (long long)B * R * R;
    const int RR = R * R;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const long long b = p / RR;
        const int s = (int)(p - b * RR);
#pragma unroll
        for (int c = 0; c < 3; ++c) out[(b * 3 + c) * RR + s] = o[p * 3 + c];
    }
}

__global__ void pack_target_kernel(const float *t, float *o, int B, int R) {
    const long long P = (long long)B * R * R;
    const int RR = R * R;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const long long b = p / RR;
        const int s = (int)(p - b * RR);
#pragma unroll
        for (int c = 0; c < 3; ++c) o[p * 3 + c] = t[(b * 3 + c) * RR + s];
    }
}

__global__ void mse_kernel(const float *o, const float *t, bf16 *dout, double *loss, long long P, double inv_count) {
    double local = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        __align__(16) bf16 row[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) row[c] = __float2bfloat16_rn(0.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = o[p * 3 + c] - t[p * 3 + c];
            local += (double)d * d;
            row[c] = __float2bfloat16_rn((float)(2.0 * inv_count) * d);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dout + p * 32);
        const uint4 *src = reinterpret_cast<const uint4 *>(row);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = src[k];
    }
    for (int o_ = 16; o_ > 0; o_ >>= 1) local += __shfl_down_sync(0xffffffffu, local, o_);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, local * inv_count);
}

__global__ void prepare_kernel(const float *params, long long off, int cin_real, int cout_real, int cin_pad,
                               int cout_pad, bf16 *wf, bf16 *wb, float *bias) {
    const long long n = (long long)cout_pad * 9 * cin_pad;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin_pad);
        const long long t = i / cin_pad;
        const int tap = (int)(t % 9);
        const int co = (int)(t / 9);
        const float w = (co < cout_real && ci < cin_real) ? params[off + ((long long)co * 9 + tap) * cin_real + ci] : 0.0f;
        const bf16 h = __float2bfloat16_rn(w);
        wf[i] = h;
        if (wb) wb[((long long)ci * 9 + (8 - tap)) * cout_pad + co] = h;
        if (i < cout_pad) bias[i] = i < cout_real ? params[off + (long long)cout_real * 9 * cin_real + i] : 0.0f;
    }
}

__global__ void adam_kernel(float *p, float *m, float *v, const float *g, long long n, float lr_t, float b1, float b2,
                            float eps_t) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr_t * mi / (sqrtf(vi) + eps_t);
    }
}

inline int blocks_for(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    if (b > 65535) b = 65535;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t conv_forward(const ConvArgs &a, cudaStream_t st) {
    if (a.Cx % 32 || a.N % 2) return cudaErrorInvalidValue;
    const long long M = (long long)a.B * a.R * a.R;
    dim3 grid((unsigned)((M + CBM - 1) / CBM), (unsigned)((a.N + CBN - 1) / CBN));
    conv_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t conv_wgrad(const WGradArgs &a, int num_sms, cudaStream_t st) {
    if (a.Cin % 8 || a.Cout % 8) return cudaErrorInvalidValue;
    const long long P = (long long)a.B * a.R * a.R;
    const long long ktiles = (P + 31) / 32;
    const int tn = (9 * a.Cin + WBN - 1) / WBN, tm = (a.Cout + WBM - 1) / WBM;
    long long splits = (4ll * num_sms + tn * tm - 1) / (tn * tm);
    if (splits > ktiles) splits = ktiles;
    if (splits < 1) splits = 1;
    const long long chunk = (ktiles + splits - 1) / splits;
    splits = (ktiles + chunk - 1) / chunk;
    wgrad_kernel<<<dim3(tn, tm, (unsigned)splits), 256, 0, st>>>(a, (int)chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long pchunk = 256;
    bias_grad_kernel<<<(unsigned)((P + pchunk - 1) / pchunk), 256, 0, st>>>(
        a.dZ, P, a.Cout, a.cout_real, pchunk, a.g + a.off + (long long)a.cout_real * 9 * a.cin_real);
    return cudaGetLastError();
}

cudaError_t silu_forward(const bf16 *z, bf16 *y, long long n, cudaStream_t st) {
    silu_fwd_kernel<<<blocks_for(n), 256, 0, st>>>(z, y, n);
    return cudaGetLastError();
}
cudaError_t silu_backward(const bf16 *z, const bf16 *dy, bf16 *dz, long long n, cudaStream_t st) {
    if (n % 8) return cudaErrorInvalidValue;
    silu_bwd_kernel<<<blocks_for(n / 8), 256, 0, st>>>(reinterpret_cast<const bf16x8 *>(z),
                                                      reinterpret_cast<const bf16x8 *>(dy),
                                                      reinterpret_cast<bf16x8 *>(dz), n / 8);
    return cudaGetLastError();
}
cudaError_t pool_forward(const bf16 *x, bf16 *y, int B, int R, int C, cudaStream_t st) {
    if (C % 8) return cudaErrorInvalidValue;
    pool_fwd_kernel<<<blocks_for((long long)B * R * R * C / 32), 256, 0, st>>>(
        reinterpret_cast<const bf16x8 *>(x), reinterpret_cast<bf16x8 *>(y), B, R, C / 8);
    return cudaGetLastError();
}
cudaError_t pool_backward(const bf16 *dy, bf16 *dx, int B, int R, int C, cudaStream_t st) {
    if (C % 8) return cudaErrorInvalidValue;
    pool_bwd_kernel<<<blocks_for((long long)B * R * R * C / 8), 256, 0, st>>>(
        reinterpret_cast<const bf16x8 *>(dy), reinterpret_cast<bf16x8 *>(dx), B, R, C / 8);
    return cudaGetLastError();
}
cudaError_t up_forward(const bf16 *x, bf16 *y, int B, int R, int C, cudaStream_t st) {
    if (C % 8) return cudaErrorInvalidValue;
    up_fwd_kernel<<<blocks_for((long long)B * R * R * C / 2), 256, 0, st>>>(
        reinterpret_cast<const bf16x8 *>(x), reinterpret_cast<bf16x8 *>(y), B, R, C / 8);
    return cudaGetLastError();
}
cudaError_t up_backward(const bf16 *dy, bf16 *dx, int B, int R, int C, cudaStream_t st) {
    if (C % 8) return cudaErrorInvalidValue;
    up_bwd_kernel<<<blocks_for((long long)B * R * R * C / 8), 256, 0, st>>>(
        reinterpret_cast<const bf16x8 *>(dy), reinterpret_cast<bf16x8 *>(dx), B, R, C / 8);
    return cudaGetLastError();
}
cudaError_t add_inplace(bf16 *dst, const bf16 *src, long long n, cudaStream_t st) {
    if (n % 8) return cudaErrorInvalidValue;
    add_kernel<<<blocks_for(n / 8), 256, 0, st>>>(reinterpret_cast<bf16x8 *>(dst),
                                                  reinterpret_cast<const bf16x8 *>(src), n / 8);
    return cudaGetLastError();
}
cudaError_t pack_input(const float *in, bf16 *x, int B, int R, cudaStream_t st) {
    pack_input_kernel<<<blocks_for((long long)B * R * R), 256, 0, st>>>(in, x, B, R);
    return cudaGetLastError();
}
cudaError_t unpack_output(const float *o, float *out, int B, int R, cudaStream_t st) {
    unpack_output_kernel<<<blocks_for((long long)B * R * R), 256, 0, st>>>(o, out, B, R);
    return cudaGetLastError();
}
cudaError_t pack_target(const float *t, float *o, int B, int R, cudaStream_t st) {
    pack_target_kernel<<<blocks_for((long long)B * R * R), 256, 0, st>>>(t, o, B, R);
    return cudaGetLastError();
}
cudaError_t mse_loss(const float *o, const float *t, bf16 *dout, double *loss, int B, int R, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long long P = (long long)B * R * R;
    mse_kernel<<<blocks_for(P), 256, 0, st>>>(o, t, dout, loss, P, 1.0 / (3.0 * (double)P));
    return cudaGetLastError();
}
cudaError_t prepare_layer(const float *params, long long off, int cin_real, int cout_real, int cin_pad,
                          int cout_pad, bf16 *wf, bf16 *wb, float *bias, cudaStream_t st) {
    prepare_kernel<<<blocks_for((long long)cout_pad * 9 * cin_pad), 256, 0, st>>>(params, off, cin_real, cout_real,
                                                                                   cin_pad, cout_pad, wf, wb, bias);
    return cudaGetLastError();
}
cudaError_t adam_step(float *p, float *m, float *v, const float *g, long long n, float lr_t, float b1, float b2,
                      float eps_t, cudaStream_t st) {
    adam_kernel<<<blocks_for(n), 256, 0, st>>>(p, m, v, g, n, lr_t, b1, b2, eps_t);
    return cudaGetLastError();
}

}  // namespace mdfnet
