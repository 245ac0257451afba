// net_tc.cu -- the warm-start network's 3 x 3 convolutions on the
// fifth-generation tensor cores: tcgen05.mma with the accumulators in tensor
// memory (TMEM), operands staged in shared memory by TMA.
//
// The product is the implicit GEMM of conv_kernel (net_kernels.cu):
// out[m][n] = sum_k A[m][k] W[n][k] (+ bias[n]) (+ skip[m][n]), m a pixel,
// n an output channel, k = (tap, c) with A[m][(tap, c)] the input at pixel m
// shifted by the tap (zero outside the image), optionally followed by the
// SiLU activation.  A persistent CTA of six warps walks 128 x BN output
// tiles:
//  * A, for every tap and chunk of BKC channels, is ONE TMA box of the NHWC
//    input, [BKC channels] x [Wx columns] x [Hy rows] x [Bn images] = 128
//    pixels, started at the tile's first pixel shifted by the tap; TMA fills
//    the coordinates outside the image with zeros, which is the convolution's
//    zero padding;
//  * W's box is [BKC channels] x [1 tap] x [BN output channels] of the
//    [N][9][C] weights;
//  * both land in shared memory in the swizzled K-major layout (rows of
//    BKC x 2 bytes: 128-byte swizzle for BKC = 64, 64-byte for BKC = 32)
//    that the MMA's shared-memory descriptors describe;
//  * warp 0 fills a ring of STAGES slots; warp 1 issues the MMAs (M = 128,
//    N = BN, K = 16 each, BF16 in, FP32 accumulated in TMEM) into one of two
//    accumulators and frees each slot with tcgen05.commit; warps 2-9 read
//    the other accumulator back (tcgen05.ld 32x32b: TMEM lane = pixel), add
//    bias and skip, apply the activation and store, so that the epilogue of
//    one tile overlaps the copies and MMAs of the next.
// Every wait is bounded (about two seconds).  A CTA that gives up records
// an error word, waits (bounded) for its own copies and MMAs to finish,
// frees its TMEM and returns; the host reports the word as MDF_E_CUDA.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "net_internal.cuh"

namespace mdfnet {

namespace {

constexpr int TC_BM = 128;
// warp 0: TMA, warp 1: MMA, warps 2-9: epilogue (two warps per TMEM lane
// quarter, each taking half of the accumulator's columns)
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);

__device__ __forceinline__ uint32_t s_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mb_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbarrier_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mb_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^32 clock cycles (about two seconds).
__device__ __forceinline__ bool mb_wait(uint64_t *bar, uint32_t parity) {
    if (mb_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mb_try_wait(bar, parity)) return true;
        if (clock64() - t0 > (1ll << 32)) return false;
    }
}

__device__ __forceinline__ void tma_load_4d(const CUtensorMap *map, uint64_t *bar, void *dst, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(s_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(s_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(const CUtensorMap *map, uint64_t *bar, void *dst, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(s_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(s_u32(bar))
        : "memory");
}

// ---- tcgen05 (tensor memory and the fifth-generation MMA)

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] x B[smem]^T, one M = 128, N = BN, K = 16 step.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major operand in the swizzled
// layout TMA writes: rows of BKC x 2 bytes, 8-row groups SBO bytes apart;
// start address and offsets in 16-byte units, version 1 (bits 46-47),
// swizzle mode in bits 61-63 (2: 128-byte, 4: 64-byte).
template <int BKC>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
    constexpr uint64_t sbo = 8 * BKC * 2;         // bytes between 8-row groups
    constexpr uint64_t layout = BKC == 64 ? 2 : 4;
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46) |
           (layout << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

struct TcTile {
    int Wx, Hy, Bn;  // the 128-pixel tile as columns x rows x images
};

// Shared memory of one CTA: STAGES ring slots of G (A box, W box) pairs,
// 1024-byte aligned for the swizzle, then the barriers.
template <int BN, int BKC, int STAGES, int G, int MT>
struct TcSmem {
    static constexpr int SUBTILE = TC_BM * BKC * 2;  // one M = 128 block of an A box
    static constexpr int A_BYTES = MT * SUBTILE;
    static constexpr int B_BYTES = BN * BKC * 2;
    static constexpr int SUB = A_BYTES + B_BYTES;  // one K step: (A box, W box)
    static constexpr int STAGE = G * SUB;         // a ring slot holds G K steps
    static constexpr int BARS = STAGES * STAGE;
    // full[STAGES], empty[STAGES], tfull[2], tempty[2], drain; TMEM address
    static constexpr int NBAR = 2 * STAGES + 5;
    static constexpr int TOTAL = BARS + NBAR * 8 + 16 + 1024;  // + alignment slack
};

// Bounded wait that also gives up as soon as another role of the CTA has
// failed (*fail set).
__device__ __forceinline__ bool mb_wait_f(uint64_t *bar, uint32_t parity, volatile int *fail) {
    if (mb_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mb_try_wait(bar, parity)) return true;
        if (*fail) return false;
        if (clock64() - t0 > (1ll << 32)) return false;
    }
}

// Persistent, warp-specialised CTA of TC_THREADS threads walking output tiles
// tile = blockIdx.x, blockIdx.x + gridDim.x, ... (tile = m_tile * ntn + n_tile):
//   warp 0, lane 0   TMA producer: the (A, W) boxes of every K step into
//                    a STAGES-deep ring (full / empty barriers);
//   warp 1           allocates 2 x BN TMEM columns (two accumulators);
//                    lane 0 issues the MMAs of a tile into accumulator
//                    t & 1 and commits it (tfull) once its last K step is in;
//   warps 2-9        epilogue: TMEM lanes 32 (w % 4) .. + 31 and half of
//                    the columns of accumulator t & 1 -> bias, skip,
//                    activation, BF16/FP32 stores, then release the
//                    accumulator (tempty) so the MMAs of tile t + 2 may use it.
// The epilogue of one tile overlaps the copies and MMAs of the next.
template <int BN, int BKC, int STAGES, int G, int MT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap,
                   const ConvArgs a, int ntiles, int ntn, int *err) {
    using S = TcSmem<BN, BKC, STAGES, G, MT>;
    constexpr int BMT = TC_BM * MT;      // pixels of a tile (MT blocks of 128)
    constexpr int ACC = MT * BN;         // TMEM columns of one accumulator
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S::BARS);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    __shared__ int s_fail;
    __shared__ int s_issued, s_consumed;
    volatile int *fail = &s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = a.R, RR = R * R;
    const long long M = (long long)a.B * RR;
    const int kchunks = a.Cx / BKC;
    const int nk = 9 * kchunks;         // K steps of a tile
    const int ns = (nk + G - 1) / G;    // ring slots of a tile (the last may hold fewer steps)

    if (tid == 0) {
        s_fail = 0;
        s_issued = s_consumed = 0;
        for (int s = 0; s < STAGES; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mb_init(&tfull[b], 1);
            mb_init(&tempty[b], TC_EPI_WARPS);  // one arrival per epilogue warp
        }
        mb_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * ACC);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int k = 0;
            for (int tile = blockIdx.x; tile < ntiles && !*fail; tile += gridDim.x) {
                const long long m0 = (long long)(tile / ntn) * BMT;
                const int n0 = (tile % ntn) * BN;
                const int b0 = (int)(m0 / RR);
                const int rem = (int)(m0 - (long long)b0 * RR);
                const int y0 = rem / R, x0 = rem - y0 * R;
                for (int j = 0; j < ns; ++j, ++k) {
                    const int s = k % STAGES;
                    if (k >= STAGES && !mb_wait_f(&empty[s], (uint32_t)(((k / STAGES) - 1) & 1), fail)) {
                        *fail = 1;
                        break;
                    }
                    const int g = nk - j * G < G ? nk - j * G : G;
                    unsigned char *sa = smem + s * S::STAGE;
                    mb_expect_tx(&full[s], (uint32_t)(g * S::SUB));
                    for (int u = 0; u < g; ++u) {
                        const int i = j * G + u;
                        const int tap = i / kchunks, c0 = (i - tap * kchunks) * BKC;
                        tma_load_4d(&xmap, &full[s], sa + u * S::SUB, c0, x0 + tap % 3 - 1, y0 + tap / 3 - 1, b0);
                        tma_load_3d(&wmap, &full[s], sa + u * S::SUB + S::A_BYTES, c0, tap, n0);
                    }
                    s_issued = k + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            constexpr uint32_t idesc = idesc_bf16(TC_BM, BN);  // every MMA is M = 128
            int k = 0, t = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
                const int acc = t & 1;
                if (t >= 2 && !mb_wait_f(&tempty[acc], (uint32_t)(((t >> 1) - 1) & 1), fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * ACC);
                for (int j = 0; j < ns; ++j, ++k) {
                    const int s = k % STAGES;
                    if (!mb_wait_f(&full[s], (uint32_t)((k / STAGES) & 1), fail)) {
                        ok = false;
                        break;
                    }
                    s_consumed = k + 1;
                    tc_fence_after();
                    const int g = nk - j * G < G ? nk - j * G : G;
                    for (int u = 0; u < g; ++u) {
                        const uint32_t sa = s_u32(smem + s * S::STAGE + u * S::SUB);
                        const uint64_t bd = kmajor_desc<BKC>(sa + S::A_BYTES);
                        const int i = j * G + u;
#pragma unroll
                        for (int mb = 0; mb < MT; ++mb) {  // the 128-pixel blocks share the W box
                            const uint64_t ad = kmajor_desc<BKC>(sa + mb * S::SUBTILE);
#pragma unroll
                            for (int kk = 0; kk < BKC / 16; ++kk)  // K = 16 is 32 bytes along the swizzled row
                                umma_f16(d + (uint32_t)(mb * BN), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                                         idesc, (i | kk) != 0);
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&tfull[acc]);
            }
            if (!ok) *fail = 1;
            // every MMA issued above has completed before TMEM is released
            umma_commit(drain);
            mb_wait(drain, 0);
        }
    } else {
        // ---- epilogue: this warp's TMEM lane quarter = rows 32 q .. 32 q + 31 of
        // a tile, columns [c_lo, c_lo + BN/2) (the other half: the warp 4 apart)
        const int q = warp & 3;
        const int c_lo = (warp - 2) < 4 ? 0 : BN / 2;
        int t = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
            const int acc = t & 1;
            bool ready = true;
            if (lane == 0) ready = mb_wait_f(&tfull[acc], (uint32_t)((t >> 1) & 1), fail);
            ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
            if (!ready) {
                if (lane == 0) *fail = 1;
                break;
            }
            tc_fence_after();
            const int n0 = (tile % ntn) * BN;
#pragma unroll 1
            for (int mb = 0; mb < MT; ++mb)
#pragma unroll 1
            for (int c = c_lo; c < c_lo + BN / 2; c += 16) {
                const long long m = (long long)(tile / ntn) * BMT + mb * TC_BM + q * 32 + lane;
                const bool mv = m < M;
                float v[16];
                __syncwarp();  // tcgen05.ld is warp-collective
                tmem_ld16(tmem + (uint32_t)(acc * ACC + mb * BN) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
                const int nb = n0 + c;
                if (!mv) continue;
                if (a.bias) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += a.bias[nb + j];
                }
                if (a.skip) {
                    const uint4 *sp = reinterpret_cast<const uint4 *>(a.skip + m * a.N + nb);
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const uint4 w = sp[h2];
                        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 f = __bfloat1622float2(h[e]);
                            v[8 * h2 + 2 * e] += f.x;
                            v[8 * h2 + 2 * e + 1] += f.y;
                        }
                    }
                }
                if (a.out) {
                    uint4 o[2];
                    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
                    for (int e = 0; e < 8; ++e) h[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                    uint4 *dp = reinterpret_cast<uint4 *>(a.out + m * a.N + nb);
                    dp[0] = o[0];
                    dp[1] = o[1];
                    if (a.act) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            h[e] = __halves2bfloat162(silu_bf16(__low2bfloat16(h[e])),
                                                      silu_bf16(__high2bfloat16(h[e])));
                        uint4 *ap = reinterpret_cast<uint4 *>(a.act + m * a.N + nb);
                        ap[0] = o[0];
                        ap[1] = o[1];
                    }
                }
                if (a.outf) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (nb + j < a.nf) a.outf[m * a.nf + nb + j] = v[j];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbarrier_arrive(&tempty[acc]);
        }
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) {
            atomicCAS(err, 0, 1);
            // the boxes that were issued but never waited for by the MMA thread
            for (int k = s_consumed; k < s_issued; ++k) mb_wait(&full[k % STAGES], (uint32_t)((k / STAGES) & 1));
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 2 * ACC);
}

// ---- host side

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> fn{nullptr};
    PFN_cuTensorMapEncodeTiled_v12000 f = fn.load();
    if (!f) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return nullptr;
        f = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        fn.store(f);
    }
    return f;
}

// The tile shape for side R: P pixels (a power of two) as whole rows of
// whole images when R <= P, a P-column piece of one row otherwise (each box
// dimension at most 256).
bool tile_for(int R, int P, TcTile *t) {
    if (R <= 0 || (R & (R - 1)) || P <= 0 || (P & (P - 1))) return false;  // powers of two only
    t->Wx = R < P ? R : P;
    t->Hy = R < P ? (R < P / R ? R : P / R) : 1;
    t->Bn = P / (t->Wx * t->Hy);
    return t->Wx * t->Hy * t->Bn == P && t->Wx <= 256 && t->Hy <= 256 && t->Bn <= 256;
}

// CTAs per SM and ring depth.  One thread issues a CTA's copies and one its
// MMAs, and each ring slot costs them a few hundred cycles of issue and
// barrier latency, so two CTAs per SM (two independent pipelines) run the
// small layers about twice as fast as one CTA with a deeper ring, and a
// slot carries as much work as its shared memory allows: two 32-channel K
// steps (G = 2), or MT = 4 blocks of 128 pixels that share one weight box
// (the 32-output-channel layers).  A ring takes about 104 KB of shared
// memory per CTA (at most 16 slots); a CTA whose two accumulators fill
// the 512 TMEM columns (BN = 256) runs alone on its SM with a 200 KB ring.
constexpr int tc_ctas_per_sm(int acc_cols) { return 2 * acc_cols <= 256 ? 2 : 1; }
constexpr int tc_stages(int stage, int acc_cols) {
    return (tc_ctas_per_sm(acc_cols) == 2 ? 104 : 200) * 1024 / stage < 16
               ? (tc_ctas_per_sm(acc_cols) == 2 ? 104 : 200) * 1024 / stage
               : 16;
}

template <int BN, int BKC, int MT>
cudaError_t launch_bn(const ConvArgs &a, int num_sms, int *err, cudaStream_t st) {
    TcTile tile;
    if (!tile_for(a.R, TC_BM * MT, &tile)) return cudaErrorInvalidValue;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const CUtensorMapSwizzle sw = BKC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap xmap, wmap;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)a.Cx, (cuuint64_t)a.R, (cuuint64_t)a.R, (cuuint64_t)a.B};
        const cuuint64_t strides[3] = {(cuuint64_t)a.Cx * 2, (cuuint64_t)a.R * a.Cx * 2,
                                       (cuuint64_t)a.R * a.R * a.Cx * 2};
        const cuuint32_t box[4] = {(cuuint32_t)BKC, (cuuint32_t)tile.Wx, (cuuint32_t)tile.Hy, (cuuint32_t)tile.Bn};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(a.X), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)a.Cx, 9, (cuuint64_t)a.N};
        const cuuint64_t strides[2] = {(cuuint64_t)a.Cx * 2, (cuuint64_t)9 * a.Cx * 2};
        const cuuint32_t box[3] = {(cuuint32_t)BKC, 1, (cuuint32_t)BN};
        const cuuint32_t es[3] = {1, 1, 1};
        if (enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(a.W), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    // 32-channel chunks (64-byte rows) of single-block tiles go two K steps
    // to a ring slot, so a slot carries the same 64 channels of K as a
    // 128-byte-row slot does
    constexpr int G = (BKC == 32 && MT == 1) ? 2 : 1;
    constexpr int STAGES = tc_stages(G * (TC_BM * MT + BN) * BKC * 2, MT * BN);
    using S = TcSmem<BN, BKC, STAGES, G, MT>;
    auto k = conv_tc_kernel<BN, BKC, STAGES, G, MT>;
    constexpr int smem = S::TOTAL;
    static std::atomic<unsigned long long> configured{0};  // devices whose attribute is set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    const long long mt = ((long long)a.B * a.R * a.R + TC_BM * MT - 1) / (TC_BM * MT);
    const int ntn = a.N / BN;
    const long long ntiles = mt * ntn;
    if (ntiles > (1ll << 30)) return cudaErrorInvalidValue;
    long long grid = (long long)num_sms * tc_ctas_per_sm(MT * BN);
    if (grid > ntiles) grid = ntiles;
    k<<<(unsigned)grid, TC_THREADS, smem, st>>>(xmap, wmap, a, (int)ntiles, ntn, err);
    return cudaGetLastError();
}

template <int BKC>
cudaError_t launch_bkc(const ConvArgs &a, int bn, int mtile, int num_sms, int *err, cudaStream_t st) {
    switch (bn) {
        case 256: return launch_bn<256, BKC, 1>(a, num_sms, err, st);
        case 128: return launch_bn<128, BKC, 1>(a, num_sms, err, st);
        case 64: return launch_bn<64, BKC, 1>(a, num_sms, err, st);
        default:
            if (BKC == 32 && mtile == 4) return launch_bn<32, 32, 4>(a, num_sms, err, st);
            return launch_bn<32, BKC, 1>(a, num_sms, err, st);
    }
}

}  // namespace

bool conv_tc_applies(const ConvArgs &a) {
    TcTile t;
    return tile_for(a.R, TC_BM, &t) && (a.Cx == 32 || a.Cx % 64 == 0) && a.N % 32 == 0 && a.N >= 32 &&
           a.N <= 1024;
}

cudaError_t conv_forward_tc(const ConvArgs &a, int num_sms, int *err, cudaStream_t st) {
    if (!conv_tc_applies(a)) return cudaErrorInvalidValue;
    const long long mt = ((long long)a.B * a.R * a.R + TC_BM - 1) / TC_BM;
    // the widest N tile (each A box read once per N tile) that still gives
    // every SM a tile
    int bn = 32;
    for (int c : {256, 128, 64}) {
        if (a.N % c == 0 && mt * (a.N / c) >= num_sms) {
            bn = c;
            break;
        }
    }
    // 32 output channels from 32 input channels: tiles of four 128-pixel
    // blocks sharing the weight box, while there is at least one such tile
    // for every CTA
    TcTile t4;
    const int mtile = (bn == 32 && a.Cx == 32 && tile_for(a.R, 4 * TC_BM, &t4) && mt >= 4ll * 2 * num_sms) ? 4 : 1;
    return a.Cx == 32 ? launch_bkc<32>(a, bn, mtile, num_sms, err, st)
                      : launch_bkc<64>(a, bn, mtile, num_sms, err, st);
}

}  // namespace mdfnet
