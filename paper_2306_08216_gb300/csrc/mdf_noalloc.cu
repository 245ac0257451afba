// mdf_noalloc.cu -- residual and momentum drift from caller buffers, with no
// allocation of any kind.
//
// Who needs this: code that runs where device memory may not be allocated --
// under an allocator (a framework's caching allocator, a memory pool sized at
// start-up) that owns all device memory and forbids side allocations, or in a
// real-time loop that must not risk an allocation failure or the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.  Such a caller passes
// its own inputs and outputs; the only scratch this path uses is the
// file-scope array below, which the CUDA loader places in device memory when
// the library is loaded (every GPU that loads the library holds it until the
// process exits).
//
// The reduction is the same FP64 two-pass reduction as mdf_residual, on a
// dense state instead of a context's padded planes, and it leaves the
// caller's snapshot untouched.
#include <mutex>

#include "../../include/mdf.h"
#include "mdf_internal.cuh"

namespace {

// Per-block partial sums: 5 doubles per block, at most kMaxBlocks blocks of
// kThreads threads, each thread folding kPerThread nodes.  This fixes the
// largest accepted field: kMaxBlocks * kThreads * kPerThread nodes
// (4096 x 4096), 160 KiB of device memory.
constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxNodes = (long long)kMaxBlocks * kThreads * kPerThread;

static __device__ __align__(256) double g_partials[kMaxBlocks * 5];

// Device address of g_partials for each device, resolved once per device
// (the first call on that device, with it current).  A device reset
// (cudaDeviceReset) unloads the module, so the cached address is not valid
// afterwards; the header says so.
constexpr int kMaxDevices = 64;
double *g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__global__ void norms_partial_kernel(const float *__restrict__ fhat, const float *__restrict__ u_prev,
                                     const float *__restrict__ v_prev, long long N, double *partials) {
    __shared__ double red[5][kThreads / 32];
    double d2 = 0.0, n2 = 0.0, su = 0.0, sv = 0.0, bad = 0.0;
    const long long base = (long long)blockIdx.x * kThreads * kPerThread + threadIdx.x;
#pragma unroll 4
    for (int k = 0; k < kPerThread; ++k) {
        const long long n = base + (long long)k * kThreads;
        if (n >= N) break;
        float u = 0.0f, v = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            u += fhat[j * N + n];
            v += fhat[(5 + j) * N + n];
        }
        if (!isfinite(u) || !isfinite(v)) bad += 1.0;
        const double du = (double)u - u_prev[n], dv = (double)v - v_prev[n];
        d2 += du * du + dv * dv;
        n2 += (double)u * u + (double)v * v;
        su += u;
        sv += v;
    }
    double vals[5] = {d2, n2, su, sv, bad};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double x = vals[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double x = lane < kThreads / 32 ? red[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) partials[(long long)blockIdx.x * 5 + q] = x;
        }
    }
}

// One block folds the partials in a fixed order and writes
// out = {residual, sum u, sum v, non-finite count}.
__global__ void norms_final_kernel(const double *partials, int nblocks, long long window, double *out) {
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
    if (threadIdx.x == 0) {
        double s[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int q = 0; q < 5; ++q) s[q] += red[q][w];
        out[0] = sqrt(s[0]) / ((double)window * sqrt(s[1]));
        out[1] = s[2];
        out[2] = s[3];
        out[3] = s[4];
    }
}

}  // namespace

extern "C" mdf_status mdf_residual_noalloc(const float *fhat, const float *u_prev, const float *v_prev, int nx,
                                           int ny, long long window, void *cuda_stream, double *out) {
    if (!fhat || !u_prev || !v_prev || !out || nx < 1 || ny < 1 || window < 1) return MDF_E_INVALID;
    const long long N = (long long)nx * ny;
    if (N > kMaxNodes) return MDF_E_INVALID;  // larger than the static scratch serves
    // an error left by an earlier, unrelated call on this thread is not this
    // call's failure: clear it before the launches are checked
    (void)cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MDF_E_CUDA;
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return MDF_E_CUDA;
            g_partials_addr[dev] = static_cast<double *>(p);
        }
        partials = g_partials_addr[dev];
    }
    const int nblocks = (int)((N + (long long)kThreads * kPerThread - 1) / ((long long)kThreads * kPerThread));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    norms_partial_kernel<<<nblocks, kThreads, 0, st>>>(fhat, u_prev, v_prev, N, partials);
    if (cudaGetLastError() != cudaSuccess) return MDF_E_CUDA;
    norms_final_kernel<<<1, 1024, 0, st>>>(partials, nblocks, window, out);
    return cudaGetLastError() == cudaSuccess ? MDF_OK : MDF_E_CUDA;
}
