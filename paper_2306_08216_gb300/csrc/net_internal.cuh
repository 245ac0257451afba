// net_internal.cuh -- kernels of the warm-start network (a 3 x 3
// convolutional U-Net, BF16 storage, FP32 accumulation on the tensor cores)
// and their launchers.  Not part of the public C ABI (include/mdf_net.h).
//
// Activations are NHWC: [B][R][R][C] BF16, C a multiple of 32.  Weights of a
// layer are kept as BF16 [Cout][9][Cin] (forward; tap t = 3 i + j is kernel
// row i, column j: input offset (i - 1, j - 1) in (y, x)) and as BF16
// [Cin][9][Cout] with the tap mirrored (8 - t) for the input gradient.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdfnet {

typedef __nv_bfloat16 bf16;

// Input planes of the network (include/mdf_net.h).
#define NET_IN_PLANES 8

// SiLU(z) = z / (1 + exp(-z)) of a BF16 value, rounded to BF16: the same
// expression in the elementwise kernels and in the convolution epilogues
// that fuse it, so both give the same bits.  The exponential and the
// reciprocal are the fast approximate ones (relative error near 1e-7,
// far below the BF16 rounding of the result).
__device__ __forceinline__ float net_sigmoid(float z) { return __frcp_rn(1.0f + __expf(-z)); }
__device__ __forceinline__ __nv_bfloat16 silu_bf16(__nv_bfloat16 zb) {
    const float v = __bfloat162float(zb);
    return __float2bfloat16_rn(v * net_sigmoid(v));
}

// out[m][n] = sum_k A[m][k] W[n][k] (+ bias[n]) (+ skip[m][n]) over
// k = (tap, c), A[m][(tap, c)] = X[pixel m shifted by tap][c] (zero outside):
// the forward convolution (X = activations, W = [Cout][9][Cin]) and the input
// gradient (X = output gradient, W = mirrored [Cin][9][Cout]).
struct ConvArgs {
    const bf16 *X;      // [B][R][R][Cx], Cx % 32 == 0
    const bf16 *W;      // [N][9][Cx]
    const float *bias;  // [N] or null
    const bf16 *skip;   // [B][R][R][N] or null
    bf16 *out;          // [B][R][R][N] (N % 2 == 0), or null if outf is set
    bf16 *act;          // SiLU of the BF16-rounded out, [B][R][R][N], or null
    float *outf;        // FP32 output [B][R][R][nf] of the first nf channels, or null
    int nf;
    int B, R, Cx, N;
};
cudaError_t conv_forward(const ConvArgs &a, cudaStream_t st);
// The same product on the tcgen05 tensor cores (net_tc.cu): TMA-staged
// operands, FP32 accumulator in tensor memory.  Applies when R is a power of
// two, Cx is 32 or a multiple of 64 and N a multiple of 32; a CTA that gives
// up waiting sets *err to a nonzero value (device memory).
bool conv_tc_applies(const ConvArgs &a);
cudaError_t conv_forward_tc(const ConvArgs &a, int num_sms, int *err, cudaStream_t st);

// Weight and bias gradients of one layer, accumulated (atomic FP32) into the
// flat parameter-gradient vector: g[off + (co * 9 + tap) * cin_real + ci]
// += sum_m dZ[m][co] X[m shifted by tap][ci] for co < cout_real,
// ci < cin_real, and g[off + cout_real * 9 * cin_real + co] += sum_m dZ[m][co].
struct WGradArgs {
    const bf16 *dZ;  // [B][R][R][Cout]
    const bf16 *X;   // [B][R][R][Cin]
    float *g;
    long long off;
    int B, R, Cin, Cout, cin_real, cout_real;
};
cudaError_t conv_wgrad(const WGradArgs &a, int num_sms, cudaStream_t st);

// Elementwise / layout kernels (n = element count unless stated).
cudaError_t silu_forward(const bf16 *z, bf16 *y, long long n, cudaStream_t st);
cudaError_t silu_backward(const bf16 *z, const bf16 *dy, bf16 *dz, long long n, cudaStream_t st);
cudaError_t pool_forward(const bf16 *x, bf16 *y, int B, int R, int C, cudaStream_t st);    // R = input side
cudaError_t pool_backward(const bf16 *dy, bf16 *dx, int B, int R, int C, cudaStream_t st); // dx = ...
cudaError_t up_forward(const bf16 *x, bf16 *y, int B, int R, int C, cudaStream_t st);      // R = input side
cudaError_t up_backward(const bf16 *dy, bf16 *dx, int B, int R, int C, cudaStream_t st);
cudaError_t add_inplace(bf16 *dst, const bf16 *src, long long n, cudaStream_t st);
// planar FP32 [B][NET_IN_PLANES][R][R] -> NHWC BF16 [B][R][R][32] (zero
// channels NET_IN_PLANES..31)
cudaError_t pack_input(const float *in, bf16 *x, int B, int R, cudaStream_t st);
// NHWC FP32 [B][R][R][3] <-> planar FP32 [B][3][R][R]
cudaError_t unpack_output(const float *o, float *out, int B, int R, cudaStream_t st);
cudaError_t pack_target(const float *t, float *o, int B, int R, cudaStream_t st);
// loss = mean (o - t)^2 (FP64 accumulation into *loss, zeroed here) and
// dOut = 2 (o - t) / count as NHWC BF16 [B][R][R][32] (zero channels 3..31)
cudaError_t mse_loss(const float *o, const float *t, bf16 *dout, double *loss, int B, int R, cudaStream_t st);
// Layer weights from the flat FP32 parameter vector: forward BF16
// [cout_pad][9][cin_pad], mirrored BF16 [cin_pad][9][cout_pad] (may be null)
// and FP32 bias [cout_pad], zero in the padding.
cudaError_t prepare_layer(const float *params, long long off, int cin_real, int cout_real, int cin_pad,
                          int cout_pad, bf16 *wf, bf16 *wb, float *bias, cudaStream_t st);
// Adam on the flat vector: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr_t m / (sqrt(v) + eps_t) with the bias-corrected step folded into
// lr_t and eps_t.
cudaError_t adam_step(float *p, float *m, float *v, const float *g, long long n, float lr_t, float b1, float b2,
                      float eps_t, cudaStream_t st);

}  // namespace mdfnet
