// net_api.cu -- runtime of the warm-start network behind include/mdf_net.h:
// buffers, the U-Net wiring of the forward and backward passes, Adam.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/mdf_net.h"
#include "net_internal.cuh"

using namespace mdfnet;

namespace {

// Input planes: scaled log Re, scaled n, node coordinates x, y and the
// metric coefficients xi_x, xi_y, eta_x, eta_y (include/mdf_net.h).
constexpr int kInPlanes = NET_IN_PLANES;

struct LayerSpec {
    const char *name;
    int cin, cout, div;  // real channels; resolution R / div
    bool act;
};

// Parameter order; inputs and skips are wired in forward()/backward().
const LayerSpec kLayers[] = {
    {"e0a", kInPlanes, 32, 1, true},     {"e0b", 32, 32, 1, true},    {"e1a", 32, 64, 2, true},
    {"e1b", 64, 64, 2, true},    {"e2a", 64, 128, 4, true},   {"e2b", 128, 128, 4, true},
    {"e3a", 128, 256, 8, true},  {"e3b", 256, 256, 8, true},  {"d2a", 256, 128, 4, true},
    {"d2b", 128, 128, 4, true},  {"d1a", 128, 64, 2, true},   {"d1b", 64, 64, 2, true},
    {"d0a", 64, 32, 1, true},    {"d0b", 32, 32, 1, true},    {"out", 32, 3, 1, false},
};
constexpr int kNL = sizeof(kLayers) / sizeof(kLayers[0]);

inline int pad32(int c) { return (c + 31) / 32 * 32; }

}  // namespace

struct mdf_net {
    int R = 0, Bmax = 0, dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    long long P = 0;
    long long off[kNL];
    int cin_pad[kNL], cout_pad[kNL];
    std::vector<void *> allocs;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wf[kNL], *wb[kNL];
    float *bias[kNL];
    // activations
    bf16 *xin = nullptr, *z[kNL], *y[kNL];
    bf16 *p0 = nullptr, *p1 = nullptr, *p2 = nullptr, *u0 = nullptr, *u1 = nullptr, *u2 = nullptr;
    float *outf = nullptr, *tgt = nullptr, *io = nullptr;
    // gradients
    bf16 *dz[kNL], *dy[kNL];
    bf16 *dp0 = nullptr, *dp1 = nullptr, *dp2 = nullptr, *du0 = nullptr, *du1 = nullptr, *du2 = nullptr;
    double *loss = nullptr, *h_loss = nullptr;
    int *err = nullptr, *h_err = nullptr;  // error word of the tensor-core kernels
    int conv_kind = 0;                     // 0: tcgen05 where it applies, 1: mma.sync
    long long adam_t = 0;
    bool prepared = false;
    char last_error[256] = {0};
};

static thread_local char g_net_error[256] = {0};

static mdf_status nfail(mdf_net *n, mdf_status st, const char *fmt, ...) {
    char *dst = n ? n->last_error : g_net_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

#define NCK(net, call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return nfail(net, e_ == cudaErrorMemoryAllocation ? MDF_E_NOMEM : MDF_E_CUDA,        \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)

template <typename T>
static mdf_status nalloc(mdf_net *n, T **p, size_t count) {
    void *q = nullptr;
    NCK(n, cudaMalloc(&q, count * sizeof(T)));
    try {
        n->allocs.push_back(q);
    } catch (const std::bad_alloc &) {
        cudaFree(q);
        return nfail(n, MDF_E_NOMEM, "host allocation failed");
    }
    *p = static_cast<T *>(q);
    return MDF_OK;
}

static void free_net(mdf_net *n) {
    if (!n) return;
    for (void *p : n->allocs) cudaFree(p);
    if (n->h_loss) cudaFreeHost(n->h_loss);
    if (n->h_err) cudaFreeHost(n->h_err);
    delete n;
}

static long long pix(const mdf_net *n, int B, int div) {
    const long long r = n->R / div;
    return (long long)B * r * r;
}

// Rebuild the BF16 layer weights from the FP32 master parameters.
static mdf_status prepare(mdf_net *n) {
    for (int l = 0; l < kNL; ++l)
        NCK(n, prepare_layer(n->params, n->off[l], kLayers[l].cin, kLayers[l].cout, n->cin_pad[l], n->cout_pad[l],
                             n->wf[l], n->wb[l], n->bias[l], n->stream));
    n->prepared = true;
    return MDF_OK;
}

// One implicit-GEMM convolution on the tcgen05 tensor cores where that
// kernel applies (and is not switched off), else on the mma.sync kernel.
static mdf_status run_conv(mdf_net *n, const ConvArgs &a) {
    if (n->conv_kind == 0 && conv_tc_applies(a)) NCK(n, conv_forward_tc(a, n->num_sms, n->err, n->stream));
    else NCK(n, conv_forward(a, n->stream));
    return MDF_OK;
}

static mdf_status conv(mdf_net *n, int l, int B, const bf16 *x, const bf16 *skip, bf16 *out, float *outf, int nf,
                       bf16 *act = nullptr) {
    ConvArgs a;
    a.X = x;
    a.W = n->wf[l];
    a.bias = n->bias[l];
    a.skip = skip;
    a.out = out;
    a.act = act;
    a.outf = outf;
    a.nf = nf;
    a.B = B;
    a.R = n->R / kLayers[l].div;
    a.Cx = n->cin_pad[l];
    a.N = n->cout_pad[l];
    return run_conv(n, a);
}

// dX of layer l's input from dZ (mirrored weights, no bias).
static mdf_status conv_dx(mdf_net *n, int l, int B, const bf16 *dZ, bf16 *dX) {
    ConvArgs a;
    a.X = dZ;
    a.W = n->wb[l];
    a.bias = nullptr;
    a.skip = nullptr;
    a.out = dX;
    a.act = nullptr;
    a.outf = nullptr;
    a.nf = 0;
    a.B = B;
    a.R = n->R / kLayers[l].div;
    a.Cx = n->cout_pad[l];
    a.N = n->cin_pad[l];
    return run_conv(n, a);
}

static mdf_status wgrad(mdf_net *n, int l, int B, const bf16 *dZ, const bf16 *X) {
    WGradArgs a;
    a.dZ = dZ;
    a.X = X;
    a.g = n->grad;
    a.off = n->off[l];
    a.B = B;
    a.R = n->R / kLayers[l].div;
    a.Cin = n->cin_pad[l];
    a.Cout = n->cout_pad[l];
    a.cin_real = kLayers[l].cin;
    a.cout_real = kLayers[l].cout;
    NCK(n, conv_wgrad(a, n->num_sms, n->stream));
    return MDF_OK;
}

#define NRET(call)                      \
    do {                                \
        mdf_status s_ = (call);         \
        if (s_ != MDF_OK) return s_;    \
    } while (0)

// Layer l with its activation: z = conv(x) + b (+ skip), y = silu(z), the
// activation written by the convolution's epilogue.
static mdf_status layer(mdf_net *n, int l, int B, const bf16 *x, const bf16 *skip) {
    return conv(n, l, B, x, skip, n->z[l], nullptr, 0, n->y[l]);
}

static mdf_status forward(mdf_net *n, int B) {
    if (!n->prepared) NRET(prepare(n));
    const int R = n->R;
    NRET(layer(n, 0, B, n->xin, nullptr));
    NRET(layer(n, 1, B, n->y[0], nullptr));                      // s0
    NCK(n, pool_forward(n->y[1], n->p0, B, R, 32, n->stream));
    NRET(layer(n, 2, B, n->p0, nullptr));
    NRET(layer(n, 3, B, n->y[2], nullptr));                      // s1
    NCK(n, pool_forward(n->y[3], n->p1, B, R / 2, 64, n->stream));
    NRET(layer(n, 4, B, n->p1, nullptr));
    NRET(layer(n, 5, B, n->y[4], nullptr));                      // s2
    NCK(n, pool_forward(n->y[5], n->p2, B, R / 4, 128, n->stream));
    NRET(layer(n, 6, B, n->p2, nullptr));
    NRET(layer(n, 7, B, n->y[6], nullptr));
    NCK(n, up_forward(n->y[7], n->u2, B, R / 8, 256, n->stream));
    NRET(layer(n, 8, B, n->u2, n->y[5]));
    NRET(layer(n, 9, B, n->y[8], nullptr));
    NCK(n, up_forward(n->y[9], n->u1, B, R / 4, 128, n->stream));
    NRET(layer(n, 10, B, n->u1, n->y[3]));
    NRET(layer(n, 11, B, n->y[10], nullptr));
    NCK(n, up_forward(n->y[11], n->u0, B, R / 2, 64, n->stream));
    NRET(layer(n, 12, B, n->u0, n->y[1]));
    NRET(layer(n, 13, B, n->y[12], nullptr));
    return conv(n, 14, B, n->y[13], nullptr, nullptr, n->outf, 3);
}

// dz[l] = silu'(z[l]) dy[l]
static mdf_status act_back(mdf_net *n, int l, int B) {
    NCK(n, silu_backward(n->z[l], n->dy[l], n->dz[l], pix(n, B, kLayers[l].div) * n->cout_pad[l], n->stream));
    return MDF_OK;
}

// Backward pass from dz[14] (dLoss/dout, set by the loss kernel) into grad.
static mdf_status backward(mdf_net *n, int B) {
    const int R = n->R;
    NCK(n, cudaMemsetAsync(n->grad, 0, n->P * sizeof(float), n->stream));
    // output layer and the R-level decoder
    NRET(wgrad(n, 14, B, n->dz[14], n->y[13]));
    NRET(conv_dx(n, 14, B, n->dz[14], n->dy[13]));
    NRET(act_back(n, 13, B));
    NRET(wgrad(n, 13, B, n->dz[13], n->y[12]));
    NRET(conv_dx(n, 13, B, n->dz[13], n->dy[12]));
    NRET(act_back(n, 12, B));
    NRET(wgrad(n, 12, B, n->dz[12], n->u0));
    NRET(conv_dx(n, 12, B, n->dz[12], n->du0));
    NCK(n, up_backward(n->du0, n->dy[11], B, R / 2, 64, n->stream));
    // R/2 decoder
    NRET(act_back(n, 11, B));
    NRET(wgrad(n, 11, B, n->dz[11], n->y[10]));
    NRET(conv_dx(n, 11, B, n->dz[11], n->dy[10]));
    NRET(act_back(n, 10, B));
    NRET(wgrad(n, 10, B, n->dz[10], n->u1));
    NRET(conv_dx(n, 10, B, n->dz[10], n->du1));
    NCK(n, up_backward(n->du1, n->dy[9], B, R / 4, 128, n->stream));
    // R/4 decoder
    NRET(act_back(n, 9, B));
    NRET(wgrad(n, 9, B, n->dz[9], n->y[8]));
    NRET(conv_dx(n, 9, B, n->dz[9], n->dy[8]));
    NRET(act_back(n, 8, B));
    NRET(wgrad(n, 8, B, n->dz[8], n->u2));
    NRET(conv_dx(n, 8, B, n->dz[8], n->du2));
    NCK(n, up_backward(n->du2, n->dy[7], B, R / 8, 256, n->stream));
    // bottleneck
    NRET(act_back(n, 7, B));
    NRET(wgrad(n, 7, B, n->dz[7], n->y[6]));
    NRET(conv_dx(n, 7, B, n->dz[7], n->dy[6]));
    NRET(act_back(n, 6, B));
    NRET(wgrad(n, 6, B, n->dz[6], n->p2));
    NRET(conv_dx(n, 6, B, n->dz[6], n->dp2));
    // encoder R/4: s2 receives the pooled path and the skip of d2a
    NCK(n, pool_backward(n->dp2, n->dy[5], B, R / 4, 128, n->stream));
    NCK(n, add_inplace(n->dy[5], n->dz[8], pix(n, B, 4) * 128, n->stream));
    NRET(act_back(n, 5, B));
    NRET(wgrad(n, 5, B, n->dz[5], n->y[4]));
    NRET(conv_dx(n, 5, B, n->dz[5], n->dy[4]));
    NRET(act_back(n, 4, B));
    NRET(wgrad(n, 4, B, n->dz[4], n->p1));
    NRET(conv_dx(n, 4, B, n->dz[4], n->dp1));
    // encoder R/2
    NCK(n, pool_backward(n->dp1, n->dy[3], B, R / 2, 64, n->stream));
    NCK(n, add_inplace(n->dy[3], n->dz[10], pix(n, B, 2) * 64, n->stream));
    NRET(act_back(n, 3, B));
    NRET(wgrad(n, 3, B, n->dz[3], n->y[2]));
    NRET(conv_dx(n, 3, B, n->dz[3], n->dy[2]));
    NRET(act_back(n, 2, B));
    NRET(wgrad(n, 2, B, n->dz[2], n->p0));
    NRET(conv_dx(n, 2, B, n->dz[2], n->dp0));
    // encoder R
    NCK(n, pool_backward(n->dp0, n->dy[1], B, R, 32, n->stream));
    NCK(n, add_inplace(n->dy[1], n->dz[12], pix(n, B, 1) * 32, n->stream));
    NRET(act_back(n, 1, B));
    NRET(wgrad(n, 1, B, n->dz[1], n->y[0]));
    NRET(conv_dx(n, 1, B, n->dz[1], n->dy[0]));
    NRET(act_back(n, 0, B));
    return wgrad(n, 0, B, n->dz[0], n->xin);
}

// Wait for the stream; a tensor-core kernel that gave up waiting for its
// copies or MMAs left a nonzero error word, reported here (and cleared).
static mdf_status wait(mdf_net *n) {
    NCK(n, cudaMemcpyAsync(n->h_err, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    if (*n->h_err) {
        *n->h_err = 0;
        NCK(n, cudaMemsetAsync(n->err, 0, sizeof(int), n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
        return nfail(n, MDF_E_CUDA, "a tensor-core convolution gave up waiting for its copies or MMAs");
    }
    return MDF_OK;
}

// Stage inputs (and targets) of `batch` samples.
static mdf_status stage(mdf_net *n, int B, const float *inputs, const float *targets, int on_device) {
    const long long RR = (long long)n->R * n->R;
    const float *in = inputs, *tg = targets;
    if (!on_device) {
        NCK(n, cudaMemcpyAsync(n->io, inputs, (size_t)B * kInPlanes * RR * sizeof(float), cudaMemcpyHostToDevice,
                               n->stream));
        in = n->io;
        if (targets) {
            NCK(n, cudaMemcpyAsync(n->io + (size_t)B * kInPlanes * RR, targets, (size_t)B * 3 * RR * sizeof(float),
                                   cudaMemcpyHostToDevice, n->stream));
            tg = n->io + (size_t)B * kInPlanes * RR;
        }
    }
    NCK(n, pack_input(in, n->xin, B, n->R, n->stream));
    if (tg) NCK(n, pack_target(tg, n->tgt, B, n->R, n->stream));
    return MDF_OK;
}

static mdf_status check_batch(mdf_net *n, int batch, const void *a, const void *b) {
    if (batch < 1 || batch > n->Bmax) return nfail(n, MDF_E_INVALID, "batch must be in [1, %d]", n->Bmax);
    if (!a || !b) return nfail(n, MDF_E_INVALID, "array arguments are required");
    return MDF_OK;
}

extern "C" {

mdf_status mdf_net_create(int resolution, int max_batch, mdf_net **out) {
    if (!out) return nfail(nullptr, MDF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (resolution < 8 || resolution % 8) return nfail(nullptr, MDF_E_INVALID, "resolution must be a multiple of 8");
    if (max_batch < 1 || (long long)max_batch * resolution * resolution > (1ll << 28))
        return nfail(nullptr, MDF_E_INVALID, "max_batch must be >= 1 and max_batch R^2 <= 2^28");
    // host allocations never throw across the C ABI
    mdf_net *n = new (std::nothrow) mdf_net();
    if (!n) return nfail(nullptr, MDF_E_NOMEM, "host allocation of the network failed");
    n->R = resolution;
    n->Bmax = max_batch;
#define NCKC(call)                                       \
    do {                                                 \
        mdf_status s_ = (call);                          \
        if (s_ != MDF_OK) {                              \
            strncpy(g_net_error, n->last_error, 255);    \
            free_net(n);                                 \
            return s_;                                   \
        }                                                \
    } while (0)
#define NCKE(call) NCKC(([&]() -> mdf_status { NCK(n, call); return MDF_OK; })())
    NCKE(cudaGetDevice(&n->dev));
    NCKE(cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, n->dev));
    long long off = 0;
    for (int l = 0; l < kNL; ++l) {
        n->off[l] = off;
        off += (long long)kLayers[l].cout * 9 * kLayers[l].cin + kLayers[l].cout;
        n->cin_pad[l] = pad32(kLayers[l].cin);
        n->cout_pad[l] = pad32(kLayers[l].cout);
    }
    n->P = off;
    NCKC(nalloc(n, &n->params, n->P));
    NCKC(nalloc(n, &n->grad, n->P));
    NCKC(nalloc(n, &n->m, n->P));
    NCKC(nalloc(n, &n->v, n->P));
    NCKE(cudaMemset(n->params, 0, n->P * sizeof(float)));
    NCKE(cudaMemset(n->m, 0, n->P * sizeof(float)));
    NCKE(cudaMemset(n->v, 0, n->P * sizeof(float)));
    const int B = max_batch;
    for (int l = 0; l < kNL; ++l) {
        const size_t w = (size_t)n->cout_pad[l] * 9 * n->cin_pad[l];
        NCKC(nalloc(n, &n->wf[l], w));
        NCKC(nalloc(n, &n->wb[l], w));
        NCKC(nalloc(n, &n->bias[l], (size_t)n->cout_pad[l]));
        const size_t act = (size_t)pix(n, B, kLayers[l].div) * n->cout_pad[l];
        NCKC(nalloc(n, &n->z[l], act));
        NCKC(nalloc(n, &n->dz[l], act));
        n->y[l] = n->dy[l] = nullptr;
        if (kLayers[l].act) {
            NCKC(nalloc(n, &n->y[l], act));
            NCKC(nalloc(n, &n->dy[l], act));
        }
    }
    const int R = resolution;
    NCKC(nalloc(n, &n->xin, (size_t)pix(n, B, 1) * 32));
    NCKC(nalloc(n, &n->p0, (size_t)pix(n, B, 2) * 32));
    NCKC(nalloc(n, &n->p1, (size_t)pix(n, B, 4) * 64));
    NCKC(nalloc(n, &n->p2, (size_t)pix(n, B, 8) * 128));
    NCKC(nalloc(n, &n->dp0, (size_t)pix(n, B, 2) * 32));
    NCKC(nalloc(n, &n->dp1, (size_t)pix(n, B, 4) * 64));
    NCKC(nalloc(n, &n->dp2, (size_t)pix(n, B, 8) * 128));
    NCKC(nalloc(n, &n->u2, (size_t)pix(n, B, 4) * 256));
    NCKC(nalloc(n, &n->u1, (size_t)pix(n, B, 2) * 128));
    NCKC(nalloc(n, &n->u0, (size_t)pix(n, B, 1) * 64));
    NCKC(nalloc(n, &n->du2, (size_t)pix(n, B, 4) * 256));
    NCKC(nalloc(n, &n->du1, (size_t)pix(n, B, 2) * 128));
    NCKC(nalloc(n, &n->du0, (size_t)pix(n, B, 1) * 64));
    NCKC(nalloc(n, &n->outf, (size_t)pix(n, B, 1) * 3));
    NCKC(nalloc(n, &n->tgt, (size_t)pix(n, B, 1) * 3));
    NCKC(nalloc(n, &n->io, (size_t)pix(n, B, 1) * (kInPlanes + 3)));
    NCKC(nalloc(n, &n->loss, 1));
    NCKE(cudaMallocHost(&n->h_loss, sizeof(double)));
    NCKC(nalloc(n, &n->err, 1));
    NCKE(cudaMemset(n->err, 0, sizeof(int)));
    NCKE(cudaMallocHost(&n->h_err, sizeof(int)));
    *n->h_err = 0;
    (void)R;
    *out = n;
    return MDF_OK;
#undef NCKE
#undef NCKC
}

void mdf_net_destroy(mdf_net *n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    free_net(n);
}

mdf_status mdf_net_set_stream(mdf_net *n, void *stream) {
    if (!n) return MDF_E_INVALID;
    n->stream = (cudaStream_t)stream;
    return MDF_OK;
}

mdf_status mdf_net_set_conv_kernel(mdf_net *n, int kind) {
    if (!n) return MDF_E_INVALID;
    if (kind != 0 && kind != 1) return nfail(n, MDF_E_INVALID, "kind must be 0 (tcgen05) or 1 (mma.sync)");
    n->conv_kind = kind;
    return MDF_OK;
}

long long mdf_net_param_count(const mdf_net *n) { return n ? n->P : -1; }
int mdf_net_layer_count(const mdf_net *n) { return n ? kNL : -1; }

mdf_status mdf_net_layer_shape(const mdf_net *n, int layer, int shape[2]) {
    if (!n || !shape || layer < 0 || layer >= kNL) return MDF_E_INVALID;
    shape[0] = kLayers[layer].cout;
    shape[1] = kLayers[layer].cin;
    return MDF_OK;
}

mdf_status mdf_net_set_params(mdf_net *n, const float *params, int on_device) {
    if (!n || !params) return n ? nfail(n, MDF_E_INVALID, "params is NULL") : MDF_E_INVALID;
    NCK(n, cudaMemcpyAsync(n->params, params, n->P * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream));
    NCK(n, cudaMemsetAsync(n->m, 0, n->P * sizeof(float), n->stream));
    NCK(n, cudaMemsetAsync(n->v, 0, n->P * sizeof(float), n->stream));
    n->adam_t = 0;
    NRET(prepare(n));
    return on_device ? MDF_OK : wait(n);
}

mdf_status mdf_net_get_params(mdf_net *n, float *params, int on_device) {
    if (!n || !params) return n ? nfail(n, MDF_E_INVALID, "params is NULL") : MDF_E_INVALID;
    NCK(n, cudaMemcpyAsync(params, n->params, n->P * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
    return on_device ? MDF_OK : wait(n);
}

mdf_status mdf_net_forward(mdf_net *n, int batch, const float *inputs, float *outputs, int on_device) {
    if (!n) return MDF_E_INVALID;
    NRET(check_batch(n, batch, inputs, outputs));
    NRET(stage(n, batch, inputs, nullptr, on_device));
    NRET(forward(n, batch));
    const long long RR = (long long)n->R * n->R;
    float *dst = on_device ? outputs : n->io;
    NCK(n, unpack_output(n->outf, dst, batch, n->R, n->stream));
    if (on_device) return MDF_OK;
    NCK(n, cudaMemcpyAsync(outputs, n->io, (size_t)batch * 3 * RR * sizeof(float), cudaMemcpyDeviceToHost,
                           n->stream));
    return wait(n);
}

static mdf_status loss_and_backward(mdf_net *n, int batch, const float *inputs, const float *targets,
                                    int on_device) {
    NRET(stage(n, batch, inputs, targets, on_device));
    NRET(forward(n, batch));
    NCK(n, mse_loss(n->outf, n->tgt, n->dz[14], n->loss, batch, n->R, n->stream));
    return backward(n, batch);
}

mdf_status mdf_net_gradient(mdf_net *n, int batch, const float *inputs, const float *targets, double *loss,
                            float *grad, int on_device) {
    if (!n) return MDF_E_INVALID;
    NRET(check_batch(n, batch, inputs, targets));
    if (!grad) return nfail(n, MDF_E_INVALID, "grad is NULL");
    NRET(loss_and_backward(n, batch, inputs, targets, on_device));
    NCK(n, cudaMemcpyAsync(grad, n->grad, n->P * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
    if (loss) NCK(n, cudaMemcpyAsync(n->h_loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    if (!on_device || loss) NRET(wait(n));
    if (loss) *loss = *n->h_loss;
    return MDF_OK;
}

mdf_status mdf_net_train_step(mdf_net *n, int batch, const float *inputs, const float *targets, double lr,
                              double *loss, int on_device) {
    if (!n) return MDF_E_INVALID;
    NRET(check_batch(n, batch, inputs, targets));
    if (!(lr > 0 && isfinite(lr))) return nfail(n, MDF_E_INVALID, "lr must be > 0");
    NRET(loss_and_backward(n, batch, inputs, targets, on_device));
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    ++n->adam_t;
    const double c1 = 1.0 - pow(b1, (double)n->adam_t), c2 = 1.0 - pow(b2, (double)n->adam_t);
    NCK(n, adam_step(n->params, n->m, n->v, n->grad, n->P, (float)(lr * sqrt(c2) / c1), (float)b1, (float)b2,
                     (float)(eps * sqrt(c2)), n->stream));
    NRET(prepare(n));
    if (loss) {
        NCK(n, cudaMemcpyAsync(n->h_loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        NRET(wait(n));
        *loss = *n->h_loss;
    } else if (!on_device) {
        NRET(wait(n));
    }
    return MDF_OK;
}

const char *mdf_net_last_error(const mdf_net *n) { return n ? n->last_error : g_net_error; }

}  // extern "C"
