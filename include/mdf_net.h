/* mdf_net.h -- C ABI of the warm-start network in libmdf.so.
 *
 * The paper has no learned component; this network is an extension of the
 * library: it predicts the steady state of a power-law lid-driven cavity
 * (the Sec. 4.4 set-up with a power-law fluid -- named by the paper, the
 * model nu = K gdot^(n-1) is the library's reading -- on the square or a
 * body-fitted trapezoid grid) from its Reynolds number, power-law index and grid
 * geometry, so that the MDF-FDLBM march (mdf_init_fields,
 * mdf_step) can start from that prediction instead of from rest and still
 * converges to the method's own steady state (the network never replaces
 * the solver's result).
 *
 * Network: a 3 x 3 convolutional U-Net on R x R nodes (R divisible by 8),
 * 15 layers (32, 64, 128, 256 channels over four resolutions, SiLU
 * activations, 2 x 2 average pooling, nearest upsampling, additive skip
 * connections), 1,755,619 parameters.  Weights and activations are stored in
 * BF16 and every convolution accumulates in FP32 on the tensor cores
 * (tcgen05 with tensor-memory accumulators; see mdf_net_set_conv_kernel); the
 * master parameters, their gradient and the Adam moments are FP32.
 *
 * Layouts (all row-major, C order):
 *   inputs   [batch][8][R][R] FP32: scaled log Re, scaled n, the node
 *            coordinates x, y and the metric coefficients xi_x, xi_y, eta_x,
 *            eta_y of the cavity's grid (derivatives of the computational
 *            coordinates xi = i/(R-1), eta = j/(R-1) with respect to x, y;
 *            1, 0, 0, 1 on the unit square)
 *   outputs  [batch][3][R][R] FP32: u / u_lid, v / u_lid, p / u_lid^2
 *   targets  as outputs
 *   params   flat FP32, layer by layer: weights [Cout][3][3][Cin] (kernel
 *            row i, column j act on the input at offset (i - 1, j - 1) in
 *            (y, x)), then bias [Cout]
 * Pointers are host memory when on_device == 0, device memory of the
 * network's GPU otherwise.  Calls enqueue on the network's stream; calls with
 * host pointers or a loss output synchronise before returning.
 * Errors: MDF_E_INVALID (bad arguments, before any CUDA call), MDF_E_NOMEM,
 * MDF_E_CUDA; mdf_net_last_error explains.
 */
#ifndef MDF_NET_H
#define MDF_NET_H

#include "mdf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdf_net mdf_net;

/* Network for R x R fields (R >= 8, R % 8 == 0) and batches of at most
 * max_batch samples; parameters start at zero (set them with
 * mdf_net_set_params). */
mdf_status mdf_net_create(int resolution, int max_batch, mdf_net **out);
void mdf_net_destroy(mdf_net *net);
mdf_status mdf_net_set_stream(mdf_net *net, void *cuda_stream);

/* Kernel of the 3 x 3 convolutions (forward and input gradient):
 * kind 0 (default) runs them on the tcgen05 tensor cores -- operands staged
 * in shared memory by TMA, FP32 accumulators in tensor memory -- wherever
 * the resolution of the layer is a power of two, and on the mma.sync kernel
 * otherwise; kind 1 runs every convolution on the mma.sync kernel (the
 * reference point the tcgen05 kernel is measured and tested against).  The
 * weight gradient runs on the mma.sync kernel.  MDF_E_INVALID for another
 * kind. */
mdf_status mdf_net_set_conv_kernel(mdf_net *net, int kind);

/* Number of parameters; layer count and the real (cout, cin) of a layer. */
long long mdf_net_param_count(const mdf_net *net);
int mdf_net_layer_count(const mdf_net *net);
mdf_status mdf_net_layer_shape(const mdf_net *net, int layer, int shape[2]);

/* Copy the parameters in (resets the Adam moments and step count) / out. */
mdf_status mdf_net_set_params(mdf_net *net, const float *params, int on_device);
mdf_status mdf_net_get_params(mdf_net *net, float *params, int on_device);

/* outputs = network(inputs) for `batch` samples. */
mdf_status mdf_net_forward(mdf_net *net, int batch, const float *inputs, float *outputs, int on_device);

/* Mean-square loss against targets and its gradient with respect to the
 * parameters (flat, mdf_net_param_count floats); no update.  loss may be
 * NULL. */
mdf_status mdf_net_gradient(mdf_net *net, int batch, const float *inputs, const float *targets, double *loss,
                            float *grad, int on_device);

/* One Adam step (beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected)
 * with learning rate lr on the mean-square loss of this batch; *loss (may
 * be NULL) receives the loss before the update. */
mdf_status mdf_net_train_step(mdf_net *net, int batch, const float *inputs, const float *targets, double lr,
                              double *loss, int on_device);

const char *mdf_net_last_error(const mdf_net *net); /* NULL: this thread's last failed create */

#ifdef __cplusplus
}
#endif

#endif /* MDF_NET_H */
