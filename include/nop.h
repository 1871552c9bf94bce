/*
 * nop.h -- C ABI of the learned warm start: a small convolutional neural
 * operator that maps the signed distance to the bodies, the Mach number and
 * the Reynolds number of a 2D case to an initial density, velocity and
 * temperature field, trained on steady fields that the solver itself
 * produces.  The converged plain solve remains the judge of the answer: the
 * network only replaces the uniform-flow start (lbm_set_fields), so it can
 * shorten the transient but not change the converged state.
 *
 * The paper has no counterpart of this component (its cases all start from
 * uniform flow, Sec. 3); the network is a production pattern added around
 * the method.
 *
 * Network (U-Net style, four levels, channels c0..c3, all convolutions 3x3
 * with zero padding, stride 1, bias; ReLU after every convolution except the
 * last; 2x2 average pooling down, nearest-neighbour x2 up-sampling, additive
 * skips):
 *   encoder, level l = 0..3 (level l has H/2^l x W/2^l pixels):
 *     a_l = relu(conv(in_l; -> c_l)),  e_l = relu(conv(a_l; c_l -> c_l)),
 *     in_0 = x (in_channels), in_l = pool(e_{l-1}) for l >= 1
 *   decoder, level l = 2, 1, 0 (g_3 = e_3):
 *     s_l = relu(conv(up(g_{l+1}); c_{l+1} -> c_l)),  t_l = s_l + e_l,
 *     g_l = relu(conv(t_l; c_l -> c_l))
 *   output  y = conv(g_0; c_0 -> out_channels)   (no activation)
 * 15 convolutions.  Parameters are one flat FP32 vector, layer after layer in
 * the order above (a_0, e_0, a_1, e_1, a_2, e_2, a_3, e_3, s_2, g_2, s_1,
 * g_1, s_0, g_0, y); layer k holds its weights W[c_out][3][3][c_in]
 * (c_in fastest; tap (ky, kx) multiplies the input pixel (y + ky - 1,
 * x + kx - 1)) followed by its bias b[c_out].
 *
 * Arithmetic: FP32 master weights (Adam moments in FP32); every convolution
 * runs on the tensor cores with BF16 operands (weights and the input
 * activations rounded to BF16 when staged) and FP32 accumulation;
 * activations and gradients are stored in FP32.  Weight gradients are summed
 * over pixels in fixed-size chunks and the chunk partials added in a fixed
 * order, so a training step is bitwise reproducible (no atomics).
 *
 * Tensors are NHWC, FP32, on the device: x[B][H][W][in_channels],
 * y[B][H][W][out_channels], batch-major.  H and W must be multiples of 8.
 *
 * Ownership: the library owns every device buffer of a nop_net; pointers
 * passed in stay owned by the caller and are only read or written during
 * the call (all calls are synchronous with respect to the host unless
 * stated otherwise).  Errors: every call returns an lbm_status (declared in
 * lbmib.h); the text of the last error of a network is returned by
 * nop_last_error.
 */
#ifndef NOP_H
#define NOP_H

#include <stddef.h>

#include "lbmib.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nop_net nop_net;

typedef struct {
  size_t struct_size;  /* sizeof(nop_config) */
  int height, width;   /* grid ny x nx of the cases (multiples of 8) */
  int max_batch;       /* largest batch passed to any call */
  int in_channels;     /* 1..16 (3: signed distance / D, Mach, Re / 200) */
  int out_channels;    /* 1..16 (4: density, two velocity components, temperature) */
  int channels[4];     /* c0..c3, each a multiple of 16 in 16..256 (32, 64, 96, 128) */
  int device;          /* CUDA device ordinal */
  void* stream;        /* cudaStream_t to run on, or NULL for a stream the net creates */
} nop_config;

/* Fill a config with the defaults: 512 x 256 grid (height 256, width 512),
 * max_batch 8, 3 input and 4 output channels, channels 32, 64, 96, 128. */
lbm_status nop_config_default(nop_config* cfg);

/* Create a network on cfg->device with all parameters zero (set them with
 * nop_set_params or nop_init_params).  LBM_EINVAL for an invalid config,
 * LBM_ENOMEM / LBM_ECUDA when the device buffers cannot be allocated. */
lbm_status nop_create(const nop_config* cfg, nop_net** out);
void nop_destroy(nop_net* net);
const char* nop_last_error(const nop_net* net);

/* Number of FP32 parameters (size of the flat vector described above). */
long long nop_param_count(const nop_net* net);

/* He-uniform initialisation of the weights from a seeded counter-based
 * generator (splitmix64 of seed and the parameter index, top 24 bits as a
 * uniform in [0, 1)), biases zero; resets the Adam state. */
lbm_status nop_init_params(nop_net* net, unsigned long long seed);

/* Copy the FP32 parameter vector in or out (nop_param_count floats);
 * is_device selects device or host memory.  Setting the parameters resets
 * the Adam state. */
lbm_status nop_set_params(nop_net* net, int is_device, const float* params);
lbm_status nop_get_params(const nop_net* net, int is_device, float* params);

/* Forward pass: y = net(x) for `batch` samples (device pointers). */
lbm_status nop_forward(nop_net* net, int batch, const float* x, float* y);

/* Forward pass, then the backward pass of a given output gradient dy
 * (device, same layout as y): dparams receives dL/dtheta (nop_param_count
 * floats, device, may be NULL) and dx receives dL/dx (device, same layout
 * as x, may be NULL). */
lbm_status nop_backward(nop_net* net, int batch, const float* x, const float* dy,
                        float* dparams, float* dx);

/* Gradient-check mode (on != 0): the 3x3 convolutions of nop_forward,
 * nop_backward and nop_train_step run on FP32 operands (weights and
 * activations unrounded, FP32 products and fixed-order FP32 sums, CUDA
 * cores) instead of the BF16-operand tensor-core path, so that the
 * gradients can be compared with the FP64 reference backward to 1e-5.
 * Slow; for checks only.  The first call with on != 0 allocates the FP32
 * weight copies (LBM_ENOMEM on failure); on = 0 returns to the BF16 path.
 * No counterpart in the paper (the network is this library's addition). */
lbm_status nop_set_fp32(nop_net* net, int on);

/* One training step on a batch: forward, mean-squared-error loss
 * L = sum (y - target)^2 / (batch H W out_channels), backward, Adam update
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, learning rate lr) of
 * the FP32 master weights.  *loss (host, may be NULL) receives L of the
 * batch before the update, in FP64. */
lbm_status nop_train_step(nop_net* net, int batch, const float* x, const float* target,
                          float lr, double* loss);

/* Warm start of a 2D solver: run the network on one sample x (device,
 * [1][H][W][in_channels]) and set the solver state to the equilibrium of
 * rho = off[0] + scale[0] y_0, u_x = off[1] + scale[1] y_1,
 * u_y = off[2] + scale[2] y_2, T = off[3] + scale[3] y_3 (lbm_set_fields).
 * The solver must be D2Q9 with nx = W, ny = H, and the network must have
 * 4 output channels; LBM_EINVAL otherwise. */
lbm_status nop_infer_into(nop_net* net, lbm_handle* h, const float* x, const double off[4],
                          const double scale[4]);

#ifdef __cplusplus
}
#endif

#endif /* NOP_H */
