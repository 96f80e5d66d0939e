/*
 * unet.h -- C ABI of the learned warm start in liblbm.so: the signed-distance
 * input field and a 3-D convolutional U-Net trained on velocity fields that
 * the LBM of lbm.h produces.
 *
 * The paper has no learned component.  The warm start feeds the LBM a better
 * initial velocity u0 (lbm_init evaluates Eq. (equilibrium) at u0); the
 * converged LBM remains the arbiter of the prediction, so a poor prediction only
 * costs steps, never accuracy.
 *
 * Conventions are those of lbm.h: LBM_* status codes, caller-owned device
 * memory, 256-byte aligned workspaces, calls asynchronous on the bound
 * stream unless they return host values.
 */
#ifndef UNET_H
#define UNET_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Truncated signed distance of a geometry, the network's input: for every
 * cell, the smallest signed distance to a solid surface -- |p - c| - r over
 * every periodic image of every sphere and, when z is not periodic, the
 * distances to the wall planes z = 1 - q_lo and z = nz - 2 + q_hi (negative
 * inside solids) -- divided by trunc and clipped to [-1, 1].
 * dev_out[nz][ny][nx] (float).  The workspace (lbm_sdf_workspace_size bytes)
 * holds the sphere images near each cell.  Synchronises `stream`. */
int lbm_sdf_workspace_size(const lbm_geometry *geom, float trunc, size_t *bytes);
int lbm_sdf(const lbm_geometry *geom, float trunc, void *dev_workspace, size_t bytes, float *dev_out, void *stream);

typedef struct unet_net unet_net;

/* A U-Net for a batch of n fields of nz x ny x nx cells (each divisible by 8).
 * Architecture: two 3x3x3 convolutions + ReLU per level with 16/32/64/128
 * channels, 2x2x2 average pooling down, nearest x2 upsampling up with the skip
 * tensor concatenated after the upsampled one, a 1x1x1 head to 3 channels;
 * convolutions pad circularly in x and y and with zeros in z.  Input channels:
 * [sdf, z in [-1, 1], 14 zeros].  Activations and weight copies are bf16,
 * every contraction accumulates in fp32 on the tensor cores; master weights,
 * gradients and Adam moments are fp32. */
int unet_create(int32_t n, int32_t nz, int32_t ny, int32_t nx, unet_net **out);
void unet_destroy(unet_net *net);

/* Number of fp32 parameters: for each 3x3x3 layer in order (enc1a, enc1b,
 * enc2a, enc2b, enc3a, enc3b, botta, bottb, dec3a, dec3b, dec2a, dec2b, dec1a,
 * dec1b) the weights [27][c_out][c_in] (tap 9(dz+1) + 3(dy+1) + (dx+1)) then
 * the bias [c_out]; then the head weights [3][16] and bias [3]. */
int unet_param_count(const unet_net *net, int64_t *n);

/* Device workspace for activations, gradients, weights and optimiser state. */
int unet_workspace_size(const unet_net *net, size_t *bytes);
int unet_bind(unet_net *net, void *dev_workspace, size_t bytes, void *stream);

/* Copy the fp32 parameter vector in (and refresh the bf16 weight copies) or
 * out; copy the gradients of the last unet_backward out. */
int unet_set_params(unet_net *net, const float *dev_params);
int unet_get_params(unet_net *net, float *dev_params);
int unet_get_grads(unet_net *net, float *dev_grads);

/* Forward pass: dev_sdf[n][nz][ny][nx] -> dev_u[n][3][nz][ny][nx] = out_scale *
 * network output (dev_u may be NULL when only the training state is wanted).
 * With out_scale = g nz^2 / nu the output is a velocity in lattice units for a
 * network trained on targets u nu / (g nz^2). */
int unet_forward(unet_net *net, const float *dev_sdf, float *dev_u, float out_scale);

/* Backward pass of the last forward: loss = mean over all voxels and the 3
 * components of (output - target_scale * dev_target)^2, dev_target laid out
 * like dev_u; accumulates the gradients of every parameter.  *host_loss (may
 * be NULL, else the call synchronises) receives the loss. */
int unet_backward(unet_net *net, const float *dev_target, float target_scale, double *host_loss);

/* One Adam step (Kingma & Ba 2015, bias-corrected) on the fp32 parameters,
 * then refresh of the bf16 weight copies. */
int unet_adam_step(unet_net *net, float lr, float beta1, float beta2, float eps);

/* One 3x3x3 convolution layer as the network runs it (its kernels exposed for
 * checks and per-layer measurements): dev_y[v][o] = bf16(act(bias[o] +
 * sum_t sum_c w[t][o][c] x[v + off_t][c])), act = ReLU when relu != 0, with
 * fp32 accumulation on the tensor cores.  bf16 values are passed as their
 * 16-bit patterns: activations [n][nz][ny][nx][c] (c fastest), weights
 * dev_w[27][co][ci] (tap 9(dz+1) + 3(dy+1) + (dx+1)); dev_bias fp32 [co] or
 * NULL.  Padding is circular in x and y and zero in z.  ci and co are
 * multiples of 16, co <= 256, n nz ny nx < 2^31.  *dev_status (caller-owned,
 * zero on entry) is set to 1 if a bounded device-side wait gave up.
 * Asynchronous on `stream`. */
int unet_conv3d(const uint16_t *dev_x, int32_t ci, const uint16_t *dev_w, const float *dev_bias, uint16_t *dev_y,
                int32_t co, int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t relu, int32_t *dev_status,
                void *stream);

/* Weight gradient of that layer: dev_dw[t][o][c] (fp32) += sum_v
 * dy[v][o] x[v + off_t][c] with the same padding; dy and x bf16 as above.
 * co <= 128 and ci <= 256, multiples of 16.  Partial sums are added with fp32
 * atomics (the order of the additions is not fixed).  Asynchronous. */
int unet_conv3d_wgrad(const uint16_t *dev_dy, int32_t co, const uint16_t *dev_x, int32_t ci, float *dev_dw,
                      int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t *dev_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* UNET_H */
