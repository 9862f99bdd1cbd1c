/* sgn_unet.h - a small periodic U-Net for the learned GMRES initial guess.
 *
 * The network maps coarse samples of a stage state to a correction of the
 * GMRES starting value for sigma (Section 3: GMRES is started from the last
 * computed sigma; the learned correction improves that start and every solve
 * still meets the same tolerance). Fixed architecture, all convolutions
 * periodic (the domain is a torus), NCHW layout, batch B:
 *
 *   in  [B][4][n][n]   (channels as the caller defines them)
 *   e0  conv3x3 4->16, ReLU;  s0 conv3x3 16->16, ReLU          n x n
 *   p0  2x2 average pool                                        n/2
 *   e1  conv3x3 16->32, ReLU; s1 conv3x3 32->32, ReLU          n/2
 *   p1  2x2 average pool                                        n/4
 *   b0  conv3x3 32->32, ReLU; b1 conv3x3 32->32, ReLU          n/4
 *   u1  nearest 2x upsample of b1, concat s1 -> 64 channels     n/2
 *   d1  conv3x3 64->32, ReLU                                    n/2
 *   u0  nearest 2x upsample of d1, concat s0 -> 48 channels     n
 *   d0  conv3x3 48->16, ReLU                                    n
 *   out conv1x1 16->1 (linear)                                  n
 *
 * Activations are stored in BF16 (act_bf16 = 1) or FP32 (0, used to check
 * gradients against the CPU oracle); weights, accumulation, gradients and the
 * Adam moments are FP32. Parameters are one contiguous FP32 array: for each
 * layer in the order above its weights [Co][Ci][k][k], then its biases [Co].
 *
 * All pointers are device pointers unless stated. Calls are asynchronous on
 * the network's stream (sgn_unet_set_stream) except where they return a host
 * value. Errors: SGN_EINVAL for bad sizes or NULL pointers, SGN_ECUDA for
 * CUDA errors (message in sgn_unet_last_error), SGN_ENOMEM in create.
 */
#ifndef SGN_UNET_H
#define SGN_UNET_H

#include "sgn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgn_unet_ctx* sgn_unet_t;

/* n: coarse grid side, a power of two in [16, 512]; max_batch >= 1. Allocates
 * parameters (Kaiming-uniform initialised from seed), gradients, Adam moments
 * and the activations of max_batch samples. */
sgn_status sgn_unet_create(int n, int max_batch, int act_bf16, unsigned long long seed, sgn_unet_t* out);
sgn_status sgn_unet_destroy(sgn_unet_t net);
sgn_status sgn_unet_set_stream(sgn_unet_t net, void* cuda_stream);
const char* sgn_unet_last_error(sgn_unet_t net);

/* number of FP32 parameters */
long long sgn_unet_num_params(sgn_unet_t net);
/* the coarse grid side n the network was created for (-1 for NULL) */
int sgn_unet_side(sgn_unet_t net);
/* copy all parameters from / to a device FP32 array of sgn_unet_num_params entries */
sgn_status sgn_unet_set_params(sgn_unet_t net, const float* params);
sgn_status sgn_unet_get_params(sgn_unet_t net, float* params);
/* copy the gradients of the last sgn_unet_backward to a device FP32 array */
sgn_status sgn_unet_get_grads(sgn_unet_t net, float* grads);

/* out[B][1][n][n] = net(in[B][4][n][n]), 1 <= B <= max_batch; out may be
 * NULL. Keeps the activations, and the pointer in (which must stay valid), for
 * sgn_unet_backward. */
sgn_status sgn_unet_forward(sgn_unet_t net, const float* in, float* out, int batch);

/* after sgn_unet_forward with the same batch: loss = mean((out - target)^2)
 * over B n^2 values (written to *loss_dev, a device double; may be NULL) and
 * the gradients of that loss with respect to every parameter (overwritten). */
sgn_status sgn_unet_backward(sgn_unet_t net, const float* target, double* loss_dev);

/* Adam (Kingma & Ba) on the current gradients, step t >= 1 for the bias
 * correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
sgn_status sgn_unet_adam_step(sgn_unet_t net, float lr, float beta1, float beta2, float eps, int t);

#ifdef __cplusplus
}
#endif

#endif /* SGN_UNET_H */
