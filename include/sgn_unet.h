/* sgn_unet.h - a periodic U-Net for the learned GMRES initial guess.
 *
 * The network maps coarse samples of a stage state to a correction of the
 * GMRES starting value for sigma (Section 3: GMRES is started from the last
 * computed sigma; the learned correction improves that start and every solve
 * still meets the same tolerance). All convolutions are periodic (the domain
 * is a torus). Depth D (resolution levels, 2..6) and widths w[0..D-1] are set
 * at creation; on an n x n input, level l works on the (n / 2^l)^2 grid:
 *
 *   in  [B][4][n][n]   (channels as the caller defines them)
 *   for l = 0 .. D-2:  e_l conv3x3 (l ? w_{l-1} : 4) -> w_l, ReLU
 *                      s_l conv3x3 w_l -> w_l, ReLU
 *                      2x2 average pool of s_l (to level l+1)
 *   level D-1:         b0 conv3x3 w_{D-2} -> w_{D-1}, ReLU; b1 w_{D-1} -> w_{D-1}, ReLU
 *   for l = D-2 .. 0:  nearest 2x upsample of the level below, concatenated
 *                      (upsampled channels first) with s_l;
 *                      d_l conv3x3 w_{l+1} + w_l -> w_l, ReLU
 *   out conv1x1 w_0 -> 1 (linear)
 *
 * sgn_unet_create makes D = 3, w = (16, 32, 32) (60,705 parameters);
 * D = 4, w = (32, 64, 64, 96) has 471,873.
 *
 * Training (sgn_unet_forward / sgn_unet_backward / sgn_unet_adam_step) runs
 * on CUDA cores with activations stored in BF16 (act_bf16 = 1) or FP32 (0,
 * used to check gradients against the CPU oracle); weights, accumulation,
 * gradients and the Adam moments are FP32. Inference (sgn_unet_infer) runs
 * the 3x3 layers after the first as BF16 tensor-core GEMMs (FP32
 * accumulation) over BF16 activations. Parameters are one contiguous FP32
 * array: for each layer in the order above (e_0, s_0, ..., b0, b1,
 * d_{D-2}, ..., d_0, out) its weights [Co][Ci][k][k], then its biases [Co].
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

/* n: coarse grid side, a power of two in [16, 512]; 1 <= max_batch <= 64.
 * Allocates parameters (Kaiming-uniform initialised from seed), gradients,
 * Adam moments and the activations of max_batch samples. The default network,
 * D = 3, w = (16, 32, 32). */
sgn_status sgn_unet_create(int n, int max_batch, int act_bf16, unsigned long long seed, sgn_unet_t* out);
/* any depth 2 <= levels <= 6 and widths (host array of levels entries, each a
 * multiple of 16 in [16, 256]); n / 2^(levels-1) >= 4. */
sgn_status sgn_unet_create_arch(int n, int max_batch, int act_bf16, unsigned long long seed, int levels,
                                const int* widths, sgn_unet_t* out);
sgn_status sgn_unet_destroy(sgn_unet_t net);
sgn_status sgn_unet_set_stream(sgn_unet_t net, void* cuda_stream);
const char* sgn_unet_last_error(sgn_unet_t net);

/* number of FP32 parameters */
long long sgn_unet_num_params(sgn_unet_t net);
/* the coarse grid side n the network was created for (-1 for NULL) */
int sgn_unet_side(sgn_unet_t net);
/* depth D, and the width of a level (-1 for NULL or a level out of range) */
int sgn_unet_levels(sgn_unet_t net);
int sgn_unet_width(sgn_unet_t net, int level);
/* copy all parameters from / to a device FP32 array of sgn_unet_num_params entries */
sgn_status sgn_unet_set_params(sgn_unet_t net, const float* params);
sgn_status sgn_unet_get_params(sgn_unet_t net, float* params);
/* copy the gradients of the last sgn_unet_backward to a device FP32 array */
sgn_status sgn_unet_get_grads(sgn_unet_t net, float* grads);

/* out[B][1][n][n] = net(in[B][4][n][n]), 1 <= B <= max_batch; out may be
 * NULL. Keeps the activations, and the pointer in (which must stay valid), for
 * sgn_unet_backward. */
sgn_status sgn_unet_forward(sgn_unet_t net, const float* in, float* out, int batch);

/* out[B][1][n][n] = net(in[B][4][n][n]) on the tensor cores, 1 <= B <=
 * max_batch: the first layer in FP32 on CUDA cores, every later 3x3 layer a
 * BF16 implicit GEMM with FP32 accumulation (weights rounded to BF16 from the
 * current parameters at each call), activations stored in BF16, the 1x1
 * output layer in FP32. Keeps nothing for sgn_unet_backward. Launches only
 * (no synchronisation, no allocation): it may be captured in a CUDA graph. */
sgn_status sgn_unet_infer(sgn_unet_t net, const float* in, float* out, int batch);

/* synchronises the network's stream and reports whether an sgn_unet_infer
 * since the last check gave up waiting for the tensor cores or the copy
 * engine (bounded waits of about a second): SGN_ECUDA then (the outputs of
 * those calls are not valid; the flag is cleared), SGN_OK otherwise. */
sgn_status sgn_unet_check(sgn_unet_t net);

/* One periodic 3x3 convolution + bias + ReLU on the tensor cores, the
 * building block of sgn_unet_infer: for every pixel (b, y, x) of a
 * batch x H x W grid and output channel o,
 *   out[b][y][x][o] = bf16(max(0, bias[o] + sum_{c, ky, kx} bf16(weight[o][c][ky][kx])
 *                                    in[b][(y + ky - 1) mod H][(x + kx - 1) mod W][c]))
 * with FP32 accumulation, where the input channels c < C0 come from src0 and
 * the next C1 from src1 (NHWC BF16, row lengths C0 and C1); with up0, src0 is
 * on the H/2 x W/2 grid and read at (y / 2, x / 2) (nearest upsampling).
 * H, W powers of two (>= 4 with up0); C0 and C1 multiples of 16 (C1 may be
 * 0, then src1 may be NULL), C0 + C1 <= 1024; Co a multiple of 16 in
 * [16, 256]. weight [Co][C0 + C1][3][3] and bias [Co] are FP32 device arrays;
 * out is NHWC BF16 [batch][H][W][Co]; workspace is a device buffer of at
 * least sgn_conv3_workspace_bytes(C0 + C1, Co) bytes (16-byte aligned; it
 * receives the BF16 weights). Synchronous on stream (NULL: the default
 * stream): SGN_ECUDA also when a bounded wait of the kernel ran out. */
sgn_status sgn_conv3_relu_bf16(int batch, int H, int W, const void* src0, int C0, int up0, const void* src1, int C1,
                               const float* weight, const float* bias, int Co, void* out, void* workspace,
                               size_t workspace_bytes, void* stream);
size_t sgn_conv3_workspace_bytes(int Ci, int Co);

/* Self-test of the tensor-core kernels' bounded waits (both kernels, a
 * 16 -> 16 channel layer on 8 x 8 and on 4 x 128 zeros): one launch whose
 * weight barrier is armed for 16 bytes more than its copy delivers, so that
 * the phase never completes, must report the run-out wait (the kernel stops,
 * drains what it has in flight and frees its tensor memory), and the same
 * layer must then run normally on the same context. SGN_OK if all of that
 * held, SGN_ECUDA otherwise. Allocates and synchronises on stream; a few
 * seconds at most (each run-out wait is bounded). */
sgn_status sgn_conv3_wait_selftest(void* stream);

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
