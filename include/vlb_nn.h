/* vlb_nn.h -- the learned warm start: a small 2D U-Net that maps a mesh's
 * geometry and forcing to an estimate of its steady fields, used to start
 * the solver (vlb_reset) closer to the steady state than a rest state. The
 * paper has no counterpart: this is a serving-style addition around the
 * method, trained on steady solutions the solver itself produces.
 *
 * Network (fixed topology, width w, input channels Ci, output channels Co,
 * on an H x W index grid with H and W multiples of 4):
 *   e1 = relu(conv3(x; Ci->w)),   s1 = relu(conv3(e1; w->w))          H x W
 *   e2 = relu(conv3(pool(s1); w->2w)), s2 = relu(conv3(e2; 2w->2w))   H/2 x W/2
 *   e3 = relu(conv3(pool(s2); 2w->4w)), b = relu(conv3(e3; 4w->4w))   H/4 x W/4
 *   d2 = relu(conv3([up(b), s2]; 6w->2w)), t2 = relu(conv3(d2; 2w->2w))
 *   d1 = relu(conv3([up(t2), s1]; 3w->w)), t1 = relu(conv3(d1; w->w))
 *   y  = conv1(t1; w->Co)
 * conv3: 3x3, zero padding, bias; pool: 2x2 average; up: 2x nearest; [a, b]:
 * channel concatenation. Layouts are NCHW, FP32 at the boundary.
 *
 * Storage: weights and activations in FP32 or bfloat16; every product is
 * accumulated in FP32. An FP32 master copy of the parameters is kept for the
 * optimizer (Adam). All pointers named d_ are device pointers owned by the
 * caller; everything else is host memory. Calls are synchronous on the
 * library's stream of the net (the default stream). Errors: VLB_EINVAL,
 * VLB_ENOMEM, VLB_ECUDA (codes of vlb.h); the message is vlb_last_error(). */
#ifndef VLB_NN_H
#define VLB_NN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum vlb_nn_storage { VLB_NN_F32 = 0, VLB_NN_BF16 = 1 };

typedef struct vlb_nn vlb_nn;

/* Create a net for batches of up to max_batch samples; parameters are drawn
 * from a counter-based generator keyed by seed (He-uniform weights, zero
 * biases). */
int vlb_nn_create(int32_t in_ch, int32_t out_ch, int32_t width, int32_t H, int32_t W, int32_t max_batch,
                  int32_t storage, uint64_t seed, vlb_nn **out);
/* Number of parameters and their order: for each of the 11 layers in the
 * order above, weights [Cout][Cin][k][k] then biases [Cout]. */
int vlb_nn_num_params(const vlb_nn *net, int64_t *n);
int vlb_nn_get_params(const vlb_nn *net, float *host);
int vlb_nn_set_params(vlb_nn *net, const float *host);
/* y = net(x); x [B][Ci][H][W], y [B][Co][H][W] device FP32, B <= max_batch.
 * Keeps what the backward pass needs. With bfloat16 storage, a 3x3 layer
 * whose Co is a power of two in [16, 256], whose grid has a multiple of 128
 * cells and whose Ci is a multiple of 8 runs on the tensor cores (tcgen05:
 * an implicit GEMM with FP32 accumulators in tensor memory); the others,
 * the FP32 storage and the backward pass run on the CUDA cores. VLB_ECUDA if
 * a tensor-core layer gave up waiting (one second) for its MMAs. */
int vlb_nn_forward(vlb_nn *net, const float *d_x, float *d_y, int32_t batch);
/* Whether bfloat16 forward passes may use the tensor cores (default 1); 0
 * runs every layer on the CUDA cores (for comparison). */
int vlb_nn_set_tensor_cores(vlb_nn *net, int32_t enable);
/* Mean-square loss over all outputs against d_target and its gradient with
 * respect to y, written to d_dy (may alias nothing else); loss is returned in
 * host *loss. */
int vlb_nn_mse(vlb_nn *net, const float *d_y, const float *d_target, float *d_dy, int32_t batch,
               double *loss);
/* Gradients of the parameters for dL/dy = d_dy, through the activations of the
 * last forward call (replaces any previous gradients). */
int vlb_nn_backward(vlb_nn *net, const float *d_dy, int32_t batch);
int vlb_nn_get_grads(const vlb_nn *net, float *host);
/* One Adam step (step index t >= 1) on the FP32 master parameters; the
 * bfloat16 copy, if any, is refreshed. */
int vlb_nn_adam(vlb_nn *net, float lr, float beta1, float beta2, float eps, int64_t t);
void vlb_nn_destroy(vlb_nn *net);

#ifdef __cplusplus
}
#endif
#endif
