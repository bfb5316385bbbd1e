/* C ABI of the learned warm start: a 2D U-Net over the N respiratory phases
 * of a slice as channels, trained on (per-phase FBP, converged TNLM) pairs
 * that the plain method generates.  The paper has no counterpart: the
 * network only supplies a start image f^(0) for the TNLM algorithm box of
 * Sec. 2.2, which still runs to its own stopping rule and decides the
 * result.
 *
 * Network (in_ch must equal out_ch): encoder levels l = 0..L-1 with c_l = base * 2^l channels, each two
 * 3x3 convolutions (zero padding, bias) with ReLU, 2x2 max pooling between
 * levels; decoder levels l = L-2..0: nearest 2x upsampling, concatenation
 * [upsampled, encoder output of level l], two 3x3 convolutions with ReLU;
 * output = input + 1x1 convolution of the last decoder level.  Loss: mean
 * squared error.  Parameters are one flat FP32 vector in the order: encoder
 * l = 0..L-1 (conv a weight, bias, conv b weight, bias), decoder l = L-2..0
 * (same), final 1x1 (weight, bias); 3x3 weights are [cout][cin][3][3].
 *
 * Numerics: the input, the weights seen by the convolutions and every
 * post-ReLU activation are stored in BF16 (round to nearest even); sums,
 * outputs, gradients, master weights and Adam moments are FP32; a gradient
 * entering a 3x3 convolution's input- and weight-gradient products is
 * rounded to BF16 (the bias gradient uses it unrounded).  The 3x3 products
 * run on the tensor cores (tcgen05, BF16 x BF16 -> FP32) where the channel
 * counts allow (forward: 32/64/128/256 outputs; input gradient: 32/64/96/
 * 128/192/256 inputs; weight gradient: width a multiple of 16), else on the
 * CUDA cores with the same rounding.  Max pooling
 * sends its gradient to the first maximum of each 2x2 window (row-major).
 * Results are deterministic.
 *
 * Tensors are device pointers, NCHW, contiguous, FP32.  h and w must be
 * multiples of 2^(L-1).  Calls are asynchronous on 'stream' (a cudaStream_t
 * or NULL) unless stated otherwise.  Errors: TNLM_ERR_INVALID_ARG (bad
 * sizes, NULL), TNLM_ERR_OOM, TNLM_ERR_CUDA; message from
 * tnlm_unet_last_error(). */
#ifndef TNLM_UNET_H
#define TNLM_UNET_H

#include "tnlm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnlm_unet tnlm_unet;

/* A network with in_ch input and out_ch output channels, base channels at
 * level 0 and 'levels' levels, on 'device'; parameters start at zero (load
 * them with tnlm_unet_set_params).  The library owns the object. */
tnlm_status tnlm_unet_create(int in_ch, int out_ch, int base, int levels, int device, tnlm_unet** out);
void tnlm_unet_destroy(tnlm_unet* net);

/* Number of FP32 parameters (weights and biases). */
long long tnlm_unet_param_count(const tnlm_unet* net);

/* Load parameters from host memory (FP32, the order above); resets the
 * Adam moments.  Synchronous. */
tnlm_status tnlm_unet_set_params(tnlm_unet* net, const float* h_params);

/* Copy the parameters and/or the gradients of the last tnlm_unet_grads call
 * to host memory (either may be NULL).  Synchronises the device. */
tnlm_status tnlm_unet_get_params(const tnlm_unet* net, float* h_params, float* h_grads);

/* d_out[batch][out_ch][h][w] = network(d_x[batch][in_ch][h][w]). */
tnlm_status tnlm_unet_forward(tnlm_unet* net, const float* d_x, float* d_out, int batch, int h, int w,
                              void* stream);

/* Forward pass, mean squared error against d_target and the gradients of
 * every parameter (kept on the device for tnlm_unet_adam_step / _get_params).
 * loss (host, may be NULL) receives the loss and makes the call synchronous. */
tnlm_status tnlm_unet_grads(tnlm_unet* net, const float* d_x, const float* d_target, int batch, int h,
                            int w, double* loss, void* stream);

/* One Adam step with the stored gradients (bias-corrected moments). */
tnlm_status tnlm_unet_adam_step(tnlm_unet* net, float lr, float beta1, float beta2, float eps,
                                void* stream);

/* Message of the last failing tnlm_unet_* call on this host thread. */
const char* tnlm_unet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TNLM_UNET_H */
