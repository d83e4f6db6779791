/*
 * rad_mlp.h -- C ABI of the learned surrogate's network.
 *
 * The surrogate (a build-side addition to the paper's method, which always
 * evaluates the full sum of Sec. 2.2) maps a sparse spectrum computed exactly
 * by the rad_* library to the dense spectrum: a ReLU multilayer perceptron
 *     h_0 = x,  z_{l+1} = h_l W_l^T + b_l,  h_{l+1} = ReLU(z_{l+1}),  y = z_L,
 * trained on the mean squared error with Adam.  Arithmetic: BF16 weights (an
 * FP32 master copy is what Adam updates), BF16 GEMM operands (activations and
 * backward gradients rounded to BF16 where they enter a product), FP32
 * accumulation on the tensor cores, FP32 biases, losses accumulated in FP64.
 * Rounding points (the CPU oracle takes the same): x -> BF16; h_{l+1} =
 * BF16(ReLU(z_{l+1})); g_L = 2 (y - t)/(B * out) in FP32, BF16 for products;
 * dW_l = BF16(g_{l+1})^T h_l; g_l = (BF16(g_{l+1}) W_l) * [z_l > 0] in FP32, BF16
 * for products; db_l = column sums of the FP32 g_{l+1}.
 *
 * Every width must be a positive multiple of 128.  Batches are padded to a
 * multiple of 128 internally (padded rows carry no gradient).  Pointers may
 * be host or device memory unless stated.  Returns RAD_MLP_OK or a negative
 * code; calls are stream ordered on the stream given at init and return after
 * their results are ready.
 *
 * The products run on the tcgen05 tensor cores (TMA-staged BF16 tiles, FP32
 * accumulators in tensor memory).  Every wait inside a GEMM block is bounded;
 * an expired wait sets a device-wide error word that the next synchronising
 * call (rad_mlp_forward, rad_mlp_gradients, rad_mlp_check) reports as
 * RAD_MLP_ETIMEOUT and clears.
 */
#ifndef RAD_MLP_H
#define RAD_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RAD_MLP_OK 0
#define RAD_MLP_EINVAL (-1)
#define RAD_MLP_ENOMEM (-2)
#define RAD_MLP_ECUDA (-3)
#define RAD_MLP_ETIMEOUT (-4) /* a GEMM block's bounded wait expired (results invalid) */

typedef struct rad_mlp rad_mlp;

/* widths: [n_layers + 1] layer widths (input first); max_batch >= 1. */
int rad_mlp_init(rad_mlp **out, const int32_t *widths, int32_t n_layers, int32_t max_batch,
                 void *cuda_stream);

/* Set layer `layer`'s FP32 weights W [out][in] and bias b [out]; resets Adam. */
int rad_mlp_set_layer(rad_mlp *m, int32_t layer, const float *W, const float *b);

/* Read a layer's FP32 weights, bias and last gradients (any pointer may be NULL). */
int rad_mlp_get_layer(rad_mlp *m, int32_t layer, float *W, float *b, float *dW, float *db);

/* y [batch][out] = network(x [batch][in]), FP32 in and out. */
int rad_mlp_forward(rad_mlp *m, int32_t batch, const float *x, float *y);

/* Forward + MSE against t [batch][out] + backward: stores dW, db of every
 * layer (read them with rad_mlp_get_layer); *loss (host, may be NULL) gets the MSE. */
int rad_mlp_gradients(rad_mlp *m, int32_t batch, const float *x, const float *t, double *loss);

/* The surrogate's data transforms, for rad_mlp_predict: per input feature
 * x' = (log10(max(x, floor_value)) - in_mu) / in_sd, per output feature
 * y = 10^(z out_sd + out_mu) ([w_0] and [w_L] FP32 values each, host or
 * device; floor_value > 0).  The statistics are the training set's. */
int rad_mlp_set_transform(rad_mlp *m, const float *in_mu, const float *in_sd, const float *out_mu,
                          const float *out_sd, float floor_value);

/* Prediction in physical units: the input transform, the forward pass and the
 * output transform, all on the device; x [batch][w_0] raw inputs, y
 * [batch][w_L] (host or device).  RAD_MLP_EINVAL before rad_mlp_set_transform. */
int rad_mlp_predict(rad_mlp *m, int32_t batch, const float *x, float *y);

/* One Adam step from the stored gradients (bias-corrected; FP32 master weights,
 * BF16 copies of W and W^T refreshed).  Stream ordered; does not wait. */
int rad_mlp_adam(rad_mlp *m, float lr, float beta1, float beta2, float eps);

/* One training step: rad_mlp_gradients followed by rad_mlp_adam in one call,
 * with no host synchronisation between the backward pass and the optimiser
 * (the gradients are stored as by rad_mlp_gradients).  Same arguments and
 * checks as the two calls; *loss (host, may be NULL) gets the MSE before the
 * update.  Waits for the stream. */
int rad_mlp_train_step(rad_mlp *m, int32_t batch, const float *x, const float *t, float lr,
                       float beta1, float beta2, float eps, double *loss);

/* The tensor-core GEMM on its own: C [M][N] (FP32, device) = op(A) op(B), BF16
 * device operands (16-byte aligned); a_kcontig != 0: A stored [M][K], else
 * [K][M]; b_kcontig != 0: B stored [N][K], else [K][N] (operands stored K-last are first
 * transposed into scratch).  M, N multiples of 128, K of 64.  Default stream;
 * returns once the work is enqueued.  Products with few 128 x 128 output tiles
 * and a long K are split over K.  Scratch comes from the default stream's
 * stream-ordered pool (RAD_MLP_ENOMEM when it cannot be had).  A, B or C
 * outside device or managed memory: RAD_MLP_EINVAL, nothing launched. */
int rad_mlp_gemm(int32_t a_kcontig, int32_t b_kcontig, int32_t M, int32_t N, int32_t K,
                 const void *A, const void *B, float *C);

/* Waits for the device and reports whether any GEMM block's bounded wait
 * expired since the last check (RAD_MLP_ETIMEOUT), clearing the flag. */
int rad_mlp_check(void);

/* Text of the last failure of a rad_mlp_* call on the calling host thread
 * (empty if none; the storage belongs to the library). */
const char *rad_mlp_last_error(void);

void rad_mlp_destroy(rad_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* RAD_MLP_H */
