/*
 * ge_sno.h -- C ABI of the learned surrogate that jumps K GE steps ahead: a
 * spectral neural operator (1D Fourier neural operator) trained on GE
 * solutions, used with the GE solver as its accuracy fallback.
 *
 * The paper has no counterpart: arXiv:1310.3422 Sec. 2 defines only the GE
 * step.  The surrogate is a deployment variant for large batches of small
 * problems: it maps (u0, r, beta_l, beta_r) on a grid of n interior points to
 * an approximation of the state after a fixed number K of GE steps (the K it
 * was trained for), and the caller re-solves with GE every problem whose
 * checked error is too large.
 *
 * Model (all sizes fixed at creation):
 *   features per point: (u0_j, x_j, r, beta_l + (beta_r - beta_l) x_j),
 *     x_j = (j + 1) / (n + 1) as in the GE mesh;
 *   lift: 4 -> width channels (affine);
 *   `layers` Fourier layers: v <- act(iDFT(R_m * DFT(v)_m, m < modes)
 *     + v W + b), act = GELU (tanh form) except after the last layer; the
 *     DFT runs along the n grid points of each channel, keeps the `modes`
 *     lowest frequencies, and R_m is a complex width x width matrix;
 *   projection: width -> hidden (GELU) -> 1, added to u0: the network
 *     predicts the change of the state over the jump (residual output).
 * Arithmetic: the parameters are FP32 masters that every forward pass rounds
 * to BF16 (the network's weights are BF16 values; ge_sno_adam_step updates
 * the masters with the gradient of the rounded network).  Activations are
 * stored as BF16; every matrix product takes BF16 operands and accumulates
 * in FP32 on the tensor cores, and GELU uses the hardware tanh approximation
 * (relative error about 2^-11).  With ge_sno_set_precision(model, 1) the
 * activations are stored in FP32 and each operand is split into two BF16
 * parts and three products are summed, so activations
 * and the DFT bases enter at about FP32 accuracy (the weights, already BF16,
 * are exact) and GELU uses the library tanh; this mode is also the one
 * checked against an FP64 reference.
 *
 * Parameter vector (FP32, in this order): W0 [4][width], b0 [width]; for each
 * layer: Rr [modes][width out][width in], Ri [modes][width][width],
 * W [width in][width out], b [width]; Q1 [width][hidden], q1 [hidden],
 * Q2 [hidden], q2 [1].
 *
 * Per-problem inputs are FP32 device arrays: u0 [batch][n] row-major, r,
 * beta_l, beta_r [batch].  Conventions otherwise as in ge.h (caller-owned
 * device buffers, asynchronous on the model's stream, ge_status returns,
 * ge_last_error() text).
 */
#ifndef GE_SNO_H
#define GE_SNO_H

#include "ge.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ge_sno ge_sno;  /* opaque; owned by the library */

/* Create a model with seeded initial parameters (Adam state zeroed).
 *   n          grid points per problem (>= 4).
 *   width      channels C (>= 1); modes M (1 <= M <= n/2); layers (>= 1);
 *   hidden     projection width (>= 1); max_batch: largest batch a call may
 *              pass (activation memory is sized for it: about
 *              max_batch * n * (4 layers + 8) * width * 4 bytes).
 *   seed       initial-parameter seed.
 * Synchronous.  Errors: GE_EINVAL, GE_ENOMEM, GE_ECUDA. */
ge_status ge_sno_create(ge_sno **out, int32_t n, int32_t width, int32_t modes, int32_t layers,
                        int32_t hidden, int32_t max_batch, uint64_t seed, void *stream);

/* Number of FP32 parameters. */
ge_status ge_sno_num_params(const ge_sno *model, int64_t *count);

/* Copy the parameter vector out of / into the model (device buffers of
 * ge_sno_num_params floats). */
ge_status ge_sno_get_params(ge_sno *model, float *dst_dev);
ge_status ge_sno_set_params(ge_sno *model, const float *src_dev);

/* split = 0: BF16 operands (default); split = 1: two-part BF16 operands. */
ge_status ge_sno_set_precision(ge_sno *model, int32_t split);

/* Inference on the fifth-generation tensor cores (on = 1, the default):
 * with BF16 operands (split = 0) and the shape its kernels are built for
 * (width 64, 16 modes, hidden 128, n a multiple of 128), forward passes that
 * keep no training state (ge_sno_forward) run each fused layer (inverse DFT
 * + pointwise path + bias + GELU) and the projection (hidden layer + GELU +
 * output dot product + residual) as tcgen05 MMAs with TMEM accumulators and
 * TMA-loaded operands; the truncated DFT and the mode mixing stay on the
 * mma.sync GEMM.  Same model and operands as the other path; results differ
 * only by FP32 accumulation order (and the BF16 rounding that follows it).
 * on = 0 uses the mma.sync GEMM throughout.  Errors: GE_EINVAL. */
ge_status ge_sno_set_tensor_cores(ge_sno *model, int32_t on);
/* *active = 1 when forward passes take the tensor-core path.  Errors: GE_EINVAL. */
ge_status ge_sno_get_tensor_cores(const ge_sno *model, int32_t *active);

/* Wait for the model's stream and report a deferred device failure: a
 * bounded wait of a tensor-core kernel that gave up (GE_ETIMEOUT; the
 * outputs of that pass are not valid; reported once).  Errors: GE_EINVAL,
 * GE_ECUDA, GE_ETIMEOUT. */
ge_status ge_sno_sync(ge_sno *model);

/* Prediction for `batch` problems (1 <= batch <= max_batch): pred_dev
 * [batch][n] receives the approximate state after K steps. */
ge_status ge_sno_forward(ge_sno *model, int32_t batch, const float *u0_dev, const float *r_dev,
                         const float *beta_l_dev, const float *beta_r_dev, float *pred_dev);

/* Loss and gradient: loss_b = ||pred_b - target_b||_2 / ||target_b||_2 per
 * problem; the gradient is that of the batch mean.  loss_dev [batch] and
 * grads_dev [num_params] may each be NULL (not copied out); the gradient is
 * kept inside the model for ge_sno_adam_step either way. */
ge_status ge_sno_loss_grad(ge_sno *model, int32_t batch, const float *u0_dev, const float *r_dev,
                           const float *beta_l_dev, const float *beta_r_dev, const float *target_dev,
                           float *loss_dev, float *grads_dev);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * the gradient of the last ge_sno_loss_grad. */
ge_status ge_sno_adam_step(ge_sno *model, float lr);

/* ge_sno_loss_grad followed by ge_sno_adam_step. */
ge_status ge_sno_train_step(ge_sno *model, int32_t batch, const float *u0_dev, const float *r_dev,
                            const float *beta_l_dev, const float *beta_r_dev, const float *target_dev,
                            float lr, float *loss_dev);

/* Fallback arbiter helpers.  GE recomputes a sample of the problems and
 * replaces any problem the surrogate fails on; these move and compare rows
 * of the model's n FP32 values on the model's stream, so that no step of
 * that check runs outside the library.  Row indices are device int64
 * arrays; an index outside [0, rows) is skipped on the device (gather and
 * scatter leave that destination row untouched, rel_err writes NaN).
 *   rows_nonfinite: flags_dev[i] = 1 if row i of u_dev ([rows][n]) holds a
 *                   NaN or an infinity, else 0.
 *   rows_gather:    dst_dev row i <- src_dev row idx[i] (src has src_rows rows).
 *   rows_scatter:   dst_dev row idx[i] <- src_dev row i (dst has dst_rows rows).
 *   rows_rel_err:   err_dev[i] = ||a row idx[i] - ref row i||_2 / ||ref row i||_2,
 *                   sums in FP64; +inf when not finite or when ref is zero
 *                   and the rows differ.
 * Errors: GE_EINVAL (NULL model or pointer, negative counts), GE_ECUDA. */
ge_status ge_sno_rows_nonfinite(ge_sno *model, const float *u_dev, int64_t rows, int32_t *flags_dev);
ge_status ge_sno_rows_gather(ge_sno *model, const float *src_dev, int64_t src_rows, const int64_t *idx_dev,
                             int64_t count, float *dst_dev);
ge_status ge_sno_rows_scatter(ge_sno *model, float *dst_dev, int64_t dst_rows, const int64_t *idx_dev,
                              const float *src_dev, int64_t count);
ge_status ge_sno_rows_rel_err(ge_sno *model, const float *a_dev, int64_t a_rows, const int64_t *idx_dev,
                              const float *ref_dev, int64_t count, float *err_dev);

/* Free the model (waits for its stream first).  NULL is a no-op. */
void ge_sno_destroy(ge_sno *model);

#ifdef __cplusplus
}
#endif

#endif /* GE_SNO_H */
