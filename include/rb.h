/*
 * rb.h - C ABI of the stamp real-bogus classifier and the candidate detector.
 *
 * The paper (Sec. 2.3.3-2.3.5) detects sources on the difference image,
 * cuts a three-channel stamp (science, template, difference) around each one
 * and scores it with a CNN in [0, 1]; alerts pass a score threshold (0.3 hot,
 * 0.6 cold).  Its network is not specified beyond that; this library's network
 * is: per-channel robust normalisation (median, 1.4826 MAD, clip +-64), three
 * 3 x 3 'same' convolutions (3 -> 32 -> 64 -> 64) each followed by ReLU and a
 * 2 x 2 max-pool (31 -> 15 -> 7 -> 3), a 576 -> 128 ReLU layer and a 128 -> 1
 * logit; score = sigmoid(logit).  Training minimises binary cross-entropy with
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights; forward and
 * backward matrix products run on BF16 tensor-core MMA with FP32 accumulation.
 *
 * Stamps are float [n][3][31][31] in raw ADU (channel 0 science, 1 template,
 * 2 difference), centred on the candidate pixel.  All data pointers are
 * DEVICE pointers unless named host_*; calls are asynchronous on `stream`
 * except where stated.  Statuses are the sfft_status_t codes of sfft.h.
 */
#ifndef RB_GB300_H
#define RB_GB300_H

#include <stddef.h>
#include <stdint.h>

#include "sfft.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RB_STAMP 31
#define RB_NPARAM 130305   /* w1 b1 w2 b2 w3 b3 w4 b4 w5 b5 */

typedef struct rb_model_s* rb_model_t;

/* desc[0] = max stamps per internal batch (1 .. 4096, else
 * SFFT_ERR_UNSUPPORTED), desc[1] = initialisation
 * seed (uniform He-style weights, zero biases).  Allocates the weights, Adam
 * state and activation scratch for desc[0] stamps on the current device. */
sfft_status_t rb_create(const int32_t* desc, rb_model_t* out);
sfft_status_t rb_destroy(rb_model_t m);

/* Weights as RB_NPARAM floats in the order w1 [32][3][3][3], b1 [32],
 * w2 [64][32][3][3], b2, w3 [64][64][3][3], b3, w4 [128][576] (input index
 * channel * 9 + row * 3 + column), b4, w5 [1][128], b5 [1].  Host buffers;
 * synchronous.  bytes must be RB_NPARAM * 4. */
sfft_status_t rb_set_weights(rb_model_t m, const void* host_buf, size_t bytes);
sfft_status_t rb_get_weights(rb_model_t m, void* host_buf, size_t bytes);
/* Gradients of the last rb_backward / rb_train_step, same layout (synchronous). */
sfft_status_t rb_get_grads(rb_model_t m, void* host_buf, size_t bytes);
/* Full training state for checkpoint/resume: weights, Adam first and second
 * moments (3 * RB_NPARAM floats, same layout) and the step count. */
sfft_status_t rb_get_state(rb_model_t m, void* host_buf, size_t bytes, int64_t* step);
sfft_status_t rb_set_state(rb_model_t m, const void* host_buf, size_t bytes, int64_t step);

/* Logits and scores of n stamps (any n; processed in internal batches). */
sfft_status_t rb_logits(rb_model_t m, const float* stamps, int64_t n, float* logit, void* stream);
sfft_status_t rb_score(rb_model_t m, const float* stamps, int64_t n, float* score, void* stream);

/* One fused inference convolution of the model, the step rb_logits runs per
 * layer: 3 x 3 'same' convolution with the model's weights rounded to BF16,
 * FP32 bias, ReLU and 2 x 2 max-pool (floor), BF16 output, on the tcgen05
 * tensor cores with FP32 accumulation.
 *   layer 1: in  = normalised stamps, BF16 [n][2888]: NHWC 31 x 31 x 3
 *            values, then 5 unused ones (a stamp is 5776 bytes);
 *            out = the conv2 input planes, (CB, WS) = (4, 8)
 *   layer 2: in  = those planes;  out = the conv3 input planes, (8, 4)
 *   layer 3: in  = those planes;  out = BF16 NHWC [n][3][3][64]
 * Planes are BF16 [CB][4][n_alloc][WS][WS][8]: the image is padded with a
 * zero border (padded pixel (r, c) = pixel (r - 1, c - 1)) and split by the
 * parities of r and c; record (r >> 1, c >> 1) of parity plane
 * 2 (r & 1) + (c & 1) holds channels 8 cb .. 8 cb + 7 of padded pixel (r, c),
 * and every record that holds no pixel must be zero.  The layer reads whole
 * planes of stamps < n and writes only the pixel records of stamps < n.
 * Device pointers, 16-byte aligned; 0 <= n <= n_alloc <= 2^24 (n = 0 does
 * nothing).  SFFT_ERR_ARG for a bad layer, sizes, alignment or null pointers.
 * Asynchronous on `stream`; a bounded wait that gave up sets the flag that
 * rb_get_error reads. */
sfft_status_t rb_conv_layer(rb_model_t m, int32_t layer, const void* in, int64_t n, int64_t n_alloc, void* out,
                            void* stream);
/* Error flags of the model's tensor-core kernels (synchronous): 0 none, bit 0
 * a bounded wait gave up.  Sticky for the model's lifetime; while set,
 * rb_logits and rb_score return NaN logits and scores. */
sfft_status_t rb_get_error(rb_model_t m, int32_t* flags);

/* Time attribution of the fused inference convolutions (a diagnostic): in a
 * build compiled with -DRBTC_WAIT_PROFILE, out[0 .. 9] receive the summed
 * cycles of layer `layer` (1-3) since the last reset: the CTAs' runs, the
 * copy warp's waits for a free buffer, conv1's plane builders waiting for
 * staged stamps / a free buffer / working, the MMA warp waiting for a full
 * buffer / a free accumulator slot / issuing, the epilogue warps waiting for
 * accumulators / working (lane 0 of each warp adds its own time).  reset != 0
 * zeroes the counters.  Synchronous.  SFFT_ERR_UNSUPPORTED in other builds. */
sfft_status_t rb_debug_conv_waits(int32_t layer, uint64_t* out, int32_t reset);

/* Mean BCE loss (written to loss_dev, float) and parameter gradients of one
 * batch of n <= max stamps with labels (float 0/1); no parameter update. */
sfft_status_t rb_backward(rb_model_t m, const float* stamps, const float* labels, int64_t n, float* loss_dev,
                          void* stream);
/* rb_backward followed by one Adam step with learning rate lr. */
sfft_status_t rb_train_step(rb_model_t m, const float* stamps, const float* labels, int64_t n, float lr,
                            float* loss_dev, void* stream);

/* The paper's classifier (Sec. 2.3.4: a rotation-invariant CNN in the cited
 * DeepHiTS framework with ResNet-style residual connections; the layer sizes
 * are this library's reading).  The normalised stamp passes in its four
 * rotations by multiples of 90 degrees through one shared stack:
 * conv1 3 -> 32 + ReLU + pool (31 -> 15); residual block relu(p1 +
 * conv_b(relu(conv_a(p1)))) at 32 channels; conv2 32 -> 64 + ReLU + pool
 * (15 -> 7); residual block relu(p2 + conv_d(relu(conv_c(p2)))) at 64
 * channels and a pool (7 -> 3); the four 576-feature vectors are averaged
 * (exact invariance under the rotations) and fed to fc1 576 -> 128 + ReLU and
 * fc2 128 -> 1.  Normalisation, loss, optimiser, precision and the call
 * semantics are those of the rb_* model above; desc[0] <= 2048.  Weights:
 * RBRI_NPARAM floats in the order w1 [32][3][3][3], b1, wa [32][32][3][3], ba,
 * wb [32][32][3][3], bb, w2 [64][32][3][3], b2, wc [64][64][3][3], bc,
 * wd [64][64][3][3], bd, w4 [128][576] (input index channel * 9 + row * 3 +
 * column), b4, w5 [1][128], b5. */
#define RBRI_NPARAM 185729

typedef struct rbri_model_s* rbri_model_t;

sfft_status_t rbri_create(const int32_t* desc, rbri_model_t* out);
sfft_status_t rbri_destroy(rbri_model_t m);
sfft_status_t rbri_set_weights(rbri_model_t m, const void* host_buf, size_t bytes);
sfft_status_t rbri_get_weights(rbri_model_t m, void* host_buf, size_t bytes);
sfft_status_t rbri_get_grads(rbri_model_t m, void* host_buf, size_t bytes);
sfft_status_t rbri_get_state(rbri_model_t m, void* host_buf, size_t bytes, int64_t* step);
sfft_status_t rbri_set_state(rbri_model_t m, const void* host_buf, size_t bytes, int64_t step);
sfft_status_t rbri_logits(rbri_model_t m, const float* stamps, int64_t n, float* logit, void* stream);
sfft_status_t rbri_score(rbri_model_t m, const float* stamps, int64_t n, float* score, void* stream);
sfft_status_t rbri_backward(rbri_model_t m, const float* stamps, const float* labels, int64_t n,
                            float* loss_dev, void* stream);
sfft_status_t rbri_train_step(rbri_model_t m, const float* stamps, const float* labels, int64_t n, float lr,
                              float* loss_dev, void* stream);

/* Candidate detection on difference images (Sec. 2.3.3's detection step,
 * here a matched filter): SNR(x) = sum_u G(u) D^(x - u) / (sigma_D ||G||_2)
 * with D^ = D at good finite pixels and 0 elsewhere (and outside the image),
 * G(u) = g(u_x) g(u_y), g(t) = exp(-t^2 / (2 psf_sigma^2)) on |t| <= r =
 * ceil(3 psf_sigma), 0 < psf_sigma <= 5; sigma_D the RMS of D about its mean
 * over the good finite pixels at least 15 px from every edge after three
 * 3-sigma clipping passes (|D - mean| <= 3 RMS of the previous pass), divided
 * by sqrt(0.97334), the share of a Gaussian's variance inside +-3 sigma.
 * Candidates are pixels at least 15 px from every edge, with no bad pixel
 * within Chebyshev distance `guard` (0 <= guard <= 15; 0: the pixel itself is
 * not bad; a subtraction's kernel half-width keeps out pixels whose D drew on
 * masked reference pixels), with SNR >= thresh and SNR >= every SNR in their
 * 5 x 5 neighbourhood.  Per CCD,
 * up to max_cand candidates are written in row-major order: xy int32
 * [batch][max_cand][2] (x, y), snr float [batch][max_cand], count int32
 * [batch] (the number found, which may exceed max_cand), and stamps float
 * [batch][max_cand][3][31][31] (S, R, D; non-finite values written as 0).
 * Entries past the count are left untouched.  D, S, R float [batch][H][W]
 * with H, W >= 31; bad uint8 or NULL.  The filter runs in FP32 and the clipped
 * statistics in FP64.  ws: device scratch of
 * rb_detect_workspace_bytes(H, W, batch, max_cand), 256-byte aligned. */
size_t rb_detect_workspace_bytes(int32_t H, int32_t W, int32_t batch, int32_t max_cand);
sfft_status_t rb_detect(int32_t H, int32_t W, int32_t batch, const float* D, const float* S, const float* R,
                        const uint8_t* bad, float psf_sigma, float thresh, int32_t guard, int32_t max_cand,
                        int32_t* xy, float* snr, int32_t* count, float* stamps, void* ws, void* stream);

/* Plain SNR/shape cuts on difference stamps (the classifier's fallback):
 * pass[i] = 1 iff snr[i] >= snr_min, the second-moment FWHM of the positive
 * central 9 x 9 lies in [0.5, 2.0] psf_fwhm, the negative-flux fraction of the
 * central 7 x 7 is below 0.3 and the axis ratio is below 2.5. */
sfft_status_t rb_shape_cuts(const float* stamps, const float* snr, int64_t n, float psf_fwhm, float snr_min,
                            int32_t* pass, void* stream);
/* The same cuts with a noise-robust size estimate (the paper's Sec. 2.3.4
 * fallback reading: SNR and PSF-shape cuts; the estimator is this library's
 * choice): the FWHM and axis ratio come from Gaussian-weighted adaptive
 * second moments of the difference channel over the central 15 x 15 (40
 * iterations of w = exp(-(r - mu)^T M^-1 (r - mu) / 2), mu = sum w I r / sum w I,
 * M = 2 sum w I (r - mu)(r - mu)^T / sum w I, starting from the PSF width at the
 * centre), which converge to a Gaussian source's own covariance and give
 * distant noise no weight.  A candidate fails when its weighted flux is not
 * positive, M is not positive definite, the centroid moves more than 3 px or
 * M grows past 25 px^2.  Same arguments and layouts as rb_shape_cuts. */
sfft_status_t rb_shape_cuts_adaptive(const float* stamps, const float* snr, int64_t n, float psf_fwhm,
                                     float snr_min, int32_t* pass, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RB_GB300_H */
