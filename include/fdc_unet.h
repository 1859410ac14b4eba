/*
 * fdc_unet.h -- C ABI of the learned denoiser's kernels.
 *
 * The denoiser is not part of the paper: it is a small 3-D U-Net that maps a
 * dose computed from few histories (plus the phantom density) to the dose of
 * many histories; the track-repeating engine of fdc.h generates its training
 * pairs and stays the fallback and the reference its error is measured against.  These calls are
 * the building blocks the network is trained and run with: BF16 tensor-core
 * convolutions with FP32 accumulation and their gradients, plus the
 * element-wise pieces.
 *
 * Conventions: all pointers are device memory owned by the caller; tensors
 * are channels-last [batch][d][h][w][c]; "bf16" arrays hold IEEE bfloat16
 * values (uint16 storage); weights are [c_out][k][k][k][c_in] (bf16) and
 * their data-gradient copy [c_in][k][k][k][c_out] (fdc_conv3d_transpose_weights).
 * Calls are asynchronous on `stream` (cudaStream_t as void *, NULL = legacy
 * default stream) and return FDC_OK, FDC_ERR_INVALID (bad shapes: channel
 * counts must be multiples of 16 and at most 2048, sizes positive and consistent) or
 * FDC_ERR_CUDA (launch failure).
 */
#ifndef FDC_UNET_H
#define FDC_UNET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A 3-D convolution: kernel ksize^3 (1, 2 or 3), stride, zero padding pad;
 * out = (in + 2 pad - ksize) / stride + 1 per axis.  relu = 1 applies
 * max(0, .) to the forward output. */
typedef struct fdc_conv3d {
    int32_t batch, in_d, in_h, in_w, out_d, out_h, out_w, c_in, c_out, ksize, stride, pad, relu;
} fdc_conv3d;

/* y[b][o][co] = act(bias[co] + sum_{tap, ci} x[b][o * stride - pad + tap][ci] w[co][tap][ci]).
 * x bf16 [batch][in...][c_in]; w bf16; bias FP32 [c_out] or NULL; outputs
 * y_bf16 [batch][out...][c_out] and/or y_f32 (either may be NULL). */
int fdc_conv3d_forward(const fdc_conv3d *g, const void *x, const void *w, const float *bias, void *y_bf16,
                       float *y_f32, void *stream);
/* The forward map of a 3^3, stride-1, padding-1 convolution (ksize 3, stride 1,
 * pad 1 required) whose input is the channel concatenation [xa | xb]: xa holds
 * the first ca channels (multiple of 16), at half resolution and read through
 * nearest x2 upsampling when upsample_a = 1 (in_d, in_h, in_w even); xb holds
 * the other c_in - ca channels at full resolution (may be NULL when ca = c_in).
 * Same result as fdc_conv3d_forward on the materialised input. */
int fdc_conv3d_forward_fused(const fdc_conv3d *g, const void *xa, int32_t ca, int32_t upsample_a, const void *xb,
                             const void *w, const float *bias, void *y_bf16, float *y_f32, void *stream);
/* The 3^3 convolution (ksize 3, stride 1, pad 1) of upsample2(xa), computed
 * on xa's own half-resolution grid by output parity class: along each axis,
 * output 2i + p reads the two coarse voxels i + p - 1 and i + p with the sums
 * of the weights of the taps that land on them, 8 collapsed taps per output
 * voxel instead of 27.  g describes the full-resolution convolution (in_d,
 * in_h, in_w even, output = input size); xa bf16 [batch][in_d/2][in_h/2][in_w/2][c_in];
 * w_up the collapsed weights of fdc_conv3d_collapse_up_weights; bias, relu and
 * outputs as in fdc_conv3d_forward.  Equals fdc_conv3d_forward_fused with
 * upsample_a = 1 up to the one BF16 rounding of each collapsed weight (unit
 * roundoff 2^-8): per output, |difference| <= 2^-8 * sum over taps and
 * channels of |w| |x| (plus FP32 accumulation order).  FDC_ERR_INVALID, launching nothing, for shapes
 * without its kernel: c_in a multiple of 16 up to 64, c_out a multiple of
 * 16, a half-resolution grid of at least 10 (h) x 16 (w), shared memory for
 * the collapsed weights of every input channel. */
int fdc_conv3d_forward_up(const fdc_conv3d *g, const void *xa, const void *w_up, const float *bias, void *y_bf16,
                          float *y_f32, void *stream);
/* Collapsed weights for fdc_conv3d_forward_up: w_up[co][pd ph][sd sh][pw sw][ci]
 * (bf16, c_out x 64 x c_in) = the sum, in FP32 rounded once to BF16, of
 * w[co][kd][kh][kw][ci] over the taps with (p + k - 1) >> 1 = p - 1 + s on each
 * axis (p: output parity, s = 0, 1: the first or second coarse voxel read).
 * g: a 3^3, stride-1, padding-1 convolution. */
int fdc_conv3d_collapse_up_weights(const fdc_conv3d *g, const void *w, void *w_up, void *stream);
/* The data gradient of fdc_conv3d_forward_up with respect to its coarse input
 * xa, computed on the coarse grid (the adjoint of the sub-pixel form): along
 * each axis, coarse voxel m receives the gradients dy[2m - 1 .. 2m + 2] of the
 * outputs that read it, each through its collapsed weight, so
 * dxa = upsample2-adjoint of the full-resolution data gradient without
 * forming the latter.  g as for fdc_conv3d_forward_up; dy bf16
 * [batch][in_d][in_h][in_w][c_out]; w_up_t from
 * fdc_conv3d_collapse_up_weights_t; relu_mask (may be NULL): xa, bf16
 * [batch][in_d/2][in_h/2][in_w/2][c_in], dxa written as zero where it is not
 * positive; dxa bf16 in xa's layout.  Equals the adjoint of the direct form up
 * to the BF16 rounding of each collapsed weight (|difference| <= 2^-8 * the
 * same sum with |w| and |dy|) and FP32 accumulation order.  FDC_ERR_INVALID,
 * launching nothing, without a kernel for the shape (full-resolution grid of
 * at least 20 (h) x 32 (w), even sizes). */
int fdc_conv3d_backward_data_up(const fdc_conv3d *g, const void *dy, const void *w_up_t, const void *relu_mask,
                                void *dxa, void *stream);
/* Transposed collapsed weights for fdc_conv3d_backward_data_up: w_up_t[ci][t][co]
 * (bf16, c_in x 64 x c_out), t = (q_d, q_h, q_w, i_d, i_h, i_w) as bits from the
 * highest, = the FP32 sum (rounded once to BF16) of w[co][kd][kh][kw][ci] over the
 * taps of each axis with (q + k - 1) >> 1 = q - i: the collapsed weight of output
 * parity q and coarse offset s = 1 - i. */
int fdc_conv3d_collapse_up_weights_t(const fdc_conv3d *g, const void *w, void *w_up_t, void *stream);
/* dx[b][i][ci] = sum over (tap, co) with i + pad - tap = stride * o of dy[b][o][co] w[co][tap][ci]
 * (the gradient of the forward map with respect to x, without this layer's ReLU).
 * dy bf16 [batch][out...][c_out]; w_t the data-gradient weights that
 * fdc_conv3d_transpose_weights produced for this convolution; dx bf16.
 * relu_mask (may be NULL): this convolution's forward input x (bf16, the
 * layout of dx); where it is not positive dx is written as zero -- the
 * derivative of the ReLU that produced x, applied in the same pass (dx is
 * then the gradient with respect to the previous layer's pre-activation). */
int fdc_conv3d_backward_data(const fdc_conv3d *g, const void *dy, const void *w_t, const void *relu_mask, void *dx,
                             void *stream);
/* The same plus a second gradient of the same activation: dx = (masked data
 * gradient) + residual, rounded once to BF16 (the U-Net adds the skip
 * connection's gradient this way).  residual bf16 in dx's layout, must not
 * alias dx.  The 2^3 stride-2 convolutions add it in the tensor-core
 * epilogue; other shapes run the data gradient, then the addition. */
int fdc_conv3d_backward_data_add(const fdc_conv3d *g, const void *dy, const void *w_t, const void *relu_mask,
                                 const void *residual, void *dx, void *stream);
/* dw[co][tap][ci] += sum_o dy[o][co] x[o * stride - pad + tap][ci] and, if db is not NULL,
 * db[co] += sum_o dy[o][co]; dw, db FP32 (accumulated: zero them first). */
int fdc_conv3d_backward_weights(const fdc_conv3d *g, const void *x, const void *dy, float *dw, float *db,
                                void *stream);
/* The gradients of fdc_conv3d_forward_fused (3^3, stride 1, padding 1), whose
 * input x = [upsample?(xa) | xb] is never materialised (xa: ca channels, at
 * half resolution when upsample_a; xb: c_in - ca channels, NULL when
 * ca = c_in):
 *   backward_weights_fused: as fdc_conv3d_backward_weights on that x;
 *   backward_data_fused: as fdc_conv3d_backward_data with relu_mask = x,
 *     the result split by channel: dxa[voxel][ca] (full resolution: the
 *     gradient with respect to upsample(xa) when upsample_a) and
 *     dxb[voxel][c_in - ca]; needs c_out <= 32 (the d-walking kernels).
 * FDC_ERR_INVALID for other geometries, ca not a multiple of 16, a missing
 * xb / dxb, or odd sizes with upsample_a. */
int fdc_conv3d_backward_weights_fused(const fdc_conv3d *g, const void *xa, int32_t ca, int32_t upsample_a,
                                      const void *xb, const void *dy, float *dw, float *db, void *stream);
int fdc_conv3d_backward_data_fused(const fdc_conv3d *g, const void *dy, const void *w_t, const void *xa, int32_t ca,
                                   int32_t upsample_a, const void *xb, void *dxa, void *dxb, void *stream);
/* Data-gradient weights (bf16, c_in x k^3 x c_out): w_t[ci][tap][co] = w[co][tap][ci], with the
 * tap reflected (tap -> k^3 - 1 - tap) for 3^3 stride-1 padding-1 convolutions, whose data
 * gradient is then a forward convolution of dy. */
int fdc_conv3d_transpose_weights(const fdc_conv3d *g, const void *w, void *w_t, void *stream);
/* The same for n layers in one launch per 32 layers: g[i], w[i], w_t[i] (host
 * arrays of geometries and device pointers) as in fdc_conv3d_transpose_weights.
 * FDC_ERR_INVALID on n < 0, a NULL array or pointer, or a bad geometry. */
int fdc_conv3d_transpose_weights_batch(int32_t n, const fdc_conv3d *g, const void *const *w, void *const *w_t,
                                       void *stream);

/* dx = dy where y > 0, else 0 (bf16, n elements). */
int fdc_relu_backward(const void *y, const void *dy, void *dx, int64_t n, void *stream);
/* Nearest-neighbour x2 upsampling of x [b][d][h][w][c] into y [b][2d][2h][2w][c]
 * (backward = 0), or its adjoint: dx[b][d][h][w][c] = sum of the 8 children of dy
 * (backward = 1, x = dy, y = dx).  bf16. */
int fdc_upsample2(const void *x, void *y, int32_t b, int32_t d, int32_t h, int32_t w, int32_t c,
                  int32_t backward, void *stream);
/* split = 0: out[r] = concat(a[r] (ca channels), b[r] (cb channels)); split = 1:
 * the inverse, a[r] and b[r] from out[r].  bf16, rows r. */
int fdc_concat_channels(void *a, int32_t ca, void *b, int32_t cb, void *out, int64_t rows, int32_t split,
                        void *stream);
/* Mean squared error of channel 0 of pred [rows][c] (FP32) against target [rows]:
 * adds mean((pred - target)^2) to *loss (FP32, device) and, if grad is not NULL,
 * writes d loss / d pred into grad [rows][c] (bf16, zero outside channel 0). */
int fdc_mse(const float *pred, int32_t c, const float *target, int64_t rows, void *grad, float *loss,
            void *stream);
/* One Adam step (Kingma & Ba 2015) at step number `step` (>= 1) on n FP32 parameters p with
 * gradient g and moments m, v; also writes the bf16 copy p_bf16 if not NULL. */
int fdc_adam(float *p, const float *g, float *m, float *v, void *p_bf16, int64_t n, float lr, float beta1,
             float beta2, float eps, int32_t step, void *stream);
/* y = bf16(x), n elements. */
int fdc_f32_to_bf16(const float *x, void *y, int64_t n, void *stream);
/* out = a + b (bf16, n elements; out may alias a or b). */
int fdc_add_bf16(const void *a, const void *b, void *out, int64_t n, void *stream);

/* Network input from a dose grid of n voxels (FP64, Gy) and its density
 * (FP32): x [n][16] bf16 with channel 0 = dose / dose_scale, channel 1 =
 * density * density_scale, channels 2..15 zero; dose_in [n] FP32 = channel 0.
 * With dose_high (a high-history dose of the same field) and target not NULL,
 * target [n] FP32 = dose_high / dose_scale - dose_in, the correction the
 * network is trained to predict.  x must be 16-byte aligned (rows are
 * written as 16-byte pieces); FDC_ERR_INVALID otherwise. */
int fdc_unet_prepare(const double *dose, const float *density, const double *dose_high, int64_t n,
                     double dose_scale, float density_scale, void *x, float *dose_in, float *target,
                     void *stream);
/* The same steps with the dose scale in device memory, so that a whole
 * denoising pass (scale, input, network, head) can be captured in one CUDA
 * graph without a device-to-host read of the scale:
 *   fdc_unet_dose_scale: *scale (FP64, device) = max of dose[n] (dose values are
 *     non-negative; 0 when all are 0);
 *   fdc_unet_prepare_dev: fdc_unet_prepare without the training target, the
 *     scale read from *scale on the device (a scale <= 0 counts as 1);
 *   fdc_unet_head_dev: fdc_unet_head's dose_out with the scale read likewise.
 * The results equal those of the host-scale calls given the same scale.
 * FDC_ERR_INVALID on NULL pointers, n < 1, c != 16 or misaligned x. */
int fdc_unet_dose_scale(const double *dose, int64_t n, double *scale, void *stream);
int fdc_unet_prepare_dev(const double *dose, const float *density, int64_t n, const double *scale,
                         float density_scale, void *x, float *dose_in, void *stream);
int fdc_unet_head_dev(const void *x, int32_t c, const void *w, const float *b, int64_t n, const float *dose_in,
                      const double *scale, double *dose_out, void *stream);
/* Training augmentation by a lateral symmetry of a field along +z (the
 * physics is unchanged by mirroring x or y or exchanging them, so a transformed
 * pair is another valid low/high-history pair): for every voxel of the d x h x w
 * grid (x fastest), x_out[z][y][x] = x[z][y'][x'] (16 bf16 channels) and, if
 * target is not NULL, target_out likewise (FP32), where (y', x') is (y, x)
 * after exchanging them (code bit 2; needs h == w), then mirroring x (bit 0)
 * and y (bit 1).  Outputs must not alias inputs.  FDC_ERR_INVALID on bad
 * sizes, a code outside 0..7 or aliasing. */
int fdc_unet_dihedral(const void *x, const float *target, int32_t d, int32_t h, int32_t w, int32_t code,
                      void *x_out, float *target_out, void *stream);
/* Device status of the tensor-core convolutions: FDC_OK, or FDC_ERR_TIMEOUT
 * once a convolution CTA gave up waiting for its accumulator (that CTA wrote
 * no output); clear != 0 resets it.  Synchronises with the device; not for
 * use inside stream capture.
 * After FDC_ERR_TIMEOUT nothing computed on the device from that launch on
 * can be trusted: the CTA that gave up frees its tensor memory and returns
 * while the matrix operations it issued may still be reading its shared
 * memory and writing the columns it freed, which later CTAs may hold.  Treat
 * the timeout as fatal to the process's GPU state: discard the outputs of
 * that and every later launch and rebuild the CUDA context. */
int fdc_unet_status(int32_t clear);
/* Test hook of that status (no counterpart in the paper): launches one thread
 * that waits on a barrier nothing completes, gives up after `cycles` SM clock
 * cycles (1 .. 4e9) and records FDC_ERR_TIMEOUT as a timed-out convolution
 * would.  It issues no matrix operation, so it exercises the bounded wait and
 * the status word only, not a convolution CTA abandoning operations in
 * flight.  Asynchronous on `stream`; FDC_ERR_INVALID for cycles out of
 * range. */
int fdc_debug_wait_timeout(int64_t cycles, void *stream);
/* Denoised dose: dose_out [n] (FP64, Gy) = max(0, (head[n][16] channel 0 + dose_in) * dose_scale). */
int fdc_unet_finish(const float *head, const float *dose_in, int64_t n, double dose_scale, double *dose_out,
                    void *stream);

/* Head of the denoiser, output channel 0 of its 1^3 convolution (the only
 * channel the loss and the denoised dose use): for every voxel i of n,
 * y_i = b[0] + sum_c w[c] x[i][c], with x [n][16] BF16 features (c must be 16;
 * 16-byte aligned), w the 16 BF16 weights of that output channel (row 0 of the
 * head's [16][16] weights) and b its FP32 bias (b[0] read on the device).
 * Products are exact, the sum FP32.  y [n] FP32 (may be NULL) receives y_i;
 * dose_out [n] FP64 (may be NULL; needs dose_in and dose_scale > 0) receives
 * max(0, (y_i + dose_in[i]) * dose_scale), the denoised dose in Gy.
 * FDC_ERR_INVALID on NULL inputs, c != 16, n < 1 or no output. */
int fdc_unet_head(const void *x, int32_t c, const void *w, const float *b, int64_t n, const float *dose_in,
                  double dose_scale, float *y, double *dose_out, void *stream);
/* Loss and gradients of that head: *loss += (1/n) sum_i (y_i - target[i])^2
 * (FP32, *loss on the device); with g_i = 2 (y_i - target[i]) / n,
 * dx [n][16] BF16 (may be NULL; 16-byte aligned, not aliasing x) =
 * bf16(w[c] g_i) where x[i][c] > 0, else 0 (the ReLU derivative of the layer
 * that produced x); dw [16] FP32 += sum_i g_i x[i][c] and db[0] += sum_i g_i
 * (both NULL, or both given).  Sums are per-block FP32 partials added with
 * atomics: their order, and so their last bits, vary from run to run.
 * FDC_ERR_INVALID on NULL inputs, c != 16, n < 1, misalignment, aliasing, or
 * exactly one of dw and db. */
int fdc_unet_head_loss(const void *x, int32_t c, const void *w, const float *b, const float *target, int64_t n,
                       float *loss, void *dx, float *dw, float *db, void *stream);

/* Gamma index (Low, Harms, Mutic & Purdy 1998) of an evaluated dose against a
 * reference dose on the same d x h x w grid (spacing sd, sh, sw cm; FP64,
 * x fastest): for every reference voxel above threshold * max(ref),
 * gamma = min over evaluated voxels within the search radius of
 * sqrt(distance^2 / dta^2 + (eval - ref)^2 / (dose_frac * max(ref))^2)
 * (global dose difference, voxel-centre sampling, no interpolation; search
 * radius ceil(1.5 dta / min spacing) voxels, at most 8).  gamma [n] FP32
 * (may be NULL) receives the values (-1 outside the threshold); scratch is a
 * device buffer of 3 uint64; *pass_rate (host, may be NULL) receives the
 * fraction of evaluated voxels with gamma <= 1 (the call then waits for the
 * stream). */
int fdc_gamma(const double *ref, const double *eval, int32_t d, int32_t h, int32_t w, double sd, double sh,
              double sw, double dose_frac, double dta, double threshold, float *gamma, uint64_t *scratch,
              double *pass_rate, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FDC_UNET_H */
