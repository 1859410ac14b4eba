// Internal interface of the learned denoiser's kernels (unet_kernels.cu):
// convolution geometry and launch functions behind include/fdc_unet.h.
#pragma once

#include <cuda_runtime.h>

namespace fdc {

// Denoiser convolutions (layout in fdc_unet.h).
struct Conv3dArgs {
    int batch, in_d, in_h, in_w, out_d, out_h, out_w, c_in, c_out, ksize, stride, pad, relu;
    // data gradient only: null, or the layer's forward input (same layout as
    // the output, BF16); output values where it is not positive become zero
    // (the ReLU derivative of the layer that produced that input)
    const void *mask;
    // data gradient of a layer whose forward input was [upsample?(a) | b]
    // (fdc_conv3d_forward_fused), read without materialising it: with
    // mask_ca > 0 the mask of channels < mask_ca is `mask` (mask_ca channels,
    // at half resolution when mask_up) and of the others `mask_b` (Nn -
    // mask_ca channels); with out_b, output channels >= mask_ca go to out_b
    // ([voxel][Nn - mask_ca]) and the others to the main output ([voxel][mask_ca]).
    const void *mask_b;
    int mask_ca, mask_up;
    void *out_b;
};
// residual (data gradient, mode 1, BF16 like the output, not aliasing it): added to the output
cudaError_t launch_conv(const Conv3dArgs &g, int mode, const void *src, const void *wt, const float *bias,
                        void *out_bf16, float *out_f32, cudaStream_t st, const void *residual = nullptr);
int tc_status(bool clear);
cudaError_t launch_wait_timeout(long long cycles, cudaStream_t st);
cudaError_t launch_conv_halo(const Conv3dArgs &g, const void *src, const void *wt, const float *bias,
                             void *out_bf16, float *out_f32, int Cs, int Nn, int relu, cudaStream_t st,
                             int ca, int up_a, const void *src_b);
// the sub-pixel convolution of upsample2(xa) (cudaErrorNotSupported, nothing
// launched, for shapes without its kernel) and its collapsed weights
cudaError_t launch_conv_up(const Conv3dArgs &g, const void *xa, const void *w_up, const float *bias, void *out_bf16,
                           float *out_f32, int relu, cudaStream_t st);
cudaError_t launch_collapse_up(const void *w, void *w_up, int co, int ci, cudaStream_t st);
// the data gradient of that convolution on the coarse grid (g.mask: the plain ReLU mask xa)
// and its transposed collapsed weights
cudaError_t launch_conv_up_dgrad(const Conv3dArgs &g, const void *dy, const void *w_up_t, void *dxa, cudaStream_t st);
cudaError_t launch_collapse_up_t(const void *w, void *w_up_t, int co, int ci, cudaStream_t st);
cudaError_t launch_flip_transpose(const void *w, void *wf, int co, int k, int ci, cudaStream_t st);
cudaError_t launch_conv_wgrad(const Conv3dArgs &g, const void *x, const void *dy, float *dw, float *db,
                              cudaStream_t st, int ca, int up_a, const void *xb);
bool conv_dwalk_enabled();
cudaError_t launch_transpose_weights(const void *w, void *wt, int co, int taps, int ci, cudaStream_t st);
cudaError_t launch_relu_bwd(const void *y, const void *dy, void *dx, long long n, cudaStream_t st);
cudaError_t launch_upsample2(const void *x, void *y, int B, int D, int H, int W, int C, int backward,
                             cudaStream_t st);
cudaError_t launch_concat(const void *a, int Ca, const void *b, int Cb, void *out, long long rows, int inverse,
                          cudaStream_t st);
cudaError_t launch_mse(const float *pred, int C, const float *target, long long rows, void *grad, float *loss,
                       cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, void *p_bf16, long long n, float lr, float b1,
                        float b2, float eps, float bc1, float bc2, cudaStream_t st);
cudaError_t launch_f32_to_bf16(const float *x, void *y, long long n, cudaStream_t st);
cudaError_t launch_add_bf16(const void *a, const void *b, void *out, long long n, cudaStream_t st);
// scale_dev (may be null): the dose scale read on the device instead of inv_scale / scale
cudaError_t launch_prepare(const double *dose, const float *density, const double *dose_high, long long n,
                           double inv_scale, float density_scale, void *x, float *dose_in, float *target,
                           cudaStream_t st, const double *scale_dev);
cudaError_t launch_dose_scale(const double *dose, long long n, double *scale, cudaStream_t st);
cudaError_t launch_finish(const float *head, const float *dose_in, long long n, double scale, double *dose_out,
                          cudaStream_t st);
cudaError_t launch_head(const void *x, const void *w, const float *b, long long n, const float *dose_in,
                        double scale, float *y, double *dose_out, cudaStream_t st, const double *scale_dev);
cudaError_t launch_head_loss(const void *x, const void *w, const float *b, const float *target, long long n,
                             float *loss, void *dx, float *dw, float *db, cudaStream_t st);
cudaError_t launch_gamma(const double *ref, const double *eval, int D, int H, int W, double sd, double sh, double sw,
                         double dd, double dta, double thr, int radius, float *gamma, unsigned long long *scratch,
                         cudaStream_t st);

}  // namespace fdc
