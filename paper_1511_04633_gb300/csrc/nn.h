// nn.h -- launchers of the surrogate's kernels (nn.cu); see nn.cu for the
// layouts.  Every launcher returns the CUDA error of its launches.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lbm {
namespace nn {

// Input features per voxel (see features_kernel).
constexpr int kFeatures = 8;

// y = act(conv_k(x, w) + bias), k in {1, 3}, n a multiple of 8; act: 0 none,
// 1 leaky ReLU (slope 0.1).  bias may be null.  bfloat16 x and w (cin a
// multiple of 8) run on tensor cores; other types on CUDA cores.
template <typename TI, typename TW, typename TO>
cudaError_t conv3d(const TI *x, const TW *w, const float *bias, TO *y, int batch, int n, int cin,
                   int cout, int k, int act, cudaStream_t s);

// dw (FP32, [tap][cout][cin]) of conv3d; scratch holds the per-chunk partials.
template <typename TI>
cudaError_t conv3d_wgrad(const TI *x, const float *dy, float *dw, float *scratch,
                         size_t scratch_floats, int batch, int n, int cin, int cout, int k,
                         cudaStream_t s);

// the same on tensor cores, with the output gradient in bfloat16; requires
// cin and cout multiples of 8 and 16-byte aligned x and dy
// (cudaErrorInvalidValue otherwise).
cudaError_t conv3d_wgrad_bf16(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *dw, float *scratch,
                              size_t scratch_floats, int batch, int n, int cin, int cout, int k,
                              cudaStream_t s);

// Number of tcgen05 convolution launches whose bounded wait ran out (their
// output is not written); reset = true clears it.  -1 on a CUDA error.
int tensor_core_errors(bool reset);

cudaError_t bias_grad(const float *dy, float *db, float *scratch, size_t scratch_floats,
                      long long voxels, int cout, cudaStream_t s);

// dy *= slope where the leaky-ReLU output yout is not positive.
template <typename T>
cudaError_t act_backward(const T *yout, float *dy, long long len, cudaStream_t s);

// act_backward (if act) and then dyn = bfloat16(dy), in one pass; len % 4 == 0,
// dy 16-byte and dyn 8-byte aligned.
template <typename T>
cudaError_t act_backward_narrow(const T *yout, float *dy, __nv_bfloat16 *dyn, long long len, int act,
                                cudaStream_t s);

// act_backward_narrow over voxels x cout values plus the bias gradient db[co]
// = sum over voxels of dy[v][co], in a fixed order; cout % 4 == 0 and cout / 4
// dividing 256; `scratch` holds 608 * cout partial sums.
template <typename T>
cudaError_t act_backward_narrow_bias(const T *yout, float *dy, __nv_bfloat16 *dyn, long long voxels, int cout,
                                     int act, float *db, float *scratch, size_t scratch_floats, cudaStream_t s);

// weights of the transposed convolution (input gradient = conv3d with them)
template <typename TW>
cudaError_t flip_transpose(const TW *w, TW *wt, int k, int cout, int cin, cudaStream_t s);

template <typename T>
cudaError_t avgpool2(const T *x, T *y, int batch, int n, int c, cudaStream_t s);
cudaError_t avgpool2_backward(const float *dy, float *dx, int batch, int n, int c, cudaStream_t s);
template <typename T>
cudaError_t up2_add(const T *x, const T *skip, T *y, int batch, int n, int c, cudaStream_t s);
cudaError_t up2_backward(const float *dy, float *dx, int batch, int n, int c, cudaStream_t s);
cudaError_t add_inplace(float *a, const float *b, long long len, cudaStream_t s);

// loss = mean((yp - tgt)^2) into *loss (device double); dy = d loss / d yp.
template <typename T>
cudaError_t mse(const T *yp, const float *tgt, float *dy, double *partials, double *loss,
                long long len, cudaStream_t s);

template <typename TW>
cudaError_t adam(float *master, TW *wstore, const float *grad, float *m1, float *m2, long long len,
                 float lr, float beta1, float beta2, float eps, int t, cudaStream_t s);
template <typename TW>
cudaError_t copy_to_store(const float *master, TW *wstore, long long len, cudaStream_t s);

template <typename T>
cudaError_t features(const double *ra, const int *wall, T *out, int batch, int n, cudaStream_t s);

// trilinear resampling of one channels-last sample [m^3][c] (c <= 5) to
// planar fields: channel k into plane[k] of out, as scale[k] * v + offset[k]
template <typename T>
cudaError_t resample(const T *in, int m, int c, float *out, int N, const int plane[5],
                     const float scale[5], const float offset[5], cudaStream_t s);

// out = bfloat16(in), rounded to nearest
cudaError_t narrow(const float *in, __nv_bfloat16 *out, long long len, cudaStream_t s);
// out = (float) in; p[0..len) = v; training target from planar fields
template <typename T>
cudaError_t widen(const T *in, float *out, long long len, cudaStream_t s);
cudaError_t fill(float *p, float v, long long len, cudaStream_t s);
cudaError_t target_from_fields(const float *u, const float *theta, const float *rho, long long vox,
                               float inv_uc, float *out, cudaStream_t s);

}  // namespace nn
}  // namespace lbm
