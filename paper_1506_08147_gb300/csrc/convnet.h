// Host interface of the learned-preconditioner network kernels (convnet.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace dgdft {

constexpr int kConvLayers = 4;
extern const int kConvChannels[kConvLayers + 1];  // 2, 16, 16, 16, 1

// weights + biases of layer l: c_out * c_in * 27 + c_out
size_t conv_param_count(int layer);

// Layer l forward on B samples of nz x ny x nx, ReLU on all but the last.
void conv_forward(int layer, const float* in, const __nv_bfloat16* w, const float* b, float* out, int B, int nz,
                  int ny, int nx, cudaStream_t st);
// Data gradient of layer l (1..3) or the input gradient of layer 0 (unused).
void conv_backward_data(int layer, const float* gout, const __nv_bfloat16* wflip, const float* bias_zero, float* gx,
                        int B, int nz, int ny, int nx, cudaStream_t st);
void conv_flip_weights(int layer, const __nv_bfloat16* w, __nv_bfloat16* wflip, cudaStream_t st);
size_t conv_wgrad_partial_floats(int B, int nz, int ny, int nx);
// Weight and bias gradients of layer l into grad (c_out*c_in*27 weights, then c_out biases).
void conv_backward_weights(int layer, const float* x, const float* gout, float* partial, float* grad, int B, int nz,
                           int ny, int nx, cudaStream_t st);
void conv_relu_mask(float* g, const float* act, size_t n, cudaStream_t st);
void conv_mse(const float* out, const float* tgt, float* gout, double* loss_part, int B, int nz, int ny, int nx,
              int lo, int hi, int nblocks, cudaStream_t st);
void conv_adam(float* master, __nv_bfloat16* wbf, float* bias, const float* grad, float* m1, float* m2, int n,
               int nweights, float lr, int step, cudaStream_t st);

}  // namespace dgdft
