// Parameters, training and inference of the learned preconditioner network.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "convnet.h"

namespace dgdft {

// All parameters concatenated per layer: weights (c_out x c_in x 27) then
// biases (c_out); 15,169 floats for the 2-16-16-16-1 network.
size_t convnet_total_params();

struct ConvNet {
  float* master[kConvLayers] = {};      // FP32 master copy (weights then bias)
  __nv_bfloat16* wbf[kConvLayers] = {};  // BF16 weights the kernels read
  float* bias[kConvLayers] = {};
  __nv_bfloat16* wflip[kConvLayers] = {};
  float* grad[kConvLayers] = {};
  float* m1[kConvLayers] = {};
  float* m2[kConvLayers] = {};
  float* bias_zero = nullptr;
  int step = 0;
  bool ready = false;

  ~ConvNet();
  // Allocate; He-normal weights from a seeded generator, zero biases.
  std::string init(uint64_t seed, cudaStream_t st);
  std::string set_params(const float* host, cudaStream_t st);
  std::string get_params(float* host, cudaStream_t st);
  std::string load_file(const char* path, cudaStream_t st);
  std::string save_file(const char* path, cudaStream_t st);
  // Forward on B samples (2 input channels each) of nz x ny x nx.  acts[0..2]
  // receive the hidden activations (B x 16 fields each) when non-null,
  // otherwise ping-pong between tmp0 and tmp1.
  void forward(const float* in, float* out, int B, int nz, int ny, int nx, float* const* acts, float* tmp0,
               float* tmp1, cudaStream_t st);
  // Loss over the interior [lo, hi) window and parameter gradients (into grad[]).
  std::string loss_and_grad(const float* in, const float* tgt, int B, int nz, int ny, int nx, int lo, int hi,
                            double* loss, cudaStream_t st);
  void adam(float lr, cudaStream_t st);
};

// Column-wise FP64 helpers for the CG solves that make training targets:
// out[j] = a_j . b_j (part: 64 * k doubles of scratch), y_j = alpha_j x_j + beta_j y_j.
void col_dot(const double* a, const double* b, int n, int k, double* part, double* out, cudaStream_t st);
void col_axpby(const double* alpha, const double* x, const double* beta, double* y, int n, int k, cudaStream_t st);

// W = rms(R) * net(R / rms(R), V) for every column of every element of the
// batch that uses the network (all elements share the grid nz x ny x nx);
// in: nel*m*2*N_g, out: nel*m*N_g, tmp0/tmp1: nel*m*16*N_g floats.
template <class real> struct Batch;
void learned_precondition(const Batch<float>& b, ConvNet& net, int nchunk, int nz, int ny, int nx, float* in,
                          float* out, float* tmp0, float* tmp1, cudaStream_t st);

void cg_alpha(const double* rr, const double* pap, double* alpha, double* nalpha, int k, cudaStream_t st);
void cg_beta(double* rr, const double* rrn, double* beta, int k, cudaStream_t st);
// rms[f] = sqrt(mean r_f^2) (1 for an all-zero field)
void field_rms(const float* r, int nfields, size_t npts, float* rms, cudaStream_t st);

// Gather B crops of edge c from fields (periodic wrap): input channels
// (r / rms, V) and target t / rms; offsets are (field, oz, oy, ox) per crop.
void gather_crops(const float* r, const float* v, const float* t, const float* rms, const int* offsets, int B,
                  int c, int nz, int ny, int nx, float* in, float* tgt, cudaStream_t st);

}  // namespace dgdft
