// Learned preconditioner: a 3-D convolutional network on the element grid,
// forward and backward, with BF16-stored weights and FP32 accumulation.
//
// It replaces the Teter preconditioner of Sec. II.B (operation 5) in the
// chosen form: inputs are the residual scaled to unit RMS and the local
// potential, 4 layers of 3x3x3 circular convolutions (2 -> 16 -> 16 -> 16
// -> 1 channels) with ReLU between layers; the correction is the output
// times the residual's RMS.  Fields are [sample][channel][z][y][x] in FP32;
// weights [c_out][c_in][27] (tap = 9 dz + 3 dy + dx, offset d - 1 per axis).
//
// Forward: a CTA computes a 4 x 8 x 16 tile of output points for every
// output channel; the input tile with its one-point halo (all input
// channels) and the layer's weights sit in shared memory.  The data
// gradient is the same convolution with flipped taps and swapped channels.
// Weight gradients reduce per CTA over its tile and then over CTAs in a
// fixed order.
#include <cuda_bf16.h>

#include <algorithm>

#include "convnet.h"
#include "internal.h"

namespace dgdft {

namespace {

constexpr int TZ = 4, TY = 8, TX = 16;                 // output tile
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;   // with halo
constexpr int HPTS = HZ * HY * HX;
constexpr int CT = TZ * TY * TX;                       // threads per CTA (512)

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// out[b][co][p] = act(bias[co] + sum_{ci,tap} w[co][ci][tap] in[b][ci][p + off(tap)])
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(CT) conv_fwd_kernel(const float* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ bias, float* __restrict__ out,
                                                      int nz, int ny, int nx) {
  __shared__ float xs[CIN][HPTS];
  __shared__ float ws[CIN * 27][COUT];
  const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + TY - 1) / TY;
  int t = blockIdx.x;
  const int bx = t % tiles_x;
  t /= tiles_x;
  const int by = t % tiles_y;
  const int bz = t / tiles_y;
  const int b = blockIdx.y;
  const size_t npts = (size_t)nz * ny * nx;
  const float* inb = in + (size_t)b * CIN * npts;
  const int z0 = bz * TZ, y0 = by * TY, x0 = bx * TX;
  for (int i = threadIdx.x; i < CIN * 27 * COUT; i += CT) {
    const int co = i / (CIN * 27), r = i - co * (CIN * 27);
    ws[r][co] = __bfloat162float(w[i]);
  }
  for (int i = threadIdx.x; i < CIN * HPTS; i += CT) {
    const int ci = i / HPTS, h = i - ci * HPTS;
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    const int gz = wrap(z0 + hz - 1, nz), gy = wrap(y0 + hy - 1, ny), gx = wrap(x0 + hx - 1, nx);
    xs[ci][h] = inb[(size_t)ci * npts + ((size_t)gz * ny + gy) * nx + gx];
  }
  __syncthreads();
  const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
  const int z = z0 + lz, y = y0 + ly, x = x0 + lx;
  if (z >= nz || y >= ny || x >= nx) return;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = bias[co];
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) {
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      const float v = xs[ci][((lz + dz) * HY + (ly + dy)) * HX + (lx + dx)];
      const float* wr = ws[ci * 27 + tap];
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wr[co], v, acc[co]);
    }
  }
  float* ob = out + (size_t)b * COUT * npts + ((size_t)z * ny + y) * nx + x;
#pragma unroll
  for (int co = 0; co < COUT; ++co) ob[(size_t)co * npts] = RELU ? fmaxf(acc[co], 0.f) : acc[co];
}

// gW[co][ci][tap] partial over one tile: sum_p gout[b][co][p] x[b][ci][p + off(tap)].
// One thread per (co, ci) pair (and the bias gradient for ci == 0).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const float* __restrict__ x, const float* __restrict__ gout,
                                                         float* __restrict__ partial, int nz, int ny, int nx) {
  __shared__ float xs[CIN][HPTS];
  __shared__ float gs[COUT][CT];
  const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + TY - 1) / TY;
  const int tiles_z = (nz + TZ - 1) / TZ;
  int t = blockIdx.x;
  const int bx = t % tiles_x;
  t /= tiles_x;
  const int by = t % tiles_y;
  const int bz = t / tiles_y;
  const int b = blockIdx.y;
  const size_t npts = (size_t)nz * ny * nx;
  const int z0 = bz * TZ, y0 = by * TY, x0 = bx * TX;
  for (int i = threadIdx.x; i < CIN * HPTS; i += blockDim.x) {
    const int ci = i / HPTS, h = i - ci * HPTS;
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    const int gz = wrap(z0 + hz - 1, nz), gy = wrap(y0 + hy - 1, ny), gx = wrap(x0 + hx - 1, nx);
    xs[ci][h] = x[(size_t)b * CIN * npts + (size_t)ci * npts + ((size_t)gz * ny + gy) * nx + gx];
  }
  for (int i = threadIdx.x; i < COUT * CT; i += blockDim.x) {
    const int co = i / CT, p = i - co * CT;
    const int lx = p % TX, ly = (p / TX) % TY, lz = p / (TX * TY);
    const int z = z0 + lz, y = y0 + ly, xx = x0 + lx;
    gs[co][p] = (z < nz && y < ny && xx < nx)
                    ? gout[(size_t)b * COUT * npts + (size_t)co * npts + ((size_t)z * ny + y) * nx + xx]
                    : 0.f;
  }
  __syncthreads();
  const int nw = COUT * CIN * 27 + COUT;
  float* pout = partial + ((size_t)b * (gridDim.x) + blockIdx.x) * nw;
  for (int pair = threadIdx.x; pair < COUT * CIN; pair += blockDim.x) {
    const int co = pair / CIN, ci = pair - co * CIN;
    float acc[27];
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) acc[tap] = 0.f;
    float gb = 0.f;
    for (int p = 0; p < CT; ++p) {
      const float g = gs[co][p];
      const int lx = p % TX, ly = (p / TX) % TY, lz = p / (TX * TY);
      gb += g;
#pragma unroll
      for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        acc[tap] = fmaf(g, xs[ci][((lz + dz) * HY + (ly + dy)) * HX + (lx + dx)], acc[tap]);
      }
    }
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) pout[(co * CIN + ci) * 27 + tap] = acc[tap];
    if (ci == 0) pout[COUT * CIN * 27 + co] = gb;
  }
  (void)tiles_z;
}

__global__ void sum_partials_kernel(const float* __restrict__ partial, int nparts, int nw, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += partial[(size_t)p * nw + i];
    out[i] = (float)s;
  }
}

// Weights of the data-gradient convolution: wt[ci][co][26 - tap] = w[co][ci][tap].
__global__ void flip_weights_kernel(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int cin,
                                    int cout) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cin * cout * 27; i += gridDim.x * blockDim.x) {
    const int co = i / (cin * 27), r = i - co * cin * 27, ci = r / 27, tap = r - ci * 27;
    wt[(ci * cout + co) * 27 + (26 - tap)] = w[i];
  }
}

__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ act, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(act[i] > 0.f)) g[i] = 0.f;
}

// loss partials and gout = 2 (out - tgt) / count over the interior window
// [lo, hi) of every axis of the crop (sample b).
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ tgt, float* __restrict__ gout,
                           double* __restrict__ loss_part, int nz, int ny, int nx, int lo, int hi, double inv_count) {
  const size_t npts = (size_t)nz * ny * nx;
  const int b = blockIdx.y;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
    const bool in = x >= lo && x < hi && y >= lo && y < hi && z >= lo && z < hi;
    const size_t k = (size_t)b * npts + i;
    const float d = in ? out[k] - tgt[k] : 0.f;
    gout[k] = (float)(2.0 * inv_count) * d;
    s += (double)d * d;
  }
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    loss_part[(size_t)b * gridDim.x + blockIdx.x] = t * inv_count;
  }
}

// Adam on FP32 master weights; the BF16 copy is what the network reads.
__global__ void adam_kernel(float* __restrict__ master, __nv_bfloat16* __restrict__ wbf, float* __restrict__ bias_dst,
                            const float* __restrict__ grad, float* __restrict__ m1, float* __restrict__ m2, int n,
                            int nweights, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float v = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    const float p = master[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    master[i] = p;
    if (i < nweights)
      wbf[i] = __float2bfloat16_rn(p);
    else
      bias_dst[i - nweights] = p;
  }
}

template <int CIN, int COUT, bool RELU>
void fwd_t(const float* in, const __nv_bfloat16* w, const float* b, float* out, int B, int nz, int ny, int nx,
           cudaStream_t st) {
  const int tiles = ((nz + TZ - 1) / TZ) * ((ny + TY - 1) / TY) * ((nx + TX - 1) / TX);
  conv_fwd_kernel<CIN, COUT, RELU><<<dim3(tiles, B), CT, 0, st>>>(in, w, b, out, nz, ny, nx);
}

template <int CIN, int COUT>
void wgrad_t(const float* x, const float* g, float* partial, float* out, int B, int nz, int ny, int nx,
             cudaStream_t st) {
  const int tiles = ((nz + TZ - 1) / TZ) * ((ny + TY - 1) / TY) * ((nx + TX - 1) / TX);
  conv_wgrad_kernel<CIN, COUT><<<dim3(tiles, B), 256, 0, st>>>(x, g, partial, nz, ny, nx);
  const int nw = COUT * CIN * 27 + COUT;
  sum_partials_kernel<<<(nw + 255) / 256, 256, 0, st>>>(partial, tiles * B, nw, out);
}

}  // namespace

const int kConvChannels[kConvLayers + 1] = {2, 16, 16, 16, 1};

size_t conv_param_count(int layer) {
  return (size_t)kConvChannels[layer + 1] * kConvChannels[layer] * 27 + kConvChannels[layer + 1];
}

void conv_forward(int layer, const float* in, const __nv_bfloat16* w, const float* b, float* out, int B, int nz,
                  int ny, int nx, cudaStream_t st) {
  switch (layer) {
    case 0: fwd_t<2, 16, true>(in, w, b, out, B, nz, ny, nx, st); break;
    case 1: fwd_t<16, 16, true>(in, w, b, out, B, nz, ny, nx, st); break;
    case 2: fwd_t<16, 16, true>(in, w, b, out, B, nz, ny, nx, st); break;
    default: fwd_t<16, 1, false>(in, w, b, out, B, nz, ny, nx, st); break;
  }
}

// gx = conv^T(gout): forward convolution with flipped, transposed weights
// and no bias (bias_zero must hold >= 16 zeros).
void conv_backward_data(int layer, const float* gout, const __nv_bfloat16* wflip, const float* bias_zero, float* gx,
                        int B, int nz, int ny, int nx, cudaStream_t st) {
  // layer l maps C_l -> C_{l+1}; its data gradient maps C_{l+1} -> C_l
  switch (layer) {
    case 0: fwd_t<16, 2, false>(gout, wflip, bias_zero, gx, B, nz, ny, nx, st); break;
    case 1: fwd_t<16, 16, false>(gout, wflip, bias_zero, gx, B, nz, ny, nx, st); break;
    case 2: fwd_t<16, 16, false>(gout, wflip, bias_zero, gx, B, nz, ny, nx, st); break;
    default: fwd_t<1, 16, false>(gout, wflip, bias_zero, gx, B, nz, ny, nx, st); break;
  }
}

void conv_flip_weights(int layer, const __nv_bfloat16* w, __nv_bfloat16* wflip, cudaStream_t st) {
  const int ci = kConvChannels[layer], co = kConvChannels[layer + 1];
  flip_weights_kernel<<<(ci * co * 27 + 255) / 256, 256, 0, st>>>(w, wflip, ci, co);
}

size_t conv_wgrad_partial_floats(int B, int nz, int ny, int nx) {
  const size_t tiles = (size_t)((nz + TZ - 1) / TZ) * ((ny + TY - 1) / TY) * ((nx + TX - 1) / TX);
  return tiles * B * (16 * 16 * 27 + 16);
}

void conv_backward_weights(int layer, const float* x, const float* gout, float* partial, float* grad, int B, int nz,
                           int ny, int nx, cudaStream_t st) {
  switch (layer) {
    case 0: wgrad_t<2, 16>(x, gout, partial, grad, B, nz, ny, nx, st); break;
    case 1: wgrad_t<16, 16>(x, gout, partial, grad, B, nz, ny, nx, st); break;
    case 2: wgrad_t<16, 16>(x, gout, partial, grad, B, nz, ny, nx, st); break;
    default: wgrad_t<16, 1>(x, gout, partial, grad, B, nz, ny, nx, st); break;
  }
}

void conv_relu_mask(float* g, const float* act, size_t n, cudaStream_t st) {
  size_t blocks = std::min<size_t>((n + 255) / 256, 8192);
  relu_mask_kernel<<<(unsigned)blocks, 256, 0, st>>>(g, act, n);
}

void conv_mse(const float* out, const float* tgt, float* gout, double* loss_part, int B, int nz, int ny, int nx,
              int lo, int hi, int nblocks, cudaStream_t st) {
  const double count = (double)B * (hi - lo) * (hi - lo) * (hi - lo);
  mse_kernel<<<dim3(nblocks, B), 256, 0, st>>>(out, tgt, gout, loss_part, nz, ny, nx, lo, hi, 1.0 / count);
}

void conv_adam(float* master, __nv_bfloat16* wbf, float* bias, const float* grad, float* m1, float* m2, int n,
               int nweights, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(master, wbf, bias, grad, m1, m2, n, nweights, lr, b1, b2, 1e-8f, c1,
                                               c2);
}

}  // namespace dgdft
