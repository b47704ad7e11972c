// Learned preconditioner network: parameters, training step, inference.
//
// Training (chosen-form preconditioner): mean squared error between the
// network output on (r / rms(r), V) and the exact correction t / rms(r),
// t solving (H - sigma I) t = r, on crops of edge c cut from full fields with
// periodic wrap; the loss is taken on the interior [4, c - 4) of each crop,
// where the 9-point receptive field of the 4 layers lies inside the crop.
// Adam updates an FP32 master copy; the kernels read a BF16 copy.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "internal.h"
#include "learned.h"

namespace dgdft {

namespace {

__global__ void gather_crops_kernel(const float* __restrict__ r, const float* __restrict__ v,
                                    const float* __restrict__ t, const float* __restrict__ rms,
                                    const int* __restrict__ offs, int c, int nz, int ny, int nx,
                                    float* __restrict__ in, float* __restrict__ tgt) {
  const int b = blockIdx.y;
  const int f = offs[4 * b], oz = offs[4 * b + 1], oy = offs[4 * b + 2], ox = offs[4 * b + 3];
  const size_t npts = (size_t)nz * ny * nx;
  const size_t cpts = (size_t)c * c * c;
  const float inv = 1.f / rms[f];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cpts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % c), y = (int)((i / c) % c), z = (int)(i / ((size_t)c * c));
    const int gz = (oz + z) % nz, gy = (oy + y) % ny, gx = (ox + x) % nx;
    const size_t g = ((size_t)gz * ny + gy) * nx + gx;
    in[(size_t)b * 2 * cpts + i] = r[(size_t)f * npts + g] * inv;
    in[(size_t)b * 2 * cpts + cpts + i] = v[(size_t)f * npts + g];
    tgt[(size_t)b * cpts + i] = t[(size_t)f * npts + g] * inv;
  }
}

struct Work {
  float* buf = nullptr;
  size_t cap = 0;
  float* get(size_t n) {
    if (n > cap) {
      if (buf) cudaFree(buf);
      buf = nullptr;
      if (cudaMalloc(&buf, n * sizeof(float)) != cudaSuccess) {
        cap = 0;
        return nullptr;
      }
      cap = n;
    }
    return buf;
  }
};

Work g_work;

// part[chunk][j] = sum over the chunk's rows of a_j . b_j (k columns of n rows)
__global__ void col_dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int n, int k,
                               double* __restrict__ part) {
  const int j = blockIdx.y;
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int beg = blockIdx.x * chunk, end = min(n, beg + chunk);
  double s = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) s += a[(size_t)j * n + i] * b[(size_t)j * n + i];
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(size_t)blockIdx.x * k + j] = t;
  }
}

__global__ void col_dot_reduce_kernel(const double* __restrict__ part, int nchunk, int k, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * k + j];
  out[j] = s;
}

// y_j = alpha_j x_j + beta_j y_j (alpha, beta device arrays; nullptr = 1)
__global__ void col_axpby_kernel(const double* __restrict__ alpha, const double* __restrict__ x,
                                 const double* __restrict__ beta, double* __restrict__ y, int n, int k) {
  const size_t total = (size_t)n * k;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / n);
    const double a = alpha ? alpha[j] : 1.0, bb = beta ? beta[j] : 1.0;
    y[i] = a * x[i] + bb * y[i];
  }
}

// CG scalars per column: alpha = rr / pAp (0 when pAp <= 0), nalpha = -alpha.
__global__ void cg_alpha_kernel(const double* __restrict__ rr, const double* __restrict__ pap,
                                double* __restrict__ alpha, double* __restrict__ nalpha, int k) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const double a = (pap[j] > 0.0) ? rr[j] / pap[j] : 0.0;
  alpha[j] = a;
  nalpha[j] = -a;
}

// beta = rr_new / rr, then rr <- rr_new.
__global__ void cg_beta_kernel(double* __restrict__ rr, const double* __restrict__ rrn, double* __restrict__ beta,
                               int k) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  beta[j] = (rr[j] > 0.0) ? rrn[j] / rr[j] : 0.0;
  rr[j] = rrn[j];
}

__global__ void field_rms_kernel(const float* __restrict__ r, size_t npts, float* __restrict__ rms) {
  const int f = blockIdx.x;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < npts; i += blockDim.x) {
    const double v = r[(size_t)f * npts + i];
    s += v * v;
  }
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const double v = sqrt(t / (double)npts);
    rms[f] = (float)(v > 0.0 ? v : 1.0);
  }
}

__device__ __forceinline__ float residual_rms(const ElemDev<float>& e, int j, int nchunk) {
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += e.rpart[((size_t)j * nchunk + c) * 4];
  const double r = sqrt(s / (double)e.ng);
  return (float)(r > 0.0 ? r : 1.0);
}

// Network input for column j of element z (sample z * m_max + j): the
// residual (in the W block) over its RMS, and V_eff.
__global__ void pack_kernel(const ElemDev<float>* __restrict__ elems, int nchunk, int m_max, int ng,
                            float* __restrict__ in) {
  const ElemDev<float>& e = elems[blockIdx.z];
  const int j = blockIdx.y;
  if (!e.state[ST_ACTIVE] || e.state[ST_TETER] || j >= e.m) return;
  const float inv = 1.f / residual_rms(e, j, nchunk);
  const float* r = e.blk[BW][0] + (size_t)j * e.ng;
  float* dst = in + ((size_t)blockIdx.z * m_max + j) * 2 * ng;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < e.ng; p += gridDim.x * blockDim.x) {
    dst[p] = r[p] * inv;
    dst[ng + p] = e.V[p];
  }
}

// W_j = rms(r_j) * network output.
__global__ void unpack_kernel(const ElemDev<float>* __restrict__ elems, int nchunk, int m_max, int ng,
                              const float* __restrict__ out) {
  const ElemDev<float>& e = elems[blockIdx.z];
  const int j = blockIdx.y;
  if (!e.state[ST_ACTIVE] || e.state[ST_TETER] || j >= e.m) return;
  const float s = residual_rms(e, j, nchunk);
  float* w = e.blk[BW][0] + (size_t)j * e.ng;
  const float* src = out + ((size_t)blockIdx.z * m_max + j) * ng;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < e.ng; p += gridDim.x * blockDim.x) w[p] = s * src[p];
}

}  // namespace

void learned_precondition(const Batch<float>& b, ConvNet& net, int nchunk, int nz, int ny, int nx, float* in,
                          float* out, float* tmp0, float* tmp1, cudaStream_t st) {
  const int ng = nz * ny * nx;
  const int m = b.s.max_m;
  pack_kernel<<<dim3(32, m, b.s.nel), 256, 0, st>>>(b.d_elems, nchunk, m, ng, in);
  net.forward(in, out, b.s.nel * m, nz, ny, nx, nullptr, tmp0, tmp1, st);
  unpack_kernel<<<dim3(32, m, b.s.nel), 256, 0, st>>>(b.d_elems, nchunk, m, ng, out);
}

void cg_alpha(const double* rr, const double* pap, double* alpha, double* nalpha, int k, cudaStream_t st) {
  cg_alpha_kernel<<<(k + 127) / 128, 128, 0, st>>>(rr, pap, alpha, nalpha, k);
}
void cg_beta(double* rr, const double* rrn, double* beta, int k, cudaStream_t st) {
  cg_beta_kernel<<<(k + 127) / 128, 128, 0, st>>>(rr, rrn, beta, k);
}
void field_rms(const float* r, int nfields, size_t npts, float* rms, cudaStream_t st) {
  field_rms_kernel<<<nfields, 256, 0, st>>>(r, npts, rms);
}

void col_dot(const double* a, const double* b, int n, int k, double* part, double* out, cudaStream_t st) {
  const int nchunk = 64;
  col_dot_kernel<<<dim3(nchunk, k), 256, 0, st>>>(a, b, n, k, part);
  col_dot_reduce_kernel<<<(k + 127) / 128, 128, 0, st>>>(part, nchunk, k, out);
}

void col_axpby(const double* alpha, const double* x, const double* beta, double* y, int n, int k, cudaStream_t st) {
  size_t blocks = std::min<size_t>(((size_t)n * k + 255) / 256, 8192);
  col_axpby_kernel<<<(unsigned)blocks, 256, 0, st>>>(alpha, x, beta, y, n, k);
}

size_t convnet_total_params() {
  size_t n = 0;
  for (int l = 0; l < kConvLayers; ++l) n += conv_param_count(l);
  return n;
}

void gather_crops(const float* r, const float* v, const float* t, const float* rms, const int* offsets, int B,
                  int c, int nz, int ny, int nx, float* in, float* tgt, cudaStream_t st) {
  gather_crops_kernel<<<dim3(64, B), 256, 0, st>>>(r, v, t, rms, offsets, c, nz, ny, nx, in, tgt);
}

ConvNet::~ConvNet() {
  for (int l = 0; l < kConvLayers; ++l) {
    for (void* p : {(void*)master[l], (void*)wbf[l], (void*)bias[l], (void*)wflip[l], (void*)grad[l], (void*)m1[l],
                    (void*)m2[l]})
      if (p) cudaFree(p);
  }
  if (bias_zero) cudaFree(bias_zero);
}

std::string ConvNet::init(uint64_t seed, cudaStream_t st) {
  for (int l = 0; l < kConvLayers; ++l) {
    const size_t n = conv_param_count(l);
    const size_t nw = n - kConvChannels[l + 1];
    if (cudaMalloc(&master[l], n * 4) || cudaMalloc(&wbf[l], nw * 2) || cudaMalloc(&bias[l], kConvChannels[l + 1] * 4) ||
        cudaMalloc(&wflip[l], nw * 2) || cudaMalloc(&grad[l], n * 4) || cudaMalloc(&m1[l], n * 4) ||
        cudaMalloc(&m2[l], n * 4))
      return "network allocation failed";
    cudaMemsetAsync(m1[l], 0, n * 4, st);
    cudaMemsetAsync(m2[l], 0, n * 4, st);
  }
  if (cudaMalloc(&bias_zero, 16 * 4)) return "network allocation failed";
  cudaMemsetAsync(bias_zero, 0, 16 * 4, st);
  std::mt19937_64 gen(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<float> host(convnet_total_params());
  size_t off = 0;
  for (int l = 0; l < kConvLayers; ++l) {
    const int ci = kConvChannels[l], co = kConvChannels[l + 1];
    const double s = std::sqrt(2.0 / (27.0 * ci));
    for (int i = 0; i < co * ci * 27; ++i) host[off++] = (float)(s * nd(gen));
    for (int i = 0; i < co; ++i) host[off++] = 0.f;
  }
  step = 0;
  ready = true;
  return set_params(host.data(), st);
}

__global__ void split_params_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ w, float* __restrict__ b,
                                    int nw, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < nw)
      w[i] = __float2bfloat16_rn(p[i]);
    else
      b[i - nw] = p[i];
  }
}

std::string ConvNet::set_params(const float* host, cudaStream_t st) {
  size_t off = 0;
  for (int l = 0; l < kConvLayers; ++l) {
    const size_t n = conv_param_count(l);
    const int nw = (int)(n - kConvChannels[l + 1]);
    if (cudaMemcpyAsync(master[l], host + off, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return "parameter upload failed";
    split_params_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(master[l], wbf[l], bias[l], nw, (int)n);
    conv_flip_weights(l, wbf[l], wflip[l], st);
    off += n;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return "parameter upload failed";
  return "";
}

std::string ConvNet::get_params(float* host, cudaStream_t st) {
  size_t off = 0;
  for (int l = 0; l < kConvLayers; ++l) {
    const size_t n = conv_param_count(l);
    if (cudaMemcpyAsync(host + off, master[l], n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return "parameter download failed";
    off += n;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return "parameter download failed";
  return "";
}

// File: 8-byte magic "DGALBNN1", int32 layer count, per layer int32 c_in,
// c_out, then the concatenated float32 parameters (weights then biases).
std::string ConvNet::save_file(const char* path, cudaStream_t st) {
  std::vector<float> host(convnet_total_params());
  std::string e = get_params(host.data(), st);
  if (!e.empty()) return e;
  FILE* f = std::fopen(path, "wb");
  if (!f) return std::string("cannot open ") + path;
  const char magic[8] = {'D', 'G', 'A', 'L', 'B', 'N', 'N', '1'};
  int32_t nl = kConvLayers;
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&nl, 4, 1, f) == 1;
  for (int l = 0; l < kConvLayers && ok; ++l) {
    int32_t cc[2] = {kConvChannels[l], kConvChannels[l + 1]};
    ok = std::fwrite(cc, 4, 2, f) == 2;
  }
  ok = ok && std::fwrite(host.data(), 4, host.size(), f) == host.size();
  std::fclose(f);
  return ok ? "" : std::string("write failed: ") + path;
}

std::string ConvNet::load_file(const char* path, cudaStream_t st) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return std::string("cannot open ") + path;
  char magic[8];
  int32_t nl = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "DGALBNN1", 8) == 0 &&
            std::fread(&nl, 4, 1, f) == 1 && nl == kConvLayers;
  for (int l = 0; l < kConvLayers && ok; ++l) {
    int32_t cc[2];
    ok = std::fread(cc, 4, 2, f) == 2 && cc[0] == kConvChannels[l] && cc[1] == kConvChannels[l + 1];
  }
  std::vector<float> host(convnet_total_params());
  ok = ok && std::fread(host.data(), 4, host.size(), f) == host.size();
  std::fclose(f);
  if (!ok) return std::string("not a weights file for this network: ") + path;
  for (float v : host)
    if (!std::isfinite(v)) return "non-finite network weight";
  return set_params(host.data(), st);
}

void ConvNet::forward(const float* in, float* out, int B, int nz, int ny, int nx, float* const* acts, float* tmp0,
                      float* tmp1, cudaStream_t st) {
  const float* cur = in;
  for (int l = 0; l < kConvLayers; ++l) {
    float* dst;
    if (l == kConvLayers - 1)
      dst = out;
    else if (acts)
      dst = acts[l];
    else
      dst = (l & 1) ? tmp1 : tmp0;
    conv_forward(l, cur, wbf[l], bias[l], dst, B, nz, ny, nx, st);
    cur = dst;
  }
}

std::string ConvNet::loss_and_grad(const float* in, const float* tgt, int B, int nz, int ny, int nx, int lo, int hi,
                                   double* loss, cudaStream_t st) {
  const size_t pts = (size_t)nz * ny * nx;
  const size_t hid = (size_t)B * 16 * pts;
  const size_t part = conv_wgrad_partial_floats(B, nz, ny, nx);
  const int nblk = 64;
  // workspace: 3 activations, output, gout, 2 gradient fields, partials, loss parts (as doubles)
  float* w = g_work.get(3 * hid + 2 * (size_t)B * pts + 2 * hid + part + 2 * (size_t)B * nblk);
  if (!w) return "network workspace allocation failed";
  float* acts[3] = {w, w + hid, w + 2 * hid};
  float* out = w + 3 * hid;
  float* gout = out + (size_t)B * pts;
  float* ga = gout + (size_t)B * pts;
  float* gb = ga + hid;
  float* partial = gb + hid;
  double* lpart = reinterpret_cast<double*>(partial + part);
  forward(in, out, B, nz, ny, nx, acts, nullptr, nullptr, st);
  conv_mse(out, tgt, gout, lpart, B, nz, ny, nx, lo, hi, nblk, st);
  // layer 3 (16 -> 1)
  conv_backward_weights(3, acts[2], gout, partial, grad[3], B, nz, ny, nx, st);
  conv_backward_data(3, gout, wflip[3], bias_zero, ga, B, nz, ny, nx, st);
  conv_relu_mask(ga, acts[2], hid, st);
  // layers 2, 1 (16 -> 16)
  float* g_in = ga;
  float* g_out = gb;
  for (int l = 2; l >= 1; --l) {
    conv_backward_weights(l, acts[l - 1], g_in, partial, grad[l], B, nz, ny, nx, st);
    conv_backward_data(l, g_in, wflip[l], bias_zero, g_out, B, nz, ny, nx, st);
    conv_relu_mask(g_out, acts[l - 1], hid, st);
    float* tmp = g_in;
    g_in = g_out;
    g_out = tmp;
  }
  conv_backward_weights(0, in, g_in, partial, grad[0], B, nz, ny, nx, st);
  std::vector<double> lp((size_t)B * nblk);
  if (cudaMemcpyAsync(lp.data(), lpart, lp.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return "network loss readback failed";
  double s = 0.0;
  for (double v : lp) s += v;
  *loss = s;
  return "";
}

void ConvNet::adam(float lr, cudaStream_t st) {
  ++step;
  for (int l = 0; l < kConvLayers; ++l) {
    const int n = (int)conv_param_count(l);
    const int nw = n - kConvChannels[l + 1];
    conv_adam(master[l], wbf[l], bias[l], grad[l], m1[l], m2[l], n, nw, lr, step, st);
    conv_flip_weights(l, wbf[l], wflip[l], st);
  }
}

}  // namespace dgdft
