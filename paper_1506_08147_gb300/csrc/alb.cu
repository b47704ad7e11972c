// Restriction of Ritz vectors to the element and precision conversions.
//
// Sec. II.A / Sec. II.B: the lowest J_K eigenvectors on Q_K are restricted to
// E_K before orthonormalisation.  The gather reads the E_K sub-box of each of
// the first J columns (x fastest) and writes an n_E x J FP64 block.
#include "internal.h"

namespace dgdft {

namespace {

template <class real>
__global__ void restrict_kernel(const real* __restrict__ x, int ng, int nx, int ny, int lo0, int lo1,
                                int lo2, int ex, int ey, int ez, int J, double* __restrict__ out) {
  const int ne = ex * ey * ez;
  const int j = blockIdx.y;
  if (j >= J) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ne; t += gridDim.x * blockDim.x) {
    const int i = t % ex;
    const int r = t / ex;
    const int jy = r % ey, kz = r / ey;
    const size_t g = (size_t)(lo0 + i) + (size_t)nx * ((lo1 + jy) + (size_t)ny * (lo2 + kz));
    out[t + (size_t)j * ne] = (double)x[g + (size_t)j * ng];
  }
}

template <class A, class B>
__global__ void convert_kernel(const A* __restrict__ in, B* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

__global__ void scale_kernel(double* __restrict__ x, size_t n, double s) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

__global__ void nonfinite_kernel(const double* __restrict__ x, size_t n, int* __restrict__ flag) {
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Orthonormalisation products, all elements of a wave in one launch each.
// Gram: each CTA sums a 32 x 32 tile of A^T A over one chunk of rows (2 x 2
// outputs per thread); the chunk partials are reduced in a fixed order.
constexpr int OT = 32;

__global__ void __launch_bounds__(256) ortho_gram_kernel(const OrthoTask* __restrict__ tasks, int tiles, int chunk,
                                                         double* __restrict__ partial) {
  const OrthoTask T = tasks[blockIdx.z];
  const int ti = blockIdx.y / tiles, tj = blockIdx.y - ti * tiles;
  const int i0 = ti * OT, j0 = tj * OT;
  __shared__ double As[OT][OT + 1], Bs[OT][OT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  const int k_beg = blockIdx.x * chunk, k_end = min(T.rows, k_beg + chunk);
  if (i0 < T.J && j0 < T.J) {
    for (int k0 = k_beg; k0 < k_end; k0 += OT) {
      for (int idx = threadIdx.x; idx < OT * OT; idx += blockDim.x) {
        const int c = idx / OT, r = idx - c * OT;
        const int k = k0 + r;
        As[r][c] = (k < k_end && i0 + c < T.J) ? T.a[k + (size_t)(i0 + c) * T.rows] : 0.0;
        Bs[r][c] = (k < k_end && j0 + c < T.J) ? T.a[k + (size_t)(j0 + c) * T.rows] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int r = 0; r < OT; ++r) {
        const double a0 = As[r][2 * ty], a1 = As[r][2 * ty + 1];
        const double b0 = Bs[r][2 * tx], b1 = Bs[r][2 * tx + 1];
        acc[0][0] += a0 * b0;
        acc[0][1] += a0 * b1;
        acc[1][0] += a1 * b0;
        acc[1][1] += a1 * b1;
      }
      __syncthreads();
    }
  }
  double* out = partial + (((size_t)blockIdx.z * gridDim.x + blockIdx.x) * gridDim.y + blockIdx.y) * (OT * OT);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) out[(2 * ty + a) * OT + 2 * tx + b] = acc[a][b];
}

__global__ void ortho_gram_reduce_kernel(const OrthoTask* __restrict__ tasks, int tiles, int nchunk,
                                         const double* __restrict__ partial) {
  const OrthoTask T = tasks[blockIdx.z];
  const int ti = blockIdx.x / tiles, tj = blockIdx.x - ti * tiles;
  for (int idx = threadIdx.x; idx < OT * OT; idx += blockDim.x) {
    const int r = idx / OT, c = idx - r * OT;
    const int i = ti * OT + r, j = tj * OT + c;
    if (i >= T.J || j >= T.J) continue;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch)
      s += partial[(((size_t)blockIdx.z * nchunk + ch) * (tiles * tiles) + blockIdx.x) * (OT * OT) + idx];
    T.out[i + (size_t)j * T.J] = s;
  }
}

// out = A Y (rows x K times K x J): a thread per row, 32 output columns per
// CTA, the Y columns staged in shared memory.
__global__ void __launch_bounds__(256) ortho_apply_kernel(const OrthoTask* __restrict__ tasks) {
  const OrthoTask T = tasks[blockIdx.z];
  const int c0 = blockIdx.y * OT;
  if (c0 >= T.J) return;
  const int K = T.K > 0 ? T.K : T.J;
  extern __shared__ double ys[];  // K x OT
  for (int idx = threadIdx.x; idx < K * OT; idx += blockDim.x) {
    const int k = idx / OT, c = idx - k * OT;
    ys[idx] = (c0 + c < T.J) ? T.y[k + (size_t)(c0 + c) * K] : 0.0;
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= T.rows) return;
  double acc[OT];
#pragma unroll
  for (int c = 0; c < OT; ++c) acc[c] = 0.0;
  for (int k = 0; k < K; ++k) {
    const double a = T.a[r + (size_t)k * T.rows];
#pragma unroll
    for (int c = 0; c < OT; ++c) acc[c] += a * ys[k * OT + c];
  }
  const int nc = min(OT, T.J - c0);
  for (int c = 0; c < nc; ++c) T.out[r + (size_t)(c0 + c) * T.rows] = acc[c];
}

}  // namespace

size_t ortho_partial_doubles(int ntask, int max_rows, int max_J) {
  const int tiles = (max_J + OT - 1) / OT;
  const int nchunk = (max_rows + ORTHO_CHUNK - 1) / ORTHO_CHUNK;
  return (size_t)ntask * nchunk * tiles * tiles * OT * OT;
}

void launch_ortho_gram(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, double* partial,
                       cudaStream_t st) {
  if (ntask <= 0) return;
  const int tiles = (max_J + OT - 1) / OT;
  const int nchunk = (max_rows + ORTHO_CHUNK - 1) / ORTHO_CHUNK;
  ortho_gram_kernel<<<dim3(nchunk, tiles * tiles, ntask), 256, 0, st>>>(d_tasks, tiles, ORTHO_CHUNK, partial);
  ortho_gram_reduce_kernel<<<dim3(tiles * tiles, 1, ntask), 256, 0, st>>>(d_tasks, tiles, nchunk, partial);
}

void launch_ortho_apply(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, int max_K, cudaStream_t st) {
  if (ntask <= 0) return;
  const size_t smem = sizeof(double) * (size_t)(max_K > max_J ? max_K : max_J) * OT;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute((const void*)ortho_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ortho_apply_kernel<<<dim3((max_rows + 255) / 256, (max_J + OT - 1) / OT, ntask), 256, smem, st>>>(d_tasks);
}

void launch_nonfinite(const double* x, size_t n, int* flag, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  nonfinite_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, flag);
}

template <class real>
void launch_restrict(const real* x, int ng, int nx, int ny, const int* lo, const int* hi, int J, double* out,
                     cudaStream_t st) {
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int ne = ex * ey * ez;
  const int bx = (ne + 255) / 256 < 64 ? (ne + 255) / 256 : 64;
  restrict_kernel<real><<<dim3(bx, J), 256, 0, st>>>(x, ng, nx, ny, lo[0], lo[1], lo[2], ex, ey, ez, J, out);
}

template <class A, class B>
void launch_convert(const A* in, B* out, size_t n, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  convert_kernel<A, B><<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
}

void launch_scale(double* x, size_t n, double s, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  scale_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, s);
}

template void launch_restrict<double>(const double*, int, int, int, const int*, const int*, int, double*,
                                      cudaStream_t);
template void launch_restrict<float>(const float*, int, int, int, const int*, const int*, int, double*,
                                     cudaStream_t);
template void launch_convert<double, float>(const double*, float*, size_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, size_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, size_t, cudaStream_t);

}  // namespace dgdft
