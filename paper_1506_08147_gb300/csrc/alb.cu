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
// Gram G = A^T A over chunks of ORTHO_CHUNK rows: the chunk's rows are staged
// OG_R at a time for every column; each thread owns a 2 x 2 output tile of
// the upper triangle (tiles numbered densely, 256 per CTA, grid.y over groups
// of 256), so no thread computes an output that does not exist; the chunk
// partials are summed in a fixed order and mirrored to the lower triangle.
constexpr int OG_R = 16;

__device__ __forceinline__ void ortho_tile_of(int t, int nt, int* ti, int* tj) {
  int i = 0, base = 0;
  while (t >= base + (nt - i)) {
    base += nt - i;
    ++i;
  }
  *ti = i;
  *tj = i + (t - base);
}

__global__ void __launch_bounds__(256) ortho_gram_kernel(const OrthoTask* __restrict__ tasks, int chunk,
                                                         int nchunk, int ld, size_t stride,
                                                         double* __restrict__ partial) {
  extern __shared__ double As_[];  // OG_R x ld (ld >= the padded J of every task)
  const OrthoTask T = tasks[blockIdx.z];
  const int J = T.J, nt = (J + 1) / 2, ntiles = nt * (nt + 1) / 2;
  const int tile0 = blockIdx.y * 256;
  if (tile0 >= ntiles) return;
  const int mytile = tile0 + threadIdx.x;
  const bool active = mytile < ntiles;
  int ti = 0, tj = 0;
  if (active) ortho_tile_of(mytile, nt, &ti, &tj);
  const int i0 = 2 * ti, j0 = 2 * tj;
  const int k_beg = blockIdx.x * chunk, k_end = min(T.rows, k_beg + chunk);
  const int Jp = (J + 1) & ~1;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
  for (int k0 = k_beg; k0 < k_end; k0 += OG_R) {
    for (int q = threadIdx.x; q < OG_R * Jp; q += blockDim.x) {
      const int c = q / OG_R, r = q - c * OG_R, k = k0 + r;
      As_[r * ld + c] = (k < k_end && c < J) ? T.a[k + (size_t)c * T.rows] : 0.0;
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int r = 0; r < OG_R; ++r) {
        const double* row = As_ + r * ld;
        const double x0 = row[i0], x1 = row[i0 + 1], y0 = row[j0], y1 = row[j0 + 1];
        a00 = fma(x0, y0, a00);
        a01 = fma(x0, y1, a01);
        a10 = fma(x1, y0, a10);
        a11 = fma(x1, y1, a11);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  // each (task, chunk) owns `stride` doubles (the launch's largest J^2)
  double* out = partial + ((size_t)blockIdx.z * nchunk + blockIdx.x) * stride;
  const double v[2][2] = {{a00, a01}, {a10, a11}};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
      if (i0 + a < J && j0 + b < J) out[(size_t)(i0 + a) * J + j0 + b] = v[a][b];
}

__global__ void ortho_gram_reduce_kernel(const OrthoTask* __restrict__ tasks, int nchunk, size_t stride,
                                         const double* __restrict__ partial) {
  const OrthoTask T = tasks[blockIdx.z];
  const int J = T.J;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < J * J; q += gridDim.x * blockDim.x) {
    int i = q / J, j = q - (q / J) * J;
    const int oi = i, oj = j;
    if (i / 2 > j / 2) {  // only tiles with i/2 <= j/2 were written
      const int t = i;
      i = j;
      j = t;
    }
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += partial[((size_t)blockIdx.z * nchunk + ch) * stride + i * J + j];
    T.out[oi + (size_t)oj * J] = s;
  }
}

// out = A Y (rows x K times K x J): a thread per row, NC output columns per
// CTA (the smallest of 8 ... 64 that covers J, else tiles of 64), the Y
// columns staged in shared memory.
template <int NC>
__global__ void __launch_bounds__(256) ortho_apply_kernel(const OrthoTask* __restrict__ tasks) {
  const OrthoTask T = tasks[blockIdx.z];
  const int c0 = blockIdx.y * NC;
  if (c0 >= T.J) return;
  const int K = T.K > 0 ? T.K : T.J;
  extern __shared__ double ys[];  // K x NC
  for (int idx = threadIdx.x; idx < K * NC; idx += blockDim.x) {
    const int k = idx / NC, c = idx - k * NC;
    ys[idx] = (c0 + c < T.J) ? T.y[k + (size_t)(c0 + c) * K] : 0.0;
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= T.rows) return;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int k = 0; k < K; ++k) {
    const double a = T.a[r + (size_t)k * T.rows];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = fma(a, ys[k * NC + c], acc[c]);
  }
  const int nc = min(NC, T.J - c0);
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (c < nc) T.out[r + (size_t)(c0 + c) * T.rows] = acc[c];
}

template <int NC>
void launch_apply_nc(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, int max_K, cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)max_K * NC;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute((const void*)ortho_apply_kernel<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ortho_apply_kernel<NC><<<dim3((max_rows + 255) / 256, (max_J + NC - 1) / NC, ntask), 256, smem, st>>>(d_tasks);
}

}  // namespace

size_t ortho_partial_doubles(int ntask, int max_rows, int max_J) {
  const int nchunk = (max_rows + ORTHO_CHUNK - 1) / ORTHO_CHUNK;
  return (size_t)ntask * nchunk * max_J * max_J;
}

void launch_ortho_gram(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, double* partial,
                       cudaStream_t st) {
  if (ntask <= 0) return;
  const int nchunk = (max_rows + ORTHO_CHUNK - 1) / ORTHO_CHUNK;
  const int nt = (max_J + 1) / 2, ntiles = nt * (nt + 1) / 2;
  const int ld = ((max_J + 1) & ~1) + 2;
  const size_t smem = sizeof(double) * OG_R * (size_t)ld;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute((const void*)ortho_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const size_t stride = (size_t)max_J * max_J;
  ortho_gram_kernel<<<dim3(nchunk, (ntiles + 255) / 256, ntask), 256, smem, st>>>(d_tasks, ORTHO_CHUNK, nchunk, ld,
                                                                                      stride, partial);
  ortho_gram_reduce_kernel<<<dim3((max_J * max_J + 255) / 256, 1, ntask), 256, 0, st>>>(d_tasks, nchunk, stride,
                                                                                       partial);
}

void launch_ortho_apply(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, int max_K, cudaStream_t st) {
  if (ntask <= 0) return;
  if (max_J <= 8) launch_apply_nc<8>(d_tasks, ntask, max_rows, max_J, max_K, st);
  else if (max_J <= 16) launch_apply_nc<16>(d_tasks, ntask, max_rows, max_J, max_K, st);
  else if (max_J <= 24) launch_apply_nc<24>(d_tasks, ntask, max_rows, max_J, max_K, st);
  else if (max_J <= 32) launch_apply_nc<32>(d_tasks, ntask, max_rows, max_J, max_K, st);
  else if (max_J <= 40) launch_apply_nc<40>(d_tasks, ntask, max_rows, max_J, max_K, st);
  else if (max_J <= 48) launch_apply_nc<48>(d_tasks, ntask, max_rows, max_J, max_K, st);
  else launch_apply_nc<64>(d_tasks, ntask, max_rows, max_J, max_K, st);
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
