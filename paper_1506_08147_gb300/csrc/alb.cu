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

}  // namespace

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
