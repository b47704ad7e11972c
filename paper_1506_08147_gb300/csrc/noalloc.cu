// Gram product C = U^T V with no device allocation at all.
//
// Some callers cannot call cudaMalloc while they run: code inside a custom
// memory pool that must not fragment, and allocator-free real-time loops
// whose latency must not include an allocation.  This entry point serves
// them: the caller passes device inputs and the device output,
// and the split-K partial sums of the FP64 Gram kernel live in a fixed
// file-scope device array instead of an allocated buffer.  Every GPU that
// loads the library holds that array (8 MiB) until the process exits.
#include <mutex>

#include "../../include/dgdft_alb_steps.h"
#include "internal.h"

namespace dgdft {

namespace {

constexpr int NA_TILE = 64;
constexpr int NA_KS = 32;
constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)1 << 20;  // 8 MiB
constexpr int NOALLOC_MAX_COLS = 256;

// The scratch shared by every call of dgdft_alb_gram_noalloc on a device.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Per-device address of g_noalloc_scratch, looked up once per device and
// kept for the life of the process (stale after a device reset).
std::mutex g_addr_mu;
double* g_addr[64] = {nullptr};

// grid: (nchunk, tiles_a * tiles_b); block 256 (16 x 16 threads, 4 x 4 outputs each).
__global__ void __launch_bounds__(256) noalloc_gram_kernel(const double* __restrict__ U,
                                                           const double* __restrict__ V, int ng, int p,
                                                           int q, int kchunk, int tiles_b,
                                                           double* __restrict__ partial) {
  __shared__ double As[NA_KS][NA_TILE + 4];
  __shared__ double Bs[NA_KS][NA_TILE + 4];
  const int ta = blockIdx.y / tiles_b, tb = blockIdx.y - ta * tiles_b;
  const int a0 = ta * NA_TILE, b0 = tb * NA_TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k_beg = blockIdx.x * kchunk;
  const int k_end = min(ng, k_beg + kchunk);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = k_beg; k0 < k_end; k0 += NA_KS) {
    for (int i = threadIdx.x; i < NA_KS * NA_TILE; i += blockDim.x) {
      const int c = i / NA_KS, r = i - c * NA_KS;
      const int k = k0 + r;
      const bool kin = k < k_end;
      As[r][c] = (kin && a0 + c < p) ? U[(size_t)(a0 + c) * ng + k] : 0.0;
      Bs[r][c] = (kin && b0 + c < q) ? V[(size_t)(b0 + c) * ng + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < NA_KS; ++r) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[r][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[r][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
  double* out = partial + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * (NA_TILE * NA_TILE);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * NA_TILE + tx * 4 + j] = acc[i][j];
}

// Sum the chunks in a fixed order; C is p x q column-major.
__global__ void noalloc_reduce_kernel(const double* __restrict__ partial, int nchunk, int ntile, int tiles_b,
                                      int p, int q, double* __restrict__ c) {
  const int t = blockIdx.x;
  const int ta = t / tiles_b, tb = t - ta * tiles_b;
  const int a0 = ta * NA_TILE, b0 = tb * NA_TILE;
  for (int i = threadIdx.x; i < NA_TILE * NA_TILE; i += blockDim.x) {
    const int r = i / NA_TILE, cc = i - r * NA_TILE;
    if (a0 + r >= p || b0 + cc >= q) continue;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += partial[((size_t)ch * ntile + t) * (NA_TILE * NA_TILE) + i];
    c[(a0 + r) + (size_t)(b0 + cc) * p] = s;
  }
}

}  // namespace

}  // namespace dgdft

using namespace dgdft;

extern "C" dgdft_status dgdft_alb_gram_noalloc(int ng, int p, int q, const double* u, const double* v, double* c,
                                               void* stream) {
  if (ng < 1 || p < 1 || q < 1 || !u || !v || !c) return DGDFT_EINVAL;
  if (p > NOALLOC_MAX_COLS || q > NOALLOC_MAX_COLS) return DGDFT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DGDFT_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
      // the array's name is a host-side stand-in: ask the runtime for its
      // device address on the current device, once
      double* ptr = nullptr;
      if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return DGDFT_ECUDA;
      g_addr[dev] = ptr;
    }
    scratch = g_addr[dev];
  }
  const int tiles_a = (p + NA_TILE - 1) / NA_TILE, tiles_b = (q + NA_TILE - 1) / NA_TILE;
  const int ntile = tiles_a * tiles_b;
  // chunks of >= 2048 rows, as many as the scratch holds (>= 16 at 256 x 256)
  const size_t max_chunks = NOALLOC_SCRATCH_DOUBLES / ((size_t)ntile * NA_TILE * NA_TILE);
  size_t nchunk = ((size_t)ng + 2047) / 2048;
  if (nchunk > max_chunks) nchunk = max_chunks;
  const int kchunk = (int)(((size_t)ng + nchunk - 1) / nchunk);
  nchunk = ((size_t)ng + kchunk - 1) / kchunk;
  cudaStream_t st = (cudaStream_t)stream;
  int nch = (int)nchunk;
  void* a1[] = {(void*)&u, (void*)&v, (void*)&ng, (void*)&p, (void*)&q, (void*)&kchunk, (void*)&tiles_b,
                (void*)&scratch};
  if (cudaLaunchKernel((const void*)noalloc_gram_kernel, dim3((unsigned)nchunk, ntile), dim3(256), a1, 0, st) !=
      cudaSuccess)
    return DGDFT_ECUDA;
  void* a2[] = {(void*)&scratch, (void*)&nch, (void*)&ntile, (void*)&tiles_b, (void*)&p, (void*)&q, (void*)&c};
  if (cudaLaunchKernel((const void*)noalloc_reduce_kernel, dim3(ntile), dim3(256), a2, 0, st) != cudaSuccess)
    return DGDFT_ECUDA;
  return DGDFT_OK;
}
