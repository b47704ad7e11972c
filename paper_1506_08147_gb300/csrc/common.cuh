// Shared device types for the ALB generator (sm_103a).
//
// Data layout in HBM, per extended element Q_K (Sec. II.B: Psi_K is an
// N_g x J_K dense matrix):
//   * blocks X, W, P, HX, HW, HP: column-major N_g x m, x fastest inside a
//     vector; X, P, HX, HP are double-buffered (parity bit per element) so a
//     block update never reads what it overwrites;
//   * Z: FFT scratch, m half-spectra of (nx/2+1) * ny * nz complex values,
//     ordered [z][y][kx];
//   * small FP64 matrices (Gram blocks, Rayleigh-Ritz factors) per element.
// Every kernel indexes the element by blockIdx.z and skips inactive ones.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dgdft {

template <class real> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <class real> using cplx_t = typename cplx_of<real>::type;
struct dff;  // double-float scalar (dfloat.cuh)

template <class C> __host__ __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) {
  C c; c.x = a; c.y = b; return c;
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <class C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }

// Block selectors.  Double-buffered blocks have two physical buffers.
enum Blk { BX = 0, BP = 1, BHX = 2, BHP = 3, BW = 4, BHW = 5, NBLK = 6 };
enum { NDBL = 4 };  // X, P, HX, HP are double-buffered

// Per-element state words (device int array, STATE_WORDS per element).
enum {
  ST_PARITY = 0,    // which buffer of X/P/HX/HP is current
  ST_ACTIVE = 1,    // 1 while the element still iterates
  ST_HAS_P = 2,     // 1 once the P block is valid
  ST_ITER = 3,      // LOBPCG iterations done
  ST_ERROR = 4,     // bit flags, see ERR_*
  ST_CONVERGED = 5, // 1 once max residual <= tol
  ST_FALLBACK = 6,  // Rayleigh-Ritz retries without P
  ST_TETER = 7,     // 1: precondition with Teter (the learned network's fallback)
  ST_RESTART = 8,   // 1: Rayleigh-Ritz found no usable pencil; X is perturbed and P dropped
  ST_NRESTART = 9,  // restarts taken (bounded per solve)
  STATE_WORDS = 10
};
enum { ERR_CHOL = 1, ERR_NONFINITE = 2, ERR_EIG = 4, ERR_TIMEOUT = 8 };  // ERR_TIMEOUT: a bounded device wait ran out

constexpr int MAX_STAGES = 8;
enum { TW_H = 0, TW_X = 1, TW_Y = 2, TW_Z = 3 };

struct FftPlan {
  int n;                    // transform length
  int nstage;
  int radix[MAX_STAGES];
};

// Everything a kernel needs to know about one element, in working precision.
template <class real> struct ElemDev {
  using C = cplx_t<real>;
  int nx, ny, nz, ng;       // grid, N_g
  int nh, nxh, nspec;       // nx/2, nx/2+1, nxh*ny*nz
  int m, J;                 // block size, kept vectors
  double scale;             // 2 / N_g: normalisation of r2c forward + c2r inverse
  double tol;
  double ecut;              // planewave set |G|^2/2 <= ecut (Ha); 0: every G of the grid
  FftPlan px, py, pz;       // x plan is for the half length nh
  // twiddle tables e^{-2 pi i t / n} per axis: [TW_H] n = nx/2 (t < nh),
  // [TW_X] n = nx (t <= nh, r2c post-processing), [TW_Y] n = ny, [TW_Z] n = nz;
  // in working precision and in FP64 (the same table for FP64 waves)
  const C* tw[4];
  const double2* tw64[4];
  // the FP64 tables as FP32 pairs (hi, lo of re, hi, lo of im), FP64 waves
  // only: for FFT passes in double-float arithmetic
  const float4* twdf[4];
  const double* gx2;        // (2 pi kx / Lx)^2 / 2, kx = 0..nh
  const double* gy2;        // (2 pi f_y / Ly)^2 / 2 over y index (|f| <= ny/2)
  const double* gz2;
  const float* gx2f;        // the same symbols in FP32 (FP32 stage arithmetic)
  const float* gy2f;
  const float* gz2f;
  const real* V;            // V_eff^{Q_K}, N_g
  // Kleinman-Bylander projectors, CSR by projector
  int n_proj;
  const int* p_ptr;         // n_proj + 1
  const int* p_idx;
  const real* p_val;
  const double* p_gamma;    // n_proj
  // the same nonzeros grouped by grid point, for the fused scatter
  int n_sup;
  const int* s_plane;       // nz + 1: support entries of plane z
  const int* s_off;         // in-plane offset y*nx + x of support entry
  const int* s_ptr;         // n_sup + 1 into (s_proj, s_gv)
  const int* s_proj;
  const real* s_gv;         // gamma_p * v_p(point)
  // the same per point padded to 4 nonzeros (zero weight, projector 0), when
  // no point has more than 4; nullptr otherwise
  const int* s_proj4;
  const real* s_gv4;
  real* Ccoef;              // n_proj x m projector coefficients (column j contiguous)
  // blocks
  real* blk[NBLK][2];       // [sel][buffer]; single-buffered blocks use [0]
  void* Z;                  // FFT scratch, m * nspec complex of up to FP64 size
  // small FP64 workspace
  double* gram;             // 2 x (3m)^2: A then B (ld 3m)
  double* gxw;              // m x m: X^T W
  double* Y;                // 3m x m Rayleigh-Ritz coefficients
  float* Yf;                // the same in FP32 (FP32 waves: read by the block updates)
  double* theta;            // m
  double* res;              // m
  double* tkin;             // m
  // spectral shift of the FP32 stage: [0] sigma, [1] the change made this
  // iteration.  Kernels of the FP32 stage apply H - sigma I, so Ritz values
  // and H-images are stored relative to sigma (always 0 for FP64 waves).
  double* sigma;
  double* rr_work;          // dense eigensolver workspace
  double* rpart;            // residual partial sums
  int* state;               // STATE_WORDS
};

// Asynchronous global -> shared copies (cp.async).  src_bytes < size fills
// the rest of the destination with zeros (src must still be a valid address).
__device__ __forceinline__ uint32_t shared_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(shared_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(shared_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Twiddle table of axis `a` in the transform's compute precision TC.
template <class TC, class real>
__device__ __forceinline__ const cplx_t<TC>* twp(const ElemDev<real>& e, int a) {
  if constexpr (std::is_same<TC, dff>::value) {
    return reinterpret_cast<const cplx_t<TC>*>(e.twdf[a]);
  } else if constexpr (sizeof(TC) == sizeof(double)) {
    return e.tw64[a];
  } else {
    return reinterpret_cast<const cplx_t<TC>*>(e.tw[a]);
  }
}

template <class real>
__device__ __forceinline__ real* cur_blk(const ElemDev<real>& e, int sel) {
  int par = (sel < NDBL) ? (e.state[ST_PARITY] & 1) : 0;
  return e.blk[sel][par];
}
template <class real>
__device__ __forceinline__ real* next_blk(const ElemDev<real>& e, int sel) {
  int par = (sel < NDBL) ? ((e.state[ST_PARITY] & 1) ^ 1) : 0;
  return e.blk[sel][par];
}

}  // namespace dgdft
