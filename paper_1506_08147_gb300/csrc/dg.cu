// DG Hamiltonian assembly from the adaptive local basis (Eq. DGHamiltonian;
// Sec. II.B, "Construction of the DG Hamiltonian").
//
// Per batch of elements, FP64 throughout:
//   1. interpolation of the J columns from Q_K's uniform grid to E_K's LGL
//      grid: three passes of a small dense matrix applied along one axis
//      (the real trigonometric interpolant over Q_K, sampled at the nodes);
//   2. Eq. orthonormal under the LGL quadrature: the mass matrix
//      M = phi~^T W phi~ (W the LGL weights), its Cholesky factor M = L L^T
//      and phi = phi~ L^-T.  Orthonormalising before the integrals keeps the
//      rounding of ill-conditioned mass matrices (restricted Ritz vectors
//      are nearly dependent on E_K) amplified by cond(L), not cond(M);
//   3. gradients: the LGL differentiation matrix along each axis;
//   4. volume integrals: weighted Gram products phi^T W V phi and
//      (d_d phi)^T W (d_d phi);
//   5. face traces (values and normal derivative on the six faces) and the
//      KB coefficients <b_p, phi_j>;
// then over all elements:
//   6. face integrals: weighted Gram products of the traces of both sides of
//      every face;
//   7. every block H_{K,K'} summed from its volume, KB and face terms.
// Density (Eq. density, the DIAG route for small systems): H^DG scattered
// into a dense matrix, its eigenpairs by a one-sided Jacobi eigensolver over
// the whole GPU (one cooperative kernel), the density matrix blocks
// P_K = Y_K Y_K^T of the lowest n_occ, and rho = sum_jj' phi_j P_K,jj' phi_j'
// on the LGL grids.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/dgdft_dg.h"
#include "dfloat.cuh"

namespace {

constexpr int AX_THREADS = 256;
constexpr int AX_TC = 64;                      // columns per CTA tile
constexpr int AX_LD = AX_TC + 1;               // odd stride: conflict-free column walks
constexpr int AX_NR = AX_THREADS / AX_TC;      // row groups
constexpr int AX_MAXR = 32;                    // output rows per thread: n_out <= 128
constexpr int MAX_NL = AX_MAXR * AX_NR;
constexpr int MAX_J = 128;

constexpr int GR_R = 16;                       // staged points per step
constexpr int GR_CH = 2048;                    // points per split-K chunk

constexpr double PI = 3.14159265358979323846;

// Arithmetic of the contractions: FP64, or double-float pairs (FP32 h + l,
// ~2^-48 relative per operation, on the FP32 pipes).
using dgdft::dfl;
__device__ __forceinline__ double to_t(double v, double*) { return v; }
__device__ __forceinline__ dfl to_t(double v, dfl*) { return dgdft::dfl_of(v); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ dfl fma_t(dfl a, dfl b, dfl c) { return dgdft::dfl_fma(a, b, c); }
__device__ __forceinline__ double val_t(double a) { return a; }
__device__ __forceinline__ double val_t(dfl a) { return dgdft::dfl_val(a); }
template <class T> __device__ __forceinline__ T zero_t() { return to_t(0.0, (T*)nullptr); }

// ------------------------------------------------------------------ kernels

// One pass of a small dense matrix A (n_out x n_in, row-major; element e uses
// A + e * a_stride) along one axis of every element's array viewed as
// [O][n_in][S]: out[o][r][s] = sum_i A[r][i] in[o][i][s].  FAST (S == 1): a
// tile is 64 consecutive lines, staged transposed so loads and stores stay
// coalesced; otherwise a tile is 64 consecutive (o, s) columns, s fastest.
// Each thread owns R output rows of one column (R >= n_out / AX_NR, a
// compile-time count, so no FP64 instruction issues for rows that do not
// exist beyond the last group of AX_NR).
struct AxisJob {
  const double* const* in;
  double* const* out;
  const double* A;
  long long a_stride;
  int n_in, n_out, S;
  long long O;
};

template <bool FAST, int R, class T>
__global__ void __launch_bounds__(AX_THREADS) dg_axis_kernel(AxisJob jb) {
  extern __shared__ double sm[];
  const int nin = jb.n_in, nout = jb.n_out, S = jb.S;
  T* As = reinterpret_cast<T*>(sm);
  T* Xs = As + nout * nin;
  const double* __restrict__ in = jb.in[blockIdx.y];
  double* __restrict__ out = jb.out[blockIdx.y];
  const double* __restrict__ A = jb.A + blockIdx.y * jb.a_stride;
  const int t = threadIdx.x;
  for (int i = t; i < nout * nin; i += AX_THREADS) As[i] = to_t(A[i], (T*)nullptr);
  const long long ncols_total = FAST ? jb.O : jb.O * (long long)S;
  const long long g0 = (long long)blockIdx.x * AX_TC;
  const int ncol = (int)min((long long)AX_TC, ncols_total - g0);
  if (FAST) {
    const double* src = in + g0 * nin;
    for (int q = t; q < ncol * nin; q += AX_THREADS) {
      const int c = q / nin, i = q - c * nin;
      Xs[i * AX_LD + c] = to_t(src[q], (T*)nullptr);
    }
  } else {
    for (int q = t; q < nin * AX_TC; q += AX_THREADS) {
      const int i = q / AX_TC, c = q - i * AX_TC;
      double v = 0.0;
      if (c < ncol) {
        const long long g = g0 + c, o = g / S, s = g - o * S;
        v = in[(o * nin + i) * S + s];
      }
      Xs[i * AX_LD + c] = to_t(v, (T*)nullptr);
    }
  }
  __syncthreads();
  const int c = t % AX_TC, r = t / AX_TC;
  // rows r, r + AX_NR, ...: the last ones may not exist (row >= nout); their
  // matrix row is clamped to a valid one and the result is not stored
  int arow[R];
#pragma unroll
  for (int k = 0; k < R; ++k) arow[k] = min(r + k * AX_NR, nout - 1) * nin;
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = zero_t<T>();
  for (int i = 0; i < nin; ++i) {
    const T x = Xs[i * AX_LD + c];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = fma_t(As[arow[k] + i], x, acc[k]);
  }
  if (FAST) {
    __syncthreads();
    double* Xd = reinterpret_cast<double*>(Xs);  // the tile again, as doubles
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int row = r + k * AX_NR;
      if (row < nout) Xd[row * AX_LD + c] = val_t(acc[k]);
    }
    __syncthreads();
    double* dst = out + g0 * nout;
    for (int q = t; q < ncol * nout; q += AX_THREADS) {
      const int cc = q / nout, i = q - cc * nout;
      dst[q] = Xd[i * AX_LD + cc];
    }
  } else if (c < ncol) {
    const long long g = g0 + c, o = g / S, s = g - o * S;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int row = r + k * AX_NR;
      if (row < nout) out[(o * nout + row) * S + s] = val_t(acc[k]);
    }
  }
}

// Weighted Gram products C = X^T diag(w v) Y over n points (X, Y column-major
// with leading dimensions ldx, ldy), split into chunks of GR_CH points whose
// partial J1 x J2 sums are added in a fixed order by dg_gram_reduce_kernel.
// Each thread owns a 2 x 2 output tile; tiles are numbered densely (row-major,
// or the upper triangle ti <= tj when sym: X = Y, the lower half mirrored by
// the reduction), 256 per CTA, grid.z over groups of 256 tiles.
struct GramTask {
  const double* X;
  const double* Y;
  const double* w;  // n weights
  const double* v;  // optional second factor (NULL = 1)
  double* out;      // J1 x J2 row-major
  long long part;   // offset of this task's partials
  int n, ldx, ldy, J1, J2, nchunk, sym;
};

__device__ __forceinline__ void gram_tile_of(int t, int nt, int sym, int* ti, int* tj) {
  if (!sym) {
    *ti = t / nt;
    *tj = t - *ti * nt;
    return;
  }
  // upper triangle, row by row: row i holds nt - i tiles
  int i = 0, base = 0;
  while (t >= base + (nt - i)) {
    base += nt - i;
    ++i;
  }
  *ti = i;
  *tj = i + (t - base);
}

template <class T>
__global__ void __launch_bounds__(256) dg_gram_kernel(const GramTask* __restrict__ tasks,
                                                      double* __restrict__ partial) {
  __shared__ T Xs[GR_R][MAX_J + 2];
  __shared__ T Ys[GR_R][MAX_J + 2];
  const GramTask Tk = tasks[blockIdx.y];
  const int chunk = blockIdx.x;
  if (chunk >= Tk.nchunk) return;
  const int nti = (Tk.J1 + 1) / 2, ntj = (Tk.J2 + 1) / 2;
  const int ntiles = Tk.sym ? nti * (nti + 1) / 2 : nti * ntj;
  const int tile0 = blockIdx.z * 256;
  if (tile0 >= ntiles) return;
  const int mytile = tile0 + threadIdx.x;
  int ti = 0, tj = 0;
  const bool active = mytile < ntiles;
  if (active) gram_tile_of(mytile, Tk.sym ? nti : ntj, Tk.sym, &ti, &tj);
  const int i0 = 2 * ti, j0 = 2 * tj;
  const int p0 = chunk * GR_CH, p1 = min(Tk.n, p0 + GR_CH);
  T acc00 = zero_t<T>(), acc01 = zero_t<T>(), acc10 = zero_t<T>(), acc11 = zero_t<T>();
  const int J1p = (Tk.J1 + 1) & ~1, J2p = (Tk.J2 + 1) & ~1;
  for (int p = p0; p < p1; p += GR_R) {
    for (int q = threadIdx.x; q < GR_R * J1p; q += 256) {
      const int col = q / GR_R, rr = q - col * GR_R, pt = p + rr;
      double xv = 0.0;
      if (pt < p1 && col < Tk.J1) {
        double wt = Tk.w[pt];
        if (Tk.v) wt *= Tk.v[pt];
        xv = Tk.X[(size_t)col * Tk.ldx + pt] * wt;
      }
      Xs[rr][col] = to_t(xv, (T*)nullptr);
    }
    for (int q = threadIdx.x; q < GR_R * J2p; q += 256) {
      const int col = q / GR_R, rr = q - col * GR_R, pt = p + rr;
      Ys[rr][col] = to_t((pt < p1 && col < Tk.J2) ? Tk.Y[(size_t)col * Tk.ldy + pt] : 0.0, (T*)nullptr);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int rr = 0; rr < GR_R; ++rr) {
        const T a0 = Xs[rr][i0], a1 = Xs[rr][i0 + 1];
        const T b0 = Ys[rr][j0], b1 = Ys[rr][j0 + 1];
        acc00 = fma_t(a0, b0, acc00);
        acc01 = fma_t(a0, b1, acc01);
        acc10 = fma_t(a1, b0, acc10);
        acc11 = fma_t(a1, b1, acc11);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  double* dst = partial + Tk.part + (size_t)chunk * Tk.J1 * Tk.J2;
  const double v[2][2] = {{val_t(acc00), val_t(acc01)}, {val_t(acc10), val_t(acc11)}};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int ii = i0 + a, jj = j0 + b;
      if (ii < Tk.J1 && jj < Tk.J2) dst[(size_t)ii * Tk.J2 + jj] = v[a][b];
    }
}

__global__ void dg_gram_reduce_kernel(const GramTask* __restrict__ tasks, const double* __restrict__ partial) {
  const GramTask T = tasks[blockIdx.y];
  const int n = T.J1 * T.J2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int i = q / T.J2, j = q - (q / T.J2) * T.J2;
    // symmetric tasks hold the tiles with i/2 <= j/2 only
    if (T.sym && i / 2 > j / 2) {
      const int t = i;
      i = j;
      j = t;
    }
    const int src = i * T.J2 + j;
    double s = 0.0;
    for (int c = 0; c < T.nchunk; ++c) s += partial[T.part + (size_t)c * n + src];
    T.out[q] = s;
  }
}

// Face traces: for every element of the batch and each of its six faces
// (slot = 2 d + high), the values of phi and of d_d phi on the face plane,
// copied to compact n_face x J arrays.
struct TraceJob {
  const double* phi;     // batch base: element e at phi + e * J * nL
  const double* grad[3];
  double* traces;        // element e (global index g0 + e) at traces + (g0 + e) * tr_elem
  long long tr_elem;     // doubles per element
  long long tr_off[6];   // offset of slot's F; DF follows at + n_face * J
  int nf[6];
  int nl[3], J, nL, g0;
};

__global__ void dg_trace_kernel(TraceJob jb) {
  const int e = blockIdx.z, slot = blockIdx.y;
  const int d = slot >> 1, high = slot & 1;
  const int nfc = jb.nf[slot];
  const int nx = jb.nl[0], ny = jb.nl[1], nz = jb.nl[2];
  const double* phi = jb.phi + (size_t)e * jb.J * jb.nL;
  const double* gd = jb.grad[d] + (size_t)e * jb.J * jb.nL;
  double* F = jb.traces + (size_t)(jb.g0 + e) * jb.tr_elem + jb.tr_off[slot];
  double* DF = F + (size_t)nfc * jb.J;
  const long long total = (long long)nfc * jb.J;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(q / nfc), p = (int)(q - (long long)j * nfc);
    int idx;
    if (d == 0) {  // p = y + ny z
      const int y = p % ny, z = p / ny;
      idx = (high ? nx - 1 : 0) + nx * (y + ny * z);
    } else if (d == 1) {  // p = x + nx z
      const int x = p % nx, z = p / nx;
      idx = x + nx * ((high ? ny - 1 : 0) + ny * z);
    } else {  // p = x + nx y
      idx = p + nx * ny * (high ? nz - 1 : 0);
    }
    F[q] = phi[(size_t)j * jb.nL + idx];
    DF[q] = gd[(size_t)j * jb.nL + idx];
  }
}

// KB coefficients c[row][j] = sum_i (w_i b_p(x_i)) phi_j(x_i) for every
// projector row of the batch's elements; one CTA per row, a warp per j.
struct KbJob {
  const double* phi;        // batch base
  const int* row_elem;      // batch-local element of each row
  const long long* row_ptr; // CSR over (idx, wval), global rows
  const int* idx;
  const double* wval;       // w_i b_p(x_i)
  double* coef;             // row r at coef + r * J
  int row0, J, nL;
};

__global__ void dg_kb_kernel(KbJob jb) {
  const int r = jb.row0 + blockIdx.x;
  const int e = jb.row_elem[blockIdx.x];
  const double* phi = jb.phi + (size_t)e * jb.J * jb.nL;
  const long long b = jb.row_ptr[r], nnz = jb.row_ptr[r + 1] - b;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < jb.J; j += nw) {
    double s = 0.0;
    for (long long i = lane; i < nnz; i += 32) s = fma(jb.wval[b + i], phi[(size_t)j * jb.nL + jb.idx[b + i]], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) jb.coef[(size_t)r * jb.J + j] = s;
  }
}

// Cholesky M~ = L L^T of every element's mass matrix (in shared memory) and
// the lower triangular L^-1 (written column by column to global memory, each
// column by one thread), one CTA per element.
__global__ void __launch_bounds__(256) dg_chol_kernel(const double* __restrict__ mass, long long mass_stride,
                                                      double* __restrict__ linv, int J, int* __restrict__ bad) {
  extern __shared__ double Ls[];  // J x J
  const int e = blockIdx.x, t = threadIdx.x;
  const double* M = mass + (size_t)e * mass_stride;
  for (int q = t; q < J * J; q += blockDim.x) Ls[q] = M[q];
  __shared__ int fail;
  if (t == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < J; ++k) {
    if (t == 0) {
      const double d = Ls[k * J + k];
      const bool ok = d > 0.0 && isfinite(d);
      if (!ok) fail = 1;
      Ls[k * J + k] = ok ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double piv = Ls[k * J + k];
    for (int i = k + 1 + t; i < J; i += blockDim.x) Ls[i * J + k] /= piv;
    __syncthreads();
    const int m = J - k - 1;
    for (int q = t; q < m * m; q += blockDim.x) {
      const int i = k + 1 + q / m, j = k + 1 + q % m;
      if (j <= i) Ls[i * J + j] -= Ls[i * J + k] * Ls[j * J + k];
    }
    __syncthreads();
  }
  double* X = linv + (size_t)e * J * J;
  for (int j = t; j < J; j += blockDim.x) {  // column j of L^-1: solve L x = e_j
    for (int i = 0; i < j; ++i) X[i * J + j] = 0.0;
    for (int i = j; i < J; ++i) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) s -= Ls[i * J + k] * X[k * J + j];
      X[i * J + j] = s / Ls[i * J + i];
    }
  }
  if (t == 0) bad[e] = fail;
}

// Every block: sum of coef * pool matrix (or its transpose) and of the KB
// outer products gamma c_a c_b^T.
struct MatTerm {
  double coef;
  long long mat;  // offset in the matrix pool
  int trans;
  int pad;
};
struct KbTerm {
  double gamma;
  int ra, rb;  // KB coefficient rows of the two elements
};
struct BlockJob {
  const double* pool;
  const MatTerm* terms;
  const int* term_ptr;
  const KbTerm* kb;
  const int* kb_ptr;
  const double* coef;  // KB coefficients
  double* out;         // H (nblk x J x J)
  int J;
};

__global__ void dg_block_sum_kernel(BlockJob jb) {
  const int b = blockIdx.y, J = jb.J;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= J * J) return;
  const int i = q / J, j = q - i * J;
  double s = 0.0;
  for (int t = jb.term_ptr[b]; t < jb.term_ptr[b + 1]; ++t) {
    const MatTerm T = jb.terms[t];
    s = fma(T.coef, jb.pool[T.mat + (T.trans ? (size_t)j * J + i : (size_t)i * J + j)], s);
  }
  for (int t = jb.kb_ptr[b]; t < jb.kb_ptr[b + 1]; ++t) {
    const KbTerm K = jb.kb[t];
    s = fma(K.gamma * jb.coef[(size_t)K.ra * J + i], jb.coef[(size_t)K.rb * J + j], s);
  }
  jb.out[(size_t)b * J * J + q] = s;
}

// Dense H^DG (element-major, row K J + i) from the stored blocks.
__global__ void dg_dense_kernel(const double* __restrict__ H, const int2* __restrict__ blk_kk, double* __restrict__ A,
                                int J, long long n) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= J * J) return;
  const int i = q / J, j = q - i * J;
  const int2 kk = blk_kk[b];
  A[((long long)kk.x * J + i) * n + (long long)kk.y * J + j] = H[(size_t)b * J * J + q];
}

// P_K[j][j'] = sum_i Y[K J + j, i] Y[K J + j', i] (Y column-major n x m).
__global__ void dg_dm_kernel(const double* __restrict__ Y, double* __restrict__ P, int J, long long n, int m) {
  const int k = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= J * J) return;
  const int j = q / J, jp = q - j * J;
  const double* a = Y + (long long)k * J + j;
  const double* b = Y + (long long)k * J + jp;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s = fma(a[(long long)i * n], b[(long long)i * n], s);
  P[(size_t)k * J * J + q] = s;
}

// rho[p] = sum_j phi[j][p] T[j][p] for every element of a batch (grid.y).
__global__ void dg_rho_kernel(const double* __restrict__ phi, const double* __restrict__ T, double* __restrict__ rho,
                              int J, int nL) {
  const size_t off = (size_t)blockIdx.y * J * nL;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nL; p += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < J; ++j) s = fma(phi[off + (size_t)j * nL + p], T[off + (size_t)j * nL + p], s);
    rho[(size_t)blockIdx.y * nL + p] = s;
  }
}

// One-sided (Hestenes) Jacobi eigensolver for a symmetric matrix, FP64, over
// the whole GPU.  B = A + sigma I is positive definite (sigma from a
// Gershgorin bound); rotations of column pairs make the columns of W = B V
// mutually orthogonal, so that at convergence w_i = lambda_i(B) v_i:
// eigenvalues |w_i| - sigma, eigenvectors w_i / |w_i| (V itself is never
// formed).  Each sweep visits
// every pair once in n_pad - 1 rounds of disjoint pairs (the round-robin
// tournament: index 0 fixed, the others rotating); a CTA rotates one pair,
// and the grid synchronises between rounds (a cooperative launch, so every
// CTA is resident).  The sweeps stop when no pair's cosine |w_i . w_j| /
// (|w_i| |w_j|) exceeds tol, or after max_sweeps.  W is column-major n x n;
// off[s] (zeroed by the host) collects sweep s's largest cosine.
__device__ __forceinline__ int jacobi_player(int i, int r, int n_pad) {
  return i == 0 ? 0 : 1 + (i - 1 + r) % (n_pad - 1);
}

constexpr int JC_THREADS = 128;

__global__ void __launch_bounds__(JC_THREADS) dg_jacobi_kernel(double* __restrict__ W, int n,
                                                               int n_pad, int max_sweeps, double tol,
                                                               unsigned long long* __restrict__ off,
                                                               int* __restrict__ sweeps) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[JC_THREADS / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int npairs = n_pad / 2;
  int s = 0;
  for (; s < max_sweeps; ++s) {
    double worst = 0.0;
    for (int r = 0; r < n_pad - 1; ++r) {
      for (int k = blockIdx.x; k < npairs; k += gridDim.x) {
        // pair k of round r: (pos k, pos n_pad - 1 - k) on the circle
        int p = jacobi_player(k, r, n_pad), q = jacobi_player(n_pad - 1 - k, r, n_pad);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= n) continue;  // the padding column of an odd n
        double* wp = W + (size_t)p * n;
        double* wq = W + (size_t)q * n;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = threadIdx.x; i < n; i += JC_THREADS) {
          const double x = wp[i], y = wq[i];
          a = fma(x, x, a);
          b = fma(y, y, b);
          g = fma(x, y, g);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (lane == 0) {
          red[warp][0] = a;
          red[warp][1] = b;
          red[warp][2] = g;
        }
        __syncthreads();
        a = b = g = 0.0;
#pragma unroll
        for (int w = 0; w < JC_THREADS / 32; ++w) {
          a += red[w][0];
          b += red[w][1];
          g += red[w][2];
        }
        __syncthreads();  // red is reused by the next pair
        if (a <= 0.0 || b <= 0.0) continue;
        const double cosv = fabs(g) / sqrt(a * b);
        worst = fmax(worst, cosv);
        if (cosv <= tol) continue;
        // the rotation that makes the two columns orthogonal
        const double zeta = (b - a) / (2.0 * g);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int i = threadIdx.x; i < n; i += JC_THREADS) {
          const double x = wp[i], y = wq[i];
          wp[i] = c * x - sn * y;
          wq[i] = sn * x + c * y;
        }
      }
      grid.sync();
    }
    // the sweep's largest cosine (non-negative doubles order as their bits)
    if (threadIdx.x == 0 && worst > 0.0) atomicMax(off + s, (unsigned long long)__double_as_longlong(worst));
    grid.sync();
    const double sweep_worst = __longlong_as_double((long long)*(volatile unsigned long long*)(off + s));
    if (sweep_worst <= tol) {
      ++s;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps = s;
}

// Gershgorin lower bound per row: a_ii - sum_{j != i} |a_ij| (row-major A).
__global__ void dg_gershgorin_kernel(const double* __restrict__ A, long long n, double* __restrict__ lo) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = A + (size_t)warp * n;
  double s = 0.0;
  for (long long j = lane; j < n; j += 32)
    if (j != warp) s += fabs(row[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) lo[warp] = row[warp] - s;
}

// W = A + sigma I (column-major; A symmetric).
__global__ void dg_jacobi_init_kernel(const double* __restrict__ A, double* __restrict__ W, long long n,
                                      double sigma) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q % n, j = q / n;
    W[q] = A[i * n + j] + (i == j ? sigma : 0.0);
  }
}

// |w_i| per column (one warp each).
__global__ void dg_colnorm_kernel(const double* __restrict__ W, long long n, double* __restrict__ nrm) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* col = W + (size_t)warp * n;
  double s = 0.0;
  for (long long i = lane; i < n; i += 32) s = fma(col[i], col[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) nrm[warp] = sqrt(s);
}

// Y[:, c] = w_k / |w_k|, k = order[c], for the lowest m (column-major, n rows).
__global__ void dg_gather_kernel(const double* __restrict__ W, const double* __restrict__ nrm,
                                 const int* __restrict__ order, double* __restrict__ Y, long long n, int m) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * m;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = q / n, i = q % n;
    const int k = order[c];
    Y[q] = W[(size_t)k * n + i] / nrm[k];
  }
}

// ------------------------------------------------------------------ host tables

// P_N(x) and P_{N-1}(x) by the three-term recurrence.
void legendre_pair(int N, double x, double* pn, double* pn1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (N == 0) {
    *pn = 1.0;
    *pn1 = 0.0;
    return;
  }
  for (int k = 2; k <= N; ++k) {
    const double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *pn1 = a;
}

// LGL rule on [-1, 1]: the end points and the roots of P'_N (N = n - 1),
// found by Newton's method from the Chebyshev extrema, with P'_N from
// (x^2 - 1) P'_N = N (x P_N - P_{N-1}) and P''_N from Legendre's equation;
// weights 2 / (N (N + 1) P_N(x)^2).
bool lgl_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  const int N = n - 1;
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(PI * j / N);
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre_pair(N, t, &pn, &pn1);
      const double d1 = N * (t * pn - pn1) / (t * t - 1.0);
      const double d2 = (2.0 * t * d1 - N * (N + 1.0) * pn) / (1.0 - t * t);
      const double dt = d1 / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-15) {
        ok = true;
        break;
      }
    }
    if (!ok) return false;
    x[j] = t;
  }
  for (int j = 0; j < n / 2; ++j) {  // exact symmetry
    const double a = 0.5 * (x[N - j] - x[j]);
    x[j] = -a;
    x[N - j] = a;
  }
  if (n % 2) x[n / 2] = 0.0;
  for (int j = 0; j < n; ++j) {
    double pn, pn1;
    legendre_pair(N, x[j], &pn, &pn1);
    w[j] = 2.0 / (N * (N + 1.0) * pn * pn);
  }
  return true;
}

// LGL differentiation matrix on [-1, 1] (Legendre closed form):
// D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j, D_00 = -N(N+1)/4,
// D_NN = N(N+1)/4, other diagonal entries 0.
std::vector<double> lgl_diff(const std::vector<double>& x) {
  const int n = (int)x.size(), N = n - 1;
  std::vector<double> p(n), D((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double pn1;
    legendre_pair(N, x[i], &p[i], &pn1);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (i != j) D[(size_t)i * n + j] = p[i] / (p[j] * (x[i] - x[j]));
  D[0] = -0.25 * N * (N + 1.0);
  D[(size_t)N * n + N] = 0.25 * N * (N + 1.0);
  return D;
}

// Value at t of the real trigonometric interpolant of the unit sample at
// k h (n samples over the period L): the Dirichlet kernel
// sin((M + 1/2) th) / sin(th / 2) / n over |m| <= M, th = 2 pi (t - k h) / L,
// plus cos(n th / 2) / n for the Nyquist mode of even n.
double trig_weight(int n, double L, double t, int k) {
  const double th = 2.0 * PI * (t - k * (L / n)) / L;
  const int M = (n - 1) / 2;
  const double s = std::sin(0.5 * th);
  double v = (std::fabs(s) < 1e-13) ? (2.0 * M + 1.0) : std::sin((M + 0.5) * th) / s;
  if (n % 2 == 0) v += std::cos(0.5 * n * th);
  return v / n;
}

}  // namespace

// ------------------------------------------------------------------ context

struct dgdft_dg {
  dgdft_dg_config cfg{};
  std::string err;
  cudaStream_t st = nullptr;
  int nel = 0, J = 0, nL = 0, ngq = 0;
  int nl[3]{}, nq[3]{}, nf[3]{};  // nf[d]: points of a face normal to d
  std::vector<double> xr[3], wr[3], local[3], w1[3];
  double le[3]{}, e_off[3]{};
  // device tables
  double *d_I[3]{}, *d_D[3]{}, *d_w = nullptr, *d_wf[3]{};
  // inputs
  double* d_v = nullptr;  // nel x nL
  std::vector<double> gamma;
  struct Proj {
    std::vector<int> pid;
    std::vector<long long> ptr;
    std::vector<int> idx;
    std::vector<double> val;
  };
  std::vector<Proj> proj;
  // persistent results
  double* d_pool = nullptr;   // volume (5 per element) and face (7 per face) matrices
  double* d_traces = nullptr;
  long long tr_elem = 0, tr_off[6]{};
  double* d_linv = nullptr;
  double* d_H = nullptr;      // all blocks, row by row
  int* d_bad = nullptr;
  std::vector<std::vector<int>> nb;
  std::vector<int> row_first;  // first block of each row
  int nblk = 0;
  bool assembled = false;
  double ms[6]{};
  double density_ms[2]{};  // eigensolve, density evaluation
  int density_sweeps = 0;  // Jacobi sweeps of the last density
  int launches = 0;
  // batch scratch
  int batch = 0;
  double *d_z = nullptr, *d_t1 = nullptr, *d_t2 = nullptr, *d_phi = nullptr, *d_g[3]{};
  double* d_part = nullptr;
  size_t part_cap = 0;
  size_t t1_elem = 0, t2_elem = 0;

  dgdft_status fail(dgdft_status s, const std::string& m) {
    err = m;
    return s;
  }
  long long vol_mat(int e, int k) const { return ((long long)e * 5 + k) * J * J; }
  long long face_mat(int e, int d, int k) const { return (((long long)nel * 5) + ((long long)e * 3 + d) * 7 + k) * J * J; }
  int index(int ix, int iy, int iz) const {
    const int* n = cfg.ne;
    ix = ((ix % n[0]) + n[0]) % n[0];
    iy = ((iy % n[1]) + n[1]) % n[1];
    iz = ((iz % n[2]) + n[2]) % n[2];
    return ix + n[0] * (iy + n[1] * iz);
  }
  void coords(int k, int* c) const {
    c[0] = k % cfg.ne[0];
    c[1] = (k / cfg.ne[0]) % cfg.ne[1];
    c[2] = k / (cfg.ne[0] * cfg.ne[1]);
  }
};

namespace {

bool cuda_ok(dgdft_dg* dg, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  dg->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

template <class T> bool dmalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

template <class T> bool upload(dgdft_dg* dg, T** p, const std::vector<T>& h) {
  if (!dmalloc(p, h.size())) return false;
  if (h.empty()) return true;
  return cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, dg->st) == cudaSuccess &&
         cudaStreamSynchronize(dg->st) == cudaSuccess;
}

size_t axis_smem(int nin, int nout) {
  return sizeof(double) * ((size_t)nout * nin + (size_t)std::max(nin, nout) * AX_LD);
}

template <bool FAST, int R>
void launch_axis_r(dgdft_dg* dg, const AxisJob& jb, unsigned tiles, int nelem, size_t sm) {
  if (dg->cfg.arith)
    dg_axis_kernel<FAST, R, dfl><<<dim3(tiles, nelem), AX_THREADS, sm, dg->st>>>(jb);
  else
    dg_axis_kernel<FAST, R, double><<<dim3(tiles, nelem), AX_THREADS, sm, dg->st>>>(jb);
}

template <bool FAST>
void launch_axis_fast(dgdft_dg* dg, const AxisJob& jb, unsigned tiles, int nelem, size_t sm) {
  const int need = (jb.n_out + AX_NR - 1) / AX_NR;
  if (need <= 4) launch_axis_r<FAST, 4>(dg, jb, tiles, nelem, sm);
  else if (need <= 8) launch_axis_r<FAST, 8>(dg, jb, tiles, nelem, sm);
  else if (need <= 12) launch_axis_r<FAST, 12>(dg, jb, tiles, nelem, sm);
  else if (need <= 16) launch_axis_r<FAST, 16>(dg, jb, tiles, nelem, sm);
  else if (need <= 20) launch_axis_r<FAST, 20>(dg, jb, tiles, nelem, sm);
  else if (need <= 24) launch_axis_r<FAST, 24>(dg, jb, tiles, nelem, sm);
  else launch_axis_r<FAST, 32>(dg, jb, tiles, nelem, sm);
}

template <bool FAST, int R> bool set_smem_r(int bytes) {
  return cudaFuncSetAttribute(dg_axis_kernel<FAST, R, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes) == cudaSuccess &&
         cudaFuncSetAttribute(dg_axis_kernel<FAST, R, dfl>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess;
}

template <bool FAST> bool set_axis_smem(int bytes) {
  return set_smem_r<FAST, 4>(bytes) && set_smem_r<FAST, 8>(bytes) && set_smem_r<FAST, 12>(bytes) &&
         set_smem_r<FAST, 16>(bytes) && set_smem_r<FAST, 20>(bytes) && set_smem_r<FAST, 24>(bytes) &&
         set_smem_r<FAST, 32>(bytes);
}

// A (n_out x n_in) along one axis of nelem arrays [O][n_in][S]; element e
// uses A + e * a_stride.
bool launch_axis(dgdft_dg* dg, const double* const* d_in, double* const* d_out, int nelem, const double* A,
                 int nin, int nout, int S, long long O, long long a_stride = 0) {
  AxisJob jb{d_in, d_out, A, a_stride, nin, nout, S, O};
  const long long cols = (S == 1) ? O : O * S;
  const unsigned tiles = (unsigned)((cols + AX_TC - 1) / AX_TC);
  const size_t sm = axis_smem(nin, nout);
  if (S == 1)
    launch_axis_fast<true>(dg, jb, tiles, nelem, sm);
  else
    launch_axis_fast<false>(dg, jb, tiles, nelem, sm);
  ++dg->launches;
  return cuda_ok(dg, cudaGetLastError(), "axis kernel");
}

bool run_grams(dgdft_dg* dg, std::vector<GramTask>& tasks) {
  if (tasks.empty()) return true;
  long long part = 0;
  int maxc = 0, maxJ1 = 0, maxJ2 = 0;
  for (GramTask& t : tasks) {
    t.nchunk = (t.n + GR_CH - 1) / GR_CH;
    t.part = part;
    part += (long long)t.nchunk * t.J1 * t.J2;
    maxc = std::max(maxc, t.nchunk);
    maxJ1 = std::max(maxJ1, t.J1);
    maxJ2 = std::max(maxJ2, t.J2);
  }
  if ((size_t)part > dg->part_cap) {
    cudaFree(dg->d_part);
    dg->d_part = nullptr;
    dg->part_cap = 0;
    if (!dmalloc(&dg->d_part, (size_t)part)) {
      dg->err = "Gram partials: out of memory";
      return false;
    }
    dg->part_cap = (size_t)part;
  }
  GramTask* d_t = nullptr;
  std::vector<GramTask> h(tasks);
  if (!dmalloc(&d_t, h.size())) {
    dg->err = "Gram tasks: out of memory";
    return false;
  }
  bool ok = cuda_ok(dg, cudaMemcpyAsync(d_t, h.data(), h.size() * sizeof(GramTask), cudaMemcpyHostToDevice, dg->st),
                    "Gram tasks");
  const int ntiles = ((maxJ1 + 1) / 2) * ((maxJ2 + 1) / 2);
  if (ok) {
    const dim3 grid(maxc, (unsigned)h.size(), (ntiles + 255) / 256);
    if (dg->cfg.arith)
      dg_gram_kernel<dfl><<<grid, 256, 0, dg->st>>>(d_t, dg->d_part);
    else
      dg_gram_kernel<double><<<grid, 256, 0, dg->st>>>(d_t, dg->d_part);
    dg_gram_reduce_kernel<<<dim3(std::max(1, (maxJ1 * maxJ2 + 255) / 256), (unsigned)h.size()), 256, 0, dg->st>>>(
        d_t, dg->d_part);
    dg->launches += 2;
    ok = cuda_ok(dg, cudaGetLastError(), "Gram kernel") && cuda_ok(dg, cudaStreamSynchronize(dg->st), "Gram kernel");
  }
  cudaFree(d_t);
  return ok;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Interpolation of a batch's columns to the LGL grids (into d_phi).
bool interp_batch(dgdft_dg* dg, int nb, const double* const* h_in) {
  const int J = dg->J;
  std::vector<const double*> cin;
  std::vector<double*> cout;
  for (int e = 0; e < nb; ++e) cin.push_back(h_in[e]);
  for (int e = 0; e < nb; ++e) cin.push_back(dg->d_t1 + e * dg->t1_elem);
  for (int e = 0; e < nb; ++e) cin.push_back(dg->d_t2 + e * dg->t2_elem);
  for (int e = 0; e < nb; ++e) cout.push_back(dg->d_t1 + e * dg->t1_elem);
  for (int e = 0; e < nb; ++e) cout.push_back(dg->d_t2 + e * dg->t2_elem);
  for (int e = 0; e < nb; ++e) cout.push_back(dg->d_phi + (size_t)e * J * dg->nL);
  const double** d_in = nullptr;
  double** d_out = nullptr;
  if (!dmalloc(&d_in, cin.size()) || !dmalloc(&d_out, cout.size())) {
    cudaFree(d_in);
    dg->err = "pointer tables: out of memory";
    return false;
  }
  bool ok = cuda_ok(dg, cudaMemcpyAsync(d_in, cin.data(), cin.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                    "pointer tables") &&
            cuda_ok(dg, cudaMemcpyAsync(d_out, cout.data(), cout.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                    "pointer tables");
  const int *nq = dg->nq, *nl = dg->nl;
  Timer tm(dg->st);
  // x: lines of Q_K (J nqz nqy lines of nqx) -> nlx
  ok = ok && launch_axis(dg, d_in, d_out, nb, dg->d_I[0], nq[0], nl[0], 1, (long long)J * nq[2] * nq[1]);
  // y: [J nqz][nqy][nlx] -> nly
  ok = ok && launch_axis(dg, d_in + nb, d_out + nb, nb, dg->d_I[1], nq[1], nl[1], nl[0], (long long)J * nq[2]);
  // z: [J][nqz][nly nlx] -> nlz
  ok = ok && launch_axis(dg, d_in + 2 * nb, d_out + 2 * nb, nb, dg->d_I[2], nq[2], nl[2], nl[0] * nl[1], J);
  dg->ms[0] += tm.stop();
  ok = ok && cuda_ok(dg, cudaStreamSynchronize(dg->st), "interpolation");
  cudaFree(d_in);
  cudaFree(d_out);
  return ok;
}

// Gradients of the batch's d_phi along x, y, z (into d_g[0..2]).
bool grad_batch(dgdft_dg* dg, int nb) {
  const int J = dg->J;
  std::vector<const double*> cin;
  std::vector<double*> cout;
  for (int e = 0; e < nb; ++e) cin.push_back(dg->d_phi + (size_t)e * J * dg->nL);
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < nb; ++e) cout.push_back(dg->d_g[d] + (size_t)e * J * dg->nL);
  const double** d_in = nullptr;
  double** d_out = nullptr;
  if (!dmalloc(&d_in, cin.size()) || !dmalloc(&d_out, cout.size())) {
    cudaFree(d_in);
    dg->err = "pointer tables: out of memory";
    return false;
  }
  bool ok = cuda_ok(dg, cudaMemcpyAsync(d_in, cin.data(), cin.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                    "pointer tables") &&
            cuda_ok(dg, cudaMemcpyAsync(d_out, cout.data(), cout.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                    "pointer tables");
  const int* nl = dg->nl;
  ok = ok && launch_axis(dg, d_in, d_out, nb, dg->d_D[0], nl[0], nl[0], 1, (long long)J * nl[2] * nl[1]);
  ok = ok && launch_axis(dg, d_in, d_out + nb, nb, dg->d_D[1], nl[1], nl[1], nl[0], (long long)J * nl[2]);
  ok = ok && launch_axis(dg, d_in, d_out + 2 * nb, nb, dg->d_D[2], nl[2], nl[2], nl[0] * nl[1], J);
  ok = ok && cuda_ok(dg, cudaStreamSynchronize(dg->st), "gradients");
  cudaFree(d_in);
  cudaFree(d_out);
  return ok;
}

// Eq. orthonormal for the batch's d_phi: mass matrices (into mass, J x J per
// element), Cholesky and L^-1 (into linv), phi = phi~ L^-T (written to d_g[2],
// whose buffer then becomes d_phi).  bad[e] = 1 where M is not positive definite.
bool ortho_batch(dgdft_dg* dg, int nb, double* mass, long long mass_stride, double* linv, int* bad) {
  const int J = dg->J;
  std::vector<GramTask> tasks;
  for (int e = 0; e < nb; ++e) {
    GramTask t{};
    t.X = t.Y = dg->d_phi + (size_t)e * J * dg->nL;
    t.w = dg->d_w;
    t.out = mass + (size_t)e * mass_stride;
    t.n = t.ldx = t.ldy = dg->nL;
    t.J1 = t.J2 = J;
    t.sym = 1;
    tasks.push_back(t);
  }
  if (!run_grams(dg, tasks)) return false;
  dg_chol_kernel<<<nb, 256, (size_t)J * J * sizeof(double), dg->st>>>(mass, mass_stride, linv, J, bad);
  ++dg->launches;
  if (!cuda_ok(dg, cudaGetLastError(), "orthonormalisation")) return false;
  // phi = phi~ L^-T: L^-1 along the J axis of [1][J][n_LGL]
  std::vector<const double*> cin;
  std::vector<double*> cout;
  for (int e = 0; e < nb; ++e) cin.push_back(dg->d_phi + (size_t)e * J * dg->nL);
  for (int e = 0; e < nb; ++e) cout.push_back(dg->d_g[2] + (size_t)e * J * dg->nL);
  const double** d_in = nullptr;
  double** d_out = nullptr;
  if (!dmalloc(&d_in, cin.size()) || !dmalloc(&d_out, cout.size())) {
    cudaFree(d_in);
    dg->err = "pointer tables: out of memory";
    return false;
  }
  bool ok = cuda_ok(dg, cudaMemcpyAsync(d_in, cin.data(), cin.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                    "pointer tables") &&
            cuda_ok(dg, cudaMemcpyAsync(d_out, cout.data(), cout.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                    "pointer tables") &&
            launch_axis(dg, d_in, d_out, nb, linv, J, J, dg->nL, 1, (long long)J * J) &&
            cuda_ok(dg, cudaStreamSynchronize(dg->st), "orthonormalisation");
  cudaFree(d_in);
  cudaFree(d_out);
  std::swap(dg->d_phi, dg->d_g[2]);
  return ok;
}

bool ensure_batch(dgdft_dg* dg, int nb) {
  if (nb <= dg->batch) return true;
  for (double* p : {dg->d_z, dg->d_t1, dg->d_t2, dg->d_phi, dg->d_g[0], dg->d_g[1], dg->d_g[2]}) cudaFree(p);
  dg->d_z = dg->d_t1 = dg->d_t2 = dg->d_phi = dg->d_g[0] = dg->d_g[1] = dg->d_g[2] = nullptr;
  dg->batch = 0;
  const size_t per = (size_t)dg->J * dg->nL;
  if (!dmalloc(&dg->d_z, (size_t)nb * dg->J * dg->ngq) || !dmalloc(&dg->d_t1, nb * dg->t1_elem) ||
      !dmalloc(&dg->d_t2, nb * dg->t2_elem) || !dmalloc(&dg->d_phi, nb * per) || !dmalloc(&dg->d_g[0], nb * per) ||
      !dmalloc(&dg->d_g[1], nb * per) || !dmalloc(&dg->d_g[2], nb * per)) {
    dg->err = "batch scratch: out of memory";
    return false;
  }
  dg->batch = nb;
  return true;
}

size_t batch_bytes(const dgdft_dg* dg) {
  const size_t per = (size_t)dg->J * dg->nL;
  const size_t nchunk = (dg->nL + GR_CH - 1) / GR_CH;
  return sizeof(double) * ((size_t)dg->J * dg->ngq + dg->t1_elem + dg->t2_elem + 4 * per +
                           5 * nchunk * dg->J * dg->J);
}

}  // namespace

extern "C" {

dgdft_status dgdft_dg_create(const dgdft_dg_config* cfg, dgdft_dg** out) {
  if (!out) return DGDFT_EINVAL;
  *out = nullptr;
  if (!cfg) return DGDFT_EINVAL;
  dgdft_dg* dg = new dgdft_dg();
  *out = dg;
  dg->cfg = *cfg;
  const dgdft_dg_config& c = *cfg;
  for (int d = 0; d < 3; ++d) {
    if (c.ne[d] < 1) return dg->fail(DGDFT_EINVAL, "ne must be >= 1");
    if (!(c.cell[d] > 0.0) || !std::isfinite(c.cell[d])) return dg->fail(DGDFT_EINVAL, "cell must be positive");
    if (!(c.q_span[d] == 3 || (c.q_span[d] == 1 && c.ne[d] == 1)))
      return dg->fail(DGDFT_EINVAL, "q_span must be 3, or 1 with ne = 1");
    if (c.nq[d] < 2 || c.nq[d] > 1024) return dg->fail(DGDFT_EINVAL, "nq out of range");
    if (c.nl[d] < 2 || c.nl[d] > MAX_NL) return dg->fail(DGDFT_EINVAL, "nl out of range (2..128)");
  }
  if (c.J < 1 || c.J > MAX_J) return dg->fail(DGDFT_EINVAL, "J out of range (1..128)");
  if (!(c.alpha >= 0.0) || !std::isfinite(c.alpha)) return dg->fail(DGDFT_EINVAL, "alpha must be >= 0");
  if (c.n_proj < 0) return dg->fail(DGDFT_EINVAL, "n_proj must be >= 0");
  if (c.arith != 0 && c.arith != 1) return dg->fail(DGDFT_EINVAL, "arith must be 0 (FP64) or 1 (double-float)");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return dg->fail(DGDFT_ECUDA, "no CUDA device");
  if (c.device < 0 || c.device >= ndev || cudaSetDevice(c.device) != cudaSuccess)
    return dg->fail(DGDFT_ECUDA, "bad device");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c.device) != cudaSuccess || prop.major != 10 || prop.minor != 3)
    return dg->fail(DGDFT_ECUDA, "an sm_103 device is required");
  dg->st = static_cast<cudaStream_t>(c.cuda_stream);
  dg->nel = c.ne[0] * c.ne[1] * c.ne[2];
  dg->J = c.J;
  for (int d = 0; d < 3; ++d) {
    dg->nl[d] = c.nl[d];
    dg->nq[d] = c.nq[d];
    dg->le[d] = c.cell[d] / c.ne[d];
    dg->e_off[d] = dg->le[d] * (c.q_span[d] / 2);
  }
  dg->nL = dg->nl[0] * dg->nl[1] * dg->nl[2];
  dg->ngq = dg->nq[0] * dg->nq[1] * dg->nq[2];
  dg->nf[0] = dg->nl[1] * dg->nl[2];
  dg->nf[1] = dg->nl[0] * dg->nl[2];
  dg->nf[2] = dg->nl[0] * dg->nl[1];
  dg->t1_elem = (size_t)c.J * dg->nq[2] * dg->nq[1] * dg->nl[0];
  dg->t2_elem = (size_t)c.J * dg->nq[2] * dg->nl[1] * dg->nl[0];
  // shared memory of every axis pass
  size_t smax = axis_smem(c.J, c.J);
  for (int d = 0; d < 3; ++d) smax = std::max({smax, axis_smem(dg->nq[d], dg->nl[d]), axis_smem(dg->nl[d], dg->nl[d])});
  if (smax > 220 * 1024) return dg->fail(DGDFT_EINVAL, "grids too large for the interpolation kernel");
  if (!set_axis_smem<true>((int)smax) || !set_axis_smem<false>((int)smax) ||
      cudaFuncSetAttribute(dg_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(c.J * c.J * sizeof(double))) != cudaSuccess)
    return dg->fail(DGDFT_ECUDA, "kernel attributes");
  // tables
  std::vector<double> hI[3], hD[3];
  for (int d = 0; d < 3; ++d) {
    if (!lgl_rule(dg->nl[d], dg->xr[d], dg->wr[d])) return dg->fail(DGDFT_EINVAL, "LGL nodes did not converge");
    dg->local[d].resize(dg->nl[d]);
    dg->w1[d].resize(dg->nl[d]);
    for (int j = 0; j < dg->nl[d]; ++j) {
      dg->local[d][j] = 0.5 * (dg->xr[d][j] + 1.0) * dg->le[d];
      dg->w1[d][j] = 0.5 * dg->wr[d][j] * dg->le[d];
    }
    hD[d] = lgl_diff(dg->xr[d]);
    for (double& v : hD[d]) v *= 2.0 / dg->le[d];
    const double lq = dg->le[d] * c.q_span[d];
    hI[d].resize((size_t)dg->nl[d] * dg->nq[d]);
    for (int j = 0; j < dg->nl[d]; ++j)
      for (int k = 0; k < dg->nq[d]; ++k)
        hI[d][(size_t)j * dg->nq[d] + k] = trig_weight(dg->nq[d], lq, dg->e_off[d] + dg->local[d][j], k);
  }
  std::vector<double> hw(dg->nL), hf[3];
  for (int z = 0; z < dg->nl[2]; ++z)
    for (int y = 0; y < dg->nl[1]; ++y)
      for (int x = 0; x < dg->nl[0]; ++x)
        hw[x + dg->nl[0] * (y + dg->nl[1] * z)] = dg->w1[0][x] * dg->w1[1][y] * dg->w1[2][z];
  hf[0].resize(dg->nf[0]);
  for (int z = 0; z < dg->nl[2]; ++z)
    for (int y = 0; y < dg->nl[1]; ++y) hf[0][y + dg->nl[1] * z] = dg->w1[1][y] * dg->w1[2][z];
  hf[1].resize(dg->nf[1]);
  for (int z = 0; z < dg->nl[2]; ++z)
    for (int x = 0; x < dg->nl[0]; ++x) hf[1][x + dg->nl[0] * z] = dg->w1[0][x] * dg->w1[2][z];
  hf[2].resize(dg->nf[2]);
  for (int y = 0; y < dg->nl[1]; ++y)
    for (int x = 0; x < dg->nl[0]; ++x) hf[2][x + dg->nl[0] * y] = dg->w1[0][x] * dg->w1[1][y];
  for (int d = 0; d < 3; ++d)
    if (!upload(dg, &dg->d_I[d], hI[d]) || !upload(dg, &dg->d_D[d], hD[d]) || !upload(dg, &dg->d_wf[d], hf[d]))
      return dg->fail(DGDFT_ENOMEM, "tables");
  if (!upload(dg, &dg->d_w, hw)) return dg->fail(DGDFT_ENOMEM, "tables");
  // neighbourhoods and block rows
  dg->nb.resize(dg->nel);
  dg->row_first.resize(dg->nel + 1, 0);
  for (int k = 0; k < dg->nel; ++k) {
    int cc[3];
    dg->coords(k, cc);
    std::vector<int> s;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        for (int g = -1; g <= 1; ++g) s.push_back(dg->index(cc[0] + a, cc[1] + b, cc[2] + g));
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    dg->nb[k] = s;
    dg->row_first[k + 1] = dg->row_first[k] + (int)s.size();
  }
  dg->nblk = dg->row_first[dg->nel];
  // face trace layout per element: slot = 2 d + high, F then DF
  long long off = 0;
  for (int slot = 0; slot < 6; ++slot) {
    dg->tr_off[slot] = off;
    off += 2LL * dg->nf[slot / 2] * c.J;
  }
  dg->tr_elem = off;
  const size_t JJ = (size_t)c.J * c.J;
  dg->proj.resize(dg->nel);
  dg->gamma.assign(c.n_proj, 0.0);
  if (!dmalloc(&dg->d_v, (size_t)dg->nel * dg->nL) ||
      !dmalloc(&dg->d_pool, ((size_t)dg->nel * 5 + (size_t)dg->nel * 3 * 7) * JJ) ||
      !dmalloc(&dg->d_traces, (size_t)dg->nel * dg->tr_elem) || !dmalloc(&dg->d_linv, (size_t)dg->nel * JJ) ||
      !dmalloc(&dg->d_H, (size_t)dg->nblk * JJ) ||
      !dmalloc(&dg->d_bad, (size_t)dg->nel))
    return dg->fail(DGDFT_ENOMEM, "element storage");
  if (cudaMemsetAsync(dg->d_v, 0, sizeof(double) * dg->nel * dg->nL, dg->st) != cudaSuccess ||
      cudaStreamSynchronize(dg->st) != cudaSuccess)
    return dg->fail(DGDFT_ECUDA, "init");
  return DGDFT_OK;
}

dgdft_status dgdft_dg_lgl_points(dgdft_dg* dg, int elem, double* x, double* y, double* z) {
  if (!dg || elem < 0 || elem >= dg->nel || !x || !y || !z) return DGDFT_EINVAL;
  int c[3];
  dg->coords(elem, c);
  double* o[3] = {x, y, z};
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < dg->nl[d]; ++j) o[d][j] = c[d] * dg->le[d] + dg->local[d][j];
  return DGDFT_OK;
}

dgdft_status dgdft_dg_set_potential(dgdft_dg* dg, int elem, const double* v, int on_device) {
  if (!dg || elem < 0 || elem >= dg->nel || !v) return DGDFT_EINVAL;
  if (cudaMemcpyAsync(dg->d_v + (size_t)elem * dg->nL, v, sizeof(double) * dg->nL,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, dg->st) != cudaSuccess ||
      cudaStreamSynchronize(dg->st) != cudaSuccess)
    return dg->fail(DGDFT_ECUDA, "set_potential copy");
  dg->assembled = false;
  return DGDFT_OK;
}

dgdft_status dgdft_dg_set_gamma(dgdft_dg* dg, const double* gamma) {
  if (!dg || (!gamma && dg->cfg.n_proj > 0)) return DGDFT_EINVAL;
  for (int p = 0; p < dg->cfg.n_proj; ++p) {
    if (!std::isfinite(gamma[p])) return dg->fail(DGDFT_EINVAL, "gamma must be finite");
    dg->gamma[p] = gamma[p];
  }
  dg->assembled = false;
  return DGDFT_OK;
}

dgdft_status dgdft_dg_set_projectors(dgdft_dg* dg, int elem, int n_p, const int* pid, const int64_t* row_ptr,
                                     const int* idx, const double* val) {
  if (!dg || elem < 0 || elem >= dg->nel || n_p < 0) return DGDFT_EINVAL;
  if (n_p > 0 && (!pid || !row_ptr)) return DGDFT_EINVAL;
  dgdft_dg::Proj P;
  P.ptr.push_back(0);
  std::vector<int> seen;
  for (int r = 0; r < n_p; ++r) {
    if (pid[r] < 0 || pid[r] >= dg->cfg.n_proj) return dg->fail(DGDFT_EINVAL, "projector id out of range");
    seen.push_back(pid[r]);
    if (row_ptr[r + 1] < row_ptr[r] || (row_ptr[r + 1] > row_ptr[r] && (!idx || !val)))
      return dg->fail(DGDFT_EINVAL, "bad projector CSR");
    for (int64_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
      if (idx[q] < 0 || idx[q] >= dg->nL) return dg->fail(DGDFT_EINVAL, "projector index out of range");
      if (!std::isfinite(val[q])) return dg->fail(DGDFT_EINVAL, "projector value not finite");
      P.idx.push_back(idx[q]);
      P.val.push_back(val[q]);
    }
    P.pid.push_back(pid[r]);
    P.ptr.push_back((long long)P.idx.size());
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return dg->fail(DGDFT_EINVAL, "duplicate projector id");
  dg->proj[elem] = std::move(P);
  dg->assembled = false;
  return DGDFT_OK;
}

dgdft_status dgdft_dg_neighbours(dgdft_dg* dg, int elem, int* nb, int* n_nb) {
  if (!dg || elem < 0 || elem >= dg->nel || !nb || !n_nb) return DGDFT_EINVAL;
  *n_nb = (int)dg->nb[elem].size();
  for (int s = 0; s < *n_nb; ++s) nb[s] = dg->nb[elem][s];
  return DGDFT_OK;
}

dgdft_status dgdft_dg_assemble(dgdft_dg* dg, const double* const* z, int on_device) {
  if (!dg) return DGDFT_EINVAL;
  if (!z) return dg->fail(DGDFT_EINVAL, "z is NULL");
  for (int k = 0; k < dg->nel; ++k)
    if (!z[k]) return dg->fail(DGDFT_EINVAL, "z[" + std::to_string(k) + "] is NULL");
  dg->assembled = false;
  for (double& m : dg->ms) m = 0.0;
  dg->launches = 0;
  const int J = dg->J, nel = dg->nel;
  const size_t JJ = (size_t)J * J;
  // batch size from the scratch budget
  size_t cap = dg->cfg.hbm_cap_bytes;
  if (!cap) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return dg->fail(DGDFT_ECUDA, "cudaMemGetInfo");
    cap = fr / 4;
  }
  const int nbat = (int)std::max<size_t>(1, std::min<size_t>(nel, cap / std::max<size_t>(1, batch_bytes(dg))));
  if (!ensure_batch(dg, nbat)) return DGDFT_ENOMEM;
  // KB rows: global numbering over elements
  std::vector<long long> kb_ptr_h{0};
  std::vector<int> kb_idx_h, row_elem_global, row_first_of(nel + 1, 0);
  std::vector<double> kb_wval_h;
  std::vector<double> hw(dg->nL);
  for (int zz = 0; zz < dg->nl[2]; ++zz)
    for (int y = 0; y < dg->nl[1]; ++y)
      for (int x = 0; x < dg->nl[0]; ++x)
        hw[x + dg->nl[0] * (y + dg->nl[1] * zz)] = dg->w1[0][x] * dg->w1[1][y] * dg->w1[2][zz];
  for (int k = 0; k < nel; ++k) {
    const auto& P = dg->proj[k];
    row_first_of[k] = (int)row_elem_global.size();
    for (size_t r = 0; r < P.pid.size(); ++r) {
      for (long long q = P.ptr[r]; q < P.ptr[r + 1]; ++q) {
        kb_idx_h.push_back(P.idx[q]);
        kb_wval_h.push_back(hw[P.idx[q]] * P.val[q]);
      }
      kb_ptr_h.push_back((long long)kb_idx_h.size());
      row_elem_global.push_back(k);
    }
  }
  row_first_of[nel] = (int)row_elem_global.size();
  const int nrows = (int)row_elem_global.size();
  long long* d_kb_ptr = nullptr;
  int *d_kb_idx = nullptr, *d_row_elem = nullptr;
  double *d_kb_wval = nullptr, *d_coef = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_kb_ptr);
    cudaFree(d_kb_idx);
    cudaFree(d_row_elem);
    cudaFree(d_kb_wval);
    cudaFree(d_coef);
  };
  if (!upload(dg, &d_kb_ptr, kb_ptr_h) || !upload(dg, &d_kb_idx, kb_idx_h) || !upload(dg, &d_kb_wval, kb_wval_h) ||
      !dmalloc(&d_coef, (size_t)std::max(1, nrows) * J) || !dmalloc(&d_row_elem, (size_t)std::max(1, nrows))) {
    cleanup();
    return dg->fail(DGDFT_ENOMEM, "KB storage");
  }
  // ---- per batch: interpolation, gradients, volume Grams, traces, KB
  for (int g0 = 0; g0 < nel; g0 += nbat) {
    const int nb = std::min(nbat, nel - g0);
    std::vector<const double*> src(nb);
    for (int e = 0; e < nb; ++e) {
      if (on_device) {
        src[e] = z[g0 + e];
      } else {
        double* dst = dg->d_z + (size_t)e * J * dg->ngq;
        if (cudaMemcpyAsync(dst, z[g0 + e], sizeof(double) * J * dg->ngq, cudaMemcpyHostToDevice, dg->st) !=
            cudaSuccess) {
          cleanup();
          return dg->fail(DGDFT_ECUDA, "copy of z");
        }
        src[e] = dst;
      }
    }
    if (!interp_batch(dg, nb, src.data())) {
      cleanup();
      return DGDFT_ECUDA;
    }
    {
      Timer tm(dg->st);
      if (!ortho_batch(dg, nb, dg->d_pool + dg->vol_mat(g0, 0), 5 * (long long)JJ, dg->d_linv + (size_t)g0 * JJ,
                       dg->d_bad + g0) ||
          !grad_batch(dg, nb)) {
        cleanup();
        return DGDFT_ECUDA;
      }
      dg->ms[1] += tm.stop();
    }
    {
      Timer tm(dg->st);
      std::vector<GramTask> tasks;
      for (int e = 0; e < nb; ++e) {
        const int k = g0 + e;
        const double* phi = dg->d_phi + (size_t)e * J * dg->nL;
        GramTask t{};
        t.n = dg->nL;
        t.ldx = t.ldy = dg->nL;
        t.J1 = t.J2 = J;
        t.w = dg->d_w;
        t.X = t.Y = phi;
        t.sym = 1;
        t.v = dg->d_v + (size_t)k * dg->nL;  // V_eff
        t.out = dg->d_pool + dg->vol_mat(k, 1);
        tasks.push_back(t);
        t.v = nullptr;
        for (int d = 0; d < 3; ++d) {
          t.X = t.Y = dg->d_g[d] + (size_t)e * J * dg->nL;
          t.out = dg->d_pool + dg->vol_mat(k, 2 + d);
          tasks.push_back(t);
        }
      }
      if (!run_grams(dg, tasks)) {
        cleanup();
        return DGDFT_ECUDA;
      }
      dg->ms[2] += tm.stop();
    }
    {
      Timer tm(dg->st);
      TraceJob tj{};
      tj.phi = dg->d_phi;
      for (int d = 0; d < 3; ++d) tj.grad[d] = dg->d_g[d];
      tj.traces = dg->d_traces;
      tj.tr_elem = dg->tr_elem;
      for (int s = 0; s < 6; ++s) {
        tj.tr_off[s] = dg->tr_off[s];
        tj.nf[s] = dg->nf[s / 2];
      }
      for (int d = 0; d < 3; ++d) tj.nl[d] = dg->nl[d];
      tj.J = J;
      tj.nL = dg->nL;
      tj.g0 = g0;
      dg_trace_kernel<<<dim3(64, 6, nb), 256, 0, dg->st>>>(tj);
      ++dg->launches;
      const int r0 = row_first_of[g0], r1 = row_first_of[g0 + nb];
      if (r1 > r0) {
        std::vector<int> re(r1 - r0);
        for (int r = r0; r < r1; ++r) re[r - r0] = row_elem_global[r] - g0;
        if (cudaMemcpyAsync(d_row_elem, re.data(), sizeof(int) * re.size(), cudaMemcpyHostToDevice, dg->st) !=
            cudaSuccess) {
          cleanup();
          return dg->fail(DGDFT_ECUDA, "KB rows");
        }
        KbJob kj{dg->d_phi, d_row_elem, d_kb_ptr, d_kb_idx, d_kb_wval, d_coef, r0, J, dg->nL};
        dg_kb_kernel<<<r1 - r0, 128, 0, dg->st>>>(kj);
        ++dg->launches;
      }
      if (!cuda_ok(dg, cudaGetLastError(), "trace/KB kernels") ||
          !cuda_ok(dg, cudaStreamSynchronize(dg->st), "trace/KB kernels")) {
        cleanup();
        return DGDFT_ECUDA;
      }
      dg->ms[3] += tm.stop();
    }
  }
  // ---- face integrals: face (a, d) between a (its high face, side 0) and
  // b = a + e_d (its low face, side 1); pool matrices 0..3 = S_fd[s][t]
  // (s = 2 * s + t), 4 = S_ff[0][0], 5 = S_ff[0][1], 6 = S_ff[1][1]
  {
    Timer tm(dg->st);
    std::vector<GramTask> tasks;
    for (int a = 0; a < nel; ++a) {
      int c[3];
      dg->coords(a, c);
      for (int d = 0; d < 3; ++d) {
        int cb[3] = {c[0], c[1], c[2]};
        cb[d] += 1;
        const int b = dg->index(cb[0], cb[1], cb[2]);
        const int nfc = dg->nf[d];
        const double* F[2] = {dg->d_traces + (size_t)a * dg->tr_elem + dg->tr_off[2 * d + 1],
                              dg->d_traces + (size_t)b * dg->tr_elem + dg->tr_off[2 * d]};
        const double* DF[2] = {F[0] + (size_t)nfc * J, F[1] + (size_t)nfc * J};
        GramTask t{};
        t.n = nfc;
        t.ldx = t.ldy = nfc;
        t.J1 = t.J2 = J;
        t.w = dg->d_wf[d];
        for (int s = 0; s < 2; ++s)
          for (int u = 0; u < 2; ++u) {
            t.X = F[s];
            t.Y = DF[u];
            t.out = dg->d_pool + dg->face_mat(a, d, 2 * s + u);
            tasks.push_back(t);
          }
        const int ff[3][2] = {{0, 0}, {0, 1}, {1, 1}};
        for (int q = 0; q < 3; ++q) {
          t.X = F[ff[q][0]];
          t.Y = F[ff[q][1]];
          t.sym = ff[q][0] == ff[q][1];
          t.out = dg->d_pool + dg->face_mat(a, d, 4 + q);
          tasks.push_back(t);
        }
      }
    }
    if (!run_grams(dg, tasks)) {
      cleanup();
      return DGDFT_ECUDA;
    }
    dg->ms[4] += tm.stop();
  }
  // ---- factorisation and blocks
  Timer tm(dg->st);
  std::vector<MatTerm> terms;
  std::vector<int> term_ptr{0}, kb_ptr{0};
  std::vector<KbTerm> kbt;
  const double alpha = dg->cfg.alpha;
  for (int k = 0; k < nel; ++k) {
    int c[3];
    dg->coords(k, c);
    for (int k2 : dg->nb[k]) {
      if (k2 == k) {
        terms.push_back({1.0, dg->vol_mat(k, 1), 0, 0});
        for (int d = 0; d < 3; ++d) terms.push_back({0.5, dg->vol_mat(k, 2 + d), 0, 0});
      }
      for (int d = 0; d < 3; ++d) {
        int cl[3] = {c[0], c[1], c[2]};
        cl[d] -= 1;
        const int lower = dg->index(cl[0], cl[1], cl[2]);
        std::vector<int> as{k};
        if (lower != k) as.push_back(lower);
        for (int a : as) {
          int ca[3];
          dg->coords(a, ca);
          ca[d] += 1;
          const int b = dg->index(ca[0], ca[1], ca[2]);
          auto in_face = [&](int e) { return e == a || e == b; };
          if (!in_face(k) || !in_face(k2)) continue;
          // jump and average coefficients of each side
          auto eps = [&](int s, int e) { return s == 0 ? (e == a ? 1.0 : 0.0) : (e == b ? -1.0 : 0.0); };
          auto del = [&](int s, int e) { return s == 0 ? (e == a ? 0.5 : 0.0) : (e == b ? 0.5 : 0.0); };
          for (int s = 0; s < 2; ++s)
            for (int u = 0; u < 2; ++u) {
              const double c1 = -0.5 * eps(s, k) * del(u, k2);  // jump_k W avg_k2^T
              const double c2 = -0.5 * del(s, k) * eps(u, k2);  // avg_k W jump_k2^T
              const double c3 = alpha * eps(s, k) * eps(u, k2);
              if (c1 != 0.0) terms.push_back({c1, dg->face_mat(a, d, 2 * s + u), 0, 0});
              if (c2 != 0.0) terms.push_back({c2, dg->face_mat(a, d, 2 * u + s), 1, 0});
              if (c3 != 0.0) {
                if (s == 1 && u == 0)
                  terms.push_back({c3, dg->face_mat(a, d, 5), 1, 0});
                else
                  terms.push_back({c3, dg->face_mat(a, d, 4 + (s == 0 && u == 0 ? 0 : (s == 0 ? 1 : 2))), 0, 0});
              }
            }
        }
      }
      term_ptr.push_back((int)terms.size());
      // KB: projectors present in both elements
      const auto& P1 = dg->proj[k];
      const auto& P2 = dg->proj[k2];
      for (size_t r1 = 0; r1 < P1.pid.size(); ++r1)
        for (size_t r2 = 0; r2 < P2.pid.size(); ++r2)
          if (P1.pid[r1] == P2.pid[r2])
            kbt.push_back({dg->gamma[P1.pid[r1]], row_first_of[k] + (int)r1, row_first_of[k2] + (int)r2});
      kb_ptr.push_back((int)kbt.size());
    }
  }
  MatTerm* d_terms = nullptr;
  KbTerm* d_kbt = nullptr;
  int *d_term_ptr = nullptr, *d_kbp = nullptr;
  bool ok = upload(dg, &d_terms, terms) && upload(dg, &d_kbt, kbt) && upload(dg, &d_term_ptr, term_ptr) &&
            upload(dg, &d_kbp, kb_ptr);
  if (ok) {
    BlockJob bj{dg->d_pool, d_terms, d_term_ptr, d_kbt, d_kbp, d_coef, dg->d_H, J};
    const unsigned gx = (unsigned)((JJ + 255) / 256);
    dg_block_sum_kernel<<<dim3(gx, dg->nblk), 256, 0, dg->st>>>(bj);
    ++dg->launches;
    ok = cuda_ok(dg, cudaGetLastError(), "block kernels") && cuda_ok(dg, cudaStreamSynchronize(dg->st), "block kernels");
  } else {
    dg->err = "block term lists: out of memory";
  }
  dg->ms[5] += tm.stop();
  for (void* p : {(void*)d_terms, (void*)d_kbt, (void*)d_term_ptr, (void*)d_kbp}) cudaFree(p);
  cleanup();
  if (!ok) return DGDFT_ECUDA;
  std::vector<int> bad(nel);
  if (cudaMemcpy(bad.data(), dg->d_bad, sizeof(int) * nel, cudaMemcpyDeviceToHost) != cudaSuccess)
    return dg->fail(DGDFT_ECUDA, "status copy");
  for (int k = 0; k < nel; ++k)
    if (bad[k])
      return dg->fail(DGDFT_ENOTCONV, "mass matrix of element " + std::to_string(k) + " is not positive definite");
  dg->assembled = true;
  return DGDFT_OK;
}

dgdft_status dgdft_dg_get_row(dgdft_dg* dg, int elem, double* blocks, int on_device) {
  if (!dg || elem < 0 || elem >= dg->nel || !blocks) return DGDFT_EINVAL;
  if (!dg->assembled) return dg->fail(DGDFT_ESTATE, "get_row before a successful assemble");
  const size_t JJ = (size_t)dg->J * dg->J;
  const size_t n = dg->nb[elem].size() * JJ;
  if (cudaMemcpyAsync(blocks, dg->d_H + (size_t)dg->row_first[elem] * JJ, n * sizeof(double),
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, dg->st) != cudaSuccess ||
      cudaStreamSynchronize(dg->st) != cudaSuccess)
    return dg->fail(DGDFT_ECUDA, "get_row copy");
  return DGDFT_OK;
}

dgdft_status dgdft_dg_lgl_basis(dgdft_dg* dg, int elem, const double* z, int z_on_device, double* phi,
                                int on_device) {
  if (!dg || elem < 0 || elem >= dg->nel || !z || !phi) return DGDFT_EINVAL;
  if (!ensure_batch(dg, 1)) return DGDFT_ENOMEM;
  const int J = dg->J;
  const double* src = z;
  if (!z_on_device) {
    if (cudaMemcpyAsync(dg->d_z, z, sizeof(double) * J * dg->ngq, cudaMemcpyHostToDevice, dg->st) != cudaSuccess)
      return dg->fail(DGDFT_ECUDA, "copy of z");
    src = dg->d_z;
  }
  const double* srcs[1] = {src};
  if (!interp_batch(dg, 1, srcs)) return DGDFT_ECUDA;
  double *d_mass = nullptr, *d_linv = nullptr;
  int* d_bad = nullptr;
  if (!dmalloc(&d_mass, (size_t)J * J) || !dmalloc(&d_linv, (size_t)J * J) || !dmalloc(&d_bad, 1)) {
    cudaFree(d_mass);
    cudaFree(d_linv);
    return dg->fail(DGDFT_ENOMEM, "lgl_basis scratch");
  }
  int bad = 0;
  bool ok = ortho_batch(dg, 1, d_mass, 0, d_linv, d_bad) &&
            cuda_ok(dg, cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, dg->st), "status") &&
            cuda_ok(dg, cudaMemcpyAsync(phi, dg->d_phi, sizeof(double) * J * dg->nL,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, dg->st),
                    "basis copy") &&
            cuda_ok(dg, cudaStreamSynchronize(dg->st), "lgl_basis");
  cudaFree(d_mass);
  cudaFree(d_linv);
  cudaFree(d_bad);
  if (!ok) return DGDFT_ECUDA;
  if (bad) return dg->fail(DGDFT_ENOTCONV, "mass matrix is not positive definite");
  return DGDFT_OK;
}

dgdft_status dgdft_dg_density(dgdft_dg* dg, const double* const* z, int z_on_device, int n_occ, double* eig,
                              double* rho, int on_device) {
  if (!dg) return DGDFT_EINVAL;
  const int J = dg->J, nel = dg->nel;
  const long long n = (long long)nel * J;
  if (!z || !eig || !rho || n_occ < 1 || n_occ > n) return dg->fail(DGDFT_EINVAL, "density: bad arguments");
  if (n > 4096) return dg->fail(DGDFT_EINVAL, "density: n_elem * J above 4096");
  for (int k = 0; k < nel; ++k)
    if (!z[k]) return dg->fail(DGDFT_EINVAL, "density: z[" + std::to_string(k) + "] is NULL");
  if (!dg->assembled) return dg->fail(DGDFT_ESTATE, "density before a successful assemble");
  const size_t JJ = (size_t)J * J;
  double *dA = nullptr, *dW = nullptr, *dY = nullptr, *dlo = nullptr, *dnrm = nullptr, *dP = nullptr,
         *drho = nullptr;
  int2* dkk = nullptr;
  int *dord = nullptr, *dsweeps = nullptr;
  unsigned long long* doff = nullptr;
  constexpr int MAX_SWEEPS = 40;
  auto release = [&]() {
    for (void* p : {(void*)dA, (void*)dW, (void*)dY, (void*)dlo, (void*)dnrm, (void*)dP, (void*)drho, (void*)dkk,
                    (void*)dord, (void*)dsweeps, (void*)doff})
      cudaFree(p);
  };
  std::vector<int2> kk;
  for (int k = 0; k < nel; ++k)
    for (int k2 : dg->nb[k]) kk.push_back(make_int2(k, k2));
  if (!dmalloc(&dA, (size_t)(n * n)) || !dmalloc(&dW, (size_t)(n * n)) || !dmalloc(&dY, (size_t)(n * n_occ)) || !dmalloc(&dlo, (size_t)n) || !dmalloc(&dnrm, (size_t)n) ||
      !dmalloc(&dP, (size_t)nel * JJ) || !dmalloc(&dord, (size_t)n_occ) || !dmalloc(&dsweeps, 1) ||
      !dmalloc(&doff, (size_t)MAX_SWEEPS) || !upload(dg, &dkk, kk) ||
      (!on_device && !dmalloc(&drho, (size_t)nel * dg->nL))) {
    release();
    return dg->fail(DGDFT_ENOMEM, "density storage");
  }
  double t_ms[2] = {0.0, 0.0};
  bool ok = cuda_ok(dg, cudaMemsetAsync(dA, 0, sizeof(double) * n * n, dg->st), "density") &&
            cuda_ok(dg, cudaMemsetAsync(doff, 0, sizeof(unsigned long long) * MAX_SWEEPS, dg->st), "density");
  {
    Timer tm(dg->st);
    const unsigned gx = (unsigned)((JJ + 255) / 256);
    const unsigned gw = (unsigned)((n * 32 + 255) / 256);
    std::vector<double> lo(n), lam(n);
    if (ok) {
      dg_dense_kernel<<<dim3(gx, dg->nblk), 256, 0, dg->st>>>(dg->d_H, dkk, dA, J, n);
      dg_gershgorin_kernel<<<gw, 256, 0, dg->st>>>(dA, n, dlo);
      ok = cuda_ok(dg, cudaGetLastError(), "density matrix") &&
           cuda_ok(dg, cudaMemcpyAsync(lo.data(), dlo, sizeof(double) * n, cudaMemcpyDeviceToHost, dg->st),
                   "Gershgorin bound") &&
           cuda_ok(dg, cudaStreamSynchronize(dg->st), "Gershgorin bound");
    }
    int sweeps = 0;
    if (ok) {
      // B = A + sigma I with every eigenvalue >= 1
      const double sigma = std::max(0.0, 1.0 - *std::min_element(lo.begin(), lo.end()));
      dg_jacobi_init_kernel<<<1024, 256, 0, dg->st>>>(dA, dW, n, sigma);
      int occ = 0, nsm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dg_jacobi_kernel, JC_THREADS, 0);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dg->cfg.device);
      const int n_pad = (int)(n + (n & 1));
      const int grid = std::max(1, std::min(n_pad / 2, std::max(1, occ) * std::max(1, nsm)));
      int nn = (int)n, maxs = MAX_SWEEPS;
      // stop at a pair cosine of sqrt(n) 1e-15 (the columns' rounding level)
      double tol = std::sqrt((double)n) * 1e-15;
      void* args[] = {&dW, &nn, (void*)&n_pad, &maxs, &tol, &doff, &dsweeps};
      ok = cuda_ok(dg, cudaLaunchCooperativeKernel((const void*)dg_jacobi_kernel, grid, JC_THREADS, args, 0, dg->st),
                   "Jacobi eigensolver");
      dg_colnorm_kernel<<<gw, 256, 0, dg->st>>>(dW, n, dnrm);
      ok = ok && cuda_ok(dg, cudaGetLastError(), "Jacobi eigensolver") &&
           cuda_ok(dg, cudaMemcpyAsync(lam.data(), dnrm, sizeof(double) * n, cudaMemcpyDeviceToHost, dg->st),
                   "eigenvalues") &&
           cuda_ok(dg, cudaMemcpyAsync(&sweeps, dsweeps, sizeof(int), cudaMemcpyDeviceToHost, dg->st), "sweeps") &&
           cuda_ok(dg, cudaStreamSynchronize(dg->st), "Jacobi eigensolver");
      if (ok) {
        for (double& v : lam) v -= sigma;
        std::vector<int> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lam[x] < lam[y]; });
        order.resize(n_occ);
        for (int i = 0; i < n_occ; ++i) eig[i] = lam[order[i]];
        ok = cuda_ok(dg, cudaMemcpyAsync(dord, order.data(), sizeof(int) * n_occ, cudaMemcpyHostToDevice, dg->st),
                     "order");
        if (ok) {
          dg_gather_kernel<<<1024, 256, 0, dg->st>>>(dW, dnrm, dord, dY, n, n_occ);
          dg_dm_kernel<<<dim3(gx, nel), 256, 0, dg->st>>>(dY, dP, J, n, n_occ);
          ok = cuda_ok(dg, cudaGetLastError(), "density matrix blocks") &&
               cuda_ok(dg, cudaStreamSynchronize(dg->st), "density matrix blocks");
        }
      }
    }
    dg->density_sweeps = sweeps;
    if (ok && std::getenv("DGDFT_TRACE")) {
      std::vector<unsigned long long> h(MAX_SWEEPS);
      cudaMemcpy(h.data(), doff, sizeof(unsigned long long) * MAX_SWEEPS, cudaMemcpyDeviceToHost);
      std::fprintf(stderr, "[dgdft] Jacobi, largest pair cosine per sweep:");
      for (int i = 0; i < sweeps; ++i) {
        double v;
        std::memcpy(&v, &h[i], sizeof(v));
        std::fprintf(stderr, " %.1e", v);
      }
      std::fprintf(stderr, "\n");
    }
    if (ok && sweeps >= MAX_SWEEPS) {
      release();
      return dg->fail(DGDFT_ENOTCONV, "density: the Jacobi sweeps did not converge");
    }
    t_ms[0] = tm.stop();
  }
  // density on each batch: phi from z again, then T = P_K phi and rho
  size_t cap = dg->cfg.hbm_cap_bytes;
  if (ok && !cap) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cap = fr / 4;
  }
  const int nbat = (int)std::max<size_t>(1, std::min<size_t>(nel, cap / std::max<size_t>(1, batch_bytes(dg))));
  if (ok && !ensure_batch(dg, nbat)) ok = false;
  double* d_mass = nullptr;
  int* d_bad = nullptr;
  double* d_linv = nullptr;
  if (ok && (!dmalloc(&d_mass, (size_t)nbat * JJ) || !dmalloc(&d_linv, (size_t)nbat * JJ) ||
             !dmalloc(&d_bad, (size_t)nbat))) {
    dg->err = "density scratch: out of memory";
    ok = false;
  }
  Timer tm(dg->st);
  for (int g0 = 0; ok && g0 < nel; g0 += nbat) {
    const int nb = std::min(nbat, nel - g0);
    std::vector<const double*> src(nb);
    for (int e = 0; e < nb && ok; ++e) {
      if (z_on_device) {
        src[e] = z[g0 + e];
      } else {
        double* dst = dg->d_z + (size_t)e * J * dg->ngq;
        ok = cuda_ok(dg, cudaMemcpyAsync(dst, z[g0 + e], sizeof(double) * J * dg->ngq, cudaMemcpyHostToDevice, dg->st),
                     "copy of z");
        src[e] = dst;
      }
    }
    ok = ok && interp_batch(dg, nb, src.data()) && ortho_batch(dg, nb, d_mass, (long long)JJ, d_linv, d_bad);
    if (!ok) break;
    std::vector<const double*> cin;
    std::vector<double*> cout;
    for (int e = 0; e < nb; ++e) cin.push_back(dg->d_phi + (size_t)e * J * dg->nL);
    for (int e = 0; e < nb; ++e) cout.push_back(dg->d_g[0] + (size_t)e * J * dg->nL);
    const double** d_in = nullptr;
    double** d_out = nullptr;
    if (!dmalloc(&d_in, cin.size()) || !dmalloc(&d_out, cout.size())) {
      cudaFree(d_in);
      dg->err = "pointer tables: out of memory";
      ok = false;
      break;
    }
    ok = cuda_ok(dg, cudaMemcpyAsync(d_in, cin.data(), cin.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                 "pointer tables") &&
         cuda_ok(dg, cudaMemcpyAsync(d_out, cout.data(), cout.size() * sizeof(void*), cudaMemcpyHostToDevice, dg->st),
                 "pointer tables") &&
         launch_axis(dg, d_in, d_out, nb, dP + (size_t)g0 * JJ, J, J, dg->nL, 1, (long long)JJ);
    if (ok) {
      double* out = (on_device ? rho : drho) + (size_t)g0 * dg->nL;
      dg_rho_kernel<<<dim3(256, nb), 256, 0, dg->st>>>(dg->d_phi, dg->d_g[0], out, J, dg->nL);
      ok = cuda_ok(dg, cudaGetLastError(), "density kernel") && cuda_ok(dg, cudaStreamSynchronize(dg->st), "density");
    }
    cudaFree(d_in);
    cudaFree(d_out);
  }
  t_ms[1] = tm.stop();
  cudaFree(d_mass);
  cudaFree(d_linv);
  cudaFree(d_bad);
  if (ok && !on_device)
    ok = cuda_ok(dg, cudaMemcpy(rho, drho, sizeof(double) * nel * dg->nL, cudaMemcpyDeviceToHost), "density copy");
  dg->density_ms[0] = t_ms[0];
  dg->density_ms[1] = t_ms[1];
  release();
  return ok ? DGDFT_OK : DGDFT_ECUDA;
}

dgdft_status dgdft_dg_density_info(dgdft_dg* dg, int* sweeps) {
  if (!dg || !sweeps) return DGDFT_EINVAL;
  *sweeps = dg->density_sweeps;
  return DGDFT_OK;
}

dgdft_status dgdft_dg_last_timing(dgdft_dg* dg, double* ms, int n, int* launches) {
  if (!dg || (n > 0 && !ms) || n > 8) return DGDFT_EINVAL;
  for (int i = 0; i < n; ++i) ms[i] = i < 6 ? dg->ms[i] : dg->density_ms[i - 6];
  if (launches) *launches = dg->launches;
  return DGDFT_OK;
}

const char* dgdft_dg_last_error(const dgdft_dg* dg) { return dg ? dg->err.c_str() : "null handle"; }

void dgdft_dg_destroy(dgdft_dg* dg) {
  if (!dg) return;
  if (dg->batch || dg->d_v) cudaStreamSynchronize(dg->st);
  for (int d = 0; d < 3; ++d) {
    cudaFree(dg->d_I[d]);
    cudaFree(dg->d_D[d]);
    cudaFree(dg->d_wf[d]);
    cudaFree(dg->d_g[d]);
  }
  for (void* p : {(void*)dg->d_w, (void*)dg->d_v, (void*)dg->d_pool, (void*)dg->d_traces, (void*)dg->d_linv,
                  (void*)dg->d_H, (void*)dg->d_bad, (void*)dg->d_z, (void*)dg->d_t1,
                  (void*)dg->d_t2, (void*)dg->d_phi, (void*)dg->d_part})
    cudaFree(p);
  delete dg;
}

}  // extern "C"
