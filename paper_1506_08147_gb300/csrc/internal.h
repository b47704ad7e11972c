// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace dgdft {

// A block operand: either one of the element's blocks (current or next
// buffer) or, for single-element step calls, an explicit device pointer.
template <class real> struct BRef {
  int sel;
  int next;
  real* ptr;
};
template <class real> inline BRef<real> bref(int sel, int next = 0) { return BRef<real>{sel, next, nullptr}; }
template <class real> inline BRef<real> bptr(real* p) { return BRef<real>{0, 0, p}; }

template <class real>
__device__ __forceinline__ real* resolve(const ElemDev<real>& e, const BRef<real>& r) {
  if (r.ptr) return r.ptr;
  return r.next ? next_blk(e, r.sel) : cur_blk(e, r.sel);
}

// Launch geometry of a batch of elements resident on the device.
struct BatchShape {
  int nel = 0;        // elements in the batch
  int max_nz = 0, max_ny = 0, max_nxh = 0, max_nplane = 0, max_m = 0, max_ng = 0;
  int max_nproj = 0, max_rows_e = 0;
  // grid shared by every element (0 when the batch mixes grids): selects
  // FFT kernels specialised for the line lengths at compile time
  int uni_nx = 0, uni_ny = 0, uni_nz = 0;
  bool ng_mult4 = true;  // every element's N_g is a multiple of 4 (16-byte columns)
  // FP64 wave of the mixed form: Gram products in double-float arithmetic
  // (FP32 pairs) instead of on the FP64 pipe
  bool dfloat = false;
  // 128-row tiles per CTA of the FP32 block update (tsmm_rows_kernel); a
  // launch shape only (each output's arithmetic is the same), tuned per
  // batch shape when the context has an autotune cache
  int tsmm_tiles = 8;
};

template <class real> struct Batch {
  const ElemDev<real>* d_elems = nullptr;  // device array of nel descriptors
  BatchShape s;
};

enum { ZM_KINETIC = 0, ZM_TETER = 1, ZM_MASK = 2 };
enum { XI_HAMILTONIAN = 0, XI_PLAIN = 1 };

// hamiltonian.cu
// Orthogonal projection onto the span of the planewaves with |G|^2/2 <=
// ecut (each element's own ecut): dst = F^-1 mask F src.
void launch_project(const Batch<double>& b, BRef<double> src, BRef<double> dst, int ncols, cudaStream_t st);
void launch_project(const Batch<float>& b, BRef<float> src, BRef<float> dst, int ncols, cudaStream_t st);
template <class real>
void launch_apply_h(const Batch<real>& b, BRef<real> src, BRef<real> dst, int ncols, cudaStream_t st,
                    bool fwd64 = false);
template <class real>
void launch_teter(const Batch<real>& b, BRef<real> src, BRef<real> dst, const double* tkin_override,
                  int ncols, cudaStream_t st, int only_teter_elems = 0);

void init_hamiltonian_kernels();

// fft_mono.cu: the three H / Teter passes for FP32 batches on one monolayer
// grid (48 x 64 x 40 or 48 x 64 x 48, mono_grid); all three run together
// (their half spectrum is ordered [z][kx][y])
bool mono_grid(const BatchShape& s);
void mono_xy_fwd(const Batch<float>& b, BRef<float> src, int ncols, int filt, cudaStream_t st);
void mono_z(const Batch<float>& b, int mode, int ncols, const double* tkin_override, int filt, cudaStream_t st);
void mono_xy_inv(const Batch<float>& b, int mode, BRef<float> dst, BRef<float> xsrc, int ncols, int filt,
                 cudaStream_t st);
void init_mono_kernels();
void opt_in_dynamic_smem(const void* kernel);
template <class real>
void launch_proj_coef(const Batch<real>& b, BRef<real> src, int ncols, cudaStream_t st);
template <class real>
void launch_h_pass(const Batch<real>& b, int pass, BRef<real> src, BRef<real> dst, int ncols, cudaStream_t st);

// blas.cu
// Gram products U_a^T V_b over the rows of each element, split over row
// chunks; FP64 partial sums are reduced in a fixed order.
enum { OUT_GRAM_A = 0, OUT_GRAM_B = 1, OUT_GXW = 2, OUT_PTR = 3 };
constexpr int MAX_PAIRS = 12;
template <class real> struct GramJob {
  int npairs = 0;
  BRef<real> a[MAX_PAIRS], b[MAX_PAIRS];
  int needs_p[MAX_PAIRS];   // 1: skip the pair while the element has no P block
  int out_id[MAX_PAIRS];
  int brow[MAX_PAIRS], bcol[MAX_PAIRS];  // placement, in units of the column count
  int ncols_a = 0, ncols_b = 0;          // <= 0: the element's m
  int rows = 0;                          // <= 0: the element's N_g
  int ld_in = 0;                         // leading dim of explicit pointers (<=0: rows)
  int ld_out = 0;                        // <= 0: 3m for gram A/B, m for X^T W
  double* out_ptr = nullptr;             // OUT_PTR target (single element)
};
template <class real>
void launch_gram(const Batch<real>& b, const GramJob<real>& job, double* partial, size_t partial_cap,
                 cudaStream_t st);

// Tall-skinny update out = alpha * sum_i in_i Y_i + beta * out, Y in FP64.
enum { Y_RR = 0, Y_GXW = 1, Y_PTR = 2 };
template <class real> struct TsmmJob {
  int nin = 0;
  BRef<real> in[3];
  int needs_p[3] = {0, 0, 0};
  int yrow[3] = {0, 0, 0};   // first Y row of input i, in units of the column count
  int y_id = Y_RR;
  const double* y_ptr = nullptr;
  int ldy = 0;               // <= 0: 3m for Y_RR, m for Y_GXW
  int ycol = 0;              // first Y column, in units of the column count
  int ncols = 0;             // columns per input and output (<= 0: m)
  int rows = 0;              // <= 0: N_g
  int ld_in = 0;             // explicit pointer leading dim (<= 0: rows)
  BRef<real> out;
  double alpha = 1.0, beta = 0.0;
  // optional second output: out2 = sum over inputs i >= from2 of in_i Y_i
  // (alpha 1, beta 0), written on the way to out; from2 < 0: none
  int from2 = -1;
  BRef<real> out2;
};
template <class real>
void launch_tsmm(const Batch<real>& b, const TsmmJob<real>& job, cudaStream_t st);
void init_blas_kernels();

// Residual R = HX - X diag(theta) into W, with per-column partial sums.
template <class real>
void launch_residual(const Batch<real>& b, int nchunk, cudaStream_t st);
// Reduces the partial sums: residual norms, kinetic energies for Teter,
// convergence and iteration bookkeeping.
template <class real>
void launch_post_residual(const Batch<real>& b, int nchunk, int maxit, cudaStream_t st);
// r.r partial sums of the W block in the residual kernel's chunks,
// replacing that kernel's first sum: after W = P R was projected.
void launch_rnorm(const Batch<double>& b, int nchunk, cudaStream_t st);
void launch_rnorm(const Batch<float>& b, int nchunk, cudaStream_t st);
// End of an iteration: flip the X/P/HX/HP buffers, mark P valid.
template <class real>
void launch_restart(const Batch<real>& b, cudaStream_t st);
template <class real>
void launch_iter_finish(const Batch<real>& b, int set_p, cudaStream_t st);
// FP32 stage: HX -= d X, HP -= d P for elements whose shift moved by d this
// iteration (post_residual decides d).
template <class real>
void launch_shift(const Batch<real>& b, cudaStream_t st);
// theta = 0 (mode 0) or the Rayleigh quotients from the residual sums (mode 1)
template <class real>
void launch_theta(const Batch<real>& b, int nchunk, int mode, cudaStream_t st);

// dense.cu: FP64 Rayleigh-Ritz on one CTA per task.
enum { RR_FIXED = 0, RR_INITIAL = 1, RR_LOBPCG = 2 };
struct RRTask {
  const double* A;   // n x n (ld), symmetric up to rounding
  const double* B;   // n x n (ld), symmetric positive definite
  int ld;
  int mode;          // RR_FIXED: n = n_fixed; RR_INITIAL: n = m; RR_LOBPCG: 2m or 3m
  int n_fixed;
  int m;             // eigenpairs wanted (lowest)
  double* Y;         // n x m output (ldy); LOBPCG rows of a dropped P are zeroed
  float* Yf;         // optional FP32 copy of Y (same layout), or nullptr
  int ldy;
  double* theta;     // m
  double* work;      // rr_work_doubles(n_max, m) doubles
  int* state;        // element state words, or nullptr
  double cond_max;   // Cholesky condition limit on the equilibrated B
  // > 0 (LOBPCG tasks of the FP32 stage): when no pencil passes, not even X
  // alone (condition limit 1e6 there), Y = [I; 0] keeps X and the element is
  // marked for a restart (ST_RESTART) instead of failing, at most this many
  // times; 0: such an element fails with ERR_CHOL
  int restart_max;
};
size_t rr_work_doubles(int n_max, int m);
// n_max, m_max bound the tasks' pencil sizes; pencils that fit use the
// shared-memory kernel.  n_max <= 0 forces the global-memory kernel.
// dfloat: the FP32 stage's reduction in double-float arithmetic (rr_df.cu)
// where the pencil fits that kernel, FP64 otherwise.
void launch_rr(const RRTask* d_tasks, int ntask, cudaStream_t st, int n_max, int m_max, bool dfloat = false);
void init_rr_kernels();
bool rr_df_eligible(int n_max, int m_max);
void launch_rr_df(const RRTask* d_tasks, int ntask, cudaStream_t st, int n_max, int m_max);
void init_rr_df_kernel();

// solver-level helpers are in solver.cu

std::string cuda_err_string(cudaError_t e);

}  // namespace dgdft

namespace dgdft {
// tf32_gram.cu: tcgen05 TF32-split Gram products of the FP32 stage, operands
// loaded by TMA (m <= 48, N_g % 4 == 0)
bool tf32_gram_eligible(const BatchShape& s);
// encodes the 10 block tensor maps of each element (128 bytes each) into
// host_out; returns "" or the reason it could not
std::string encode_tf32_gram_maps(const ElemDev<float>* h, int nel, void* host_out);
void init_tf32_gram_kernel();
// Tensor-core block updates of the FP32 stage (tf32_update.cu): the same
// jobs as launch_tsmm for blocks of the batch's elements (m <= 48, N_g a
// multiple of 4, default rows/columns/leading dimensions); false when the
// job or batch is not eligible and the SIMT kernel must run.
bool tf32_update_eligible(const BatchShape& s);
std::string encode_tf32_update_maps(const ElemDev<float>* h, int nel, void* host_out);
void init_tf32_update_kernel();
bool launch_tf32_update(const Batch<float>& b, const TsmmJob<float>& job, const void* d_maps, uint32_t polls,
                        cudaStream_t st);
// mode 0: the 12 LOBPCG Gram blocks into gram (A, B); mode 1: X^T W into gxw.
// polls: bound of every device wait (0: the default, about a second).
// Returns false (nothing launched) when the partial buffer is too small.
bool launch_tf32_gram(const Batch<float>& b, const void* d_maps, int mode, double* partial, size_t partial_cap,
                      uint32_t polls, cudaStream_t st);

// alb.cu
// One product of the FP64 orthonormalisation for one element: the Gram
// out = A^T A (J x J) or the update out = A Y (rows x J); column-major.
struct OrthoTask {
  const double* a;  // rows x K (K = J for a Gram task: the J x J Gram of a)
  const double* y;  // K x J (update only)
  double* out;
  int rows, J;
  int K;            // columns of a in an update task (0: J)
};
constexpr int ORTHO_CHUNK = 1024;  // rows per CTA of the Gram
size_t ortho_partial_doubles(int ntask, int max_rows, int max_J);
void launch_ortho_gram(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, double* partial,
                       cudaStream_t st);
// the K x 32 Y columns of a CTA are staged in shared memory (K <= 900)
void launch_ortho_apply(const OrthoTask* d_tasks, int ntask, int max_rows, int max_J, int max_K, cudaStream_t st);
template <class real>
void launch_restrict(const real* x, int ng, int nx, int ny, const int* lo, const int* hi, int J, double* out,
                     cudaStream_t st);
template <class A, class B>
void launch_convert(const A* in, B* out, size_t n, cudaStream_t st);
void launch_scale(double* x, size_t n, double s, cudaStream_t st);
// flag |= 1 when any of x[0..n) is not finite
void launch_nonfinite(const double* x, size_t n, int* flag, cudaStream_t st);
}  // namespace dgdft
