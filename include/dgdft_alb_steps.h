/*
 * dgdft_alb_steps.h -- step-level entry points of the ALB generator.
 *
 * Each call runs one stage of the hot path on the GPU, in the context's
 * precision, on data the caller supplies, so every kernel can be compared
 * with an independent implementation.  Grid, block and ownership
 * conventions are those of dgdft_alb.h.  Inputs and outputs are double on
 * both sides of the ABI; in DGDFT_PREC_MIXED contexts they are rounded to the
 * working precision on entry.  The element's potential (and projectors,
 * where used) must have been set.  Calls are synchronous.
 */
#ifndef DGDFT_ALB_STEPS_H
#define DGDFT_ALB_STEPS_H

#include "dgdft_alb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* H applied to k vectors (Sec. II.B, operation 1; Eq. localproblem):
 * hx = -1/2 Lap x + V_eff x + sum_p gamma_p v_p (v_p^T x).  The Laplacian is
 * spectral over every G of the FFT grid, Nyquist plane included.  stage
 * picks the solver stage whose kernels run: 0 the bulk stage (FP32 in
 * DGDFT_PREC_MIXED), 1 the FP64 stage (in DGDFT_PREC_MIXED FP64 vectors with
 * the transforms in double-float arithmetic, ~2^-46 per operation; plain
 * FP64 in DGDFT_PREC_FP64, where both stages are the same).
 * x, hx: N_g x k column-major.  1 <= k <= n_compute. */
dgdft_status dgdft_alb_apply_h(dgdft_alb_ctx* ctx, int elem, int stage, int k, const double* x, double* hx,
                               int on_device);

/* Teter-Payne-Allan preconditioner (Sec. II.B, operation 5), per column:
 * w_i = F^-1 [ K((|G|^2/2) / t_kin[i]) F r_i ] with
 * K(s) = (27+18s+12s^2+8s^3) / (27+18s+12s^2+8s^3+16s^4).
 * r, w: N_g x k; t_kin: k positive kinetic-energy scales (Ha, host). */
dgdft_status dgdft_alb_apply_teter(dgdft_alb_ctx* ctx, int elem, int k, const double* r,
                                   const double* t_kin, double* w, int on_device);

/* Gram product C = U^T V (Sec. II.B, operation 2) over ng rows:
 * U is ng x p, V is ng x q (column-major), C is p x q column-major (host,
 * FP64).  Computed by the solver's split-K SIMT kernels in the context's
 * precision (FP32 with compensated accumulation in DGDFT_PREC_MIXED,
 * FP64 otherwise); the solver's tensor-core Gram is exercised through
 * dgdft_alb_lobpcg_gram. */
dgdft_status dgdft_alb_gram(dgdft_alb_ctx* ctx, int ng, int p, int q, const double* u,
                            const double* v, double* c, int on_device);

/* The Gram products of one LOBPCG iteration (Sec. II.B, operation 2: the 12
 * products Phi^T Psi), computed on caller blocks by the same kernels and
 * with the same precision choices as the solver for element `elem`, in the
 * stage `stage` selects: 0 the bulk stage (in DGDFT_PREC_MIXED the FP32
 * stage: tensor cores unless bulk_kernels = 1), 1 the FP64 stage (in
 * DGDFT_PREC_MIXED double-float products, FP32 pairs with exact products
 * and two-sum accumulation, ~2^-44 relative; plain FP64 in
 * DGDFT_PREC_FP64, where both stages are the same).  blocks holds
 * six N_g x m column-major blocks one after another: X, W, P, H X, H W, H P
 * (m = n_compute; P and H P are ignored when has_p = 0).  With S = [X W P]:
 * a = (H S)^T S and b = S^T S, each 3m x 3m column-major, are returned in
 * their upper block triangle (the diagonal blocks included), which is all
 * the Rayleigh-Ritz step reads; the rest is zero, and so is every P row and
 * column when has_p = 0.  In the upper triangle the H-image is on the
 * earlier block: a(i, j) = (H s_i)^T s_j for block(i) <= block(j).  xtw =
 * X^T W (m x m).  a, b, xtw are host arrays; blocks is on the device when
 * on_device = 1.  DGDFT_ETIMEOUT when a bounded device wait ran out. */
dgdft_status dgdft_alb_lobpcg_gram(dgdft_alb_ctx* ctx, int elem, int stage, int has_p, const double* blocks,
                                   double* a, double* b, double* xtw, int on_device);

/* The block updates of one LOBPCG iteration (Sec. II.B, operation 4: the
 * paper's Phi C products), computed on caller blocks by the same kernels
 * and precision choices as the solver for element `elem` in stage `stage`
 * (0: the bulk stage, in DGDFT_PREC_MIXED the FP32 stage, tensor cores when
 * bulk_kernels = 2; 1: the FP64 stage, double-float in DGDFT_PREC_MIXED).
 * blocks holds six N_g x m column-major blocks: X, W, P, H X, H W, H P (P
 * and H P ignored when has_p = 0); y is the 3m x m column-major coefficient
 * block [Y_x; Y_w; Y_p] of a Rayleigh-Ritz step.  out receives three N_g x m
 * blocks: X' = [X W P] Y, P' = [W P] [Y_w; Y_p] and (H P)' = [H W H P]
 * [Y_w; Y_p] (the P terms dropped when has_p = 0).  blocks and out are on
 * the device when on_device = 1, else host arrays; y is a host array.
 * DGDFT_ETIMEOUT when a bounded device wait ran out. */
dgdft_status dgdft_alb_lobpcg_update(dgdft_alb_ctx* ctx, int elem, int stage, int has_p, const double* blocks,
                                     const double* y, double* out, int on_device);

/* Rayleigh-Ritz on a symmetric pencil (Sec. II.B, operation 4) on the GPU:
 * the lowest m eigenpairs of A y = theta B y with B positive definite.
 * stage picks the arithmetic of a solve's two stages: 0 = the FP32 LOBPCG
 * stage's reduction, double-float (FP32 pairs, ~2^-46 relative) in a
 * DGDFT_PREC_MIXED context when n <= 160 and m <= 64, FP64 otherwise;
 * 1 = FP64 (the FP64 continuation, and every stage of an FP64 context).
 * A, B: n x n column-major (host, both symmetric); theta: m ascending;
 * y: n x m with y^T B y = I.  Returns DGDFT_EINVAL when B is not positive
 * definite to working accuracy or stage is not 0 or 1.
 * n <= 3 * max n_compute of the context. */
dgdft_status dgdft_alb_rayleigh_ritz(dgdft_alb_ctx* ctx, int stage, int n, int m, const double* a,
                                     const double* b, double* theta, double* y);

/* Restriction to E_K and orthonormalisation (Sec. II.A; Sec. II.B): the
 * first J columns of the N_g x k block x are restricted to E_K's points and
 * replaced by the left singular vectors of that n_E x J block, scaled by
 * 1/sqrt(dV); with the context's restrict_all = 1, all k columns are
 * restricted and the J left singular vectors of the largest singular values
 * kept.  phi: n_E x J column-major.  J <= k. */
dgdft_status dgdft_alb_restrict_orthonormalise(dgdft_alb_ctx* ctx, int elem, int k,
                                               int J, const double* x, double* phi,
                                               int on_device);

/* The converged Ritz block of element `elem` after a solve or SCF step: x is
 * N_g x m (the m = n_compute Ritz vectors, Euclidean-orthonormal, ascending
 * Ritz values), host or device per on_device.  Read from the host copy that
 * keep_block = 1 keeps, else from the resident wave of a workload that fits
 * one memory-admission wave (valid until the next solve or step).
 * DGDFT_ESTATE before a solve, or when neither holds the block. */
dgdft_status dgdft_alb_get_block(dgdft_alb_ctx* ctx, int elem, double* x, int on_device);

/* Projection onto the sphere-cutoff planewave set of the context
 * (dgdft_alb_config.ecut > 0): px_i = F^-1 [ mask F x_i ], mask(G) = 1
 * where |G|^2/2 <= ecut, else 0 (the orthogonal projector P of the solve's
 * Galerkin problem), with the FP64 stage's passes (FP64; double-float,
 * ~2^-44 relative, in DGDFT_PREC_MIXED).  x, px: N_g x k column-major, 1 <= k <=
 * n_compute.  DGDFT_EINVAL when the context has ecut = 0, DGDFT_ESTATE
 * before the element's potential is set. */
dgdft_status dgdft_alb_project_cutoff(dgdft_alb_ctx* ctx, int elem, int k, const double* x, double* px,
                                      int on_device);

/* Gram product C = U^T V in FP64 that allocates nothing.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory while
 * they run (code inside a custom memory pool that must not fragment, or
 * allocator-free real-time loops whose latency must not include an
 * allocation).  It needs no context.  u is ng x p, v is ng x q, c is p x q, all column-major
 * FP64 *device* pointers on the current device, owned by the caller; the
 * work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without waiting for it.
 * Limits: 1 <= p, q <= 256 and ng >= 1; anything else returns DGDFT_EINVAL
 * before any GPU work.  The split-K partial sums live in one fixed 8 MiB
 * device array inside the library, held by every GPU that loads it until
 * the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress).  That address is cached per device
 * for the life of the process: do not use this entry point across a device
 * reset (cudaDeviceReset, or a reset of the primary context), after which
 * the cached address is stale.  Every call reuses the same array:
 * calls that can overlap on the GPU (different streams, or the same
 * stream from different host threads without ordering) race and corrupt
 * each other's results; serialise them.  Returns DGDFT_ECUDA if the launch
 * fails.  No cudaMalloc, cudaFree or allocating library call is made. */
dgdft_status dgdft_alb_gram_noalloc(int ng, int p, int q, const double* u, const double* v, double* c,
                                    void* stream);

/* ---- Learned preconditioner (the chosen form's replacement of the Teter
 * preconditioner of Sec. II.B, operation 5).  A 3-D convolutional network:
 * inputs (r / rms(r), V_eff), 4 layers of 3x3x3 circular convolutions,
 * 2 -> 16 -> 16 -> 16 -> 1 channels, ReLU between layers; correction =
 * rms(r) * output.  Weights are stored in BF16 (FP32 master copy for
 * training), arithmetic accumulates in FP32.  Parameter vector layout: per
 * layer, weights [c_out][c_in][3][3][3] (taps dz, dy, dx = offsets -1..1)
 * then c_out biases; DGDFT_PRECOND_PARAMS floats in total.  Fields are
 * [sample][channel][z][y][x] float32. */
#define DGDFT_PRECOND_PARAMS 15169

/* He-normal initial weights from `seed`, zero biases. */
dgdft_status dgdft_alb_precond_init(dgdft_alb_ctx* ctx, uint64_t seed);
dgdft_status dgdft_alb_precond_set_params(dgdft_alb_ctx* ctx, const float* params);
dgdft_status dgdft_alb_precond_get_params(dgdft_alb_ctx* ctx, float* params);
/* Weights file: "DGALBNN1", int32 layer count, per layer int32 c_in, c_out,
 * then the float32 parameter vector.  The same file can be named in
 * dgdft_alb_config.precond_weights. */
dgdft_status dgdft_alb_precond_save(dgdft_alb_ctx* ctx, const char* path);
dgdft_status dgdft_alb_precond_load(dgdft_alb_ctx* ctx, const char* path);

/* Network output for B samples of nz x ny x nx: in is B x 2 fields, out is
 * B x 1 fields (float32, host or device per on_device). */
dgdft_status dgdft_alb_precond_forward(dgdft_alb_ctx* ctx, int B, int nz, int ny, int nx, const float* in,
                                       float* out, int on_device);

/* Mean squared error of the output against tgt over the window [lo, hi) of
 * every axis (mean over B samples and window points) and its gradient with
 * respect to every parameter (host array, parameter layout). */
dgdft_status dgdft_alb_precond_loss_grad(dgdft_alb_ctx* ctx, int B, int nz, int ny, int nx, int lo, int hi,
                                         const float* in, const float* tgt, double* loss, float* grads,
                                         int on_device);

/* Train with Adam (lr, betas 0.9/0.999) on `steps` batches of `batch` random
 * crops of edge `crop` (periodic wrap) from nfields fields r, v, t (device
 * arrays, nfields x nz x ny x nx each): input (r / rms(r), v), target
 * t / rms(r), loss on the crop interior [4, crop - 4).  Reports the mean loss
 * of the first and last min(10, steps) batches. */
dgdft_status dgdft_alb_precond_train(dgdft_alb_ctx* ctx, int nfields, int nz, int ny, int nx, const float* r,
                                     const float* v, const float* t, int crop, int batch, int steps, double lr,
                                     uint64_t seed, double* loss_first, double* loss_last);

/* Training pairs from the plain solver: for each snapshot q the FP64 LOBPCG
 * of element `elem` is run from its initial block for snap_iters[q]
 * iterations; its residual block R (m fields) goes to r_out, and
 * t = (H - sigma I)^-1 R, sigma = (lowest Ritz value) - 1 Ha, solved by FP64
 * conjugate gradients to relative residual 1e-10, goes to t_out (device
 * float32, nsnap x m x N_g each).  sigma and CG iteration counts per snapshot
 * are returned when the pointers are non-NULL. */
dgdft_status dgdft_alb_precond_make_data(dgdft_alb_ctx* ctx, int elem, int nsnap, const int* snap_iters,
                                         float* r_out, float* t_out, double* sigma, int* cg_iters);

/* Kernel stages that dgdft_alb_time_stage can time in isolation. */
enum {
  DGDFT_STAGE_XY_FWD = 0,   /* FFT pass 1: r2c along x, FFT along y (H apply)  */
  DGDFT_STAGE_Z_MULT = 1,   /* FFT pass 2: FFT along z, kinetic symbol, inverse */
  DGDFT_STAGE_XY_INV = 2,   /* FFT pass 3: inverse y, c2r x, + V psi + KB       */
  DGDFT_STAGE_GRAM = 3,     /* the 12 Gram blocks of S^T H S, S^T S + reduction */
  DGDFT_STAGE_UPDATE = 4,   /* one block update X <- [X W P] Y                  */
  DGDFT_STAGE_RR = 5,       /* FP64 Rayleigh-Ritz of every element              */
  DGDFT_STAGE_RESIDUAL = 6, /* R = HX - X Theta with partial sums               */
  DGDFT_STAGE_COUNT = 7
};

/* Average device time (ms) of one launch of `stage` over all elements kept
 * resident by the last dgdft_alb_solve (the bulk-precision wave: FP32 for
 * DGDFT_PREC_MIXED), measured with CUDA events on the context stream over
 * `reps` back-to-back launches after one untimed launch.  The stage runs on
 * the solve's final data with every element marked active; the solve's
 * results (basis, eigenvalues, residuals) are not affected.  Also reports
 * the number of elements and the working-precision size in bytes.
 * DGDFT_ESTATE when no wave is resident (memory-limited multi-wave solves
 * do not keep one). */
dgdft_status dgdft_alb_time_stage(dgdft_alb_ctx* ctx, int stage, int reps, double* ms_per_launch,
                                  int* n_elem, int* real_bytes);

#ifdef __cplusplus
}
#endif
#endif /* DGDFT_ALB_STEPS_H */
