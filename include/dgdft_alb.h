/*
 * dgdft_alb.h -- C-ABI of the GB300 adaptive-local-basis (ALB) generator.
 *
 * Operation (Hu, Lin, Yang, "DGDFT: A Massively Parallel Method for Large
 * Scale Density Functional Theory Calculations", Sec. II.A and Sec. II.B):
 * for every element E_K of a domain decomposition, solve the local Kohn-Sham
 * eigenproblem of Eq. localproblem on the extended element Q_K,
 *
 *     (-1/2 Lap + V_eff^{Q_K} + V_nl^{Q_K}) phi~_{K,j} = lambda_{K,j} phi~_{K,j},
 *
 * discretised by planewaves on a uniform periodic grid (grid rule Eq. Ngecut;
 * every G of the grid, or the sphere |G|^2/2 <= ecut, see
 * dgdft_alb_config.ecut), by LOBPCG (Sec. II.B, operations 1-5) for the lowest n_compute (m)
 * eigenpairs; restrict the lowest n_keep (J) eigenvectors to E_K,
 * orthonormalise them (so that the ALB overlap matrix is the identity,
 * Eq. orthonormal) and return them on E_K's grid points (zero elsewhere).
 *
 * Conventions shared by every entry point:
 *   - A grid function on Q_K is a real array of N_g = nx*ny*nz values, flat
 *     index i + nx*(j + ny*k) (x fastest), point (i*Lx/nx, j*Ly/ny, k*Lz/nz)
 *     relative to Q_K's corner.  Q_K is treated as a periodic box.
 *   - A block of k grid functions is column-major N_g x k (each vector
 *     contiguous).  All host-visible floating-point data is double.
 *   - The local problem uses the Euclidean inner product of grid vectors; the
 *     returned ALBs are scaled to the L2 normalisation sum phi_i phi_j dV =
 *     delta_ij with dV = Lx*Ly*Lz / N_g.
 *   - Ownership: the caller owns every buffer it passes; set_* calls copy
 *     the data in before returning, get_* calls copy out.  Pointers flagged
 *     on_device = 1 are CUDA device pointers valid on the context's device;
 *     they need to stay valid only until the call returns.
 *   - Errors: every call returns a dgdft_status; no exception, abort or
 *     device trap crosses the ABI.  dgdft_alb_last_error() describes the
 *     most recent failure on a context.  A context is not thread-safe.
 *   - The library needs a CUDA device of compute capability 10.3 (sm_103a).
 *     There is no CPU fallback: without a usable device create() fails with
 *     DGDFT_ECUDA.
 */
#ifndef DGDFT_ALB_H
#define DGDFT_ALB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgdft_alb_ctx dgdft_alb_ctx; /* opaque, owned by the library */

typedef enum {
  DGDFT_OK = 0,
  DGDFT_EINVAL = 1,   /* bad argument, size or non-finite input             */
  DGDFT_ENOMEM = 2,   /* device or host allocation failed                   */
  DGDFT_ECUDA = 3,    /* CUDA runtime error (message in last_error)         */
  DGDFT_ENOTCONV = 4, /* some element did not reach tol within maxit        */
  DGDFT_ETIMEOUT = 5, /* a bounded device-side wait ran out                 */
  DGDFT_ESTATE = 6    /* call out of order (e.g. get_basis before solve)    */
} dgdft_status;

/* Arithmetic of the LOBPCG operations (H apply, preconditioner, Gram
 * products, block updates, Rayleigh-Ritz).  The final restriction and
 * orthonormalisation are FP64 in every mode.                               */
enum {
  DGDFT_PREC_FP64 = 0,  /* plain: FP64 everywhere                             */
  DGDFT_PREC_MIXED = 1  /* chosen form: an FP32 stage (FP32 storage, FFTs
                           and block updates, Gram products on tensor cores
                           or compensated SIMT (see bulk_kernels), the
                           Rayleigh-Ritz in double-float, ~2^-46), then the
                           FP64 check and FP64-accurate iterations to the
                           tolerance (FP64 storage and residuals,
                           double-float FFT passes, Gram and update
                           products and Rayleigh-Ritz, ~2^-46 relative)    */
};

enum {
  DGDFT_PRECOND_TETER = 0,   /* Teter-Payne-Allan kinetic preconditioner      */
  DGDFT_PRECOND_LEARNED = 1  /* learned 3-D conv net, Teter as fallback        */
};

/* One extended element Q_K and its element E_K. */
typedef struct {
  int nx, ny, nz;        /* grid of Q_K: factors 2, 3, 5, nx even,
                            (nx/2+1)*ny <= 7000, nz <= 400                   */
  double Lx, Ly, Lz;     /* side lengths of Q_K in bohr                       */
  int e_lo[3], e_hi[3];  /* E_K as the half-open grid-index box [lo, hi)      */
  int n_compute;         /* m: eigenpairs computed by LOBPCG (>= n_keep)      */
  int n_keep;            /* J: ALBs kept                                      */
} dgdft_element_desc;

typedef struct {
  int precision;          /* DGDFT_PREC_*                                     */
  int precond;            /* DGDFT_PRECOND_*                                  */
  double tol;             /* residual tolerance (Ha): max_{j<J} |Hx-theta x|/|x| */
  int maxit;              /* LOBPCG iteration limit per element (> 0)         */
  int check_every;        /* iterations between host convergence polls (>= 1) */
  size_t hbm_cap_bytes;   /* device memory the solve may use; 0 = 90% of free */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = library stream    */
  int device;             /* CUDA device ordinal; -1 = current device         */
  int keep_block;         /* 1: keep each converged N_g x m Ritz block on the
                             host after solve (for dgdft_alb_get_block)        */
  int bulk_kernels;       /* Gram products and block updates of the FP32
                             stage.  0 (default): Gram products on tcgen05
                             tensor cores where every element of a wave has
                             m <= 48 and N_g % 4 == 0 (TMA copies of the
                             blocks, each FP32 value split into two TF32
                             parts, ~2^-22 relative per product, FP32
                             accumulation in tensor memory over 256 rows,
                             then compensated), else the SIMT kernel; block
                             updates in SIMT FP32.  1: SIMT FP32 kernels
                             only (compensated Gram accumulation).  2: as 0,
                             and the block updates on tensor cores too (the
                             same split, sums of up to 3m products in tensor
                             memory).  Other values give DGDFT_EINVAL.     */
  int h_fp64_forward;     /* FP64 forward FFT in the FP32 stage's H apply
                             (its rounding, amplified by |G|^2/2, sets the
                             stage's residual floor near 2e-6 Ha): 0 never;
                             1 every apply (~4x slower passes); 2 only H X'
                             once the median residual is below 1e-5        */
  const char* autotune_cache;   /* optional path of the autotuner's JSON cache
                                   (a flat object of "key": integer launch
                                   shapes per batch shape), read when a wave is
                                   built; missing keys are tuned then (timed on
                                   the wave's own blocks) and written back.
                                   Tuned today: the FP32 block update's
                                   128-row tiles per CTA (2, 4, 8 or 16), a
                                   launch shape that changes no result.  NULL
                                   = no tuning (defaults).  The string is
                                   copied at create.                         */
  const char* precond_weights;  /* learned preconditioner weights; NULL = none */
  int device_wait_polls;  /* bound on every device-side wait of the tensor-core
                             kernels, in polls: 0 (default) about a second;
                             a small value makes the waits run out, which is
                             how failure handling is tested: the element's
                             report (and the call) then return
                             DGDFT_ETIMEOUT.  Negative gives DGDFT_EINVAL. */
  int restrict_all;       /* restriction and orthonormalisation (Sec. II.A;
                             Eq. orthonormal).  0 (default, the paper's
                             procedure): the lowest J Ritz vectors are
                             restricted to E_K and all J left singular
                             vectors kept.  1: all m computed vectors are
                             restricted and the J left singular vectors of
                             the largest singular values kept.  Other
                             values give DGDFT_EINVAL.                      */
  double ecut;            /* planewave set of the local problem.  0 (default):
                             every G of the FFT grid.  > 0 (Ha): the sphere
                             |G|^2/2 <= ecut (the kinetic-energy cutoff
                             that Eq. Ngecut turns into the grid; with
                             Eq. Ngecut's value (pi n_d / L_d)^2 / 2 the
                             sphere inscribed in the grid's frequencies),
                             solved as the Galerkin problem on the span of
                             those planewaves: the starting block is
                             projected onto it, residuals are measured as
                             |P (H x - theta x)| with P that projection,
                             and the returned vectors lie in it.  Three
                             more FFT round trips per iteration (R, X', P'
                             projected).  In DGDFT_PREC_MIXED the FP32
                             stage decides the mask in FP32 (a frequency
                             within FP32 rounding of the sphere may be
                             decided differently there) and the FP64 check
                             and iterations project with the FP64 decision,
                             which fixes the result.  Needs the Teter
                             preconditioner and at least 3 n_compute
                             planewaves in the set of every element;
                             otherwise, or when negative or not finite,
                             DGDFT_EINVAL.                                 */
} dgdft_alb_config;

/* Per-element outcome of dgdft_alb_solve. */
typedef struct {
  int status;        /* DGDFT_OK, DGDFT_ENOTCONV, or DGDFT_ETIMEOUT when a
                        bounded device wait ran out for the element (its
                        FP32-stage products were then abandoned; the FP64
                        stage may still have converged it: see max_resid) */
  int iterations;    /* LOBPCG iterations taken (all precision stages)        */
  double max_resid;  /* max_{j<J} residual (Ha) at exit, FP64-checked         */
  int fallbacks;     /* Rayleigh-Ritz retries without P / preconditioner falls */
  int wave;          /* memory-admission wave the element ran in              */
  double seconds;    /* wall time of the element's wave                       */
  int iterations_bulk; /* of `iterations`, those run in the FP32 stage (mixed) */
  double resid_bulk;   /* max_{j<J} residual (Ha) when the FP32 stage ended   */
  long long graph_kernels; /* kernels launched through the per-iteration CUDA
                              graphs of this element's wave (both stages);
                              set-up, verify and orthonormalisation kernels
                              outside the graphs are not counted           */
  int restarts;      /* FP32-stage restarts: every Rayleigh-Ritz level failed,
                        so X was perturbed and P dropped (also counted in
                        `fallbacks`)                                        */
} dgdft_solve_report;

/* Fill cfg with defaults: FP64, Teter, tol 1e-6, maxit 400, check_every 4. */
void dgdft_alb_config_init(dgdft_alb_config* cfg);

/* Create a context for n_elem elements.  Validates every descriptor
 * (sizes, 0 < n_keep <= n_compute, E_K inside Q_K, grid factors) and selects
 * the device.  Nothing is allocated on the device until set_potential.
 * Returns DGDFT_EINVAL on a bad descriptor, DGDFT_ECUDA without a device. */
dgdft_status dgdft_alb_create(const dgdft_alb_config* cfg, int n_elem,
                              const dgdft_element_desc* elems,
                              dgdft_alb_ctx** out);

/* Restricted effective potential V_eff^{Q_K} of element `elem` (Sec. II.A):
 * N_g doubles in the grid convention above.  Non-finite values give
 * DGDFT_EINVAL. */
dgdft_status dgdft_alb_set_potential(dgdft_alb_ctx* ctx, int elem,
                                     const double* veff, int on_device);

/* Kleinman-Bylander projectors of the atoms whose centres lie in Q_K
 * (Eq. DGvar, nonlocal term): projector p has nonzeros
 * grid_idx[row_ptr[p] .. row_ptr[p+1]) with values val (= b_p * sqrt(dV), so
 * that sum val^2 = 1) and weight gamma[p] (Ha).  The discrete operator is
 * V_nl = sum_p gamma_p v_p v_p^T.  Host pointers; n_proj may be 0.  Indices
 * outside [0, N_g) or non-finite values give DGDFT_EINVAL. */
dgdft_status dgdft_alb_set_projectors(dgdft_alb_ctx* ctx, int elem, int n_proj,
                                      const int64_t* row_ptr, const int32_t* grid_idx,
                                      const double* val, const double* gamma);

/* Optional initial block X0 (N_g x m, column-major) for element `elem`; the
 * default is a seeded standard-normal block.  Also the warm start for a
 * repeated solve (Sec. II.B: previous Psi_K as the starting guess). */
dgdft_status dgdft_alb_set_initial(dgdft_alb_ctx* ctx, int elem, const double* x0,
                                   int on_device);

/* Run ALB generation for every element with a potential.  Writes n_elem
 * reports when per_elem is non-NULL.  Returns DGDFT_ENOTCONV when some
 * element missed tol (its basis is still available), DGDFT_ETIMEOUT when a
 * bounded device wait ran out for some element (this takes precedence),
 * DGDFT_ESTATE when an element has no potential. */
dgdft_status dgdft_alb_solve(dgdft_alb_ctx* ctx, dgdft_solve_report* per_elem);

/* One SCF step of ALB generation (Sec. II.B: in each SCF iteration the ALBs
 * are refined by a few LOBPCG iterations that start from those of the
 * previous SCF step, under the updated V_eff set by dgdft_alb_set_potential).
 * Every element runs exactly n_iter (>= 0) LOBPCG iterations, in the
 * context's precision (FP32 storage and arithmetic with an FP64
 * Rayleigh-Ritz in the mixed form), from the block given by
 * dgdft_alb_set_initial since the last solve or step, else from its own
 * Ritz block of the previous solve or step; then the FP64 residual check,
 * restriction to E_K and orthonormalisation as in dgdft_alb_solve.  There is
 * no tolerance: a report's status is DGDFT_OK unless the element failed, and
 * max_resid is the FP64 residual after the step.  The workload must fit one
 * memory-admission wave (it stays resident between steps; changing the
 * projectors drops the resident blocks).  n_iter = 0 runs no iteration: the
 * starting block is rotated to its Ritz vectors under the current potential
 * (FP64 Rayleigh-Ritz) and their FP64 residuals are reported, which tells a
 * caller how far the previous ALBs are from the new problem.  Returns
 * DGDFT_ESTATE when an element has no block to start from, DGDFT_EINVAL for
 * n_iter < 0. */
dgdft_status dgdft_alb_scf_step(dgdft_alb_ctx* ctx, int n_iter, dgdft_solve_report* per_elem);

/* Copy out element `elem`'s ALBs: phi is n_E x J column-major (n_E = product
 * of e_hi - e_lo, points ordered x fastest within E_K), eig the J lowest
 * eigenvalues (Ha), resid their residuals (Ha).  Any pointer may be NULL.
 * DGDFT_ESTATE before a solve. */
dgdft_status dgdft_alb_get_basis(dgdft_alb_ctx* ctx, int elem, double* phi,
                                 double* eig, double* resid, int on_device);

/* Human-readable description of the last failure on ctx ("" if none). */
const char* dgdft_alb_last_error(const dgdft_alb_ctx* ctx);

/* Release every device and host resource of ctx.  NULL is a no-op. */
void dgdft_alb_destroy(dgdft_alb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGDFT_ALB_H */
