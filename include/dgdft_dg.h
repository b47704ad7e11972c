/* DG Hamiltonian assembly from the adaptive local basis functions.
 *
 * Eq. DGHamiltonian defines H^DG_{K',j';K,j} in three groups:
 *   (1) 1/2 <grad phi_{K,j'}, grad phi_{K,j}> + <phi_{K,j'}, V_eff phi_{K,j}>
 *       over E_K (diagonal blocks);
 *   (2) sum_p gamma_p <phi_{K',j'}, b_p> <b_p, phi_{K,j}> (the blocks of every
 *       pair of elements a projector b_p touches);
 *   (3) -1/2 <[phi'], {grad phi}> - 1/2 <{grad phi'}, [phi]> + alpha <[phi'], [phi]>
 *       over the faces shared by neighbouring elements.
 * Sec. II.B ("Construction of the DG Hamiltonian") evaluates every integral by
 * Legendre-Gauss-Lobatto (LGL) quadrature on each element and the gradients by
 * LGL differentiation matrices; Sec. III uses twice as many LGL points per
 * direction as the uniform grid has.  The K-th block row is assembled from E_K
 * and its neighbours, as in the paper's per-element ownership.
 *
 * Readings (the paper is silent on them):
 *   - the ALB functions of E_K are the real trigonometric interpolants over the
 *     periodic box Q_K of J columns given on Q_K's uniform grid (after an ALB
 *     solve: the lowest J Ritz vectors), restricted to E_K;
 *   - Eq. orthonormal is imposed under the LGL quadrature by the Cholesky factor
 *     of the mass matrix, M = L L^T, phi = phi~ L^-T (unique given the
 *     columns), before any integral of H^DG is evaluated;
 *   - on the face between E_a and its +e_d neighbour E_b the jump is
 *     (u_a - u_b) e_d and the average of the normal derivative
 *     (d_d u_a + d_d u_b) / 2; with one element along d the face joins the
 *     element to itself across the periodic boundary.
 *
 * Arithmetic: FP64 by default, double-float pairs as an option (arith).
 * All compute runs on the GPU on the stream of the configuration; there is
 * no CPU path.
 */
#ifndef DGDFT_DG_H
#define DGDFT_DG_H

#include <stddef.h>
#include <stdint.h>

#include "dgdft_alb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgdft_dg dgdft_dg;

typedef struct {
  int ne[3];          /* elements per direction of the periodic cell;
                         element K = ix + ne[0] (iy + ne[1] iz)            */
  double cell[3];     /* periodic cell (bohr)                              */
  int q_span[3];      /* elements per direction spanned by Q_K: 3, or 1 when
                         ne = 1 (Q_K then spans the cell along that axis)   */
  int nq[3];          /* Q_K's uniform grid (x, y, z), each >= 2            */
  int nl[3];          /* LGL points per direction on E_K, 2..128           */
  int J;              /* basis functions per element, 1..128               */
  double alpha;       /* interior-penalty parameter of Eq. DGvar, >= 0      */
  int n_proj;         /* projectors of the system (ids 0..n_proj-1)         */
  void* cuda_stream;  /* cudaStream_t to run on; NULL = the legacy stream   */
  int device;         /* CUDA device ordinal                               */
  size_t hbm_cap_bytes; /* bound on the per-batch scratch (0 = a quarter of
                           the free device memory); elements are processed
                           in batches that fit it                          */
  int arith;            /* contractions (interpolation, orthonormalisation,
                           differentiation, Gram products): 0 = FP64;
                           1 = double-float pairs on the FP32 pipes
                           (~2^-48 relative per operation, ~3x faster).
                           With nearly dependent columns (mass-matrix
                           condition kappa) both forms lose about
                           kappa^(1/2) of their unit in the basis's weak
                           directions, double-float from its larger unit */
} dgdft_dg_config;

/* Validate the configuration, build the LGL, differentiation and
 * interpolation tables and allocate the per-element storage.
 * DGDFT_EINVAL on an invalid field, DGDFT_ECUDA without a usable sm_103
 * device, DGDFT_ENOMEM when the storage does not fit.  Whenever out and cfg
 * are non-NULL, *out receives a handle, on failure too (its
 * dgdft_dg_last_error says why); the caller frees it with dgdft_dg_destroy. */
dgdft_status dgdft_dg_create(const dgdft_dg_config* cfg, dgdft_dg** out);

/* The LGL nodes of element `elem` in cell coordinates (bohr): x[nl[0]],
 * y[nl[1]], z[nl[2]] (host arrays, ascending), so the caller can evaluate
 * V_eff and the projectors there.  DGDFT_EINVAL on a bad element.          */
dgdft_status dgdft_dg_lgl_points(dgdft_dg* dg, int elem, double* x, double* y, double* z);

/* V_eff of element `elem` at its LGL points: n = nl[0] nl[1] nl[2] values,
 * x fastest (host or device pointer per on_device; copied).                */
dgdft_status dgdft_dg_set_potential(dgdft_dg* dg, int elem, const double* v, int on_device);

/* Projection weights gamma[n_proj] (host, copied).                          */
dgdft_status dgdft_dg_set_gamma(dgdft_dg* dg, const double* gamma);

/* The projectors touching element `elem`, sampled at its LGL points (host
 * arrays, copied): n_p projectors with global ids pid[n_p] (distinct, in
 * [0, n_proj)), CSR row_ptr[n_p + 1] over idx (flat LGL index, x fastest)
 * and val (b_p at that point, no quadrature weight).  Replaces any earlier
 * set for the element.  DGDFT_EINVAL on an id or index out of range.        */
dgdft_status dgdft_dg_set_projectors(dgdft_dg* dg, int elem, int n_p, const int* pid,
                                     const int64_t* row_ptr, const int* idx, const double* val);

/* Assemble every block row of H^DG.  z[K] (K = 0 .. n_elem-1) points to the
 * J columns of element K on Q_K's uniform grid: nq[0] nq[1] nq[2] x J,
 * column-major, x fastest (device pointers when on_device, else host; read
 * only, not retained).  Results stay on the device until dgdft_dg_get_row.
 * DGDFT_EINVAL on a NULL pointer; DGDFT_ENOTCONV when a mass matrix is not
 * positive definite (columns linearly dependent on E_K; the element is named
 * in dgdft_dg_last_error); DGDFT_ECUDA on a CUDA error.                     */
dgdft_status dgdft_dg_assemble(dgdft_dg* dg, const double* const* z, int on_device);

/* The distinct elements of the 3 x 3 x 3 periodic neighbourhood of `elem`,
 * ascending: nb[*n_nb] (host, room for 27).  Block s of the row couples elem
 * with nb[s].                                                             */
dgdft_status dgdft_dg_neighbours(dgdft_dg* dg, int elem, int* nb, int* n_nb);

/* Block row `elem` after dgdft_dg_assemble: n_nb blocks of J x J, block s
 * holding H_{elem, nb[s]} row-major (row i = basis function i of elem,
 * column j = basis function j of nb[s]).  DGDFT_ESTATE before assembly.      */
dgdft_status dgdft_dg_get_row(dgdft_dg* dg, int elem, double* blocks, int on_device);

/* The orthonormal ALBs of element `elem` on its LGL grid from its columns z
 * (as in assemble, z_on_device): phi (n_LGL x J column-major, x fastest).   */
dgdft_status dgdft_dg_lgl_basis(dgdft_dg* dg, int elem, const double* z, int z_on_device, double* phi,
                                int on_device);

/* Density (Eq. density) by dense diagonalisation of the assembled H^DG (the
 * DIAG route of Sec. II.B, for small systems): the lowest n_occ eigenpairs
 * of H^DG c = lambda c (the basis is orthonormal, so a standard problem) by
 * an FP64 one-sided Jacobi eigensolver over the whole GPU (sweeps until no
 * pair of columns has a cosine above sqrt(n) 1e-15, at most 40; DGDFT_ENOTCONV
 * beyond), then rho(x) = sum_{i < n_occ}
 * |psi_i(x)|^2 with psi_i = sum_{K,j} c_{i;K,j} phi_{K,j}, one electron per
 * state as Eq. density is written, on every element's LGL grid.  z: the same
 * columns as the last assemble (z_on_device as there; the basis is rebuilt
 * from them).  eig: n_occ eigenvalues, ascending (host).  rho: n_elem x n_LGL
 * (element-major, x fastest; device when on_device, else host).
 * DGDFT_ESTATE before a successful assemble; DGDFT_EINVAL for n_occ outside
 * 1..n_elem J or n_elem J above 4096.                                      */
dgdft_status dgdft_dg_density(dgdft_dg* dg, const double* const* z, int z_on_device, int n_occ, double* eig,
                              double* rho, int on_device);

/* Sweeps of the Jacobi eigensolver in the last dgdft_dg_density (host int). */
dgdft_status dgdft_dg_density_info(dgdft_dg* dg, int* sweeps);

/* Kernel time of the last assembly per stage (CUDA events on the stream):
 * ms[0] interpolation, ms[1] orthonormalisation and gradients, ms[2] volume
 * integrals, ms[3] face traces and KB coefficients, ms[4] face integrals,
 * ms[5] block assembly, and of the last density: ms[6] eigensolve, ms[7]
 * density evaluation; *launches = kernels of the last assembly.  n = entries
 * of ms (<= 8).                                                            */
dgdft_status dgdft_dg_last_timing(dgdft_dg* dg, double* ms, int n, int* launches);

const char* dgdft_dg_last_error(const dgdft_dg* dg);
void dgdft_dg_destroy(dgdft_dg* dg);

#ifdef __cplusplus
}
#endif

#endif /* DGDFT_DG_H */
