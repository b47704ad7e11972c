"""Local Kohn-Sham Hamiltonian on an extended element (oracle, FP64).

Sec. II.A, Eq. localproblem: H = -1/2 Lap + V_eff^{Q_K} + V_nl^{Q_K} on Q_K,
discretised by planewaves on a uniform grid (Sec. II.B, Eq. Ngecut).
Readings taken where the paper is silent:
  * Q_K is a periodic box; the planewave set is every G of the FFT grid,
    the Nyquist plane included with |G| built from |n/2|, so the
    discrete kinetic operator is exactly F^-1 diag(|G|^2/2) F;
  * grid vectors use the Euclidean inner product (dV is a constant factor
    that does not change the eigenproblem); the nonlocal term of Eq. DGvar,
    gamma <b, psi> b, becomes sum_p gamma_p v_p (v_p^T psi) with
    v_p = b_p sqrt(dV) of unit Euclidean norm.
Blocks are arrays of shape (k, N_g): row i is vector i, flat index x fastest.
"""

from __future__ import annotations

import numpy as np


def gvectors(n, L):
    """Per-axis reciprocal components 2 pi f / L_d, f in FFT order."""
    return tuple(2.0 * np.pi * np.fft.fftfreq(int(nd), d=1.0 / int(nd)) / float(ld)
                 for nd, ld in zip(n, L))


def kinetic_symbol(n, L) -> np.ndarray:
    """|G|^2 / 2 on the (nz, ny, nx) FFT grid (the symbol of -1/2 Lap)."""
    gx, gy, gz = gvectors(n, L)
    return 0.5 * (gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2)


def _grid(block, n):
    return block.reshape(block.shape[0], n[2], n[1], n[0])


def apply_kinetic(block: np.ndarray, n, L) -> np.ndarray:
    """-1/2 Lap applied spectrally to every row of the block."""
    sym = kinetic_symbol(n, L)
    f = np.fft.fftn(_grid(block, n), axes=(1, 2, 3))
    out = np.fft.ifftn(f * sym[None], axes=(1, 2, 3)).real
    return out.reshape(block.shape)


def nonlocal_matrix(el):
    """Projector rows as a dense (P, N_g) matrix (small cases and tests)."""
    p = el.n_proj
    dense = np.zeros((p, el.ng))
    for i in range(p):
        s, e = el.proj_row_ptr[i], el.proj_row_ptr[i + 1]
        dense[i, el.proj_idx[s:e]] = el.proj_val[s:e]
    return dense


def projector_coefficients(block: np.ndarray, el) -> np.ndarray:
    """C[p, i] = v_p^T psi_i (the inner products <b_p, psi_i>)."""
    c = np.zeros((el.n_proj, block.shape[0]))
    for p in range(el.n_proj):
        s, e = el.proj_row_ptr[p], el.proj_row_ptr[p + 1]
        c[p] = block[:, el.proj_idx[s:e]] @ el.proj_val[s:e]
    return c


def apply_nonlocal(block: np.ndarray, el) -> np.ndarray:
    """sum_p gamma_p v_p (v_p^T psi) for every row psi of the block."""
    out = np.zeros_like(block)
    if el.n_proj == 0:
        return out
    c = projector_coefficients(block, el)
    for p in range(el.n_proj):
        s, e = el.proj_row_ptr[p], el.proj_row_ptr[p + 1]
        out[:, el.proj_idx[s:e]] += el.proj_gamma[p] * np.outer(c[p], el.proj_val[s:e])
    return out


def apply_h(block: np.ndarray, el) -> np.ndarray:
    """H psi = -1/2 Lap psi + V_eff psi + V_nl psi (Eq. localproblem)."""
    block = np.atleast_2d(block)
    return (apply_kinetic(block, el.n, el.L)
            + block * el.veff.reshape(1, -1)
            + apply_nonlocal(block, el))


def dense_h(el) -> np.ndarray:
    """Dense N_g x N_g matrix of H, assembled column by column (small grids)."""
    return apply_h(np.eye(el.ng), el).T
