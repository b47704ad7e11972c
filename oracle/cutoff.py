"""Sphere-cutoff planewave set for the local problem (oracle, FP64).

TEST INFRASTRUCTURE: used only by the tests (see the package docstring).

Eq. Ngecut fixes the grid of Q_K from the kinetic-energy cutoff; the paper
names that cutoff the same as in planewave codes (Sec. III), whose basis is
the set of G with |G|^2/2 <= E_cut.  The grid variant of this package keeps
every G of the FFT grid; this module is the other reading: the local problem
discretised in the span of the planewaves inside the sphere.

Readings:
  * the set is closed, |G|^2/2 <= ecut, with G from the grid's frequencies
    (the Nyquist index with |n/2|, as in ``hamiltonian``); it is symmetric
    under G -> -G, so its span holds real grid functions and the spectral
    mask is an orthogonal projector P on them;
  * the discretised problem is the Galerkin one: the eigenpairs of H
    restricted to range(P), i.e. of Q^T H Q for an orthonormal basis Q of
    range(P) (the same H as the grid variant: kinetic, V_eff on the grid,
    KB projectors);
  * with Eq. Ngecut's ecut, (pi n_d / L_d)^2 / 2, the sphere is the one
    inscribed in the grid's box of frequencies.
"""

from __future__ import annotations

import numpy as np

from .hamiltonian import apply_h, kinetic_symbol


def ngecut_ecut(n, L) -> float:
    """The cutoff that Eq. Ngecut turns into the grid n on the box L: the
    smallest over the axes of (pi n_d / L_d)^2 / 2 (all equal when the
    spacing is)."""
    return float(min(0.5 * (np.pi * nd / ld) ** 2 for nd, ld in zip(n, L)))


def cutoff_mask(n, L, ecut: float) -> np.ndarray:
    """Boolean (nz, ny, nx) mask of the grid frequencies inside the sphere."""
    return kinetic_symbol(n, L) <= ecut


def project(block: np.ndarray, n, L, ecut: float) -> np.ndarray:
    """P applied to every row: the component in the span of the set."""
    block = np.atleast_2d(block)
    g = block.reshape(block.shape[0], n[2], n[1], n[0])
    f = np.fft.fftn(g, axes=(1, 2, 3)) * cutoff_mask(n, L, ecut)[None]
    return np.fft.ifftn(f, axes=(1, 2, 3)).real.reshape(block.shape)


def set_basis(n, L, ecut: float) -> np.ndarray:
    """Orthonormal basis of range(P) as (N_g, N_set) columns: the
    eigenvectors of the dense projector with eigenvalue 1."""
    ng = int(np.prod(n))
    p = project(np.eye(ng), n, L, ecut)
    p = 0.5 * (p + p.T)
    w, v = np.linalg.eigh(p)
    return v[:, w > 0.5]


def galerkin_eigenpairs(el, ecut: float, k: int):
    """Lowest k eigenpairs of H on the span of the set, by dense
    diagonalisation of Q^T H Q.  Returns (theta, vectors as (k, N_g) rows)."""
    h = apply_h(np.eye(el.ng), el)
    h = 0.5 * (h + h.T)
    q = set_basis(el.n, el.L, ecut)
    hs = q.T @ h @ q
    theta, z = np.linalg.eigh(0.5 * (hs + hs.T))
    return theta[:k], (q @ z[:, :k]).T


def full_eigenpairs(el, k: int):
    """Lowest k eigenpairs of H over the whole grid space (dense)."""
    h = apply_h(np.eye(el.ng), el)
    theta, z = np.linalg.eigh(0.5 * (h + h.T))
    return theta[:k], z[:, :k].T
