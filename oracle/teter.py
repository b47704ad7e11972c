"""Teter-Payne-Allan kinetic preconditioner (oracle, FP64).

Sec. II.B applies the preconditioner of Payne, Teter, Allan et al. (1992)
to every residual column independently.  The paper does not print its
formula.  Reading used on both sides: for residual r_i of Ritz vector x_i,

    w_i = F^-1 [ K(s) F r_i ],   s = (|G|^2 / 2) / T_i,
    K(s) = (27 + 18 s + 12 s^2 + 8 s^3) / (27 + 18 s + 12 s^2 + 8 s^3 + 16 s^4),
    T_i  = <x_i, -1/2 Lap x_i> / <x_i, x_i>   (kinetic energy of x_i).

Pins: K(0) = 1 with K - 1 = O(s^4), K(s) -> 1/(2 s) as s -> infinity,
0 < K <= 1.  The choice of T_i itself is "parity unpinned": nothing in the
paper fixes it, so both sides share this reading.
"""

from __future__ import annotations

import numpy as np

from .hamiltonian import apply_kinetic, kinetic_symbol


def teter_k(s):
    """The rational Teter function K(s)."""
    s = np.asarray(s, dtype=np.float64)
    num = 27.0 + s * (18.0 + s * (12.0 + s * 8.0))
    return num / (num + 16.0 * s ** 4)


def kinetic_energy(block: np.ndarray, n, L) -> np.ndarray:
    """T_i = <x_i, -1/2 Lap x_i> / <x_i, x_i> for every row x_i."""
    kx = apply_kinetic(block, n, L)
    return np.einsum("ij,ij->i", block, kx) / np.einsum("ij,ij->i", block, block)


def precondition(resid: np.ndarray, x: np.ndarray, n, L) -> np.ndarray:
    """Apply K((|G|^2/2)/T_i) in G-space to residual row i."""
    t = kinetic_energy(x, n, L)
    sym = kinetic_symbol(n, L)
    r = resid.reshape(resid.shape[0], n[2], n[1], n[0])
    f = np.fft.fftn(r, axes=(1, 2, 3))
    k = teter_k(sym[None] / t[:, None, None, None])
    return np.fft.ifftn(f * k, axes=(1, 2, 3)).real.reshape(resid.shape)
