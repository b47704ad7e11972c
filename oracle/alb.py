"""Restriction to the element and orthonormalisation (oracle, FP64).

Sec. II.A: the lowest J_K eigenfunctions on Q_K are restricted to E_K; the
truncated vectors are not orthonormal, so they are orthonormalised and set
to zero outside E_K, which makes the ALB overlap matrix the identity
(Eq. orthonormal).  Sec. II.B repeats this after LOBPCG.  The paper does not
name the orthonormalisation; the reading used is the thin SVD
Phi~ = U Sigma V^T keeping all J left singular vectors, scaled by
1/sqrt(dV) so that sum_pts phi_i phi_j dV = delta_ij.  A variant restricts
all m computed vectors and keeps the J left singular vectors of the largest
singular values (orthonormalise_top).  Results are compared as spans
(principal angles), never column by column.
"""

from __future__ import annotations

import numpy as np

from .lobpcg import lobpcg


def element_indices(el) -> np.ndarray:
    """Flat Q_K grid indices of E_K's points, x fastest within the box."""
    lo, hi, n = el.e_lo, el.e_hi, el.n
    k, j, i = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                          np.arange(lo[0], hi[0]), indexing="ij")
    return (i + n[0] * (j + n[1] * k)).reshape(-1)


def restrict(x: np.ndarray, el, keep: int | None = None) -> np.ndarray:
    """Rows of the lowest `keep` eigenvectors restricted to E_K: (J, N_E)."""
    keep = el.J if keep is None else keep
    return x[:keep][:, element_indices(el)]


def orthonormalise(phi_t: np.ndarray, dv: float) -> np.ndarray:
    """Left singular vectors of the (N_E x J) restricted block, L2-scaled."""
    u, _, _ = np.linalg.svd(phi_t.T, full_matrices=False)
    return u.T / np.sqrt(dv)


def orthonormalise_top(phi_t: np.ndarray, dv: float, keep: int) -> np.ndarray:
    """Variant of the restriction step: the (k, N_E) restricted block of all
    k computed vectors -> the `keep` left singular vectors of the largest
    singular values, L2-scaled (rows)."""
    u, _, _ = np.linalg.svd(phi_t.T, full_matrices=False)  # singular values descending
    return u[:, :keep].T / np.sqrt(dv)


def generate_alb(el, x0: np.ndarray, **kw):
    """Full ALB generation for one element: LOBPCG, restriction, SVD."""
    out = lobpcg(el, x0, **kw)
    phi = orthonormalise(restrict(out["X"], el), el.dv)
    out["phi"] = phi
    return out


def principal_angles(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Principal angles (radians) between the row spaces of a and b."""
    qa, _ = np.linalg.qr(a.T)
    qb, _ = np.linalg.qr(b.T)
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return np.arccos(np.clip(s, -1.0, 1.0))


def sin_max_angle(a: np.ndarray, b: np.ndarray) -> float:
    """sin of the largest principal angle, computed stably via projections."""
    qa, _ = np.linalg.qr(a.T)
    qb, _ = np.linalg.qr(b.T)
    resid = qb - qa @ (qa.T @ qb)
    return float(np.linalg.norm(resid, 2))
