"""Comparison of GPU Ritz blocks with the oracle's stored Ritz values.

Helpers for the GPU parity tests (test infrastructure, like oracle/).  The
oracle's Ritz values and residuals are stored by tests/golden/make_golden.py
(oracle LOBPCG to 1e-9 Ha on the lowest J + 4 pairs).  The subspace of the
GPU's lowest J Ritz vectors is compared with the oracle's through the
Davis-Kahan sin-theta theorem: for an orthonormal block X with residual
R = H X - X Theta, the sine of the largest angle to the invariant subspace of
the lowest J eigenvalues is at most |R|_2 / delta, delta the distance from
Theta's largest value to lambda_{J+1}.  The same bound for the oracle's block
(from its stored residuals) added to it bounds the angle between the two
computed subspaces.
"""

import os

import numpy as np

from oracle import hamiltonian as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ritz_golden(name):
    """(theta, residual) arrays of the oracle's lowest J + 4 Ritz pairs."""
    d = np.loadtxt(os.path.join(GOLDEN, f"{name}_ritz.txt"))
    return d[:, 0], d[:, 1]


def angle_bound(x, theta, el, gold_theta, gold_res):
    """Davis-Kahan bound on sin(angle) between span(x[:J]) and the oracle's
    J-dimensional Ritz subspace, and the gap lambda_{J+1} - lambda_J.

    x: GPU Ritz block rows (>= J), theta: its J Ritz values; residuals are
    recomputed with the oracle's H.  lambda_{J+1} is taken from below as the
    oracle's Ritz value minus its residual."""
    J = el.J
    q, _ = np.linalg.qr(x[:J].T)
    xq = q.T
    hx = H.apply_h(xq, el)
    th = np.einsum("ij,ij->i", xq, hx)
    r = hx - th[:, None] * xq
    r2 = float(np.linalg.norm(r, 2))
    lam_next = gold_theta[J] - gold_res[J]
    d_gpu = lam_next - float(np.max(th))
    d_or = lam_next - gold_theta[J - 1]
    r_or = float(np.sqrt(np.sum(gold_res[:J] ** 2)))
    if d_gpu <= 0 or d_or <= 0:
        return float("inf"), gold_theta[J] - gold_theta[J - 1]
    return r2 / d_gpu + r_or / d_or, gold_theta[J] - gold_theta[J - 1]
