"""LOBPCG for the lowest eigenpairs of the local Hamiltonian (oracle, FP64).

Sec. II.B solves the local problem of Eq. localproblem with LOBPCG (Knyazev
2001).  Its five operations are: 1) H applied to the block, 2) Gram products
Phi^T Psi, 3) block updates Phi C, 4) Rayleigh-Ritz on an O(J_K) matrix,
5) the preconditioner.  One iteration applies H once, forms 12 Gram products
(the 6 + 6 distinct blocks of S^T H S and S^T S for S = [X W P]) and 7 block
updates; the steps below follow that order.

  start: X <- X0 orthonormalised (Cholesky-QR), HX = H X, Rayleigh-Ritz on X.
  loop:  R = HX - X Theta; stop when max_{i<J} |r_i| / |x_i| <= tol.
         W = T(R) (Teter); W <- W - X (X^T W); columns of W normalised.
         HW = H W.
         A = S^T (H S), B = S^T S, S = [X W P], both symmetrised.
         B = L L^T; on failure or cond(B) > 1e14 drop P and retry; if that
         fails too, Cholesky-QR W and retry.
         eig(L^-1 A L^-T) -> lowest m pairs (Theta, Z); Y = L^-T Z.
         X = S Y, HX = (HS) Y, P = [W P] Y_WP, HP = [HW HP] Y_WP, then the
         columns of P (and HP with them) scaled to unit norm.
Blocks are (k, N_g) arrays whose rows are the vectors.  The residual is the
absolute Euclidean norm |H x - theta x| / |x| in Ha, max over the kept J, no
locking.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .hamiltonian import apply_h
from .teter import precondition

COND_MAX = 1e14


def cholesky_qr(block: np.ndarray) -> np.ndarray:
    """Rows orthonormalised: block = R^T Q with R upper triangular."""
    g = block @ block.T
    r = sla.cholesky(0.5 * (g + g.T), lower=False)
    return sla.solve_triangular(r, block, trans="T", lower=False)


def _chol_checked(b: np.ndarray):
    if not np.all(np.isfinite(b)) or np.linalg.cond(b) > COND_MAX:
        return None
    try:
        return sla.cholesky(b, lower=True)
    except np.linalg.LinAlgError:
        return None


def rayleigh_ritz(s, hs, m):
    """Lowest m Ritz pairs of the pencil (S^T H S, S^T S); returns
    (theta, Y) or None when the Cholesky factorisation of S^T S fails."""
    a = s @ hs.T
    a = 0.5 * (a + a.T)
    b = s @ s.T
    b = 0.5 * (b + b.T)
    low = _chol_checked(b)
    if low is None:
        return None
    c = sla.solve_triangular(low, a, lower=True)
    c = sla.solve_triangular(low, c.T, lower=True)
    c = 0.5 * (c + c.T)
    theta, z = np.linalg.eigh(c)
    y = sla.solve_triangular(low, z[:, :m], lower=True, trans="T")
    return theta[:m], y


def lobpcg(el, x0: np.ndarray, tol: float | None = None, maxit: int = 500,
           apply=None, precond=None, keep: int | None = None):
    """Run LOBPCG on element `el` from the (m, N_g) block x0.

    Returns a dict with X, HX (rows), theta, res, iterations, converged and a
    per-iteration history of Ritz values and residuals.
    """
    apply = (lambda b: apply_h(b, el)) if apply is None else apply
    precond = (lambda r, x: precondition(r, x, el.n, el.L)) if precond is None else precond
    tol = el.tol if tol is None else tol
    keep = el.J if keep is None else keep
    m = x0.shape[0]
    x = cholesky_qr(np.array(x0, dtype=np.float64))
    hx = apply(x)
    a = x @ hx.T
    theta, z = np.linalg.eigh(0.5 * (a + a.T))
    x = z.T @ x
    hx = z.T @ hx
    p = hp = None
    hist = {"theta": [], "res": [], "dropped_p": 0}
    converged = False
    it = 0
    while True:
        r = hx - theta[:, None] * x
        res = np.linalg.norm(r, axis=1) / np.linalg.norm(x, axis=1)
        hist["theta"].append(theta.copy())
        hist["res"].append(res.copy())
        if np.max(res[:keep]) <= tol:
            converged = True
            break
        if it >= maxit:
            break
        it += 1
        w = precond(r, x)
        w = w - (w @ x.T) @ x
        w = w / np.linalg.norm(w, axis=1)[:, None]
        hw = apply(w)
        out = None
        if p is not None:
            out = rayleigh_ritz(np.vstack([x, w, p]), np.vstack([hx, hw, hp]), m)
            if out is None:
                hist["dropped_p"] += 1
        if out is None:
            out = rayleigh_ritz(np.vstack([x, w]), np.vstack([hx, hw]), m)
            if out is None:
                w = cholesky_qr(w)
                hw = apply(w)
                out = rayleigh_ritz(np.vstack([x, w]), np.vstack([hx, hw]), m)
            s_wp, hs_wp = w, hw
        else:
            s_wp, hs_wp = np.vstack([w, p]), np.vstack([hw, hp])
        theta, y = out
        s = np.vstack([x, s_wp])
        hs = np.vstack([hx, hs_wp])
        y_wp = y[m:]
        x, hx = y.T @ s, y.T @ hs
        p, hp = y_wp.T @ s_wp, y_wp.T @ hs_wp
        # unit columns for P: a rescaling of the basis, which leaves the
        # Rayleigh-Ritz result unchanged but keeps cond(S^T S) a measure of
        # linear dependence rather than of the shrinking step length
        pn = np.linalg.norm(p, axis=1)
        pn[pn == 0.0] = 1.0
        p, hp = p / pn[:, None], hp / pn[:, None]
    return {"X": x, "HX": hx, "theta": theta, "res": res, "iterations": it,
            "converged": converged, "history": hist}
