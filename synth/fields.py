"""Effective potential and Kleinman-Bylander projectors sampled on grids.

Local pseudopotential per atom: v(r) = -Z erf(r / rc) / r.  Its periodic
lattice sum is conditionally convergent (Coulomb tail), so it is built in
reciprocal space with a neutralising background:

    V(G) = -(4 pi Z / (Omega |G|^2)) exp(-|G|^2 rc^2 / 4) sum_I exp(-i G.R_I),
    V(G = 0) = 0,

over the reciprocal vectors of the periodic cell's own uniform grid, then
summed as a Fourier series at the points of an extended element's grid
(whose origin may sit at a fractional grid offset of the cell grid).  The
real part is kept, which symmetrises the Nyquist terms.

Projectors (two per atom): b_s = exp(-r^2 / (2 sigma^2)),
b_p = (z - Z_I) exp(-r^2 / (2 sigma^2)), sigma = 0.5, truncated at
r_c = 2.0 bohr, minimum image in the periodic cell, grid points outside the
extended element dropped (no wrap inside it), normalised to sum b^2 dV = 1.
They are handed out as CSR rows of values b * sqrt(dV), so the Euclidean norm
of each row is 1 and the discrete nonlocal operator is
sum_p gamma_p v_p v_p^T (Eq. DGvar, nonlocal term).
"""

from __future__ import annotations

import numpy as np

from .geometry import min_image

ZVAL = 5.0
RC_LOC = 0.8
SIGMA_KB = 0.5
RCUT_KB = 2.0


def _freqs(n: int, length: float) -> np.ndarray:
    return 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / length


def local_potential_coeffs(atoms: np.ndarray, cell: np.ndarray, ngrid,
                           z: float = ZVAL, rc: float = RC_LOC) -> dict:
    """Fourier coefficients of the periodic local potential on the cell's grid."""
    gx, gy, gz = (_freqs(int(n), float(l)) for n, l in zip(ngrid, cell))
    omega = float(np.prod(cell))
    g2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        vg = -(4.0 * np.pi * z / (omega * g2)) * np.exp(-g2 * rc * rc / 4.0)
    vg[0, 0, 0] = 0.0
    # structure factor sum_I exp(-i G.R_I), separable per atom
    ex = np.exp(-1j * np.outer(atoms[:, 0], gx))
    ey = np.exp(-1j * np.outer(atoms[:, 1], gy))
    ez = np.exp(-1j * np.outer(atoms[:, 2], gz))
    sf = np.einsum("ic,ib,ia->cba", ez, ey, ex, optimize=True)
    return {"coef": vg * sf, "g": (gx, gy, gz)}


def eval_series(coeffs: dict, origin, spacing, npts) -> np.ndarray:
    """Sum the Fourier series at origin + (i hx, j hy, k hz); shape (nz, ny, nx)."""
    gx, gy, gz = coeffs["g"]
    c = coeffs["coef"]
    ex = np.exp(1j * np.outer(gx, origin[0] + spacing[0] * np.arange(npts[0])))
    ey = np.exp(1j * np.outer(gy, origin[1] + spacing[1] * np.arange(npts[1])))
    ez = np.exp(1j * np.outer(gz, origin[2] + spacing[2] * np.arange(npts[2])))
    v = np.einsum("cba,ai->cbi", c, ex, optimize=True)
    v = np.einsum("cbi,bj->cji", v, ey, optimize=True)
    v = np.einsum("cji,ck->kji", v, ez, optimize=True)
    return np.ascontiguousarray(v.real)


def kb_projectors(atoms: np.ndarray, cell: np.ndarray, origin, spacing, npts,
                  gamma: np.ndarray, wrap_inside: bool = False):
    """Tabulate s and p projectors of atoms whose centres lie in the box.

    Returns (row_ptr int64[P+1], idx int32[nnz], val float64[nnz],
    gamma float64[P]); idx is the flat grid index (x fastest).  gamma has
    shape (n_atoms, 2) and is indexed by the global atom id so an atom keeps
    its weights in every extended element that contains it.
    """
    origin = np.asarray(origin, float)
    spacing = np.asarray(spacing, float)
    npts = np.asarray(npts, int)
    box = spacing * npts
    dv = float(np.prod(spacing))
    rel = np.mod(atoms - origin, cell)
    inside = np.all(rel < box + 1e-12, axis=1)
    row_ptr = [0]
    idx_all, val_all, gam_all = [], [], []
    reach = np.ceil(RCUT_KB / spacing).astype(int) + 1
    for a in np.nonzero(inside)[0]:
        centre = rel[a]  # position relative to the box origin
        c_idx = np.floor(centre / spacing).astype(int)
        axes = []
        for d in range(3):
            r = np.arange(c_idx[d] - reach[d], c_idx[d] + reach[d] + 2)
            if not wrap_inside:
                r = r[(r >= 0) & (r < npts[d])]
            axes.append(r)
        kk, jj, ii = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        pts = np.stack([ii, jj, kk], axis=-1).reshape(-1, 3)
        d = pts * spacing - centre
        d = min_image(d, cell if not wrap_inside else box)
        r2 = np.sum(d * d, axis=1)
        keep = r2 <= RCUT_KB ** 2
        pts, d, r2 = pts[keep], d[keep], r2[keep]
        if wrap_inside:
            pts = np.mod(pts, npts)
        flat = pts[:, 0] + npts[0] * (pts[:, 1] + npts[1] * pts[:, 2])
        order = np.argsort(flat, kind="stable")
        flat, d, r2 = flat[order], d[order], r2[order]
        gauss = np.exp(-r2 / (2.0 * SIGMA_KB ** 2))
        for ell, b in enumerate((gauss, d[:, 2] * gauss)):
            nrm = np.sqrt(np.sum(b * b) * dv)
            if nrm == 0.0:
                continue
            b = b / nrm * np.sqrt(dv)  # Euclidean-normalised row: b * sqrt(dV)
            idx_all.append(flat.astype(np.int32))
            val_all.append(b)
            gam_all.append(gamma[a, ell])
            row_ptr.append(row_ptr[-1] + len(flat))
    if idx_all:
        idx = np.concatenate(idx_all)
        val = np.concatenate(val_all)
    else:
        idx = np.zeros(0, np.int32)
        val = np.zeros(0, np.float64)
    return (np.asarray(row_ptr, np.int64), idx, val, np.asarray(gam_all, np.float64))
