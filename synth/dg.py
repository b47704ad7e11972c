"""Inputs of the DG Hamiltonian assembly (Eq. DGHamiltonian).

The periodic cell is cut into ne_x x ne_y x ne_z equal element boxes E_K,
K = ix + ne_x (iy + ne_y iz).  Each extended element Q_K is the box of
q_span elements per direction centred on E_K (q_span 3, or 1 where one
element spans the cell, as along z of the monolayer), sampled on its own
uniform nq grid.  The ALB functions of E_K are spanned by J columns given on
Q_K's grid (after an ALB solve, the lowest J Ritz vectors).

What this module provides, for either side to consume:
  * the domain description (sizes, counts, the penalty alpha, and the
    number of Legendre-Gauss-Lobatto points per direction: twice the uniform
    points that E_K's own extent holds at Q_K's spacing, Sec. III);
  * V_eff and the KB projection functions evaluated at points the caller
    passes in (each side computes its own quadrature nodes);
  * seeded smooth blocks on the Q_K grids (band-limited random series).

It holds none of the assembly's arithmetic: no quadrature, interpolation,
differentiation or integral is computed here.  Projection functions are the
fixture of the local problem (s and p Gaussians, sigma 0.5, cut at 2 bohr,
minimum image in the cell) normalised to unit L2 norm over the cut ball.
"""

from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np
from scipy import integrate

from . import fields
from .geometry import min_image, monolayer, random_atoms, rng
from .workloads import _monolayer_coeffs, _monolayer_system


@dataclass
class DGDomain:
    cell: np.ndarray      # periodic cell (bohr)
    ne: tuple             # elements per direction
    q_span: tuple         # elements per direction covered by Q_K (3, or 1 with ne = 1)
    nq: tuple             # Q_K uniform grid (x, y, z)
    J: int                # basis functions per element
    alpha: float          # penalty parameter of Eq. DGvar
    atoms: np.ndarray
    gamma: np.ndarray     # (n_atoms, 2): s and p weights
    coeffs: dict          # Fourier coefficients of the cell's V_eff
    seed_key: tuple

    @property
    def n_elem(self) -> int:
        return int(np.prod(self.ne))

    @property
    def le(self) -> np.ndarray:
        return np.asarray(self.cell, float) / np.asarray(self.ne)

    @property
    def lq(self) -> np.ndarray:
        return self.le * np.asarray(self.q_span)

    @property
    def e_off(self) -> np.ndarray:
        """Lower corner of E_K inside Q_K."""
        return self.le * (np.asarray(self.q_span) // 2)

    @property
    def nl(self) -> tuple:
        h = self.lq / np.asarray(self.nq)
        return tuple(int(2 * round(float(l / hh))) for l, hh in zip(self.le, h))

    @property
    def ng_q(self) -> int:
        return int(np.prod(self.nq))

    @property
    def n_lgl(self) -> int:
        return int(np.prod(self.nl))

    def index(self, ix, iy, iz) -> int:
        nx, ny, nz = self.ne
        return int(ix % nx + nx * ((iy % ny) + ny * (iz % nz)))

    def coords(self, k: int) -> tuple:
        nx, ny, _ = self.ne
        return k % nx, (k // nx) % ny, k // (nx * ny)

    def corner(self, k: int) -> np.ndarray:
        """Lower corner of E_K in the cell."""
        return np.asarray(self.coords(k), float) * self.le


def potential_at(dom: DGDomain, xs, ys, zs) -> np.ndarray:
    """V_eff (the cell's Fourier series) at the tensor points; (nz, ny, nx)."""
    gx, gy, gz = dom.coeffs["g"]
    c = dom.coeffs["coef"]
    ex = np.exp(1j * np.outer(gx, xs))
    ey = np.exp(1j * np.outer(gy, ys))
    ez = np.exp(1j * np.outer(gz, zs))
    v = np.einsum("cba,ai->cbi", c, ex, optimize=True)
    v = np.einsum("cbi,bj->cji", v, ey, optimize=True)
    v = np.einsum("cji,ck->kji", v, ez, optimize=True)
    return np.ascontiguousarray(v.real)


@lru_cache(maxsize=None)
def _kb_norms() -> tuple:
    """1 / ||b||_2 over the cut ball for the s and p shapes."""
    s2 = fields.SIGMA_KB ** 2
    rc = fields.RCUT_KB
    ss = integrate.quad(lambda r: 4 * np.pi * r * r * np.exp(-r * r / s2), 0.0, rc,
                        epsabs=0, epsrel=1e-12)[0]
    # z^2 averages to r^2 / 3 over the sphere
    pp = integrate.quad(lambda r: 4 * np.pi / 3 * r ** 4 * np.exp(-r * r / s2), 0.0, rc,
                        epsabs=0, epsrel=1e-12)[0]
    return 1.0 / np.sqrt(ss), 1.0 / np.sqrt(pp)


def projectors_at(dom: DGDomain, xs, ys, zs):
    """KB projection functions at the tensor points (absolute cell coordinates).

    Returns (pid int32[P], row_ptr int64[P+1], idx int32[nnz], val float64[nnz])
    for every projector with a point inside r <= r_c; idx is the flat index of
    the tensor grid (x fastest); pid = 2 * atom + l (l = 0 s, 1 p).  Weights
    gamma[pid] come from gamma_table(dom).
    """
    xs, ys, zs = (np.asarray(a, float) for a in (xs, ys, zs))
    ns, np_ = _kb_norms()
    rc2 = fields.RCUT_KB ** 2
    cell = np.asarray(dom.cell, float)
    pid, row_ptr, idx_all, val_all = [], [0], [], []
    nx, ny = len(xs), len(ys)
    for a, r0 in enumerate(dom.atoms):
        dx = min_image(xs - r0[0], cell[0])
        dy = min_image(ys - r0[1], cell[1])
        dz = min_image(zs - r0[2], cell[2])
        ix = np.nonzero(np.abs(dx) <= fields.RCUT_KB)[0]
        iy = np.nonzero(np.abs(dy) <= fields.RCUT_KB)[0]
        iz = np.nonzero(np.abs(dz) <= fields.RCUT_KB)[0]
        if not (len(ix) and len(iy) and len(iz)):
            continue
        kk, jj, ii = np.meshgrid(iz, iy, ix, indexing="ij")
        r2 = dx[ii] ** 2 + dy[jj] ** 2 + dz[kk] ** 2
        keep = r2 <= rc2
        if not keep.any():
            continue
        ii, jj, kk, r2 = ii[keep], jj[keep], kk[keep], r2[keep]
        flat = (ii + nx * (jj + ny * kk)).astype(np.int64)
        order = np.argsort(flat, kind="stable")
        flat, r2, zk = flat[order], r2[order], dz[kk[order]]
        gauss = np.exp(-r2 / (2.0 * fields.SIGMA_KB ** 2))
        for ell, b in enumerate((ns * gauss, np_ * zk * gauss)):
            pid.append(2 * a + ell)
            idx_all.append(flat.astype(np.int32))
            val_all.append(b)
            row_ptr.append(row_ptr[-1] + len(flat))
    idx = np.concatenate(idx_all) if idx_all else np.zeros(0, np.int32)
    val = np.concatenate(val_all) if val_all else np.zeros(0, np.float64)
    return (np.asarray(pid, np.int32), np.asarray(row_ptr, np.int64), idx, val)


def gamma_table(dom: DGDomain) -> np.ndarray:
    """gamma[pid] for pid = 2 * atom + l."""
    return np.ascontiguousarray(dom.gamma.reshape(-1))


def smooth_block(dom: DGDomain, k: int, kmax=(3, 3, 3)) -> np.ndarray:
    """Seeded band-limited random functions on Q_K's grid, shape (J, N_gQ)
    (row j is column j of the N_gQ x J block, x fastest): the real part of a
    Fourier series over |m_d| <= kmax_d with complex normal coefficients
    damped as 1 / (1 + |m|^2), scaled to unit mean square."""
    gen = np.random.default_rng([*dom.seed_key, 7, k])
    nx, ny, nz = dom.nq
    out = np.empty((dom.J, nz, ny, nx))
    mz, my, mx = (np.fft.fftfreq(n, d=1.0 / n) for n in (nz, ny, nx))
    band = ((np.abs(mz)[:, None, None] <= kmax[2]) & (np.abs(my)[None, :, None] <= kmax[1])
            & (np.abs(mx)[None, None, :] <= kmax[0]))
    damp = 1.0 / (1.0 + mz[:, None, None] ** 2 + my[None, :, None] ** 2 + mx[None, None, :] ** 2)
    for j in range(dom.J):
        c = (gen.standard_normal((nz, ny, nx)) + 1j * gen.standard_normal((nz, ny, nx))) * damp * band
        f = np.fft.ifftn(c).real
        out[j] = f / np.sqrt(np.mean(f * f))
    return out.reshape(dom.J, -1)


def dg_config2(J: int = 40, alpha: float = 20.0) -> DGDomain:
    """The 576-atom monolayer of the ALB workload (6 x 6 x 1 elements,
    Q_K on 48 x 64 x 40 spanning 3 x 3 elements and the cell's z)."""
    atoms, cell, gamma = _monolayer_system(2, 12, 12)
    nq = (48, 64, 40)
    le = cell / np.array([6, 6, 1])
    h = le * np.array([3, 3, 1]) / np.asarray(nq)
    ngrid = tuple(int(round(c / hh)) for c, hh in zip(cell, h))
    co = _monolayer_coeffs(2, 12, 12, ngrid)
    return DGDomain(cell=cell, ne=(6, 6, 1), q_span=(3, 3, 1), nq=nq, J=J, alpha=alpha,
                    atoms=atoms, gamma=gamma, coeffs=co, seed_key=(2, 9))


def dg_config5(J: int = 120, alpha: float = 20.0) -> DGDomain:
    """The 3,456-atom monolayer of the large workload (24 x 9 x 1 elements,
    Q_K on 48 x 64 x 48 spanning 3 x 3 elements and the cell's z)."""
    atoms, cell, gamma = _monolayer_system(5, 48, 18)
    nq = (48, 64, 48)
    le = cell / np.array([24, 9, 1])
    h = le * np.array([3, 3, 1]) / np.asarray(nq)
    ngrid = tuple(int(round(c / hh)) for c, hh in zip(cell, h))
    co = _monolayer_coeffs(5, 48, 18, ngrid)
    return DGDomain(cell=cell, ne=(24, 9, 1), q_span=(3, 3, 1), nq=nq, J=J, alpha=alpha,
                    atoms=atoms, gamma=gamma, coeffs=co, seed_key=(5, 9))


def dg_small_layer(J: int = 8, alpha: float = 20.0) -> DGDomain:
    """3 x 2 cells of the monolayer (24 atoms) cut into 3 x 3 x 1 elements;
    Q_K (3 x 3 elements) is the whole in-plane cell, on 24 x 24 x 30."""
    atoms, cell = monolayer(3, 2, perturb=0.2, gen=rng(6, 3))
    gamma = rng(6, 1).uniform(0.5, 2.0, size=(len(atoms), 2))
    nq = (24, 24, 30)
    co = fields.local_potential_coeffs(atoms, cell, nq)
    return DGDomain(cell=cell, ne=(3, 3, 1), q_span=(3, 3, 1), nq=nq, J=J, alpha=alpha,
                    atoms=atoms, gamma=gamma, coeffs=co, seed_key=(6, 9))


def dg_small_cube(J: int = 6, alpha: float = 20.0) -> DGDomain:
    """A 12 bohr periodic cube with 6 random atoms cut into 3 x 3 x 3
    elements; Q_K (3 x 3 x 3 elements) is the cell, on 18^3."""
    cell = np.array([12.0, 12.0, 12.0])
    atoms = random_atoms(6, cell, 2.5, rng(7, 0))
    gamma = rng(7, 1).uniform(0.5, 2.0, size=(len(atoms), 2))
    nq = (18, 18, 18)
    co = fields.local_potential_coeffs(atoms, cell, nq)
    return DGDomain(cell=cell, ne=(3, 3, 3), q_span=(3, 3, 3), nq=nq, J=J, alpha=alpha,
                    atoms=atoms, gamma=gamma, coeffs=co, seed_key=(7, 9))
