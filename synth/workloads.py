"""Per-element inputs for the five synthetic workloads.

Seeds: numpy default_rng([config id, purpose(, index)]) with purposes
0 = positions, 1 = projector weights gamma, 2 = initial block, 3 = position
perturbations.  The single-element free-electron/atoms case draws its initial
block from the literal default_rng(0).

Workloads (sizes in bohr, grids x by y by z):
  1  one periodic 10^3 box on 16^3, 8 random atoms (min separation 2.5),
     local potential only, 16 eigenpairs, residual 1e-8 Ha.
  2  puckered monolayer 12 x 12 cells (576 atoms, 75.12 x 103.44 x 24) cut
     into 6 x 6 elements; extended element = 3 x 3 elements on 48 x 64 x 40;
     144 atoms / 288 projectors each; 48 computed, 40 kept, residual 1e-6 Ha.
  3  128 standalone periodic elements, grids drawn from {24^3, 32^3,
     40x40x48, 48x48x64} at spacing 0.78, 4..40 random atoms,
     J = 16 + round(80 (n_at - 4) / 36), m = 8 ceil(1.2 J / 8).
  5  monolayer 48 x 18 cells (3,456 atoms) cut into 24 x 9 elements; extended
     element on 48 x 64 x 48; 144 computed, 120 kept.
Small boxes for the sphere-cutoff planewave set (config id 8): two standalone
periodic boxes at spacing 0.78 on 12 x 12 x 16 and 16 x 12 x 12 points, with
4 and 5 random atoms and their projectors, residual 1e-8 Ha.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

from . import fields
from .geometry import monolayer, random_atoms, rng


@dataclass
class ElementInput:
    """One extended element Q_K with its element box E_K (grid index box)."""

    n: tuple            # (nx, ny, nz)
    L: tuple            # (Lx, Ly, Lz) bohr; periodic box of the local problem
    veff: np.ndarray    # float64, shape (nz, ny, nx) -> flat index x fastest
    proj_row_ptr: np.ndarray  # int64[P+1]
    proj_idx: np.ndarray      # int32[nnz] flat grid indices
    proj_val: np.ndarray      # float64[nnz], rows with unit Euclidean norm
    proj_gamma: np.ndarray    # float64[P]
    e_lo: tuple         # E_K lower grid index (inclusive)
    e_hi: tuple         # E_K upper grid index (exclusive)
    m: int              # block size computed
    J: int              # ALBs kept
    tol: float          # residual tolerance, Ha
    seed_key: tuple = field(default=())

    @property
    def ng(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def dv(self) -> float:
        return float(np.prod(np.asarray(self.L) / np.asarray(self.n)))

    @property
    def n_proj(self) -> int:
        return int(len(self.proj_row_ptr) - 1)

    @property
    def n_e(self) -> int:
        return int(np.prod(np.asarray(self.e_hi) - np.asarray(self.e_lo)))


def element_box(n) -> tuple:
    """E_K = points with coordinate in [L/3, 2L/3) along x and y, all z."""
    lo = (math.ceil(n[0] / 3), math.ceil(n[1] / 3), 0)
    hi = (math.ceil(2 * n[0] / 3), math.ceil(2 * n[1] / 3), n[2])
    return lo, hi


def initial_block(el: ElementInput, key=None) -> np.ndarray:
    """Random normal initial block, shape (m, N_g): row i is column i of the
    N_g x m column-major block."""
    key = el.seed_key if key is None else key
    gen = np.random.default_rng(list(key)) if key != (0,) else np.random.default_rng(0)
    return gen.standard_normal((el.m, el.ng))


def _empty_proj():
    return (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float64),
            np.zeros(0, np.float64))


def config1() -> ElementInput:
    cell = np.array([10.0, 10.0, 10.0])
    n = (16, 16, 16)
    atoms = random_atoms(8, cell, 2.5, rng(1, 0))
    co = fields.local_potential_coeffs(atoms, cell, n)
    v = fields.eval_series(co, (0.0, 0.0, 0.0), cell / np.asarray(n), n)
    rp, idx, val, gam = _empty_proj()
    return ElementInput(n=n, L=tuple(cell), veff=v, proj_row_ptr=rp, proj_idx=idx,
                        proj_val=val, proj_gamma=gam, e_lo=(0, 0, 0), e_hi=n,
                        m=16, J=16, tol=1e-8, seed_key=(0,))


@lru_cache(maxsize=4)
def _monolayer_system(cfg: int, nxc: int, nyc: int):
    atoms, cell = monolayer(nxc, nyc, perturb=0.2, gen=rng(cfg, 3))
    gamma = rng(cfg, 1).uniform(0.5, 2.0, size=(len(atoms), 2))
    return atoms, cell, gamma


@lru_cache(maxsize=4)
def _monolayer_coeffs(cfg: int, nxc: int, nyc: int, ngrid: tuple):
    atoms, cell, _ = _monolayer_system(cfg, nxc, nyc)
    return fields.local_potential_coeffs(atoms, cell, ngrid)


def _monolayer_elements(cfg, nxc, nyc, nex, ney, nq, m, J, tol, elems=None):
    atoms, cell, gamma = _monolayer_system(cfg, nxc, nyc)
    ex_w, ey_w = cell[0] / nex, cell[1] / ney
    lq = np.array([3 * ex_w, 3 * ey_w, cell[2]])
    h = lq / np.asarray(nq)
    ngrid = tuple(int(round(c / hh)) for c, hh in zip(cell, h))
    co = _monolayer_coeffs(cfg, nxc, nyc, ngrid)
    e_lo, e_hi = element_box(nq)
    out = []
    ids = range(nex * ney) if elems is None else elems
    for k in ids:
        ix, iy = k % nex, k // nex
        origin = np.array([(ix - 1) * ex_w, (iy - 1) * ey_w, 0.0])
        origin = np.mod(origin, cell)
        v = fields.eval_series(co, origin, h, nq)
        rp, idx, val, gam = fields.kb_projectors(atoms, cell, origin, h, nq, gamma)
        out.append(ElementInput(n=tuple(nq), L=tuple(lq), veff=v, proj_row_ptr=rp,
                                proj_idx=idx, proj_val=val, proj_gamma=gam,
                                e_lo=e_lo, e_hi=e_hi, m=m, J=J, tol=tol,
                                seed_key=(cfg, 2, k)))
    return out


def config2(elems=None):
    """36 extended elements of the 576-atom monolayer (6 x 6 elements)."""
    return _monolayer_elements(2, 12, 12, 6, 6, (48, 64, 40), 48, 40, 1e-6, elems)


def config4(perturbation: int, elems=(0,)):
    """Elements of the 576-atom monolayer geometry with its own seeded
    +-0.2 bohr perturbation (perturbation = 0..63): training geometries of
    the learned preconditioner."""
    atoms, cell = monolayer(12, 12, perturb=0.2, gen=rng(4, 3, perturbation))
    gamma = rng(4, 1, perturbation).uniform(0.5, 2.0, size=(len(atoms), 2))
    nex = ney = 6
    nq = (48, 64, 40)
    ex_w, ey_w = cell[0] / nex, cell[1] / ney
    lq = np.array([3 * ex_w, 3 * ey_w, cell[2]])
    h = lq / np.asarray(nq)
    ngrid = tuple(int(round(c / hh)) for c, hh in zip(cell, h))
    co = fields.local_potential_coeffs(atoms, cell, ngrid)
    e_lo, e_hi = element_box(nq)
    out = []
    for k in elems:
        ix, iy = k % nex, k // nex
        origin = np.mod(np.array([(ix - 1) * ex_w, (iy - 1) * ey_w, 0.0]), cell)
        v = fields.eval_series(co, origin, h, nq)
        rp, idx, val, gam = fields.kb_projectors(atoms, cell, origin, h, nq, gamma)
        out.append(ElementInput(n=tuple(nq), L=tuple(lq), veff=v, proj_row_ptr=rp, proj_idx=idx,
                                proj_val=val, proj_gamma=gam, e_lo=e_lo, e_hi=e_hi, m=48, J=40,
                                tol=1e-6, seed_key=(4, 2, perturbation, k)))
    return out


def config5(elems=None):
    """216 extended elements of the 3,456-atom monolayer (24 x 9 elements)."""
    return _monolayer_elements(5, 48, 18, 24, 9, (48, 64, 48), 144, 120, 1e-6, elems)


CONFIG3_GRIDS = ((24, 24, 24), (32, 32, 32), (40, 40, 48), (48, 48, 64))


def random_element(cfg: int, k: int, n, n_atoms: int, J: int, m: int,
                   tol: float = 1e-6, spacing: float = 0.78) -> ElementInput:
    """A standalone periodic element box with random atoms and projectors."""
    cell = np.asarray(n, float) * spacing
    atoms = random_atoms(n_atoms, cell, 2.5, rng(cfg, 0, k))
    gamma = rng(cfg, 1, k).uniform(0.5, 2.0, size=(n_atoms, 2))
    co = fields.local_potential_coeffs(atoms, cell, n)
    h = cell / np.asarray(n)
    v = fields.eval_series(co, (0.0, 0.0, 0.0), h, n)
    rp, idx, val, gam = fields.kb_projectors(atoms, cell, (0.0, 0.0, 0.0), h, n, gamma,
                                             wrap_inside=True)
    e_lo, e_hi = element_box(n)
    return ElementInput(n=tuple(n), L=tuple(cell), veff=v, proj_row_ptr=rp, proj_idx=idx,
                        proj_val=val, proj_gamma=gam, e_lo=e_lo, e_hi=e_hi, m=m, J=J,
                        tol=tol, seed_key=(cfg, 2, k))


def config3(elems=None):
    """128 uneven standalone elements."""
    draw = rng(3, 4)
    specs = []
    for k in range(128):
        n = CONFIG3_GRIDS[int(draw.integers(0, len(CONFIG3_GRIDS)))]
        n_at = int(draw.integers(4, 41))
        J = 16 + int(round(80 * (n_at - 4) / 36))
        m = 8 * math.ceil(1.2 * J / 8)
        specs.append((n, n_at, J, m))
    ids = range(128) if elems is None else elems
    return [random_element(3, k, *specs[k]) for k in ids]


CUTOFF_BOXES = (((12, 12, 16), 4, 8, 12), ((16, 12, 12), 5, 10, 16))


def cutoff_boxes(elems=None):
    """Two small standalone boxes (grid, atoms, J, m as in CUTOFF_BOXES)
    whose dense Hamiltonians the sphere-cutoff oracle diagonalises."""
    ids = range(len(CUTOFF_BOXES)) if elems is None else elems
    return [random_element(8, k, *CUTOFF_BOXES[k], tol=1e-8) for k in ids]
