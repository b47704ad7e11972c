"""Atom positions for the synthetic workloads.

The paper's test systems are phosphorene monolayers (Sec. III, P140/P3500/
P14000) whose coordinates are not printed.  The stand-in is a puckered
4-atom orthorhombic cell (two sub-layers 4.0 bohr apart) tiled in-plane with
vacuum along z.  Fractional in-plane positions and absolute heights of the
cell are this project's choice; the minimum interatomic distance is about
4.06 bohr.
"""

from __future__ import annotations

import numpy as np

# Orthorhombic puckered cell, bohr.
CELL_A = 6.26
CELL_B = 8.62
PUCKER = 4.0
VACUUM = 20.0
# (fractional x, fractional y, height relative to the layer mid-plane)
CELL_SITES = (
    (0.0, 0.10, -0.5 * PUCKER),
    (0.5, 0.40, -0.5 * PUCKER),
    (0.5, 0.60, +0.5 * PUCKER),
    (0.0, 0.90, +0.5 * PUCKER),
)


def rng(*key: int) -> np.random.Generator:
    """Seeded generator; key = (config id, purpose[, index])."""
    return np.random.default_rng(list(key))


def monolayer(nx_cells: int, ny_cells: int, perturb: float = 0.0,
              gen: np.random.Generator | None = None):
    """Tile the puckered cell nx_cells x ny_cells; return (atoms[N,3], cell[3]).

    The layer mid-plane sits at the centre of the z extent (PUCKER + VACUUM).
    With perturb > 0 every coordinate gets an independent U[-perturb, perturb]
    displacement drawn from gen.
    """
    lz = PUCKER + VACUUM
    cell = np.array([nx_cells * CELL_A, ny_cells * CELL_B, lz])
    pos = []
    for cy in range(ny_cells):
        for cx in range(nx_cells):
            for fx, fy, dz in CELL_SITES:
                pos.append(((cx + fx) * CELL_A, (cy + fy) * CELL_B, 0.5 * lz + dz))
    atoms = np.asarray(pos, dtype=np.float64)
    if perturb > 0.0:
        atoms = atoms + gen.uniform(-perturb, perturb, size=atoms.shape)
    atoms = np.mod(atoms, cell)
    return atoms, cell


def min_image(d: np.ndarray, cell: np.ndarray) -> np.ndarray:
    """Minimum-image displacement in an orthorhombic periodic cell."""
    return d - cell * np.round(d / cell)


def random_atoms(n_atoms: int, cell: np.ndarray, min_sep: float,
                 gen: np.random.Generator, max_tries: int = 100000) -> np.ndarray:
    """Uniform random positions with minimum-image separation >= min_sep
    (rejection sampling, one candidate at a time)."""
    atoms = []
    tries = 0
    while len(atoms) < n_atoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_atoms: could not place atoms")
        c = gen.uniform(0.0, 1.0, size=3) * cell
        if atoms:
            d = min_image(np.asarray(atoms) - c, cell)
            if np.min(np.linalg.norm(d, axis=1)) < min_sep:
                continue
        atoms.append(c)
    return np.asarray(atoms, dtype=np.float64)
