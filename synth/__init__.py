"""Seeded synthetic inputs for the ALB-generation hot path.

This package builds the inputs of the per-element local Kohn-Sham problem of
DGDFT (Sec. II.A, Eq. localproblem): atom positions on a puckered-monolayer
lattice or at random, the restricted effective potential V_eff^{Q_K} on each
extended element's uniform grid, the tabulated Kleinman-Bylander projection
vectors b_{I,l} with weights gamma_{I,l} (Eq. DGvar, nonlocal term), the
element box E_K inside Q_K and the random initial block.

It holds none of the eigensolver's arithmetic.  Both the CPU oracle and the
GPU library consume exactly these arrays, so input construction (lattice
sums, projector sampling) is never part of a parity comparison.
"""

from .workloads import (  # noqa: F401
    ElementInput,
    config1,
    config2,
    config3,
    config4,
    config5,
    cutoff_boxes,
    element_box,
    initial_block,
    random_element,
)
