"""Plain FP64 CPU oracle for DGDFT's adaptive-local-basis generation.

TEST INFRASTRUCTURE.  Nothing in the product path may import, call, link or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library; both sides only consume the seeded inputs built by ``synth``.

What it computes, per extended element Q_K (Sec. II.A, Eq. localproblem):
  * the discretised local Hamiltonian -1/2 Lap + V_eff + V_nl on a periodic
    uniform grid, kinetic term spectral over every G of the FFT grid
    (``hamiltonian``; Eq. Ngecut for the grid, Sec. II.B operation 1);
  * the Teter-Payne-Allan kinetic preconditioner (``teter``; Sec. II.B);
  * LOBPCG for the lowest m eigenpairs (``lobpcg``; Sec. II.B operations
    1-5, the 12 Gram products and 7 block updates per iteration);
  * restriction of the lowest J eigenvectors to E_K and their
    orthonormalisation by SVD (``alb``; Sec. II.A, Sec. II.B);
  * the learned preconditioner's 3-D convolutional network, forward and
    backward (``convnet``);
  * the DG Hamiltonian assembled from the ALBs (Eq. DGHamiltonian): LGL
    quadrature and differentiation, trigonometric interpolation from Q_K's
    grid, the volume, KB and interior-penalty face blocks (``dg``).
  * the sphere-cutoff planewave set (|G|^2/2 <= ecut, Eq. Ngecut's
    cutoff): its projector and the Galerkin eigenpairs of H on its span by
    dense diagonalisation (``cutoff``).

Pins (tests/test_oracle_*.py) tie every function to closed forms, brute-force
diagonalisation and invariants rather than to itself.  Functions whose
definition is a reading of a silent passage say so; the Teter
preconditioner's scale parameter is "parity unpinned" beyond the limits of
its rational function (see ``teter``).
"""
