"""Plain, slow, float64 CPU oracle of the constrained DTT/FFT elasticity solver
(Gelebart & Amouzou-Adoun, "Constrained minimization problems and FFT-based solvers").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check of
__graft_entry__ and the cpu_baseline / reference legs of bench.py may import it.  The
CUDA product path never calls it and shares no code with it.

Modules:
  transforms   -- DCT1/DCT3/DST1/DST3/DFT as naive O(n^2) trigonometric sums
                  (Section 3.2.2, Tables 2-3, Eq. 7)
  discrete     -- grid, BCs, HEX1/TETRA2 operators, stress (small strain) and first
                  Piola-Kirchhoff stress (finite strain, Section 5.2), divergence, Paux R0
                  and its symbol, Green step, Eq. 5 residual (Sections 3.1-3.2)
  constraints  -- strong / weak / smooth / tie rows, proj_U and proj_P, reactions,
                  sphere-contact geometry (Sections 4.1-4.2, 5.1)
  solver       -- Anderson acceleration, Algorithm 1, Algorithm 2 (Algorithm 3 with
                  kinematics="FS")
  kkt          -- element-by-element stiffness and dense multiplier solve (Section 4.3)
  hertz        -- Eq. 30

Parity status: every function is pinned by a "not gpu" test.  The Anderson
combination rule, which the paper cites without printing an accelerated iterate, is
pinned by a closed form (the first accelerated iterate of an affine map whose start
error lies in a four-dimensional invariant subspace) and by accelerated solves that
reach the dense multiplier system's solution.
"""
from . import transforms, discrete, constraints, solver, kkt, hertz  # noqa: F401
