"""Plain, slow complex128 CPU oracle for the moving-PML sweeping preconditioner.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code,
tables or constants with the CUDA library; the two meet only through the
seeded input generators, which hold none of the method's arithmetic.

Every function restates the paper (Engquist & Ying, "Sweeping preconditioner
for the Helmholtz equation: moving perfectly matched layers", 2010) in the
order and notation of the paper, with library primitives (sparse LU, LAPACK
band LU, dense solve) as steps:

* ``helmholtz2d`` -- PML profile (Eq. sigma), stretch factors, the 5-point
  discretisation (Eq. helmd) of A and of the shifted operator A_alpha
  (Eq. helmalpha).
* ``sweep2d``     -- block partition (two fronts, d layers per step,
  Sec. 2.3), moving-PML subproblems H_m (Eq. helma), their banded LU in the
  x2-first ordering (Algorithm 3), the approximate sweep M_alpha
  (Algorithm 4), and the exact block LDL^t sweep (Algorithms 1 and 2).
* ``krylov``      -- right-preconditioned flexible GMRES and the paper's
  left-preconditioned GMRES on M_alpha A (Sec. 2.3).
* ``helmholtz3d`` -- the 7-point operator (Eq. helmd3) and the slab sweep
  (Algorithms 5 and 6) with exact sparse solves of each slab problem.
* ``cnn``         -- FP64 reference of the 3-layer convolutional
  post-correction (forward, backward, Adam).
* ``polar``       -- the scattering problem of Sec. 3 (sound-soft disk, polar
  grid periodic in theta, radial PML) and its radial sweep (Algorithms 3 and 4
  on rings); the CUDA library has no counterpart for this variant.

Each function's docstring states the passage it follows and the readings
of passages the paper leaves open; the tests pin every function against
values and limits the paper and the mathematics fix (hand-computed profiles,
exact solves, Green's functions, finite differences).
"""
