"""Plain, slow FP64 CPU oracle of the MLSDC-SH method (Hamon, Schreiber, Minion,
"Multi-Level Spectral Deferred Corrections Scheme for the Shallow Water
Equations on the Rotating Sphere").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import anything from this
package.  The CUDA product path never imports it, and this package imports
nothing from the CUDA path: the two share no code.  The only module both
sides use is the seeded input generator ``paper_1805_07923_gb300.inputs``,
which holds no arithmetic of the method.

Everything here is float64 numpy, written step by step after the paper; a
library primitive (matmul, polynomial roots, LU) is used only where it is a
step of a plain definition.  Modules:

  quadrature  Gaussian latitudes, Gauss-Lobatto time nodes, the collocation
              matrix Q, the forward-Euler and LU-trick matrices, Lagrange
              interpolation matrices (Sec. 3, Sec. 4.2, Sec. 4.3.3)
  legendre    normalised associated Legendre functions and
              H = (1 - mu^2) dP/dmu (Sec. 3, Eq. spectral_to_physical_space)
  sht         spherical-harmonic synthesis / analysis, scalar and vector
              (Sec. 3, Eqs. spectral_to_physical_space, fourier_transform,
              legendre_transform; Sec. 2 Helmholtz decomposition)
  swe         shallow-water right-hand sides F_E, F_I and the implicit
              solve (Sec. 2, Sec. 4.1, Sec. 4.4)
  sdc         IMEX SDC sweep, SDC step, two-level MLSDC step (Sec. 4.2,
              Sec. 4.3, Algorithm 1)
  cost        the cost model and theoretical speedup (Sec. 4.5)
  adjoint     tangent-linear and adjoint of the SDC/MLSDC step
"""
