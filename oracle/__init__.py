"""FP64 CPU oracle for the DGDFT hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  The product path (the CUDA
library and its Python binding) never calls it; there is no CPU fallback.

It is a plain, slow, obviously correct NumPy/SciPy restatement of the method
(Sec. II.A of the paper) and shares no code with the CUDA path:

* ``local_operator`` -- the local Kohn-Sham Hamiltonian on an extended element
  (Eq. LocalKS) in the plane-wave / real-grid basis, and its dense matrix.
* ``chefsi``         -- Chebyshev-filtered subspace iteration (Alg. CheFSI)
  with Lanczos upper bound, Cholesky-QR and Rayleigh-Ritz.
* ``alb``            -- restriction to the element and SVD truncation (the
  ALB functions, Sec. II.A.1).
* ``dg``             -- interior-penalty DG Hamiltonian blocks (Eq.
  DGHamiltonian) and the dense assembled matrix (Eq. DGEigenvalue).
* ``grad``           -- Fermi-smeared band energy and its Hellmann-Feynman
  gradient (the local analogue of Eq. hfforce).
* ``dg_solve``       -- eigenpairs of the assembled DG Hamiltonian (Eq.
  DGEigenvalue) by CheFSI applied block by block, and the DG electron density
  (the next steps of the method).
* ``lobpcg``         -- LOBPCG with the Teter preconditioner (Alg. LOBPCG, Eqs. 3-5), the
  paper's default local solver, as a second route to the same eigenpairs.
* ``driver``         -- all of the above over every element of a workload.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
brute force and finite differences.  Parity unpinned: the Chebyshev filter's
bound heuristics (Lanczos step count, lower bound from the largest Ritz
value) only change iteration counts, not the converged result.
"""
from . import local_operator, chefsi, alb, dg, grad, driver, dg_solve, lobpcg  # noqa: F401
