"""FP64 CPU oracle for the adaptive-conditioning conic solver (arXiv 2103.00736).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, readable restatement
of the paper's method used to check the CUDA library.  Only the test suite,
the smoke check and the CPU-baseline leg of the benchmark may import it; the
library itself never does, and this package never imports the library.  It
shares no code with the CUDA path: the only common dependency is the seeded
instance generator, which holds none of the method's arithmetic.

Contents
  cones     -- proj_K / abs_K of Definition 1 for products of Lorentz cones
  subspace  -- the subspace range(A_hat') and its reflection abs_A (Alg. 1, step 5)
  alg       -- Algorithm 1 and Algorithm 2 step by step, in FP64
  kkt       -- KKT residuals of the primal/dual pair (Eqs. 19a-19c)
  vertex    -- brute-force vertex enumeration for tiny LPs (ground truth)

Parity status of each function is stated in its docstring; every function
here is pinned by the not-gpu tests unless it says "parity unpinned".
"""
from . import cones, subspace, alg, kkt, vertex  # noqa: F401
