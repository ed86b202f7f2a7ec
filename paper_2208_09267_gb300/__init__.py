"""GB300 (sm_103a) solver for the consistent lattice Boltzmann scheme of the
volume averaged Navier-Stokes equations (Bukreev et al., arXiv 2208.09267).

Modules:
  lbm     -- ctypes binding of the C ABI in include/lbm_vanse.h (the solver,
             single lattices and batches of lattices)
  build   -- in-tree nvcc build of liblbm_vanse.so
  tune    -- autotuner of the step kernels' launch variants, cached per size
             bucket and read by lbm, the batch and the server
  serve   -- continuous-batching request loop
  inputs  -- seeded synthetic input fields (no method arithmetic)

Importing the package loads nothing; the shared library is loaded on first
use and every solver call fails loudly if it cannot be.
"""
__all__ = ["lbm", "build", "inputs", "serve", "tune"]
