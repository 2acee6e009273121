"""GB300-native direct-summation N-body library (softened forces + Hermite-4
block time steps), hand-written sm_103a CUDA behind a C ABI.

Submodules (import them explicitly):
  ``paper_1411_5234_gb300.nbody``  -- ctypes binding of ``libnbody_gb300.so``;
  ``paper_1411_5234_gb300.build``  -- nvcc build of that library (sm_103a);
  ``paper_1411_5234_gb300.inputs`` -- seeded synthetic initial conditions.
Importing the package itself loads nothing, so the input generators work on
machines without a GPU; the binding raises when the library is missing.
"""
