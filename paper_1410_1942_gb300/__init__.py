"""GB300-native (sm_103a) variable-coefficient pressure Poisson solver.

The solve of ``div((1/rho) grad p) = s`` from the pressure projection of a Cartesian-grid
two-phase ship-wave method (Formulation, eq. (pois); Numerical Time Integration), by
preconditioned conjugate gradients in hand-written CUDA behind the C ABI of ``include/poisson.h``.

``paper_1410_1942_gb300.capi`` is the thin ctypes binding to ``libpoisson.so``;
``paper_1410_1942_gb300.inputs`` makes the seeded synthetic fields.  Importing the package does not
load the CUDA library; the binding loads it on first use and raises if it is missing.
"""
