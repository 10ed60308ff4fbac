"""GB300-native (sm_103a) Hamilton-Jacobi level-set solver.

The hot path (Algorithm 1 of arXiv 2204.05520: upwind/ENO2 derivatives,
bang-bang optimal inputs, Lax-Friedrichs Hamiltonian with a grid-wide or
per-node alpha, CFL step, Euler / TVD-RK2 update, the BRT min and the
reach-avoid obstacle max) and the time-to-reach sweep (Algorithm 2) run in the
CUDA library ``libodp.so`` behind a C ABI (``include/odp.h``), with batched
and served modes.  ``odp`` is its thin ctypes binding; ``inputs`` holds the
seeded synthetic workloads.

Importing the package loads nothing; ``odp.load()`` (called by every binding
function) loads the library and raises if it is missing.
"""
