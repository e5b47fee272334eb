"""GB300-native (sm_103a) Lagrangian large-deformation lattice Boltzmann solver.

The solver itself lives in the C-ABI shared library built from ``csrc/``; the
Python module :mod:`paper_2208_13769_gb300.lbm` binds it through ctypes.
Importing the package does not load the library (so that the seeded input
generators in :mod:`paper_2208_13769_gb300.workloads` work on machines
without a GPU).
"""
__all__ = ["workloads", "lbm"]
