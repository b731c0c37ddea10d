"""GB300-native fourth-order entropy-stable vectorial lattice Boltzmann scheme.

The composite time step of Bellotti, Helluy and Navoret (arXiv 2403.13406)
as hand-written sm_103a CUDA kernels behind a C ABI (``include/eslbm.h``),
with a thin ctypes binding in :mod:`paper_2403_13406_gb300.eslbm`.

Importing the package does not load the CUDA library; the binding loads it
on first use and raises if it has not been built.
"""
__all__ = ["eslbm", "inputs"]
