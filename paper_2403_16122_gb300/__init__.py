"""GB300-native (sm_103a) time step of the phase-field lattice Boltzmann method
for freezing with volume change (arXiv 2403.16122).

The compute path is the CUDA library ``liblbmfreeze.so`` behind the C-ABI
declared in ``include/lbm.h``; :mod:`paper_2403_16122_gb300.lbm` is its thin
ctypes binding. :mod:`paper_2403_16122_gb300.inputs` states the seeded
synthetic workloads. Importing the package loads nothing; the binding loads
the library on first use and raises if it is missing.
"""
__all__ = ["inputs", "lbm"]
