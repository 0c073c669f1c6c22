"""GB300-native lattice Boltzmann stream-and-collide library (sm_103a).

The compute path is the C-ABI shared library built from ``csrc/`` (see
``include/lbm.h``); ``lbm`` is its thin ctypes binding and fails loudly when
the library has not been built.  ``workloads`` holds seeded input generators.
Import ``paper_1311_2404_gb300.lbm`` explicitly; importing the package alone
does not load the CUDA library.
"""
__all__ = ["lbm", "workloads"]
