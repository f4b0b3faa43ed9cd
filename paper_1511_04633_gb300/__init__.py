"""GB300-native double-MRT thermal lattice Boltzmann solver (arXiv:1511.04633).

The compute path is the CUDA library ``libdmrt.so`` (sources in ``csrc/``,
ABI in ``include/dmrt.h``); ``dmrt`` is its ctypes binding.  ``inputs`` holds
the seeded synthetic input generators.  Importing the package does not load
the library; ``from paper_1511_04633_gb300 import dmrt`` does, and fails if
the library cannot be built or loaded.
"""

__version__ = "0.1.0"
