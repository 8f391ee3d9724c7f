"""GB300-native entropy-limited lattice Boltzmann step (D1Q3 / D2Q9 LBGK).

The compute path is the CUDA library ``liblbm.so`` built from ``csrc/``;
``paper_0704_0043_gb300.lbm`` is a thin ctypes binding over its C ABI
(``include/lbm.h``).  Importing this package does not load the library; the
first use of ``lbm`` does, and raises if the library has not been built.
"""
