"""GB300-native deflated block-Jacobi Schur-complement GMRES for the SMPM
Poisson-Neumann and per-Fourier-mode Helmholtz problems (Joshi, Thomsen &
Diamessis, arXiv:1512.01756).

The solver lives in the C-ABI library ``libsmpm.so`` (CUDA sm_103a kernels plus
a C++ host runtime, sources in ``csrc/``, API in ``include/smpm.h``).  The
Python module ``smpm`` is a thin ctypes binding with the same entry-point
names; ``inputs`` holds the seeded synthetic input recipes.
"""
