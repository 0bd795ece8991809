"""CPU oracle for the SMPM Poisson/Helmholtz Schur-complement method (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.  It shares no code with the CUDA library; the only
module both sides use is the seeded input generator, which holds none of the
method's arithmetic.

Modules
-------
``lgl``       Gauss-Lobatto-Legendre nodes, weights, differentiation matrix (Sec. 2.2).
``smpm``      Grid geometry and explicit node-by-node assembly of the SMPM operator L
              (Eq. smpm_poisson), its strip split L = A + E B (Sec. 2.3) and the
              direct (dense) solve used on tiny grids.
``schur``     Schur complement S = I + B A^-1 E, null vectors (Claims 1-2), Alg. schur.
``dbj``       Block-Jacobi + deflation GMRES on the Schur system (Sec. 3, Alg. seq),
              Householder-Arnoldi GMRES (Sec. 3.1).
``fourier``   3-D y-periodic extension through per-mode Helmholtz solves (Sec. 5, Alg. 3d).
"""
