"""CPU oracle for the Laplace KIFMM hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from this package.
The CUDA library never depends on it, and it never depends on the CUDA
library: the two share no code, tables or constants.  Only the seeded input
generators (``paper_2303_08394_gb300.workloads``) feed both sides.

Contents
  direct   FP64 direct sum of Eq. (1), plain C with OpenMP (``direct.c``).
  kifmm    FP64 kernel-independent FMM with dense M2L, numpy, following the
           operator sequence of the "Fast Multipole Method" and
           "Computational structure of FMM operators" sections.

Parity status of each function is stated in its module header.
"""
