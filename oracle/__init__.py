"""Oracle for the coupled shell-cavity frequency sweep and its rational Arnoldi ROM.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, CPU FP64 restatement
of what the method computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path (``paper_2310_04734_gb300``) and neither
imports the other; both read their inputs from ``workloads``.

Modules
-------
fem   element matrices by isoparametric Gauss quadrature and global assembly
      (problem statement Sec. 2, Eq. 1-3; coupling matrix Eq. 5; complex
      stiffness Sec. 3.3 after Eq. 8).
fom   the full-order solution x(w) = A(w)^-1 f by dense GEPP and by a
      block-banded GEPP with pivoting across the stacked panel; receivers and
      SPL (Eq. 1, Eq. 8).
rom   rational Arnoldi Krylov bases (Eq. 9 second-order, Eq. 10 first-order),
      CGS2, Galerkin projection and the reduced sweep (Eq. 11), greedy choice of
      expansion points and the error measure of Sec. 3.3.
"""
