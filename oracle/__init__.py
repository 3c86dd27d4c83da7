"""CPU FP64 oracle for factorized CG / BiCGSTAB on A X + X B = C1 C2^T.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
CUDA library (``paper_2605_28274_gb300``) shares no code with it: no kernels,
no helpers, no constants; the two meet only through the seeded inputs of
``workloads``.

Plain, slow and readable on purpose: numpy/scipy in float64, every function
following one passage of the paper (Satake, Fukaya, Sogabe, Zhang,
"Factorized Krylov subspace methods for solving large Sylvester equations"):

* ``matrix_oriented``: Algorithms 2.1 (CG) and 2.2 (BiCGSTAB) on the full
  n x m iterate (the plain definition the factorized methods must reproduce,
  Sec. 5.1).
* ``factorized``: thin QR, block Lanczos / block Arnoldi (eq. 3.4 relation),
  the factored Sylvester operator (eq. 3.7), Algorithms 4.1 and 4.2 and the
  Lyapunov specialisation of Sec. 4.3.
* ``exact``: Bartels-Stewart (library), Kronecker solve, closed forms.
* ``residual``: the true residual ||C1 C2^T - A X - X B||_F, directly and in
  factored form.

Parity status: every function here is pinned by a test in
``tests/test_oracle_pins.py`` against closed forms, library routines,
invariants or brute force; none is "parity unpinned".
"""
from . import exact, factorized, matrix_oriented, residual  # noqa: F401
