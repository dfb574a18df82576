"""CPU FP64 oracle for the JFNK hot path (test infrastructure only).

This package is the independent reference that the CUDA library is checked
against. It is test infrastructure: only the tests, the smoke check and the
CPU-baseline leg of the benchmark import it; the library never calls it and
has no CPU fallback through it.

It is written from the paper ("Robust Matrix-Free Newton-Krylov Solvers via
Automatic Differentiation") in plain numpy, in float64, without blocking,
fusion or reordering beyond what each definition states:

* ``pdes``     discrete residuals G and the theta-method residual F
               (Eq. 2; App. A and the benchmark variants);
* ``jvp``      the Gateaux derivative (Eq. 6) by the complex step, the
               finite-difference quotient (Eq. 7) with both step rules (Eq. 8
               and the scaled rule), and the dense Jacobian;
* ``krylov``   restarted GMRES with classical Gram-Schmidt applied twice and
               Givens rotations, BiCGSTAB and CG (Sec. 2, Sec. 3.1);
* ``newton``   Newton with backtracking line search and the relative stopping
               test (Eqs. 4-5), time stepping and the Born start (Sec. 3.1).

Every function is pinned by tests/test_oracle_*.py against what the paper and
the mathematics fix (closed forms, Taylor remainders, manufactured solutions,
conservation, special cases reducing to library routines). It shares no code
with the CUDA path; both read inputs from ``synthetic_inputs`` only.
"""
from . import pdes, jvp, krylov, newton  # noqa: F401
