"""CPU oracle for the AVU-GSR hot path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package. It is a plain FP64 restatement of
the paper's Eq. 2 and Eq. 3 (aprod 1 / aprod 2) and of Paige & Saunders' LSQR,
and it shares no code with the CUDA library.

Pins (each checked by a CPU test, see ``tests/test_oracle_*.py``):
  aprod1/aprod2  - explicit dense A built independently from the packed rows,
                   the adjoint identity, hand-worked single-row fixture;
  colnorm2       - dense column sums of squares;
  lsqr           - dense QR least squares (LAPACK), planted x* from a
                   consistent b, scipy's independent LSQR iterates, the
                   normal-equation residual, monotone residual norms;
  variance       - diag((A^T A)^-1) on tiny fully converged systems;
  mlp            - FP64 finite differences (``oracle.mlp``).
"""
from .core import (  # noqa: F401
    build_oracle,
    n_unknowns,
    n_equations,
    aprod1,
    aprod2,
    colnorm2,
    lsqr,
)
