"""FP64 CPU oracle for the explicit DOM transient step of the phonon BTE (arXiv 2306.14181).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU
baseline leg may import this package.  The product library never uses it, and the two share
no code: the oracle has its own quadrature (``oracle.quadrature``), its own step
(``oracle/bte_oracle.c``) and its own adjoint.
"""
from .oracle import Problem, build_oracle, load_oracle  # noqa: F401
from . import quadrature  # noqa: F401
