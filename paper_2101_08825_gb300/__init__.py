"""GB300 (sm_103a) implementation of the mollified nonlocal finite-element assembly of
Aulisa, Capodaglio, Chierici and D'Elia (arXiv 2101.08825): pair search and CSR pattern,
Algorithm 1 adaptive quadrature with the eps-mollifier, right-hand side with lifting and
Krylov solves, behind the C ABI of include/nl.h (libnl.so).

The Python layer (:mod:`.nl`) only marshals arguments; every step runs in the library's
CUDA kernels.
"""
from . import nl  # noqa: F401
from .build import build  # noqa: F401
