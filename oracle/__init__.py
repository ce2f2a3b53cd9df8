"""FP64 CPU oracle for the GridPull optimisation step (test infrastructure).

This package is the plain, slow reference that the CUDA path is checked
against.  It is test infrastructure only: the tests, the smoke check and the
benchmark's CPU-baseline leg use it; the library never imports it, and it
imports nothing from the library.  See ``oracle.gridpull`` for the functions
and the passage of the paper each one follows.
"""
from . import gridpull  # noqa: F401
