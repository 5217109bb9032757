"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only generates inputs (grids, coefficient fields, CSR matrices,
manufactured solutions).  It holds none of the solver method's arithmetic and
imports neither the oracle nor the CUDA library.
"""
from . import cd, configs, rng  # noqa: F401
from .cd import System  # noqa: F401
