"""GB300-native projection solve of the low Mach number method (arXiv 1910.12979).

The solve  div((beta0/rho) grad phi) = div(beta0 U) - beta0 S  (Eq. 6, with the
base state frozen) by geometric multigrid, MAC and nodal projections, FP64 or
mixed precision, behind the C ABI of include/mg.h (libmgproj.so).  This package
is the thin Python binding: ``native`` wraps the C entry points one to one,
``solver`` adds a torch-tensor convenience class.
"""
from . import native  # noqa: F401
from .solver import ProjectionSolver, project_batch, solve_batch  # noqa: F401

__all__ = ["native", "ProjectionSolver", "project_batch", "solve_batch"]
