"""B300-native (sm_103a) R-tree algebraic-geometric multilevel preconditioned CG.

Hot path: CG preconditioned by one V-cycle of the R-tree agglomerate
hierarchy (point- or cell-based agglomeration, box Q^{p'} prolongation, Galerkin
levels, Chebyshev-Jacobi smoothing, dense Cholesky on the coarsest level),
all inside libr3mg (``include/r3mg.h``).  This package is the thin Python
binding: ``Hierarchy`` (setup / vcycle / pcg / introspection),
``partition`` / ``partition_cells`` (host-only R-tree) and ``R3MGSolve`` (autograd).
"""
from ._lib import R3MGError, build as _build_lib, SO_PATH


def build(force: bool = False, verbose: bool = False) -> str:
    return _build_lib(force=force, verbose=verbose)


def __getattr__(name):
    if name in ("Hierarchy", "BatchHierarchy", "partition", "partition_cells", "group_rows", "default_params", "measure_fp64_rates",
                "wait_selftest"):
        from . import solver
        return getattr(solver, name)
    if name in ("R3MGSolve", "solve"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)


__all__ = ["build", "Hierarchy", "BatchHierarchy", "partition", "partition_cells", "group_rows", "default_params", "R3MGSolve", "solve", "R3MGError", "SO_PATH"]
