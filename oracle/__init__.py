"""CPU FP64 oracle for the R-tree algebraic-geometric multilevel preconditioner.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
calls this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow restatement of the method of the paper
"R3MG-C: a high-order algebraic-geometric multilevel preconditioner for
continuous finite element discretizations", written from the paper and
sharing no code, table or constant generator with the CUDA library:

  rtree.py      point-based agglomeration by a deterministic R-tree
                bisection (Section 3, Definition of the R-tree; Section 4,
                point-based agglomeration)
  basis.py      GLL nodes and the tensor Q^{p'} Lagrange basis on a box
                (Section 4; Section 5, eq. (localinterpolation))
  transfer.py   fine-to-level-1 prolongation P and inter-level P~ (Section 4)
  hierarchy.py  Galerkin operators A_{l+1} = P^T A_l P, diagonal, Lanczos
                eigenvalue estimate, coarsest Cholesky, the tables' H and h
                (Sections 1, 4, 6)
  solve.py      Chebyshev-Jacobi smoother, V-cycle (FP64, or FP32 for the
                mixed-precision path), PCG and flexible CG with their
                condition estimates and stop tests (Section 4; Section 5,
                Remark on the smoother; Section 6)
  adjoint.py    gradient of a quadratic loss through the solve

Everything is float64 numpy/scipy.  A library primitive (sparse product,
sort, dense eigenvalues of a tiny tridiagonal) serves as a step where the
paper's definition is that primitive.  Where the paper is silent the
reading taken is stated in the function that takes it.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
a closed form, an invariant, a hand-worked example or a dense direct
computation; none is "parity unpinned".
"""
from .basis import gll_nodes01, lagrange_1d, box_basis
from .rtree import Partition, cell_partition, rtree_partition
from .transfer import prolongation_fine, prolongation_coarse, coarse_nodes
from .hierarchy import (Hierarchy, build_hierarchy, galerkin, block_pattern, lanczos_lmax, cholesky_lower, cholesky_solve,
                        mesh_stats)
from .solve import chebyshev_sweep, vcycle, pcg, fcg, PCGResult, as_precision
from .adjoint import solve_adjoint_grads
from .rng import splitmix64_uniform

__all__ = [
    "gll_nodes01", "lagrange_1d", "box_basis", "Partition", "rtree_partition", "cell_partition", "prolongation_fine",
    "prolongation_coarse", "coarse_nodes", "Hierarchy", "build_hierarchy", "galerkin", "block_pattern",
    "lanczos_lmax", "cholesky_lower", "cholesky_solve", "chebyshev_sweep", "vcycle", "pcg", "fcg", "PCGResult",
    "solve_adjoint_grads", "splitmix64_uniform", "mesh_stats", "as_precision",
]
