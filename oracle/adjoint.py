"""Gradient of a loss of the solution u = A^{-1} b with respect to b and to A's stored values.

For L(u) with g = dL/du and A symmetric, the adjoint lambda solves
A lambda = g; then dL/db = lambda and dL/dA_ij = -lambda_i u_j on every
stored entry (i, j) of A's pattern.  Here both solves are dense direct
solves (the oracle's definition; the GPU library reuses its multilevel
hierarchy and PCG for the adjoint solve).
"""
import numpy as np


def solve_adjoint_grads(rowptr, colidx, vals, b, g_of_u):
    """Returns (u, grad_b, grad_vals) for loss gradient function g_of_u(u) -> dL/du (dense solves)."""
    n = len(rowptr) - 1
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    A[rows, colidx] = vals
    u = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, g_of_u(u))
    grad_vals = -lam[rows] * u[colidx]
    return u, lam, grad_vals
