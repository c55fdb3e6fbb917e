"""Chebyshev-Jacobi smoother, V-cycle preconditioner, PCG and flexible CG.

Section 4 / Section 6: one V-cycle of the agglomerated hierarchy is the
preconditioner of the conjugate gradient method; the smoother is the
Chebyshev acceleration of Jacobi (Section 5, Remark on the smoother;
Section 6) with 2 pre- and 2 post-smoothing steps.

Chebyshev recurrence (Saad, Iterative Methods for Sparse Linear Systems,
2nd ed., Algorithm 12.1, preconditioned by D^{-1}) for the interval
[lam_lo, lam_hi] of D^{-1} A:
    theta = (hi + lo)/2, delta = (hi - lo)/2, sigma = theta/delta
    r = b - A x;  d = D^{-1} r / theta;  rho = 1/sigma
    repeat k-1 times:
        x += d;  r -= A d;  rho' = 1/(2 sigma - rho)
        d = rho' rho d + (2 rho'/delta) D^{-1} r;  rho = rho'
    x += d
Reading taken: one smoothing "step" of the paper is one such degree-k
sweep; pre- and post-smoothing use the same polynomial, so the V-cycle is
a symmetric operator.  The coarsest level is solved exactly (Cholesky).
"""
from dataclasses import dataclass

import numpy as np

from .hierarchy import cholesky_solve


def chebyshev_sweep(A, dinv, b, x, lam, k):
    lo, hi = lam
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    x = x.copy()
    r = b - A @ x
    d = dinv * r / theta
    rho = 1.0 / sigma
    for _ in range(k - 1):
        x = x + d
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x + d


def vcycle(H, r, level: int = 0):
    """z = M^{-1} r: one V-cycle of the hierarchy H applied at `level` to right-hand side r."""
    prm = H.params
    if level == prm.levels - 1:
        return cholesky_solve(H.Lc, r)
    A, dinv, lam = H.A[level], H.dinv[level], H.lam[level]
    x = np.zeros_like(r)
    for _ in range(prm.sweeps):
        x = chebyshev_sweep(A, dinv, r, x, lam, prm.cheb_degree)
    res = r - A @ x
    P = H.P[level]
    e = vcycle(H, P.T @ res, level + 1)
    x = x + P @ e
    for _ in range(prm.sweeps):
        x = chebyshev_sweep(A, dinv, r, x, lam, prm.cheb_degree)
    return x


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    relres: float
    converged: bool
    history: list
    cond_estimate: float


def _cond_from_cg(alphas, betas):
    k = len(alphas)
    if k == 0:
        return 1.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


def pcg(A, b, precond, rtol=1e-8, maxit=500, x0=None):
    """Preconditioned CG (Hestenes-Stiefel).  Stops when ||r||_2 <= rtol ||b||_2.

    Iterations = number of completed updates of x.  The condition estimate
    (the "Cond." column of the paper's tables) is the ratio of extreme
    eigenvalues of the Lanczos tridiagonal built from the CG coefficients.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    bnorm = float(np.linalg.norm(b))
    r = b - A @ x
    hist = [float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0]
    if bnorm == 0.0 or hist[0] <= rtol:
        return PCGResult(x, 0, hist[0], True, hist, 1.0)
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    for it in range(1, maxit + 1):
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            raise ArithmeticError("PCG breakdown: p^T A p <= 0")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        alphas.append(alpha)
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if rel <= rtol:
            return PCGResult(x, it, rel, True, hist, _cond_from_cg(alphas, betas))
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    return PCGResult(x, maxit, hist[-1], False, hist, _cond_from_cg(alphas, betas))


def fcg(A, b, precond, rtol=1e-8, maxit=500, x0=None):
    """Flexible CG with one retained direction (Notay, SIAM J. Sci. Comput. 22, 2000).

    p_0 = z_0;  alpha_k = p_k^T r_k / p_k^T A p_k;  x += alpha p;  r -= alpha A p;
    z = M(r);  p_{k+1} = z - (z^T A p_k / p_k^T A p_k) p_k.
    With a fixed SPD preconditioner this equals PCG in exact arithmetic; it
    stays convergent when M varies slightly (a lower-precision V-cycle).
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    bnorm = float(np.linalg.norm(b))
    r = b - A @ x
    hist = [float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0]
    if bnorm == 0.0 or hist[0] <= rtol:
        return PCGResult(x, 0, hist[0], True, hist, 1.0)
    p = precond(r)
    for it in range(1, maxit + 1):
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            raise ArithmeticError("FCG breakdown: p^T A p <= 0")
        alpha = float(p @ r) / pq
        x = x + alpha * p
        r = r - alpha * q
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if rel <= rtol:
            return PCGResult(x, it, rel, True, hist, float("nan"))
        z = precond(r)
        beta = float(z @ q) / pq
        p = z - beta * p
    return PCGResult(x, maxit, hist[-1], False, hist, float("nan"))
