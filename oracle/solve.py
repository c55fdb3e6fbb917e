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
from dataclasses import dataclass, replace

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


def as_precision(H, dtype):
    """The hierarchy H with its operators (A_l, P_l, D_l^{-1}, the coarsest Cholesky factor)
    rounded to `dtype`.  With float32, ``vcycle`` on it runs every step in single precision
    with single-precision accumulation (numpy and scipy keep float32 operands in float32), which
    is the FP32 V-cycle of the mixed-precision solver: the benchmark spec fixes FP32 values,
    vectors and accumulation for the V-cycle inside an FP64 outer iteration.  The Chebyshev
    interval stays a pair of Python floats, rounded to `dtype` where it meets an array."""
    cast = lambda M: M.astype(dtype)
    return replace(H, A=[cast(A) for A in H.A], P=[cast(P) for P in H.P], dinv=[d.astype(dtype) for d in H.dinv],
                   Lc=H.Lc.astype(dtype))


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


def _threshold(rtol, bnorm, atol, reduction, r0norm):
    """Stop threshold on ||r||_2: max(rtol ||b||, atol, reduction ||r_0||).  atol = reduction = 0
    is the relative test of the workloads; rtol = 0, atol = 1e-9, reduction = 1e-6 is the rule
    of Section 6 (absolute residual below 1e-9, or six orders of reduction)."""
    return max(rtol * bnorm, atol, reduction * r0norm)


def pcg(A, b, precond, rtol=1e-8, maxit=500, x0=None, atol=0.0, reduction=0.0):
    """Preconditioned CG (Hestenes-Stiefel).  Stops when ||r||_2 <= max(rtol ||b||_2, atol,
    reduction ||r_0||_2) (by default the relative test ||r|| <= rtol ||b||).

    Iterations = number of completed updates of x.  The condition estimate
    (the "Cond." column of the paper's tables) is the ratio of extreme
    eigenvalues of the Lanczos tridiagonal built from the CG coefficients.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    bnorm = float(np.linalg.norm(b))
    r = b - A @ x
    r0norm = float(np.linalg.norm(r))
    thr = _threshold(rtol, bnorm, atol, reduction, r0norm)
    hist = [r0norm / bnorm if bnorm > 0 else 0.0]
    if bnorm == 0.0 or r0norm <= thr:
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
        rnorm = float(np.linalg.norm(r))
        rel = rnorm / bnorm
        hist.append(rel)
        if rnorm <= thr:
            return PCGResult(x, it, rel, True, hist, _cond_from_cg(alphas, betas))
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    return PCGResult(x, maxit, hist[-1], False, hist, _cond_from_cg(alphas, betas))


def fcg(A, b, precond, rtol=1e-8, maxit=500, x0=None, atol=0.0, reduction=0.0):
    """Flexible CG with one retained direction (Notay, SIAM J. Sci. Comput. 22, 2000).

    p_0 = z_0;  alpha_k = p_k^T r_k / p_k^T A p_k;  x += alpha p;  r -= alpha A p;
    z = M(r);  p_{k+1} = z - (z^T A p_k / p_k^T A p_k) p_k.
    With a fixed SPD preconditioner this equals PCG in exact arithmetic; it
    stays convergent when M varies slightly (a lower-precision V-cycle).
    In exact arithmetic with a fixed SPD M, z_{k+1}^T A p_k = -r_{k+1}^T z_{k+1} / alpha_k and
    p_k^T A p_k = r_k^T z_k / alpha_k, so the coefficient above is minus the PCG beta: the
    condition estimate takes the alphas and the negated coefficients as PCG's.
    Stop test as in ``pcg``.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    bnorm = float(np.linalg.norm(b))
    r = b - A @ x
    r0norm = float(np.linalg.norm(r))
    thr = _threshold(rtol, bnorm, atol, reduction, r0norm)
    hist = [r0norm / bnorm if bnorm > 0 else 0.0]
    if bnorm == 0.0 or r0norm <= thr:
        return PCGResult(x, 0, hist[0], True, hist, 1.0)
    p = precond(r)
    alphas, betas = [], []
    for it in range(1, maxit + 1):
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            raise ArithmeticError("FCG breakdown: p^T A p <= 0")
        alpha = float(p @ r) / pq
        x = x + alpha * p
        r = r - alpha * q
        alphas.append(alpha)
        rnorm = float(np.linalg.norm(r))
        rel = rnorm / bnorm
        hist.append(rel)
        if rnorm <= thr:
            return PCGResult(x, it, rel, True, hist, _cond_from_cg(alphas, betas))
        z = precond(r)
        beta = float(z @ q) / pq
        betas.append(-beta)
        p = z - beta * p
    return PCGResult(x, maxit, hist[-1], False, hist, _cond_from_cg(alphas, betas))
