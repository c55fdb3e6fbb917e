"""Pins of the oracle's smoother, V-cycle, PCG, FCG and adjoint (Sections 4, 5, 6)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.adjoint import solve_adjoint_grads
from oracle.hierarchy import Params, build_hierarchy
from oracle.solve import chebyshev_sweep, fcg, pcg, vcycle


def _sym_eig(A, dinv):
    s = np.sqrt(dinv)
    lam, V = np.linalg.eigh(s[:, None] * A.toarray() * s[None, :])
    return lam, V, s


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_chebyshev_error_polynomial(k):
    """Error after one sweep = T_k((theta - lambda)/delta) / T_k(theta/delta) in the eigenbasis of D^{-1}A."""
    P = W.poisson(2, 5, 2, perturb=0.1, seed=5)
    A = P.scipy()
    dinv = 1 / A.diagonal()
    lam, V, s = _sym_eig(A, dinv)
    lo, hi = 0.1 * lam[-1], 1.05 * lam[-1]
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    rng = np.random.default_rng(k)
    xs = rng.standard_normal(P.n)
    b = A @ xs
    x0 = rng.standard_normal(P.n)
    x1 = chebyshev_sweep(A, dinv, b, x0, (lo, hi), k)
    T = np.polynomial.chebyshev.Chebyshev.basis(k)
    g = T((theta - lam) / delta) / T(theta / delta)
    # D^{1/2} e is propagated by V diag(g) V^T
    e0 = (x0 - xs) / s
    e1 = (x1 - xs) / s
    assert np.allclose(e1, V @ (g * (V.T @ e0)), atol=1e-11 * np.abs(e0).max())


def test_degree1_is_damped_jacobi():
    """k = 1: x += D^{-1} r / theta, damped Jacobi with omega = 1/theta (Section 5, R = omega D^{-1})."""
    P = W.poisson(2, 4, 2)
    A = P.scipy(); dinv = 1 / A.diagonal()
    x0 = np.random.default_rng(0).standard_normal(P.n)
    x1 = chebyshev_sweep(A, dinv, P.b, x0, (0.2, 1.8), 1)
    assert np.allclose(x1, x0 + dinv * (P.b - A @ x0) / 1.0, atol=1e-14)


def _small_hierarchy(L=2, pp=1, k=3):
    P = W.poisson(2, 6, 2, perturb=0.2, seed=8)
    H = build_hierarchy(P.coords, P.scipy(), Params(30, pp, L, cheb_degree=k))
    return P, H


def test_vcycle_symmetric():
    P, H = _small_hierarchy(3)
    M = np.stack([vcycle(H, e) for e in np.eye(P.n)], 1)
    assert np.max(np.abs(M - M.T)) <= 1e-13 * np.abs(M).max()
    assert np.linalg.eigvalsh((M + M.T) / 2)[0] > 0


def test_two_level_matches_textbook_operator():
    """L = 2: I - M^{-1}A = S (I - P A_c^{-1} P^T A) S with S the smoother's error polynomial
    (applied `sweeps` times), the two-grid error operator of the subspace-correction framework (Section 5)."""
    P, H = _small_hierarchy(2, 1, 3)
    A = H.A[0].toarray(); n = A.shape[0]
    dinv = H.dinv[0]
    lam, V, s = _sym_eig(H.A[0], dinv)
    lo, hi = H.lam[0]
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = np.polynomial.chebyshev.Chebyshev.basis(3)
    g = T((theta - lam) / delta) / T(theta / delta)
    S1 = (s[:, None] * (V * g) @ V.T) / s[None, :]        # error map of one sweep
    S = np.linalg.matrix_power(S1, H.params.sweeps)
    Pm = H.P[0].toarray()
    Ac = Pm.T @ A @ Pm
    E = S @ (np.eye(n) - Pm @ np.linalg.solve(Ac, Pm.T @ A)) @ S
    M = np.stack([vcycle(H, e) for e in np.eye(n)], 1)
    assert np.allclose(np.eye(n) - M @ A, E, atol=1e-11)


@pytest.mark.parametrize("d,p,pp,L", [(2, 2, 1, 3), (2, 3, 2, 2), (3, 2, 1, 2)])
def test_pcg_matches_direct_solve(d, p, pp, L):
    P = W.poisson(d, 8 if d == 2 else 3, p, perturb=0.2, seed=9)
    A = P.scipy()
    H = build_hierarchy(P.coords, A, Params(40, pp, L))
    res = pcg(A, P.b, lambda r: vcycle(H, r), rtol=1e-13)
    xd = np.linalg.solve(A.toarray(), P.b)
    assert res.converged
    assert np.linalg.norm(res.x - xd) <= 1e-10 * np.linalg.norm(xd)
    r2 = fcg(A, P.b, lambda r: vcycle(H, r), rtol=1e-13)
    assert abs(r2.iterations - res.iterations) <= 1
    assert np.linalg.norm(r2.x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_condition_estimate_matches_dense():
    P, H = _small_hierarchy(2)
    A = H.A[0]
    res = pcg(A, P.b, lambda r: vcycle(H, r), rtol=1e-14, maxit=200)
    M = np.stack([vcycle(H, e) for e in np.eye(P.n)], 1)
    ev = np.sort(np.linalg.eigvals(M @ A.toarray()).real)
    assert abs(res.cond_estimate - ev[-1] / ev[0]) < 0.05 * ev[-1] / ev[0]


def test_higher_pprime_fewer_iterations():
    """Qualitative trend of the structured-square tables: p' = 1 needs fewer iterations than p' = 0."""
    P = W.poisson(2, 16, 2)
    A = P.scipy()
    its = []
    for pp in (0, 1):
        H = build_hierarchy(P.coords, A, Params(64, pp, 2))
        its.append(pcg(A, P.b, lambda r: vcycle(H, r), rtol=1e-8).iterations)
    assert its[1] < its[0]


def test_adjoint_against_finite_differences():
    P = W.poisson(2, 3, 2, perturb=0.1, seed=6)
    ut = np.random.default_rng(1).standard_normal(P.n)
    loss = lambda u: 0.5 * np.sum((u - ut) ** 2)
    u, gb, gv = solve_adjoint_grads(P.rowptr, P.colidx, P.vals, P.b, lambda u: u - ut)
    A = P.scipy().toarray()
    h = 1e-6
    for i in [0, 3, P.n - 1]:
        e = np.zeros(P.n); e[i] = h
        fd = (loss(np.linalg.solve(A, P.b + e)) - loss(np.linalg.solve(A, P.b - e))) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * max(1, abs(gb[i]))
    rows = np.repeat(np.arange(P.n), np.diff(P.rowptr))
    for k in [0, 5, len(P.vals) // 2]:
        Ap = A.copy(); Am = A.copy()
        Ap[rows[k], P.colidx[k]] += h; Am[rows[k], P.colidx[k]] -= h
        fd = (loss(np.linalg.solve(Ap, P.b)) - loss(np.linalg.solve(Am, P.b))) / (2 * h)
        assert abs(fd - gv[k]) <= 1e-6 * max(1, abs(gv[k]))
