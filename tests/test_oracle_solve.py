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


def test_fcg_condition_estimate_is_pcg_estimate():
    """With a fixed SPD preconditioner flexible CG is PCG: its alphas and negated betas give the
    same Lanczos tridiagonal, so both estimates agree (and match the dense spectrum of M^{-1}A
    as pinned above)."""
    P, H = _small_hierarchy(3)
    A = H.A[0]
    rp = pcg(A, P.b, lambda r: vcycle(H, r), rtol=1e-12, maxit=200)
    rf = fcg(A, P.b, lambda r: vcycle(H, r), rtol=1e-12, maxit=200)
    assert rp.iterations == rf.iterations
    assert abs(rf.cond_estimate - rp.cond_estimate) <= 1e-6 * rp.cond_estimate
    M = np.stack([vcycle(H, e) for e in np.eye(P.n)], 1)
    ev = np.sort(np.linalg.eigvals(M @ A.toarray()).real)
    # Ritz values lie inside the spectrum: the estimate never exceeds the true condition number
    assert rf.cond_estimate <= ev[-1] / ev[0] * (1 + 1e-9)
    assert rf.cond_estimate > 0.95 * ev[-1] / ev[0]


@pytest.mark.parametrize("solver", [pcg, fcg])
def test_paper_stop_rule_stops_at_first_admissible_iterate(solver):
    """Section 6's rule (absolute residual < atol or a `reduction` drop of the initial residual)
    stops at the first iterate that meets either part; the iterates before it are those of a run
    that never stops early (same arithmetic), so the stopping index is read off that run."""
    P, H = _small_hierarchy(3)
    A = H.A[0]
    ref = solver(A, P.b, lambda r: vcycle(H, r), rtol=0.0, maxit=25)   # never stops early
    bnorm = np.linalg.norm(P.b)
    res = np.array(ref.history) * bnorm             # ||r_k||, k = 0, 1, ...
    for atol, red in [(1e-9, 1e-6), (0.0, 1e-3), (res[4] * 1.0000001, 0.0), (1e-30, 1e-30)]:
        thr = max(atol, red * res[0])
        want = next((k for k in range(len(res)) if res[k] <= thr), None)
        out = solver(A, P.b, lambda r: vcycle(H, r), rtol=0.0, maxit=25, atol=atol, reduction=red)
        if want is None:
            assert not out.converged and out.iterations == 25
        else:
            assert out.converged and out.iterations == want
            assert np.array_equal(out.history, ref.history[:want + 1])


def test_float32_vcycle_rounds_every_step():
    """as_precision(H, float32): every operator in single precision, so the V-cycle returns
    float32, differs from the FP64 V-cycle at the single-precision level (relative 1e-7..1e-4,
    never 0) and float64 gives the FP64 V-cycle bit for bit."""
    from oracle.solve import as_precision
    P, H = _small_hierarchy(3)
    r = np.random.default_rng(4).standard_normal(P.n)
    z64 = vcycle(H, r)
    assert np.array_equal(vcycle(as_precision(H, np.float64), r), z64)
    z32 = vcycle(as_precision(H, np.float32), r.astype(np.float32))
    assert z32.dtype == np.float32
    err = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
    assert 1e-8 < err < 1e-4, err
    assert as_precision(H, np.float32).A[0].dtype == np.float32 and H.A[0].dtype == np.float64


def test_threaded_products_give_the_same_bits():
    """The all-core evaluation (row blocks on a thread pool) forms every row sum as the serial
    product does: V-cycle and PCG give identical bits."""
    from oracle.parallel import threaded
    P, H = _small_hierarchy(3)
    A = H.A[0]
    Hp, Ap = threaded(H, A, 3)
    r = np.random.default_rng(8).standard_normal(P.n)
    assert np.array_equal(vcycle(Hp, r), vcycle(H, r))
    a = pcg(A, P.b, lambda v: vcycle(H, v), rtol=1e-10)
    b = pcg(Ap, P.b, lambda v: vcycle(Hp, v), rtol=1e-10)
    assert a.iterations == b.iterations and np.array_equal(a.x, b.x)
