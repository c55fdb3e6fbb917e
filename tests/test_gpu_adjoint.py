"""Differentiation through the solve (adjoint + sampled outer product) on the GPU.

Checks: autograd gradients against the oracle's dense-solve gradient (1e-8 relative), against
central finite differences through the GPU solver itself (step 1e-6, 1e-6 relative, symmetric
perturbations since the solver requires a symmetric A), and the rebuild-on-new-values rule.
Workload: -div(kappa grad u) = 1 with kappa = exp(g), g a sum of 16 seeded Fourier modes.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle.adjoint import solve_adjoint_grads

pytestmark = pytest.mark.gpu


def _problem(dim=2, N=6, p=2):
    return W.poisson(dim, N, p, perturb=0.1, seed=31, kappa_modes=16, rhs="one")


def _solver(P, **kw):
    from paper_2607_28235_b300.autograd import R3MGSolver
    prm = dict(leaf_size=24, pprime=1, levels=3, rtol=1e-14)
    prm.update(kw)
    return R3MGSolver(P.coords, P.rowptr, P.colidx, P.vals, **prm)


def _loss_grads(S, P, ut):
    vals = torch.tensor(P.vals, device="cuda", requires_grad=True)
    b = torch.tensor(P.b, device="cuda", requires_grad=True)
    u = S.solve(vals, b)
    L = 0.5 * torch.sum((u - ut) ** 2)
    L.backward()
    return float(L.detach()), vals.grad.cpu().numpy(), b.grad.cpu().numpy(), u.detach().cpu().numpy()


@pytest.mark.parametrize("dim,N,p", [(2, 6, 2), (3, 3, 2)])
def test_gradients_match_oracle_dense(dim, N, p):
    P = _problem(dim, N, p)
    S = _solver(P, leaf_size=24 if dim == 2 else 30)
    ut_np = np.random.default_rng(2).standard_normal(P.n)
    ut = torch.tensor(ut_np, device="cuda")
    L, gv, gb, u = _loss_grads(S, P, ut)
    u_o, gb_o, gv_o = solve_adjoint_grads(P.rowptr, P.colidx, P.vals, P.b, lambda v: v - ut_np)
    assert np.linalg.norm(u - u_o) <= 1e-10 * np.linalg.norm(u_o)
    assert np.linalg.norm(gb - gb_o) <= 1e-8 * np.linalg.norm(gb_o)
    assert np.linalg.norm(gv - gv_o) <= 1e-8 * np.linalg.norm(gv_o)


def test_gradients_match_finite_differences():
    P = _problem(2, 6, 2)
    S = _solver(P)
    ut = torch.tensor(np.random.default_rng(4).standard_normal(P.n), device="cuda")
    L0, gv, gb, _ = _loss_grads(S, P, ut)
    h = 1e-6
    rows = np.repeat(np.arange(P.n), np.diff(P.rowptr))

    def loss_at(vals, b):
        with torch.no_grad():
            u = S.solve(torch.tensor(vals, device="cuda"), torch.tensor(b, device="cuda"))
            return float(0.5 * torch.sum((u - ut) ** 2))

    # right-hand side entries
    for i in np.argsort(-np.abs(gb))[:3]:
        e = np.zeros(P.n); e[i] = h
        fd = (loss_at(P.vals, P.b + e) - loss_at(P.vals, P.b - e)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * abs(gb[i])
    # matrix entries: symmetric pair (i, j) and (j, i) moved together
    key = {(int(rows[k]), int(P.colidx[k])): k for k in range(P.nnz)}
    off = [k for k in np.argsort(-np.abs(gv)) if rows[k] != P.colidx[k]][:2]
    diag = [k for k in np.argsort(-np.abs(gv)) if rows[k] == P.colidx[k]][:1]
    for k in off + diag:
        i, j = int(rows[k]), int(P.colidx[k])
        kt = key[(j, i)]
        E = np.zeros(P.nnz); E[k] += h
        if kt != k:
            E[kt] += h
        fd = (loss_at(P.vals + E, P.b) - loss_at(P.vals - E, P.b)) / (2 * h)
        an = gv[k] + (gv[kt] if kt != k else 0.0)
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)


def test_hierarchy_rebuilt_only_when_values_change():
    P = _problem(2, 6, 2)
    S = _solver(P)
    b = torch.tensor(P.b, device="cuda")
    v = torch.tensor(P.vals, device="cuda")
    S.solve(v, b)
    n0 = S.rebuilds
    S.solve(v, b)
    assert S.rebuilds == n0
    u2 = S.solve(v * 2.0, b)
    assert S.rebuilds == n0 + 1
    u1 = S.solve(v, b)
    assert torch.allclose(u2 * 2.0, u1, rtol=1e-10, atol=0)
