"""Input generator checks (FE model problem of Section 2; not the multilevel method)."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import workloads as W


def test_sizes_match_structured_counts():
    # free DoFs (N p - 1)^d; the totals (N p + 1)^d match the DoF counts quoted for structured meshes
    assert W.sizes(2, 32, 2)[0] == 63 ** 2
    assert W.sizes(3, 32, 3) == (857375, 101847563)
    assert W.sizes(3, 64, 3)[0] == 191 ** 3


@pytest.mark.parametrize("perturb", [0.0, 0.2])
def test_bitwise_symmetric_and_constant_kernel(perturb):
    P = W.poisson(3, 3, 2, perturb=perturb, seed=7)
    A = P.scipy()
    assert (A != A.T).nnz == 0
    # rows whose support touches no boundary node: constants are in the kernel of the stiffness form
    F = P.N * P.p - 1
    idx = np.arange(P.n)
    I = np.stack([idx % F, (idx // F) % F, idx // (F * F)], 1) + 1
    # coupling reaches at most p nodes away
    far = np.all((I > P.p) & (I < P.N * P.p - P.p), axis=1)
    rs = A @ np.ones(P.n)
    assert far.any()
    assert np.max(np.abs(rs[far])) < 1e-13 * np.max(np.abs(A.diagonal()))


def test_linear_patch_affine_mesh():
    # on an affine mesh a linear function is reproduced: A u_lin = 0 on rows away from the boundary
    P = W.poisson(2, 4, 3)
    A = P.scipy()
    u = 0.3 + 2.0 * P.coords[:, 0] - 1.5 * P.coords[:, 1]
    F = P.N * P.p - 1
    idx = np.arange(P.n)
    I = np.stack([idx % F, idx // F], 1) + 1
    far = np.all((I > P.p) & (I < P.N * P.p - P.p), axis=1)
    assert np.max(np.abs((A @ u)[far])) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fe_error_rate(p):
    errs = []
    for N in (4, 8, 16):
        P = W.poisson(2, N, p, perturb=0.15, seed=3)
        u = sla.spsolve(P.scipy().tocsc(), P.b)
        errs.append(W.l2_error(P, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.35, rates


def test_gll_fine_nodes():
    assert np.allclose(W.gll01(3), [0, (1 - 5 ** -0.5) / 2, (1 + 5 ** -0.5) / 2, 1], atol=1e-15)
