"""Pins of the oracle's Galerkin hierarchy, Lanczos estimate and Cholesky (Sections 1, 4, 6)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.hierarchy import (NotSPDError, Params, block_pattern, build_hierarchy, cholesky_lower,
                              cholesky_solve, galerkin, lanczos_lmax)
from oracle.rtree import rtree_partition
from oracle.transfer import prolongation_fine


def test_galerkin_pprime0_closed_form():
    """p' = 0: A_1[B, B'] = sum_{i in B, j in B'} A_ij."""
    P = W.poisson(2, 6, 2, perturb=0.1, seed=1)
    A = P.scipy()
    part = rtree_partition(P.coords, 20, 2)
    Ac = galerkin(A, prolongation_fine(P.coords, part, 0)).toarray()
    nb = part.nboxes(1)
    ref = np.zeros((nb, nb))
    Ad = A.toarray()
    box = part.box_of_point[1]
    for i in range(P.n):
        for j in range(P.n):
            ref[box[i], box[j]] += Ad[i, j]
    assert np.allclose(Ac, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("d,pp,L", [(2, 1, 3), (2, 2, 3), (3, 1, 3), (3, 2, 2)])
def test_levels_symmetric_spd_and_pattern(d, pp, L):
    P = W.poisson(d, 8 if d == 2 else 3, 2 if d == 2 else 3, perturb=0.2, seed=2)
    H = build_hierarchy(P.coords, P.scipy(), Params(32 if d == 2 else 64, pp, L))
    b = (pp + 1) ** d
    for lev in range(1, L):
        Ad = H.A[lev].toarray()
        assert np.max(np.abs(Ad - Ad.T)) <= 1e-13 * np.abs(Ad).max()
        assert np.linalg.eigvalsh(Ad)[0] > 0
        # values only inside the structural block pattern, and every pattern block is hit
        nb = Ad.shape[0] // b
        mask = np.zeros((nb, nb), bool)
        for B, nbrs in enumerate(H.patterns[lev]):
            mask[B, nbrs] = True
        blocks = np.abs(Ad.reshape(nb, b, nb, b)).max(axis=(1, 3))
        assert not np.any((blocks > 0) & ~mask)
        assert np.all(mask == mask.T)


def test_cholesky_reconstructs():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((40, 40)); M = M @ M.T + 40 * np.eye(40)
    L = cholesky_lower(M)
    assert np.allclose(np.triu(L, 1), 0) and np.all(np.diag(L) > 0)
    assert np.allclose(L @ L.T, M, rtol=1e-14, atol=1e-12)
    r = rng.standard_normal(40)
    z = cholesky_solve(L, r)
    assert np.linalg.norm(M @ z - r) <= 1e-13 * np.linalg.norm(r) * np.linalg.cond(M)
    with pytest.raises(NotSPDError):
        cholesky_lower(np.diag([1.0, -1.0]))


def test_lanczos_estimate_bounds():
    P = W.poisson(2, 8, 2, perturb=0.1, seed=4)
    A = P.scipy()
    dinv = 1 / A.diagonal()
    Ad = A.toarray()
    lam = np.linalg.eigvalsh(np.sqrt(dinv)[:, None] * Ad * np.sqrt(dinv)[None, :])
    est = lanczos_lmax(A, 10, 1)
    assert est <= lam[-1] * (1 + 1e-12) and est > 0.9 * lam[-1]
    assert abs(lanczos_lmax(A, A.shape[0], 1) - lam[-1]) < 1e-8 * lam[-1]
    # tiny system: the Krylov space is exhausted early, estimate is exact
    T = sp.csr_matrix(np.array([[2.0, -1, 0], [-1, 2, -1], [0, -1, 2]]))
    ex = np.linalg.eigvalsh(np.array([[2.0, -1, 0], [-1, 2, -1], [0, -1, 2]]) / 2)[-1]
    assert abs(lanczos_lmax(T, 10, 9) - ex) < 1e-12
