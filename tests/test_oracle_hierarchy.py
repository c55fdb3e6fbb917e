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
        # values only inside the structural block pattern (the exact pattern is pinned below)
        nb = Ad.shape[0] // b
        mask = np.zeros((nb, nb), bool)
        for B, nbrs in enumerate(H.patterns[lev]):
            mask[B, nbrs] = True
        blocks = np.abs(Ad.reshape(nb, b, nb, b)).max(axis=(1, 3))
        assert not np.any((blocks > 0) & ~mask)
        assert np.all(mask == mask.T)


@pytest.mark.parametrize("d,N,p,leaf,L", [(2, 8, 2, 32, 3), (2, 12, 1, 8, 4), (3, 3, 3, 64, 3), (3, 4, 2, 6, 4)])
def test_block_patterns_are_exact(d, N, p, leaf, L):
    """The block pattern of every level is exactly the set of box pairs with a structurally
    nonzero block of P^T A P: with p' = 0 (P the 0/1 box indicator, Section 1) and every stored
    entry of A set to 1, A_1[B, B'] counts the stored entries between B and B', and the coarser
    levels sum those of their children, so a block is > 0 iff the pair is adjacent.  The pattern
    must equal {blocks > 0} (no missing pair, no extra pair such as a neighbour's neighbour)."""
    P = W.poisson(d, N, p, perturb=0.2, seed=3)
    A = P.scipy().copy()
    A.data[:] = 1.0
    H = build_hierarchy(P.coords, A, Params(leaf, 0, L))
    for lev in range(1, L):
        nb = H.A[lev].shape[0]
        mask = np.zeros((nb, nb), bool)
        for B, nbrs in enumerate(H.patterns[lev]):
            mask[B, nbrs] = True
        blocks = H.A[lev].toarray()
        assert np.all(blocks >= 0)
        assert np.array_equal(mask, blocks > 0), lev
        if lev == 1:   # the counting reading itself, by brute force over the stored entries
            box = H.part.box_of_point[1]
            cnt = np.zeros((nb, nb))
            Ac = A.tocoo()
            np.add.at(cnt, (box[Ac.row], box[Ac.col]), 1.0)
            assert np.array_equal(cnt, blocks)


def test_mesh_stats_closed_forms():
    """h on unperturbed structured meshes is the cell diagonal sqrt(d)/N (opposite vertices of an
    interior cell are coupled; no two farther points share a cell); H on the hand-worked 2D
    R-tree example (tests/golden/rtree_hand_2d.txt): the leaves' MBRs have diagonals
    1.5 sqrt(2), sqrt(2), sqrt(2.5), sqrt(2.5), so H = 1.5 sqrt(2) with 2 levels; with 3 levels
    the coarsest box is the root, MBR [0, 4] x [0, 3.5], H = sqrt(16 + 12.25)."""
    from oracle.hierarchy import mesh_stats
    for d, N, p in [(2, 8, 1), (2, 6, 3), (3, 4, 2)]:
        P = W.poisson(d, N, p)
        part = rtree_partition(P.coords, 16, 2)
        st = mesh_stats(P.coords, P.scipy(), part)
        assert abs(st["h"] - np.sqrt(d) / N) <= 1e-15, (d, N, p, st["h"])
    pts = np.array([[0.0, 0.0], [4.0, 1.0], [1.0, 3.0], [2.0, 2.0], [3.0, 0.5], [0.5, 1.5], [3.5, 3.5],
                    [2.5, 1.0], [1.5, 0.2], [2.0, 3.0]])
    A = sp.csr_matrix(([1.0, 1.0], ([0, 3], [3, 0])), shape=(10, 10))   # couples points 0 and 3 only
    st2 = mesh_stats(pts, A, rtree_partition(pts, 3, 2))
    assert np.isclose(st2["H"], 1.5 * np.sqrt(2.0), rtol=1e-15, atol=0) and st2["h"] == np.sqrt(8.0)
    assert st2["H_over_h"] == st2["H"] / st2["h"]
    st3 = mesh_stats(pts, A, rtree_partition(pts, 3, 3))
    assert np.isclose(st3["H"], np.sqrt(16.0 + 12.25), rtol=1e-15, atol=0)


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
