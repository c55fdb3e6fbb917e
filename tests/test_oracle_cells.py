"""Cell-based agglomeration in the oracle (Section 4): an R-tree over cells, then first-come
ownership of the support points by the agglomerates in their listed order.

Pins: a hand-worked 4x4 example (tests/golden/cells_q1_4x4.txt); the ownership rule checked by
brute force (each point's owner is the first agglomerate, in order, with a cell holding it);
owned points inside their boxes and nested boxes; polynomial reproduction and the
piecewise-constant (p' = 0) Galerkin sum rule on a cell-based hierarchy; the V-cycle symmetry.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.hierarchy import Params
from oracle.rtree import cell_partition

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cells_q1_4x4.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out[k] = np.array([float(t) for t in v])
    return out


def test_hand_example():
    P = W.poisson(2, 4, 1)
    ptr, pts = W.cells(2, 4, 1)
    part = cell_partition(P.coords, ptr, pts, 4, 2)
    g = _golden()
    assert part.depth == 2
    assert np.array_equal(part.box_of_point[1], g["owner"].astype(np.int64))
    assert np.array_equal(part.mbr_lo[1].ravel(), g["box_lo"])
    assert np.array_equal(part.mbr_hi[1].ravel(), g["box_hi"])


CASES = [(2, 8, 2, 0.2, 3, 4, 3), (2, 12, 1, 0.1, 4, 6, 3), (3, 4, 2, 0.2, 5, 4, 2), (3, 4, 1, 0.15, 6, 2, 3)]


@pytest.mark.parametrize("d,N,p,pert,seed,leaf,L", CASES)
def test_first_come_ownership_brute_force(d, N, p, pert, seed, leaf, L):
    P = W.poisson(d, N, p, perturb=pert, seed=seed)
    ptr, pts = W.cells(d, N, p)
    part = cell_partition(P.coords, ptr, pts, leaf, L)
    n1 = part.nboxes(1)
    # the rule on its definition: a point's owner is the first agglomerate, in the listed order,
    # that has a cell holding the point (cell sets from an independent loop restatement)
    owner = part.box_of_point[1]
    first = np.full(P.n, np.iinfo(np.int64).max)
    cell_agg = _cell_agglomerates(P.coords, ptr, pts, leaf, d)
    for c, K in cell_agg.items():
        for i in pts[ptr[c]:ptr[c + 1]]:
            if i >= 0:
                first[i] = min(first[i], K)
    assert np.array_equal(owner, first)
    # owned points inside their box on every level; boxes nest
    for lev in range(1, L):
        B = part.box_of_point[lev]
        assert np.all(P.coords >= part.mbr_lo[lev][B]) and np.all(P.coords <= part.mbr_hi[lev][B])
        if lev > 1:
            child_parent = np.arange(part.nboxes(lev - 1)) >> d
            assert np.all(part.mbr_lo[lev - 1] >= part.mbr_lo[lev][child_parent])
            assert np.all(part.mbr_hi[lev - 1] <= part.mbr_hi[lev][child_parent])
    # every point owned once, tree order groups points by owner
    assert np.array_equal(np.sort(part.perm), np.arange(P.n))
    assert np.all(np.diff(owner[part.perm]) >= 0)
    assert n1 == 1 << part.depth


def _cell_agglomerates(coords, ptr, pts, leaf, d):
    """Independent restatement of the cell bisection (loops, no shared helper): cell -> level-1
    agglomerate."""
    x = np.asarray(coords)
    cells = []
    lo = {}; hi = {}
    for c in range(len(ptr) - 1):
        q = [i for i in pts[ptr[c]:ptr[c + 1]] if i >= 0]
        if q:
            cells.append(c)
            lo[c] = x[q].min(axis=0); hi[c] = x[q].max(axis=0)
    D = 0
    while -(-len(cells) // (1 << D)) > leaf:
        D += 1
    nodes = [cells]
    for _ in range(D):
        nxt = []
        for S in nodes:
            mn = np.min([lo[c] for c in S], axis=0); mx = np.max([hi[c] for c in S], axis=0)
            ext = mx - mn
            a = 0
            for k in range(1, d):
                if ext[k] > ext[a]:
                    a = k
            def key(c):
                m = (lo[c] + hi[c]) / 2
                return tuple(m[(a + k) % d] for k in range(d)) + (c,)
            S2 = sorted(S, key=key)
            h = (len(S2) + 1) // 2
            nxt += [S2[:h], S2[h:]]
        nodes = nxt
    return {c: K for K, S in enumerate(nodes) for c in S}


@pytest.mark.parametrize("pp,leaf", [(1, 6), (2, 12)])
def test_polynomial_reproduction_cells(pp, leaf):
    P = W.poisson(2, 12, 2, perturb=0.2, seed=7)
    ptr, pts = W.cells(2, 12, 2)
    part = cell_partition(P.coords, ptr, pts, leaf, 3)
    P0 = O.prolongation_fine(P.coords, part, pp)
    nodes_all = []
    for B in range(part.nboxes(1)):
        nodes_all.append(O.coarse_nodes(part.mbr_lo[1][B], part.mbr_hi[1][B], pp))
    xi = np.concatenate(nodes_all)
    for ax in range(pp + 1):
        for ay in range(pp + 1):
            c = xi[:, 0] ** ax * xi[:, 1] ** ay
            f = P.coords[:, 0] ** ax * P.coords[:, 1] ** ay
            assert np.max(np.abs(P0 @ c - f)) <= 1e-13


def test_piecewise_constant_galerkin_cells():
    P = W.poisson(2, 10, 2, perturb=0.1, seed=8)
    ptr, pts = W.cells(2, 10, 2)
    A = P.scipy()
    H = O.build_hierarchy(P.coords, A, Params(8, 0, 3, cheb_degree=2), cells=(ptr, pts))
    own = H.part.box_of_point[1]
    nb = H.part.nboxes(1)
    ref = np.zeros((nb, nb))
    Ad = A.toarray()
    for i in range(P.n):
        for j in range(P.n):
            ref[own[i], own[j]] += Ad[i, j]
    assert np.max(np.abs(H.A[1].toarray() - ref)) <= 1e-12 * np.abs(ref).max()


def test_vcycle_symmetric_cells():
    P = W.poisson(3, 4, 2, perturb=0.2, seed=9)
    ptr, pts = W.cells(3, 4, 2)
    H = O.build_hierarchy(P.coords, P.scipy(), Params(4, 1, 2, cheb_degree=3), cells=(ptr, pts))
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(P.n), rng.standard_normal(P.n)
    a, b = O.vcycle(H, u) @ v, u @ O.vcycle(H, v)
    assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)
    # the preconditioned solve converges to the direct solution
    x = np.linalg.solve(P.scipy().toarray(), P.b)
    r = O.pcg(P.scipy(), P.b, lambda z: O.vcycle(H, z), rtol=1e-12)
    assert np.linalg.norm(r.x - x) <= 1e-9 * np.linalg.norm(x)
