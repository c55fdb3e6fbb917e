"""Pins of the oracle's transfer operators (Section 4; Section 5, partition-of-unity remark)."""
import numpy as np
import pytest

import workloads as W
from oracle.basis import gll_nodes01
from oracle.rtree import rtree_partition
from oracle.transfer import UnisolventError, coarse_nodes, prolongation_coarse, prolongation_fine


def _setup(d, pp, L, perturb=0.2):
    P = W.poisson(d, 6 if d == 2 else 3, 3, perturb=perturb, seed=11)
    leaf = 24 if d == 2 else 40
    part = rtree_partition(P.coords, leaf, L)
    return P, part


@pytest.mark.parametrize("d,pp", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_polynomial_reproduction(d, pp):
    """Every polynomial of per-axis degree <= p' is reproduced exactly by P_0 (proof of the
    two-level theorem uses this): P_0 applied to its box-nodal values gives its point values."""
    P, part = _setup(d, pp, 2)
    P0 = prolongation_fine(P.coords, part, pp).toarray()
    b = (pp + 1) ** d
    for alpha in np.ndindex(*([pp + 1] * d)):
        f = lambda y: np.prod(y ** np.array(alpha), axis=1)
        coef = np.concatenate([f(coarse_nodes(part.mbr_lo[1][B], part.mbr_hi[1][B], pp))
                               for B in range(part.nboxes(1))])
        assert coef.shape[0] == part.nboxes(1) * b
        assert np.allclose(P0 @ coef, f(P.coords), atol=1e-12)


@pytest.mark.parametrize("d,pp", [(2, 0), (2, 1), (3, 2)])
def test_partition_of_unity(d, pp):
    """Remark (partition of unity): sum over boxes and q of the coarse functions is 1 on the free DoFs."""
    P, part = _setup(d, pp, 2)
    P0 = prolongation_fine(P.coords, part, pp)
    assert np.allclose(P0 @ np.ones(P0.shape[1]), 1.0, atol=1e-13)


def test_pprime0_is_nicolaides_indicator():
    """p' = 0: P_0 is the 0/1 indicator of the box owning each point (Nicolaides space, Section 1)."""
    P, part = _setup(2, 0, 2)
    P0 = prolongation_fine(P.coords, part, 0).toarray()
    ind = np.zeros_like(P0)
    ind[np.arange(P.n), part.box_of_point[1]] = 1.0
    assert np.array_equal(P0, ind)


@pytest.mark.parametrize("d,pp", [(2, 1), (2, 2), (3, 1)])
def test_nestedness(d, pp):
    """Section 4: P_2 = P_0 P~_1 equals the direct interpolation of the level-2 box polynomials."""
    P, part = _setup(d, pp, 3)
    P0 = prolongation_fine(P.coords, part, pp)
    Pt = prolongation_coarse(part, 1, pp)
    comp = (P0 @ Pt).toarray()
    # direct: a partition whose level-1 boxes are the level-2 boxes of `part`
    direct = np.zeros_like(comp)
    b = (pp + 1) ** d
    from oracle.basis import box_basis
    for B in range(part.nboxes(2)):
        mem = part.perm[part.box_offsets[2][B]:part.box_offsets[2][B + 1]]
        direct[np.ix_(mem, B * b + np.arange(b))] = box_basis(P.coords[mem], part.mbr_lo[2][B], part.mbr_hi[2][B], pp)
    assert np.allclose(comp, direct, atol=1e-12)


def test_structural_pattern_kept():
    """Point on a GLL node line gives an exact zero value that stays in the stored pattern."""
    x = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, 0.5], [0.5, 0.0], [0.0, 0.5],
                  [1.0, 0.5], [0.5, 1.0]])
    part = rtree_partition(x, 9, 2)
    P0 = prolongation_fine(x, part, 2)
    assert P0.nnz == 9 * 9
    assert (P0.data == 0.0).sum() > 0


def test_unisolvent_errors():
    x = np.stack([np.linspace(0, 1, 20), np.zeros(20)], 1)   # collinear: zero extent in y
    part = rtree_partition(x, 20, 2)
    with pytest.raises(UnisolventError):
        prolongation_fine(x, part, 1)
    prolongation_fine(x, part, 0)
    # points on 2 x-lines only cannot carry degree 2 in x... (3 distinct x needed)
    x2 = np.array([[0, 0], [0, 1], [0, 0.5], [1, 0], [1, 1], [1, 0.5], [0, 0.2], [1, 0.7], [0, 0.9]], float)
    part2 = rtree_partition(x2, 9, 2)
    with pytest.raises(UnisolventError):
        prolongation_fine(x2, part2, 2)
