"""Pins of the oracle's R-tree bisection (Section 3, R-tree definition; Section 4, point-based agglomeration)."""
import os

import numpy as np
import pytest

from oracle.rtree import DepthError, rtree_partition, tree_depth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    pts, kv, mbr = [], {}, []
    mode = None
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line == "points":
            mode = "pts"; continue
        tok = line.split()
        if mode == "pts" and len(tok) == 3 and tok[0].isdigit():
            pts.append([float(tok[1]), float(tok[2])]); continue
        mode = None
        if tok[0] == "mbr":
            mbr.append([float(t) for t in tok[1:]])
        else:
            kv[tok[0]] = [float(t) if "." in t else int(t) for t in tok[1:]]
    return np.array(pts), kv, np.array(mbr)


def test_hand_worked_irregular():
    pts, kv, mbr = _read("rtree_hand_2d.txt")
    part = rtree_partition(pts, kv["leaf_size"][0], 2)
    assert part.depth == kv["depth"][0]
    assert part.perm.tolist() == kv["perm"]
    assert part.box_offsets[1].tolist() == kv["leaf_offsets"]
    assert np.array_equal(np.hstack([part.mbr_lo[1], part.mbr_hi[1]]), mbr)


def test_hand_worked_grid_tie():
    _, kv, _ = _read("rtree_grid_4x4.txt")
    i, j = np.meshgrid(np.arange(4.0), np.arange(4.0), indexing="xy")
    pts = np.stack([i.ravel(), j.ravel()], 1)     # index i + 4 j
    part = rtree_partition(pts, 4, 3)
    assert part.perm.tolist() == kv["perm"]
    assert part.box_offsets[1].tolist() == kv["leaf_offsets"]
    assert part.box_offsets[2].tolist() == [0, 16]


@pytest.mark.parametrize("n,d,leaf,L", [(1000, 2, 17, 3), (4097, 3, 64, 3), (777, 3, 5, 4), (64, 2, 64, 2)])
def test_invariants(n, d, leaf, L):
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, (n, d))
    x[::7] = x[3]        # duplicated points exercise the index tie-break
    part = rtree_partition(x, leaf, L)
    D = part.depth
    assert -(-n // (1 << D)) <= leaf and (D == 0 or -(-n // (1 << (D - 1))) > leaf)
    assert np.array_equal(np.sort(part.perm), np.arange(n))
    for lev in range(1, L):
        off = part.box_offsets[lev]
        sizes = np.diff(off)
        t = D - d * (lev - 1)
        assert set(sizes.tolist()) <= {n // (1 << t), -(-n // (1 << t))}
        for B in range(len(sizes)):
            mem = part.perm[off[B]:off[B + 1]]
            assert np.all(part.box_of_point[lev][mem] == B)
            assert np.all(x[mem] >= part.mbr_lo[lev][B]) and np.all(x[mem] <= part.mbr_hi[lev][B])
            assert np.all(x[mem].min(0) == part.mbr_lo[lev][B])
        if lev >= 2:
            fan = 1 << d
            for c in range(part.nboxes(lev - 1)):
                B = c // fan
                assert np.all(part.mbr_lo[lev - 1][c] >= part.mbr_lo[lev][B])
                assert np.all(part.mbr_hi[lev - 1][c] <= part.mbr_hi[lev][B])


def test_depth_error():
    x = np.random.default_rng(0).uniform(0, 1, (100, 3))
    assert tree_depth(100, 64) == 1
    with pytest.raises(DepthError):
        rtree_partition(x, 64, 3)


def test_order_independent_of_input_order():
    """The key is a total order, so any correct sort gives the same tree (up to relabelling)."""
    rng = np.random.default_rng(5)
    x = np.round(rng.uniform(0, 1, (500, 3)), 1)     # many coordinate ties
    part = rtree_partition(x, 20, 3)
    sh = rng.permutation(500)
    part2 = rtree_partition(x[sh], 20, 3)
    # boxes as sets of coordinates must agree where no two points are identical in all coordinates + index;
    # with exact duplicates the index decides, so compare box sizes and MBRs
    assert np.array_equal(part.box_offsets[1], part2.box_offsets[1])
    assert np.array_equal(part.mbr_lo[1], part2.mbr_lo[1]) and np.array_equal(part.mbr_hi[1], part2.mbr_hi[1])
