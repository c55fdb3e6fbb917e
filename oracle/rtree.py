"""Point-based agglomeration by a deterministic R-tree bisection.

Section 3 (Definition of an R-tree of order (m, M)) and Section 4 (point-based
agglomeration: an R-tree whose leaves are the fine support points; each
point is owned by exactly one box).  The paper builds its tree by R*-tree
insertion (Boost.Geometry) with M = 2m and skips the leaf level (Section 6).
Insertion heuristics are not reproducible between two codes, so this
reading replaces them by a bulk-loaded, balanced bisection tree that keeps
what the method needs: nested axis-aligned boxes, a fan-out of 2^d between
consecutive agglomerated levels (so H/h doubles per level, as in the
structured-mesh tables), and unique ownership of every point.

Rule (identical in the CUDA library's host code):
  D = smallest t >= 0 with ceil(n / 2^t) <= leaf_size.
  Every node above depth D is split in two:
    1. MBR of the node's points (exact min / max);
    2. axis a = argmax_a (max_a - min_a), ties to the smallest a;
    3. order the node's points by the key
       (x_a, x_{(a+1) mod d}, ..., x_{(a+d-1) mod d}, original index);
    4. left child = first ceil(|S|/2) points, right child = the rest.
  Level l (l = 1 .. L-1) agglomerates are the nodes at depth D - d (l-1),
  numbered left to right.  Level 0 is the fine level.
The permutation lists the points in final tree order (leaves left to right,
inside a leaf in the order of its parent's split key).
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Partition:
    n: int
    dim: int
    depth: int                   # D
    levels: int                  # L (fine level included)
    perm: np.ndarray             # perm[k] = original index of the k-th point in tree order
    box_offsets: list            # box_offsets[l] (l >= 1): start of each level-l box in tree order (nbox_l + 1)
    box_of_point: list           # box_of_point[l][i] for original i (l >= 1)
    mbr_lo: list                 # mbr_lo[l] (nbox_l, d)
    mbr_hi: list

    def nboxes(self, level: int) -> int:
        return len(self.box_offsets[level]) - 1


class DepthError(ValueError):
    pass


def tree_depth(n: int, leaf_size: int) -> int:
    t = 0
    while -(-n // (1 << t)) > leaf_size:
        t += 1
    return t


def _split_key_order(x: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Order of the points idx (original indices) by the split rule's key."""
    pts = x[idx]
    d = x.shape[1]
    ext = pts.max(axis=0) - pts.min(axis=0)
    a = int(np.argmax(ext))          # first maximum: ties go to the smallest axis
    keys = [idx] + [pts[:, (a + k) % d] for k in reversed(range(d))]
    # np.lexsort sorts by the LAST key first: primary x_a, then x_{a+1}, ..., then original index
    return idx[np.lexsort(keys)]


def rtree_partition(coords: np.ndarray, leaf_size: int, levels: int) -> Partition:
    x = np.ascontiguousarray(coords, dtype=np.float64)
    n, d = x.shape
    if levels < 2:
        raise ValueError("need at least two levels (fine + coarsest)")
    if leaf_size < 2 or n < 1:
        # leaf_size 1 would allow empty leaves (n < 2^D); every box must own a point
        raise ValueError("empty problem or leaf_size < 2")
    D = tree_depth(n, leaf_size)
    if D - d * (levels - 2) < 0:
        raise DepthError(f"tree depth {D} too shallow for {levels} levels in {d}D")
    # nodes at the current depth: list of index arrays, left to right
    nodes = [np.arange(n, dtype=np.int64)]
    for _ in range(D):
        nxt = []
        for idx in nodes:
            order = _split_key_order(x, idx)
            h = -(-len(order) // 2)
            nxt.append(order[:h])
            nxt.append(order[h:])
        nodes = nxt
    perm = np.concatenate(nodes) if nodes else np.zeros(0, np.int64)
    leaf_sizes = np.array([len(v) for v in nodes], np.int64)
    leaf_off = np.concatenate(([0], np.cumsum(leaf_sizes)))
    box_offsets, box_of_point, lo, hi = [None], [None], [None], [None]
    for lev in range(1, levels):
        stride = 1 << (d * (lev - 1))
        off = leaf_off[::stride]
        nb = len(off) - 1
        bop = np.empty(n, np.int64)
        blo = np.empty((nb, d)); bhi = np.empty((nb, d))
        for B in range(nb):
            members = perm[off[B]:off[B + 1]]
            bop[members] = B
            blo[B] = x[members].min(axis=0)
            bhi[B] = x[members].max(axis=0)
        box_offsets.append(off); box_of_point.append(bop); lo.append(blo); hi.append(bhi)
    return Partition(n, d, D, levels, perm, box_offsets, box_of_point, lo, hi)


# ---------------------------------------------------------------- cell-based agglomeration
def cell_mbrs(coords: np.ndarray, cell_ptr: np.ndarray, cell_pts: np.ndarray):
    """MBR of every cell from the coordinates of its support points that belong to the
    system (entries < 0 are eliminated points).  Returns (lo, hi, valid); cells without any
    point of the system are not valid and take no part in the agglomeration."""
    x = np.ascontiguousarray(coords, dtype=np.float64)
    nc = len(cell_ptr) - 1
    d = x.shape[1]
    lo = np.zeros((nc, d)); hi = np.zeros((nc, d))
    valid = np.zeros(nc, bool)
    for c in range(nc):
        pts = cell_pts[cell_ptr[c]:cell_ptr[c + 1]]
        pts = pts[pts >= 0]
        if len(pts) == 0:
            continue
        valid[c] = True
        lo[c] = x[pts].min(axis=0)
        hi[c] = x[pts].max(axis=0)
    return lo, hi, valid


def cell_partition(coords: np.ndarray, cell_ptr: np.ndarray, cell_pts: np.ndarray, leaf_size: int,
                   levels: int) -> Partition:
    """Cell-based agglomeration (Section 4): an R-tree whose leaves are the cells' MBRs, then
    unique ownership of the support points by the agglomerates in the order they are listed.

    Tree: the bisection rule of rtree_partition applied to cells, with
      * the node MBR = union of its cells' MBRs (axis of longest extent, ties to the smaller axis),
      * the split key of a cell = (m_a, m_{a+1}, ..., cell index), m = its MBR centre (lo + hi) / 2,
      * D = smallest t with ceil(ncells / 2^t) <= leaf_size (leaf_size counts cells).
    Level-l agglomerates are the nodes at depth D - d (l - 1), left to right; the box B_K of an
    agglomerate is the union of its cells' MBRs.
    Ownership (the three-step procedure of Section 4): the level-1 agglomerates are visited in
    order; each takes every support point of its cells that no earlier agglomerate took.  A
    point's level-l agglomerate is the level-l ancestor of its level-1 owner (the spaces nest).
    Points are listed in tree order by (level-1 owner, original index).
    """
    x = np.ascontiguousarray(coords, dtype=np.float64)
    n, d = x.shape
    if levels < 2:
        raise ValueError("need at least two levels (fine + coarsest)")
    clo, chi, valid = cell_mbrs(x, cell_ptr, cell_pts)
    cells = np.nonzero(valid)[0].astype(np.int64)
    ncv = len(cells)
    if leaf_size < 2 or ncv < 1:
        # leaf_size 1 would allow empty agglomerates (ncells < 2^D)
        raise ValueError("no cells with points of the system, or leaf_size < 2")
    D = tree_depth(ncv, leaf_size)
    if D - d * (levels - 2) < 0:
        raise DepthError(f"tree depth {D} too shallow for {levels} levels in {d}D")
    centre = 0.5 * (clo + chi)
    nodes = [cells]
    for _ in range(D):
        nxt = []
        for idx in nodes:
            ext = chi[idx].max(axis=0) - clo[idx].min(axis=0)
            a = int(np.argmax(ext))
            keys = [idx] + [centre[idx, (a + k) % d] for k in reversed(range(d))]
            order = idx[np.lexsort(keys)]
            h = -(-len(order) // 2)
            nxt.append(order[:h])
            nxt.append(order[h:])
        nodes = nxt
    # level-1 agglomerates = the nodes at depth D; first-come ownership of the points
    owner = np.full(n, -1, np.int64)
    for K, cl in enumerate(nodes):
        for c in cl:
            pts = cell_pts[cell_ptr[c]:cell_ptr[c + 1]]
            for i in pts:
                if i >= 0 and owner[i] < 0:
                    owner[i] = K
    if np.any(owner < 0):
        raise ValueError("a support point belongs to no cell")
    n1 = len(nodes)
    perm = np.lexsort((np.arange(n), owner)).astype(np.int64)
    counts1 = np.bincount(owner, minlength=n1)
    box_offsets, box_of_point, lo, hi = [None], [None], [None], [None]
    for lev in range(1, levels):
        shift = d * (lev - 1)
        nb = n1 >> shift
        bop = owner >> shift
        cnt = counts1.reshape(nb, 1 << shift).sum(axis=1)
        off = np.concatenate(([0], np.cumsum(cnt))).astype(np.int64)
        blo = np.empty((nb, d)); bhi = np.empty((nb, d))
        for B in range(nb):
            members = np.concatenate(nodes[B << shift:(B + 1) << shift])
            blo[B] = clo[members].min(axis=0)
            bhi[B] = chi[members].max(axis=0)
        box_offsets.append(off); box_of_point.append(bop); lo.append(blo); hi.append(bhi)
    return Partition(n, d, D, levels, perm, box_offsets, box_of_point, lo, hi)
