"""C-ABI library checks that need no GPU: symbols, host R-tree bit-exactness, error codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2607_28235_b300 as R
from paper_2607_28235_b300 import _lib
from oracle.rtree import rtree_partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    R.build()
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "r3mg.h")).read()
    names = set(re.findall(r"\b(r3mg_[a-z_]+)\s*\(", hdr))
    assert len(names) >= 15
    raw = ctypes.CDLL(_lib.SO_PATH)
    for nm in sorted(names):
        assert hasattr(raw, nm), nm


def test_default_params(lib):
    p = R.default_params()
    assert p["cheb_degree"] == 3 and p["sweeps"] == 2 and p["lanczos_steps"] == 10
    assert p["eig_safety"] == 1.1 and p["eig_ratio"] == 30.0


@pytest.mark.parametrize("n,d,leaf,L,seed", [(1000, 2, 17, 3, 0), (4097, 3, 64, 3, 1), (777, 3, 5, 4, 2),
                                             (64, 2, 64, 2, 3), (5000, 3, 40, 3, 4), (3, 2, 2, 2, 5)])
def test_partition_bit_exact_vs_oracle(lib, n, d, leaf, L, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, d))
    x[::5] = np.round(x[::5], 1)        # coordinate ties exercise the secondary keys
    x[::11] = x[2]                      # full duplicates exercise the index tie-break
    perm, off, D = R.partition(x, leaf, L)
    part = rtree_partition(x, leaf, L)
    assert D == part.depth
    assert np.array_equal(perm, part.perm)
    assert np.array_equal(off, part.box_offsets[1] if L >= 2 else off)


def test_partition_fe_points(lib):
    import workloads as W
    P = W.poisson(3, 6, 3, perturb=0.2, seed=3)
    perm, off, D = R.partition(P.coords, 50, 3)
    part = rtree_partition(P.coords, 50, 3)
    assert np.array_equal(perm, part.perm) and np.array_equal(off, part.box_offsets[1])


def test_partition_hand_example(lib):
    pts = np.array([[0, 0], [4, 1], [1, 3], [2, 2], [3, .5], [.5, 1.5], [3.5, 3.5], [2.5, 1], [1.5, .2], [2, 3]], float)
    perm, off, D = R.partition(pts, 3, 2)
    assert perm.tolist() == [0, 8, 5, 3, 2, 4, 7, 1, 9, 6] and off.tolist() == [0, 3, 5, 8, 10] and D == 2


def test_partition_errors(lib):
    x = np.random.default_rng(0).uniform(0, 1, (100, 3))
    with pytest.raises(R.R3MGError) as e:
        R.partition(x, 64, 3)
    assert e.value.name == "E_DEPTH"
    with pytest.raises(R.R3MGError) as e:
        R.partition(x, 1, 2)
    assert e.value.name == "E_ARG"
    x[3, 1] = np.nan
    with pytest.raises(R.R3MGError) as e:
        R.partition(x, 8, 2)
    assert e.value.name == "E_ARG"


# ---------------------------------------------------------------- cell-based agglomeration
CELL_CASES = [(2, 4, 1, 0.0, 0, 4, 2), (2, 8, 2, 0.2, 3, 4, 3), (2, 12, 1, 0.1, 4, 6, 3), (3, 4, 2, 0.2, 5, 4, 2),
              (3, 4, 1, 0.15, 6, 2, 3), (3, 6, 3, 0.2, 7, 8, 3)]


@pytest.mark.parametrize("d,N,p,pert,seed,leaf,L", CELL_CASES)
def test_partition_cells_bit_exact_vs_oracle(lib, d, N, p, pert, seed, leaf, L):
    import workloads as W
    from oracle.rtree import cell_partition
    P = W.poisson(d, N, p, perturb=pert, seed=seed)
    ptr, pts = W.cells(d, N, p)
    perm, off, lo, hi, D = R.partition_cells(P.coords, ptr, pts, leaf, L)
    part = cell_partition(P.coords, ptr, pts, leaf, L)
    assert D == part.depth
    assert np.array_equal(perm, part.perm)
    assert np.array_equal(off, part.box_offsets[1])
    assert np.array_equal(lo, part.mbr_lo[1]) and np.array_equal(hi, part.mbr_hi[1])


def test_partition_cells_errors(lib):
    import workloads as W
    P = W.poisson(2, 4, 1)
    ptr, pts = W.cells(2, 4, 1)
    with pytest.raises(RuntimeError):
        R.partition_cells(P.coords, ptr, pts, 1, 2)            # leaf < 2
    with pytest.raises(RuntimeError):
        R.partition_cells(P.coords, ptr, pts, 4, 4)            # too shallow
    bad = pts.copy()
    bad[0] = P.n                                              # index out of range
    with pytest.raises(RuntimeError):
        R.partition_cells(P.coords, ptr, bad, 4, 2)
    orphan = np.where(pts == 4, -1, pts)                      # point 4 in no cell
    with pytest.raises(RuntimeError):
        R.partition_cells(P.coords, ptr, orphan, 4, 2)


def test_null_handles_and_pointers_are_argument_errors(lib):
    """Every solve-path entry point refuses a null hierarchy or null buffers with R3MG_E_ARG before
    touching the GPU (so these checks run without one)."""
    import ctypes
    null = ctypes.c_void_p(0)
    one = ctypes.c_void_p(8)          # a non-null pointer that is never dereferenced
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    E_ARG = 1
    assert lib.r3mg_pcg(null, one, one, 1e-8, 10, ctypes.byref(it), ctypes.byref(rel), null) == E_ARG
    assert lib.r3mg_vcycle(null, one, one, null) == E_ARG
    assert lib.r3mg_level_apply(null, 0, one, one, null) == E_ARG
    assert lib.r3mg_coarse_solve(null, one, one, null) == E_ARG
    assert lib.r3mg_update_values(null, one, null) == E_ARG
    its = np.zeros(4, np.int32)
    rels = np.zeros(4)
    assert lib.r3mg_pcg_multi(null, 4, one, one, 1e-8, 10, its.ctypes.data, rels.ctypes.data, null) == E_ARG
    assert lib.r3mg_vcycle_multi(null, 4, one, one, null) == E_ARG
    assert lib.r3mg_level_apply_multi(null, 0, 4, 0, one, one, null) == E_ARG
    s = ctypes.c_int(0)
    assert lib.r3mg_block_config(null, 0, 1, ctypes.byref(s)) == E_ARG
    assert lib.r3mg_set_block_config(null, 0, 1, 4) == E_ARG
    assert lib.r3mg_level0_apply_noalloc(null, one, one, null) == E_ARG
    lib.r3mg_destroy(null)            # a no-op


def _expected_groups(rp, br, ix):
    """Brute force of the grouping rule: per box, rows with equal index lists in increasing row
    order, cut into groups of 8, then 4, 2 and 1; per size, boxes in order."""
    per_size = {8: [], 4: [], 2: [], 1: []}
    for B in range(len(br) - 1):
        runs = {}
        for r in range(br[B], br[B + 1]):
            runs.setdefault(tuple(ix[rp[r]:rp[r + 1]].tolist()), []).append(r)
        box = {8: [], 4: [], 2: [], 1: []}
        for run in runs.values():
            i = 0
            for R_ in (8, 4, 2, 1):
                while len(run) - i >= R_:
                    box[R_].append(tuple(run[i:i + R_]))
                    i += R_
        for R_ in (8, 4, 2, 1):
            per_size[R_].append(sorted(box[R_]))
    return per_size


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_group_rows_vs_brute_force(lib, seed):
    """Host grouping of the block kernels' grouped fine level: every row once, each group one index
    list inside one box, sizes 8/4/2/1 cut in increasing row order, sizes then boxes in order."""
    rng = np.random.default_rng(seed)
    nbox = 5
    lists, box_row = [], [0]
    for B in range(nbox):
        base = [rng.integers(0, 200, size=4 * rng.integers(1, 6)).astype(np.uint16) for _ in range(4)]
        # a box's rows: repeats of a few lists (runs of 1 .. 19 rows), interleaved, plus distinct rows
        # of equal length (same key length, different contents)
        rows = []
        for j, lst in enumerate(base):
            rows += [lst] * int(rng.integers(1, 20))
        rows += [np.concatenate([base[0][:-1], [np.uint16(199 - k)]]) for k in range(3)]
        order = rng.permutation(len(rows))
        lists += [rows[k] for k in order]
        box_row.append(len(lists))
    rp = np.zeros(len(lists) + 1, np.int64)
    rp[1:] = np.cumsum([len(x) for x in lists])
    ix = np.concatenate(lists).astype(np.uint16)
    br = np.array(box_row, np.int64)
    counts, rows = R.group_rows(rp, br, ix)
    assert sorted(rows.tolist()) == list(range(len(lists)))
    want = _expected_groups(rp, br, ix)
    pos = 0
    for c, R_ in enumerate((8, 4, 2, 1)):
        assert counts[c] == sum(len(b) for b in want[R_])
        got = [tuple(rows[pos + k * R_: pos + (k + 1) * R_].tolist()) for k in range(int(counts[c]))]
        pos += int(counts[c]) * R_
        # boxes in order within a size, and within a box the expected set of groups
        k = 0
        for B, groups in enumerate(want[R_]):
            mine = sorted(got[k:k + len(groups)])
            assert mine == groups, (R_, B)
            for g in mine:
                assert all(br[B] <= r < br[B + 1] for r in g)
            k += len(groups)


def test_group_rows_errors(lib):
    rp = np.array([0, 4, 8], np.int64)
    ix = np.zeros(8, np.uint16)
    with pytest.raises(R.R3MGError) as e:
        R.group_rows(rp, np.array([0, 1], np.int64), ix)        # boxes cover 1 of 2 rows
    assert e.value.name == "E_ARG"
    with pytest.raises(R.R3MGError) as e:
        R.group_rows(np.array([0, 4, 2], np.int64), np.array([0, 2], np.int64), ix)   # decreasing row_ptr
    assert e.value.name == "E_ARG"
    counts, rows = R.group_rows(rp, np.array([0, 2], np.int64), ix)   # two equal rows: one group of 2
    assert counts.tolist() == [0, 0, 1, 0] and rows.tolist() == [0, 1]
