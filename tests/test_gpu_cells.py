"""Cell-based agglomeration on the GPU path (through the C ABI) against the oracle.

Agglomerates and block patterns bit-exact; P values 1e-14; Galerkin blocks 1e-12 of the largest
entry; one FP64 V-cycle 1e-12 relative; PCG iterations +-1 and the solution within 1e-10 of the
oracle's; the mixed-precision solve reaches the FP64 residual (same tolerances and reasons as the
point-based parity tests).  A late agglomerate left with too few points is reported as
R3MG_E_UNISOLVENT by both sides.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.hierarchy import Params
from oracle.transfer import UnisolventError

pytestmark = pytest.mark.gpu

# (dim, N, p, perturb, seed, leaf cells, p', levels, Chebyshev degree)
CASES = [
    (2, 16, 2, 0.2, 1, 8, 1, 3, 3),
    (2, 24, 1, 0.1, 2, 16, 1, 3, 2),
    (3, 6, 2, 0.2, 3, 8, 1, 3, 3),
    (3, 4, 3, 0.2, 4, 4, 2, 2, 3),
    (2, 10, 3, 0.15, 6, 4, 2, 3, 3),
]


def _setup(case, precision=0):
    import paper_2607_28235_b300 as R
    d, N, p, pert, seed, leaf, pp, L, k = case
    P = W.poisson(d, N, p, perturb=pert, seed=seed)
    cells = W.cells(d, N, p)
    H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, cells=cells, leaf_size=leaf, pprime=pp, levels=L,
                    cheb_degree=k, precision=precision)
    return P, cells, H


@pytest.fixture(scope="module", params=CASES, ids=[f"{c[0]}d_q{c[2]}_{c[1]}_pp{c[6]}_L{c[7]}" for c in CASES])
def trio(request):
    case = request.param
    P, cells, H = _setup(case)
    d, N, p, pert, seed, leaf, pp, L, k = case
    Ho = O.build_hierarchy(P.coords, P.scipy(), Params(leaf, pp, L, cheb_degree=k), cells=cells)
    return case, P, H, Ho


def test_agglomerates_and_patterns(trio):
    case, P, H, Ho = trio
    L = case[7]
    for lev in range(1, L):
        assert np.array_equal(H.agglomerates(lev), Ho.part.box_of_point[lev])
        ptr, nbr = H.level_pattern(lev)
        ref = Ho.patterns[lev]
        assert np.array_equal(np.diff(ptr), [len(v) for v in ref])
        assert np.array_equal(nbr, np.concatenate(ref))


def test_prolongation_and_galerkin(trio):
    case, P, H, Ho = trio
    b = H.b
    P0 = H.prolongation(0)
    ref = Ho.P[0].toarray()
    box = Ho.part.box_of_point[1]
    got = np.zeros_like(ref)
    for q in range(b):
        got[np.arange(P.n), box * b + q] = P0[:, q]
    assert np.max(np.abs(got - ref)) <= 1e-14
    for lev in range(1, case[7]):
        blocks = H.level_blocks(lev)
        ptr, nbr = H.level_pattern(lev)
        refA = Ho.A[lev].toarray()
        gotA = np.zeros_like(refA)
        for B in range(len(ptr) - 1):
            for e in range(ptr[B], ptr[B + 1]):
                gotA[B * b:(B + 1) * b, nbr[e] * b:(nbr[e] + 1) * b] = blocks[e]
        assert np.max(np.abs(gotA - refA)) <= 1e-12 * np.abs(refA).max()


def test_vcycle_and_pcg(trio):
    case, P, H, Ho = trio
    r = np.random.default_rng(3).standard_normal(P.n)
    z = H.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    ref = O.vcycle(Ho, r)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    rtol = 1e-10
    x, it, rel = H.pcg(torch.tensor(P.b, device="cuda"), rtol=rtol)
    refs = O.pcg(P.scipy(), P.b, lambda v: O.vcycle(Ho, v), rtol=rtol)
    assert abs(it - refs.iterations) <= 1
    assert np.linalg.norm(x.cpu().numpy() - refs.x) <= 1e-10 * np.linalg.norm(refs.x)


def test_mixed_precision_and_block_solve(trio):
    case, P, H, Ho = trio
    _, _, Hm = _setup(case, precision=1)
    A = P.scipy()
    x, it, rel = Hm.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-10)
    assert np.linalg.norm(P.b - A @ x.cpu().numpy()) <= 1e-10 * np.linalg.norm(P.b)
    B = np.random.default_rng(4).standard_normal((4, P.n))
    X, its, rels = Hm.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-10)
    X = X.cpu().numpy()
    for c in range(4):
        assert np.linalg.norm(B[c] - A @ X[c]) <= 1e-10 * np.linalg.norm(B[c])
    Hm.close()


def test_too_few_points_is_unisolvent():
    case = (3, 8, 1, 0.1, 5, 16, 1, 3, 3)
    d, N, p, pert, seed, leaf, pp, L, k = case
    P = W.poisson(d, N, p, perturb=pert, seed=seed)
    with pytest.raises(UnisolventError):
        O.build_hierarchy(P.coords, P.scipy(), Params(leaf, pp, L, cheb_degree=k), cells=W.cells(d, N, p))
    with pytest.raises(RuntimeError) as e:
        _setup(case)
    assert e.value.status == 5           # R3MG_E_UNISOLVENT
