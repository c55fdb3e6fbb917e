"""Full-size workloads on the GPU, checked through properties and sampled oracle outputs.

* 3D Q3 32^3 perturbed (857,375 DoFs, the bench workload), leaf 128, p' 2, 4 levels, launched
  as the bench launches it: R-tree agglomerates bit-exact against the oracle; level-1 block
  pattern bit-exact against the oracle's structural adjacency; sampled level-1 Galerkin blocks
  against the oracle's definition P_B^T A[B, B'] P_B' (1e-12 relative); the fine-level Lanczos
  interval against the oracle's; PCG (FP64 and mixed) to 1e-8 with the true residual checked
  independently by scipy.
* 3D Q4 24^3 with kappa = exp(g) (857,375 DoFs, 174.7M nonzeros): gradient of
  L = 1/2 ||u - u_t||^2 with respect to the matrix values along a random symmetric direction
  and with respect to b, against central finite differences (step 1e-6) through the solver.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bench_problem():
    return W.poisson(3, 32, 3, perturb=0.2, seed=1)


def test_bench_workload_structure_and_blocks(bench_problem):
    import paper_2607_28235_b300 as R
    P = bench_problem
    H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, leaf_size=128, pprime=2, levels=4, cheb_degree=3)
    part = O.rtree_partition(P.coords, 128, 4)
    for lev in range(1, 4):
        assert np.array_equal(H.agglomerates(lev), part.box_of_point[lev])
    A = P.scipy()
    box = part.box_of_point[1]
    pat = O.block_pattern(box, box, A, part.nboxes(1))
    ptr, nbr = H.level_pattern(1)
    assert np.array_equal(np.diff(ptr), [len(v) for v in pat])
    assert np.array_equal(nbr, np.concatenate(pat))
    # sampled Galerkin blocks by the definition A_1[B, B'] = P_B^T A[B, B'] P_B'
    blocks = H.level_blocks(1)
    b = 27
    rng = np.random.default_rng(0)
    for B in rng.choice(part.nboxes(1), 12, replace=False):
        mB = part.perm[part.box_offsets[1][B]:part.box_offsets[1][B + 1]]
        PB = O.box_basis(P.coords[mB], part.mbr_lo[1][B], part.mbr_hi[1][B], 2)
        for e in range(ptr[B], ptr[B + 1], max(1, (ptr[B + 1] - ptr[B]) // 4)):
            C = nbr[e]
            mC = part.perm[part.box_offsets[1][C]:part.box_offsets[1][C + 1]]
            PC = O.box_basis(P.coords[mC], part.mbr_lo[1][C], part.mbr_hi[1][C], 2)
            ref = PB.T @ A[mB][:, mC].toarray() @ PC
            assert np.max(np.abs(blocks[e] - ref)) <= 1e-12 * np.max(np.abs(ref)) + 1e-300
    # fine-level smoother interval
    lam = O.lanczos_lmax(A, 10, 0x5EED)
    assert abs(H.info()["lam_hi"][0] - 1.1 * lam) <= 1e-10 * lam
    # solves
    bvec = torch.tensor(P.b, device="cuda")
    for prec in (0, 1):
        Hs = H if prec == 0 else R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, leaf_size=128, pprime=2,
                                             levels=4, cheb_degree=3, precision=1)
        x, it, rel = Hs.pcg(bvec, rtol=1e-8)
        r = np.linalg.norm(P.b - A @ x.cpu().numpy()) / np.linalg.norm(P.b)
        assert r <= 1e-8 and it <= 12, (prec, r, it)


def test_config3_kappa_gradients_full_size():
    from paper_2607_28235_b300.autograd import R3MGSolver
    P = W.poisson(3, 24, 4, perturb=0.0, seed=3, kappa_modes=16, rhs="one")
    assert P.n == 857375 and P.nnz == 174676879
    S = R3MGSolver(P.coords, P.rowptr, P.colidx, P.vals, rtol=1e-12, maxit=400, leaf_size=128, pprime=2, levels=4,
                   cheb_degree=3)
    rng = np.random.default_rng(5)
    ut = torch.tensor(rng.standard_normal(P.n), device="cuda")
    vals = torch.tensor(P.vals, device="cuda", requires_grad=True)
    b = torch.tensor(P.b, device="cuda", requires_grad=True)
    u = S.solve(vals, b)
    L = 0.5 * torch.sum((u - ut) ** 2)
    L.backward()
    gv, gb = vals.grad.cpu().numpy(), b.grad.cpu().numpy()
    # random symmetric direction on the pattern, scaled like the matrix
    A = P.scipy()
    R = sp.csr_matrix((rng.standard_normal(P.nnz), P.colidx, P.rowptr), shape=A.shape)
    E = (R + R.T).tocsr()
    E.sort_indices()
    Eval = E.data * np.abs(A.data).mean()      # the step 1e-6 is relative to the entries' scale
    # b direction along the gradient, scaled to ||b||: a random direction's derivative cancels to a
    # value far below the rounding of a loss of this size
    db = gb / np.linalg.norm(gb) * np.linalg.norm(P.b)
    h = 1e-6

    def loss(v, bb):
        with torch.no_grad():
            uu = S.solve(torch.tensor(v, device="cuda"), torch.tensor(bb, device="cuda"))
            return float(0.5 * torch.sum((uu - ut) ** 2))

    fd_v = (loss(P.vals + h * Eval, P.b) - loss(P.vals - h * Eval, P.b)) / (2 * h)
    an_v = float(gv @ Eval)
    fd_b = (loss(P.vals, P.b + h * db) - loss(P.vals, P.b - h * db)) / (2 * h)
    an_b = float(gb @ db)
    print(f"config3 directional: values fd {fd_v:.10e} an {an_v:.10e}; b fd {fd_b:.10e} an {an_b:.10e}")
    assert abs(fd_v - an_v) <= 1e-6 * abs(an_v)
    assert abs(fd_b - an_b) <= 1e-6 * abs(an_b)
