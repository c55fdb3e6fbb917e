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


# ---- P_p simplices on the Kuhn triangulation (the simplicial elements of Section 5)

def _interior_rows(P, margin):
    """Free rows whose lattice index lies at least `margin` nodes away from the boundary."""
    F = P.N * P.p - 1
    idx = np.arange(P.n)
    ok = np.ones(P.n, bool)
    for a in range(P.dim):
        i = (idx // F ** a) % F + 1
        ok &= (i > margin) & (i < F + 1 - margin)
    return np.nonzero(ok)[0]


def test_simplex_p1_reproduces_the_finite_difference_stencils():
    # P1 on the Kuhn triangulation of a uniform grid: 2D gives the 5-point stencil (4, -1 x 4);
    # 3D gives h times the 7-point stencil (6, -1 x 6) (the couplings along the cube diagonals cancel)
    P = W.poisson_simplex(2, 8, 1)
    A = P.scipy().tocsr()
    for i in _interior_rows(P, 2):
        row = np.sort(A[i].data[np.abs(A[i].data) > 1e-14])   # the diagonal neighbours couple with 0
        assert np.allclose(row, [-1, -1, -1, -1, 4], atol=1e-13), (i, row)
    P = W.poisson_simplex(3, 6, 1)
    A = P.scipy().tocsr()
    h = 1.0 / 6
    for i in _interior_rows(P, 2):
        row = np.sort(A[i].data[np.abs(A[i].data) > 1e-14])
        assert np.allclose(row / h, [-1] * 6 + [6], atol=1e-12), (i, row / h)


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 2)])
@pytest.mark.parametrize("perturb", [0.0, 0.2])
def test_simplex_bitwise_symmetric_spd_constant_kernel(dim, p, perturb):
    P = W.poisson_simplex(dim, 4, p, perturb=perturb, seed=5)
    A = P.scipy()
    assert (A != A.T).nnz == 0
    assert np.linalg.eigvalsh(A.toarray()).min() > 0
    # constants lie in the kernel of the Laplacian: rows coupled to free nodes only sum to zero
    rs = np.asarray(A.sum(axis=1)).ravel()
    rows = _interior_rows(P, p + 1)
    assert len(rows) > 0
    assert np.abs(rs[rows]).max() <= 1e-12 * np.abs(A).max()


def test_simplex_support_points_form_the_lattice():
    # unperturbed: the P_p nodes of all simplices are the points I / (N p) of the grid
    P = W.poisson_simplex(3, 3, 2)
    F = P.N * P.p - 1
    idx = np.arange(P.n)
    for a in range(3):
        assert np.allclose(P.coords[:, a], ((idx // F ** a) % F + 1) / (P.N * P.p), atol=1e-15)


@pytest.mark.parametrize("dim,p,Ns", [(2, 1, (16, 32)), (2, 2, (8, 16)), (2, 3, (4, 8)), (3, 2, (4, 8))])
def test_simplex_fe_error_rate(dim, p, Ns):
    # the discrete solution converges at the optimal L2 rate p + 1 (manufactured sine solution)
    errs = []
    for N in Ns:
        P = W.poisson_simplex(dim, N, p, perturb=0.0, seed=1)
        u = sla.spsolve(P.scipy().tocsc(), P.b)
        errs.append(W.l2_error(P, u))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 0.8, (errs, rate)


def test_oracle_pcg_converges_on_simplices():
    # the point-based R-tree hierarchy needs only support points, so it serves P_p simplices as
    # it serves Q_p cells (Section 5): a few PCG iterations on perturbed 2D and 3D P_2 meshes
    import oracle as O
    from oracle.hierarchy import Params
    for dim, N, leaf in ((2, 24, 64), (3, 5, 40)):
        P = W.poisson_simplex(dim, N, 2, perturb=0.1, seed=3)
        Ho = O.build_hierarchy(P.coords, P.scipy(), Params(leaf, 1, 3, cheb_degree=3))
        r = O.pcg(P.scipy(), P.b, lambda v: O.vcycle(Ho, v), rtol=1e-10)
        assert r.iterations <= 15
        assert np.linalg.norm(P.b - P.scipy() @ r.x) <= 1e-10 * np.linalg.norm(P.b)
