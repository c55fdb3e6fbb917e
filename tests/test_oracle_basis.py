"""Pins of the oracle's GLL nodes and box basis (Section 4; Section 5, GLL-norm lemma)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle.basis import box_basis, gll_nodes01, lagrange_1d


def test_gll_closed_forms():
    assert np.allclose(gll_nodes01(1), [0, 1], atol=0)
    assert np.allclose(gll_nodes01(2), [0, 0.5, 1], atol=1e-16)
    s5 = 1 / np.sqrt(5)
    assert np.allclose(gll_nodes01(3), [0, (1 - s5) / 2, (1 + s5) / 2, 1], atol=1e-15)
    s37 = np.sqrt(3 / 7)
    assert np.allclose(gll_nodes01(4), [0, (1 - s37) / 2, 0.5, (1 + s37) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_gll_norm_lemma(p):
    """Section 5, lemma on GLL shape functions: ||psi_j||^2_{L2(-1,1)} = 2p/(2p+1) w_j,
    w_j = 2 / (p (p+1) L_p(xi_j)^2).  A wrong node set breaks the identity."""
    xi = 2 * gll_nodes01(p) - 1
    c = np.zeros(p + 1); c[p] = 1
    Lp = npleg.legval(xi, c)
    w = 2.0 / (p * (p + 1) * Lp ** 2)
    tq, wq = np.polynomial.legendre.leggauss(p + 2)       # exact for degree 2p
    psi = lagrange_1d(xi, tq)
    norms = (wq[:, None] * psi ** 2).sum(0)
    assert np.allclose(norms, 2 * p / (2 * p + 1) * w, rtol=1e-13)
    assert abs(w.sum() - 2) < 1e-14


def test_lagrange_cardinal():
    z = gll_nodes01(4)
    assert np.allclose(lagrange_1d(z, z), np.eye(5), atol=1e-14)


@pytest.mark.parametrize("d,pp", [(2, 1), (2, 2), (3, 1), (3, 2), (3, 3)])
def test_box_basis_reproduces_qpprime(d, pp):
    rng = np.random.default_rng(d * 10 + pp)
    lo = rng.uniform(-1, 0, d); hi = lo + rng.uniform(0.5, 2, d)
    x = lo + (hi - lo) * rng.uniform(0, 1, (50, d))
    phi = box_basis(x, lo, hi, pp)
    assert np.allclose(phi.sum(1), 1.0, atol=1e-13)           # partition of unity
    # every monomial with per-axis degree <= p' is reproduced from its values at the box's GLL nodes
    z = gll_nodes01(pp)
    nb1 = pp + 1
    nodes = np.array([[lo[a] + z[(q // nb1 ** a) % nb1] * (hi[a] - lo[a]) for a in range(d)] for q in range(nb1 ** d)])
    for alpha in np.ndindex(*([nb1] * d)):
        f = lambda y: np.prod(y ** np.array(alpha), axis=1)
        assert np.allclose(phi @ f(nodes), f(x), atol=1e-12)


def test_splitmix64_published_outputs():
    """splitmix64 (Steele, Lea, Flood 2014) from state 0 yields 0xE220A8397B1DCDAF, then
    0x6E789E6AA1B965F4; the oracle maps each to 2 * (top 53 bits / 2^53) - 1."""
    from oracle.rng import splitmix64_uniform
    u = splitmix64_uniform(0, 2)
    for v, z in zip(u, (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4)):
        assert v == 2.0 * ((z >> 11) / 2.0 ** 53) - 1.0
