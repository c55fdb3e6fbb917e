"""GLL nodes and the tensor-product Q^{p'} Lagrange basis on an axis-aligned box.

Section 4: on each agglomerate K with bounding box B_K the coarse functions
come from a basis of Q^{p'}(B_K); Section 5, eq. (localinterpolation) and the
definition of V_i^c.  The paper leaves the basis open ("a basis of
Q^{p'}(B_i)"); its analysis (Section 5, the GLL-norm lemma) works with
Gauss-Lobatto-Legendre nodes, and the partition-of-unity remark needs the
basis to sum to one.  Reading taken: Lagrange polynomials on the p'+1 GLL
nodes of each box edge, coefficient index q lexicographic with x fastest.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_nodes01(p: int) -> np.ndarray:
    """The p+1 Gauss-Lobatto-Legendre nodes mapped to [0, 1], ascending.

    Interior nodes are the roots of P_p' (derivative of the Legendre
    polynomial of degree p); the end points are 0 and 1.
    """
    if p == 0:
        return np.array([0.5])  # unused: degree 0 has the constant basis
    if p == 1:
        return np.array([0.0, 1.0])
    c = np.zeros(p + 1); c[p] = 1.0
    inner = np.sort(npleg.legroots(npleg.legder(c)).real)
    t = np.concatenate(([-1.0], inner, [1.0]))
    return 0.5 * (t + 1.0)


def lagrange_1d(nodes: np.ndarray, t: np.ndarray) -> np.ndarray:
    """L[k, a] = ell_a(t_k), the Lagrange polynomial of node a evaluated at t_k."""
    t = np.asarray(t, np.float64)
    m = len(nodes)
    L = np.ones((t.shape[0], m))
    for a in range(m):
        for k in range(m):
            if k != a:
                L[:, a] *= (t - nodes[k]) / (nodes[a] - nodes[k])
    return L


def box_basis(x: np.ndarray, lo: np.ndarray, hi: np.ndarray, pprime: int) -> np.ndarray:
    """phi[j, q] = prod_a ell_{q_a}((x_ja - lo_a) / (hi_a - lo_a)) for points x (m, d).

    q = q_0 + (p'+1) q_1 + (p'+1)^2 q_2 (x fastest).  Degree 0 gives phi = 1
    (the piecewise-constant Nicolaides space, Section 1).
    """
    x = np.atleast_2d(x)
    m, d = x.shape
    if pprime == 0:
        return np.ones((m, 1))
    z = gll_nodes01(pprime)
    per_axis = []
    for a in range(d):
        t = (x[:, a] - lo[a]) / (hi[a] - lo[a])
        per_axis.append(lagrange_1d(z, t))
    nb1 = pprime + 1
    b = nb1 ** d
    phi = np.ones((m, b))
    for q in range(b):
        r = q
        for a in range(d):
            phi[:, q] *= per_axis[a][:, r % nb1]
            r //= nb1
    return phi
