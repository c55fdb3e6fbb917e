"""Transfer operators of the agglomerated hierarchy (Section 4).

Fine -> level 1 (point-based agglomeration, Section 4): the coarse function
(B, q) is the interpolant, at the fine support points owned by box B, of the
box polynomial phi_{B,q} in Q^{p'}(B); every fine point has exactly the
b = (p'+1)^d entries of its own box.  The stored pattern is structural: an
entry whose value happens to be 0 is kept.

Level l -> level l+1 (l >= 1): the natural injection P~ between agglomerated
levels (Section 4, P_i = P_{M-1} P~ ... P~).  A parent box polynomial
restricted to a child box is again in Q^{p'} of the child box, so it is
represented in the child's Lagrange basis by its values at the child's GLL
nodes: P~[(c, q'), (B, q)] = phi_{B,q}(xi_{c,q'}).  This makes the spaces
nested, V^{l+1} inside V^l (Section 4).

Coarse DoF numbering (the paper gives none): box * b + q.
"""
import numpy as np
import scipy.sparse as sp

from .basis import box_basis, gll_nodes01


class UnisolventError(ValueError):
    pass


def _check_box(lo, hi, pprime, npts, b):
    if npts < b:
        raise UnisolventError(f"box owns {npts} points < {b} coarse functions")
    if pprime >= 1 and np.any(hi <= lo):
        raise UnisolventError("box has zero extent along an axis")


def unisolvence_ok(phi: np.ndarray) -> bool:
    """Rank test of the owned-point evaluation matrix V (points x b).

    Reading taken for "enough support points to build the local
    interpolation" (Section 4, Remark on (m, M)): the Gram matrix V^T V must
    admit a Cholesky factorisation whose every pivot exceeds 1e-12 times its
    largest diagonal entry.  Textbook column Cholesky, FP64.
    """
    G = phi.T @ phi
    b = G.shape[0]
    tol = 1e-12 * np.max(np.diag(G))
    L = np.zeros_like(G)
    for j in range(b):
        s = G[j, j] - np.dot(L[j, :j], L[j, :j])
        if not s > tol:
            return False
        L[j, j] = np.sqrt(s)
        for i in range(j + 1, b):
            L[i, j] = (G[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return True


def prolongation_fine(coords: np.ndarray, part, pprime: int) -> sp.csr_matrix:
    """P_0 (n x nbox_1 * b), rows in the caller's (original) point numbering."""
    x = np.asarray(coords, np.float64)
    n, d = x.shape
    b = (pprime + 1) ** d
    nb = part.nboxes(1)
    rows, cols, vals = [], [], []
    for B in range(nb):
        members = part.perm[part.box_offsets[1][B]:part.box_offsets[1][B + 1]]
        lo, hi = part.mbr_lo[1][B], part.mbr_hi[1][B]
        _check_box(lo, hi, pprime, len(members), b)
        phi = box_basis(x[members], lo, hi, pprime)
        if pprime >= 1 and not unisolvence_ok(phi):
            raise UnisolventError(f"level-1 box {B}: points cannot carry Q^{pprime}")
        rows.append(np.repeat(members, b))
        cols.append(np.tile(B * b + np.arange(b), len(members)))
        vals.append(phi.ravel())
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, nb * b))
    P.sort_indices()
    return P


def coarse_nodes(lo: np.ndarray, hi: np.ndarray, pprime: int) -> np.ndarray:
    """Physical GLL nodes xi_{c,q'} of a box (b, d), q' lexicographic with x fastest."""
    d = len(lo)
    if pprime == 0:
        return ((lo + hi) / 2.0)[None, :]
    z = gll_nodes01(pprime)
    nb1 = pprime + 1
    b = nb1 ** d
    out = np.empty((b, d))
    for q in range(b):
        r = q
        for a in range(d):
            out[q, a] = lo[a] + z[r % nb1] * (hi[a] - lo[a])
            r //= nb1
    return out


def prolongation_coarse(part, level: int, pprime: int) -> sp.csr_matrix:
    """P~_l: level l+1 -> level l, (nbox_l * b) x (nbox_{l+1} * b), l >= 1."""
    d = part.dim
    b = (pprime + 1) ** d
    fan = 1 << d
    nc = part.nboxes(level)
    npar = part.nboxes(level + 1)
    rows, cols, vals = [], [], []
    for c in range(nc):
        B = c // fan                     # parents hold 2^d consecutive children
        lo_c, hi_c = part.mbr_lo[level][c], part.mbr_hi[level][c]
        lo_B, hi_B = part.mbr_lo[level + 1][B], part.mbr_hi[level + 1][B]
        _check_box(lo_B, hi_B, pprime, b, b)
        xi = coarse_nodes(lo_c, hi_c, pprime)
        blk = box_basis(xi, lo_B, hi_B, pprime)       # blk[q', q] = phi_{B,q}(xi_{c,q'})
        rows.append(np.repeat(c * b + np.arange(b), b))
        cols.append(np.tile(B * b + np.arange(b), b))
        vals.append(blk.ravel())
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nc * b, npar * b))
    P.sort_indices()
    return P
