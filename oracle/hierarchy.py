"""Galerkin hierarchy, smoother constants and coarsest factorisation.

Section 1 / Section 4: the level operators are inherited,
A_i = P_i^T A P_i, which level by level is A_1 = P_0^T A P_0 and
A_{l+1} = P~_l^T A_l P~_l.  Section 6: the smoother is a degree-3
Chebyshev-accelerated Jacobi iteration whose parameters come from Lanczos
eigenvalue estimates; the paper's coarse solver is a sparse direct method,
replaced here by a dense Cholesky factorisation of the coarsest operator.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .rng import splitmix64_uniform
from .rtree import Partition, cell_partition, rtree_partition
from .transfer import prolongation_coarse, prolongation_fine


class NotSPDError(ValueError):
    pass


def galerkin(A: sp.csr_matrix, P: sp.csr_matrix) -> sp.csr_matrix:
    """A_c = P^T A P (library sparse products; Section 1)."""
    return (P.T.tocsr() @ (A @ P)).tocsr()


def block_pattern(rows_box: np.ndarray, cols_box: np.ndarray, A: sp.csr_matrix, nbox: int) -> list:
    """Structural box adjacency of A: for each row box B, sorted boxes B' with some A_ij stored, i in B, j in B'."""
    A = A.tocoo()
    pairs = np.unique(rows_box[A.row].astype(np.int64) * nbox + cols_box[A.col].astype(np.int64))
    out = [[] for _ in range(nbox)]
    for pr in pairs:
        out[int(pr // nbox)].append(int(pr % nbox))
    return [np.array(v, np.int64) for v in out]


def coarse_block_pattern(fine_pattern: list, fan: int, nbox_coarse: int) -> list:
    """Block adjacency of A_{l+1} from that of A_l: parents of adjacent children (P~ is block diagonal by parent)."""
    out = [set() for _ in range(nbox_coarse)]
    for c, nbrs in enumerate(fine_pattern):
        for cp in nbrs:
            out[c // fan].add(int(cp) // fan)
    return [np.array(sorted(s), np.int64) for s in out]


def lanczos_lmax(A: sp.csr_matrix, steps: int, seed: int) -> float:
    """Largest Ritz value of D^{-1} A after `steps` Jacobi-preconditioned CG steps (Section 6).

    Reading taken (the paper only says "Lanczos iterations"): CG on
    A x = v, x_0 = 0, v uniform in [-1, 1) from splitmix64(seed), Jacobi
    preconditioner D = diag(A); the CG coefficients give the Lanczos
    tridiagonal T with T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1} and
    T_{j,j+1} = sqrt(beta_j)/alpha_j; the estimate is lambda_max(T).
    The loop stops early when r^T z is exactly 0 (Krylov space exhausted).
    """
    n = A.shape[0]
    dinv = 1.0 / A.diagonal()
    r = splitmix64_uniform(seed, n)
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    for _ in range(min(steps, n)):
        q = A @ p
        pq = float(p @ q)
        alpha = rz / pq
        r = r - alpha * q
        z = dinv * r
        rz_new = float(r @ z)
        alphas.append(alpha)
        beta = rz_new / rz
        betas.append(beta)
        if rz_new == 0.0:
            break
        p = z + beta * p
        rz = rz_new
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return float(np.linalg.eigvalsh(T)[-1])


def cholesky_lower(M: np.ndarray) -> np.ndarray:
    """Dense Cholesky M = L L^T, left-looking column form (textbook); raises NotSPDError on a pivot <= 0."""
    n = M.shape[0]
    L = np.zeros_like(M, dtype=np.float64)
    for j in range(n):
        s = M[j, j] - L[j, :j] @ L[j, :j]
        if not s > 0.0:
            raise NotSPDError(f"pivot {j} = {s}")
        L[j, j] = np.sqrt(s)
        if j + 1 < n:
            L[j + 1:, j] = (M[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def cholesky_solve(L: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = L^{-T} L^{-1} r by forward then back substitution (textbook loops), in the precision
    of L and r (float64 unless both are float32)."""
    n = L.shape[0]
    dt = np.result_type(L.dtype, np.asarray(r).dtype)
    y = np.empty(n, dt)
    for i in range(n):
        y[i] = (r[i] - L[i, :i] @ y[:i]) / L[i, i]
    z = np.empty(n, dt)
    for i in reversed(range(n)):
        z[i] = (y[i] - L[i + 1:, i] @ z[i + 1:]) / L[i, i]
    return z


def mesh_stats(coords, A: sp.csr_matrix, part: Partition) -> dict:
    """The mesh quantities of the paper's tables (Section 6, table legend): H = the largest box
    size on the coarsest level, read as the diameter (Euclidean length of the MBR diagonal) of a
    coarsest-level box, the paper's "maximal diameter of an agglomerate" (Section 1); h = the
    largest element size on the fine level.  The method sees support points, not elements:
    two support points share a stored entry of A exactly when they share an element, so h is
    read as the largest distance between two points coupled by a stored entry (the largest
    element diameter over the elements whose vertices are all unknowns)."""
    x = np.asarray(coords, np.float64)
    Ac = sp.csr_matrix(A).tocoo()
    h = float(np.sqrt(np.max(np.sum((x[Ac.row] - x[Ac.col]) ** 2, axis=1))))
    L = part.levels
    ext = np.asarray(part.mbr_hi[L - 1]) - np.asarray(part.mbr_lo[L - 1])
    H = float(np.sqrt(np.max(np.sum(ext ** 2, axis=1))))
    return {"H": H, "h": h, "H_over_h": H / h}


@dataclass
class Params:
    leaf_size: int
    pprime: int
    levels: int
    cheb_degree: int = 3          # Section 6: degree-3 Chebyshev
    sweeps: int = 2               # Section 6: 2 pre- and 2 post-smoothing steps
    lanczos_steps: int = 10
    eig_safety: float = 1.1       # reading: upper bound 1.1 * Ritz estimate
    eig_ratio: float = 30.0       # reading: lower bound = upper / 30
    seed: int = 0x5EED


@dataclass
class Hierarchy:
    params: Params
    part: Partition
    A: list                       # A[l] csr; A[0] in original numbering, A[l>=1] in box*b+q numbering
    P: list                       # P[l]: level l+1 -> level l
    dinv: list
    lam: list                     # Chebyshev interval (lo, hi) per smoothed level
    Lc: np.ndarray                # Cholesky factor of A[L-1] (dense)
    patterns: list = field(default_factory=list)   # block adjacency per coarse level (l >= 1)


def build_hierarchy(coords, A: sp.csr_matrix, prm: Params, cells=None) -> Hierarchy:
    """Setup: partition, transfers, Galerkin operators, smoother constants, coarsest Cholesky.

    cells = (cell_ptr, cell_pts) selects cell-based agglomeration (leaf_size counts cells);
    the default is point-based agglomeration (leaf_size counts support points)."""
    A0 = sp.csr_matrix(A, dtype=np.float64)
    if cells is None:
        part = rtree_partition(coords, prm.leaf_size, prm.levels)
    else:
        part = cell_partition(coords, cells[0], cells[1], prm.leaf_size, prm.levels)
    d = part.dim
    As, Ps, pats = [A0], [], [None]
    P0 = prolongation_fine(coords, part, prm.pprime)
    Ps.append(P0)
    As.append(galerkin(A0, P0))
    b = (prm.pprime + 1) ** d
    box_of_fine = part.box_of_point[1]
    pats.append(block_pattern(box_of_fine, box_of_fine, A0, part.nboxes(1)))
    for lev in range(1, prm.levels - 1):
        Pt = prolongation_coarse(part, lev, prm.pprime)
        Ps.append(Pt)
        As.append(galerkin(As[lev], Pt))
        pats.append(coarse_block_pattern(pats[lev], 1 << d, part.nboxes(lev + 1)))
    dinv, lam = [], []
    for lev in range(prm.levels - 1):
        diag = As[lev].diagonal()
        if np.any(~(diag > 0.0)):
            raise NotSPDError(f"level {lev} has a non-positive diagonal entry")
        dinv.append(1.0 / diag)
        lmax = lanczos_lmax(As[lev], prm.lanczos_steps, prm.seed + lev)
        hi = prm.eig_safety * lmax
        lam.append((hi / prm.eig_ratio, hi))
    Ac = As[-1].toarray()
    Lc = cholesky_lower(Ac)
    return Hierarchy(prm, part, As, Ps, dinv, lam, Lc, pats)
