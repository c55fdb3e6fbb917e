"""Seeded synthetic finite-element workloads (inputs only).

Builds the Poisson systems the R-tree multilevel solver is applied to: the
model problem of Section 2 (eqs. (poisson), (weakform), (discweakform)),
continuous Q_p Lagrange elements on a structured, optionally perturbed
[0,1]^d mesh, or continuous P_p elements on its Kuhn triangulation (the
simplicial elements of Section 5), Dirichlet nodes eliminated.  This module holds none of the
multilevel method's arithmetic; the CPU oracle and the GPU library both
consume what it returns, and neither is imported here.

The C assembler (``fem.c``) is compiled on first use into ``_build/`` next
to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libfem.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile fem.c into _build/libfem.so (gcc, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "fem.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.fem_sizes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i64p]
        lib.fem_sizes.restype = ctypes.c_int
        lib.fem_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 6
        lib.fem_assemble.restype = ctypes.c_int
        lib.fem_l2_error.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_void_p]
        lib.fem_l2_error.restype = ctypes.c_double
        lib.fem_gll01.argtypes = [ctypes.c_int, ctypes.c_void_p]
        lib.fem_gll01.restype = None
        lib.fem_simplex_sizes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i64p]
        lib.fem_simplex_sizes.restype = ctypes.c_int
        lib.fem_simplex_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_uint64, ctypes.c_int] + [ctypes.c_void_p] * 6
        lib.fem_simplex_assemble.restype = ctypes.c_int
        lib.fem_simplex_l2_error.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_uint64, ctypes.c_void_p]
        lib.fem_simplex_l2_error.restype = ctypes.c_double
        _lib = lib
    return _lib


@dataclass
class Problem:
    """A free-DoF system A u = b with support-point coordinates."""
    dim: int
    N: int
    p: int
    perturb: float
    seed: int
    coords: np.ndarray      # (n, dim) float64, C-contiguous
    rowptr: np.ndarray      # (n+1,) int64
    colidx: np.ndarray      # (nnz,) int32, ascending within a row
    vals: np.ndarray        # (nnz,) float64, bitwise symmetric
    b: np.ndarray           # (n,) float64 load vector
    u_exact: np.ndarray     # (n,) float64 nodal values of the manufactured solution (zeros if f = 1)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.n, self.n))


def sizes(dim: int, N: int, p: int) -> tuple[int, int]:
    lib = _load()
    n = ctypes.c_int64(); nnz = ctypes.c_int64()
    if lib.fem_sizes(dim, N, p, ctypes.byref(n), ctypes.byref(nnz)) != 0:
        raise ValueError("bad mesh parameters")
    return int(n.value), int(nnz.value)


def poisson(dim: int, N: int, p: int, perturb: float = 0.0, seed: int = 0, kappa_modes: int = 0,
            rhs: str = "sine") -> Problem:
    """Assemble -div(kappa grad u) = f on [0,1]^dim, Q_p on an N^dim mesh.

    perturb: interior vertices move by U(-perturb*h, perturb*h) in each component (h = 1/N).
    kappa_modes: number of seeded random Fourier modes of g = log kappa (unit variance); 0 -> kappa = 1.
    rhs: "sine" (manufactured u = prod sin(pi x_a)) or "one" (f = 1).
    """
    lib = _load()
    n, nnz = sizes(dim, N, p)
    coords = np.empty((n, dim), np.float64)
    rowptr = np.empty(n + 1, np.int64)
    colidx = np.empty(nnz, np.int32)
    vals = np.empty(nnz, np.float64)
    b = np.empty(n, np.float64)
    uex = np.empty(n, np.float64)
    kind = {"sine": 0, "one": 1}[rhs]
    rc = lib.fem_assemble(dim, N, p, float(perturb), int(seed) & (2**64 - 1), int(kappa_modes), kind,
                          coords.ctypes.data, rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data,
                          b.ctypes.data, uex.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"fem_assemble failed ({rc})")
    return Problem(dim, N, p, perturb, seed, coords, rowptr, colidx, vals, b, uex,
                   meta={"kappa_modes": kappa_modes, "rhs": rhs})


def poisson_simplex(dim: int, N: int, p: int, perturb: float = 0.0, seed: int = 0, rhs: str = "sine") -> Problem:
    """Assemble -lap u = f on [0,1]^dim with continuous P_p elements on the Kuhn triangulation
    of the N^dim mesh (every cell split into dim! simplices the same way; p <= 4 in 2D, <= 3 in
    3D).  Support points are the equispaced barycentric lattice points of the affine simplices,
    which together form the (N p + 1)^dim grid; boundary nodes are eliminated and the free nodes
    numbered lexicographically as for Q_p.  perturb and seed move the interior cell vertices as
    in poisson(); rhs as in poisson()."""
    lib = _load()
    n = ctypes.c_int64(); nnz = ctypes.c_int64()
    if lib.fem_simplex_sizes(dim, N, p, ctypes.byref(n), ctypes.byref(nnz)) != 0:
        raise ValueError("bad simplex mesh parameters")
    n, nnz = int(n.value), int(nnz.value)
    coords = np.empty((n, dim), np.float64)
    rowptr = np.empty(n + 1, np.int64)
    colidx = np.empty(nnz, np.int32)
    vals = np.empty(nnz, np.float64)
    b = np.empty(n, np.float64)
    uex = np.empty(n, np.float64)
    kind = {"sine": 0, "one": 1}[rhs]
    rc = lib.fem_simplex_assemble(dim, N, p, float(perturb), int(seed) & (2**64 - 1), kind, coords.ctypes.data,
                                  rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data, b.ctypes.data,
                                  uex.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"fem_simplex_assemble failed ({rc})")
    return Problem(dim, N, p, perturb, seed, coords, rowptr, colidx, vals, b, uex,
                   meta={"kappa_modes": 0, "rhs": rhs, "element": "P"})


def l2_error(prob: Problem, u: np.ndarray) -> float:
    """L2 error of the FE function with free coefficients u against prod sin(pi x_a)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = lib.fem_simplex_l2_error if prob.meta.get("element") == "P" else lib.fem_l2_error
    return float(f(prob.dim, prob.N, prob.p, float(prob.perturb), int(prob.seed) & (2**64 - 1), u.ctypes.data))


def gll01(p: int) -> np.ndarray:
    """GLL nodes on [0,1] used for the fine support points."""
    x = np.empty(p + 1, np.float64)
    _load().fem_gll01(p, x.ctypes.data)
    return x


def gaussian(n: int, seed: int, count: int = 1) -> np.ndarray:
    """Seeded standard-normal vectors (n,) or (count, n), float64."""
    g = np.random.default_rng(seed).standard_normal((count, n))
    return g[0] if count == 1 else g


def cells(dim: int, N: int, p: int) -> tuple[np.ndarray, np.ndarray]:
    """Cell -> support-point connectivity of the structured Q_p mesh in the free-DoF numbering.

    Cell c = (c_0, ..., c_{d-1}) (lexicographic, c_0 fastest) holds the (p+1)^d grid nodes
    i_a = c_a p + k_a, k_a = 0..p; the free DoFs are the interior nodes of the (Np+1)^d grid,
    numbered lexicographically (x fastest), and eliminated boundary nodes appear as -1.
    Returns (cell_ptr (ncells+1,), cell_pts (ncells*(p+1)^d,)), both int64.
    """
    M = N * p
    k1 = np.arange(p + 1)
    c1 = np.arange(N)
    node1 = c1[:, None] * p + k1[None, :]                         # (N, p+1) grid index per axis
    free1 = np.where((node1 >= 1) & (node1 <= M - 1), node1 - 1, -1)
    per = (p + 1) ** dim
    if dim == 2:
        # cells (cy, cx) with cx fastest; nodes (ky, kx) with kx fastest
        fx = free1[None, :, None, :]                               # (1, N, 1, p+1)
        fy = free1[:, None, :, None]                               # (N, 1, p+1, 1)
        idx = fx + fy * (M - 1)
        ok = (fx >= 0) & (fy >= 0)
        pts = np.where(ok, idx, -1).reshape(N * N, per)
    else:
        fx = free1[None, None, :, None, None, :]
        fy = free1[None, :, None, None, :, None]
        fz = free1[:, None, None, :, None, None]
        idx = fx + fy * (M - 1) + fz * (M - 1) ** 2
        ok = (fx >= 0) & (fy >= 0) & (fz >= 0)
        pts = np.where(ok, idx, -1).reshape(N ** 3, per)
    ptr = np.arange(pts.shape[0] + 1, dtype=np.int64) * per
    return ptr, pts.reshape(-1).astype(np.int64)
