"""Python binding of libr3mg: argument marshalling only.

Every step of the solver runs inside libr3mg (CUDA kernels for sm_103a and
host C++ for the R-tree); PyTorch tensors only provide device memory and
the current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import R3MGError, _Params, lib


# level-operator kernel forms, in the order of r3mg_kernel_config's codes
FORMS = ["register", "tma", "register_persistent", "register_l2_prefetch", "symmetric_block", "register_pipelined",
         "register_pipelined_l2_prefetch", "symmetric_block_staged"]


def _p(a) -> ctypes.c_void_p:
    if isinstance(a, torch.Tensor):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc: int, h=None):
    if rc != 0:
        raise R3MGError(rc, lib().r3mg_last_error(h).decode())


def default_params() -> dict:
    p = _Params()
    lib().r3mg_default_params(ctypes.byref(p))
    return {f: getattr(p, f) for f, _ in _Params._fields_}


def partition(coords: np.ndarray, leaf_size: int, levels: int):
    """Host-only R-tree bisection: (perm, leaf_offsets, depth); perm[k] = caller index at tree position k."""
    x = np.ascontiguousarray(coords, dtype=np.float64)
    n, d = x.shape
    perm = np.empty(n, np.int64)
    depth = ctypes.c_int(0)
    # leaf offsets need 2^D + 1 entries; D <= ceil(log2(n)) + 1
    off = np.empty((1 << (max(int(np.ceil(np.log2(max(n, 1)))), 0) + 1)) + 1, np.int64)
    rc = lib().r3mg_partition(n, d, _p(x), int(leaf_size), int(levels), _p(perm), _p(off), ctypes.byref(depth))
    _check(rc)
    return perm, off[: (1 << depth.value) + 1].copy(), depth.value


def partition_cells(coords: np.ndarray, cell_ptr: np.ndarray, cell_pts: np.ndarray, leaf_size: int, levels: int):
    """Host-only cell-based agglomeration: (perm, level-1 box offsets, box lo, box hi, depth)."""
    x = np.ascontiguousarray(coords, dtype=np.float64)
    n, d = x.shape
    cptr = np.ascontiguousarray(cell_ptr, dtype=np.int64)
    cpts = np.ascontiguousarray(cell_pts, dtype=np.int64)
    nc = len(cptr) - 1
    perm = np.empty(n, np.int64)
    cap = 1 << (max(int(np.ceil(np.log2(max(nc, 1)))), 0) + 1)
    off = np.empty(cap + 1, np.int64)
    lo = np.empty(cap * d, np.float64)
    hi = np.empty(cap * d, np.float64)
    depth = ctypes.c_int(0)
    rc = lib().r3mg_partition_cells(n, d, _p(x), nc, _p(cptr), _p(cpts), int(leaf_size), int(levels), _p(perm),
                                    _p(off), _p(lo), _p(hi), ctypes.byref(depth))
    _check(rc)
    nb = 1 << depth.value
    return perm, off[:nb + 1].copy(), lo[:nb * d].reshape(nb, d).copy(), hi[:nb * d].reshape(nb, d).copy(), depth.value


def group_rows(row_ptr: np.ndarray, box_row: np.ndarray, idx: np.ndarray):
    """Host-only row groups of the grouped block form: (counts of groups of 8, 4, 2, 1 rows, rows in group order)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    br = np.ascontiguousarray(box_row, dtype=np.int64)
    ix = np.ascontiguousarray(idx, dtype=np.uint16)
    n = len(rp) - 1
    counts = np.zeros(4, np.int64)
    rows = np.empty(max(n, 1), np.int32)
    _check(lib().r3mg_group_rows(n, _p(rp), len(br) - 1, _p(br), _p(ix) if len(ix) else None, _p(counts),
                                 _p(rows)))
    return counts, rows[:n].copy()


def wait_selftest(limit_cycles: int) -> tuple:
    """(status, expired): a one-CTA kernel whose mbarrier wait can only run out (status 10 = E_TIMEOUT)."""
    e = ctypes.c_int(0)
    rc = lib().r3mg_wait_selftest(int(limit_cycles), ctypes.byref(e), _stream())
    return rc, e.value


def measure_fp64_rates() -> dict:
    """Sustained FP64 FMA and FP64 tensor-core (mma.sync) rates of the current GPU, TFLOP/s."""
    f = ctypes.c_double(0)
    m = ctypes.c_double(0)
    _check(lib().r3mg_measure_fp64_rates(ctypes.byref(f), ctypes.byref(m), _stream()))
    return {"fma_tflops": f.value, "mma_tflops": m.value}


class Hierarchy:
    """R-tree multilevel hierarchy on the current CUDA device."""

    def __init__(self, coords, rowptr, colidx, vals, cells=None, **params):
        """cells = (cell_ptr, cell_pts) selects cell-based agglomeration (leaf_size counts
        cells; entries < 0 in cell_pts are points not in the system)."""
        p = _Params()
        lib().r3mg_default_params(ctypes.byref(p))
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = {f: getattr(p, f) for f, _ in _Params._fields_}
        x = np.ascontiguousarray(coords, dtype=np.float64)
        self.n, self.dim = x.shape
        on_device = isinstance(rowptr, torch.Tensor) and rowptr.is_cuda
        rp = None if on_device else np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = None if on_device else np.ascontiguousarray(colidx, dtype=np.int32)
        va = None if on_device else np.ascontiguousarray(vals, dtype=np.float64)
        self.nnz = 0 if on_device else int(rp[-1])
        self.b = (p.pprime + 1) ** self.dim
        h = ctypes.c_void_p()
        if isinstance(rowptr, torch.Tensor) and rowptr.is_cuda:
            # CSR arrays in device memory (r3mg_setup_device reads them back for the host analysis)
            assert cells is None, "cell-based setup takes host arrays"
            drp = rowptr.contiguous().to(torch.int64)
            dci = colidx.contiguous().to(torch.int32)
            dva = vals.contiguous().to(torch.float64)
            self.nnz = int(drp[-1].item())
            self.b = (p.pprime + 1) ** self.dim
            rc = lib().r3mg_setup_device(self.n, self.dim, _p(x), _p(drp), _p(dci), _p(dva), ctypes.byref(p),
                                         _stream(), ctypes.byref(h))
            _check(rc)
            self._h = h
            self.levels = self.info()["levels"]
            return
        if cells is None:
            rc = lib().r3mg_setup(self.n, self.dim, _p(x), _p(rp), _p(ci), _p(va), ctypes.byref(p), _stream(),
                                  ctypes.byref(h))
        else:
            cptr = np.ascontiguousarray(cells[0], dtype=np.int64)
            cpts = np.ascontiguousarray(cells[1], dtype=np.int64)
            rc = lib().r3mg_setup_cells(self.n, self.dim, _p(x), _p(rp), _p(ci), _p(va), len(cptr) - 1, _p(cptr),
                                        _p(cpts), ctypes.byref(p), _stream(), ctypes.byref(h))
        _check(rc)
        self._h = h
        info = self.info()
        self.levels = info["levels"]

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().r3mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ solves
    def vcycle(self, r: torch.Tensor) -> torch.Tensor:
        r = r.contiguous()
        assert r.is_cuda and r.dtype == torch.float64 and r.numel() == self.n
        z = torch.empty_like(r)
        _check(lib().r3mg_vcycle(self._h, _p(r), _p(z), _stream()), self._h)
        return z

    def pcg(self, b: torch.Tensor, x0: torch.Tensor | None = None, rtol: float = 1e-8, maxit: int = 500,
            raise_on_noconv: bool = True):
        b = b.contiguous()
        assert b.is_cuda and b.dtype == torch.float64 and b.numel() == self.n
        x = torch.zeros_like(b) if x0 is None else x0.clone().contiguous()
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0)
        rc = lib().r3mg_pcg(self._h, _p(b), _p(x), float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rel),
                            _stream())
        if rc != 0 and not (rc == 7 and not raise_on_noconv):
            _check(rc, self._h)
        return x, it.value, rel.value

    def pcg_multi(self, B: torch.Tensor, X0: torch.Tensor | None = None, rtol: float = 1e-8, maxit: int = 500,
                  raise_on_noconv: bool = True):
        """m <= 16 right-hand sides at once: B is (m, n) float64 on the GPU, one system per row."""
        B = B.contiguous()
        assert B.is_cuda and B.dtype == torch.float64 and B.dim() == 2 and B.shape[1] == self.n
        m = B.shape[0]
        X = torch.zeros_like(B) if X0 is None else X0.clone().contiguous()
        its = np.zeros(m, np.int32)
        rel = np.zeros(m, np.float64)
        rc = lib().r3mg_pcg_multi(self._h, m, _p(B), _p(X), float(rtol), int(maxit), _p(its), _p(rel), _stream())
        if rc != 0 and not (rc == 7 and not raise_on_noconv):
            _check(rc, self._h)
        return X, its, rel

    def vcycle_multi(self, R: torch.Tensor) -> torch.Tensor:
        R = R.contiguous()
        assert R.is_cuda and R.dtype == torch.float64 and R.dim() == 2 and R.shape[1] == self.n
        Z = torch.empty_like(R)
        _check(lib().r3mg_vcycle_multi(self._h, R.shape[0], _p(R), _p(Z), _stream()), self._h)
        return Z

    def level_apply_multi(self, level: int, X: torch.Tensor, fp32: bool = False) -> torch.Tensor:
        X = X.contiguous()
        assert X.is_cuda and X.dtype == torch.float64 and X.dim() == 2
        Y = torch.empty_like(X)
        _check(lib().r3mg_level_apply_multi(self._h, int(level), X.shape[0], 1 if fp32 else 0, _p(X), _p(Y),
                                            _stream()), self._h)
        return Y

    def block_config(self, fp32: bool = False) -> list:
        """Per level: entry slots of the block kernel (0 = staged coarse window, -1 = untuned)."""
        out = []
        for lev in range(self.levels):
            s = ctypes.c_int(0)
            _check(lib().r3mg_block_config(self._h, lev, 1 if fp32 else 0, ctypes.byref(s)), self._h)
            out.append(s.value)
        return out

    def set_block_config(self, level: int, slots: int, fp32: bool = False):
        _check(lib().r3mg_set_block_config(self._h, int(level), 1 if fp32 else 0, int(slots)), self._h)

    def pcg_host(self, b: np.ndarray, x0: np.ndarray | None = None, rtol: float = 1e-8, maxit: int = 500,
                 out: np.ndarray | None = None):
        """Host buffers in and out; the copies happen inside the library call.  `out` (optional,
        float64, n, e.g. a view of pinned memory) holds the initial guess on entry (x0 is copied
        into it when given) and receives the solution."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if out is not None:
            assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == b.shape
            x = out
            if x0 is not None:
                x[:] = x0
        else:
            x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0)
        rc = lib().r3mg_pcg_host(self._h, _p(b), _p(x), float(rtol), int(maxit), ctypes.byref(it),
                                 ctypes.byref(rel), _stream())
        _check(rc, self._h)
        return x, it.value, rel.value

    def update_values(self, vals: torch.Tensor):
        vals = vals.contiguous()
        assert vals.is_cuda and vals.dtype == torch.float64 and vals.numel() == self.nnz
        _check(lib().r3mg_update_values(self._h, _p(vals), _stream()), self._h)

    def coarse_solve(self, r: torch.Tensor, fp32: bool = False) -> torch.Tensor:
        """z = A_{L-1}^{-1} r on the coarsest level (coarsest-level numbering); fp32: the FP32 inverse."""
        r = r.contiguous()
        assert r.is_cuda and r.dtype == torch.float64
        z = torch.empty_like(r)
        _check(lib().r3mg_coarse_solve_prec(self._h, 1 if fp32 else 0, _p(r), _p(z), _stream()), self._h)
        return z

    def level_apply(self, level: int, x: torch.Tensor, fp32: bool = False) -> torch.Tensor:
        """y = A_l x with the V-cycle's kernel; fp32 uses the FP32 values (FP32 V-cycle hierarchies)."""
        x = x.contiguous()
        y = torch.empty_like(x)
        _check(lib().r3mg_level_apply_prec(self._h, int(level), 1 if fp32 else 0, _p(x), _p(y), _stream()), self._h)
        return y

    def cheb_step(self, level: int, x: torch.Tensor, r: torch.Tensor, d: torch.Tensor, a: float, c: float):
        """One fused Chebyshev-Jacobi step in the V-cycle precision: (x + d, r - A d, a d + c D^-1 (r - A d))."""
        x = x.contiguous(); r = r.contiguous(); d = d.contiguous()
        xo = torch.empty_like(x); ro = torch.empty_like(r); do = torch.empty_like(d)
        _check(lib().r3mg_level_cheb_step(self._h, int(level), _p(x), _p(r), _p(d), float(a), float(c), _p(xo), _p(ro),
                                          _p(do), _stream()), self._h)
        return xo, ro, do

    def set_stop_rule(self, atol: float = 0.0, reduction: float = 0.0):
        """Stop when ||r|| <= max(rtol ||b||, atol, reduction ||r_0||) (rtol = 0, 1e-9, 1e-6: the paper's rule)."""
        _check(lib().r3mg_set_stop_rule(self._h, float(atol), float(reduction)), self._h)

    def cond_estimate(self, column: int = -1) -> dict:
        """Condition estimate of the last solve (column >= 0: that column of the last block solve)."""
        c = ctypes.c_double(0); lo = ctypes.c_double(0); hi = ctypes.c_double(0); k = ctypes.c_int(0)
        _check(lib().r3mg_cond_estimate(self._h, int(column), ctypes.byref(c), ctypes.byref(lo), ctypes.byref(hi),
                                        ctypes.byref(k)), self._h)
        return {"cond": c.value, "lmin": lo.value, "lmax": hi.value, "steps": k.value}

    def stats(self) -> dict:
        """H (largest coarsest-box diameter), h (largest coupled-point distance), H/h, Ritz values per level."""
        H = ctypes.c_double(0); hh = ctypes.c_double(0); q = ctypes.c_double(0)
        ritz = np.zeros(self.levels, np.float64)
        _check(lib().r3mg_stats(self._h, ctypes.byref(H), ctypes.byref(hh), ctypes.byref(q), _p(ritz)), self._h)
        return {"H": H.value, "h": hh.value, "H_over_h": q.value, "ritz": ritz}

    def transfer_pattern(self, level: int, values: bool = True):
        """CSR (rowptr, cols, vals) of the transfer from level l+1 to level l (vals None unless values)."""
        nl = int(self.info()["n"][level])
        rp = np.empty(nl + 1, np.int64)
        cols = np.empty(nl * self.b, np.int32)
        vals = np.empty(nl * self.b, np.float64) if values else None
        _check(lib().r3mg_get_transfer_pattern(self._h, int(level), _p(rp), _p(cols), _p(vals) if values else None),
               self._h)
        return rp, cols, vals

    def level_matrix(self, level: int):
        """CSR (rowptr, cols, vals) of the Galerkin operator A_l, l >= 1, in coarse numbering."""
        nl = int(self.info()["n"][level])
        rp = np.empty(nl + 1, np.int64)
        _check(lib().r3mg_get_level_matrix(self._h, int(level), _p(rp), None, None), self._h)
        cols = np.empty(int(rp[-1]), np.int32)
        vals = np.empty(int(rp[-1]), np.float64)
        _check(lib().r3mg_get_level_matrix(self._h, int(level), _p(rp), _p(cols), _p(vals)), self._h)
        return rp, cols, vals

    def set_coarse_mode(self, mode: int):
        """Coarsest solve: 0 = explicit inverse (GEMV), 1 = forward and back substitution with L."""
        _check(lib().r3mg_set_coarse_mode(self._h, int(mode)), self._h)

    def set_wait_limit(self, cycles: int = 0, withhold_first_copy: bool = False):
        """Limit of the streamed kernels' bounded waits (0 = default); withhold_first_copy tests the expiry path."""
        _check(lib().r3mg_set_wait_limit(self._h, int(cycles), 1 if withhold_first_copy else 0), self._h)

    def device_status(self) -> int:
        """Status code of the bounded device waits since the last check (0, or 10 = E_TIMEOUT)."""
        return lib().r3mg_device_status(self._h, _stream())

    def sampled_outer(self, lam: torch.Tensor, u: torch.Tensor, alpha: float = -1.0) -> torch.Tensor:
        """out[k] = alpha * lam[i] * u[j] on every stored entry (i, j), in the setup CSR order."""
        lam = lam.contiguous(); u = u.contiguous()
        out = torch.empty(self.nnz, dtype=torch.float64, device=lam.device)
        _check(lib().r3mg_sampled_outer(self._h, _p(lam), _p(u), float(alpha), _p(out), _stream()), self._h)
        return out

    # ------------------------------------------------------------------ instrumentation
    def profile(self, on: bool = True):
        _check(lib().r3mg_profile_enable(self._h, 1 if on else 0), self._h)

    def profile_read(self) -> dict:
        """Per kind: (total ms, launches, algorithmic bytes per launch); plus kernel launches."""
        out = {}
        nl = ctypes.c_int64(0)
        for kind in range(self.levels + 1):
            ms = ctypes.c_double(0); n = ctypes.c_int64(0); by = ctypes.c_double(0)
            _check(lib().r3mg_profile_read(self._h, kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by),
                                           ctypes.byref(nl)), self._h)
            name = "cg_product_f64" if kind == 0 else f"cheb_step_level{kind - 1}"
            out[name] = {"ms": ms.value, "launches": n.value, "bytes_per_launch": by.value}
        out["kernel_launches"] = nl.value
        return out

    # ------------------------------------------------------------------ introspection
    def info(self) -> dict:
        L = ctypes.c_int(0)
        D = ctypes.c_int(0)
        _check(lib().r3mg_info(self._h, ctypes.byref(L), ctypes.byref(D), None, None, None, None), self._h)
        n = np.zeros(L.value, np.int64); nnz = np.zeros(L.value, np.int64); nb = np.zeros(L.value, np.int64)
        lam = np.zeros(L.value, np.float64)
        _check(lib().r3mg_info(self._h, None, None, _p(n), _p(nnz), _p(nb), _p(lam)), self._h)
        return {"levels": L.value, "depth": D.value, "n": n, "nnz": nnz, "nbox": nb, "lam_hi": lam}

    def kernel_config(self) -> list:
        """Per level: the level-operator kernel chosen for FP64 and FP32 (form, lanes, threads, tuned ms)."""
        out = []
        for lev in range(self.levels):
            row = {}
            for fp32, key in ((0, "f64"), (1, "f32")):
                f = ctypes.c_int(0); g = ctypes.c_int(0); t = ctypes.c_int(0); ms = ctypes.c_float(0)
                _check(lib().r3mg_kernel_config(self._h, lev, fp32, ctypes.byref(f), ctypes.byref(g), ctypes.byref(t),
                                                ctypes.byref(ms)), self._h)
                un = ctypes.c_int(0)
                _check(lib().r3mg_kernel_unroll(self._h, lev, fp32, ctypes.byref(un)), self._h)
                row[key] = {"form": FORMS[f.value], "lanes": g.value,
                            "threads": t.value, "unroll": un.value,
                            "tuned_ms": round(ms.value, 5)}
            out.append(row)
        return out

    def set_kernel_config(self, config: list):
        """Replay a configuration returned by kernel_config() (same hierarchy shape)."""
        forms = {name: i for i, name in enumerate(FORMS)}
        for lev, row in enumerate(config):
            for fp32, key in ((0, "f64"), (1, "f32")):
                if key not in row or (fp32 and self.params["precision"] != 1):
                    continue
                c = row[key]
                _check(lib().r3mg_set_kernel_config2(self._h, lev, fp32, forms[c["form"]], int(c["lanes"]),
                                                     int(c["threads"]), int(c.get("unroll", 0))), self._h)

    def agglomerates(self, level: int) -> np.ndarray:
        out = np.empty(self.n, np.int64)
        _check(lib().r3mg_get_agglomerates(self._h, int(level), _p(out)), self._h)
        return out

    def level_pattern(self, level: int):
        nbox = int(self.info()["nbox"][level])
        ptr = np.empty(nbox + 1, np.int64)
        _check(lib().r3mg_get_level_pattern(self._h, int(level), _p(ptr), None), self._h)
        nbr = np.empty(int(ptr[-1]), np.int64)
        _check(lib().r3mg_get_level_pattern(self._h, int(level), _p(ptr), _p(nbr)), self._h)
        return ptr, nbr

    def level_blocks(self, level: int) -> np.ndarray:
        ptr, _ = self.level_pattern(level)
        out = np.empty((int(ptr[-1]), self.b, self.b), np.float64)
        _check(lib().r3mg_get_level_blocks(self._h, int(level), _p(out)), self._h)
        return out

    def prolongation(self, level: int) -> np.ndarray:
        if level == 0:
            out = np.empty((self.n, self.b), np.float64)
        else:
            nbox = int(self.info()["nbox"][level])
            out = np.empty((nbox, self.b, self.b), np.float64)
        _check(lib().r3mg_get_prolongation(self._h, int(level), _p(out)), self._h)
        return out


class BatchHierarchy(Hierarchy):
    """Many independent problems (uneven sizes) in one block-diagonal hierarchy on the device."""

    def __init__(self, problems, **params):
        """problems: sequence of (coords, rowptr, colidx, vals), each in its own numbering."""
        p = _Params()
        lib().r3mg_default_params(ctypes.byref(p))
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = {f: getattr(p, f) for f, _ in _Params._fields_}
        self._keep = []
        ns, cs, rs, ks, vs = [], [], [], [], []
        for coords, rowptr, colidx, vals in problems:
            x = np.ascontiguousarray(coords, dtype=np.float64)
            rp = np.ascontiguousarray(rowptr, dtype=np.int64)
            ci = np.ascontiguousarray(colidx, dtype=np.int32)
            va = np.ascontiguousarray(vals, dtype=np.float64)
            self._keep += [x, rp, ci, va]
            ns.append(x.shape[0]); cs.append(x.ctypes.data); rs.append(rp.ctypes.data)
            ks.append(ci.ctypes.data); vs.append(va.ctypes.data)
        self.dim = np.asarray(problems[0][0]).shape[1]
        self.nprob = len(ns)
        narr = np.asarray(ns, np.int64)
        arr = lambda v: (ctypes.c_void_p * len(v))(*v)
        h = ctypes.c_void_p()
        rc = lib().r3mg_batch_setup(self.nprob, self.dim, _p(narr), arr(cs), arr(rs), arr(ks), arr(vs),
                                    ctypes.byref(p), _stream(), ctypes.byref(h))
        self._keep = None
        _check(rc)
        self._h = h
        self.n = int(narr.sum())
        self.sizes = narr
        self.offsets = np.concatenate([[0], np.cumsum(narr)])
        self.b = (p.pprime + 1) ** self.dim
        self.levels = self.info()["levels"]

    def set_batch_mode(self, mode: int):
        """0: the iteration loop as a graph of per-step kernels; 1: one persistent cooperative kernel;
        2 (default): automatic, the faster of the two as timed on the first two solves."""
        _check(lib().r3mg_set_batch_mode(self._h, int(mode)), self._h)

    def batch_mode(self) -> dict:
        """Loop mode setting (0 graph, 1 persistent, 2 automatic), the form the last solve used, and
        the automatic mode's per-iteration times of both forms (ms, -1 until measured)."""
        m = ctypes.c_int(0); u = ctypes.c_int(0); g = ctypes.c_float(0); pk = ctypes.c_float(0)
        _check(lib().r3mg_get_batch_mode(self._h, ctypes.byref(m), ctypes.byref(u), ctypes.byref(g), ctypes.byref(pk)),
               self._h)
        return {"mode": m.value, "used": u.value, "ms_per_iteration": {"graph": g.value, "persistent": pk.value}}

    def level_offsets(self, level: int) -> np.ndarray:
        out = np.empty(self.nprob + 1, np.int64)
        _check(lib().r3mg_batch_offsets(self._h, int(level), None, _p(out)), self._h)
        return out

    def pcg(self, b: torch.Tensor, x0: torch.Tensor | None = None, rtol: float = 1e-8, maxit: int = 500,
            raise_on_noconv: bool = True):
        b = b.contiguous()
        assert b.is_cuda and b.dtype == torch.float64 and b.numel() == self.n
        x = torch.zeros_like(b) if x0 is None else x0.clone().contiguous()
        its = np.zeros(self.nprob, np.int32)
        rel = np.zeros(self.nprob, np.float64)
        rc = lib().r3mg_batch_pcg(self._h, _p(b), _p(x), float(rtol), int(maxit), _p(its), _p(rel), _stream())
        if rc != 0 and not (rc == 7 and not raise_on_noconv):
            _check(rc, self._h)
        return x, its, rel
