"""ctypes loader and compiler driver for libr3mg (CUDA sm_103a + host C++).

The shared library is built in-tree into ``_build/libr3mg.so`` by
``build()``.  Loading never falls back to anything else: a missing or stale
library raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(_HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
SO_PATH = os.path.join(_HERE, "_build", "libr3mg.so")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC,-fopenmp,-O3", "-shared"]


def sources() -> list[str]:
    out = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cpp")):
            out.append(os.path.join(CSRC, name))
    return out


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "r3mg.h"))
    return files


def stale() -> bool:
    if not os.path.exists(SO_PATH):
        return True
    t = os.path.getmtime(SO_PATH)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libr3mg.so for sm_103a with nvcc (host code with OpenMP)."""
    if not force and not stale():
        return SO_PATH
    os.makedirs(os.path.dirname(SO_PATH), exist_ok=True)
    tmp = SO_PATH + f".tmp{os.getpid()}"
    cmd = ["nvcc", *NVCC_FLAGS, "-o", tmp, *sources(), "-lgomp"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, SO_PATH)
    return SO_PATH


class _Params(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("pprime", ctypes.c_int), ("levels", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("sweeps", ctypes.c_int), ("lanczos_steps", ctypes.c_int),
                ("eig_safety", ctypes.c_double), ("eig_ratio", ctypes.c_double), ("precision", ctypes.c_int),
                ("group_lanes", ctypes.c_int), ("seed", ctypes.c_uint64), ("kernel_form", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError(f"libr3mg is not built ({SO_PATH}); run paper_2607_28235_b300.build()")
    L = ctypes.CDLL(SO_PATH)
    vp, i64, i32, dbl, ip = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "r3mg_default_params": (None, [P(_Params)]),
        "r3mg_partition": (ip, [i64, i32, vp, i32, i32, vp, vp, P(ctypes.c_int)]),
        "r3mg_setup": (ip, [i64, i32, vp, vp, vp, vp, P(_Params), vp, P(vp)]),
        "r3mg_setup_cells": (ip, [i64, i32, vp, vp, vp, vp, i64, vp, vp, P(_Params), vp, P(vp)]),
        "r3mg_partition_cells": (ip, [i64, i32, vp, i64, vp, vp, i32, i32, vp, vp, vp, vp, P(ctypes.c_int)]),
        "r3mg_group_rows": (ip, [i64, vp, i64, vp, vp, vp, vp]),
        "r3mg_update_values": (ip, [vp, vp, vp]),
        "r3mg_vcycle": (ip, [vp, vp, vp, vp]),
        "r3mg_pcg": (ip, [vp, vp, vp, dbl, i32, P(ctypes.c_int), P(ctypes.c_double), vp]),
        "r3mg_pcg_host": (ip, [vp, vp, vp, dbl, i32, P(ctypes.c_int), P(ctypes.c_double), vp]),
        "r3mg_level_apply": (ip, [vp, i32, vp, vp, vp]),
        "r3mg_coarse_solve": (ip, [vp, vp, vp, vp]),
        "r3mg_pcg_multi": (ip, [vp, i32, vp, vp, dbl, i32, vp, vp, vp]),
        "r3mg_vcycle_multi": (ip, [vp, i32, vp, vp, vp]),
        "r3mg_level_apply_multi": (ip, [vp, i32, i32, i32, vp, vp, vp]),
        "r3mg_block_config": (ip, [vp, i32, i32, P(ctypes.c_int)]),
        "r3mg_set_block_config": (ip, [vp, i32, i32, i32]),
        "r3mg_info": (ip, [vp, P(ctypes.c_int), P(ctypes.c_int), vp, vp, vp, vp]),
        "r3mg_get_agglomerates": (ip, [vp, i32, vp]),
        "r3mg_get_level_pattern": (ip, [vp, i32, vp, vp]),
        "r3mg_get_level_blocks": (ip, [vp, i32, vp]),
        "r3mg_get_prolongation": (ip, [vp, i32, vp]),
        "r3mg_profile_enable": (ip, [vp, i32]),
        "r3mg_profile_read": (ip, [vp, i32, P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_double),
                                   P(ctypes.c_int64)]),
        "r3mg_kernel_config": (ip, [vp, i32, i32, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                    P(ctypes.c_float)]),
        "r3mg_level0_apply_noalloc": (ip, [vp, vp, vp, vp]),
        "r3mg_set_kernel_config": (ip, [vp, i32, i32, i32, i32, i32]),
        "r3mg_set_kernel_config2": (ip, [vp, i32, i32, i32, i32, i32, i32]),
        "r3mg_kernel_unroll": (ip, [vp, i32, i32, P(ctypes.c_int)]),
        "r3mg_sampled_outer": (ip, [vp, vp, vp, dbl, vp, vp]),
        "r3mg_batch_setup": (ip, [i32, i32, vp, vp, vp, vp, vp, P(_Params), vp, P(vp)]),
        "r3mg_batch_pcg": (ip, [vp, vp, vp, dbl, i32, vp, vp, vp]),
        "r3mg_batch_offsets": (ip, [vp, i32, P(ctypes.c_int), vp]),
        "r3mg_measure_fp64_rates": (ip, [P(ctypes.c_double), P(ctypes.c_double), vp]),
        "r3mg_level_apply_prec": (ip, [vp, i32, i32, vp, vp, vp]),
        "r3mg_level_cheb_step": (ip, [vp, i32, vp, vp, vp, dbl, dbl, vp, vp, vp, vp]),
        "r3mg_coarse_solve_prec": (ip, [vp, i32, vp, vp, vp]),
        "r3mg_set_stop_rule": (ip, [vp, dbl, dbl]),
        "r3mg_cond_estimate": (ip, [vp, i32, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                    P(ctypes.c_int)]),
        "r3mg_stats": (ip, [vp, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), vp]),
        "r3mg_get_transfer_pattern": (ip, [vp, i32, vp, vp, vp]),
        "r3mg_get_level_matrix": (ip, [vp, i32, vp, vp, vp]),
        "r3mg_device_status": (ip, [vp, vp]),
        "r3mg_set_wait_limit": (ip, [vp, ctypes.c_longlong, i32]),
        "r3mg_set_coarse_mode": (ip, [vp, i32]),
        "r3mg_set_batch_mode": (ip, [vp, i32]),
        "r3mg_get_batch_mode": (ip, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_float), P(ctypes.c_float)]),
        "r3mg_wait_selftest": (ip, [ctypes.c_longlong, P(ctypes.c_int), vp]),
        "r3mg_setup_device": (ip, [i64, i32, vp, vp, vp, vp, P(_Params), vp, P(vp)]),
        "r3mg_last_error": (ctypes.c_char_p, [vp]),
        "r3mg_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


STATUS = {0: "OK", 1: "E_ARG", 2: "E_CUDA", 3: "E_OOM", 4: "E_DEPTH", 5: "E_UNISOLVENT", 6: "E_NOT_SPD",
          7: "E_NOCONV", 8: "E_BREAKDOWN", 9: "E_LIMIT", 10: "E_TIMEOUT"}


class R3MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"r3mg {STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))
