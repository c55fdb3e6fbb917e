"""The allocation-free fine-level product, called through the C ABI.

r3mg_level0_apply_noalloc serves callers that cannot allocate device memory when they apply
the operator (for example while recording their own CUDA graph by stream capture); its
scratch is a static device array inside the library.  Its output must equal the ordinary
r3mg_level_apply(h, 0, ...) product, on two calls in a row (the shared scratch keeps the
previous call's contents, which must not leak into the next result).
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,N,p,pp,leaf,L", [(2, 32, 2, 1, 64, 3), (3, 5, 3, 2, 64, 3)])
def test_level0_apply_noalloc_matches_level_apply(dim, N, p, pp, leaf, L):
    import paper_2607_28235_b300 as R
    from paper_2607_28235_b300._lib import lib
    P = W.poisson(dim, N, p, perturb=0.2, seed=21)
    H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, leaf_size=leaf, pprime=pp, levels=L)
    rng = np.random.default_rng(3)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = P.scipy()
    for call in range(2):
        x = torch.tensor(rng.standard_normal(P.n), device="cuda")
        y = torch.full_like(x, float("nan"))
        rc = lib().r3mg_level0_apply_noalloc(H._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                             stream)
        assert rc == 0, lib().r3mg_last_error(H._h).decode()
        y_ref = H.level_apply(0, x)
        torch.cuda.synchronize()
        yn, yr = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.linalg.norm(yn - yr) <= 1e-13 * np.linalg.norm(yr), call
        assert np.linalg.norm(yn - A @ x.cpu().numpy()) <= 1e-13 * np.linalg.norm(yr), call
    H.close()


def test_level0_apply_noalloc_rejects_oversize():
    """A hierarchy larger than the static scratch (2^20 DoFs) is refused with R3MG_E_LIMIT before
    anything is launched: the output buffer keeps its contents.  2D Q1 on a 1026 x 1026 mesh has
    1025^2 = 1,050,625 free DoFs, just above 1,048,576."""
    import paper_2607_28235_b300 as R
    from paper_2607_28235_b300._lib import lib
    P = W.poisson(2, 1026, 1)
    assert P.n == 1025 * 1025 > (1 << 20)
    H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, leaf_size=64, pprime=1, levels=3, kernel_form=1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.ones(P.n, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, 7.25)
    rc = lib().r3mg_level0_apply_noalloc(H._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)
    torch.cuda.synchronize()
    assert rc == 9, rc                                   # R3MG_E_LIMIT
    assert "scratch limit" in lib().r3mg_last_error(H._h).decode()
    assert bool(torch.all(y == 7.25))
    H.close()
