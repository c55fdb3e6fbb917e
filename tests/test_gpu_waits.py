"""Bounded device waits run out without faulting or hanging the GPU, and the host hears of it.

Every mbarrier wait in the library's copy-engine-streamed kernels has an iteration limit; on
expiry the kernel raises a flag, waits (bounded) for the copies it still has in flight and
returns, and the next synchronising call reports R3MG_E_TIMEOUT.  The tests make waits run out
on purpose in the two ways that leave nothing unsafe behind: an arrival that announces bytes no
copy ever delivers (a one-CTA self-test kernel), and the TMA level kernel with its first
descriptor copy withheld.  Afterwards the context is still usable and results are correct.
"""
import numpy as np
import pytest
import torch

import oracle as O
from tests.gpu_cases import CASES, make

pytestmark = pytest.mark.gpu


def test_wait_selftest_runs_out_and_context_survives():
    import paper_2607_28235_b300 as R
    for limit in (1000, 200000):
        rc, expired = R.wait_selftest(limit)
        assert rc == 10 and expired == 1, (rc, expired)        # R3MG_E_TIMEOUT
    x = torch.arange(1000, dtype=torch.float64, device="cuda")
    assert float((x * 2).sum()) == 999000.0                    # the context still works


def test_tma_level_kernel_wait_expiry_is_reported():
    import paper_2607_28235_b300 as R
    P, params = make(CASES[1])                                 # 3D Q3, windows that fit the TMA stages
    H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, **dict(params, kernel_form=2))
    cfg = H.kernel_config()
    tma_levels = [l for l in range(params["levels"] - 1) if cfg[l]["f64"]["form"] == "tma"]
    if not tma_levels:
        H.close()
        pytest.skip("no level on the TMA form")
    lev = tma_levels[0]
    A = O.build_hierarchy(P.coords, P.scipy(), O.hierarchy.Params(params["leaf_size"], params["pprime"],
                                                                   params["levels"])).A[lev]
    x = torch.tensor(np.random.default_rng(51).standard_normal(A.shape[0]), device="cuda")
    assert H.device_status() == 0
    H.set_wait_limit(200000, withhold_first_copy=True)
    H.level_apply(lev, x)
    assert H.device_status() == 10                             # reported once ...
    assert H.device_status() == 0                              # ... and cleared
    H.set_wait_limit(0, withhold_first_copy=False)
    y = H.level_apply(lev, x).cpu().numpy()
    ref = A @ x.cpu().numpy()
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    assert H.device_status() == 0
    H.close()


def test_staged_symmetric_wait_expiry_is_reported():
    """The staged symmetric kernel's per-stage mbarrier wait runs out when CTA 0's first bulk copy
    is withheld: the step reports R3MG_E_TIMEOUT once, and the next step is exact again."""
    import paper_2607_28235_b300 as R
    P, params = make(CASES[1])
    H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, precision=1, **params)
    cfg = H.kernel_config()
    lev = 1
    cfg[lev]["f32"] = {"form": "symmetric_block_staged", "lanes": 1, "threads": 128}
    try:
        H.set_kernel_config(cfg[:-1])
    except RuntimeError:
        H.close()
        pytest.skip("level 1 has no staged symmetric form")
    n = H.info()["n"][lev]
    rng = np.random.default_rng(52)
    v = [torch.tensor(rng.standard_normal(n), device="cuda") for _ in range(3)]
    ref = [t.cpu().numpy() for t in H.cheb_step(lev, *v, 0.37, 0.71)]
    assert H.device_status() == 0
    H.set_wait_limit(200000, withhold_first_copy=True)
    H.cheb_step(lev, *v, 0.37, 0.71)
    assert H.device_status() == 10
    assert H.device_status() == 0
    H.set_wait_limit(0, withhold_first_copy=False)
    out = [t.cpu().numpy() for t in H.cheb_step(lev, *v, 0.37, 0.71)]
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)
    assert H.device_status() == 0
    H.close()
