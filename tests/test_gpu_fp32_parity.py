"""The FP32 arithmetic of the mixed-precision solver against the oracle, element by element.

The headline solve runs the V-cycle in FP32 (values, vectors, accumulation, transfers, the
coarsest inverse) inside FP64 flexible CG.  The outer iteration would absorb a wrong FP32 kernel,
so every FP32 stage is checked here on its own, under a bound derived from FP32 rounding
(u = 2^-24, round to nearest):

* Level product y = A_l x (one launch of the level kernel the V-cycle uses, every kernel form the
  tuner can pick): the kernel reads A_l rounded to FP32 (error <= u |a_ij|) and x rounded to FP32
  (the test rounds x the same way, so x32 is exact), then sums k products in FP32 in some order,
  which errs by at most gamma_{k-1} (|A||x32|)_i with gamma_m = m u / (1 - m u).  So
      |y_i - (A x32)_i| <= (k_i + 2) u (|A| |x32|)_i,
  k_i the stored entries of row i (the oracle's A differs from the library's FP64 A_l by
  1e-12 of the largest entry at most, far below u).
* Fused Chebyshev step (x' = x + d; r' = r - A d; d' = a d + c D^{-1} r'): x' is one FP32
  addition (bit for bit equal to numpy's float32 sum); r' is the product bound plus one rounding
  of the subtraction; d' is at most four roundings of two products and a sum, with D^{-1} rounded
  to FP32 from the library's FP64 diagonal (which may differ from the oracle's by one unit in
  the last place), so |d'_i - (a d + c dinv r')_i| <= 5 u (|a d_i| + |c dinv_i r'_i|).
* Coarsest solve with the FP32 inverse: r and A_c^{-1} rounded (2 u), an n_c-term FP32 dot
  product (gamma_{n_c}), and the FP64 inverse itself (kappa(A_c) 1e-14 relative):
      |z_i - (A_c^{-1} r32)_i| <= (n_c + 3) u (|A_c^{-1}| |r32|)_i + 1e-14 kappa(A_c) ||z||_inf.
* The whole V-cycle: z~ - z = sum_s G_s delta_s, where delta_s is the rounding of stage s (each
  bounded as above) and G_s the exact linear map from stage s to the output.  Composing the
  stage bounds through |G_s| gives a useless worst case (|A| has no cancellation), so the bound
  is set by an independent FP32 evaluation of the same stages: the oracle's V-cycle with every
  operator and vector in float32 (``oracle.as_precision``; numpy/scipy keep float32 operands
  and accumulation in float32) has local errors under the same stage bounds, in its own
  summation order.  The library's FP32 V-cycle must stay within 8 times that evaluation's
  distance from the FP64 oracle, in the max norm and in the 2-norm (floor: 64 u ||z||).  A
  dropped, duplicated or mis-scaled entry, coefficient or transfer moves z by orders of
  magnitude more than FP32 rounding does.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
from oracle.hierarchy import Params
from tests.gpu_cases import CASES, make

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
FORMS = ["register", "tma", "register_persistent", "register_l2_prefetch", "register_pipelined",
         "register_pipelined_l2_prefetch", "symmetric_block", "symmetric_block_staged"]
FINE_ONLY = set()               # forms of the fine level only
SYMMETRIC = {"symmetric_block", "symmetric_block_staged"}   # Chebyshev steps only, coarse levels only
COARSE_ONLY = SYMMETRIC
PRODUCT_FORMS = [f for f in FORMS if f not in SYMMETRIC]


def _lanes_threads(form, lanes):
    if form == "symmetric_block":
        return 16, 128
    if form == "symmetric_block_staged":
        return 4, 128                   # lanes field: resident CTAs per SM
    return lanes, 512 if form == "tma" else 256


def _hier(P, params, precision=1, **kw):
    import paper_2607_28235_b300 as R
    return R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, precision=precision, **dict(params, **kw))


def _oracle(P, params):
    return O.build_hierarchy(P.coords, P.scipy(), Params(params["leaf_size"], params["pprime"], params["levels"],
                                                          cheb_degree=params["cheb_degree"]))


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    P, params = make(request.param)
    return P, params, _oracle(P, params)


def _pin_form(H, form, levels, fp32=True):
    """Pin one kernel form on the given levels (FP32 configuration); False when a level cannot host it."""
    cfg = H.kernel_config()
    key = "f32" if fp32 else "f64"
    for lev in levels:
        if (form in COARSE_ONLY and lev == 0) or (form in FINE_ONLY and lev > 0):
            continue
        lanes, threads = _lanes_threads(form, cfg[lev][key]["lanes"] if cfg[lev][key]["lanes"] >= 4 else 16)
        cfg[lev][key] = {"form": form, "lanes": lanes, "threads": threads}
    try:
        H.set_kernel_config(cfg[:-1])
    except Exception:
        return False
    return True


def _row_len(A):
    return np.diff(sp.csr_matrix(A).indptr)


@pytest.mark.parametrize("form", PRODUCT_FORMS)
def test_fp32_level_product_rowwise_bound(case, form):
    P, params, Ho = case
    H = _hier(P, params)
    L = params["levels"]
    if not _pin_form(H, form, range(L - 1)):
        H.close()
        pytest.skip(f"{form} cannot host this case's windows")
    rng = np.random.default_rng(11)
    for lev in range(L - 1):
        A = Ho.A[lev]
        x32 = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
        y = H.level_apply(lev, torch.tensor(x32, device="cuda"), fp32=True).cpu().numpy()
        ref = A @ x32
        mag = abs(A) @ np.abs(x32)
        bound = (_row_len(A) + 2) * U32 * mag
        bad = np.abs(y - ref) > bound
        assert not bad.any(), (lev, form, int(bad.sum()), float(np.max(np.abs(y - ref) / np.maximum(mag, 1e-300))))
    H.close()


@pytest.mark.parametrize("form", FORMS)
def test_fp32_cheb_step_bounds(case, form):
    P, params, Ho = case
    H = _hier(P, params)
    L = params["levels"]
    if not _pin_form(H, form, range(L - 1)):
        H.close()
        pytest.skip(f"{form} cannot host this case's windows")
    _cheb_step_checks(H, Ho, range(L - 1), form)
    H.close()


def _cheb_step_checks(H, Ho, levels, form):
    rng = np.random.default_rng(12)
    a, c = 0.37, 0.71
    a32, c32 = float(np.float32(a)), float(np.float32(c))
    for lev in levels:
        A = Ho.A[lev]
        n = A.shape[0]
        x, r, d = (rng.standard_normal(n).astype(np.float32).astype(np.float64) for _ in range(3))
        xo, ro, do = (t.cpu().numpy() for t in H.cheb_step(lev, *(torch.tensor(v, device="cuda") for v in (x, r, d)),
                                                              a, c))
        # x' = x + d: one FP32 addition, bit for bit
        assert np.array_equal(xo, (x.astype(np.float32) + d.astype(np.float32)).astype(np.float64)), (lev, form)
        # r' = r - A d
        mag = np.abs(r) + abs(A) @ np.abs(d)
        assert np.all(np.abs(ro - (r - A @ d)) <= (_row_len(A) + 3) * U32 * mag), (lev, form)
        # d' = a d + c D^{-1} r'  (with the library's r')
        dinv32 = (1.0 / A.diagonal()).astype(np.float32).astype(np.float64)
        exact = a32 * d + c32 * dinv32 * ro
        assert np.all(np.abs(do - exact) <= 5 * U32 * (np.abs(a32 * d) + np.abs(c32 * dinv32 * ro))), (lev, form)


@pytest.mark.parametrize("lanes", [16, 4])   # 8-row and 4-row load waves
def test_fp32_cheb_step_bounds_symmetric_96_threads(case, lanes):
    """The symmetric form on 96-thread CTAs (one thread per four-column group of a 27-row box's
    upper window) keeps the FP32 Chebyshev-step bounds on every coarse level."""
    P, params, Ho = case
    H = _hier(P, params)
    L = params["levels"]
    cfg = H.kernel_config()
    for lev in range(1, L - 1):
        cfg[lev]["f32"] = {"form": "symmetric_block", "lanes": lanes, "threads": 96}
    try:
        H.set_kernel_config(cfg[:-1])
    except RuntimeError:
        H.close()
        pytest.skip("no symmetric coarse level")
    assert all(H.kernel_config()[lev]["f32"]["threads"] == 96 for lev in range(1, L - 1))
    _cheb_step_checks(H, Ho, range(1, L - 1), "symmetric_block/96")
    H.close()


def test_fp32_coarse_solve_bound(case):
    P, params, Ho = case
    H = _hier(P, params)
    Ac = Ho.A[-1].toarray()
    Ainv = np.linalg.inv(Ac)
    kappa = np.linalg.cond(Ac)
    nc = Ac.shape[0]
    r32 = np.random.default_rng(13).standard_normal(nc).astype(np.float32).astype(np.float64)
    z = H.coarse_solve(torch.tensor(r32, device="cuda"), fp32=True).cpu().numpy()
    ref = Ainv @ r32
    bound = (nc + 3) * U32 * (np.abs(Ainv) @ np.abs(r32)) + 1e-14 * kappa * np.abs(ref).max()
    assert np.all(np.abs(z - ref) <= bound), float(np.max(np.abs(z - ref) / bound))
    H.close()


def fp32_vcycle_check(H, Ho, r, what=""):
    """The library's FP32 V-cycle against the FP64 oracle, within 8x the distance of the oracle's
    own FP32 evaluation of the same stages (max norm and 2-norm; floor 64 u ||z||)."""
    z64 = O.vcycle(Ho, r)
    z32o = O.vcycle(O.as_precision(Ho, np.float32), r.astype(np.float32)).astype(np.float64)
    z = H.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    ref_inf = max(np.abs(z32o - z64).max(), 64 * U32 * np.abs(z64).max())
    ref_2 = max(np.linalg.norm(z32o - z64), 64 * U32 * np.linalg.norm(z64))
    err_inf = np.abs(z - z64).max()
    err_2 = np.linalg.norm(z - z64)
    assert err_inf <= 8 * ref_inf, (what, err_inf / ref_inf)
    assert err_2 <= 8 * ref_2, (what, err_2 / ref_2)
    return err_2 / np.linalg.norm(z64), ref_2 / np.linalg.norm(z64)


def test_fp32_vcycle_vs_oracle_autotuned(case):
    P, params, Ho = case
    H = _hier(P, params)
    rng = np.random.default_rng(14)
    for trial in range(2):
        r = rng.standard_normal(P.n) if trial else P.b.copy()
        fp32_vcycle_check(H, Ho, r, f"autotuned trial {trial}")
    H.close()


@pytest.mark.parametrize("form", FORMS)
def test_fp32_vcycle_vs_oracle_each_form(case, form):
    P, params, Ho = case
    H = _hier(P, params)
    if not _pin_form(H, form, range(params["levels"] - 1)):
        H.close()
        pytest.skip(f"{form} cannot host this case's windows")
    r = np.random.default_rng(15).standard_normal(P.n)
    fp32_vcycle_check(H, Ho, r, form)
    H.close()


@pytest.mark.parametrize("form,cps", [("symmetric_block_staged", 1), ("symmetric_block_staged", 4),
                                      ("symmetric_block", 4)])   # the last: 4-row load waves
def test_staged_symmetric_step_same_bits_as_streamed(case, form, cps):
    """The staged symmetric kernel (one bulk copy of each box's upper slice into shared memory;
    with a stage sized for 4 CTAs per SM the largest slices are read from global memory instead)
    computes every box exactly as the streamed one: the Chebyshev step outputs agree bit for bit
    on every coarse level."""
    P, params, Ho = case
    H1, H2 = _hier(P, params), _hier(P, params)
    L = params["levels"]
    ok = _pin_form(H1, "symmetric_block", range(1, L - 1))
    cfg = H2.kernel_config()
    for lev in range(1, L - 1):
        cfg[lev]["f32"] = {"form": form, "lanes": cps, "threads": 128}
    try:
        H2.set_kernel_config(cfg[:-1])
    except RuntimeError:
        ok = False
    if not ok:
        H1.close(); H2.close()
        pytest.skip("no symmetric coarse level")
    rng = np.random.default_rng(16)
    for lev in range(1, L - 1):
        n = Ho.A[lev].shape[0]
        v = [torch.tensor(rng.standard_normal(n), device="cuda") for _ in range(3)]
        o1 = [t.cpu().numpy() for t in H1.cheb_step(lev, *v, 0.37, 0.71)]
        o2 = [t.cpu().numpy() for t in H2.cheb_step(lev, *v, 0.37, 0.71)]
        for a, b in zip(o1, o2):
            assert np.array_equal(a, b), lev
    H1.close(); H2.close()
