"""GPU path (through the C ABI) against the CPU oracle, element by element.

Tolerances (FP64 path): structure bit-exact; P values 1e-14 absolute (products of
O(1) Lagrange factors); Galerkin blocks and level products 1e-12 relative to the
largest entry (sums of O(nnz_row * b) FP64 terms in a different order); one
V-cycle 1e-12 relative (2-norm); PCG iterations +-1 and the solution within
1e-10 relative of the oracle's.  FP32 V-cycle: the flexible CG still reaches
the FP64 tolerance; its solution is compared with the oracle's at rtol * 1e3.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle.hierarchy import Params
from tests.gpu_cases import CASES, make

pytestmark = pytest.mark.gpu


def _hier(P, params, precision=0):
    import paper_2607_28235_b300 as R
    return R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, precision=precision, **params)


def _oracle(P, params):
    return O.build_hierarchy(P.coords, P.scipy(), Params(params["leaf_size"], params["pprime"], params["levels"],
                                                          cheb_degree=params["cheb_degree"]))


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    P, params = make(request.param)
    return P, params, _hier(P, params), _oracle(P, params)


def test_agglomerates_and_patterns_bit_exact(pair):
    P, params, H, Ho = pair
    for lev in range(1, params["levels"]):
        assert np.array_equal(H.agglomerates(lev), Ho.part.box_of_point[lev])
        ptr, nbr = H.level_pattern(lev)
        ref = Ho.patterns[lev]
        assert np.array_equal(np.diff(ptr), [len(v) for v in ref])
        assert np.array_equal(nbr, np.concatenate(ref))


def test_prolongation_values(pair):
    P, params, H, Ho = pair
    b = H.b
    P0 = H.prolongation(0)
    ref = Ho.P[0].toarray()
    box = Ho.part.box_of_point[1]
    got = np.zeros_like(ref)
    for q in range(b):
        got[np.arange(P.n), box * b + q] = P0[:, q]
    assert np.max(np.abs(got - ref)) <= 1e-14
    for lev in range(1, params["levels"] - 1):
        Pt = H.prolongation(lev)
        R = Ho.P[lev].toarray()
        fan = 1 << P.dim
        for c in range(Pt.shape[0]):
            Bp = c // fan
            assert np.max(np.abs(Pt[c] - R[c * b:(c + 1) * b, Bp * b:(Bp + 1) * b])) <= 1e-14


def test_galerkin_blocks(pair):
    P, params, H, Ho = pair
    b = H.b
    for lev in range(1, params["levels"]):
        blocks = H.level_blocks(lev)
        ptr, nbr = H.level_pattern(lev)
        ref = Ho.A[lev].toarray()
        got = np.zeros_like(ref)
        for B in range(len(ptr) - 1):
            for e in range(ptr[B], ptr[B + 1]):
                got[B * b:(B + 1) * b, nbr[e] * b:(nbr[e] + 1) * b] = blocks[e]
        scale = np.abs(ref).max()
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (lev, np.max(np.abs(got - ref)) / scale)


def test_level_apply_and_lambda(pair):
    P, params, H, Ho = pair
    info = H.info()
    rng = np.random.default_rng(1)
    for lev in range(params["levels"]):
        A = Ho.A[lev]
        x = rng.standard_normal(A.shape[0])
        y = H.level_apply(lev, torch.tensor(x, device="cuda")).cpu().numpy()
        ref = A @ x
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
        if lev < params["levels"] - 1:
            assert abs(info["lam_hi"][lev] - Ho.lam[lev][1]) <= 1e-11 * Ho.lam[lev][1]


def test_coarsest_solve(pair):
    """The coarsest solve (explicit inverse from the dense Cholesky factor) against the oracle's
    Cholesky solve, within cond(A_c) * 1e-14 relative (forming and applying the inverse and the
    two triangular solves each err by a modest multiple of cond(A_c) * eps)."""
    P, params, H, Ho = pair
    Ac = Ho.A[-1].toarray()
    r = np.random.default_rng(9).standard_normal(Ac.shape[0])
    z = H.coarse_solve(torch.tensor(r, device="cuda")).cpu().numpy()
    ref = O.cholesky_solve(Ho.Lc, r)
    tol = 1e-14 * np.linalg.cond(Ac)
    assert np.linalg.norm(z - ref) <= tol * np.linalg.norm(ref), (np.linalg.norm(z - ref) / np.linalg.norm(ref), tol)
    assert np.linalg.norm(Ac @ z - r) <= tol * np.linalg.norm(Ac) * np.linalg.norm(z)


def test_vcycle_fp64_parity(pair):
    P, params, H, Ho = pair
    rng = np.random.default_rng(2)
    for trial in range(2):
        r = rng.standard_normal(P.n) if trial else P.b.copy()
        z = H.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
        ref = O.vcycle(Ho, r)
        err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
        assert err <= 1e-12, err
        # twice in a row gives the same bits (graph replay is deterministic)
        z2 = H.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
        assert np.array_equal(z, z2)


def test_pcg_fp64_parity(pair):
    P, params, H, Ho = pair
    rtol = 1e-10
    x, it, rel = H.pcg(torch.tensor(P.b, device="cuda"), rtol=rtol)
    ref = O.pcg(P.scipy(), P.b, lambda r: O.vcycle(Ho, r), rtol=rtol)
    assert abs(it - ref.iterations) <= 1, (it, ref.iterations)
    x = x.cpu().numpy()
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x) * max(1.0, 1e10 * rtol)
    assert np.linalg.norm(P.b - P.scipy() @ x) <= rtol * np.linalg.norm(P.b)


def test_pcg_mixed_precision(pair):
    P, params, H, Ho = pair
    Hm = _hier(P, params, precision=1)
    rtol = 1e-10
    x, it, rel = Hm.pcg(torch.tensor(P.b, device="cuda"), rtol=rtol)
    ref = O.pcg(P.scipy(), P.b, lambda r: O.vcycle(Ho, r), rtol=rtol)
    x = x.cpu().numpy()
    assert np.linalg.norm(P.b - P.scipy() @ x) <= rtol * np.linalg.norm(P.b)
    assert np.linalg.norm(x - ref.x) <= 1e3 * rtol * np.linalg.norm(ref.x)
    assert it <= ref.iterations + 3
    Hm.close()


def test_pcg_host_buffers(pair):
    P, params, H, Ho = pair
    x, it, rel = H.pcg_host(P.b, rtol=1e-9)
    assert np.linalg.norm(P.b - P.scipy() @ x) <= 1e-9 * np.linalg.norm(P.b)


def test_initial_guess_and_zero_rhs(pair):
    P, params, H, Ho = pair
    xs = np.linalg.solve(P.scipy().toarray(), P.b) if P.n < 3000 else None
    x0 = torch.tensor(P.b * 0.0, device="cuda")
    x, it, rel = H.pcg(torch.zeros(P.n, dtype=torch.float64, device="cuda"), x0=x0)
    assert it == 0 and float(x.abs().max()) == 0.0
    if xs is not None:
        x, it, rel = H.pcg(torch.tensor(P.b, device="cuda"), x0=torch.tensor(xs, device="cuda"), rtol=1e-8)
        assert it == 0


@pytest.mark.parametrize("form", [1, 2])
def test_kernel_forms_match_oracle(pair, form):
    """Both level-operator kernels (register-streamed, TMA-streamed) give the oracle's V-cycle."""
    P, params, H, Ho = pair
    Hf = _hier(P, dict(params, kernel_form=form))
    r = np.random.default_rng(7).standard_normal(P.n)
    z = Hf.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    ref = O.vcycle(Ho, r)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    Hf.close()


@pytest.mark.parametrize("form", ["register", "tma", "register_persistent", "register_l2_prefetch", "symmetric_block",
                                  "register_pipelined", "register_pipelined_l2_prefetch", "symmetric_block_staged"])
def test_set_kernel_config_each_form(pair, form):
    """Every kernel form, pinned through r3mg_set_kernel_config, gives a converged mixed-precision
    PCG (the symmetric block form exists on coarse FP32 levels only)."""
    P, params, H, Ho = pair
    Hf = _hier(P, params, precision=1)
    cfg = Hf.kernel_config()
    for lev, row in enumerate(cfg[:-1]):
        for key in ("f64", "f32"):
            if form.startswith("symmetric_block") and (lev == 0 or key == "f64"):
                continue
            if form == "symmetric_block_staged":    # lanes field: CTAs per SM
                row[key] = {"form": form, "lanes": 4, "threads": 128}
                continue
            row[key] = {"form": form, "lanes": row[key]["lanes"] if row[key]["lanes"] >= 4 else 16, "threads": 512}
    try:
        Hf.set_kernel_config(cfg[:-1])
    except Exception as e:       # a form a level cannot host (windows too large for two buffers)
        pytest.skip(str(e))
    got = Hf.kernel_config()
    first = 1 if form.startswith("symmetric_block") else 0
    assert all(got[l]["f32"]["form"] == form for l in range(first, len(cfg) - 1))
    x, it, rel = Hf.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-10)
    assert np.linalg.norm(P.b - P.scipy() @ x.cpu().numpy()) <= 1e-10 * np.linalg.norm(P.b)
    Hf.close()


def test_symmetric_block_form_vcycle_matches_full_form(pair):
    """The symmetric block form of the coarse FP32 levels gives the same V-cycle as the full form
    to FP32 rounding (same operator; the transposed blocks are taken from the upper ones)."""
    P, params, H, Ho = pair
    if params["levels"] < 3:
        pytest.skip("no smoothed coarse level")
    Hf = _hier(P, dict(params, kernel_form=1), precision=1)
    Hs = _hier(P, dict(params, kernel_form=1), precision=1)
    cfg = Hs.kernel_config()
    for lev in range(1, len(cfg) - 1):
        cfg[lev]["f32"] = {"form": "symmetric_block", "lanes": 16, "threads": 128}
    Hs.set_kernel_config(cfg[:-1])
    r = torch.tensor(np.random.default_rng(3).standard_normal(P.n), device="cuda")
    zf = Hf.vcycle(r).cpu().numpy()
    zs = Hs.vcycle(r).cpu().numpy()
    assert np.linalg.norm(zs - zf) <= 1e-5 * np.linalg.norm(zf)
    zs2 = Hs.vcycle(r).cpu().numpy()
    assert np.array_equal(zs, zs2)     # deterministic
    Hf.close(); Hs.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_loop_graph_matches_host_loop(pair, precision):
    """The solve loop as one conditional-graph launch (profiling off) and the host-driven loop
    (profiling on) run the same kernels in the same order on the same hierarchy (same tuned
    kernel configurations): same iterations, same bits."""
    P, params, H, Ho = pair
    Hg = _hier(P, params, precision=precision)
    b = torch.tensor(P.b, device="cuda")
    xg, itg, _ = Hg.pcg(b, rtol=1e-10)
    xg2, itg2, _ = Hg.pcg(b, rtol=1e-10)          # replay of the captured loop
    bg, ibg, _ = Hg.pcg(b, rtol=1e-14, maxit=2, raise_on_noconv=False)
    Hg.profile(True)
    xh, ith, _ = Hg.pcg(b, rtol=1e-10)
    bh, ibh, _ = Hg.pcg(b, rtol=1e-14, maxit=2, raise_on_noconv=False)
    Hg.profile(False)
    assert itg == ith == itg2 and itg > 0
    assert torch.equal(xg, xh) and torch.equal(xg, xg2)
    # a budget the loop cannot meet: stops after exactly maxit iterations, same bits again
    assert ibg == ibh == 2
    assert torch.equal(bg, bh)
    Hg.close()


def test_update_values_recaptures(pair):
    """New values on the same pattern (A2 = D A D, D positive diagonal) after graphs were captured:
    the V-cycle and the solve follow the oracle's hierarchy of A2, not the old coefficients."""
    P, params, H, Ho = pair
    Hu = _hier(P, params)
    r = np.random.default_rng(5).standard_normal(P.n)
    Hu.vcycle(torch.tensor(r, device="cuda"))
    Hu.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-8)
    d = np.random.default_rng(6).uniform(0.5, 2.0, P.n)
    rows = np.repeat(np.arange(P.n), np.diff(P.rowptr))
    vals2 = d[rows] * P.vals * d[P.colidx]
    Hu.update_values(torch.tensor(vals2, device="cuda"))
    A2 = P.scipy().copy()
    A2.data = vals2.copy()
    Ho2 = O.build_hierarchy(P.coords, A2, Params(params["leaf_size"], params["pprime"], params["levels"],
                                                 cheb_degree=params["cheb_degree"]))
    z = Hu.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    ref = O.vcycle(Ho2, r)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    x, it, rel = Hu.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-10)
    refs = O.pcg(A2, P.b, lambda v: O.vcycle(Ho2, v), rtol=1e-10)
    assert abs(it - refs.iterations) <= 1
    assert np.linalg.norm(P.b - A2 @ x.cpu().numpy()) <= 1e-10 * np.linalg.norm(P.b)
    Hu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_coarse_substitution_form(pair, precision):
    """The coarsest solve by forward and back substitution with the Cholesky factor (the
    oracle's own method) against the oracle, and the V-cycle with it against the V-cycle with
    the explicit inverse: the two forms of A_c^{-1} differ by kappa(A_c) eps at most."""
    P, params, H, Ho = pair
    Hc = _hier(P, params, precision=precision)
    Ac = Ho.A[-1].toarray()
    kappa = np.linalg.cond(Ac)
    r = np.random.default_rng(19).standard_normal(Ac.shape[0])
    z0 = Hc.coarse_solve(torch.tensor(r, device="cuda"), fp32=bool(precision)).cpu().numpy()
    rv = np.random.default_rng(20).standard_normal(P.n)
    v0 = Hc.vcycle(torch.tensor(rv, device="cuda")).cpu().numpy()
    Hc.set_coarse_mode(1)
    z1 = Hc.coarse_solve(torch.tensor(r, device="cuda"), fp32=bool(precision)).cpu().numpy()
    v1 = Hc.vcycle(torch.tensor(rv, device="cuda")).cpu().numpy()
    ref = O.cholesky_solve(Ho.Lc, r)
    eps = 2.0 ** -53 if precision == 0 else 2.0 ** -24
    tol = 64 * eps * kappa
    assert np.linalg.norm(z1 - ref) <= tol * np.linalg.norm(ref), (np.linalg.norm(z1 - ref) / np.linalg.norm(ref), tol)
    assert np.linalg.norm(z0 - z1) <= tol * np.linalg.norm(ref)
    assert np.linalg.norm(v1 - v0) <= tol * np.linalg.norm(v0)
    if precision == 0:
        assert np.linalg.norm(v1 - O.vcycle(Ho, rv)) <= 1e-12 * np.linalg.norm(v1)
    x, it, rel = Hc.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-10)
    assert rel <= 1e-10
    Hc.set_coarse_mode(0)
    Hc.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_every_lane_count_on_every_level(pair, fp32):
    """The register kernel with 2 (FP64 fine level only), 4, 8, 16 and 32 lanes per row (32 on
    coarse levels only) and 128 or 256 threads gives the oracle's level products on every
    smoothed level: FP64 within 1e-12 of the largest entry of the result, FP32 within the
    row-wise rounding bound (row entries + 2) 2^-24 (|A||x|)_i."""
    P, params, H, Ho = pair
    Hx = _hier(P, params, precision=1) if fp32 else H
    key = "f32" if fp32 else "f64"
    rng = np.random.default_rng(61)
    L = params["levels"]
    for lanes in (2, 4, 8, 16, 32):
        for threads in (128, 256):
            cfg = Hx.kernel_config()
            levels = [l for l in range(L - 1) if not (l == 0 and lanes == 32) and not (lanes == 2 and (l > 0 or fp32))]
            if not levels:
                continue
            for lev in levels:
                cfg[lev][key] = {"form": "register", "lanes": lanes, "threads": threads}
            Hx.set_kernel_config(cfg[:-1])
            for lev in levels:
                A = Ho.A[lev]
                x = rng.standard_normal(A.shape[0])
                if fp32:
                    x = x.astype(np.float32).astype(np.float64)
                y = Hx.level_apply(lev, torch.tensor(x, device="cuda"), fp32=fp32).cpu().numpy()
                ref = A @ x
                if fp32:
                    bound = (np.diff(A.indptr) + 2) * 2.0 ** -24 * (abs(A) @ np.abs(x))
                    assert np.all(np.abs(y - ref) <= bound), (lev, lanes, threads)
                else:
                    assert np.max(np.abs(y - ref)) <= 1e-12 * np.abs(ref).max(), (lev, lanes, threads)
    if fp32:
        Hx.close()
