"""The rest of the C ABI against the oracle: the paper's table diagnostics and the CSR exports.

* r3mg_stats: H (largest coarsest-box diameter), h (largest coupled-point distance), H/h
  (Section 6, table legend) against ``oracle.mesh_stats`` (same definition, 1e-14 relative);
  the Lanczos Ritz values against the oracle's (1e-11).
* r3mg_cond_estimate: the "Cond." column, from the CG coefficients the solve keeps on the
  device; FP64 PCG against the oracle's PCG estimate (1e-6 relative, same iterations); the
  FP32-V-cycle flexible CG against the oracle's FCG estimate with the FP64 V-cycle (the FP32
  preconditioner differs from the FP64 one at 1e-6, so 1e-3); block solves per column.
* r3mg_set_stop_rule: the paper's stop test (absolute residual < 1e-9 or six orders of
  reduction), against the oracle's PCG with the same rule (iterations +-1) and checked on the
  true residual.
* r3mg_get_transfer_pattern / r3mg_get_level_matrix: structure bit-exact against the oracle's
  structural patterns (P: b entries per row at the owner's columns; A_l: the oracle's block
  pattern expanded to dense b x b blocks), values against the oracle's P and A_l (1e-12).
* r3mg_setup_device: the same hierarchy as r3mg_setup (the V-cycle agrees bit for bit).
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle.hierarchy import Params
from tests.gpu_cases import CASES, make

pytestmark = pytest.mark.gpu


def _hier(P, params, precision=0, **kw):
    import paper_2607_28235_b300 as R
    return R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, precision=precision, **dict(params, **kw))


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    P, params = make(request.param)
    Ho = O.build_hierarchy(P.coords, P.scipy(), Params(params["leaf_size"], params["pprime"], params["levels"],
                                                        cheb_degree=params["cheb_degree"]))
    return P, params, Ho, _hier(P, params)


def test_stats_match_oracle(case):
    P, params, Ho, H = case
    st = H.stats()
    ref = O.mesh_stats(P.coords, P.scipy(), Ho.part)
    for k in ("H", "h", "H_over_h"):
        assert abs(st[k] - ref[k]) <= 1e-14 * ref[k], (k, st[k], ref[k])
    for lev in range(params["levels"] - 1):
        ritz = Ho.lam[lev][1] / Ho.params.eig_safety
        assert abs(st["ritz"][lev] - ritz) <= 1e-11 * ritz
    assert st["ritz"][-1] == 0.0


def test_cond_estimate_fp64_pcg(case):
    P, params, Ho, H = case
    rtol = 1e-10
    x, it, rel = H.pcg(torch.tensor(P.b, device="cuda"), rtol=rtol)
    ref = O.pcg(P.scipy(), P.b, lambda r: O.vcycle(Ho, r), rtol=rtol)
    ce = H.cond_estimate()
    assert it == ref.iterations and ce["steps"] == it
    assert abs(ce["cond"] - ref.cond_estimate) <= 1e-6 * ref.cond_estimate, (ce, ref.cond_estimate)
    assert 0 < ce["lmin"] <= ce["lmax"]


def test_cond_estimate_mixed_fcg(case):
    P, params, Ho, _ = case
    Hm = _hier(P, params, precision=1)
    rtol = 1e-10
    x, it, rel = Hm.pcg(torch.tensor(P.b, device="cuda"), rtol=rtol)
    ref = O.fcg(P.scipy(), P.b, lambda r: O.vcycle(Ho, r), rtol=rtol)
    ce = Hm.cond_estimate()
    assert abs(it - ref.iterations) <= 1
    assert abs(ce["cond"] - ref.cond_estimate) <= 1e-3 * ref.cond_estimate, (ce, ref.cond_estimate)
    Hm.close()


def test_cond_estimate_block_columns(case):
    P, params, Ho, H = case
    rng = np.random.default_rng(31)
    B = np.stack([P.b, rng.standard_normal(P.n), rng.standard_normal(P.n)])
    X, its, rel = H.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-10)
    for c in range(3):
        ref = O.pcg(P.scipy(), B[c], lambda r: O.vcycle(Ho, r), rtol=1e-10)
        ce = H.cond_estimate(c)
        assert abs(its[c] - ref.iterations) <= 1
        assert abs(ce["cond"] - ref.cond_estimate) <= 1e-6 * ref.cond_estimate, (c, ce, ref.cond_estimate)
    with pytest.raises(Exception):
        H.cond_estimate(3)


@pytest.mark.parametrize("atol,red", [(1e-9, 1e-6), (0.0, 1e-4), (1e-6, 0.0)])
def test_paper_stop_rule(case, atol, red):
    P, params, Ho, H = case
    A = P.scipy()
    H.set_stop_rule(atol, red)
    try:
        x, it, rel = H.pcg(torch.tensor(P.b, device="cuda"), rtol=0.0)
        X, its, rels = H.pcg_multi(torch.tensor(np.stack([P.b, 0.5 * P.b]), device="cuda"), rtol=0.0)
    finally:
        H.set_stop_rule(0.0, 0.0)
    ref = O.pcg(A, P.b, lambda r: O.vcycle(Ho, r), rtol=0.0, atol=atol, reduction=red)
    assert ref.converged and abs(it - ref.iterations) <= 1, (it, ref.iterations)
    res = np.linalg.norm(P.b - A @ x.cpu().numpy())
    assert res <= max(atol, red * np.linalg.norm(P.b))
    # per column: the half right-hand side meets the absolute part later than the full one
    for c, scale in ((0, 1.0), (1, 0.5)):
        rc = O.pcg(A, scale * P.b, lambda r: O.vcycle(Ho, r), rtol=0.0, atol=atol, reduction=red)
        assert abs(its[c] - rc.iterations) <= 1, (c, its[c], rc.iterations)
    # the default rule again: relative
    x2, it2, rel2 = H.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-10)
    assert rel2 <= 1e-10


def test_transfer_pattern_matches_oracle(case):
    P, params, Ho, H = case
    b = H.b
    for lev in range(params["levels"] - 1):
        rp, cols, vals = H.transfer_pattern(lev)
        ref = Ho.P[lev].tocsr()
        n = ref.shape[0]
        assert np.array_equal(rp, np.arange(n + 1) * b)
        # structural pattern: the owner box's b coarse DoFs (the oracle keeps structural zeros)
        owner = Ho.part.box_of_point[1] if lev == 0 else (np.arange(n) // b) // (1 << P.dim)
        want = (owner[:, None] * b + np.arange(b)[None, :]).ravel()
        assert np.array_equal(cols, want)
        dense = ref.toarray()
        got = np.zeros_like(dense)
        got[np.repeat(np.arange(n), b), cols] = vals
        assert np.max(np.abs(got - dense)) <= 1e-12


def test_level_matrix_matches_oracle(case):
    P, params, Ho, H = case
    b = H.b
    for lev in range(1, params["levels"]):
        rp, cols, vals = H.level_matrix(lev)
        pat = Ho.patterns[lev]
        n = len(pat) * b
        want_rp = [0]
        want_cols = []
        for B, nbrs in enumerate(pat):
            row = (np.asarray(nbrs)[:, None] * b + np.arange(b)[None, :]).ravel()
            for q in range(b):
                want_cols.append(row)
                want_rp.append(want_rp[-1] + len(row))
        assert np.array_equal(rp, want_rp)
        assert np.array_equal(cols, np.concatenate(want_cols))
        dense = Ho.A[lev].toarray()
        rows = np.repeat(np.arange(n), np.diff(rp))
        assert np.max(np.abs(vals - dense[rows, cols])) <= 1e-12 * np.abs(dense).max()
        # and nothing of A_l lies outside the exported pattern
        got = np.zeros_like(dense)
        got[rows, cols] = vals
        assert np.max(np.abs(got - dense)) <= 1e-12 * np.abs(dense).max()


def test_setup_from_device_csr(case):
    """Device CSR in, the same hierarchy out (fixed kernel form so both run identical kernels)."""
    import paper_2607_28235_b300 as R
    P, params, Ho, _ = case
    Hh = _hier(P, params, kernel_form=1)
    Hd = R.Hierarchy(P.coords, torch.tensor(P.rowptr, device="cuda"), torch.tensor(P.colidx, device="cuda"),
                     torch.tensor(P.vals, device="cuda"), **dict(params, kernel_form=1))
    r = torch.tensor(np.random.default_rng(32).standard_normal(P.n), device="cuda")
    for lev in range(1, params["levels"]):
        assert np.array_equal(Hd.agglomerates(lev), Hh.agglomerates(lev))
    assert torch.equal(Hd.vcycle(r), Hh.vcycle(r))
    sd, sh = Hd.stats(), Hh.stats()
    assert sd["H"] == sh["H"] and sd["h"] == sh["h"] and np.array_equal(sd["ritz"], sh["ritz"])
    assert Hd.device_status() == 0
    Hd.close(); Hh.close()
