"""Several right-hand sides on one hierarchy (block vectors, through the C ABI) against the oracle,
column by column.

Tolerances: FP64 block level products 1e-13 relative (as the single-vector product); FP32 block
products within (row entries + 2) * 2^-24 * (|A| |x|)_i per row, the rounding bound of a
length-k FP32 dot product with rounded inputs; FP64 block V-cycle 1e-12 relative per column;
FP32 block V-cycle no less accurate against the FP64 oracle than the single-vector FP32
V-cycle (4x its error, plus 4 x 3 * 2^-20 relative where a coarse level runs on the tensor
cores, whose TF32 operand splitting costs up to 3 * 2^-20 per product); PCG per column: iterations +-1 and the solution within 1e-10 relative
of the oracle's PCG (FP64), or the FP64 residual reached and the solution within 1e3 * rtol (FP32
V-cycle inside FCG).
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


def _oracle(P, params, A=None):
    return O.build_hierarchy(P.coords, P.scipy() if A is None else A,
                             Params(params["leaf_size"], params["pprime"], params["levels"],
                                    cheb_degree=params["cheb_degree"]))


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def trio(request):
    P, params = make(request.param)
    return P, params, _hier(P, params), _hier(P, params, precision=1), _oracle(P, params)


def _rhs(P, m, seed):
    B = np.random.default_rng(seed).standard_normal((m, P.n))
    B[0] = P.b
    return B


@pytest.mark.parametrize("m", [1, 5, 16])
def test_block_level_products(trio, m):
    P, params, H, Hm, Ho = trio
    rng = np.random.default_rng(10 + m)
    for lev in range(params["levels"]):
        A = Ho.A[lev]
        X = rng.standard_normal((m, A.shape[0]))
        ref = (A @ X.T).T
        Y = H.level_apply_multi(lev, torch.tensor(X, device="cuda")).cpu().numpy()
        for c in range(m):
            assert np.linalg.norm(Y[c] - ref[c]) <= 1e-13 * np.linalg.norm(ref[c]), (lev, c)
        if lev == params["levels"] - 1:          # the coarsest level has no FP32 values
            with pytest.raises(RuntimeError):
                Hm.level_apply_multi(lev, torch.tensor(X, device="cuda"), fp32=True)
            continue
        # FP32 values and inputs, FP32 accumulation; the bound of the form the tuner chose
        # (the tensor-core form adds its TF32 head/tail splitting error, see below)
        Y32 = Hm.level_apply_multi(lev, torch.tensor(X, device="cuda"), fp32=True).cpu().numpy()
        absA = abs(A)
        k = np.diff(A.indptr)
        form = Hm.block_config(fp32=True)[min(lev, params["levels"] - 2)]
        kk = 2 * k + 64 if form == 3 else k + 2
        for c in range(m):
            bound = kk * 2.0 ** -24 * (absA @ np.abs(X[c]))
            assert np.all(np.abs(Y32[c] - ref[c]) <= bound), (lev, c, form)


@pytest.mark.parametrize("m", [3, 16])
def test_block_vcycle(trio, m):
    P, params, H, Hm, Ho = trio
    R = _rhs(P, m, 20 + m)
    Z = H.vcycle_multi(torch.tensor(R, device="cuda")).cpu().numpy()
    Z32 = Hm.vcycle_multi(torch.tensor(R, device="cuda")).cpu().numpy()
    # where the tuner put a coarse level on the tensor cores, their operand splitting costs up
    # to 3 * 2^-20 relative per product (against 2^-24 for FP32 rounding): allow 4x that,
    # relative to the result, on top of the single-vector FP32 V-cycle's error
    cfg = Hm.block_config(fp32=True)
    extra = 4 * 3 * 2.0 ** -20 if any(f == 3 for f in cfg[1:params["levels"] - 1]) else 1e-7
    for c in range(m):
        ref = O.vcycle(Ho, R[c])
        assert np.linalg.norm(Z[c] - ref) <= 1e-12 * np.linalg.norm(ref), c
        single32 = Hm.vcycle(torch.tensor(R[c], device="cuda")).cpu().numpy()
        e1 = np.linalg.norm(single32 - ref)
        e2 = np.linalg.norm(Z32[c] - ref)
        assert e2 <= 4 * e1 + extra * np.linalg.norm(ref), (c, e1, e2, cfg)
    # a replay gives the same bits
    Z2 = H.vcycle_multi(torch.tensor(R, device="cuda")).cpu().numpy()
    assert np.array_equal(Z, Z2)


def test_block_pcg_fp64_per_column(trio):
    P, params, H, Hm, Ho = trio
    m, rtol = 16, 1e-10
    B = _rhs(P, m, 31)
    X, its, rel = H.pcg_multi(torch.tensor(B, device="cuda"), rtol=rtol)
    X = X.cpu().numpy()
    A = P.scipy()
    for c in range(m):
        ref = O.pcg(A, B[c], lambda r: O.vcycle(Ho, r), rtol=rtol)
        assert abs(int(its[c]) - ref.iterations) <= 1, (c, its[c], ref.iterations)
        assert np.linalg.norm(X[c] - ref.x) <= 1e-10 * np.linalg.norm(ref.x), c
        assert np.linalg.norm(B[c] - A @ X[c]) <= rtol * np.linalg.norm(B[c]), c
        assert rel[c] <= rtol


def test_block_pcg_mixed_per_column(trio):
    P, params, H, Hm, Ho = trio
    m, rtol = 16, 1e-10
    B = _rhs(P, m, 32)
    X, its, rel = Hm.pcg_multi(torch.tensor(B, device="cuda"), rtol=rtol)
    X = X.cpu().numpy()
    A = P.scipy()
    for c in range(m):
        ref = O.pcg(A, B[c], lambda r: O.vcycle(Ho, r), rtol=rtol)
        assert np.linalg.norm(B[c] - A @ X[c]) <= rtol * np.linalg.norm(B[c]), c
        assert np.linalg.norm(X[c] - ref.x) <= 1e3 * rtol * np.linalg.norm(ref.x), c
        assert its[c] <= ref.iterations + 3, (c, its[c], ref.iterations)


def test_block_pcg_edge_columns(trio):
    """A zero right-hand side, an exact initial guess and ordinary columns side by side; one
    column (m = 1, padded block) agrees with the single-vector solve."""
    P, params, H, Hm, Ho = trio
    A = P.scipy()
    m = 5
    B = _rhs(P, m, 33)
    B[2] = 0.0
    X0 = np.zeros_like(B)
    if P.n < 3000:
        X0[3] = np.linalg.solve(A.toarray(), B[3])
    X, its, rel = H.pcg_multi(torch.tensor(B, device="cuda"), X0=torch.tensor(X0, device="cuda"), rtol=1e-9)
    X = X.cpu().numpy()
    assert its[2] == 0 and np.all(X[2] == 0.0) and rel[2] == 0.0
    if P.n < 3000:
        assert its[3] == 0
    for c in (0, 1, 4):
        assert np.linalg.norm(B[c] - A @ X[c]) <= 1e-9 * np.linalg.norm(B[c])
    x1, it1, _ = H.pcg(torch.tensor(P.b, device="cuda"), rtol=1e-10)
    Xs, itss, _ = H.pcg_multi(torch.tensor(P.b[None, :], device="cuda"), rtol=1e-10)
    assert abs(int(itss[0]) - it1) <= 1
    assert torch.allclose(Xs[0], x1, rtol=0, atol=1e-9 * float(x1.abs().max()))


def test_block_pcg_budget_and_arguments(trio):
    P, params, H, Hm, Ho = trio
    B = torch.tensor(_rhs(P, 4, 34), device="cuda")
    X, its, rel = H.pcg_multi(B, rtol=1e-15, maxit=2, raise_on_noconv=False)
    assert np.all(its == 2)
    with pytest.raises(RuntimeError):
        H.pcg_multi(torch.zeros((17, P.n), dtype=torch.float64, device="cuda"))


def test_block_pcg_after_update_values(trio):
    """New values on the same pattern after the block loop graph was captured."""
    P, params, H, Hm, Ho = trio
    Hu = _hier(P, params)
    B = _rhs(P, 4, 35)
    Hu.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-8)
    d = np.random.default_rng(36).uniform(0.5, 2.0, P.n)
    rows = np.repeat(np.arange(P.n), np.diff(P.rowptr))
    vals2 = d[rows] * P.vals * d[P.colidx]
    Hu.update_values(torch.tensor(vals2, device="cuda"))
    A2 = P.scipy().copy()
    A2.data = vals2.copy()
    Ho2 = _oracle(P, params, A2)
    X, its, rel = Hu.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-10)
    X = X.cpu().numpy()
    for c in range(4):
        ref = O.pcg(A2, B[c], lambda r: O.vcycle(Ho2, r), rtol=1e-10)
        assert abs(int(its[c]) - ref.iterations) <= 1
        assert np.linalg.norm(B[c] - A2 @ X[c]) <= 1e-10 * np.linalg.norm(B[c])
    Hu.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_block_kernel_forms_on_coarse_levels(trio, fp32):
    """Every coarse-level block kernel (window gathered through L1 with 2/4/8 entry slots, window
    staged in shared memory, block rows streamed by the copy engine, tensor cores through mma.sync,
    through tcgen05 with a TMEM accumulator, and through the warp-specialised tcgen05 kernel with
    the A operand in TMEM) gives the oracle's products."""
    P, params, H, Hm, Ho = trio
    Hx = Hm if fp32 else H
    m = 16
    rng = np.random.default_rng(40)
    X0 = torch.tensor(rng.standard_normal((m, P.n)), device="cuda")
    Hx.vcycle_multi(X0)                                     # tunes the block kernels
    for lev in range(1, params["levels"] - 1):
        A = Ho.A[lev]
        X = rng.standard_normal((m, A.shape[0]))
        ref = (A @ X.T).T
        absA = abs(A)
        k = np.diff(A.indptr)
        for slots in (6, 5, 3, 1, 0, 2, 4, 8):
            if not fp32 and slots == 8:
                continue                                    # FP64, 16 columns: 8 lanes per row slice
            if not fp32 and slots in (3, 5, 6):
                with pytest.raises(RuntimeError):           # the tensor-core form is FP32 only
                    Hx.set_block_config(lev, slots, fp32=fp32)
                continue
            Hx.set_block_config(lev, slots, fp32=fp32)
            assert Hx.block_config(fp32=fp32)[lev] == slots
            Y = Hx.level_apply_multi(lev, torch.tensor(X, device="cuda"), fp32=fp32).cpu().numpy()
            assert Hx.device_status() == 0, (lev, slots)     # no bounded wait of the kernel ran out
            for c in range(m):
                if fp32:
                    # FP32 dot-product rounding; the tensor-core form adds its TF32 head/tail
                    # splitting error (at most 3 * 2^-20 = 48 * 2^-24 per product, truncation) and
                    # tensor-core accumulation (taken as 2 units of 2^-24 per entry)
                    kk = 2 * k + 64 if slots in (3, 5, 6) else k + 2
                    bound = kk * 2.0 ** -24 * (absA @ np.abs(X[c]))
                    assert np.all(np.abs(Y[c] - ref[c]) <= bound), (lev, slots, c)
                else:
                    assert np.linalg.norm(Y[c] - ref[c]) <= 1e-13 * np.linalg.norm(ref[c]), (lev, slots, c)
        # the V-cycle with the staged form on this level still matches the oracle (FP64) or
        # converges (FP32 inside FCG)
        Hx.set_block_config(lev, 0, fp32=fp32)
    B = _rhs(P, 4, 41)
    X, its, rel = Hx.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-10)
    Xc = X.cpu().numpy()
    for c in range(4):
        assert np.linalg.norm(B[c] - P.scipy() @ Xc[c]) <= 1e-10 * np.linalg.norm(B[c])


@pytest.mark.parametrize("fp32", [False, True])
def test_block_kernel_forms_on_the_fine_level(trio, fp32):
    """Fine-level block kernels: window map in shared memory (2/4/8 entry slots), the flat row
    sweep on global column indices (12/14/18) and the groups of rows with equal column lists (20)
    give the oracle's product."""
    P, params, H, Hm, Ho = trio
    Hx = Hm if fp32 else H
    m = 16
    rng = np.random.default_rng(42)
    Hx.vcycle_multi(torch.tensor(rng.standard_normal((m, P.n)), device="cuda"))
    A = Ho.A[0]
    X = rng.standard_normal((m, P.n))
    ref = (A @ X.T).T
    absA = abs(A)
    k = np.diff(A.indptr)
    for slots in (2, 4, 8, 12, 14, 18, 20):
        if not fp32 and slots in (8, 18):
            continue                                       # FP64, 16 columns: 8 lanes per row slice
        Hx.set_block_config(0, slots, fp32=fp32)
        Y = Hx.level_apply_multi(0, torch.tensor(X, device="cuda"), fp32=fp32).cpu().numpy()
        for c in range(m):
            if fp32:
                bound = (k + 2) * 2.0 ** -24 * (absA @ np.abs(X[c]))
                assert np.all(np.abs(Y[c] - ref[c]) <= bound), (slots, c)
            else:
                assert np.linalg.norm(Y[c] - ref[c]) <= 1e-13 * np.linalg.norm(ref[c]), (slots, c)
    Hx.set_block_config(0, 14, fp32=fp32)
    B = _rhs(P, 4, 43)
    Xs, its, rel = Hx.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-10)
    Xs = Xs.cpu().numpy()
    for c in range(4):
        assert np.linalg.norm(B[c] - P.scipy() @ Xs[c]) <= 1e-10 * np.linalg.norm(B[c])


def test_grouped_fine_level_follows_value_updates(trio):
    """The grouped fine level keeps its own entry-major copy of the values; after new matrix values
    (here 2 A, which scales every product exactly) the block product uses them, and the block
    solve with the grouped form still converges."""
    P, params, H, Hm, Ho = trio
    m = 16
    rng = np.random.default_rng(77)
    X = torch.tensor(rng.standard_normal((m, P.n)), device="cuda")
    for Hx, fp32 in ((H, False), (Hm, True)):
        Hx.vcycle_multi(torch.tensor(rng.standard_normal((m, P.n)), device="cuda"))
        Hx.set_block_config(0, 20, fp32=fp32)
        assert Hx.block_config(fp32=fp32)[0] == 20
        Y1 = Hx.level_apply_multi(0, X, fp32=fp32)
        try:
            Hx.update_values(torch.tensor(2.0 * P.vals, device="cuda"))
            Y2 = Hx.level_apply_multi(0, X, fp32=fp32)
        finally:
            Hx.update_values(torch.tensor(P.vals, device="cuda"))
        assert torch.equal(Y2, 2.0 * Y1)
        assert torch.equal(Hx.level_apply_multi(0, X, fp32=fp32), Y1)
        B = _rhs(P, m, 44)                       # 16 columns: the grouped form stays configured
        Xs, its, rel = Hx.pcg_multi(torch.tensor(B, device="cuda"), rtol=1e-10)
        assert Hx.block_config(fp32=fp32)[0] == 20
        Xs = Xs.cpu().numpy()
        for c in range(m):
            assert np.linalg.norm(B[c] - P.scipy() @ Xs[c]) <= 1e-10 * np.linalg.norm(B[c])
        Hx.set_block_config(0, 4, fp32=fp32)


@pytest.mark.parametrize("precision", [0, 1])
def test_block_loop_graph_matches_host_loop(trio, precision):
    """The block solve loop as one conditional-graph launch and the profiled, host-driven loop run
    the same kernels in the same order: same iterations per column, same bits."""
    P, params, H, Hm, Ho = trio
    Hx = Hm if precision else H
    B = torch.tensor(_rhs(P, 6, 44), device="cuda")
    Xg, itg, _ = Hx.pcg_multi(B, rtol=1e-10)
    Hx.profile(True)
    Xh, ith, _ = Hx.pcg_multi(B, rtol=1e-10)
    Hx.profile(False)
    assert np.array_equal(itg, ith) and np.all(itg > 0)
    assert torch.equal(Xg, Xh)
