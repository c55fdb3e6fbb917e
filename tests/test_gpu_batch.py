"""Batched solves: independent problems of uneven size in one block-diagonal hierarchy.

Every problem of the batch must behave exactly as if solved alone: agglomerates bit-exact
against the oracle's partition of that problem, one batched V-cycle equal (1e-12 relative) to
the oracle V-cycle of each problem, PCG iteration counts within +-1 of the oracle's and
solutions within 1e-10 (FP64 V-cycle) or reaching the tolerance (FP32 V-cycle).  The loop of
the batched solve is one graph launch; a second call reuses the graph and reproduces the result.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.hierarchy import Params

pytestmark = pytest.mark.gpu

SPECS = [(10, 1), (13, 2), (6, 4), (16, 1), (9, 3), (7, 2)]   # (N, p) of uneven 2D problems
PRM = dict(leaf_size=24, pprime=1, levels=3, cheb_degree=3)


@pytest.fixture(scope="module")
def batch():
    import paper_2607_28235_b300 as R
    probs = [W.poisson(2, N, p, perturb=0.15, seed=100 + k) for k, (N, p) in enumerate(SPECS)]
    rng = np.random.default_rng(9)
    bs = [rng.standard_normal(P.n) for P in probs]
    H = R.BatchHierarchy([(P.coords, P.rowptr, P.colidx, P.vals) for P in probs], **PRM)
    Hm = R.BatchHierarchy([(P.coords, P.rowptr, P.colidx, P.vals) for P in probs], precision=1, **PRM)
    orc = [O.build_hierarchy(P.coords, P.scipy(), Params(PRM["leaf_size"], PRM["pprime"], PRM["levels"],
                                                         cheb_degree=PRM["cheb_degree"])) for P in probs]
    return probs, bs, H, Hm, orc


def test_offsets_and_agglomerates(batch):
    probs, bs, H, Hm, orc = batch
    off = H.level_offsets(0)
    assert np.array_equal(np.diff(off), [P.n for P in probs])
    for lev in (1, 2):
        agg = H.agglomerates(lev)
        boxoff = H.level_offsets(lev) // H.b
        for k, (P, Ho) in enumerate(zip(probs, orc)):
            assert np.array_equal(agg[off[k]:off[k + 1]] - boxoff[k], Ho.part.box_of_point[lev])


def test_batched_vcycle_equals_each_problem(batch):
    probs, bs, H, Hm, orc = batch
    off = H.level_offsets(0)
    r = np.concatenate(bs)
    z = H.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    for k, Ho in enumerate(orc):
        ref = O.vcycle(Ho, bs[k])
        zk = z[off[k]:off[k + 1]]
        assert np.linalg.norm(zk - ref) <= 1e-12 * np.linalg.norm(ref), k


def test_batched_pcg_fp64(batch):
    probs, bs, H, Hm, orc = batch
    off = H.level_offsets(0)
    b = torch.tensor(np.concatenate(bs), device="cuda")
    x, its, rel = H.pcg(b, rtol=1e-10)
    x = x.cpu().numpy()
    for k, (P, Ho) in enumerate(zip(probs, orc)):
        ref = O.pcg(P.scipy(), bs[k], lambda v: O.vcycle(Ho, v), rtol=1e-10)
        assert abs(int(its[k]) - ref.iterations) <= 1, (k, its[k], ref.iterations)
        xk = x[off[k]:off[k + 1]]
        assert np.linalg.norm(xk - ref.x) <= 1e-10 * np.linalg.norm(ref.x), k
        assert rel[k] <= 1e-10
    x2, its2, rel2 = H.pcg(b, rtol=1e-10)
    assert np.array_equal(x2.cpu().numpy(), x) and np.array_equal(its2, its)


def test_batched_fcg_mixed(batch):
    probs, bs, H, Hm, orc = batch
    off = Hm.level_offsets(0)
    b = torch.tensor(np.concatenate(bs), device="cuda")
    x, its, rel = Hm.pcg(b, rtol=1e-8)
    x = x.cpu().numpy()
    for k, (P, Ho) in enumerate(zip(probs, orc)):
        xk = x[off[k]:off[k + 1]]
        assert np.linalg.norm(bs[k] - P.scipy() @ xk) <= 1e-8 * np.linalg.norm(bs[k]), k
        ref = O.pcg(P.scipy(), bs[k], lambda v: O.vcycle(Ho, v), rtol=1e-8)
        assert its[k] <= ref.iterations + 3


def _pin_register(Hb):
    """Pin the register form on every level (the persistent solve runs the register form) so that
    both loop modes run identical level kernels."""
    cfg = Hb.kernel_config()
    for row in cfg[:-1]:
        for key in ("f64", "f32"):
            row[key] = {"form": "register", "lanes": row[key]["lanes"] if row[key]["lanes"] >= 4 else 16, "threads": 256}
    Hb.set_kernel_config(cfg[:-1])


@pytest.mark.parametrize("precision", [0, 1])
def test_persistent_batched_solve_equals_graph_loop(batch, precision):
    """The whole batched iteration loop in one persistent cooperative kernel gives every problem
    the same iterates (same bits, same iteration counts) as the graph of per-step kernels; stopped
    problems are skipped, so problems that converge early keep their solution untouched."""
    probs, bs, H, Hm, orc = batch
    Hb = Hm if precision else H
    _pin_register(Hb)
    b = torch.tensor(np.concatenate(bs), device="cuda")
    Hb.set_batch_mode(0)
    xg, itg, relg = Hb.pcg(b, rtol=1e-9)
    Hb.set_batch_mode(1)
    xp, itp, relp = Hb.pcg(b, rtol=1e-9)
    xp2, itp2, _ = Hb.pcg(b, rtol=1e-9)        # the captured launch replayed
    Hb.set_batch_mode(0)
    assert np.array_equal(itg, itp) and np.array_equal(itp, itp2)
    assert torch.equal(xg, xp) and torch.equal(xp, xp2)
    assert np.all(relp <= 1e-9)
    assert len(set(itp.tolist())) > 1          # problems stop at different iterations


def test_automatic_batch_mode_times_both_forms(batch):
    """The default loop mode runs the graph form on the first solve and the persistent form on the
    second, timing each per loop iteration, and keeps the faster afterwards; every solve gives the
    same bits."""
    probs, bs, H, Hm, orc = batch
    b = torch.tensor(np.concatenate(bs), device="cuda")
    H.set_batch_mode(2)
    m0 = H.batch_mode()
    assert m0["mode"] == 2 and m0["ms_per_iteration"] == {"graph": -1.0, "persistent": -1.0}
    xs = []
    for k in range(3):
        x, its, rel = H.pcg(b, rtol=1e-9)
        xs.append(x)
        m = H.batch_mode()
        if k < 2:
            assert m["used"] == k
    t = m["ms_per_iteration"]
    assert t["graph"] > 0 and t["persistent"] > 0
    assert m["used"] == (1 if t["persistent"] < t["graph"] else 0)
    assert torch.equal(xs[0], xs[1]) and torch.equal(xs[1], xs[2])
    H.set_batch_mode(0)


def test_persistent_batched_barrier_expiry_is_reported(batch):
    """A grid-barrier wait that cannot complete (CTA 0 withholds its first arrival) runs out after
    the wait limit: every CTA leaves, the solve reports R3MG_E_TIMEOUT, and the next solve works."""
    import paper_2607_28235_b300 as R
    probs, bs, H, Hm, orc = batch
    b = torch.tensor(np.concatenate(bs), device="cuda")
    H.set_batch_mode(1)
    H.set_wait_limit(2_000_000, withhold_first_copy=True)
    with pytest.raises(R.R3MGError) as e:
        H.pcg(b, rtol=1e-9)
    assert e.value.status == 10
    H.set_wait_limit(0, withhold_first_copy=False)
    x, its, rel = H.pcg(b, rtol=1e-9)
    assert np.all(rel <= 1e-9)
    H.set_batch_mode(0)
