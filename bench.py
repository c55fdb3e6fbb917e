#!/usr/bin/env python3
"""Benchmark: PCG solve to 1e-8 relative residual, preconditioned by one R-tree V-cycle.

Workload (one GPU): 3D Poisson on the unit cube, Q3 Lagrange elements on a 32^3 hex
mesh with interior vertices perturbed by up to 0.2 h per component (seeded uniform),
manufactured right-hand side; 857,375 free DoFs, 101.8M nonzeros.  Hierarchy: R-tree
leaf 128 points, p' = 2, 4 levels, Chebyshev-Jacobi degree 3, 2 + 2 sweeps.
A step is one complete PCG solve (hierarchy already set up, inputs resident in HBM).
The headline form is the FP32 V-cycle inside FP64 flexible CG; the plain FP64 solve is
timed beside it.  The matrix (0.6-1.2 GB per level) is far larger than L2, so no flush
is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (the single solve does not shard); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the oracle timing uses one host thread: BLAS threads off (OpenMP of the library's host setup untouched)
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")


def _one_thread():
    """Limit BLAS pools to one thread when threadpoolctl is available (env vars cover the rest)."""
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(1)
    except ImportError:
        import contextlib
        return contextlib.nullcontext()

WORKLOAD = dict(name="poisson3d_q3_32cube_perturbed", dim=3, N=32, p=3, perturb=0.2, seed=1, leaf_size=128,
                pprime=2, levels=4, cheb_degree=3, sweeps=2, rtol=1e-8)
# the same problem with cell-based agglomeration: R-tree over the 32^3 cells, 4 cells per
# level-1 agglomerate (8192 agglomerates, as many as the point-based boxes)
CELLS = dict(WORKLOAD, name="poisson3d_q3_32cube_perturbed_cells", leaf_size=4, cells=True)
# smaller instance for ncu captures (inputs still larger than L2, a few GB on the device)
SMALL = dict(WORKLOAD, name="poisson3d_q3_24cube_perturbed", N=24)
METRIC = "PCG solve ms to 1e-8 rel-res"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _problem(w):
    import workloads as W
    return W.poisson(w["dim"], w["N"], w["p"], perturb=w["perturb"], seed=w["seed"])


def max_over_ranks(value: float, device) -> float:
    """The slowest replica's time: the max of `value` over the ranks of the default process group
    (identity without one).  Replicas share nothing else: the single solve does not shard."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _hparams(w, precision):
    return dict(leaf_size=w["leaf_size"], pprime=w["pprime"], levels=w["levels"], cheb_degree=w["cheb_degree"],
                sweeps=w["sweeps"], precision=precision)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="r3mg_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if getattr(self, "_summary", None) is None:
            self._summary = self._read()
        return self._summary

    def _read(self):
        rows = []
        text = open(self.path).read()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in text.splitlines()[1:]:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts))
            except ValueError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, _, parts in rows:
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def _traffic(kernel_name, source="kernels_level.cuh"):
    """dram bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", f"{kernel_name}.md")
    if not os.path.exists(prof):
        return None
    src = open(os.path.join(ROOT, "paper_2607_28235_b300", "csrc", source), "rb").read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    vals = {}
    for line in open(prof):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != digest:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _host_cpu():
    """CPU model and logical core count of the host the oracle runs on."""
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"model": model, "logical_cores": os.cpu_count()}


def _oracle_setup(w):
    """The oracle's hierarchy of workload w (one host thread), its fine matrix and the problem."""
    import oracle as O
    from oracle.hierarchy import Params
    P = _problem(w)
    with _one_thread():
        A = P.scipy()
        t = time.perf_counter()
        H = O.build_hierarchy(P.coords, A, Params(w["leaf_size"], w["pprime"], w["levels"],
                                                  cheb_degree=w["cheb_degree"], sweeps=w["sweeps"]))
        setup_s = time.perf_counter() - t
    return P, A, H, setup_s


def _oracle_solve(A, H, b, rtol, threads):
    """One oracle PCG solve; threads > 1 splits its sparse products over a thread pool (same bits)."""
    import oracle as O
    if threads > 1:
        from oracle.parallel import threaded
        H, A = threaded(H, A, threads)
    with _one_thread():
        t = time.perf_counter()
        r = O.pcg(A, b, lambda v: O.vcycle(H, v), rtol=rtol)
        return (time.perf_counter() - t) * 1e3, r


def cpu_baseline():
    """The oracle as it stands on the host cores, on the bench workload itself (32^3, setup
    excluded): one solve on one thread (the value), and the same solve with the sparse products
    split over all cores (all_cores)."""
    import numpy as np
    w = WORKLOAD
    P, A, H, setup_s = _oracle_setup(w)
    ms1, ref = _oracle_solve(A, H, P.b, w["rtol"], 1)
    ncores = os.cpu_count() or 1
    msn, refn = _oracle_solve(A, H, P.b, w["rtol"], ncores)
    out = {"value": ms1, "unit": "ms", "cores": 1, "kind": "oracle", "host": _host_cpu(),
           "sample": (f"one oracle PCG solve of the whole {w['name']} workload ({P.n} DoFs, {P.nnz} nnz, "
                      f"{ref.iterations} iterations to {w['rtol']}), hierarchy built beforehand "
                      f"({setup_s:.1f} s, not timed), one host thread"),
           "iterations": ref.iterations, "oracle_setup_s": setup_s,
           "all_cores": {"value": msn, "unit": "ms", "cores": ncores,
                         "kind": "oracle with its sparse products split over a thread pool (same bits)",
                         "same_solution_bits": bool(np.array_equal(ref.x, refn.x))}}
    return out, ref


def error_vs_oracle(ref, x_mixed, x_fp64, iters_mixed, iters_fp64):
    """The GPU solves of the bench workload (mixed and FP64) against the oracle's PCG solution of
    the same workload: relative 2-norm difference and iterations."""
    import numpy as np
    out = {"problem": WORKLOAD["name"], "oracle_iterations": ref.iterations}
    for key, x, it in (("mixed", x_mixed, iters_mixed), ("fp64", x_fp64, iters_fp64)):
        out[key] = {"solution_reldiff": float(np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)), "iterations": it}
    return out


BATCH = dict(name="poisson2d_batch256_uneven", nprob=256, seed=4, leaf_size=64, pprime=1, levels=3, cheb_degree=3,
             sweeps=2, rtol=1e-8)


def _batch_problems(w):
    """256 independent 2D problems: N uniform in {16..128}, Q_p with p uniform in {1..4}, seeded random f."""
    import numpy as np
    import workloads as W
    rng = np.random.default_rng(w["seed"])
    probs, rhs = [], []
    for k in range(w["nprob"]):
        N = int(rng.integers(16, 129)); p = int(rng.integers(1, 5))
        P = W.poisson(2, N, p, perturb=0.0, seed=k)
        probs.append(P)
        rhs.append(W.gaussian(P.n, seed=10_000 + k))
    return probs, rhs


def run_batch(args):
    """Batched workload: one block-diagonal hierarchy, the solve loop as one graph launch."""
    import numpy as np
    import torch
    import paper_2607_28235_b300 as R
    w = BATCH
    t0 = time.perf_counter()
    probs, rhs = _batch_problems(w)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = R.BatchHierarchy([(P.coords, P.rowptr, P.colidx, P.vals) for P in probs], leaf_size=w["leaf_size"],
                         pprime=w["pprime"], levels=w["levels"], cheb_degree=w["cheb_degree"], sweeps=w["sweeps"],
                         precision=1)
    t_setup = time.perf_counter() - t0
    b = torch.tensor(np.concatenate(rhs), device="cuda")

    def timed_mode(mode):
        H.set_batch_mode(mode)
        for _ in range(args.warmup):
            H.pcg(b, rtol=w["rtol"])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            out = H.pcg(b, rtol=w["rtol"])
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, out

    # the loop as a graph of per-step kernels (mode 0) and as one persistent kernel (mode 1);
    # the faster is the one the line reports
    mode_ms = {}
    outs = {}
    for mode in (0, 1):
        mode_ms[mode], outs[mode] = timed_mode(mode)
    best = min(mode_ms, key=mode_ms.get)
    H.set_batch_mode(best)
    ms = mode_ms[best]
    x, its, rel = outs[best]
    same_bits = bool(torch.equal(outs[0][0], outs[1][0]))
    xs = x.cpu().numpy()
    off = H.level_offsets(0)
    chk = max(float(np.linalg.norm(rhs[k] - probs[k].scipy() @ xs[off[k]:off[k + 1]]) / np.linalg.norm(rhs[k]))
              for k in range(len(probs)))
    # per-kernel event times of the batched level steps (profiled V-cycles of all problems at once)
    H.profile(True)
    nvc = 5 * args.steps
    for _ in range(nvc):
        H.vcycle(b)
    prof = H.profile_read()
    H.profile(False)
    kinds = {k: v for k, v in prof.items() if isinstance(v, dict) and v["launches"] > 0}
    top = max(kinds, key=lambda k: kinds[k]["ms"])
    tk = kinds[top]
    avg_ms = tk["ms"] / tk["launches"]
    peak, peak_kind = _peaks()
    achieved = tk["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    # end to end: pinned host right-hand sides in, solutions out, inside the timed region
    bh = torch.tensor(np.concatenate(rhs)).pin_memory()
    xh = torch.empty_like(bh).pin_memory()

    def e2e():
        xd, _, _ = H.pcg(bh.to("cuda", non_blocking=True), rtol=w["rtol"])
        xh.copy_(xd, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e()
    t = time.perf_counter()
    for _ in range(args.steps):
        e2e()
    e2e_ms = (time.perf_counter() - t) * 1e3 / args.steps
    cpu = _batch_cpu_baseline(probs, rhs, w) if not args.no_cpu_baseline else None
    line = {"metric": "batched PCG solve ms to 1e-8 rel-res (all problems)", "value": ms, "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": w["name"], "problems": len(probs), "dofs_total": int(H.n),
                       "dofs_min": int(min(P.n for P in probs)), "dofs_max": int(max(P.n for P in probs)),
                       "nnz_total": int(sum(P.nnz for P in probs)), "leaf_size": w["leaf_size"], "pprime": w["pprime"],
                       "levels": w["levels"], "precision": "FP32 V-cycle in FP64 flexible CG",
                       "loop": "one graph launch: conditional WHILE over per-step kernels, or one persistent "
                               "cooperative kernel (the faster of the two, loop_mode)"},
            "iterations": {"min": int(its.min()), "max": int(its.max()), "mean": float(its.mean())},
            "max_true_relres": chk, "dofs_per_s": H.n / (ms * 1e-3),
            "loop_modes_ms": {"graph_of_kernels": mode_ms[0], "persistent_kernel": mode_ms[1]},
            "loop_mode": ["graph_of_kernels", "persistent_kernel"][best],
            "modes_same_solution_bits": same_bits,
            "setup_s": t_setup, "assembly_s": t_asm,
            "roofline": {"bound": "hbm", "kernel": f"batched_{top}_f32", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "timing": f"CUDA events around each launch in {nvc} profiled batched V-cycles",
                         "bytes_per_launch": tk["bytes_per_launch"], "avg_launch_ms": avg_ms, "traffic": None},
            "kernel_ms_per_vcycle": {k: v["ms"] / nvc for k, v in kinds.items()},
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 8 * int(H.n),
                    "d2h_bytes_per_step": 8 * int(H.n), "host_buffers": "pinned (right-hand sides in, solutions out)"},
            "gpu_launches": int(prof["kernel_launches"])}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def _batch_cpu_baseline(probs, rhs, w, budget_s=20.0):
    """The oracle (one thread) on a bounded sample of the batch: problems in order, each set up and
    solved to the batch tolerance, until about budget_s of solve time; scaled to the whole batch by
    the nonzeros solved (setup not timed)."""
    import oracle as O
    from oracle.hierarchy import Params
    t_solve, nnz_done, k = 0.0, 0, 0
    with _one_thread():
        while k < len(probs) and t_solve < budget_s:
            P = probs[k]
            A = P.scipy()
            Hk = O.build_hierarchy(P.coords, A, Params(w["leaf_size"], w["pprime"], w["levels"],
                                                       cheb_degree=w["cheb_degree"], sweeps=w["sweeps"]))
            t = time.perf_counter()
            O.fcg(A, rhs[k], lambda v: O.vcycle(Hk, v), rtol=w["rtol"])
            t_solve += time.perf_counter() - t
            nnz_done += P.nnz
            k += 1
    total = sum(P.nnz for P in probs)
    return {"value": t_solve * 1e3 * total / nnz_done, "unit": "ms", "cores": 1, "kind": "oracle",
            "host": _host_cpu(),
            "sample": (f"oracle solves of the first {k} of {len(probs)} problems ({nnz_done} of {total} nonzeros, "
                       f"{t_solve:.1f} s, one thread, setup not timed), scaled by the nonzero ratio")}


MULTI = dict(WORKLOAD, name="poisson3d_q3_64cube_perturbed_16rhs", N=64, leaf_size=256, levels=5, nrhs=16,
             rhs_seed=500)
# the same 16-column block solve on the 24^3 instance, for ncu captures (inputs > L2, a few GB)
MULTI_SMALL = dict(MULTI, name="poisson3d_q3_24cube_perturbed_16rhs", N=24, leaf_size=128, levels=4)


def run_multi(args):
    """16 seeded Gaussian right-hand sides on the 64^3 Q3 problem, solved in one block solve
    (every level operator reads its matrix once for all 16 columns), against 16 single solves."""
    import numpy as np
    import torch
    import workloads as W
    import paper_2607_28235_b300 as R
    w = MULTI_SMALL if args.workload == "rhs16_small" else MULTI
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    P = _problem(w)
    t_asm = time.perf_counter() - t0
    m = w["nrhs"]
    B = np.stack([W.gaussian(P.n, seed=w["rhs_seed"] + k) for k in range(m)])
    t0 = time.perf_counter()
    Hm = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, **_hparams(w, 1))
    setup_m = time.perf_counter() - t0
    Bd = torch.tensor(B, device=dev)
    stream = torch.cuda.current_stream()
    if args.pin_block:               # one block solve tunes every level, then the pins replace the choice
        Hm.pcg_multi(Bd, rtol=w["rtol"])
        for pin in args.pin_block:
            lev, slots = (int(v) for v in pin.split(":"))
            Hm.set_block_config(lev, slots, fp32=True)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            out = fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out

    clocks = Clocks(0)
    with clocks:
        ms_block, (X, its, rel) = timed(lambda: Hm.pcg_multi(Bd, rtol=w["rtol"]), args.steps, args.warmup)
    # one profiled block solve: per-kind event times of the level operators
    Hm.profile(True)
    torch.cuda.profiler.start()     # ncu --profile-from-start off sees this pass only
    for _ in range(args.steps):
        Hm.pcg_multi(Bd, rtol=w["rtol"])
    torch.cuda.profiler.stop()
    prof = Hm.profile_read()
    Hm.profile(False)
    block_cfg = {"fp32": Hm.block_config(fp32=True), "fp64": Hm.block_config(fp32=False)}
    # the same 16 systems one after another with the single-vector solver
    ms_seq, its_seq = timed(lambda: [Hm.pcg(Bd[c], rtol=w["rtol"])[1] for c in range(m)], 1, 1)
    # end to end: pinned host blocks in, solutions out, inside the timed region
    Bh = torch.tensor(B).pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()

    def e2e():
        Xd, _, _ = Hm.pcg_multi(Bh.to(dev, non_blocking=True), rtol=w["rtol"])
        Xh.copy_(Xd, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e()
    t = time.perf_counter()
    for _ in range(args.steps):
        e2e()
    e2e_ms = (time.perf_counter() - t) * 1e3 / args.steps
    # the plain FP64 block solve beside it
    t0 = time.perf_counter()
    Hd = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, **_hparams(w, 0))
    setup_d = time.perf_counter() - t0
    ms_block64, (X64, its64, rel64) = timed(lambda: Hd.pcg_multi(Bd, rtol=w["rtol"]), max(1, args.steps // 2), 1)
    # independent check of four columns on the host (scipy)
    A = P.scipy()
    Xc = X.cpu().numpy()
    chk = max(float(np.linalg.norm(B[c] - A @ Xc[c]) / np.linalg.norm(B[c])) for c in range(0, m, 4))
    peak, peak_kind = _peaks()
    kinds = {k: v for k, v in prof.items() if isinstance(v, dict) and v["launches"] > 0}
    top = max(kinds, key=lambda k: kinds[k]["ms"])
    tk = kinds[top]
    avg_ms = tk["ms"] / tk["launches"]
    achieved = tk["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    kname = f"block_{top}_{'f64' if top.startswith('cg') else 'f32'}"
    info = Hm.info()
    line = {
        "metric": "block PCG solve ms to 1e-8 rel-res (16 right-hand sides)", "value": ms_block, "unit": "ms",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_block,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": w["name"], "dofs_free": P.n, "nnz": P.nnz, "rhs": m, "leaf_size": w["leaf_size"],
                   "pprime": w["pprime"], "levels": w["levels"], "cheb_degree": w["cheb_degree"],
                   "sweeps": w["sweeps"], "rtol": w["rtol"], "precision": "FP32 V-cycle in FP64 flexible CG",
                   "l2": "inputs larger than L2 (fine matrix 5 GB FP32)", "level_n": info["n"].tolist(),
                   "level_nnz": info["nnz"].tolist()},
        "iterations": {"min": int(its.min()), "max": int(its.max())}, "max_true_relres_sampled": chk,
        "sequential_single_solves_ms": ms_seq, "block_vs_sequential_speedup": ms_seq / ms_block,
        "sequential_iterations": {"min": int(min(its_seq)), "max": int(max(its_seq))},
        "fp64_block": {"ms": ms_block64, "iterations_max": int(its64.max())},
        "mixed_vs_fp64_speedup": ms_block64 / ms_block,
        "setup_s": {"mixed": setup_m, "fp64": setup_d}, "assembly_s": t_asm,
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "limiter": "the L1 data path serving the gathers of X (ncu: L1 throughput 80%, DRAM 17%)",
                     "bytes_per_launch": tk["bytes_per_launch"], "avg_launch_ms": avg_ms,
                     "traffic": _traffic(kname, "kernels_mrhs.cuh")},
        "kernel_time_share": {k: round(v["ms"] / (ms_block * args.steps), 4) for k, v in kinds.items()},
        "block_config": block_cfg,
        # the tensor-core coarse forms (3, 5, 6) split FP32 operands into TF32 head and tail
        "tensor_core_levels": [lev for lev, sl in enumerate(block_cfg["fp32"]) if sl in (3, 5, 6)],
        "tensor_core_arithmetic": "levels listed in tensor_core_levels run the 3-pass TF32 head/tail product: "
                                  "about 22 bits per product against FP32's 24 (parity bound (2k+64) 2^-24 "
                                  "(|A||x|)_i); the FP64 flexible CG reaches the same residual in the same "
                                  "iterations as with the exact FP32 forms",
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 8 * m * P.n, "d2h_bytes_per_step": 8 * m * P.n},
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


SWEEP = dict(MULTI, name="poisson3d_q3_64cube_perturbed_pprime_sweep", pprimes=(0, 1, 2, 3))


def run_sweep(args):
    """The 64^3 Q3 problem (6.97M DoFs, 849M nonzeros), one right-hand side, p' = 0..3: single
    solves with the FP32 V-cycle (FCG) and the FP64 V-cycle (PCG), one JSON line per p'."""
    import numpy as np
    import torch
    import paper_2607_28235_b300 as R
    w = SWEEP
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    P = _problem(w)
    t_asm = time.perf_counter() - t0
    b = torch.tensor(P.b, device=dev)
    A = P.scipy()
    for pp in w["pprimes"]:
        out = {"metric": "PCG solve ms to 1e-8 rel-res", "unit": "ms", "n_gpus": 1, "higher_is_better": False,
               "data": "synthetic", "config": {"workload": w["name"], "dofs_free": P.n, "nnz": P.nnz, "pprime": pp,
                                               "leaf_size": w["leaf_size"], "levels": w["levels"]},
               "assembly_s": t_asm}
        for prec, key in ((1, "mixed"), (0, "fp64")):
            try:
                t0 = time.perf_counter()
                H = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, **dict(_hparams(w, prec), pprime=pp))
                setup = time.perf_counter() - t0
                for _ in range(2):
                    H.pcg(b, rtol=w["rtol"])
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.steps):
                    x, it, rel = H.pcg(b, rtol=w["rtol"])
                e1.record()
                torch.cuda.synchronize()
                chk = float(np.linalg.norm(P.b - A @ x.cpu().numpy()) / np.linalg.norm(P.b))
                info = H.info()
                out[key] = {"ms": e0.elapsed_time(e1) / args.steps, "iterations": it, "relres_check": chk,
                            "setup_s": setup, "level_n": info["n"].tolist(), "level_nnz": info["nnz"].tolist()}
                H.close()
                del H
            except Exception as e:          # e.g. p' = 3: unisolvence or memory
                out[key] = {"error": str(e)[:200]}
            torch.cuda.empty_cache()
        if "ms" in out.get("mixed", {}):
            out["value"] = out["mixed"]["ms"]
        print(json.dumps(out), flush=True)


def run_coarse(args):
    """The coarsest solve of the bench hierarchy (3,456 rows) in its two forms: the explicit inverse
    applied by one GEMV (the default) and forward + back substitution with the Cholesky factor,
    in FP64 and FP32: time per application, error against an FP64 direct solve of A_c, cond(A_c),
    and the whole mixed and FP64 solves with either form."""
    import numpy as np
    import torch
    import paper_2607_28235_b300 as R
    w = WORKLOAD
    P = _problem(w)
    dev = torch.device("cuda", 0)
    Hm = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, **_hparams(w, 1))
    Hd = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, **_hparams(w, 0))
    Lc = Hd.levels - 1
    rp, cols, vals = Hd.level_matrix(Lc)
    nc = len(rp) - 1
    Ac = np.zeros((nc, nc))
    Ac[np.repeat(np.arange(nc), np.diff(rp)), cols] = vals
    cond = float(np.linalg.cond(Ac))
    r = np.random.default_rng(7).standard_normal(nc)
    zref = np.linalg.solve(Ac, r)
    rd = torch.tensor(r, device=dev)
    b = torch.tensor(P.b, device=dev)
    stream = torch.cuda.current_stream()
    out = {"metric": "coarsest solve ms per application", "unit": "ms", "n_gpus": 1,
           "config": {"workload": w["name"], "coarsest_rows": nc}, "cond_Ac": cond, "forms": {}}
    reps = 50
    for mode, name in ((0, "explicit_inverse_gemv"), (1, "substitution")):
        row = {}
        for H, fp32, key in ((Hd, False, "fp64"), (Hm, True, "fp32")):
            H.set_coarse_mode(mode)
            z = H.coarse_solve(rd, fp32=fp32)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                H.coarse_solve(rd, fp32=fp32)
            e1.record(stream)
            torch.cuda.synchronize()
            zc = z.cpu().numpy()
            row[key] = {"ms": e0.elapsed_time(e1) / reps,
                        "rel_error_vs_direct": float(np.linalg.norm(zc - zref) / np.linalg.norm(zref))}
        for H, key in ((Hm, "mixed_solve"), (Hd, "fp64_solve")):
            for _ in range(2):
                H.pcg(b, rtol=w["rtol"])
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                x, it, rel = H.pcg(b, rtol=w["rtol"])
            e1.record(stream)
            torch.cuda.synchronize()
            row[key] = {"ms": e0.elapsed_time(e1) / args.steps, "iterations": it, "relres": rel}
        out["forms"][name] = row
    Hm.set_coarse_mode(0)
    rv = torch.tensor(np.random.default_rng(8).standard_normal(P.n), device=dev)
    v0 = Hd.vcycle(rv).cpu().numpy()
    Hd.set_coarse_mode(1)
    v1 = Hd.vcycle(rv).cpu().numpy()
    out["fp64_vcycle_reldiff_between_forms"] = float(np.linalg.norm(v1 - v0) / np.linalg.norm(v0))
    print(json.dumps(out), flush=True)


def run_fp64_rate(args):
    """FP64 FMA and FP64 tensor-core (mma.sync m8n8k4) rates of this GPU: the denominators of the
    FP64 kernels' ALU roofline (one FMA per 8-10 bytes of matrix stream)."""
    import torch
    import paper_2607_28235_b300 as R
    torch.cuda.set_device(0)
    clocks = Clocks(0)
    with clocks:
        runs = [R.measure_fp64_rates() for _ in range(max(args.steps, 1))]
    best = {k: max(r[k] for r in runs) for k in runs[0]}
    line = {"metric": "FP64 rates", "fma_tflops": best["fma_tflops"], "mma_tflops": best["mma_tflops"],
            "fma_tfma_per_s": best["fma_tflops"] / 2, "unit": "TFLOP/s", "n_gpus": 1, "steps": len(runs),
            "runs": runs, "clocks": clocks.summary(),
            "method": "8 independent FMA chains (4 mma chains) per thread, 8 x 256-thread CTAs per SM, "
                      "CUDA events around one launch after a warm-up; best of the runs"}
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The oracle arm: the oracle's PCG solve of the bench workload itself (32^3, hierarchy built
    once beforehand), its sparse products split over all host cores (same bits as one thread);
    warm-up solves, then `steps` timed solves."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    w = WORKLOAD
    P, A, H, setup_s = _oracle_setup(w)
    ncores = os.cpu_count() or 1
    for _ in range(args.warmup):
        _oracle_solve(A, H, P.b, w["rtol"], ncores)
    times = []
    for _ in range(args.steps):
        ms, r = _oracle_solve(A, H, P.b, w["rtol"], ncores)
        times.append(ms)
    val = sum(times) / max(len(times), 1)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "dofs_free": P.n, "nnz": P.nnz, "leaf_size": w["leaf_size"],
                       "pprime": w["pprime"], "levels": w["levels"], "cheb_degree": w["cheb_degree"],
                       "sweeps": w["sweeps"], "rtol": w["rtol"], "iterations": r.iterations},
            "cpu_baseline": {"value": val, "unit": "ms", "cores": ncores, "kind": "oracle", "host": _host_cpu(),
                             "sample": (f"the whole workload: oracle PCG solve per step ({P.n} DoFs, "
                                        f"{r.iterations} iterations), sparse products over {ncores} threads, "
                                        f"hierarchy built once beforehand ({setup_s:.1f} s, not timed)")},
            "e2e": {"value": val, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import paper_2607_28235_b300 as R

    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = {"small": SMALL, "cells": CELLS}.get(args.workload, WORKLOAD)
    P = _problem(w)
    cells = None
    if w.get("cells"):
        import workloads as W
        cells = W.cells(w["dim"], w["N"], w["p"])
    t0 = time.perf_counter()
    Hm = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, cells=cells, **_hparams(w, 1))
    setup_mixed_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    Hd = R.Hierarchy(P.coords, P.rowptr, P.colidx, P.vals, cells=cells, **_hparams(w, 0))
    setup_fp64_s = time.perf_counter() - t0
    if args.kernel_config:
        cfg = json.load(open(args.kernel_config))
        Hm.set_kernel_config(cfg["mixed"])
        Hd.set_kernel_config(cfg["fp64"])
    for pins, H, key in ((args.pin_form, Hm, "f32"), (args.pin_form64, Hd, "f64")):
        for pin in pins or []:
            # level:form[:lanes[:threads]] pins the level kernel of one level (FP32 of the mixed
            # hierarchy, or FP64 of the FP64 hierarchy)
            parts = pin.split(":")
            lev = int(parts[0])
            cfg = H.kernel_config()
            row = cfg[lev][key]
            row["form"] = parts[1]
            if len(parts) > 2:
                row["lanes"] = int(parts[2])
            elif parts[1] != "symmetric_block_staged" and row["lanes"] < 4:
                row["lanes"] = 16        # the tuned form kept CTAs per SM in the lanes field
            if len(parts) > 3:
                row["threads"] = int(parts[3])
            H.set_kernel_config(cfg[:-1])
    if args.save_config:
        os.makedirs(os.path.dirname(os.path.abspath(args.save_config)), exist_ok=True)
        json.dump({"mixed": Hm.kernel_config(), "fp64": Hd.kernel_config()}, open(args.save_config, "w"))
    info = Hm.info()
    b = torch.tensor(P.b, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(H, steps, warmup, profile=False, ncu_region=False):
        """Unprofiled solves (the loop is one graph launch) give the time; then, with profile,
        the same solves once more with CUDA events around every level-operator launch (the
        host-driven loop runs the same kernels) give the per-kernel times."""
        for _ in range(warmup):
            H.pcg(b, rtol=w["rtol"])
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = []
        for _ in range(steps):
            x, it, rel = H.pcg(b, rtol=w["rtol"])
            its.append(it)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        prof = None
        if profile:
            H.profile(True)
            if ncu_region:
                # ncu --profile-from-start off sees this pass: the kernels of the timed solves,
                # launched one by one (a profiler does not enter the loop graph's conditional body)
                torch.cuda.profiler.start()
            for _ in range(steps):
                H.pcg(b, rtol=w["rtol"])
            if ncu_region:
                torch.cuda.profiler.stop()
            prof = H.profile_read()
            H.profile(False)
        ms = max_over_ranks(ms, dev)
        return ms, its, x, rel, prof

    clocks = Clocks(local)
    with clocks:
        ms_mixed, its_m, x_m, rel_m, prof = timed(Hm, args.steps, args.warmup, profile=True,
                                                  ncu_region=args.ncu_region == "mixed")
    ms_fp64, its_d, x_d, rel_d, prof_d = timed(Hd, max(1, args.steps // 2), max(3, args.warmup // 2), profile=True,
                                               ncu_region=args.ncu_region == "fp64")
    # end to end through the C ABI with host buffers (copies inside the call)
    # pinned host buffers: b, and x (zero initial guess in, solution out) written every step
    bh = torch.tensor(P.b).pin_memory().numpy()
    xh = torch.zeros(P.n, dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        xh.fill(0.0)
        Hm.pcg_host(bh, rtol=w["rtol"], out=xh)
    t = time.perf_counter()
    for _ in range(args.steps):
        xh.fill(0.0)
        _, ith, relh = Hm.pcg_host(bh, rtol=w["rtol"], out=xh)
    e2e_ms = (time.perf_counter() - t) * 1e3 / args.steps
    # independent check of the answers (scipy on the host)
    A = P.scipy()
    bn = np.linalg.norm(P.b)
    chk_m = float(np.linalg.norm(P.b - A @ x_m.cpu().numpy()) / bn)
    chk_d = float(np.linalg.norm(P.b - A @ x_d.cpu().numpy()) / bn)
    diff_md = float(np.linalg.norm(x_m.cpu().numpy() - x_d.cpu().numpy()) / np.linalg.norm(x_d.cpu().numpy()))
    # the paper's table columns for this solve (Section 6): iterations, the PCG condition
    # estimate, H, h and H/h
    st = Hm.stats()
    diag = {"iterations": its_d[-1], "cond_estimate": Hd.cond_estimate()["cond"],
            "cond_estimate_mixed": Hm.cond_estimate()["cond"], "H": st["H"], "h": st["h"],
            "H_over_h": st["H_over_h"]}
    if rank != 0:
        return
    peak, peak_kind = _peaks()
    kinds = {k: v for k, v in prof.items() if isinstance(v, dict) and v["launches"] > 0}
    top = max(kinds, key=lambda k: kinds[k]["ms"])
    tk = kinds[top]
    avg_ms = tk["ms"] / tk["launches"]
    achieved = tk["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    kernel_name = f"{top}_{'f64' if top.startswith('cg') else 'f32'}"
    kernel_src = "kernels_level.cuh"
    if top.startswith("cheb_step_level"):    # the symmetric forms have summaries of their own
        form = Hm.kernel_config()[int(top[len("cheb_step_level"):])]["f32"]["form"]
        if form.startswith("symmetric_block"):
            kernel_name += "_" + form
            kernel_src = "kernels_level_sym.cuh"
    # share of the unprofiled solve time taken by each kind (event times of the profiled pass)
    share = {k: round(v["ms"] / (ms_mixed * args.steps), 4) for k, v in kinds.items()}
    kinds_d = {k: v for k, v in prof_d.items() if isinstance(v, dict) and v["launches"] > 0}
    top_d = max(kinds_d, key=lambda k: kinds_d[k]["ms"])
    td = kinds_d[top_d]
    avg_d = td["ms"] / td["launches"]
    # the FP64 solve's top kernel is bound by the FP64 pipe: one FMA per stored value of its level
    # against the FMA rate of this GPU, measured now by the library's probe (8 independent FMA chains)
    rates = R.measure_fp64_rates()
    lev_d = 0 if top_d.startswith("cg") else int(top_d[len("cheb_step_level"):])
    fma = float(info["nnz"][lev_d])
    fp64_roof = {"bound": "alu", "kernel": f"{top_d}_f64", "achieved": fma / (avg_d * 1e-3) / 1e12,
                 "peak": rates["fma_tflops"] / 2, "unit": "T FMA/s",
                 "frac": fma / (avg_d * 1e-3) / 1e12 / (rates["fma_tflops"] / 2),
                 "peak_source": "measured FP64 FMA rate (r3mg_measure_fp64_rates)", "fma_per_launch": fma,
                 "avg_launch_ms": avg_d, "traffic": _traffic(f"{top_d}_f64")}
    line = {
        "metric": METRIC, "value": ms_mixed, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": w["name"], "dofs_free": P.n, "nnz": P.nnz, "leaf_size": w["leaf_size"],
                   "pprime": w["pprime"], "levels": w["levels"], "cheb_degree": w["cheb_degree"],
                   "sweeps": w["sweeps"], "rtol": w["rtol"], "precision": "FP32 V-cycle in FP64 flexible CG",
                   "agglomeration": "cell-based (leaf_size counts cells)" if cells is not None else "point-based",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (level matrices 0.6-1.4 GB)", "level_n": info["n"].tolist(),
                   "level_nnz": info["nnz"].tolist()},
        "iterations": its_m[-1], "relres_check": chk_m,
        "fp64": {"ms": ms_fp64, "iterations": its_d[-1], "relres_check": chk_d,
                 "top_kernel": top_d, "top_kernel_avg_ms": avg_d,
                 "top_kernel_achieved_gbs": td["bytes_per_launch"] / (avg_d * 1e-3) / 1e9,
                 "top_kernel_frac_of_fp64_bound": fp64_roof["frac"],
                 "roofline": fp64_roof,
                 "kernel_config": [row["f64"] for row in Hd.kernel_config()],
                 "kernel_ms": {k: v["ms"] / max(v["launches"], 1) for k, v in kinds_d.items()}},
        "mixed_vs_fp64_speedup": ms_fp64 / ms_mixed, "mixed_vs_fp64_solution_reldiff": diff_md,
        "paper_diagnostics": diag,
        "setup_s": {"mixed": setup_mixed_s, "fp64": setup_fp64_s},
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "timing": "CUDA events around each launch of this kernel in a profiled pass of the same solves",
                     "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_launch": tk["bytes_per_launch"], "avg_launch_ms": avg_ms,
                     "traffic": _traffic(kernel_name, kernel_src)},
        "kernel_time_share": share,
        "kernel_config": Hm.kernel_config(),
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * 8 * P.n, "d2h_bytes_per_step": 8 * P.n,
                "host_buffers": "pinned (b in; x: zero initial guess in, solution out)"},
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clocks.summary(),
    }
    print("gpu part: " + json.dumps(line), file=sys.stderr, flush=True)
    if not args.no_cpu_baseline and w is WORKLOAD:
        line["cpu_baseline"], ref = cpu_baseline()
        line["error_vs_oracle"] = error_vs_oracle(ref, x_m.cpu().numpy(), x_d.cpu().numpy(), its_m[-1], its_d[-1])
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--save-config", default=None, help="write the autotuned kernel configuration (JSON)")
    ap.add_argument("--kernel-config", default=None, help="replay a saved kernel configuration (JSON)")
    ap.add_argument("--pin-form", action="append", default=None,
                    help="level:form[:lanes[:threads]]: pin the FP32 level kernel of one level (repeatable)")
    ap.add_argument("--pin-form64", action="append", default=None,
                    help="level:form[:lanes[:threads]]: pin the FP64 level kernel of one level (repeatable)")
    ap.add_argument("--pin-block", action="append", default=None,
                    help="level:slots: pin the FP32 block kernel of one level in the block workloads (repeatable; "
                         "slots as r3mg_set_block_config: 3 mma.sync, 5 tcgen05, ...)")
    ap.add_argument("--ncu-region", default="mixed", choices=["mixed", "fp64"],
                    help="which profiled pass lies between cudaProfilerStart/Stop (ncu --profile-from-start off)")
    ap.add_argument("--workload", default="full", choices=["full", "small", "cells", "batch256", "rhs16",
                                                           "rhs16_small", "pprime_sweep", "fp64_rate", "coarse"],
                    help="small: the 24^3 instance used for ncu captures (not a bench line); "
                         "batch256: 256 uneven 2D problems in one batched solve; "
                         "cells: the full problem with cell-based agglomeration; "
                         "rhs16: 16 right-hand sides on the 64^3 Q3 problem in one block solve "
                         "(rhs16_small: its 24^3 instance for ncu captures); "
                         "pprime_sweep: the 64^3 Q3 problem with p' = 0..3")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload in ("rhs16", "rhs16_small"):
        run_multi(args)
    elif args.workload == "pprime_sweep":
        run_sweep(args)
    elif args.workload == "fp64_rate":
        run_fp64_rate(args)
    elif args.workload == "coarse":
        run_coarse(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
