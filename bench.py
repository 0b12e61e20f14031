"""Benchmark: time to the 1e-6 duality gap of plain DROT, and HBM GB/s of the fused DR step.

One "step" of this benchmark is one complete solve of the workload: Algorithm 1
from X_0 = p q^T until the stopping test fires at tol 1e-6.  By default the test
is the metric's own condition, the duality gap of Sec. 3.1,
|<C,X> - (p^T phi + q^T psi)/rho| <= 1e-6 (``--stop gap``); ``--stop full`` also
requires ||X1 - p||_1 + ||X^T 1 - q||_1 <= 1e-6 (the library's default rule).  The
default workload is the largest single-GPU one, 20000 x 20000 (points uniform in
[0,1]^3, uniform marginals, FP32 plan and cost, FP64 reductions).

The gap alone can fall below 1e-6 long before the plan is feasible (primal and dual
objectives cross), so the line also carries:
  tolerance_met   which of gap <= tol and l1 residual <= tol hold at the stop;
  final.certificate  FP64 bounds on the optimal value from the returned (X, mu, nu):
                  a feasible plan's cost (X rounded onto the marginals) above it and a
                  dual-feasible objective (the c-transform of mu) below it;
  full_rule       one solve under the full test (gap and l1 residual <= tol) of the
                  8192 x 6144 workload, with its time, iterations, status and certificate;
  batched         one solve of the 512-problem batch (one problem per uneven shape)
                  with the fraction of the HBM roofline over the whole solve;
  c_skip          one solve of the default workload with C-load skipping (Claim 1 of
                  Sec. 3.3: 10 instead of 12 bytes per entry on average).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is the mean time to tolerance in seconds (lower is
better); `roofline` reports the fused step kernel's algorithmic HBM traffic
(12 bytes per plan entry per launch: read X, read C, write X) over its
CUDA-event-timed launch duration; `e2e` is the same solve through the C ABI with
host buffers (copies inside the timed region); `cpu_baseline` is the FP64 CPU
oracle timed on a bounded sample of the same workload, on all host cores (OpenMP
build) and on one core.

Multi-GPU (torchrun): every rank solves its own replica of the problem (there
is no exchange between independent solves), the max time over ranks is taken,
and `value` stays the time to tolerance of each replica ("replicas only").
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 gap & HBM GB/s of fused DR step: plain vs batched / warm-start"
BYTES_PER_ENTRY = 12  # read X (4) + read C (4) + write X (4), FP32
L2_BYTES = 126 * 1024 * 1024

# Iterations to the stopping test at tol 1e-6 (seed 0) used by the reference (CPU
# oracle) arm to extrapolate its per-iteration time.  plain_256: the FP64 oracle's own
# count (full rule: gap and l1 residual), run to completion on the CPU.  The larger
# workloads cannot be run to completion by the oracle in a bench run; their counts are
# those the FP32 GPU solver needed ("GPU count, extrapolated" in the printed line; the
# step-parity tests show both follow the same iterates, and on plain_256 the counts
# agree to 0.5 %: 21535 vs 21434).
ITERS_TO_TOL = {
    ("plain_20000", "gap"): (470, "GPU count, extrapolated"),
    ("plain_8192x6144", "gap"): (9526, "GPU count, extrapolated"),
    ("plain_256", "full"): (21434, "oracle's own count"),
}

DEFAULT_WORKLOAD = "plain_20000"
FULL_RULE_WORKLOAD = "plain_8192x6144"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    for rel in ("paper_2110_11738_b300/csrc/drot_kernels.cuh",):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e nominal bandwidth (context beside the measured copy peak)


def _step_kernel_name(prof, c_skip):
    """Name of the fused-step kernel the solve ran, from the plan it reports."""
    v, k, st = prof["step_variant"], prof["tile_k"], prof["stages"]
    if c_skip:
        return f"drot_step_kernel<{k},1,1|2>"
    return {1: f"drot_step_kernel<{k},1,0>", 2: f"drot_step_tma_kernel<{k},{st}>",
            3: f"drot_step_async_kernel<{k},{st}>", 4: f"drot_cluster_kernel<{st}>",
            5: "drot_step_f64_kernel<1>"}.get(v, f"variant {v}")


def _traffic_per_launch(workload, kernel=None):
    """DRAM bytes per fused-step launch from the committed ncu summary, if it is current
    (same kernel source) and was taken on the kernel that ran."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("kernel_source_sha256_16") != _kernel_source_hash():
        return None
    rec = d.get("workloads", {}).get(workload)
    if rec is None or (kernel is not None and rec.get("kernel") != kernel):
        return None
    return float(rec["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.out = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x, world, device):
    """The largest x over all ranks of the default process group (x itself on one rank):
    the job's time is that of its slowest replica."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _host_problem(workload, seed, pr=None):
    """FP64 cost and marginals of the workload on the host (the oracle's inputs).  With ``pr``
    (the problem already built on the GPU by the bit-identical torch builder) the FP32 cost is
    copied back instead of being rebuilt."""
    import numpy as np

    import workloads

    if pr is None:
        pr = workloads.make_problem(workload, seed=seed)
        C32 = pr.C
    else:
        C32 = pr.C[:, : pr.n].cpu().numpy()
    return pr, np.ascontiguousarray(C32, dtype=np.float64)


def _time_oracle_iterations(C, pr, iters, all_cores):
    """Seconds per Algorithm-1 iteration of the FP64 oracle over `iters` iterations from
    X_0 = p q^T, and the thread count it used."""
    import numpy as np

    import oracle

    st = oracle.StepState(C, pr.p, pr.q, pr.rho, np.outer(pr.p, pr.q), np.zeros(pr.m), np.zeros(pr.n),
                          all_cores=all_cores)
    t0 = time.perf_counter()
    for _ in range(iters):
        st.step()
    per_iter = (time.perf_counter() - t0) / iters
    del st
    return per_iter, oracle.threads(all_cores)


def _cpu_baseline(workload, seed, iters_to_tol, count_kind, omp_iters, single_iters, pr=None):
    """The FP64 oracle as it stands, timed on this host: on every core (its OpenMP build) and on
    one core, each on a bounded sample of whole iterations of the full problem, extrapolated to
    `iters_to_tol` iterations.  plain_256 is small enough for the oracle's own complete solve."""
    import numpy as np

    import oracle

    if workload == "plain_256":
        pr, C = _host_problem(workload, seed, None)
        t0 = time.perf_counter()
        out = oracle.drot_solve(C, pr.p, pr.q, pr.rho, tol=1e-6, max_iter=1_000_000)
        secs = time.perf_counter() - t0
        return {"value": secs, "unit": "s", "cores": 1, "kind": "oracle",
                "sample": f"the oracle's complete solve to gap and l1 residual <= 1e-6 ({out['iters']} iterations, "
                          f"FP64 C oracle, one core)"}
    pr, C = _host_problem(workload, seed, pr)
    omp_s, omp_threads = _time_oracle_iterations(C, pr, omp_iters, True)
    one_s, _ = _time_oracle_iterations(C, pr, single_iters, False)
    out = {
        "value": omp_s * iters_to_tol, "unit": "s", "cores": omp_threads, "kind": "oracle",
        "sample": (f"{omp_iters} Algorithm-1 iterations of the full {pr.m}x{pr.n} problem (FP64 C oracle, OpenMP "
                   f"build on {omp_threads} threads of {os.cpu_count()} host cores, {omp_s:.3f} s/iteration), "
                   f"extrapolated to {iters_to_tol} iterations to tol ({count_kind})"),
        "seconds_per_iteration": omp_s, "nproc": os.cpu_count(),
        "single_thread": {"value": one_s * iters_to_tol, "unit": "s", "cores": 1,
                          "seconds_per_iteration": one_s,
                          "sample": f"{single_iters} iterations on one core (the parity build), extrapolated the "
                                    f"same way"},
    }
    del C
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    entry = ITERS_TO_TOL.get((args.workload, args.stop))
    if entry is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no iteration count to extrapolate the oracle to for "
                                                              f"{args.workload} under --stop {args.stop}"}))
        return 0
    iters, count_kind = entry
    pr, C = _host_problem(args.workload, args.seed)
    t_steps = []
    per_iter = []
    if args.workload == "plain_256":
        # small enough for the oracle's complete solve, every step
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            out = oracle.drot_solve(C, pr.p, pr.q, pr.rho, tol=args.tol, max_iter=1_000_000)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                t_steps.append(dt)
        sample = f"the oracle's complete solve ({out['iters']} iterations, one core), every step"
        cores = 1
    else:
        import numpy as np

        # one oracle state for the whole run: each step times the next iteration of the solve
        st = oracle.StepState(C, pr.p, pr.q, pr.rho, np.outer(pr.p, pr.q), np.zeros(pr.m), np.zeros(pr.n),
                              all_cores=True)
        cores = oracle.threads(True)
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            st.step()
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                t_steps.append(dt * iters)
                per_iter.append(dt)
        sample = (f"each step: the next Algorithm-1 iteration of the full {pr.m}x{pr.n} problem (FP64 C oracle, OpenMP "
                  f"build on {cores} threads of {os.cpu_count()} host cores, mean "
                  f"{statistics.mean(per_iter):.3f} s/iteration), extrapolated to {iters} iterations ({count_kind})")
    value = statistics.mean(t_steps) if t_steps else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None if value is None else value * 1000.0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "m": pr.m, "n": pr.n, "seed": args.seed, "tol": args.tol,
                   "stop_rule": _rule_text(args.stop), "iterations_to_tol": iters, "iteration_count": count_kind},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _rule_text(stop):
    return {"gap": "gap<=tol", "full": "gap<=tol and l1 residual<=tol"}[stop]


def _certificate(C, p, q, X, mu, nu, block_rows=2048):
    """Bounds on the optimal value of eq. ot:dist from a returned (X, mu, nu), in FP64.

    upper: X rounded onto the transport polytope (rows scaled down to at most p_i, then columns
           to at most q_j, the missing mass added as the rank-one plan e_r e_c^T / ||e_r||_1) is a
           feasible plan, so its cost is >= the optimum;
    lower: with the c-transform nu'_j = min_i (C_ij - mu_i), (mu, nu') is dual feasible, so
           p^T mu + q^T nu' is <= the optimum (weak duality, eq. ot:dist:dual).
    upper - lower bounds how far the rounded plan (and the dual) are from optimal.  Evaluation
    only (outside every timed region): plain torch reductions over row blocks."""
    import torch

    m, n = X.shape
    dev = X.device
    p = p.to(torch.float64)
    q = q.to(torch.float64)
    rows = torch.zeros(m, dtype=torch.float64, device=dev)
    cmin = torch.full((n,), float("inf"), dtype=torch.float64, device=dev)
    primal = 0.0
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        Xb = X[i0:i1].to(torch.float64)
        Cb = C[i0:i1].to(torch.float64)
        rows[i0:i1] = Xb.sum(1)
        primal += float((Cb * Xb).sum())
        cmin = torch.minimum(cmin, (Cb - mu[i0:i1, None]).min(0).values)
    xs = torch.where(rows > p, p / rows, torch.ones_like(rows))
    cols = torch.zeros(n, dtype=torch.float64, device=dev)
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        cols += (X[i0:i1].to(torch.float64) * xs[i0:i1, None]).sum(0)
    ys = torch.where(cols > q, q / cols, torch.ones_like(cols))
    rows2 = torch.zeros(m, dtype=torch.float64, device=dev)
    cost2 = 0.0
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        Xb = X[i0:i1].to(torch.float64) * xs[i0:i1, None] * ys[None, :]
        rows2[i0:i1] = Xb.sum(1)
        cost2 += float((C[i0:i1].to(torch.float64) * Xb).sum())
    er = (p - rows2).clamp_min(0.0)
    ec = (q - cols * ys).clamp_min(0.0)
    s = float(er.sum())
    if s > 0.0:
        Cec = torch.zeros(m, dtype=torch.float64, device=dev)
        for i0 in range(0, m, block_rows):
            i1 = min(m, i0 + block_rows)
            Cec[i0:i1] = C[i0:i1].to(torch.float64) @ ec
        cost2 += float(er @ Cec) / s
    lower = float(p @ mu + q @ cmin)
    upper = cost2
    return {"primal": primal, "upper_rounded_plan": upper, "lower_c_transform": lower,
            "certified_rel_gap": (upper - lower) / abs(lower) if lower != 0 else None,
            "moved_mass": s}


def _device_problem(workload, seed, dev, m=None, n=None):
    """The workload built on the GPU (bit-identical to the host builder) with an X buffer of the
    same row pitch; returns (problem, C view, p, q, X view, mu, nu)."""
    import torch

    import workloads

    spec = workloads.CONFIGS[workload]
    nn = int(spec["n"] if n is None else n)
    pr = workloads.make_problem(workload, seed=seed, m=m, n=n, device=dev, ld=workloads.pad_ld(nn))
    C = pr.C[:, : pr.n]
    ld = C.stride(0)
    X = torch.empty((pr.m, ld), dtype=torch.float32, device=dev)[:, : pr.n]
    p = torch.as_tensor(pr.p, device=dev)
    q = torch.as_tensor(pr.q, device=dev)
    mu = torch.zeros(pr.m, dtype=torch.float64, device=dev)
    nu = torch.zeros(pr.n, dtype=torch.float64, device=dev)
    return pr, C, p, q, X, mu, nu


def _final(res):
    return {k: res[k] for k in ("iters", "primal_obj", "dual_obj", "gap", "res_l1", "dual_res", "nnz")}


def _full_rule_record(args, dev, local):
    """One solve of `args.full_rule_workload` under the full stopping test (gap and l1 residual
    <= tol), timed with CUDA events, with its certificate and the smallest l1 residual of each
    tenth of the run."""
    import numpy as np
    import torch

    from paper_2110_11738_b300 import drot

    pr, C, p, q, X, mu, nu = _device_problem(args.full_rule_workload, args.seed, dev)
    rule = drot.STOP_GAP | drot.STOP_RES_L1
    # the solver's trace (<C, X_k> and the l1 residual of every iteration, written by the finish
    # kernel) shows how the l1 residual decays over the run
    trace = torch.full((2 * args.full_rule_max_iter,), float("nan"), dtype=torch.float64, device=dev)
    with drot.Solver(device=local, stop_rule=rule, autotune=True, trace=trace) as s:
        # the untimed first solve builds the plan and the graphs (a few iterations suffice)
        s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=64, X=X, mu=mu, nu=nu, check=False)
        s.reset_profile()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(local)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.full_rule_max_iter, X=X, mu=mu, nu=nu,
                      check=False)
        e1.record()
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        secs = e0.elapsed_time(e1) / 1e3
        prof = s.profile()
    cert = _certificate(C, p, q, X, mu, nu)
    l1 = trace.view(-1, 2)[: res["iters"], 1].cpu().numpy()
    del trace
    win = max(1, len(l1) // 10)
    decay = [{"iters": int(min(len(l1), (w + 1) * win)), "res_l1_min": float(np.nanmin(l1[w * win:(w + 1) * win]))}
             for w in range((len(l1) + win - 1) // win)]
    # the same workload under the gap alone, for comparison
    with drot.Solver(device=local, stop_rule=drot.STOP_GAP, autotune=True) as s:
        s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=64, X=X, mu=mu, nu=nu, check=False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        gres = s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu, check=False)
        gsecs = time.perf_counter() - t0
    gcert = _certificate(C, p, q, X, mu, nu)
    out = {"workload": args.full_rule_workload, "m": pr.m, "n": pr.n, "rule": _rule_text("full"),
           "tol": args.tol, "max_iter": args.full_rule_max_iter, "seconds": secs, "status": res["status_name"],
           "ms_per_iter": secs * 1e3 / max(1, res["iters"]), "final": dict(_final(res), certificate=cert),
           "clocks": clocks, "gpu_launches": int(prof["kernel_launches"]),
           "res_l1_decay": decay,
           "gap_rule_same_workload": {"seconds": gsecs, "status": gres["status_name"],
                                      "final": dict(_final(gres), certificate=gcert)}}
    return out


def _c_skip_record(args, C, p, q, X, mu, nu, pr, local, rule):
    """One solve of the default workload with C-load skipping (Claim 1, Sec. 3.3): passes alternate
    between reading X and C (storing X - rho C) and reading that array alone, 10 bytes per entry
    on average; the stopping test runs after the C-reading passes.  Timed with CUDA events, and
    once more with events around every fused-step launch for its roofline (10 B per entry)."""
    import torch

    from paper_2110_11738_b300 import drot

    dev = torch.device("cuda", local)
    with drot.Solver(device=local, stop_rule=rule, c_skip=True) as s:
        s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)  # warm-up
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)
        e1.record()
        torch.cuda.synchronize(dev)
        secs = e0.elapsed_time(e1) / 1e3
        plan = s.profile()
    with drot.Solver(device=local, stop_rule=rule, c_skip=True, profile=True, tile_k=plan["tile_k"]) as s:
        s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)
        s.reset_profile()
        s.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)
        prof = s.profile()
    step_ms = prof["step_ms_total"] / max(1, prof["step_launches"])
    achieved = 10.0 * pr.m * pr.n / (step_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    return {"seconds": secs, "iters": res["iters"], "status": res["status_name"],
            "ms_per_iter": secs * 1e3 / max(1, res["iters"]), "final": _final(res),
            "roofline": {"bound": "hbm", "alg_bytes_per_entry": 10, "step_ms": step_ms, "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "kernel": "drot_step_kernel<%d,1,1|2>" % prof["tile_k"]}}


def run_ours(args):
    import numpy as np
    import torch

    import workloads
    from paper_2110_11738_b300 import drot

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    pr, C, p, q, X, mu, nu = _device_problem(args.workload, args.seed, dev)
    m, n = pr.m, pr.n
    ld = C.stride(0)

    rule = {"gap": drot.STOP_GAP, "full": drot.STOP_GAP | drot.STOP_RES_L1}[args.stop]
    solver = drot.Solver(device=local, profile=False, stop_rule=rule, step_variant=args.step_variant,
                         tile_k=args.tile_k, autotune=not args.no_autotune and not args.persistent,
                         deterministic=args.deterministic, persistent=args.persistent, c_skip=args.c_skip,
                         serpentine=args.serpentine)

    def one_solve():
        return solver.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)

    for _ in range(args.warmup):
        last = one_solve()
    solver.reset_profile()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    stream = torch.cuda.current_stream(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(one_solve())
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    # the solves run on the library's stream and return after a full synchronisation,
    # so the host-side wall clock brackets them exactly; events bracket the same region
    elapsed_ms = ev0.elapsed_time(ev1)
    prof = solver.profile()

    ms_per_solve = _max_over_ranks(elapsed_ms / args.steps, world, dev)
    iters = [r["iters"] for r in results]
    statuses = sorted({r["status_name"] for r in results})
    final = _final(results[-1])
    final["certificate"] = _certificate(C, p, q, X, mu, nu)

    # Second timed region: the same solve with a CUDA event recorded around every
    # fused-step launch inside the iteration graphs (the events sit between kernels, so
    # this pass runs without programmatic dependent launch; the kernels are the same).
    psolver = drot.Solver(device=local, profile=True, stop_rule=rule, step_variant=prof["step_variant"],
                          tile_k=prof["tile_k"], deterministic=args.deterministic, persistent=args.persistent,
                          c_skip=args.c_skip, serpentine=args.serpentine)
    psolver.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)  # warm-up
    psolver.reset_profile()
    barrier()
    t0 = time.perf_counter()
    psolver.solve(C, p, q, rho=pr.rho, tol=args.tol, max_iter=args.max_iter, X=X, mu=mu, nu=nu)
    barrier()
    prof_wall_ms = (time.perf_counter() - t0) * 1e3
    pprof = psolver.profile()
    psolver.close()
    step_ms = pprof["step_ms_total"] / max(1, pprof["step_launches"])
    # C-skipping alternates 12-byte and 8-byte passes: 10 bytes per entry on average
    alg_bytes = (10 if args.c_skip else BYTES_PER_ENTRY) * m * n
    achieved = alg_bytes / (step_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    iter_ms = ms_per_solve / statistics.mean(iters)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Ch = torch.empty((m, ld), dtype=torch.float32, pin_memory=True)
        Ch.copy_(pr.C)
        ph = torch.as_tensor(pr.p).pin_memory()
        qh = torch.as_tensor(pr.q).pin_memory()
        Xh = torch.empty((m, ld), dtype=torch.float32, pin_memory=True)
        muh = torch.zeros(m, dtype=torch.float64).pin_memory()
        nuh = torch.zeros(n, dtype=torch.float64).pin_memory()
        host_call = lambda: drot.drot_solve(solver.handle, Ch[:, :n], ph, qh, rho=pr.rho, tol=args.tol,  # noqa
                                            max_iter=args.max_iter, X=Xh[:, :n], mu=muh, nu=nuh, n=n)
        host_call()  # warm the staging buffers
        barrier()
        t0 = time.perf_counter()
        e_res = [host_call() for _ in range(max(1, args.e2e_steps))]
        e_ms = (time.perf_counter() - t0) * 1e3 / max(1, args.e2e_steps)
        e2e = {"value": _max_over_ranks(e_ms, world, dev) / 1e3, "unit": "s",
               "h2d_bytes_per_step": int(Ch.numel() * 4 + ph.numel() * 8 + qh.numel() * 8),
               "d2h_bytes_per_step": int(Xh.numel() * 4 + muh.numel() * 8 + nuh.numel() * 8),
               "iters": [r["iters"] for r in e_res]}
        del Ch, Xh

    # C-load skipping (Claim 1) on the same workload
    c_skip_rec = None
    if args.c_skip_record and not args.c_skip:
        c_skip_rec = _c_skip_record(args, C, p, q, X, mu, nu, pr, local, rule)

    # the full stopping test on the 8192 x 6144 workload, and one batched solve
    full_rule = None
    if args.full_rule_workload != "none":
        full_rule = _full_rule_record(args, dev, local)
    batched = None
    if args.batched_record:
        batched = _batched_record(args, dev, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = _cpu_baseline(args.workload, args.seed, int(round(statistics.mean(iters))), "GPU count, extrapolated",
                                args.sample_iters, args.single_sample_iters, pr=pr)
        except MemoryError:
            cpu = None

    kernel_name = _step_kernel_name(pprof, args.c_skip)
    traffic = _traffic_per_launch(args.workload, kernel_name)
    tol_met = {"gap": results[-1]["gap"] <= args.tol, "res_l1": results[-1]["res_l1"] <= args.tol,
               "res_l1_at_stop": results[-1]["res_l1"],
               "note": None if results[-1]["res_l1"] <= args.tol else
               "the gap fell below tol while the plan's l1 marginal residual is still above it: see full_rule for "
               "the time to both, and final.certificate for how far the stopped plan is from optimal"}
    line = {
        "metric": METRIC,
        "value": ms_per_solve / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_solve,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "n": n, "ld": ld, "seed": args.seed, "tol": args.tol,
                   "rho": pr.rho, "stop_rule": _rule_text(args.stop),
                   "l2": f"inputs larger than L2 (C+X = {2 * m * ld * 4 / 1e6:.0f} MB > 126 MB)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "sums": "fixed-order partials" if args.deterministic else "FP64 atomics",
                   "plan": "autotuned" if not args.no_autotune and not args.persistent else "default",
                   "iteration": "persistent cooperative launch" if args.persistent else "CUDA graphs",
                   "c_skip": bool(args.c_skip),
                   "pass_order": "forward" if args.serpentine < 0 else "serpentine"},
        "iters_to_tol": iters,
        "status": statuses,
        "tolerance_met": tol_met,
        "ms_per_iter": iter_ms,
        "gpu_launches": int(prof["kernel_launches"]),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel_name,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "step_ms": step_ms, "timed_launches": int(pprof["step_launches"]),
                     "finish_ms": pprof["finish_ms_total"] / max(1, pprof["step_launches"]),
                     "step_plus_finish_ms": pprof["iter_ms_total"] / max(1, pprof["step_launches"]),
                     "iter_ms": iter_ms,
                     "iter_frac": alg_bytes / (iter_ms * 1e-3) / 1e9 / peak,
                     "timed_region": "separate profiled solve (events around each fused step); iter_ms from the "
                                     "main timed region (whole solves / iterations)",
                     "profiled_solve_ms": prof_wall_ms,
                     "alg_bytes_per_launch": alg_bytes,
                     "plan": {k: prof[k] for k in ("tile_k", "grid_ctas", "col_tiles", "graph_iters",
                                                   "step_variant", "stages")}},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "final": final,
        "c_skip": c_skip_rec,
        "full_rule": full_rule,
        "batched": batched,
    }
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["plain_8192x6144", "plain_256", "plain_20000", "batched_512", "warm_1024"])
    ap.add_argument("--batch", type=int, default=512, help="problems of the batched workload")
    ap.add_argument("--train-problems", type=int, default=1024, help="warm_1024: problems the network is trained on")
    ap.add_argument("--train-steps", type=int, default=2000, help="warm_1024: Adam steps")
    ap.add_argument("--label-tol", type=float, default=1e-4, help="warm_1024: full-rule tolerance of the labels")
    ap.add_argument("--warm-full-tol", type=float, default=1e-5,
                    help="warm_1024: tolerance of the full-rule cold/warm comparison")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--stop", choices=["gap", "full"], default="gap")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default plan")
    ap.add_argument("--persistent", action="store_true", help="one cooperative launch runs the iterations")
    ap.add_argument("--c-skip", action="store_true", help="skip the C load every other iteration (Claim 1)")
    ap.add_argument("--tile-k", type=int, default=0, choices=[0, 1, 2, 4], help="float4 chunks per lane (0: auto)")
    ap.add_argument("--deterministic", action="store_true", help="fixed-order partial sums instead of atomics")
    ap.add_argument("--step-variant", type=int, default=0, choices=[0, 1, 2, 3],
                    help="fused step: 1 register-fed, 2 TMA-fed, 3 async-copy-fed, 0 library default")
    ap.add_argument("--serpentine", type=int, default=0, choices=[-1, 0, 1],
                    help="pass order of the register-fed step: 1 alternate, -1 forward only, 0 library default")
    ap.add_argument("--max-iter", type=int, default=3_000_000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--sample-iters", type=int, default=4,
                    help="cpu_baseline: oracle iterations timed on all host cores")
    ap.add_argument("--single-sample-iters", type=int, default=2,
                    help="cpu_baseline: oracle iterations timed on one core")
    ap.add_argument("--full-rule-workload", default="auto",
                    choices=["auto", "none", "plain_8192x6144", "plain_256", "plain_20000"],
                    help="workload of the full_rule sub-record (one solve to gap and l1 residual <= tol); "
                         "auto: plain_8192x6144 on the default workload, none otherwise")
    ap.add_argument("--full-rule-max-iter", type=int, default=3_000_000)
    ap.add_argument("--batched-record", default="auto", choices=["auto", "on", "off"],
                    help="one-solve batched sub-record; auto: on for the default workload only")
    ap.add_argument("--c-skip-record", default="auto", choices=["auto", "on", "off"],
                    help="one solve with C-load skipping on the same workload; auto: default workload only")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    # the sub-records (minutes of extra work) belong to the single-GPU default line only: under
    # torchrun every rank would repeat them
    default_line = args.workload == DEFAULT_WORKLOAD and _dist()[0] == 1
    if args.full_rule_workload == "auto":
        args.full_rule_workload = FULL_RULE_WORKLOAD if default_line else "none"
    args.batched_record = args.batched_record == "on" or (args.batched_record == "auto" and default_line)
    args.c_skip_record = args.c_skip_record == "on" or (args.c_skip_record == "auto" and default_line)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up solves", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_512":
        return run_batched(args)
    if args.workload == "warm_1024":
        return run_warm(args)
    return run_ours(args)


def run_warm(args):
    """The learned warm start at m = n = 1024 (mixtures of four Gaussians, Dirichlet marginals).

    The network is trained on DROT's own solutions of `--train-problems` problems (labels from
    batched solves under the full stopping test at `--label-tol`, then Adam).  One bench step is
    one held-out problem solved cold (X_0 = p q^T) and warm (the network's dual seed, c-transform
    completed; its inference inside the timed region), both to the `--stop` test at `--tol`;
    `value` is the mean warm time.  Each held-out problem is also solved cold and warm under the
    full test (gap and l1 residual) at `--warm-full-tol`, and every gap-rule stop is certified
    (rounded feasible plan above, c-transform dual below), so the line shows what the seed
    buys under each rule."""
    import numpy as np
    import torch

    import workloads
    from paper_2110_11738_b300 import drot, warmstart

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rule = {"gap": drot.STOP_GAP, "full": drot.STOP_GAP | drot.STOP_RES_L1}[args.stop]
    full = drot.STOP_GAP | drot.STOP_RES_L1
    m = n = workloads.CONFIGS["warm_1024"]["m"]
    held = [workloads.make_problem("warm_1024", seed=20_000 + args.seed + s) for s in range(args.warmup + args.steps)]
    net = drot.Mlp(local, workloads.mlp_init_params(args.seed))
    # training problems built on the device (costs bit-identical to the host builder), labelled and
    # turned into feature rows one chunk of 512 at a time
    t0 = time.perf_counter()
    with drot.Solver(device=local, stop_rule=full, autotune=True) as lab:
        ts, lres = warmstart.labelled_training_set(
            lambda k: workloads.make_problem("warm_1024", seed=10_000 + k, device=dev), args.train_problems, net,
            lab, tol=args.label_tol, max_iter=min(args.max_iter, 2_000_000), device=local, chunk=512)
    torch.cuda.synchronize(dev)
    label_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = warmstart.train(net, ts, steps=args.train_steps, batch=8, lr=2e-3, seed=args.seed)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return out, e0.elapsed_time(e1) / 1e3

    def cert(out):
        return _certificate(out["C"], out["p"], out["q"], out["X"], out["mu"], out["nu"])["certified_rel_gap"]

    rows = []
    sampler = ClockSampler(local)
    with drot.Solver(device=local, stop_rule=rule) as solver, drot.Solver(device=local, stop_rule=full) as fsolver:
        for k, pr in enumerate(held):
            if k == args.warmup:
                sampler.start()
            cold, tc = timed(lambda: warmstart.cold_solve(solver, pr, args.tol, args.max_iter, device=local))
            warm, tw = timed(lambda: warmstart.warm_solve(net, solver, pr, args.tol, args.max_iter, device=local))
            if k < args.warmup:
                continue
            row = dict(cold_s=tc, warm_s=tw, cold_iters=cold["iters"], warm_iters=warm["iters"],
                       seeded=bool(warm["seeded"]), cold_obj=cold["primal_obj"], warm_obj=warm["primal_obj"],
                       cold_l1=cold["res_l1"], warm_l1=warm["res_l1"], cold_cert=cert(cold), warm_cert=cert(warm))
            fc, ftc = timed(lambda: warmstart.cold_solve(fsolver, pr, args.warm_full_tol, args.max_iter,
                                                         device=local))
            fw, ftw = timed(lambda: warmstart.warm_solve(net, fsolver, pr, args.warm_full_tol, args.max_iter,
                                                         device=local, fallback=False))
            row.update(full_cold_s=ftc, full_warm_s=ftw, full_cold_iters=fc["iters"], full_warm_iters=fw["iters"],
                       full_status=sorted({fc["status_name"], fw["status_name"]}))
            rows.append(row)
            del cold, warm, fc, fw
    clocks = sampler.stop()
    net.close()
    warm_s = statistics.mean(r["warm_s"] for r in rows)
    cold_s = statistics.mean(r["cold_s"] for r in rows)
    fwarm = statistics.mean(r["full_warm_iters"] for r in rows)
    fcold = statistics.mean(r["full_cold_iters"] for r in rows)
    line = {
        "metric": METRIC, "value": warm_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": warm_s * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (plan, cost), bf16 x bf16 -> f32 (network)", "data": "synthetic",
        "config": {"workload": "warm_1024", "m": m, "n": n, "seed": args.seed, "tol": args.tol,
                   "stop_rule": _rule_text(args.stop), "train_problems": args.train_problems,
                   "train_steps": args.train_steps,
                   "labels": f"batched DROT, cold start, to gap and l1 residual <= {args.label_tol:g}",
                   "l2": "problems smaller than L2 (C+X = 8 MB): latency-bound, not an HBM test"},
        "warm_vs_cold": {"rule": _rule_text(args.stop), "warm_s": warm_s, "cold_s": cold_s,
                         "speedup": cold_s / warm_s,
                         "warm_iters": [r["warm_iters"] for r in rows], "cold_iters": [r["cold_iters"] for r in rows],
                         "seeded": [r["seeded"] for r in rows],
                         "warm_res_l1": [r["warm_l1"] for r in rows], "cold_res_l1": [r["cold_l1"] for r in rows],
                         "warm_certified_rel_gap": [r["warm_cert"] for r in rows],
                         "cold_certified_rel_gap": [r["cold_cert"] for r in rows],
                         "objective_rel_diff": max(abs(r["warm_obj"] - r["cold_obj"]) / abs(r["cold_obj"])
                                                   for r in rows)},
        "warm_vs_cold_full_rule": {"rule": f"gap<={args.warm_full_tol:g} and l1 residual<={args.warm_full_tol:g}",
                                   "cold_iters": [r["full_cold_iters"] for r in rows],
                                   "warm_iters": [r["full_warm_iters"] for r in rows],
                                   "iteration_ratio_cold_over_warm": fcold / fwarm,
                                   "cold_s": statistics.mean(r["full_cold_s"] for r in rows),
                                   "warm_s": statistics.mean(r["full_warm_s"] for r in rows),
                                   "status": sorted({s for r in rows for s in r["full_status"]})},
        "training": {"label_s": label_s, "train_s": train_s,
                     "label_iters_mean": float(np.mean([r["iters"] for r in lres])),
                     "label_status": sorted({r["status_name"] for r in lres}),
                     "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:]))},
        "roofline": None,
        "e2e": None,
        "cpu_baseline": None,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _batched_problems(specs, dev):
    """Device buffers of a batch built by workloads.make_batch(device=...)."""
    import torch

    out = []
    for pr in specs:
        Cb = pr.C
        out.append(dict(C=Cb[:, : pr.n], X=torch.zeros_like(Cb)[:, : pr.n], p=torch.as_tensor(pr.p, device=dev),
                        q=torch.as_tensor(pr.q, device=dev), mu=torch.zeros(pr.m, dtype=torch.float64, device=dev),
                        nu=torch.zeros(pr.n, dtype=torch.float64, device=dev), rho=pr.rho))
    return out


def _batched_summary(specs, res, ms, tol):
    import numpy as np

    iters = np.array([r["iters"] for r in res])
    l1 = np.array([r["res_l1"] for r in res])
    alg_bytes = float(sum(12.0 * pr.m * pr.n * r["iters"] for pr, r in zip(specs, res)))
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    return {
        "iters_to_tol": {"mean": float(iters.mean()), "max": int(iters.max()), "min": int(iters.min())},
        "status": sorted({r["status_name"] for r in res}),
        "res_l1_at_stop": {"median": float(np.median(l1)), "max": float(l1.max()),
                           "share_le_tol": float((l1 <= tol).mean())},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind, "kernel": "drot_batched_step_kernel + drot_batched_narrow_kernel (whole solve)",
                     "alg_bytes": alg_bytes, "note": "12 B per entry per iteration of every unconverged problem, "
                                                     "over the whole solve's CUDA-event time"},
    }


def _batched_record(args, dev, local):
    """One solve of the 512-problem batch (gap rule), timed with CUDA events, as a sub-record."""
    import torch

    import workloads
    from paper_2110_11738_b300 import drot

    specs = workloads.make_batch(B=args.batch, seed=args.seed, device=dev)
    probs = _batched_problems(specs, dev)
    rule = {"gap": drot.STOP_GAP, "full": drot.STOP_GAP | drot.STOP_RES_L1}[args.stop]
    with drot.Solver(device=local, stop_rule=rule, autotune=True) as s:
        s.solve_batched(probs, tol=args.tol, max_iter=64, check=False)  # tile policy, graphs
        s.reset_profile()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(local)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = s.solve_batched(probs, tol=args.tol, max_iter=args.max_iter, check=False)
        e1.record()
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        prof = s.profile()
    ms = e0.elapsed_time(e1)
    out = {"workload": "batched_512", "B": len(specs), "seconds": ms / 1e3, "stop_rule": _rule_text(args.stop),
           "total_entries": int(sum(pr.m * pr.n for pr in specs)), "gpu_launches": int(prof["kernel_launches"]),
           "clocks": clocks}
    out.update(_batched_summary(specs, res, ms, args.tol))
    del probs, specs
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """The batched workload: B independent problems (m, n uniform in [64, 2048]) solved together by
    drot_solve_batched; one step = the whole batch to the stopping test.  Also times the first 32
    problems solved one after another with drot_solve for the plain-vs-batched comparison."""
    import numpy as np
    import torch

    import workloads
    from paper_2110_11738_b300 import drot

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = workloads.make_batch(B=args.batch, seed=args.seed, device=dev)
    probs = _batched_problems(specs, dev)
    rule = {"gap": drot.STOP_GAP, "full": drot.STOP_GAP | drot.STOP_RES_L1}[args.stop]
    solver = drot.Solver(device=local, stop_rule=rule, autotune=not args.no_autotune, serpentine=args.serpentine)
    for _ in range(args.warmup):
        solver.solve_batched(probs, tol=args.tol, max_iter=args.max_iter, check=False)
    sampler = ClockSampler(local)
    torch.cuda.synchronize(dev)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    results = []
    for _ in range(args.steps):
        results.append(solver.solve_batched(probs, tol=args.tol, max_iter=args.max_iter, check=False))
    ev1.record()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    prof = solver.profile()
    ms = ev0.elapsed_time(ev1) / args.steps
    res = results[-1]
    summ = _batched_summary(specs, res, ms, args.tol)
    # plain (one problem at a time) on the first 32 problems, same stopping test
    sub = min(32, len(probs))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for P in probs[:sub]:
        solver.solve(P["C"], P["p"], P["q"], rho=P["rho"], tol=args.tol, max_iter=args.max_iter, X=P["X"],
                     mu=P["mu"], nu=P["nu"], check=False)
    seq_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    solver.solve_batched(probs[:sub], tol=args.tol, max_iter=args.max_iter, check=False)
    bat_ms = (time.perf_counter() - t0) * 1e3
    solver.close()
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched_512", "B": len(specs), "m_n_range": [64, 2048], "seed": args.seed,
                   "tiles": "autotuned" if not args.no_autotune else "default",
                   "tol": args.tol, "stop_rule": args.stop, "total_entries": int(sum(pr.m * pr.n for pr in specs)),
                   "pass_order": "forward" if args.serpentine < 0 else "serpentine"},
        "iters_to_tol": summ["iters_to_tol"],
        "status": summ["status"],
        "res_l1_at_stop": summ["res_l1_at_stop"],
        "gpu_launches": int(prof["kernel_launches"]),
        "roofline": summ["roofline"],
        "plain_vs_batched_first32_ms": {"plain": seq_ms, "batched": bat_ms},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
