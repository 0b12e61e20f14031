"""Batched solver (drot_solve_batched on device buffers) against the single-problem solver
and the FP64 oracle.

Each problem of a batch runs Algorithm 1 (Sec. 3.1) with its own state and stopping test;
only the launches are shared.  So every problem must match (a) the oracle step by step from
a seeded start and (b) drot_solve on the same problem at convergence."""

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2110_11738_b300 import drot

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _dev_problem(pr, X0=None, mu0=None, nu0=None):
    ld = workloads.pad_ld(pr.n)
    Cb = torch.zeros((pr.m, ld), dtype=torch.float32, device="cuda")
    Cb[:, : pr.n] = torch.as_tensor(pr.C)
    Xb = torch.zeros_like(Cb)
    if X0 is not None:
        Xb[:, : pr.n] = torch.as_tensor(X0)
    mu = torch.as_tensor(np.zeros(pr.m) if mu0 is None else mu0, dtype=torch.float64, device="cuda").clone()
    nu = torch.as_tensor(np.zeros(pr.n) if nu0 is None else nu0, dtype=torch.float64, device="cuda").clone()
    return dict(C=Cb[:, : pr.n], X=Xb[:, : pr.n], p=torch.as_tensor(pr.p, device="cuda"),
                q=torch.as_tensor(pr.q, device="cuda"), mu=mu, nu=nu, rho=pr.rho)


def _shapes():
    return [(1, 1), (3, 7), (64, 2048), (517, 63), (200, 1029), (1000, 130), (33, 4100), (257, 257), (301, 700)]


# default: alternating pass directions within each graph; graph_iters=1: one iteration per
# replay, so the direction comes from the parity word the host rewrites between replays;
# serpentine=-1: every pass forwards; tile_k 1 and 2: 128- and 256-column tiles for every
# problem (the step kernel's narrower tile widths, which the tile-policy autotuner may pick);
# batch_narrow=1: tiles of at most 256 columns in the kernel that packs rows ((517, 63), (200, 1029),
# (33, 4100) eight rows per warp iteration, (1000, 130) and (301, 700) four; with tile_k 1 or 2 every
# tile),
# batch_narrow=-1: every tile in the wide-tile kernel
@pytest.mark.parametrize("cfg", [{}, {"graph_iters": 1}, {"serpentine": -1}, {"tile_k": 1}, {"tile_k": 2},
                                 {"tile_k": 1, "serpentine": -1}, {"batch_narrow": 1},
                                 {"batch_narrow": 1, "graph_iters": 1}, {"batch_narrow": 1, "serpentine": -1},
                                 {"batch_narrow": 1, "tile_k": 1}, {"batch_narrow": 1, "tile_k": 2},
                                 {"batch_narrow": -1}])
def test_batched_step_parity_with_oracle(cfg):
    probs, starts, specs = [], [], []
    for b, (m, n) in enumerate(_shapes()):
        pr = workloads.make_problem("plain_8192x6144", seed=100 + b, m=m, n=n)
        X0, mu0, nu0 = workloads.random_start(m, n, seed=200 + b)
        probs.append(_dev_problem(pr, X0, mu0, nu0))
        starts.append((X0, mu0, nu0))
        specs.append(pr)
    with drot.Solver(device=0, **cfg) as s:
        res = s.solve_batched(probs, tol=-1.0, max_iter=3, warm=True)
    for pr, P, (X0, mu0, nu0), r in zip(specs, probs, starts, res):
        assert r["status"] == drot.DROT_NOT_CONVERGED and r["iters"] == 3
        ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, 3, X0=X0.astype(np.float64),
                              mu0=mu0, nu0=nu0)
        S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0), np.abs(ref["X"]).max())
        Xg = P["X"].cpu().numpy().astype(np.float64)
        assert np.abs(Xg - ref["X"]).max() <= 8 * EPS32 * S * 3 * 4
        assert np.abs(P["mu"].cpu().numpy() - ref["mu"]).max() <= 64 * EPS32 * S / pr.rho * 3 + 1e-12
        assert np.abs(P["nu"].cpu().numpy() - ref["nu"]).max() <= 64 * EPS32 * S / pr.rho * 3 + 1e-12
        h = ref["history"][-1]
        assert abs(r["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9


@pytest.mark.parametrize("narrow", [0, 1])
def test_batched_solves_match_single_solves(narrow):
    specs = [workloads.make_problem("plain_256", seed=s, m=m, n=n)
             for s, (m, n) in enumerate([(40, 60), (96, 80), (61, 190), (128, 128), (20, 300)])]
    probs = [_dev_problem(pr) for pr in specs]
    with drot.Solver(device=0, batch_narrow=narrow) as s:
        res = s.solve_batched(probs, tol=1e-6, max_iter=2_000_000)
        for pr, P, r in zip(specs, probs, res):
            assert r["status"] == drot.DROT_OK, r
            Q = _dev_problem(pr)
            one = s.solve(Q["C"], Q["p"], Q["q"], rho=pr.rho, tol=1e-6, max_iter=2_000_000, X=Q["X"], mu=Q["mu"],
                          nu=Q["nu"])
            assert one["status"] == drot.DROT_OK
            obj = one["primal_obj"]
            assert abs(r["primal_obj"] - obj) <= 1e-5 * abs(obj)
            assert abs(r["iters"] - one["iters"]) <= 0.05 * one["iters"] + 5
            Xg = P["X"].cpu().numpy().astype(np.float64)
            st = oracle.plan_stats(pr.C.astype(np.float64), pr.p, pr.q, Xg, P["mu"].cpu().numpy(),
                                   P["nu"].cpu().numpy())
            assert st["res_l1"] <= 1.5e-6 and st["gap"] <= 1.5e-6
            assert r["nnz"] == int((Xg > 0).sum())


def test_batched_reports_per_problem_status():
    good = workloads.make_problem("plain_256", seed=1, m=30, n=40)
    bad = workloads.make_problem("plain_256", seed=2, m=30, n=40)
    P_good, P_bad = _dev_problem(good), _dev_problem(bad)
    P_bad["q"] = P_bad["q"] * 1.5  # mass mismatch
    with drot.Solver(device=0) as s:
        res = s.solve_batched([P_good, P_bad, _dev_problem(good)], tol=1e-6, max_iter=1_000_000, check=False)
    assert res[0]["status"] == drot.DROT_OK and res[2]["status"] == drot.DROT_OK
    assert res[1]["status"] == drot.DROT_ERR_MARGINALS
    assert res[0]["primal_obj"] == pytest.approx(res[2]["primal_obj"], rel=1e-6)


@pytest.mark.parametrize("narrow", [0, 1])
def test_batched_uneven_config_subset_iteration_cap(narrow):
    # 24 problems drawn like the 512-problem workload (m, n uniform in [64, 2048], shifted
    # clouds, Dirichlet marginals), a fixed iteration budget: every problem must agree with
    # its own single solve after the same number of iterations
    specs = workloads.make_batch(B=24, seed=3)
    probs = [_dev_problem(pr) for pr in specs]
    with drot.Solver(device=0, batch_narrow=narrow) as s:
        res = s.solve_batched(probs, tol=-1.0, max_iter=200)
        for pr, P, r in zip(specs[:6], probs[:6], res[:6]):
            assert r["iters"] == 200
            Q = _dev_problem(pr)
            one = s.solve(Q["C"], Q["p"], Q["q"], rho=pr.rho, tol=-1.0, max_iter=200, X=Q["X"], mu=Q["mu"], nu=Q["nu"])
            assert abs(r["primal_obj"] - one["primal_obj"]) <= 1e-5 * abs(one["primal_obj"])
            assert abs(r["res_l1"] - one["res_l1"]) <= 1e-4 * one["res_l1"] + 1e-9
            S = pr.rho * 4
            assert float((P["X"] - Q["X"]).abs().max()) <= 8 * EPS32 * S * 200


def test_batched_autotuned_tiles_keep_parity():
    """The tile-policy autotuner times the step on the caller's X before the cold start
    writes X_0 and then zeroes the totals it touched: the solve must agree with the
    untuned one, problem by problem, and a warm batch on the same handle must be untouched."""
    specs = workloads.make_batch(B=16, seed=5)
    with drot.Solver(device=0) as s:
        base = [_dev_problem(pr) for pr in specs]
        ref = s.solve_batched(base, tol=-1.0, max_iter=150)
    with drot.Solver(device=0, autotune=True) as s:
        for _ in range(2):  # the second call reuses the tuned policy
            probs = [_dev_problem(pr) for pr in specs]
            for P in probs:
                P["X"].fill_(float("nan"))  # whatever X holds before a cold start is overwritten
            res = s.solve_batched(probs, tol=-1.0, max_iter=150)
            for pr, P, r, r0, B0 in zip(specs, probs, res, ref, base):
                assert r["iters"] == 150
                assert abs(r["primal_obj"] - r0["primal_obj"]) <= 1e-5 * abs(r0["primal_obj"])
                assert abs(r["res_l1"] - r0["res_l1"]) <= 1e-4 * r0["res_l1"] + 1e-9
                assert float((P["X"] - B0["X"]).abs().max()) <= 8 * EPS32 * pr.rho * 4 * 150
        # warm start from the untuned results: no tuning launches touch the given X
        warm = [dict(P, X=P["X"].clone(), mu=P["mu"].clone(), nu=P["nu"].clone()) for P in base]
        X_in = [P["X"].clone() for P in warm]
        res_w = s.solve_batched(warm, tol=-1.0, max_iter=0, warm=True)
        for P, X0 in zip(warm, X_in):
            assert torch.equal(P["X"], X0)


def test_full_512_problem_batch_in_the_benchmark_configuration():
    """The whole 512-problem workload (m, n uniform in [64, 2048], seed 0), launched the way the
    benchmark launches it: cold start, autotuned tile policy, duality-gap stopping rule, serpentine
    passes.  Three iterations of every problem; then, for all 512, properties that hold at any size
    (X >= 0, the reported <C, X> and l1 marginal residual equal an FP64 recomputation from the
    returned plan), and for six sampled problems (the largest, the smallest, four seeded picks) the
    plan, the duals and the objective against the FP64 oracle run from the same X_0 = p q^T
    (rounded to FP32 as the GPU stores it)."""
    k = 3
    specs = workloads.make_batch(B=512, seed=0)
    probs = [_dev_problem(pr) for pr in specs]
    with drot.Solver(device=0, stop_rule=drot.STOP_GAP, autotune=True) as s:
        res = s.solve_batched(probs, tol=-1.0, max_iter=k, check=False)
    assert len(res) == 512
    for pr, P, r in zip(specs, probs, res):
        assert r["status"] == drot.DROT_NOT_CONVERGED and r["iters"] == k, (pr.name, r)
        Xd = P["X"].to(torch.float64)
        assert float(Xd.min()) >= 0.0
        Cd = P["C"].to(torch.float64)
        primal = float((Cd * Xd).sum())
        res_l1 = float((Xd.sum(1) - P["p"]).abs().sum() + (Xd.sum(0) - P["q"]).abs().sum())
        assert abs(primal - r["primal_obj"]) <= 1e-5 * abs(primal) + 1e-12, (pr.name, primal, r["primal_obj"])
        assert abs(res_l1 - r["res_l1"]) <= 1e-5 * res_l1 + 1e-7, (pr.name, res_l1, r["res_l1"])
    sizes = np.array([pr.m * pr.n for pr in specs])
    picks = {int(sizes.argmax()), int(sizes.argmin())}
    picks |= {int(b) for b in np.random.default_rng(1).choice(512, size=4, replace=False)}
    for b in sorted(picks):
        pr, P, r = specs[b], probs[b], res[b]
        X0 = np.outer(pr.p, pr.q).astype(np.float32).astype(np.float64)
        ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, k, X0=X0, mu0=np.zeros(pr.m),
                              nu0=np.zeros(pr.n))
        S = max(np.abs(X0).max(), pr.rho, np.abs(ref["X"]).max())
        Xg = P["X"].cpu().numpy().astype(np.float64)
        assert np.abs(Xg - ref["X"]).max() <= 8 * EPS32 * S * k * 4, pr.name
        assert np.abs(P["mu"].cpu().numpy() - ref["mu"]).max() <= 64 * EPS32 * S / pr.rho * k + 1e-12, pr.name
        assert np.abs(P["nu"].cpu().numpy() - ref["nu"]).max() <= 64 * EPS32 * S / pr.rho * k + 1e-12, pr.name
        h = ref["history"][-1]
        assert abs(r["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9, pr.name
        assert abs(r["res_l1"] - h[oracle.RES_L1]) <= 1e-5 * abs(h[oracle.RES_L1]) + 1e-7, pr.name


def test_batched_with_host_buffers_matches_the_oracle():
    """drot_solve_batched on host (NumPy) buffers stages each problem through the device and
    solves it with drot_solve's path; five cold-started iterations of each problem must match
    the FP64 oracle from the same X_0 = p q^T (rounded to FP32)."""
    k = 5
    specs, probs = [], []
    for b, (m, n) in enumerate([(3, 7), (130, 257), (64, 2048)]):
        pr = workloads.make_problem("plain_8192x6144", seed=700 + b, m=m, n=n)
        ld = workloads.pad_ld(n)
        Ch = np.zeros((m, ld), np.float32)
        Ch[:, :n] = pr.C
        Xh = np.full((m, ld), 5.0, np.float32)  # a cold start overwrites the plan; the padding stays
        probs.append(dict(C=Ch[:, :n], X=Xh[:, :n], p=pr.p.copy(), q=pr.q.copy(), mu=np.zeros(m), nu=np.zeros(n),
                          rho=pr.rho, Xfull=Xh))
        specs.append(pr)
    with drot.Solver(device=0) as s:
        res = drot.drot_solve_batched(s.handle, probs, tol=-1.0, max_iter=k, check=False)
    for pr, P, r in zip(specs, probs, res):
        assert r["status"] == drot.DROT_NOT_CONVERGED and r["iters"] == k
        X0 = np.outer(pr.p, pr.q).astype(np.float32).astype(np.float64)
        ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, k, X0=X0, mu0=np.zeros(pr.m),
                              nu0=np.zeros(pr.n))
        S = max(np.abs(X0).max(), pr.rho, np.abs(ref["X"]).max())
        assert np.abs(P["X"].astype(np.float64) - ref["X"]).max() <= 8 * EPS32 * S * k * 4
        assert np.abs(P["mu"] - ref["mu"]).max() <= 64 * EPS32 * S / pr.rho * k + 1e-12
        assert np.abs(P["nu"] - ref["nu"]).max() <= 64 * EPS32 * S / pr.rho * k + 1e-12
        assert np.all(P["Xfull"][:, pr.n:] == 5.0)
        h = ref["history"][-1]
        assert abs(r["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9
