"""CUDA path vs the FP64 oracle, through the C ABI.

Two kinds of comparison:
* step parity: both sides start from the same seeded state (X_0, mu_0, nu_0) and
  run exactly k iterations of Algorithm 1; X_k is compared entry by entry and
  the duals and stopping quantities value by value;
* solve parity: both sides run to the stopping test at tol 1e-6; objective,
  dual objective and residuals are compared (the optimal plan and the duals
  need not be unique, Prop. 1, so X and the duals are not compared entrywise).

Tolerances follow from FP32 iterates: each entry update x + phi + psi - rho c
rounds at most a few times at unit roundoff eps32 = 2^-24 of the largest term
S = max(|x|, |phi|, |psi|, rho |c|), so |x_gpu - x_ref| <= 8 eps32 S per step;
the row and column sums that feed phi and psi inherit n (or m) such errors and
are divided by n (m), so mu and nu move by O(eps32 S / rho).
"""

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2110_11738_b300 import drot

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def solver():
    s = drot.Solver(device=0)
    yield s
    s.close()


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def _gpu_inputs(pr, X0=None, mu0=None, nu0=None):
    C = drot.padded_matrix(pr.C, device="cuda")
    X = torch.zeros_like(C.as_strided((C.shape[0], C.stride(0)), (C.stride(0), 1)))[:, : pr.n]
    if X0 is not None:
        X.copy_(torch.as_tensor(X0, dtype=torch.float32))
    mu = _dev(mu0 if mu0 is not None else np.zeros(pr.m), torch.float64)
    nu = _dev(nu0 if nu0 is not None else np.zeros(pr.n), torch.float64)
    return C, _dev(pr.p, torch.float64), _dev(pr.q, torch.float64), X, mu, nu


def _step_parity(solver, pr, k, seed, stats_k=None):
    X0, mu0, nu0 = workloads.random_start(pr.m, pr.n, seed)
    C, p, q, X, mu, nu = _gpu_inputs(pr, X0, mu0, nu0)
    out = solver.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=k, X=X, mu=mu, nu=nu, warm=True)
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == k
    ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, k, X0=X0.astype(np.float64), mu0=mu0, nu0=nu0)
    Xg = X.cpu().numpy().astype(np.float64)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0), np.abs(ref["X"]).max())
    tol_x = 8 * EPS32 * S * k * 4
    err_x = np.abs(Xg - ref["X"]).max()
    assert err_x <= tol_x, (err_x, tol_x)
    assert Xg.min() >= 0.0
    tol_d = 64 * EPS32 * S / pr.rho * k + 1e-12
    assert np.abs(mu.cpu().numpy() - ref["mu"]).max() <= tol_d
    assert np.abs(nu.cpu().numpy() - ref["nu"]).max() <= tol_d
    h = ref["history"][(stats_k or k) - 1]
    assert abs(out["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9
    assert abs(out["res_l1"] - h[oracle.RES_L1]) <= 1e-5 * abs(h[oracle.RES_L1]) + 1e-7
    assert abs(out["dual_res"] - h[oracle.DUAL_RES_PREV]) <= 1e-4 * abs(h[oracle.DUAL_RES_PREV]) + 1e-6
    return out


@pytest.mark.parametrize("m,n", [(1, 1), (1, 5), (2, 2), (3, 7), (2, 31), (31, 33), (33, 129), (130, 257),
                                 (257, 1031), (300, 2053), (64, 4100), (17, 3)])
@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("cluster", [0, 1])  # automatic choice (cluster-resident when it fits) / streaming path
def test_step_parity_small_and_ragged(m, n, k, cluster):
    pr = workloads.make_problem("plain_8192x6144", seed=m * 1000 + n, m=m, n=n)
    with drot.Solver(device=0, cluster=cluster) as s:
        _step_parity(s, pr, k, seed=m + n + k)


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("tile_k", [1, 2, 4])
@pytest.mark.parametrize("grid", [37, 0])
def test_step_parity_every_variant_and_tile_width(variant, tile_k, grid):
    pr = workloads.make_problem("plain_256", seed=5, m=203, n=1337)
    with drot.Solver(device=0, tile_k=tile_k, grid_ctas=grid, step_variant=variant) as s:
        _step_parity(s, pr, 2, seed=9)
        assert s.profile()["step_variant"] == variant and s.profile()["tile_k"] == tile_k


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("tile_k", [1, 4])
@pytest.mark.parametrize("k", [2, 5])
def test_forward_only_order_keeps_parity(variant, tile_k, k):
    """serpentine=-1: every pass walks forwards; the default alternates (odd passes
    walk each CTA's rows backwards).  Both are the same iteration in another order of
    the partial sums."""
    pr = workloads.make_problem("plain_256", seed=6, m=211, n=1100)
    with drot.Solver(device=0, tile_k=tile_k, grid_ctas=29, step_variant=variant, serpentine=-1) as s:
        _step_parity(s, pr, k, seed=10)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_serpentine_first_pass_is_forward_and_orders_agree(variant):
    pr = workloads.make_problem("plain_8192x6144", seed=17, m=333, n=1500)
    X0, mu0, nu0 = workloads.random_start(pr.m, pr.n, seed=3)
    res = {}
    for serp in (1, -1):
        for k in (1, 40):
            C, p, q, X, mu, nu = _gpu_inputs(pr, X0, mu0, nu0)
            with drot.Solver(device=0, deterministic=True, step_variant=variant, grid_ctas=41,
                             serpentine=serp) as s:
                s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=k, X=X, mu=mu, nu=nu, warm=True)
            res[serp, k] = (X.cpu().numpy(), mu.cpu().numpy())
    # one pass: both orders walk forwards, bit for bit the same
    assert np.array_equal(res[1, 1][0], res[-1, 1][0]) and np.array_equal(res[1, 1][1], res[-1, 1][1])
    # forty passes: the orders differ only in the rounding of the partial sums
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0))
    assert np.abs(res[1, 40][0].astype(np.float64) - res[-1, 40][0]).max() <= 8 * EPS32 * S * 40
    assert np.abs(res[1, 40][1] - res[-1, 40][1]).max() <= 64 * EPS32 * S / pr.rho * 40


def test_serpentine_with_an_odd_replay_length():
    """An odd graph length puts two passes of one direction back to back at every replay
    boundary: only the order changes, the iterates still follow the oracle."""
    pr = workloads.make_problem("plain_256", seed=8, m=150, n=700)
    with drot.Solver(device=0, graph_iters=3, grid_ctas=23) as s:
        _step_parity(s, pr, 7, seed=12)


def test_variants_agree_bitwise_on_a_solve():
    # the three fused-step variants perform the same FP32 operations in the same order
    # per entry, walk the rows in the same (serpentine) order and write the same
    # partials, so whole runs agree bit for bit
    pr = workloads.make_problem("plain_8192x6144", seed=12, m=517, n=1029)
    outs = {}
    for v in (1, 2, 3):
        C, p, q, X, mu, nu = _gpu_inputs(pr)
        with drot.Solver(device=0, step_variant=v, tile_k=2, grid_ctas=53, deterministic=True) as s:
            o = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=300, X=X, mu=mu, nu=nu)
        outs[v] = (X.cpu().numpy(), mu.cpu().numpy(), o["primal_obj"])
    for v in (2, 3):
        assert np.array_equal(outs[1][0], outs[v][0])
        assert np.array_equal(outs[1][1], outs[v][1]) and outs[1][2] == outs[v][2]


def test_step_parity_full_size_8192x6144(solver):
    pr = workloads.make_problem("plain_8192x6144", seed=0)
    _step_parity(solver, pr, 2, seed=1)


@pytest.mark.slow
def test_step_parity_full_size_20000(solver):
    # three passes: forward, backward (serpentine order) and forward again over 40 column tiles
    # (the last one 32 columns wide), every CTA of the fused step
    pr = workloads.make_problem("plain_20000", seed=0)
    _step_parity(solver, pr, 3, seed=2)


def _solve_parity(solver, pr, tol=1e-6, rel_obj=1e-5):
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    out = solver.solve(C, p, q, rho=pr.rho, tol=tol, max_iter=2_000_000, X=X, mu=mu, nu=nu)
    assert out["status"] == drot.DROT_OK, out
    ref = oracle.drot_solve(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, tol, 2_000_000)
    assert ref["status"] == oracle.STATUS_CONVERGED
    obj = ref["stats"]["primal"]
    assert abs(out["primal_obj"] - obj) <= rel_obj * abs(obj)
    # both runs end with gap <= tol, so their dual objectives differ by at most the
    # primal difference plus 2 tol (the runs may stop a few iterations apart)
    assert abs(out["dual_obj"] - ref["stats"]["dual"]) <= rel_obj * abs(obj) + 2 * tol
    # residuals recomputed in FP64 from the returned plan
    Xg = X.cpu().numpy().astype(np.float64)
    st = oracle.plan_stats(pr.C.astype(np.float64), pr.p, pr.q, Xg, mu.cpu().numpy(), nu.cpu().numpy())
    assert st["res_l1"] <= 1e-6 * 1.5
    assert abs(st["primal"] - out["primal_obj"]) <= 1e-6 * abs(obj)
    assert st["gap"] <= 1e-6 * 1.5
    return out, ref


def test_solve_parity_plain_256(solver):
    pr = workloads.make_problem("plain_256", seed=0)
    out, ref = _solve_parity(solver, pr)
    assert 0.5 * ref["iters"] <= out["iters"] <= 2.0 * ref["iters"]


@pytest.mark.parametrize("name,m,n", [("warm_1024", 96, 80), ("plain_8192x6144", 130, 47), ("plain_256", 61, 190)])
def test_solve_parity_other_shapes(solver, name, m, n):
    pr = workloads.make_problem(name, seed=1, m=m, n=n)
    _solve_parity(solver, pr)


def test_golden_lp_optima(solver):
    import json
    import os
    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lp_optima.json")))["cases"]
    for case in cases:
        pr = workloads.make_problem(case["config"], seed=case["seed"], m=case["m"], n=case["n"])
        C, p, q, X, mu, nu = _gpu_inputs(pr)
        out = solver.solve(C, p, q, rho=pr.rho, tol=1e-6, max_iter=2_000_000, X=X, mu=mu, nu=nu)
        assert out["status"] == drot.DROT_OK
        opt = case["lp_optimum"]
        assert abs(out["primal_obj"] - opt) <= 1e-5 * abs(opt) + 2e-6, (case, out["primal_obj"])


def test_full_size_8192x6144_certificate(solver):
    """At the full size the oracle cannot run to convergence; after a fixed number of
    iterations check properties that hold at any size: nonnegativity, the reported
    stopping quantities against an FP64 recomputation from the returned plan and duals,
    and weak duality: the c-transform nu'_j = min_i (C_ij - mu_i) makes (mu, nu') dual
    feasible, so p^T mu + q^T nu' is a lower bound on the optimum."""
    pr = workloads.make_problem("plain_8192x6144", seed=0)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    out = solver.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=60_000, X=X, mu=mu, nu=nu)
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == 60_000
    Cd = torch.as_tensor(pr.C, device="cuda", dtype=torch.float64)
    Xd = X.to(torch.float64)
    r = Xd.sum(1) - p
    s_ = Xd.sum(0) - q
    res_l1 = float(r.abs().sum() + s_.abs().sum())
    primal = float((Cd * Xd).sum())
    dual = float(p @ mu + q @ nu)
    assert float(X.min()) >= 0.0
    assert abs(res_l1 - out["res_l1"]) <= 1e-3 * res_l1 + 1e-9
    assert abs(primal - out["primal_obj"]) <= 1e-6 * primal
    assert abs(dual - out["dual_obj"]) <= 1e-6 * abs(dual) + 1e-12
    assert out["res_l1"] < 1e-3 and out["gap"] < 1e-4
    nu_c = (Cd - mu[:, None]).min(dim=0).values
    lower = float(p @ mu + q @ nu_c)
    opt_gap = primal - lower
    assert opt_gap >= -2 * res_l1  # an infeasible plan may undercut the optimum by at most ~res_l1 * max C
    assert opt_gap <= 1e-2 * primal, (primal, lower)
    del Cd, Xd


@pytest.mark.parametrize("rule", [drot.STOP_GAP, drot.STOP_GAP | drot.STOP_RES_L1 | drot.STOP_DUAL_RES])
def test_stop_rules_match_oracle(rule):
    pr = workloads.make_problem("plain_256", seed=11, m=48, n=40)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    tol = 1e-6 if rule == drot.STOP_GAP else 1e-5
    with drot.Solver(device=0, stop_rule=rule) as s:
        out = s.solve(C, p, q, rho=pr.rho, tol=tol, max_iter=2_000_000, X=X, mu=mu, nu=nu)
    ref = oracle.drot_solve(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, tol, 2_000_000, stop_rule=rule)
    assert out["status"] == drot.DROT_OK and ref["status"] == oracle.STATUS_CONVERGED
    assert out["gap"] <= tol
    if rule & drot.STOP_DUAL_RES:
        assert out["dual_res"] <= tol and out["res_l1"] <= tol
    assert 0.5 * ref["iters"] <= out["iters"] <= 2.0 * ref["iters"] + 5


@pytest.mark.parametrize("m,n", [(300, 2600), (1000, 200)])
def test_autotune_picks_a_plan_and_keeps_parity(m, n):
    pr = workloads.make_problem("plain_8192x6144", seed=m + n, m=m, n=n)
    with drot.Solver(device=0, autotune=True, cluster=1) as s:
        _step_parity(s, pr, 2, seed=5)
        prof = s.profile()
        assert prof["step_variant"] in (1, 2, 3) and prof["tile_k"] in (1, 2, 4)
        first = (prof["step_variant"], prof["tile_k"])
        _step_parity(s, pr, 1, seed=6)  # the choice is cached per shape
        prof = s.profile()
        assert (prof["step_variant"], prof["tile_k"]) == first


@pytest.mark.parametrize("m,n", [(1, 1), (3, 7), (33, 129), (257, 1031), (300, 2053), (1000, 64)])
def test_persistent_step_parity(m, n):
    pr = workloads.make_problem("plain_8192x6144", seed=m * 7 + n, m=m, n=n)
    with drot.Solver(device=0, persistent=True) as s:
        _step_parity(s, pr, 3, seed=m + 2 * n)
        assert s.profile()["kernel_launches"] >= 1


def test_persistent_solve_parity_plain_256():
    pr = workloads.make_problem("plain_256", seed=0)
    with drot.Solver(device=0, persistent=True) as s:
        out, ref = _solve_parity(s, pr)
    assert 0.5 * ref["iters"] <= out["iters"] <= 2.0 * ref["iters"]


def test_persistent_matches_graph_iteration():
    pr = workloads.make_problem("plain_8192x6144", seed=21, m=900, n=700)
    outs = []
    for persistent in (False, True):
        C, p, q, X, mu, nu = _gpu_inputs(pr)
        with drot.Solver(device=0, persistent=persistent, step_variant=1) as s:
            o = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=500, X=X, mu=mu, nu=nu)
        outs.append((X.cpu().numpy().astype(np.float64), o))
    assert outs[0][1]["iters"] == outs[1][1]["iters"] == 500
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 1e-6 * np.abs(outs[0][0]).max()
    assert abs(outs[0][1]["primal_obj"] - outs[1][1]["primal_obj"]) <= 1e-6 * outs[0][1]["primal_obj"]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("m,n", [(33, 129), (257, 1031), (64, 4100)])
def test_c_skip_step_parity(m, n, k):
    # Claim 1 schedule: the array holds X - rho C after each C-reading pass; the solver
    # restores X when it stops on one, so X_k matches the oracle for odd and even k
    pr = workloads.make_problem("plain_8192x6144", seed=m + 3 * n, m=m, n=n)
    with drot.Solver(device=0, c_skip=True) as s:
        # after a C-free pass the stopping quantities are those of the preceding C-reading pass
        _step_parity(s, pr, k, seed=k + m, stats_k=k if k % 2 else k - 1)


def test_c_skip_solve_parity_plain_256():
    pr = workloads.make_problem("plain_256", seed=0)
    with drot.Solver(device=0, c_skip=True) as s:
        out, ref = _solve_parity(s, pr)
    assert out["iters"] % 2 == 1  # the test only runs after C-reading passes
    assert 0.5 * ref["iters"] <= out["iters"] <= 2.0 * ref["iters"]


@pytest.mark.parametrize("m,n", [(16, 16), (33, 129), (256, 256), (100, 700), (300, 64), (517, 200)])
@pytest.mark.parametrize("k", [1, 4])
def test_cluster_step_parity(m, n, k):
    pr = workloads.make_problem("plain_8192x6144", seed=m * 11 + n, m=m, n=n)
    with drot.Solver(device=0, cluster=2) as s:
        _step_parity(s, pr, k, seed=m + n + 5 * k)
        assert s.profile()["step_variant"] == 4  # cluster-resident path taken


def test_cluster_solve_parity_plain_256():
    pr = workloads.make_problem("plain_256", seed=0)
    with drot.Solver(device=0, cluster=2) as s:
        out, ref = _solve_parity(s, pr)
        assert s.profile()["step_variant"] == 4
    assert 0.5 * ref["iters"] <= out["iters"] <= 2.0 * ref["iters"]


# grid-resident solve (cluster=3): the rows of X and C in the shared memory of one CTA per SM,
# one CTA per row block (a single row for m <= 148), ragged last blocks, columns owned in blocks
@pytest.mark.parametrize("m,n", [(1, 1), (3, 7), (33, 129), (148, 200), (149, 301), (300, 2053), (1000, 1000),
                                 (1536, 2048)])
@pytest.mark.parametrize("k", [1, 4])
def test_grid_resident_step_parity(m, n, k):
    pr = workloads.make_problem("plain_8192x6144", seed=m * 13 + n, m=m, n=n)
    with drot.Solver(device=0, cluster=3) as s:
        _step_parity(s, pr, k, seed=m + n + 7 * k)
        assert s.profile()["step_variant"] == 6  # grid-resident path taken


def test_grid_resident_solve_parity_plain_256():
    pr = workloads.make_problem("plain_256", seed=0)
    with drot.Solver(device=0, cluster=3) as s:
        out, ref = _solve_parity(s, pr)
        assert s.profile()["step_variant"] == 6
    assert 0.5 * ref["iters"] <= out["iters"] <= 2.0 * ref["iters"]


def test_cluster_required_but_too_large():
    pr = workloads.make_problem("plain_256", seed=1, m=1200, n=1100)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    with drot.Solver(device=0, cluster=2) as s:
        with pytest.raises(drot.DrotError) as e:
            s.solve(C, p, q, rho=pr.rho, tol=1e-6, max_iter=10, X=X, mu=mu, nu=nu)
    assert e.value.status == drot.DROT_ERR_INVALID_ARG


def test_max_iter_zero_returns_cold_start(solver):
    pr = workloads.make_problem("plain_256", seed=2, m=9, n=13)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    out = solver.solve(C, p, q, rho=pr.rho, tol=1e-6, max_iter=0, X=X, mu=mu, nu=nu)
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == 0
    ref = np.outer(pr.p, pr.q).astype(np.float32)
    assert np.array_equal(X.cpu().numpy(), ref)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_deterministic_mode_bitwise(variant):
    pr = workloads.make_problem("plain_8192x6144", seed=3, m=700, n=900)
    outs = []
    for _ in range(2):
        C, p, q, X, mu, nu = _gpu_inputs(pr)
        with drot.Solver(device=0, deterministic=True, step_variant=variant) as s:
            o = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=50, X=X, mu=mu, nu=nu)
        outs.append((X.cpu().numpy().copy(), mu.cpu().numpy().copy(), o["primal_obj"], o["gap"]))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2] and outs[0][3] == outs[1][3]


def test_host_buffers_match_device_buffers():
    solver = drot.Solver(device=0, deterministic=True)
    pr = workloads.make_problem("plain_256", seed=4, m=100, n=77)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    od = solver.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=40, X=X, mu=mu, nu=nu)
    ld = workloads.pad_ld(pr.n)
    Ch = np.zeros((pr.m, ld), np.float32)
    Ch[:, : pr.n] = pr.C
    Xh = np.zeros_like(Ch)
    muh = np.zeros(pr.m)
    nuh = np.zeros(pr.n)
    oh = drot.drot_solve(solver.handle, Ch, pr.p.copy(), pr.q.copy(), rho=pr.rho, tol=-1.0, max_iter=40, X=Xh,
                         mu=muh, nu=nuh, n=pr.n)
    assert oh["iters"] == od["iters"] == 40
    assert np.array_equal(Xh[:, : pr.n], X.cpu().numpy())
    assert np.array_equal(muh, mu.cpu().numpy())
    solver.close()


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_accumulation_and_fixed_order_modes_agree(variant):
    # the two summation modes differ only in the order of FP64 additions
    pr = workloads.make_problem("plain_8192x6144", seed=13, m=300, n=1100)
    X0, mu0, nu0 = workloads.random_start(pr.m, pr.n, seed=4)
    res = {}
    for det in (False, True):
        C, p, q, X, mu, nu = _gpu_inputs(pr, X0, mu0, nu0)
        with drot.Solver(device=0, deterministic=det, step_variant=variant) as s:
            o = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=20, X=X, mu=mu, nu=nu, warm=True)
        res[det] = (X.cpu().numpy().astype(np.float64), mu.cpu().numpy(), o)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0))
    assert np.abs(res[False][0] - res[True][0]).max() <= 8 * EPS32 * S * 20
    assert np.abs(res[False][1] - res[True][1]).max() <= 64 * EPS32 * S / pr.rho * 20
    assert abs(res[False][2]["primal_obj"] - res[True][2]["primal_obj"]) <= 1e-6 * abs(res[True][2]["primal_obj"])


def test_padding_columns_untouched(solver):
    pr = workloads.make_problem("plain_256", seed=6, m=20, n=29)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    base = X.as_strided((pr.m, X.stride(0)), (X.stride(0), 1))
    base[:, pr.n:] = 7.0
    solver.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=5, X=X, mu=mu, nu=nu)
    assert float(base[:, pr.n:].sub(7.0).abs().max()) == 0.0


def test_argument_errors(solver):
    pr = workloads.make_problem("plain_256", seed=7, m=8, n=8)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    h = solver.handle
    with pytest.raises(drot.DrotError) as e:
        drot.drot_solve(h, C, p, q, X=X, mu=mu, nu=nu, max_iter=-1)
    assert e.value.status == drot.DROT_ERR_INVALID_ARG
    bad_q = q * 1.01
    with pytest.raises(drot.DrotError) as e:
        drot.drot_solve(h, C, p, bad_q, X=X, mu=mu, nu=nu)
    assert e.value.status == drot.DROT_ERR_MARGINALS
    neg = p.clone()
    neg[0] = -neg[0]
    neg[1] += 2 * p[0]
    with pytest.raises(drot.DrotError) as e:
        drot.drot_solve(h, C, neg, q, X=X, mu=mu, nu=nu)
    assert e.value.status == drot.DROT_ERR_MARGINALS
    # unaligned C: offset the base by one float
    raw = torch.zeros(8 * 8 + 1, device="cuda", dtype=torch.float32)
    Cu = raw[1:].view(8, 8)
    with pytest.raises(drot.DrotError) as e:
        drot.drot_solve(h, Cu, p, q, X=X, mu=mu, nu=nu)
    assert e.value.status == drot.DROT_ERR_INVALID_ARG
    # mixed host/device buffers
    with pytest.raises(drot.DrotError) as e:
        drot.drot_solve(h, C, pr.p.copy(), q, X=X, mu=mu, nu=nu)
    assert e.value.status == drot.DROT_ERR_INVALID_ARG


def test_nonfinite_cost_is_reported(solver):
    pr = workloads.make_problem("plain_256", seed=8, m=16, n=16)
    C, p, q, X, mu, nu = _gpu_inputs(pr)
    C[3, 5] = float("nan")
    out = drot.drot_solve(solver.handle, C, p, q, rho=pr.rho, tol=1e-6, max_iter=100, X=X, mu=mu, nu=nu,
                          check=False)
    assert out["status"] == drot.DROT_ERR_NONFINITE
    assert out["iters"] == 1


@pytest.mark.parametrize("cfg", [{"cluster": 1}, {"cluster": 2}, "batched"])
def test_resume_from_returned_state_retraces_the_run(cfg):
    """Checkpoint and resume: the state an interrupted solve returns, (X_k, mu_k, nu_k), is a
    complete checkpoint, because a warm start rebuilds a, b and alpha from their definitions
    (a = Y e - p with Y = X + phi e^T + f psi^T, Sec. 3.1).  Three iterations, then three more
    from the returned state, must match six uninterrupted iterations of the FP64 oracle."""
    k1, k2 = 3, 3
    pr = workloads.make_problem("plain_8192x6144", seed=41, m=130, n=257)
    X0, mu0, nu0 = workloads.random_start(pr.m, pr.n, seed=42)
    C, p, q, X, mu, nu = _gpu_inputs(pr, X0, mu0, nu0)
    with drot.Solver(device=0, **({} if cfg == "batched" else cfg)) as s:
        for k in (k1, k2):
            if cfg == "batched":
                out = s.solve_batched([dict(C=C, p=p, q=q, X=X, mu=mu, nu=nu, rho=pr.rho)], tol=-1.0, max_iter=k,
                                      warm=True, check=False)[0]
            else:
                out = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=k, X=X, mu=mu, nu=nu, warm=True, check=False)
            assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == k
    k = k1 + k2
    ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, k, X0=X0.astype(np.float64), mu0=mu0, nu0=nu0)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0), np.abs(ref["X"]).max())
    assert np.abs(X.cpu().numpy().astype(np.float64) - ref["X"]).max() <= 8 * EPS32 * S * k * 4
    tol_d = 64 * EPS32 * S / pr.rho * k + 1e-12
    assert np.abs(mu.cpu().numpy() - ref["mu"]).max() <= tol_d
    assert np.abs(nu.cpu().numpy() - ref["nu"]).max() <= tol_d
    h = ref["history"][-1]
    assert abs(out["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9
    assert abs(out["res_l1"] - h[oracle.RES_L1]) <= 1e-5 * abs(h[oracle.RES_L1]) + 1e-7
