"""Pins for the FP64 oracle: each check compares it with something other than itself.

* the three-variable DR form (eq. drot:general:form) with Lemma 1's projection,
  itself checked against a generic least-squares projection;
* the identities of Appendix A.2 (Lemma var:repr) and the a_k recursion (Sec. 3.1);
* firm nonexpansiveness of the DR operator (Appendix A): ||Y_{k+1} - Y_k|| non-increasing;
* Theorem 1 (Sec. 3.2): distance to a fixed point Y* (built from an LP primal-dual optimum by
  Lemma opt-rel) non-increasing, the O(1/k) bound on the ergodic objective, the identity
  ||Zbar_k - Xbar_k|| = ||Y_k - Y_0|| / k with Z_k from Lemma 1's projection, and its 2||Y_0 - Y*||/k bound;
* exact optima: brute force over permutations (Birkhoff-von Neumann), the 1-D
  monotone (north-west-corner) plan, and an LP solver (HiGHS);
* Prop. 1 at convergence.
A mutation test plants each of several plausible mistakes in the oracle and
checks that at least one pin fails for every one of them.
"""

import numpy as np
import pytest

import oracle
import workloads


def _small(m, n, seed, marginals="dirichlet"):
    pr = workloads.make_problem("plain_256", seed=seed, m=m, n=n, marginals=marginals)
    return pr.C.astype(np.float64), pr.p, pr.q, pr.rho, pr


# ---------------------------------------------------------------- projections

def test_lemma1_projection_matches_least_squares():
    rng = np.random.default_rng(3)
    m, n = 7, 5
    p = rng.dirichlet(np.ones(m))
    q = rng.dirichlet(np.ones(n))
    X = rng.standard_normal((m, n))
    # generic projection onto {A vec(X) = b}: X - A^+ (A X - b)
    A = np.vstack([np.kron(np.eye(m), np.ones((1, n))), np.kron(np.ones((1, m)), np.eye(n))])
    b = np.concatenate([p, q])
    x = X.ravel()
    ref = (x - np.linalg.pinv(A) @ (A @ x - b)).reshape(m, n)
    got = oracle.project_marginals(X, p, q)
    assert np.abs(got - ref).max() < 1e-12
    assert np.abs(got.sum(1) - p).max() < 1e-13 and np.abs(got.sum(0) - q).max() < 1e-13


# ------------------------------------------------------- Algorithm 1 == 3-var DR

@pytest.mark.parametrize("m,n,seed", [(12, 9, 0), (5, 8, 1), (1, 4, 2), (6, 1, 3)])
def test_algorithm1_equals_three_variable_dr(m, n, seed):
    C, p, q, rho, _ = _small(m, n, seed)
    iters = 200
    run = oracle.drot_run(C, p, q, rho, iters)
    Xs, Zs, Ys = oracle.dr3_run(C, p, q, rho, iters, np.outer(p, q))
    scale = max(1.0, np.abs(Xs[-1]).max())
    assert np.abs(run["X"] - Xs[-1]).max() <= 1e-12 * scale
    # the implicit duals: Y_K = X_K + phi_K e^T + f psi_K^T (eq. alg:drot:y:update)
    Y = run["X"] + rho * run["mu"][:, None] + rho * run["nu"][None, :]
    assert np.abs(Y - Ys[-1]).max() <= 1e-12 * max(1.0, np.abs(Ys[-1]).max())


def test_step_state_matches_three_variable_dr_from_warm_start():
    C, p, q, rho, _ = _small(9, 11, 4)
    X0, mu0, nu0 = workloads.random_start(9, 11, seed=5)
    st = oracle.StepState(C, p, q, rho, X0.astype(np.float64), rho * mu0, rho * nu0)
    Y0 = st.Y.copy()
    Xs, Zs, Ys = oracle.dr3_run(C, p, q, rho, 30, Y0)
    for k in range(30):
        st.step()
        assert np.abs(st.X - Xs[k]).max() < 1e-14
        assert np.abs(st.Y - Ys[k + 1]).max() < 1e-14


# ------------------------------------------------------------- invariants

def test_a_b_alpha_recursion_invariant():
    C, p, q, rho, _ = _small(10, 7, 6)
    X0, mu0, nu0 = workloads.random_start(10, 7, seed=7)
    st = oracle.StepState(C, p, q, rho, X0.astype(np.float64), rho * mu0, rho * nu0)
    m, n = st.m, st.n
    for _ in range(50):
        st.step()
        a_def = st.X.sum(1) - p + n * st.phi + st.psi.sum()
        b_def = st.X.sum(0) - q + m * st.psi + st.phi.sum()
        assert np.abs(st.a - a_def).max() < 1e-13
        assert np.abs(st.b - b_def).max() < 1e-13
        assert abs(st.alpha - st.a.sum() / (m + n)) < 1e-13
        assert abs(st.alpha - st.b.sum() / (m + n)) < 1e-13


def test_lemma_var_repr_identities_and_nonexpansiveness():
    C, p, q, rho, _ = _small(8, 6, 8)
    st = oracle.StepState(C, p, q, rho, np.outer(p, q), np.zeros(8), np.zeros(6))
    prev_step = np.inf
    for k in range(300):
        Yk = st.Y.copy()
        stats = st.step()
        Yk1 = st.Y
        dY = Yk1 - Yk
        mu, nu = st.phi / rho, st.psi / rho
        # dual feasibility up to rho^{-1}(Y_{k+1} - Y_k)
        assert (mu[:, None] + nu[None, :] - C - dY / rho).max() <= 1e-12
        # <C, X_{k+1}> - p^T mu - q^T nu = -rho^{-1} <Y_{k+1}, Y_{k+1} - Y_k>
        lhs = (C * st.X).sum() - p @ mu - q @ nu
        rhs = -(Yk1 * dY).sum() / rho
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs))
        # the oracle's reported primal/dual agree with the definitions
        assert abs(stats[oracle.PRIMAL] - (C * st.X).sum()) < 1e-13
        assert abs(stats[oracle.DUAL] - (p @ mu + q @ nu)) < 1e-10
        step = np.sqrt((dY * dY).sum())
        assert step <= prev_step * (1 + 1e-9) + 1e-15
        prev_step = step


# ------------------------------------------------------------- Theorem 1 (Sec. 3.2)

def _theorem1_violations(C, p, q, rho, iters):
    """Run Algorithm 1 (the C oracle) from X_0 = p q^T and check Theorem 1's statements at
    every k; return the names of those that fail (an empty list when all hold).

    Y* is the fixed point Lemma opt-rel builds from an exact LP primal-dual optimum, and
    Z_{k+1} = P(2 X_{k+1} - Y_k) comes from Lemma 1's projection, independently of the
    oracle's own update of Y."""
    m, n = C.shape
    Xs, mus, nus, opt = oracle.lp_primal_dual(C, p, q)
    # the LP pair must be an exact optimum before it can define Y*
    assert (mus[:, None] + nus[None, :] - C).max() <= 1e-12
    assert abs(p @ mus + q @ nus - opt) <= 1e-12 and abs((C * Xs).sum() - opt) <= 1e-12
    Ystar = oracle.fixed_point_from_pair(Xs, mus, nus, rho)
    # T(Y*) = Y*: one step of the three-variable form from Y* returns it
    _, _, Ys = oracle.dr3_run(C, p, q, rho, 1, Ystar)
    assert np.abs(Ys[1] - Ystar).max() <= 1e-12

    st = oracle.StepState(C, p, q, rho, np.outer(p, q), np.zeros(m), np.zeros(n))
    Y0 = st.Y.copy()
    d0 = np.linalg.norm(Y0 - Ystar)
    const = np.linalg.norm(Y0) ** 2 / (2 * rho) + 2 / rho * np.linalg.norm(Xs) * d0
    bad = set()
    prev, sum_cx = d0, 0.0
    sum_X, sum_Z = np.zeros_like(C), np.zeros_like(C)
    for k in range(1, iters + 1):
        Yk = st.Y.copy()
        st.step()
        X = st.X.copy()
        sum_cx += (C * X).sum()
        sum_X += X
        sum_Z += oracle.project_marginals(2 * X - Yk, p, q)
        d = np.linalg.norm(st.Y - Ystar)
        if d > prev * (1 + 1e-12) + 1e-15:  # Fejer monotone: ||Y_k - Y*|| non-increasing
            bad.add("fejer")
        prev = d
        if sum_cx / k - opt > const / k * (1 + 1e-12):  # <C, Xbar_k> - <C, X*> <= const / k
            bad.add("objective")
        feas = np.linalg.norm(sum_Z / k - sum_X / k)
        if abs(feas - np.linalg.norm(st.Y - Y0) / k) > 1e-12 * max(1.0, feas):
            bad.add("ergodic_identity")
        if feas > 2 * d0 / k * (1 + 1e-12):
            bad.add("feasibility")
    return sorted(bad)


@pytest.mark.parametrize("m,n,seed,marginals", [(9, 7, 12, "dirichlet"), (6, 6, 3, "uniform"), (12, 5, 4, "dirichlet")])
def test_theorem1_sublinear_rate(m, n, seed, marginals):
    C, p, q, rho, _ = _small(m, n, seed, marginals)
    assert _theorem1_violations(C, p, q, rho, 300) == []


# ----------------------------------------------------------------- exact optima

@pytest.mark.parametrize("n,seed", [(3, 0), (5, 1), (6, 2), (7, 3)])
def test_permutation_brute_force(n, seed):
    C, p, q, rho, _ = _small(n, n, seed, marginals="uniform")
    out = oracle.drot_solve(C, p, q, rho, tol=1e-10, max_iter=400000)
    assert out["status"] == oracle.STATUS_CONVERGED
    assert abs(out["stats"]["primal"] - oracle.permutation_optimum(C)) < 1e-8


@pytest.mark.parametrize("m,n,seed", [(10, 7, 0), (13, 13, 1)])
def test_one_dimensional_closed_form(m, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, m)
    y = rng.uniform(0, 1, n) + 0.3
    C = workloads.sq_euclidean_cost_np(x[:, None], y[:, None]).astype(np.float64)
    p = rng.dirichlet(np.ones(m))
    q = rng.dirichlet(np.ones(n))
    q *= p.sum() / q.sum()
    P = oracle.nw_corner_1d(x, y, p, q)
    assert np.abs(P.sum(1) - p).max() < 1e-14 and np.abs(P.sum(0) - q).max() < 1e-14
    best = (C * P).sum()
    out = oracle.drot_solve(C, p, q, 2.0 / (m + n), tol=1e-10, max_iter=400000)
    assert out["status"] == oracle.STATUS_CONVERGED
    assert abs(out["stats"]["primal"] - best) < 1e-8


@pytest.mark.parametrize("m,n,seed", [(12, 9, 0), (30, 20, 1)])
def test_lp_solver_optimum(m, n, seed):
    C, p, q, rho, _ = _small(m, n, seed)
    opt, _ = oracle.lp_optimum(C, p, q)
    out = oracle.drot_solve(C, p, q, rho, tol=1e-10, max_iter=400000)
    assert out["status"] == oracle.STATUS_CONVERGED
    assert abs(out["stats"]["primal"] - opt) < 1e-8
    assert abs(out["stats"]["dual"] - opt) < 1e-8


def test_prop1_at_convergence_and_reported_stats():
    C, p, q, rho, _ = _small(16, 11, 9)
    out = oracle.drot_solve(C, p, q, rho, tol=1e-9, max_iter=400000, stop_on_dual_residual=True)
    assert out["status"] == oracle.STATUS_CONVERGED
    X, mu, nu = out["X"], out["mu"], out["nu"]
    assert X.min() >= 0.0
    st = oracle.plan_stats(C, p, q, X, mu, nu)
    assert st["res_l1"] <= 1e-9 + 1e-15 and st["gap"] <= 1e-9 + 1e-15
    assert abs(st["primal"] - out["stats"]["primal"]) < 1e-15
    assert abs(st["res_l1"] - out["stats"]["res_l1"]) < 1e-15
    assert st["dual_res"] <= 1e-7
    # basic optimal solution: at most m + n - 1 entries away from zero
    assert int((X > 1e-12).sum()) <= 16 + 11 - 1


def test_warm_start_continues_the_same_iteration():
    # Y_0 = X_0 + rho mu_0 e^T + rho f nu_0^T with a_0 = Y_0 e - p reproduces the
    # state of an interrupted run exactly, so the resumed run retraces it.
    C, p, q, rho, _ = _small(14, 10, 10)
    full = oracle.drot_run(C, p, q, rho, 100)
    half = oracle.drot_run(C, p, q, rho, 50)
    rest = oracle.drot_run(C, p, q, rho, 50, X0=half["X"], mu0=half["mu"], nu0=half["nu"])
    assert np.abs(rest["history"] - full["history"][50:]).max() < 1e-12
    assert np.abs(rest["X"] - full["X"]).max() < 1e-14


def test_warm_start_from_converged_state_stops_immediately():
    C, p, q, rho, _ = _small(14, 10, 10)
    out = oracle.drot_solve(C, p, q, rho, tol=1e-9, max_iter=400000, stop_on_dual_residual=True)
    assert out["status"] == oracle.STATUS_CONVERGED
    again = oracle.drot_solve(C, p, q, rho, tol=1e-8, max_iter=10, X0=out["X"], mu0=out["mu"], nu0=out["nu"],
                              stop_on_dual_residual=True)
    assert again["status"] == oracle.STATUS_CONVERGED and again["iters"] <= 2


def test_max_iter_and_zero_iterations():
    C, p, q, rho, _ = _small(5, 4, 11)
    out = oracle.drot_solve(C, p, q, rho, tol=1e-12, max_iter=3)
    assert out["status"] == oracle.STATUS_MAX_ITER and out["iters"] == 3
    out0 = oracle.drot_solve(C, p, q, rho, tol=1e-12, max_iter=0)
    assert out0["iters"] == 0 and np.allclose(out0["X"], np.outer(p, q))


# ------------------------------------------------------------------ mutations

def _pin_battery():
    """Return the list of pin names that fail on the current oracle build."""
    failed = []
    C, p, q, rho, _ = _small(9, 7, 12)
    run = oracle.drot_run(C, p, q, rho, 60)
    Xs, _, _ = oracle.dr3_run(C, p, q, rho, 60, np.outer(p, q))
    if not np.abs(run["X"] - Xs[-1]).max() < 1e-12:
        failed.append("dr3")
    st = oracle.StepState(C, p, q, rho, np.outer(p, q), np.zeros(9), np.zeros(7))
    for _ in range(20):
        Yk = st.Y.copy()
        stats = st.step()
        mu, nu = st.phi / rho, st.psi / rho
        lhs = stats[oracle.PRIMAL] - stats[oracle.DUAL]
        rhs = -(st.Y * (st.Y - Yk)).sum() / rho
        if abs(lhs - rhs) > 1e-9 * max(1, abs(rhs)):
            failed.append("var_repr")
            break
    if _theorem1_violations(C, p, q, rho, 200):
        failed.append("theorem1")
    opt, _ = oracle.lp_optimum(C, p, q)
    out = oracle.drot_solve(C, p, q, rho, tol=1e-9, max_iter=20000)
    if out["status"] != oracle.STATUS_CONVERGED or abs(out["stats"]["primal"] - opt) > 1e-7:
        failed.append("lp")
    return failed


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5, 6, 7])
def test_pins_catch_planted_mistakes(mutation):
    try:
        oracle.set_mutation(mutation)
        failed = _pin_battery()
    finally:
        oracle.set_mutation(0)
    assert failed, f"mutation {mutation} slipped past every pin"


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 6, 7])
def test_theorem1_pins_alone_catch_every_mistake_in_the_iteration(mutation):
    # mutation 5 changes only the reported dual objective, not the iterates
    C, p, q, rho, _ = _small(9, 7, 12)
    try:
        oracle.set_mutation(mutation)
        failed = _theorem1_violations(C, p, q, rho, 300)
    finally:
        oracle.set_mutation(0)
    assert failed, f"mutation {mutation} satisfies every statement of Theorem 1"


def test_unmutated_oracle_passes_battery():
    oracle.set_mutation(0)
    assert _pin_battery() == []


# ------------------------------------------------------------------ golden file

def test_golden_lp_optima_reached_by_oracle():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "lp_optima.json")
    cases = json.load(open(path))["cases"]
    for case in cases:
        pr = workloads.make_problem(case["config"], seed=case["seed"], m=case["m"], n=case["n"])
        # the Sec. 4 Gaussian case (48 x 48) needs about 1.6 million iterations at rho0 = 2
        out = oracle.drot_solve(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, tol=1e-10, max_iter=2_000_000,
                                stop_on_dual_residual=False)
        assert out["status"] == oracle.STATUS_CONVERGED, case
        assert abs(out["stats"]["primal"] - case["lp_optimum"]) < 1e-7, case
        if "permutation_optimum" in case:
            assert abs(case["permutation_optimum"] - case["lp_optimum"]) < 1e-12
