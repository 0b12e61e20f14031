"""Double-precision solve (drot_solve_f64) vs the FP64 oracle, and the per-iteration trace.

Both sides run Algorithm 1 (Sec. 3.1) in FP64 on the same FP64 inputs, so they differ
only in rounding order: the GPU forms d = phi + psi - rho c with one fused multiply-add
and adds rows, columns and the scalar totals in another order.  Each entry update then
differs by a few units of eps64 = 2^-53 of the largest term S = max(|x|, |phi|, |psi|,
rho |c|); Douglas-Rachford is nonexpansive, so after k iterations the plans agree to
O(k eps64 S) and the duals to O(k eps64 S / rho) — about nine orders of magnitude
tighter than the FP32 path's bounds.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2110_11738_b300 import drot

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


def _cost64(pr):
    d = pr.x[:, None, :] - pr.y[None, :, :]
    return (d * d).sum(-1) / pr.cost_scale


def _dev64(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _inputs64(pr, C64, X0=None, mu0=None, nu0=None):
    C = drot.padded_matrix(C64, device="cuda", dtype=torch.float64)
    X = torch.zeros((pr.m, C.stride(0)), dtype=torch.float64, device="cuda")[:, : pr.n]
    if X0 is not None:
        X.copy_(_dev64(X0))
    mu = _dev64(mu0 if mu0 is not None else np.zeros(pr.m))
    nu = _dev64(nu0 if nu0 is not None else np.zeros(pr.n))
    return C, _dev64(pr.p), _dev64(pr.q), X, mu, nu


@pytest.fixture(scope="module")
def solver():
    s = drot.Solver(device=0)
    yield s
    s.close()


# ragged shapes: a single column, a single row, odd n (the pitch is padded to even),
# widths just past one and several 256-column tiles
SHAPES = [(300, 250), (129, 513), (64, 1), (1, 77), (517, 1031), (40, 256), (33, 257)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_f64_step_parity(solver, m, n):
    pr = workloads.make_problem("plain_256", seed=m * 7 + n, m=m, n=n)
    C64 = _cost64(pr)
    X0, mu0, nu0 = workloads.random_start(m, n, seed=m + n)
    k = 40
    C, p, q, X, mu, nu = _inputs64(pr, C64, X0, mu0, nu0)
    out = solver.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=k, X=X, mu=mu, nu=nu, warm=True)
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == k
    ref = oracle.drot_run(C64, pr.p, pr.q, pr.rho, k, X0=X0.astype(np.float64), mu0=mu0, nu0=nu0)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0), np.abs(ref["X"]).max())
    tol_x = 64 * EPS64 * S * k
    assert np.abs(X.cpu().numpy() - ref["X"]).max() <= tol_x
    tol_dual = 64 * EPS64 * S * k / pr.rho
    assert np.abs(mu.cpu().numpy() - ref["mu"]).max() <= tol_dual
    assert np.abs(nu.cpu().numpy() - ref["nu"]).max() <= tol_dual
    st = ref["stats"]
    for key in ("primal_obj", "res_l1"):
        refv = st["primal" if key == "primal_obj" else "res_l1"]
        assert abs(out[key] - refv) <= 1e-10 * max(1.0, abs(refv)), key
    assert out["nnz"] == int((ref["X"] > 0).sum())


def test_f64_cold_solve_matches_oracle_at_tight_tolerance(solver):
    """FP64 iterates can reach a gap far below the FP32 path's floor: 1e-9 here."""
    pr = workloads.make_problem("plain_256", seed=11, m=96, n=80)
    C64 = _cost64(pr)
    C, p, q, X, mu, nu = _inputs64(pr, C64)
    out = solver.solve(C, p, q, rho=pr.rho, tol=1e-9, max_iter=2_000_000, X=X, mu=mu, nu=nu)
    ref = oracle.drot_solve(C64, pr.p, pr.q, pr.rho, 1e-9, 2_000_000)
    assert out["status"] == drot.DROT_OK and ref["status"] == 0
    assert abs(out["iters"] - ref["iters"]) <= 2
    assert out["gap"] <= 1e-9 and out["res_l1"] <= 1e-9
    assert abs(out["primal_obj"] - ref["stats"]["primal"]) <= 1e-11
    assert abs(out["dual_obj"] - ref["stats"]["dual"]) <= 1e-11
    # the optimum of the LP, to the accuracy the certificate gives
    lp, _ = oracle.lp_optimum(C64, pr.p, pr.q)
    assert abs(out["primal_obj"] - lp) <= 1e-8


def test_f64_deterministic_mode_is_bitwise_reproducible():
    pr = workloads.make_problem("plain_256", seed=3, m=200, n=300)
    C64 = _cost64(pr)
    outs = []
    with drot.Solver(device=0, deterministic=True) as s:
        for _ in range(2):
            C, p, q, X, mu, nu = _inputs64(pr, C64)
            s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=60, X=X, mu=mu, nu=nu)
            outs.append((X.cpu().numpy().copy(), mu.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_f64_host_buffers_match_device_buffers():
    pr = workloads.make_problem("plain_256", seed=4, m=70, n=90)
    C64 = _cost64(pr)
    with drot.Solver(device=0, deterministic=True) as s:
        C, p, q, X, mu, nu = _inputs64(pr, C64)
        s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=30, X=X, mu=mu, nu=nu)
        ld = C.stride(0)
        Ch = np.zeros((pr.m, ld))
        Ch[:, : pr.n] = C64
        Xh = np.zeros((pr.m, ld))
        muh, nuh = np.zeros(pr.m), np.zeros(pr.n)
        drot.drot_solve(s.handle, Ch[:, : pr.n], pr.p, pr.q, rho=pr.rho, tol=-1.0, max_iter=30, X=Xh[:, : pr.n],
                        mu=muh, nu=nuh)
    assert np.array_equal(Xh[:, : pr.n], X.cpu().numpy())
    assert np.array_equal(muh, mu.cpu().numpy())


def test_f64_rejects_what_it_does_not_support(solver):
    pr = workloads.make_problem("plain_256", seed=5, m=20, n=30)
    C64 = _cost64(pr)
    C, p, q, X, mu, nu = _inputs64(pr, C64)
    # odd pitch: rows would not start on 16-byte boundaries
    Codd = torch.zeros((pr.m, 31), dtype=torch.float64, device="cuda")[:, :30]
    Xodd = torch.zeros((pr.m, 31), dtype=torch.float64, device="cuda")[:, :30]
    out = drot.drot_solve(solver.handle, Codd, p, q, rho=pr.rho, tol=1e-6, max_iter=10, X=Xodd, mu=mu, nu=nu,
                          check=False)
    assert out["status"] == drot.DROT_ERR_INVALID_ARG
    for cfg in (dict(persistent=True), dict(c_skip=True), dict(cluster=2)):
        with drot.Solver(device=0, **cfg) as s:
            out = s.solve(C, p, q, rho=pr.rho, tol=1e-6, max_iter=10, X=X, mu=mu, nu=nu, check=False)
            assert out["status"] == drot.DROT_ERR_INVALID_ARG, cfg
    with pytest.raises(ValueError):
        drot.drot_solve(solver.handle, C, p, q, X=torch.zeros((pr.m, C.stride(0)), device="cuda")[:, :30], mu=mu,
                        nu=nu)


@pytest.mark.parametrize("f64", [False, True])
def test_trace_follows_the_oracle_history(f64):
    """The trace holds <C, X_k> and the l1 residual of every iteration, as the oracle's history does."""
    pr = workloads.make_problem("plain_256", seed=8, m=150, n=120)
    k = 200
    trace = torch.full((2 * 300,), -1.0, dtype=torch.float64, device="cuda")
    if f64:
        C64 = _cost64(pr)
        C, p, q, X, mu, nu = _inputs64(pr, C64)
    else:
        C64 = pr.C.astype(np.float64)
        C = drot.padded_matrix(pr.C, device="cuda")
        X = torch.zeros((pr.m, C.stride(0)), dtype=torch.float32, device="cuda")[:, : pr.n]
        p, q = _dev64(pr.p), _dev64(pr.q)
        mu, nu = torch.zeros(pr.m, dtype=torch.float64, device="cuda"), torch.zeros(pr.n, dtype=torch.float64,
                                                                                      device="cuda")
    with drot.Solver(device=0, trace=trace) as s:
        out = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=k, X=X, mu=mu, nu=nu)
    assert out["iters"] == k
    tr = trace.cpu().numpy().reshape(-1, 2)
    assert np.all(tr[k:] == -1.0)  # nothing past the last iteration
    hist = oracle.drot_run(C64, pr.p, pr.q, pr.rho, k)["history"]
    ref = hist[:, [oracle.PRIMAL, oracle.RES_L1]]
    tol = 1e-12 if f64 else 1e-5
    assert np.abs(tr[:k] - ref).max() <= tol * max(1.0, np.abs(ref).max())
    assert tr[k - 1, 0] == pytest.approx(out["primal_obj"], rel=1e-15, abs=0)
