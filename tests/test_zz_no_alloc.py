"""drot_solve_static: the handle-free solve that allocates no device memory.

Who needs it: code that may not call cudaMalloc while it solves - a plugin inside a host
application that reserved all GPU memory up front, a component that must stay inside another
framework's memory pool, or a latency-critical loop that must never enter the allocator.  Such
callers pass only their inputs and outputs; the workspace is a fixed 16 MiB array inside the
library.

The first test calls the entry point twice in a row through the C ABI (a cold solve to tolerance, then
a few warm-started iterations on another, ragged shape) and compares each result with drot_solve
on the same inputs, within the tolerances the other parity tests use.  It also checks that a
problem whose workspace does not fit is refused before anything runs, and that a call after the
first leaves the device's free memory unchanged.  This file is collected
last so that a failing run stopped at the first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

import workloads
from paper_2110_11738_b300 import drot

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _inputs(pr, X0=None, mu0=None, nu0=None):
    ld = workloads.pad_ld(pr.n)
    C = torch.zeros((pr.m, ld), dtype=torch.float32, device="cuda")
    C[:, : pr.n] = torch.as_tensor(pr.C)
    X = torch.zeros((pr.m, ld), dtype=torch.float32, device="cuda")
    if X0 is not None:
        X[:, : pr.n] = torch.as_tensor(X0)
    mu = torch.as_tensor(np.zeros(pr.m) if mu0 is None else mu0, dtype=torch.float64, device="cuda").clone()
    nu = torch.as_tensor(np.zeros(pr.n) if nu0 is None else nu0, dtype=torch.float64, device="cuda").clone()
    p = torch.as_tensor(pr.p, device="cuda")
    q = torch.as_tensor(pr.q, device="cuda")
    return C[:, : pr.n], p, q, X[:, : pr.n], mu, nu


def test_static_solve_matches_drot_solve_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    torch.cuda.synchronize()

    # call 1: cold start, solve to the 1e-6 stopping test
    pr = workloads.make_problem("plain_256", seed=0)
    C, p, q, X, mu, nu = _inputs(pr)
    got = drot.drot_solve_static(C, p, q, rho=pr.rho, tol=1e-6, max_iter=500_000, X=X, mu=mu, nu=nu)
    assert got["status"] == drot.DROT_OK, got
    C2, p2, q2, X2, mu2, nu2 = _inputs(pr)
    with drot.Solver(device=0, step_variant=1) as s:
        ref = s.solve(C2, p2, q2, rho=pr.rho, tol=1e-6, max_iter=500_000, X=X2, mu=mu2, nu=nu2)
    assert ref["status"] == drot.DROT_OK
    obj = ref["primal_obj"]
    assert abs(got["primal_obj"] - obj) <= 1e-5 * abs(obj)
    assert abs(got["dual_obj"] - ref["dual_obj"]) <= 1e-5 * abs(obj)
    assert got["res_l1"] <= 1e-6 and got["gap"] <= 1e-6
    assert abs(got["iters"] - ref["iters"]) <= 0.02 * ref["iters"] + 2

    # call 2: warm start from a random state on a ragged shape, exactly 3 iterations
    pr = workloads.make_problem("plain_8192x6144", seed=7, m=130, n=257)
    X0, mu0, nu0 = workloads.random_start(pr.m, pr.n, seed=3)
    C, p, q, X, mu, nu = _inputs(pr, X0, mu0, nu0)
    got = drot.drot_solve_static(C, p, q, rho=pr.rho, tol=-1.0, max_iter=3, X=X, mu=mu, nu=nu, warm=True)
    assert got["status"] == drot.DROT_NOT_CONVERGED and got["iters"] == 3
    C2, p2, q2, X2, mu2, nu2 = _inputs(pr, X0, mu0, nu0)
    with drot.Solver(device=0, step_variant=1) as s:
        ref = s.solve(C2, p2, q2, rho=pr.rho, tol=-1.0, max_iter=3, X=X2, mu=mu2, nu=nu2, warm=True)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0))
    assert float((X - X2).abs().max()) <= 8 * EPS32 * S * 3 * 4
    assert float((mu - mu2).abs().max()) <= 64 * EPS32 * S / pr.rho * 3 + 1e-12
    assert float((nu - nu2).abs().max()) <= 64 * EPS32 * S / pr.rho * 3 + 1e-12
    assert abs(got["primal_obj"] - ref["primal_obj"]) <= 1e-5 * abs(ref["primal_obj"]) + 1e-9


def test_static_solve_refuses_a_problem_larger_than_its_workspace():
    m, n = 1_000_000, 4  # needs about 24 MB of workspace; the fixed array holds 16 MiB
    C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    X = torch.zeros_like(C)
    p = torch.full((m,), 1.0 / m, dtype=torch.float64, device="cuda")
    q = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    mu = torch.zeros(m, dtype=torch.float64, device="cuda")
    nu = torch.zeros(n, dtype=torch.float64, device="cuda")
    X.fill_(3.0)
    got = drot.drot_solve_static(C, p, q, tol=1e-6, max_iter=10, X=X, mu=mu, nu=nu)
    assert got["status"] == drot.DROT_ERR_TOO_LARGE
    assert float(X.min()) == 3.0  # nothing ran


def test_static_solve_allocates_no_device_memory():
    """The property the entry point exists for: after a first call (which places the library's
    device code and its fixed array), further calls leave the device's free memory and torch's
    allocator untouched."""
    torch.cuda.set_device(0)
    pr = workloads.make_problem("plain_8192x6144", seed=11, m=300, n=517)
    C, p, q, X, mu, nu = _inputs(pr)
    first = drot.drot_solve_static(C, p, q, rho=pr.rho, tol=1e-6, max_iter=2000, X=X, mu=mu, nu=nu)
    assert first["status"] in (drot.DROT_OK, drot.DROT_NOT_CONVERGED), first
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    allocated_before = torch.cuda.memory_allocated()
    reserved_before = torch.cuda.memory_reserved()
    second = drot.drot_solve_static(C, p, q, rho=pr.rho, tol=1e-6, max_iter=2000, X=X, mu=mu, nu=nu)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert second["status"] == first["status"]
    assert abs(second["primal_obj"] - first["primal_obj"]) <= 1e-5 * abs(first["primal_obj"])
    assert free_after == free_before
    assert torch.cuda.memory_allocated() == allocated_before
    assert torch.cuda.memory_reserved() == reserved_before
