"""Device-side failure detection without a GPU fault: every wait in the persistent solve is
bounded, so a grid barrier that cannot complete in time sets a fault flag, every CTA leaves,
and the host reports DROT_ERR_TIMEOUT; the context stays usable.  The test makes the waits
run out by allowing a single poll (no kernel is broken, nothing traps)."""

import numpy as np
import pytest
import torch

import workloads
from paper_2110_11738_b300 import drot

pytestmark = pytest.mark.gpu


def _inputs(pr):
    C = drot.padded_matrix(pr.C, device="cuda")
    X = torch.zeros((pr.m, C.stride(0)), dtype=torch.float32, device="cuda")[:, : pr.n]
    p = torch.as_tensor(pr.p, device="cuda")
    q = torch.as_tensor(pr.q, device="cuda")
    mu = torch.zeros(pr.m, dtype=torch.float64, device="cuda")
    nu = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    return C, p, q, X, mu, nu


def test_persistent_barrier_timeout_is_reported_and_the_context_survives():
    pr = workloads.make_problem("plain_8192x6144", seed=2, m=2048, n=1536)
    C, p, q, X, mu, nu = _inputs(pr)
    with drot.Solver(device=0, persistent=True, wait_limit=1) as s:
        out = s.solve(C, p, q, rho=pr.rho, tol=1e-6, max_iter=1000, X=X, mu=mu, nu=nu, check=False)
    assert out["status"] == drot.DROT_ERR_TIMEOUT, out["status_name"]
    torch.cuda.synchronize()
    # the same context, a default wait limit: the persistent solve runs normally
    C, p, q, X, mu, nu = _inputs(pr)
    with drot.Solver(device=0, persistent=True) as s:
        out = s.solve(C, p, q, rho=pr.rho, tol=-1.0, max_iter=60, X=X, mu=mu, nu=nu)
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == 60
    with drot.Solver(device=0) as s:
        C2, p2, q2, X2, mu2, nu2 = _inputs(pr)
        ref = s.solve(C2, p2, q2, rho=pr.rho, tol=-1.0, max_iter=60, X=X2, mu=mu2, nu=nu2)
    assert abs(out["primal_obj"] - ref["primal_obj"]) <= 1e-5 * abs(ref["primal_obj"])
    assert np.isfinite(X.cpu().numpy()).all()
