"""Out-of-bounds detection without compute-sanitizer: red zones and poisoned padding.

Every caller buffer (C, X, p, q, mu, nu) is carved out of a larger allocation with GUARD words
on each side, and the pitch padding of C and X (columns n .. ld-1 of every row) belongs to the
caller too.  All of these words hold a NaN with a recognisable payload.  A kernel that reads one
of them into its arithmetic pulls a NaN into the plan or its totals (the solve then reports
DROT_ERR_NONFINITE or leaves the oracle); a kernel that writes one changes its bit pattern.  So
after k iterations from a seeded start every path must leave each guard and padding word bit
for bit as it was and still match the FP64 oracle (Algorithm 1, Sec. 3.1) within the step-parity
tolerances.  Reads that land in a guard and are then discarded stay legal and undetected; they
stay inside the allocation, so they cannot fault.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2110_11738_b300 import drot

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53
GUARD = 64  # words on each side: 256 B (FP32) or 512 B (FP64), so the interior keeps its alignment
POISON = {torch.float32: (torch.int32, 0x7FC0DEAD), torch.float64: (torch.int64, 0x7FF8DEADBEEFDEAD)}


class Guarded:
    """`values` (a vector, or a matrix stored with pitch `ld`) inside a larger device allocation
    whose every other word holds a NaN with a fixed payload."""

    def __init__(self, values, ld=None, dtype=torch.float32):
        a = np.asarray(values)
        rows, cols = (1, a.shape[0]) if a.ndim == 1 else a.shape
        ld = cols if ld is None else int(ld)
        body = rows * ld
        self.itype, self.pattern = POISON[dtype]
        self.flat = torch.empty(2 * GUARD + body, dtype=dtype, device="cuda")
        self.flat.view(self.itype).fill_(self.pattern)
        inner = self.flat[GUARD:GUARD + body]
        self.t = inner[:cols] if a.ndim == 1 else inner.view(rows, ld)[:, :cols]
        self.t.copy_(torch.as_tensor(a, dtype=dtype))
        self.outside = torch.ones(self.flat.numel(), dtype=torch.bool, device="cuda")
        inside = self.outside[GUARD:GUARD + body]
        if a.ndim == 1:
            inside[:cols] = False
        else:
            inside.view(rows, ld)[:, :cols] = False

    def intact(self) -> bool:
        bits = self.flat.view(self.itype)
        return bool((bits[self.outside] == self.pattern).all())


def _guarded_problem(pr, X0, mu0, nu0, dtype=torch.float32, C=None):
    vec = 16 // (4 if dtype == torch.float32 else 8)
    ld = (pr.n + vec - 1) // vec * vec
    return dict(C=Guarded(pr.C if C is None else C, ld, dtype), X=Guarded(X0, ld, dtype),
                p=Guarded(pr.p, dtype=torch.float64), q=Guarded(pr.q, dtype=torch.float64),
                mu=Guarded(mu0, dtype=torch.float64), nu=Guarded(nu0, dtype=torch.float64))


def _check_guards(bufs):
    torch.cuda.synchronize()
    for name, b in bufs.items():
        assert b.intact(), f"a word outside {name} changed"


def _check_against_oracle(pr, bufs, out, X0, mu0, nu0, k, stats_k=None, C64=None, f64=False):
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == k, out
    C_ref = pr.C.astype(np.float64) if C64 is None else C64
    ref = oracle.drot_run(C_ref, pr.p, pr.q, pr.rho, k, X0=np.asarray(X0, np.float64), mu0=mu0, nu0=nu0)
    Xg = bufs["X"].t.cpu().numpy().astype(np.float64)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0), np.abs(ref["X"]).max())
    if f64:
        tol_x, tol_d = 64 * EPS64 * S * k, 64 * EPS64 * S * k / pr.rho
    else:
        tol_x, tol_d = 8 * EPS32 * S * k * 4, 64 * EPS32 * S / pr.rho * k + 1e-12
    assert np.isfinite(Xg).all() and Xg.min() >= 0.0
    assert np.abs(Xg - ref["X"]).max() <= tol_x
    assert np.abs(bufs["mu"].t.cpu().numpy() - ref["mu"]).max() <= tol_d
    assert np.abs(bufs["nu"].t.cpu().numpy() - ref["nu"]).max() <= tol_d
    h = ref["history"][(stats_k or k) - 1]
    assert abs(out["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9
    # an FP32 plan resolves its row and column totals only to EPS32 of the mass they carry; with
    # m = n = 1 one entry carries all of it, and the residual the GPU reports at the fixed point
    # is 2^-23 where the FP64 oracle's is 0
    mass = float(pr.p.sum() + pr.q.sum())
    assert abs(out["res_l1"] - h[oracle.RES_L1]) <= 1e-5 * abs(h[oracle.RES_L1]) + 1e-7 + 2 * EPS32 * mass


SHAPES = [(1, 1), (3, 7), (31, 33), (130, 257), (257, 1031)]
CONFIGS = {
    "automatic": {},  # cluster-resident where the problem fits
    "streaming": {"cluster": 1},
    "grid_resident": {"cluster": 3},
    "registers_k1": {"step_variant": 1, "tile_k": 1},
    "tma_k2": {"step_variant": 2, "tile_k": 2},
    "async_k4": {"step_variant": 3, "tile_k": 4},
    "persistent": {"persistent": True},
    "c_skip": {"c_skip": True},
    "fixed_order": {"deterministic": True, "step_variant": 1, "tile_k": 4, "grid_ctas": 37},
}


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("name", list(CONFIGS))
def test_single_solve_stays_inside_its_buffers(name, m, n):
    k = 4
    pr = workloads.make_problem("plain_8192x6144", seed=m * 31 + n, m=m, n=n)
    X0, mu0, nu0 = workloads.random_start(m, n, seed=m + 7 * n)
    bufs = _guarded_problem(pr, X0, mu0, nu0)
    with drot.Solver(device=0, **CONFIGS[name]) as s:
        out = s.solve(bufs["C"].t, bufs["p"].t, bufs["q"].t, rho=pr.rho, tol=-1.0, max_iter=k, X=bufs["X"].t,
                      mu=bufs["mu"].t, nu=bufs["nu"].t, warm=True, check=False)
    _check_guards(bufs)
    # with C skipped every other pass the stopping quantities after pass 4 are those of pass 3
    _check_against_oracle(pr, bufs, out, X0, mu0, nu0, k, stats_k=k - 1 if name == "c_skip" else None)


@pytest.mark.parametrize("m,n", [(1, 1), (64, 1), (33, 257), (300, 250)])
def test_f64_solve_stays_inside_its_buffers(m, n):
    k = 6
    pr = workloads.make_problem("plain_256", seed=m * 5 + n, m=m, n=n)
    d = pr.x[:, None, :] - pr.y[None, :, :]
    C64 = (d * d).sum(-1) / pr.cost_scale
    X0, mu0, nu0 = workloads.random_start(m, n, seed=m + n + 1)
    X0 = X0.astype(np.float64)
    bufs = _guarded_problem(pr, X0, mu0, nu0, dtype=torch.float64, C=C64)
    with drot.Solver(device=0) as s:
        out = s.solve(bufs["C"].t, bufs["p"].t, bufs["q"].t, rho=pr.rho, tol=-1.0, max_iter=k, X=bufs["X"].t,
                      mu=bufs["mu"].t, nu=bufs["nu"].t, warm=True, check=False)
    _check_guards(bufs)
    _check_against_oracle(pr, bufs, out, X0, mu0, nu0, k, C64=C64, f64=True)


@pytest.mark.parametrize("narrow", [-1, 1])  # narrow tiles in the wide-tile kernel / in their own packed kernel
def test_batched_solve_stays_inside_every_problems_buffers(narrow):
    k = 4
    cases = []
    for b, (m, n) in enumerate([(3, 7), (130, 257), (1, 1), (257, 1031), (64, 2048), (301, 700)]):
        pr = workloads.make_problem("plain_8192x6144", seed=900 + b, m=m, n=n)
        X0, mu0, nu0 = workloads.random_start(m, n, seed=950 + b)
        cases.append((pr, X0, mu0, nu0, _guarded_problem(pr, X0, mu0, nu0)))
    probs = [dict(C=g["C"].t, X=g["X"].t, p=g["p"].t, q=g["q"].t, mu=g["mu"].t, nu=g["nu"].t, rho=pr.rho)
             for pr, _, _, _, g in cases]
    with drot.Solver(device=0, batch_narrow=narrow) as s:
        res = s.solve_batched(probs, tol=-1.0, max_iter=k, warm=True, check=False)
    for (pr, X0, mu0, nu0, g), r in zip(cases, res):
        _check_guards(g)
        _check_against_oracle(pr, g, r, X0, mu0, nu0, k)


def test_static_solve_stays_inside_its_buffers():
    k = 4
    pr = workloads.make_problem("plain_8192x6144", seed=77, m=130, n=257)
    X0, mu0, nu0 = workloads.random_start(pr.m, pr.n, seed=78)
    bufs = _guarded_problem(pr, X0, mu0, nu0)
    out = drot.drot_solve_static(bufs["C"].t, bufs["p"].t, bufs["q"].t, rho=pr.rho, tol=-1.0, max_iter=k,
                                 X=bufs["X"].t, mu=bufs["mu"].t, nu=bufs["nu"].t, warm=True)
    _check_guards(bufs)
    _check_against_oracle(pr, bufs, out, X0, mu0, nu0, k)
