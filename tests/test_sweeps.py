"""The paper-shaped sweeps (Sec. 4): their host-side pieces on the CPU, and small runs of
each sweep on the GPU checked against the FP64 oracle under the same termination rule."""

import numpy as np
import pytest

import oracle
import workloads
from paper_2110_11738_b300 import sweeps


def test_success_profile_and_first_below():
    err = [1e-3, 1e-5, float("nan"), 2e-2, float("inf")]
    assert sweeps.success_profile(err, [1e-6, 1e-4, 1e-2, 1.0]) == [0.0, 0.2, 0.4, 0.6]
    assert sweeps.first_below([0.5, 0.2, 0.09, 0.2, 0.01], 0.1) == 3
    assert sweeps.first_below([0.5, 0.2], 0.1) is None


@pytest.mark.parametrize("n", [3, 5, 7])
def test_assignment_optimum_is_the_permutation_brute_force(n):
    rng = np.random.default_rng(n)
    C = rng.uniform(0, 1, size=(n, n))
    assert sweeps.assignment_optimum(C) == pytest.approx(oracle.permutation_optimum(C), rel=1e-12)


def test_assignment_optimum_is_the_lp_optimum_for_uniform_marginals():
    """Birkhoff-von Neumann: with p = q = 1/n the LP optimum sits on a scaled permutation."""
    pr = workloads.make_problem("paper_gauss", seed=2, m=14, n=14)
    C = sweeps.cost64(pr)
    lp, _ = oracle.lp_optimum(C, pr.p, pr.q)
    assert sweeps.assignment_optimum(C) == pytest.approx(lp, rel=1e-9)


def test_paper_generator_shape_and_normalisation():
    pr = workloads.make_problem("paper_gauss", seed=3, m=40, n=40, sigma_t=10.0)
    C = sweeps.cost64(pr)
    assert C.shape == (40, 40) and C.max() == pytest.approx(1.0) and C.min() >= 0.0
    assert np.allclose(pr.p, 1 / 40) and np.allclose(pr.q, 1 / 40)
    assert np.allclose(C, pr.C, rtol=1e-6, atol=1e-7)  # the FP32 cost is this one rounded


@pytest.mark.gpu
@pytest.mark.parametrize("f64", [False, True])
def test_e1_matches_the_oracle_under_the_same_termination(f64):
    m, problems = 64, 4
    res = sweeps.robustness(problems=problems, m=m, f64=f64)
    assert len(res["rel_err"]) == problems and res["profile"] == sweeps.success_profile(res["rel_err"])
    for k in range(problems):
        pr = workloads.make_problem("paper_gauss", seed=k, m=m, n=m, sigma_t=5.0)
        C = sweeps.cost64(pr) if f64 else pr.C.astype(np.float64)
        ref = oracle.drot_solve(C, pr.p, pr.q, 2.0 / (2 * m), 1e-4, 1000, stop_rule=2)
        fstar = sweeps.assignment_optimum(sweeps.cost64(pr))
        rel_ref = abs(ref["stats"]["primal"] - fstar) / fstar
        assert abs(res["iters"][k] - ref["iters"]) <= (0 if f64 else 3)
        assert abs(res["rel_err"][k] - rel_ref) <= (1e-10 if f64 else 1e-4)


@pytest.mark.gpu
def test_e3_and_runtime_small():
    res = sweeps.time_to_accuracy(sizes=(64, 128), eps_list=(1e-1, 1e-2), runs=1, k_start=200)
    for row in res["rows"]:
        k1, k2 = row["iters"]["0.1"], row["iters"]["0.01"]
        assert k1 is not None and k2 is not None and k1 <= k2
        assert 0 < row["seconds"]["0.1"] <= row["seconds"]["0.01"] * 1.5
    rt = sweeps.runtime_per_iteration(sizes=(128, 1024), runs=3)
    for row in rt["rows"]:
        assert 0 < row["lo_us"] <= row["median_us"] <= row["hi_us"]
