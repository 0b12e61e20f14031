"""Learned warm start: the network's kernels against the FP64 reference, the seed's dual
feasibility, and what a trained network's seed buys over cold-start DROT under the full
primal-dual stopping test and under the duality gap alone.

Tolerances: the GPU multiplies BF16 operands (8 significant bits) and accumulates in FP32, and
stores activations in BF16, so each layer carries a relative error of a few 2^-8; forward
outputs are compared at 5e-2 of their scale and gradients by direction (cosine) and norm.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import mlp as ref_mlp
from paper_2110_11738_b300 import drot, warmstart

pytestmark = pytest.mark.gpu


def _bf16_features(rows, seed):
    rng = np.random.default_rng(seed)
    F = rng.uniform(-1, 1, size=(rows, 64)).astype(np.float32)
    Fb = torch.as_tensor(F, device="cuda").to(torch.bfloat16)
    return Fb, Fb.float().cpu().numpy().astype(np.float64)


# 192 rows: one full and one half 128-row block per product; 65600 rows: 513 blocks (the
# tensor cores of every SM busy), the last one ragged
@pytest.mark.parametrize("rows", [192, 65600])
def test_forward_matches_reference(rows):
    params = workloads.mlp_init_params(3)
    net = drot.Mlp(0, params)
    Fb, F64 = _bf16_features(rows, 1)
    out = torch.zeros(rows, dtype=torch.float32, device="cuda")
    net.forward(Fb, out)
    ref, _ = ref_mlp.forward(params.astype(np.float64), F64)
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 5e-2 * np.abs(ref).max()
    assert np.corrcoef(got, ref)[0, 1] > 0.999
    net.close()


# 256 rows: every weight-gradient product in one K range; 1088 rows: five K ranges per product
# (the last one partly beyond the rows, read as zeros) added with atomics, and nine 128-row
# blocks in the forward products, the last one ragged
@pytest.mark.parametrize("rows", [256, 1088])
def test_gradients_match_reference(rows):
    params = workloads.mlp_init_params(4)
    params[-257:-1] *= 8.0  # larger output weights: gradients well above rounding noise
    net = drot.Mlp(0, params)
    Fb, F64 = _bf16_features(rows, 2)
    rng = np.random.default_rng(3)
    y = rng.standard_normal(rows).astype(np.float32)
    w = rng.uniform(0.1, 1.0, rows).astype(np.float32)
    seg = rng.integers(0, 4, rows).astype(np.int32)
    seg[-10:] = -1  # padding rows
    loss, grad = net.train_step(Fb, torch.as_tensor(y, device="cuda"), torch.as_tensor(w, device="cuda"),
                                torch.as_tensor(seg, device="cuda"), 4, 0.0, update=False, want_grad=True)
    keep = seg >= 0
    L, g = ref_mlp.loss_and_grad(params.astype(np.float64), F64[keep], y[keep].astype(np.float64),
                                 w[keep].astype(np.float64), seg[keep], 4)
    assert abs(loss - L) <= 5e-2 * L
    off = 0
    for name, shape in ref_mlp.SHAPES:
        k = int(np.prod(shape))
        a, b = grad[off:off + k].astype(np.float64), g[off:off + k]
        off += k
        nb = np.linalg.norm(b)
        if nb < 1e-9:
            continue
        cos = a @ b / (np.linalg.norm(a) * nb)
        assert cos > 0.99, (name, cos)
        assert abs(np.linalg.norm(a) - nb) <= 5e-2 * nb, name
    # the update actually moves the parameters (Adam step)
    net.train_step(Fb, torch.as_tensor(y, device="cuda"), torch.as_tensor(w, device="cuda"),
                   torch.as_tensor(seg, device="cuda"), 4, 1e-3, update=True)
    assert np.abs(net.get_params() - params).max() > 1e-4
    net.close()


def test_features_match_reference():
    pr = workloads.make_problem("warm_1024", seed=5, m=300, n=250)
    net = drot.Mlp(0)
    feat = torch.zeros((320, 64), dtype=torch.bfloat16, device="cuda")
    xs = torch.as_tensor(pr.x, dtype=torch.float32, device="cuda").contiguous()
    yt = torch.as_tensor(pr.y, dtype=torch.float32, device="cuda").contiguous()
    net.features(xs, yt, torch.as_tensor(pr.p, device="cuda"), torch.as_tensor(pr.q, device="cuda"), feat, 10)
    got = feat.float().cpu().numpy()
    ref = ref_mlp.features(pr.x.astype(np.float32).astype(np.float64), pr.y.astype(np.float32).astype(np.float64),
                           pr.p, pr.q)
    assert np.abs(got[10:310] - ref).max() <= 1e-2 * max(1.0, np.abs(ref).max())
    assert np.all(got[:10] == 0) and np.all(got[310:] == 0)
    net.close()


def test_seed_is_dual_feasible_and_tight():
    pr = workloads.make_problem("warm_1024", seed=6, m=200, n=170)
    net = drot.Mlp(0, workloads.mlp_init_params(7))
    d = warmstart._device_problem(pr, 0)
    xs = torch.as_tensor(pr.x, dtype=torch.float32, device="cuda").contiguous()
    yt = torch.as_tensor(pr.y, dtype=torch.float32, device="cuda").contiguous()
    net.warm_start(xs, yt, d["p"], d["q"], pr.cost_scale, d["C"], d["X"], d["mu"], d["nu"])
    C = torch.as_tensor(pr.C, dtype=torch.float64, device="cuda")
    slack = C - d["mu"][:, None] - d["nu"][None, :]
    assert float(slack.min()) >= -1e-12
    assert float(slack.min(dim=1).values.abs().max()) <= 1e-12  # every row tight
    assert float(slack.min(dim=0).values.abs().max()) <= 1e-12  # every column tight
    assert np.array_equal(d["X"].cpu().numpy(), np.outer(pr.p, pr.q).astype(np.float32))
    net.close()


def test_seeded_step_parity_full_size_1024():
    """The seeded solve at the full 1024 x 1024 size of the warm-start workload (mixtures of four
    Gaussians, Dirichlet marginals, a held-out seed): the network's c-transform seed enters as
    (X_0 = p q^T, mu_0, nu_0) with phi_0 = rho mu_0 and psi_0 = rho nu_0 (Lemma opt-rel), and two
    iterations of the warm-started solve, launched as the benchmark launches it, match the FP64
    oracle run from the same seed: plan, duals, objective and l1 residual."""
    k = 2
    EPS32 = 2.0 ** -24
    pr = workloads.make_problem("warm_1024", seed=20_000)
    assert pr.m == 1024 and pr.n == 1024
    net = drot.Mlp(0, workloads.mlp_init_params(7))
    d = warmstart._device_problem(pr, 0)
    xs = torch.as_tensor(pr.x, dtype=torch.float32, device="cuda").contiguous()
    yt = torch.as_tensor(pr.y, dtype=torch.float32, device="cuda").contiguous()
    net.warm_start(xs, yt, d["p"], d["q"], pr.cost_scale, d["C"], d["X"], d["mu"], d["nu"])
    net.close()
    X0 = d["X"].cpu().numpy().astype(np.float64)
    mu0 = d["mu"].cpu().numpy().copy()
    nu0 = d["nu"].cpu().numpy().copy()
    with drot.Solver(device=0, stop_rule=drot.STOP_GAP) as s:
        out = s.solve(d["C"], d["p"], d["q"], rho=pr.rho, tol=-1.0, max_iter=k, X=d["X"], mu=d["mu"], nu=d["nu"],
                      warm=True)
    assert out["status"] == drot.DROT_NOT_CONVERGED and out["iters"] == k
    ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, k, X0=X0, mu0=mu0, nu0=nu0)
    S = max(np.abs(X0).max(), pr.rho * (np.abs(mu0).max() + np.abs(nu0).max() + 1.0), np.abs(ref["X"]).max())
    Xg = d["X"].cpu().numpy().astype(np.float64)
    assert Xg.min() >= 0.0
    assert np.abs(Xg - ref["X"]).max() <= 8 * EPS32 * S * k * 4
    tol_d = 64 * EPS32 * S / pr.rho * k + 1e-12
    assert np.abs(d["mu"].cpu().numpy() - ref["mu"]).max() <= tol_d
    assert np.abs(d["nu"].cpu().numpy() - ref["nu"]).max() <= tol_d
    h = ref["history"][-1]
    assert abs(out["primal_obj"] - h[oracle.PRIMAL]) <= 1e-5 * abs(h[oracle.PRIMAL]) + 1e-9
    assert abs(out["res_l1"] - h[oracle.RES_L1]) <= 1e-5 * abs(h[oracle.RES_L1]) + 1e-7


def _weighted_corr(a, b, w):
    a = a - (w * a).sum()
    b = b - (w * b).sum()
    return (w * a * b).sum() / np.sqrt((w * a * a).sum() * (w * b * b).sum())


def test_chunked_labelling_matches_the_whole_set_path():
    """labelled_training_set (problems built on the device and labelled chunk by chunk, as the bench
    does at twenty thousand problems) gives the same rows as labelling every problem first and
    building the set afterwards: the costs are bit-identical, so features, weights and segments
    match exactly; the labels are the same solves up to the order of the FP64 atomic sums, which
    depends on how a batch is split over the CTAs."""
    rule = drot.STOP_GAP | drot.STOP_RES_L1
    sizes = [(96, 80), (130, 64), (64, 200), (101, 101), (77, 150)]
    host = [workloads.make_problem("warm_1024", seed=300 + k, m=m, n=n) for k, (m, n) in enumerate(sizes)]
    net = drot.Mlp(0, workloads.mlp_init_params(2))
    with drot.Solver(device=0, stop_rule=rule) as solver:
        mus, _ = warmstart.solve_labels(host, solver, tol=1e-4, max_iter=500_000, chunk=2)
        ref = warmstart.build_training_set(host, mus, net)
        ts, res = warmstart.labelled_training_set(
            lambda k: workloads.make_problem("warm_1024", seed=300 + k, m=sizes[k][0], n=sizes[k][1], device="cuda"),
            len(sizes), net, solver, tol=1e-4, max_iter=500_000, chunk=2)
    assert len(res) == len(sizes) and all(r["status"] == drot.DROT_OK for r in res)
    assert ts.sizes == ref.sizes and ts.row0 == ref.row0
    assert ts.feat.shape == ref.feat.shape and torch.equal(ts.feat, ref.feat)
    assert torch.equal(ts.seg, ref.seg) and torch.equal(ts.weight, ref.weight)
    assert float((ts.target - ref.target).abs().max()) <= 1e-3 * float(ref.target.abs().max())
    net.close()


@pytest.fixture(scope="module")
def trained_mixture_net():
    """A network trained on DROT's own duals of 128 small mixture-of-Gaussians problems (labels
    from batched solves under the full test at 1e-5), with the untrained network it started as."""
    m = 128
    rule = drot.STOP_GAP | drot.STOP_RES_L1
    train_probs = [workloads.make_problem("warm_1024", seed=1000 + s, m=m, n=m) for s in range(128)]
    with drot.Solver(device=0, stop_rule=rule) as solver:
        mus, res = warmstart.solve_labels(train_probs, solver, tol=1e-5, max_iter=2_000_000)
    assert all(r["status"] == drot.DROT_OK for r in res)
    untrained = drot.Mlp(0, workloads.mlp_init_params(11))
    net = drot.Mlp(0, workloads.mlp_init_params(11))
    ts = warmstart.build_training_set(train_probs, mus, net)
    losses = warmstart.train(net, ts, steps=600, batch=16, lr=2e-3, seed=1)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:20])
    yield net, untrained
    net.close()
    untrained.close()


def _held_out(count, m=128):
    return [workloads.make_problem("warm_1024", seed=5000 + s, m=m, n=m) for s in range(count)]


def test_trained_network_predicts_duals_and_full_rule_solves_take_as_long_as_cold(trained_mixture_net):
    """On held-out problems of the training family the trained network's potentials correlate with
    the solved duals far better than the untrained one's, and seeded solves reach the cold-start
    objective under the full primal-dual test (gap and l1 residual).  What the seed buys there is
    measured and asserted as measured: nothing material.  The number of iterations DR needs is set
    by its slow final phase, not by how far the start is from a fixed point: in FP64 on the CPU
    (256 x 256, this family) even the exact optimal duals with X_0 = p q^T took 2494 / 12289 /
    59704 / 332247 iterations to 1e-3 / 1e-4 / 1e-5 / 1e-6 against 2846 / 12850 / 98086 / 273927
    cold.  So the test asserts that the cold / warm iteration ratio stays within [2/3, 3/2]."""
    net, untrained = trained_mixture_net
    rule = drot.STOP_GAP | drot.STOP_RES_L1
    cold, warm, corr_t, corr_u = [], [], [], []
    with drot.Solver(device=0, stop_rule=rule) as solver:
        for pr in _held_out(8):
            c = warmstart.cold_solve(solver, pr, tol=1e-5, max_iter=3_000_000)
            assert c["status"] == drot.DROT_OK
            mu_star = c["mu"].cpu().numpy()
            for model, sink in ((net, corr_t), (untrained, corr_u)):
                d = warmstart._device_problem(pr, 0)
                xs = torch.as_tensor(pr.x, dtype=torch.float32, device="cuda").contiguous()
                yt = torch.as_tensor(pr.y, dtype=torch.float32, device="cuda").contiguous()
                model.warm_start(xs, yt, d["p"], d["q"], pr.cost_scale, d["C"], d["X"], d["mu"], d["nu"])
                sink.append(_weighted_corr(d["mu"].cpu().numpy(), mu_star, pr.p))
            w = warmstart.warm_solve(net, solver, pr, tol=1e-5, max_iter=3_000_000, fallback=False)
            assert w["status"] == drot.DROT_OK
            assert abs(w["primal_obj"] - c["primal_obj"]) <= 1e-4 * c["primal_obj"] + 1e-5
            cold.append(c["iters"])
            warm.append(w["iters"])
    ratio = np.mean(cold) / np.mean(warm)
    print(f"warm-start, full rule at 1e-5: duals corr trained {np.mean(corr_t):.4f} vs untrained "
          f"{np.mean(corr_u):.4f}; iterations cold {cold} warm {warm}; cold/warm {ratio:.3f}")
    assert np.mean(corr_t) > 0.75 and np.mean(corr_t) > np.mean(corr_u) + 0.5
    assert 2.0 / 3.0 <= ratio <= 1.5, (cold, warm)


def test_gap_rule_seeded_solves_stop_sooner_but_neither_stop_is_a_solution(trained_mixture_net):
    """Under the duality gap alone (the metric's condition) the seeded solves stop after fewer
    iterations than cold ones on average, but the gap test fires where primal and dual objectives
    cross, and on this family both kinds of stop leave the plan's marginals far from met: the
    mean l1 residual at the stop exceeds 100 x tol on both sides.  How feasible a stop is varies
    from problem to problem and from run to run (measured on B300 over the same eight problems:
    mean l1 6.4e-3 cold against 6.0e-3 and 1.6e-2 warm in two runs whose networks differed only
    through the order of atomic additions in the labels, features and gradients), so no ordering
    of the two residuals is asserted; the library's default test requires the l1 residual too."""
    net, _ = trained_mixture_net
    cold, warm = [], []
    with drot.Solver(device=0, stop_rule=drot.STOP_GAP) as solver:
        for pr in _held_out(8):
            c = warmstart.cold_solve(solver, pr, tol=1e-6, max_iter=3_000_000)
            w = warmstart.warm_solve(net, solver, pr, tol=1e-6, max_iter=3_000_000, fallback=False)
            assert c["status"] == drot.DROT_OK and w["status"] == drot.DROT_OK
            cold.append((c["iters"], c["res_l1"]))
            warm.append((w["iters"], w["res_l1"]))
    print(f"warm-start, gap rule at 1e-6: (iterations, l1 at stop) cold {cold} warm {warm}")
    assert np.mean([w[0] for w in warm]) < np.mean([c[0] for c in cold])
    assert np.mean([c[1] for c in cold]) > 100 * 1e-6 and np.mean([w[1] for w in warm]) > 100 * 1e-6
