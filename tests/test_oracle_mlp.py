"""Pins for the FP64 reference of the warm-start network (oracle/mlp.py)."""

import numpy as np

import workloads
from oracle import mlp


def _data(rows=40, nseg=3, seed=0):
    rng = np.random.default_rng(seed)
    F = rng.uniform(-1, 1, size=(rows, mlp.IN))
    y = rng.standard_normal(rows)
    w = rng.uniform(0.1, 1.0, rows)
    seg = rng.integers(0, nseg, rows)
    return F, y, w, seg


def test_gradient_matches_finite_differences():
    params = workloads.mlp_init_params(1).astype(np.float64)
    F, y, w, seg = _data()
    L, g = mlp.loss_and_grad(params, F, y, w, seg, 3)
    rng = np.random.default_rng(1)
    # sample parameters of every block, including the output layer and the biases
    idx = np.concatenate([rng.integers(0, mlp.NPARAMS, 40), np.arange(mlp.NPARAMS - 5, mlp.NPARAMS)])
    h = 1e-6
    for k in idx:
        pp = params.copy()
        pp[k] += h
        pm = params.copy()
        pm[k] -= h
        fd = (mlp.loss_and_grad(pp, F, y, w, seg, 3)[0] - mlp.loss_and_grad(pm, F, y, w, seg, 3)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (k, fd, g[k])


def test_loss_is_gauge_invariant_per_problem():
    params = workloads.mlp_init_params(2).astype(np.float64)
    F, y, w, seg = _data(seed=3)
    out, _ = mlp.forward(params, F)
    L0, _ = mlp.loss(out, y, w, seg, 3)
    shift = np.array([0.3, -2.0, 5.0])[seg]
    L1, _ = mlp.loss(out, y + shift, w, seg, 3)
    assert abs(L0 - L1) < 1e-12 * max(1, L0)


def test_constant_network_loss_is_weighted_variance():
    params = np.zeros(mlp.NPARAMS)
    params[-1] = 0.7  # only the output bias: out = 0.7 everywhere
    F, y, w, seg = _data(seed=4)
    out, _ = mlp.forward(params, F)
    assert np.all(out == 0.7)
    L, _ = mlp.loss(out, y, w, seg, 3)
    ref = 0.0
    for s in range(3):
        i = seg == s
        mean = (w[i] * y[i]).sum() / w[i].sum()
        ref += (w[i] * (y[i] - mean) ** 2).sum()
    assert abs(L - ref / 3) < 1e-12


def test_features_layout():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (10, 2))
    y = rng.uniform(0, 1, (7, 2))
    p = rng.dirichlet(np.ones(10))
    q = rng.dirichlet(np.ones(7))
    F = mlp.features(x, y, p, q)
    assert F.shape == (10, 64)
    assert np.allclose(F[:, 3:19].sum(1), 1.0) and np.allclose(F[:, 19:35].sum(1), 1.0)
    assert np.allclose(F[:, 2], 10 * p) and np.all(F[:, 42] == 1.0) and np.all(F[:, 43:] == 0.0)
    assert np.allclose(F[0, 37:39], q @ y)
