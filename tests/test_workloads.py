"""The seeded generators: reproducible, well-formed, and identical across the two cost builders."""

import numpy as np
import pytest
import torch

import workloads


def test_numpy_and_torch_cost_builders_agree_bitwise():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((37, 3))
    y = rng.standard_normal((29, 3)) + 0.5
    a = workloads.sq_euclidean_cost_np(x, y, block_rows=8)
    b = workloads.sq_euclidean_cost_torch(x, y, device="cpu", ld=32, block_rows=5)
    assert b.shape == (37, 32)
    assert np.array_equal(a.view(np.uint32), b[:, :29].numpy().view(np.uint32))
    assert float(b[:, 29:].abs().max()) == 0.0
    assert a.max() == np.float32(1.0) and a.min() >= 0.0


@pytest.mark.parametrize("name", ["plain_256", "plain_8192x6144", "warm_1024", "paper_gauss", "plain_20000"])
def test_problems_are_seeded_and_well_formed(name):
    a = workloads.make_problem(name, seed=3, m=40, n=24)
    b = workloads.make_problem(name, seed=3, m=40, n=24)
    c = workloads.make_problem(name, seed=4, m=40, n=24)
    assert np.array_equal(a.C, b.C) and np.array_equal(a.p, b.p)
    assert not np.array_equal(a.C, c.C)
    assert a.C.dtype == np.float32 and a.C.shape == (40, 24)
    assert a.p.min() > 0 and a.q.min() > 0
    assert abs(a.p.sum() - 1) < 1e-12 and abs(a.p.sum() - a.q.sum()) < 1e-15
    assert abs(a.rho - 2.0 / 64) < 1e-18


def test_batch_shapes():
    probs = workloads.make_batch(B=6, seed=1)
    assert len(probs) == 6
    for pr in probs:
        assert 64 <= pr.m <= 2048 and 64 <= pr.n <= 2048
        assert pr.C.shape == (pr.m, pr.n)
        assert abs(pr.p.sum() - pr.q.sum()) < 1e-15


def test_random_start():
    X0, mu0, nu0 = workloads.random_start(13, 7, seed=2)
    assert X0.dtype == np.float32 and X0.min() >= 0 and (X0 == 0).any()
    assert mu0.shape == (13,) and nu0.shape == (7,)
    assert workloads.pad_ld(7) == 8 and workloads.pad_ld(8) == 8
