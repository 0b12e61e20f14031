"""Row-sharded Algorithm 1 (Sec. 3.1) on two gloo ranks against the unsharded FP64 oracle.

The step shards by row blocks: a rank owns rows of X, C, p, phi and a; psi, b and alpha are
replicated.  Per iteration the only exchange is one all-reduce of the n column sums and six
scalars (sum r, ||r||_1, ||r||^2, p.phi-numerator, <C,X>, sum [d]_+^2); each rank then updates
psi, b, alpha identically and phi, a for its own rows.  This is the multi-GPU formulation the
library does not build (every box here has one GPU: it runs replicas); the test pins that one
exchange of n + 6 doubles per iteration reproduces the unsharded iteration exactly (up to
summation order)."""

import os
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sharded_run(rank, world, port, k, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import workloads

    pr = workloads.make_problem("plain_256", seed=17, m=37, n=23)
    C = pr.C.astype(np.float64)
    p, q, rho = pr.p, pr.q, pr.rho
    m, n = C.shape
    rows = np.array_split(np.arange(m), world)[rank]
    Cl, pl = C[rows], p[rows]
    # cold start X_0 = p q^T, phi_0 = psi_0 = 0; a_0 = X_0 1 - p, b_0 = X_0^T 1 - q, alpha_0 = 1^T a_0 / (m + n)
    Xl = np.outer(pl, q)
    al = Xl.sum(1) - pl
    v0 = torch.as_tensor(np.concatenate([Xl.sum(0), [al.sum()]]))
    dist.all_reduce(v0)
    b = v0[:n].numpy() - q
    alpha = float(v0[n]) / (m + n)
    phil = np.zeros(len(rows))
    psi = np.zeros(n)
    for _ in range(k):
        D = phil[:, None] + psi[None, :] - rho * Cl
        Xl = np.maximum(Xl + D, 0.0)
        rl = Xl.sum(1) - pl
        payload = torch.as_tensor(np.concatenate([
            Xl.sum(0),                                               # column sums (n)
            [rl.sum(), np.abs(rl).sum(), (rl * rl).sum(),            # row-side totals
             (Cl * Xl).sum(), (np.maximum(D, 0.0) ** 2).sum(), 0.0]]))
        dist.all_reduce(payload)                                     # the one exchange per iteration
        v = payload[:n].numpy()
        sum_r = float(payload[n])
        s = v - q
        beta = sum_r / (m + n)                                       # step 5
        c = 2.0 * beta - alpha
        phil = (al - 2.0 * rl + c) / n                               # steps 6-7
        psi = (b - 2.0 * s + c) / m
        al = al - rl                                                 # step 8
        b = b - s
        alpha = alpha - beta
    out[rank] = (rows.tolist(), Xl.tolist(), float(payload[n + 3]))
    dist.destroy_process_group()


def test_row_sharded_iteration_matches_oracle():
    import oracle
    import workloads

    k = 25
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_sharded_run, args=(2, 29527, k, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    pr = workloads.make_problem("plain_256", seed=17, m=37, n=23)
    ref = oracle.drot_run(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, k)
    X = np.zeros_like(ref["X"])
    for rows, Xl, _ in res.values():
        X[rows] = np.array(Xl)
    scale = np.abs(ref["X"]).max()
    assert np.abs(X - ref["X"]).max() <= 1e-12 * scale
    # <C, X_k> assembled from the shards' partial sums by the exchange
    assert res[0][2] == res[1][2]
    assert abs(res[0][2] - ref["history"][-1][oracle.PRIMAL]) <= 1e-12 * abs(ref["history"][-1][oracle.PRIMAL])
