"""Learned warm start for DROT: data from the solver itself, training and seeded solves.

Orchestration only: features, the network's forward and backward passes, Adam, the
c-transforms of the seed and every solve run in the library's kernels (drot_mlp_* and
drot_solve / drot_solve_batched); this module moves tensors between those calls.

The network predicts each source point's dual potential mu_i in units of the squared
distance (labels are DROT's own duals mu = phi / rho times the cost scale).  A seeded solve
starts from X_0 = p q^T, mu_0 = the prediction made dual feasible by c-transforms, and
nu_0 its c-transform (phi_0 = rho mu_0, psi_0 = rho nu_0, Lemma opt-rel, Appendix A.2).
Plain cold-start DROT (the paper's X_0 = p q^T, phi_0 = psi_0 = 0) is the fallback and
the reference the warm start is judged against.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

from . import drot

ROW_PAD = 64


@dataclasses.dataclass
class TrainingSet:
    feat: object      # torch.bfloat16 (rows, 64), rows a multiple of 64
    target: object    # torch.float32 (rows,)
    weight: object    # torch.float32 (rows,)
    seg: object       # torch.int32 (rows,), -1 for padding rows
    row0: List[int]   # first row of each problem
    sizes: List[int]  # source points of each problem


def _device_problem(pr, device):
    import torch

    ld = (pr.n + 3) // 4 * 4
    C = torch.zeros((pr.m, ld), dtype=torch.float32, device=device)
    C[:, : pr.n] = torch.as_tensor(pr.C, device=device)
    X = torch.zeros_like(C)
    return dict(C=C[:, : pr.n], X=X[:, : pr.n], p=torch.as_tensor(pr.p, device=device),
                q=torch.as_tensor(pr.q, device=device),
                mu=torch.zeros(pr.m, dtype=torch.float64, device=device),
                nu=torch.zeros(pr.n, dtype=torch.float64, device=device), rho=pr.rho)


def solve_labels(problems: Sequence, solver: drot.Solver, tol: float, max_iter: int, device=0, chunk: int = 256):
    """Dual potentials of each problem from batched DROT solves (cold start, library default stop rule)."""
    mus, results = [], []
    for s in range(0, len(problems), chunk):
        part = problems[s:s + chunk]
        dev = [_device_problem(pr, device) for pr in part]
        res = solver.solve_batched(dev, tol=tol, max_iter=max_iter, check=False)
        for d, r in zip(dev, res):
            mus.append(d["mu"].cpu().numpy())
            results.append(r)
        del dev
    return mus, results


def build_training_set(problems: Sequence, mus: Sequence, net: drot.Mlp, device=0) -> TrainingSet:
    import torch

    rows0, sizes = [], []
    total = 0
    for pr in problems:
        rows0.append(total)
        sizes.append(pr.m)
        total += pr.m
    rows = (total + ROW_PAD - 1) // ROW_PAD * ROW_PAD
    feat = torch.zeros((rows, drot.MLP_FEATURES), dtype=torch.bfloat16, device=device)
    target = torch.zeros(rows, dtype=torch.float32, device=device)
    weight = torch.zeros(rows, dtype=torch.float32, device=device)
    seg = torch.full((rows,), -1, dtype=torch.int32, device=device)
    for k, (pr, mu) in enumerate(zip(problems, mus)):
        xs = torch.as_tensor(pr.x, dtype=torch.float32, device=device).contiguous()
        yt = torch.as_tensor(pr.y, dtype=torch.float32, device=device).contiguous()
        p = torch.as_tensor(pr.p, device=device)
        q = torch.as_tensor(pr.q, device=device)
        net.features(xs, yt, p, q, feat, rows0[k])
        r0 = rows0[k]
        target[r0:r0 + pr.m] = torch.as_tensor(mu * pr.cost_scale, dtype=torch.float32, device=device)
        weight[r0:r0 + pr.m] = torch.as_tensor(pr.p, dtype=torch.float32, device=device)
        seg[r0:r0 + pr.m] = k
    return TrainingSet(feat=feat, target=target, weight=weight, seg=seg, row0=rows0, sizes=sizes)


def labelled_training_set(make, count: int, net: drot.Mlp, solver: drot.Solver, tol: float, max_iter: int,
                          device=0, chunk: int = 512):
    """Label `count` problems with batched cold DROT solves and turn them into feature rows, one
    chunk at a time: ``make(k)`` builds problem k (its cost preferably already on `device`), and
    only one chunk's costs and plans are resident at once, so the set can hold tens of
    thousands of problems.  Returns (TrainingSet, the label solves' result dicts)."""
    import torch

    feats, targets, weights, segs, sizes, results = [], [], [], [], [], []
    for s in range(0, count, chunk):
        part = [make(k) for k in range(s, min(count, s + chunk))]
        dev = [_device_problem(pr, device) for pr in part]
        results.extend(solver.solve_batched(dev, tol=tol, max_iter=max_iter, check=False))
        rows = sum(pr.m for pr in part)
        feat = torch.zeros((rows, drot.MLP_FEATURES), dtype=torch.bfloat16, device=device)
        r0 = 0
        for j, (pr, d) in enumerate(zip(part, dev)):
            xs = torch.as_tensor(pr.x, dtype=torch.float32, device=device).contiguous()
            yt = torch.as_tensor(pr.y, dtype=torch.float32, device=device).contiguous()
            net.features(xs, yt, d["p"], d["q"], feat, r0)
            targets.append((d["mu"] * pr.cost_scale).to(torch.float32))
            weights.append(d["p"].to(torch.float32))
            segs.append(torch.full((pr.m,), s + j, dtype=torch.int32, device=device))
            sizes.append(pr.m)
            r0 += pr.m
        feats.append(feat)
        del dev, part
    total = sum(sizes)
    rows = (total + ROW_PAD - 1) // ROW_PAD * ROW_PAD
    pad = rows - total
    feat = torch.cat(feats + [torch.zeros((pad, drot.MLP_FEATURES), dtype=torch.bfloat16, device=device)])
    target = torch.cat(targets + [torch.zeros(pad, dtype=torch.float32, device=device)])
    weight = torch.cat(weights + [torch.zeros(pad, dtype=torch.float32, device=device)])
    seg = torch.cat(segs + [torch.full((pad,), -1, dtype=torch.int32, device=device)])
    row0 = [int(x) for x in np.cumsum([0] + sizes[:-1])]
    return TrainingSet(feat=feat, target=target, weight=weight, seg=seg, row0=row0, sizes=sizes), results


def subset(ts: TrainingSet, idx: Sequence[int], device=0) -> TrainingSet:
    """The rows of problems `idx`, renumbered 0..len(idx)-1 and padded to a multiple of 64."""
    import torch

    parts = [torch.arange(ts.row0[k], ts.row0[k] + ts.sizes[k], device=device) for k in idx]
    rows_idx = torch.cat(parts)
    total = rows_idx.numel()
    rows = (total + ROW_PAD - 1) // ROW_PAD * ROW_PAD
    feat = torch.zeros((rows, drot.MLP_FEATURES), dtype=torch.bfloat16, device=device)
    feat[:total] = ts.feat[rows_idx]
    target = torch.zeros(rows, dtype=torch.float32, device=device)
    target[:total] = ts.target[rows_idx]
    weight = torch.zeros(rows, dtype=torch.float32, device=device)
    weight[:total] = ts.weight[rows_idx]
    seg = torch.full((rows,), -1, dtype=torch.int32, device=device)
    off = 0
    row0 = []
    for j, k in enumerate(idx):
        seg[off:off + ts.sizes[k]] = j
        row0.append(off)
        off += ts.sizes[k]
    return TrainingSet(feat=feat, target=target, weight=weight, seg=seg, row0=row0,
                       sizes=[ts.sizes[k] for k in idx])


def train(net: drot.Mlp, ts: TrainingSet, steps: int, batch: int, lr: float, seed: int = 0,
          device=0) -> List[float]:
    """Adam on random minibatches of `batch` problems; returns the loss of every step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nprob = len(ts.sizes)
    losses = []
    for step in range(steps):
        idx = rng.choice(nprob, size=min(batch, nprob), replace=False)
        mb = subset(ts, list(idx), device)
        decay = 0.5 * (1.0 + np.cos(np.pi * step / max(1, steps)))  # cosine schedule
        losses.append(net.train_step(mb.feat, mb.target, mb.weight, mb.seg, len(idx), lr * (0.05 + 0.95 * decay)))
    return losses


def warm_solve(net: drot.Mlp, solver: drot.Solver, pr, tol: float, max_iter: int, device=0,
               fallback: bool = True):
    """Solve `pr` from the network's seed; returns drot_solve's result dict (with "X", "mu",
    "nu" and "seeded": whether the returned solve is the warm-started one).  If the seeded
    solve fails (any status other than converged) and ``fallback`` is set, the plain
    cold-start solve is run and returned instead."""
    import torch

    d = _device_problem(pr, device)
    xs = torch.as_tensor(pr.x, dtype=torch.float32, device=device).contiguous()
    yt = torch.as_tensor(pr.y, dtype=torch.float32, device=device).contiguous()
    net.warm_start(xs, yt, d["p"], d["q"], pr.cost_scale, d["C"], d["X"], d["mu"], d["nu"])
    out = solver.solve(d["C"], d["p"], d["q"], rho=pr.rho, tol=tol, max_iter=max_iter, X=d["X"], mu=d["mu"],
                       nu=d["nu"], warm=True, check=False)
    out.update(C=d["C"], p=d["p"], q=d["q"], seeded=True)
    if fallback and out["status"] != drot.DROT_OK:
        out = cold_solve(solver, pr, tol, max_iter, device)
        out["seeded"] = False
    return out


def cold_solve(solver: drot.Solver, pr, tol: float, max_iter: int, device=0):
    """The paper's plain solve from X_0 = p q^T; the result dict also carries the problem's device
    buffers C, p, q."""
    d = _device_problem(pr, device)
    out = solver.solve(d["C"], d["p"], d["q"], rho=pr.rho, tol=tol, max_iter=max_iter, X=d["X"], mu=d["mu"],
                       nu=d["nu"], check=False)
    out.update(C=d["C"], p=d["p"], q=d["q"])
    return out
