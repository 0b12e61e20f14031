"""Seeded synthetic OT problems shaped like the paper's workloads.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` so a
(config, seed) pair fixes the problem bit for bit.  Cost matrices are built in
FP64 as squared Euclidean distances, divided by their largest entry (so that
the entrywise max norm of C is 1, as in the paper's experiments, Sec. 4) and
then rounded once to FP32.  The FP32 matrix is the problem both solvers see:
the GPU reads it as is, the CPU oracle promotes it back to FP64.

Two cost builders produce bit-identical FP32 matrices: a NumPy one for the CPU
and a PyTorch one that can run on any device (used for the large problems,
whose FP64 intermediates would be slow to build on the host).  Both perform the
same IEEE operations in the same order: per coordinate a subtraction and a
product, accumulated in coordinate order, one division by the maximum, one
rounding to FP32.
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Named workloads.  Sizes, point distributions and marginals follow the
# configurations this library is measured on; "paper_gauss" follows the
# generator described in Sec. 4 of the paper (2-D Gaussians with random means
# and covariances, target means drawn around 5, uniform marginals).
CONFIGS = {
    "plain_256": dict(kind="uniform", m=256, n=256, dim=2, marginals="uniform", rho0=2.0, tol=1e-6),
    "plain_8192x6144": dict(kind="gauss_pair", m=8192, n=6144, dim=2, marginals="uniform_random", rho0=2.0, tol=1e-6),
    "plain_20000": dict(kind="uniform", m=20000, n=20000, dim=3, marginals="uniform", rho0=2.0, tol=1e-6),
    "batched_512": dict(kind="shifted_uniform", B=512, mn_low=64, mn_high=2048, dim=2, marginals="dirichlet", rho0=2.0, tol=1e-6),
    "warm_1024": dict(kind="mixture4", m=1024, n=1024, dim=2, marginals="dirichlet", rho0=2.0, tol=1e-6),
    "paper_gauss": dict(kind="paper_gauss", m=512, n=512, dim=2, marginals="uniform", rho0=2.0, tol=1e-4, sigma_t=5.0),
}


@dataclasses.dataclass
class Problem:
    """One OT instance: minimise <C, X> s.t. X >= 0, X 1 = p, X^T 1 = q."""

    name: str
    seed: int
    m: int
    n: int
    C: object  # np.ndarray float32 (m, n) or torch.Tensor float32
    p: np.ndarray  # float64 (m,)
    q: np.ndarray  # float64 (n,)
    rho: float
    tol: float
    x: Optional[np.ndarray] = None  # source points (m, dim), float64
    y: Optional[np.ndarray] = None  # target points (n, dim), float64
    cost_scale: float = 1.0         # C = squared distances / cost_scale


def default_rho(m: int, n: int, rho0: float = 2.0) -> float:
    """rho = rho0 / (m + n), the step-size rule of the paper's experiments."""
    return float(rho0) / float(m + n)


def pad_ld(n: int) -> int:
    """Row pitch (in floats) that keeps every row 16-byte aligned."""
    return (int(n) + 3) // 4 * 4


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def sq_euclidean_cost_np(x: np.ndarray, y: np.ndarray, block_rows: int = 4096, return_scale: bool = False):
    """FP32 matrix of ||x_i - y_j||^2 / max_ij ||x_i - y_j||^2 (built in FP64).

    With ``return_scale`` also returns the divisor max_ij ||x_i - y_j||^2.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m, d = x.shape
    n = y.shape[0]

    def block(i0, i1):
        acc = np.zeros((i1 - i0, n), dtype=np.float64)
        for k in range(d):
            diff = x[i0:i1, k][:, None] - y[:, k][None, :]
            acc += diff * diff
        return acc

    cmax = 0.0
    for i0 in range(0, m, block_rows):
        cmax = max(cmax, float(block(i0, min(m, i0 + block_rows)).max()))
    if cmax <= 0.0:
        cmax = 1.0
    out = np.empty((m, n), dtype=np.float32)
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        b = block(i0, i1)
        b /= cmax
        out[i0:i1] = b.astype(np.float32)
    return (out, cmax) if return_scale else out


def sq_euclidean_cost_torch(x: np.ndarray, y: np.ndarray, device="cpu", ld: Optional[int] = None,
                            block_rows: int = 2048, return_scale: bool = False):
    """Same matrix as :func:`sq_euclidean_cost_np`, built with torch on ``device``.

    Returns a float32 tensor of shape (m, ld) whose first n columns hold the
    cost (ld defaults to n; padding columns are zero).
    """
    import torch

    xt = torch.as_tensor(np.asarray(x, dtype=np.float64), device=device)
    yt = torch.as_tensor(np.asarray(y, dtype=np.float64), device=device)
    m, d = xt.shape
    n = yt.shape[0]
    ld = n if ld is None else int(ld)

    def block(i0, i1):
        acc = torch.zeros((i1 - i0, n), dtype=torch.float64, device=device)
        for k in range(d):
            diff = xt[i0:i1, k][:, None] - yt[:, k][None, :]
            acc += diff * diff
        return acc

    cmax = torch.zeros((), dtype=torch.float64, device=device)
    for i0 in range(0, m, block_rows):
        cmax = torch.maximum(cmax, block(i0, min(m, i0 + block_rows)).max())
    cmax_v = float(cmax)
    if cmax_v <= 0.0:
        cmax_v = 1.0
    out = torch.zeros((m, ld), dtype=torch.float32, device=device)
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        b = block(i0, i1)
        b /= cmax_v
        out[i0:i1, :n] = b.to(torch.float32)
    return (out, cmax_v) if return_scale else out


def _marginal(rng: np.random.Generator, k: int, kind: str) -> np.ndarray:
    if kind == "uniform":
        return np.full(k, 1.0 / k, dtype=np.float64)
    if kind == "uniform_random":
        w = rng.uniform(0.0, 1.0, size=k)
        return w / w.sum()
    if kind == "dirichlet":
        return rng.dirichlet(np.ones(k))
    raise ValueError(f"unknown marginal kind {kind!r}")


def _rescale_mass(p: np.ndarray, q: np.ndarray):
    """Make sum(q) equal sum(p) to the last bit where possible (both ~1)."""
    q = q * (p.sum() / q.sum())
    return p, q


def _points(rng: np.random.Generator, spec: dict, m: int, n: int):
    kind = spec["kind"]
    d = spec["dim"]
    if kind == "uniform":
        return rng.uniform(0.0, 1.0, size=(m, d)), rng.uniform(0.0, 1.0, size=(n, d))
    if kind == "gauss_pair":
        x = rng.standard_normal(size=(m, d))
        y = 1.0 + np.sqrt(0.5) * rng.standard_normal(size=(n, d))
        return x, y
    if kind == "shifted_uniform":
        x = rng.uniform(0.0, 1.0, size=(m, d))
        shift = rng.uniform(0.0, 1.0, size=(1, d))
        y = rng.uniform(0.0, 1.0, size=(n, d)) + shift
        return x, y
    if kind == "mixture4":
        def cloud(k):
            means = rng.uniform(0.2, 0.8, size=(4, d))
            comp = rng.integers(0, 4, size=k)
            pts = means[comp] + 0.06 * rng.standard_normal(size=(k, d))
            return np.clip(pts, 0.0, 1.0)
        return cloud(m), cloud(n)
    if kind == "paper_gauss":
        sigma_t = float(spec.get("sigma_t", 5.0))
        mu_s = rng.standard_normal(size=d)
        a_s = rng.uniform(0.0, 1.0, size=(d, d))
        mu_t = rng.normal(5.0, sigma_t, size=d)
        a_t = rng.uniform(0.0, 1.0, size=(d, d))
        x = mu_s + rng.standard_normal(size=(m, d)) @ a_s.T
        y = mu_t + rng.standard_normal(size=(n, d)) @ a_t.T
        return x, y
    raise ValueError(f"unknown point kind {kind!r}")


def make_problem(name: str, seed: int = 0, m: Optional[int] = None, n: Optional[int] = None,
                 device=None, ld: Optional[int] = None, **overrides) -> Problem:
    """Build the named workload.

    ``m``/``n`` override the sizes (same distributions), ``device`` selects the
    torch cost builder (returns C as a float32 tensor of shape (m, ld)); without
    it C is a NumPy float32 array of shape (m, n).
    """
    spec = dict(CONFIGS[name])
    spec.update(overrides)
    if spec["kind"] == "shifted_uniform" and (m is None or n is None):
        raise ValueError("batched workloads are built with make_batch()")
    m = int(spec["m"] if m is None else m)
    n = int(spec["n"] if n is None else n)
    rng = _rng(seed)
    x, y = _points(rng, spec, m, n)
    p = _marginal(rng, m, spec["marginals"])
    q = _marginal(rng, n, spec["marginals"])
    p, q = _rescale_mass(p, q)
    if device is None:
        C, scale = sq_euclidean_cost_np(x, y, return_scale=True)
    else:
        C, scale = sq_euclidean_cost_torch(x, y, device=device, ld=ld, return_scale=True)
    return Problem(name=name, seed=seed, m=m, n=n, C=C, p=p, q=q,
                   rho=default_rho(m, n, spec["rho0"]), tol=float(spec["tol"]), x=x, y=y, cost_scale=float(scale))


def make_batch(name: str = "batched_512", seed: int = 0, B: Optional[int] = None,
               mn_low: Optional[int] = None, mn_high: Optional[int] = None, device=None) -> list:
    """Independent problems of uneven shape, m and n each uniform in [mn_low, mn_high].

    ``device`` selects the torch cost builder (each C a float32 tensor of shape (m, pad_ld(n))
    on that device, bit-identical to the NumPy one); without it C is a NumPy (m, n) array."""
    spec = dict(CONFIGS[name])
    B = int(spec["B"] if B is None else B)
    lo = int(spec["mn_low"] if mn_low is None else mn_low)
    hi = int(spec["mn_high"] if mn_high is None else mn_high)
    rng = _rng(seed)
    shapes = rng.integers(lo, hi + 1, size=(B, 2))
    seeds = rng.integers(0, 2**31 - 1, size=B)
    probs = []
    for b in range(B):
        m, n = int(shapes[b, 0]), int(shapes[b, 1])
        r = _rng(int(seeds[b]))
        x, y = _points(r, spec, m, n)
        p = _marginal(r, m, spec["marginals"])
        q = _marginal(r, n, spec["marginals"])
        p, q = _rescale_mass(p, q)
        if device is None:
            C, scale = sq_euclidean_cost_np(x, y, return_scale=True)
        else:
            C, scale = sq_euclidean_cost_torch(x, y, device=device, ld=pad_ld(n), return_scale=True)
        probs.append(Problem(name=f"{name}[{b}]", seed=int(seeds[b]), m=m, n=n, C=C, p=p, q=q,
                             rho=default_rho(m, n, spec["rho0"]), tol=float(spec["tol"]), x=x, y=y,
                             cost_scale=float(scale)))
    return probs


def mlp_init_params(seed: int) -> np.ndarray:
    """Initial parameters of the warm-start network (flat FP32, layout of drot_mlp_set_params).

    He-normal weights (std sqrt(2 / fan_in)) for the three hidden layers, std 1/16 for the
    output weights, zero biases.
    """
    rng = _rng(seed)
    fin, width = 64, 256
    parts = [rng.standard_normal(width * fin) * np.sqrt(2.0 / fin), np.zeros(width),
             rng.standard_normal(width * width) * np.sqrt(2.0 / width), np.zeros(width),
             rng.standard_normal(width * width) * np.sqrt(2.0 / width), np.zeros(width),
             rng.standard_normal(width) / 16.0, np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def random_start(m: int, n: int, seed: int):
    """A random starting state (X0, mu0, nu0) for step-level comparisons.

    X0 has FP32-representable nonnegative entries of the size of a plan
    (about 1/(m n)), a quarter of them exactly zero; mu0, nu0 are FP64 values of
    the size of the duals of a max-normalised cost.
    """
    rng = _rng(seed)
    X0 = rng.uniform(0.0, 2.0 / (m * n), size=(m, n))
    X0[rng.uniform(size=(m, n)) < 0.25] = 0.0
    X0 = X0.astype(np.float32)
    mu0 = rng.uniform(-0.5, 0.5, size=m)
    nu0 = rng.uniform(-0.5, 0.5, size=n)
    return X0, mu0, nu0
