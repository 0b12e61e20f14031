"""FP64 CPU oracle for DROT.  TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The solver library and its Python binding
never do; the two share no code, headers or constants.  Inputs come from the
``workloads`` package (seeded generators with none of the method's
arithmetic).

Contents
--------
* :func:`drot_solve` / :func:`drot_run` - Algorithm 1 (Sec. 3.1) in plain FP64
  C (``drot_oracle.c``), with the stopping test of Sec. 3.1.
* :func:`dr3_run` - the three-variable Douglas-Rachford form
  (Sec. 3.1, eq. drot:general:form) written directly in NumPy with the
  projection of Lemma 1 (Sec. 3); an independent formulation used to pin
  the single-array Algorithm 1.
* :func:`project_marginals` - Lemma 1's closed-form projection onto
  {X : X e = p, X^T f = q}.
* :func:`lp_optimum`, :func:`permutation_optimum`, :func:`nw_corner_1d` -
  exact optima from an LP library, brute force and the 1-D closed form.
* :func:`lp_primal_dual`, :func:`fixed_point_from_pair` - an exact
  primal-dual optimum from the LP library and the DR fixed point it defines
  (Lemma opt-rel, Appendix A.2), the Y* of Theorem 1 (Sec. 3.2).
* :func:`plan_stats` - the Sec. 3.1 stopping quantities of any (X, mu, nu).
"""

from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drot_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIB_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

# Indices into the stats vector returned by the C oracle.
PRIMAL, DUAL, GAP, RES_L1, RES_L2, DUAL_RES_PREV, BETA = range(7)
NSTATS = 7

STATUS_CONVERGED = 0
STATUS_MAX_ITER = 1
STATUS_NONFINITE = 2


def _compile(out: str, extra: list, force: bool) -> str:
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle twice: plain -O2 with IEEE semantics on one thread (the parity
    reference), and the same source with -fopenmp (its row loops split across the host's
    cores; used only to time the oracle on all cores)."""
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _compile(_LIB, [], force)


def threads(all_cores: bool = True) -> int:
    """Threads an iteration of the oracle uses: 1 for the parity build; the OpenMP runtime's
    thread count (OMP_NUM_THREADS, else every host core) for the all-cores build."""
    return int(_load(all_cores).oracle_threads())


def _load(all_cores: bool = False):
    key = bool(all_cores)
    with _lock:
        if key not in _libs:
            build()
            lib = ctypes.CDLL(_LIB_OMP if key else _LIB)
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_solve.restype = ctypes.c_int
            lib.oracle_solve.argtypes = [i64, i64, d, d, d, ctypes.c_double, ctypes.c_double, i64,
                                         ctypes.c_int, ctypes.c_int, d, d, d, d,
                                         ctypes.POINTER(i64), d]
            lib.oracle_iterate.restype = None
            lib.oracle_iterate.argtypes = [i64, i64, d, d, d, ctypes.c_double, d, d, d, d, d, d, d, d]
            lib.oracle_init.restype = None
            lib.oracle_init.argtypes = [i64, i64, d, d, d, d, d, d, d, d]
            lib.oracle_set_mutation.restype = None
            lib.oracle_set_mutation.argtypes = [ctypes.c_int]
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_threads.argtypes = []
            _libs[key] = lib
    return _libs[key]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_mutation(k: int) -> None:
    """Plant mistake number k (0 = none) in the C oracle; used only by pin tests."""
    _load().oracle_set_mutation(int(k))


def drot_solve(C, p, q, rho, tol, max_iter, X0=None, mu0=None, nu0=None,
               stop_on_dual_residual=False, history=False, stop_rule=None, all_cores=False):
    """Run Algorithm 1 from X0 = p q^T (or from a warm start) until the stop rule.

    ``stop_rule`` is a bitmask (1 gap, 2 l1 residual, 4 r_dual; default 3, or 7 with
    ``stop_on_dual_residual``).  ``all_cores`` runs the OpenMP build of the same source (every
    X_ij, r_i, s_j formed as in the single-thread build; only the three scalar totals are summed
    in another order).  Returns a dict with X, mu, nu (FP64), iters, status, stats (dict) and,
    when ``history`` is true, the per-iteration stats as an (iters, 7) array.
    """
    lib = _load(all_cores)
    C = np.ascontiguousarray(np.asarray(C, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    m, n = C.shape
    warm = X0 is not None
    X = np.ascontiguousarray(np.asarray(X0, dtype=np.float64)).copy() if warm else np.zeros((m, n))
    mu = np.ascontiguousarray(np.asarray(mu0, dtype=np.float64)).copy() if warm and mu0 is not None else np.zeros(m)
    nu = np.ascontiguousarray(np.asarray(nu0, dtype=np.float64)).copy() if warm and nu0 is not None else np.zeros(n)
    stats = np.zeros(NSTATS)
    iters = ctypes.c_int64(0)
    hist = np.zeros((max(int(max_iter), 1), NSTATS)) if history else None
    rc = lib.oracle_solve(m, n, _ptr(C), _ptr(p), _ptr(q), float(rho), float(tol), int(max_iter),
                          int(stop_rule if stop_rule is not None else (7 if stop_on_dual_residual else 3)), int(warm), _ptr(X), _ptr(mu), _ptr(nu),
                          _ptr(stats), ctypes.byref(iters),
                          _ptr(hist) if hist is not None else ctypes.POINTER(ctypes.c_double)())
    if rc < 0:
        raise ValueError("oracle_solve rejected its arguments")
    out = dict(X=X, mu=mu, nu=nu, iters=int(iters.value), status=int(rc),
               stats=dict(primal=stats[PRIMAL], dual=stats[DUAL], gap=stats[GAP], res_l1=stats[RES_L1],
                          res_l2=stats[RES_L2], dual_res_prev=stats[DUAL_RES_PREV], beta=stats[BETA]))
    if hist is not None:
        out["history"] = hist[: int(iters.value)].copy()
    return out


def drot_run(C, p, q, rho, iters, X0=None, mu0=None, nu0=None):
    """Exactly ``iters`` iterations of Algorithm 1 (no early stop)."""
    return drot_solve(C, p, q, rho, tol=-1.0, max_iter=iters, X0=X0, mu0=mu0, nu0=nu0, history=True)


class StepState:
    """Explicit Algorithm 1 state (X, phi, psi, a, b, alpha) stepped by the C oracle
    (``all_cores``: the OpenMP build of the same source, for timing on every host core)."""

    def __init__(self, C, p, q, rho, X0, phi0, psi0, all_cores: bool = False):
        self.lib = _load(all_cores)
        self.C = np.ascontiguousarray(np.asarray(C, dtype=np.float64))
        self.p = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
        self.q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        self.m, self.n = self.C.shape
        self.rho = float(rho)
        self.X = np.ascontiguousarray(np.asarray(X0, dtype=np.float64)).copy()
        self.phi = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64)).copy()
        self.psi = np.ascontiguousarray(np.asarray(psi0, dtype=np.float64)).copy()
        self.a = np.zeros(self.m)
        self.b = np.zeros(self.n)
        alpha = ctypes.c_double(0.0)
        self.lib.oracle_init(self.m, self.n, _ptr(self.p), _ptr(self.q), _ptr(self.X), _ptr(self.phi),
                             _ptr(self.psi), _ptr(self.a), _ptr(self.b), ctypes.byref(alpha))
        self.alpha = alpha.value
        self._work = np.zeros(self.m + self.n)

    def step(self):
        stats = np.zeros(NSTATS)
        alpha = ctypes.c_double(self.alpha)
        self.lib.oracle_iterate(self.m, self.n, _ptr(self.C), _ptr(self.p), _ptr(self.q), self.rho,
                                _ptr(self.X), _ptr(self.phi), _ptr(self.psi), _ptr(self.a), _ptr(self.b),
                                ctypes.byref(alpha), _ptr(stats), _ptr(self._work))
        self.alpha = alpha.value
        return stats

    @property
    def Y(self):
        """The Douglas-Rachford variable Y_k = X_k + phi_k e^T + f psi_k^T (eq. alg:drot:y:update)."""
        return self.X + self.phi[:, None] + self.psi[None, :]


# ---------------------------------------------------------------------------
# Independent formulations and exact optima (NumPy / SciPy)
# ---------------------------------------------------------------------------

def project_marginals(X, p, q):
    """Lemma 1 (Sec. 3): projection onto {X : X e = p, X^T f = q}.

    P(X) = X - (1/n)((X e - p) e^T - gamma f e^T) - (1/m)(f (X^T f - q)^T - gamma f e^T),
    gamma = f^T (X e - p) / (m + n).
    """
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    e = np.ones(n)
    f = np.ones(m)
    row_res = X @ e - p
    col_res = X.T @ f - q
    gamma = f @ row_res / (m + n)
    return (X - (np.outer(row_res, e) - gamma * np.outer(f, e)) / n
            - (np.outer(f, col_res) - gamma * np.outer(f, e)) / m)


def dr3_run(C, p, q, rho, iters, Y0):
    """Three-variable DR of eq. drot:general:form (Sec. 3.1), literally:

    X_{k+1} = [Y_k - rho C]_+,  Z_{k+1} = P(2 X_{k+1} - Y_k),  Y_{k+1} = Y_k + Z_{k+1} - X_{k+1}.
    Returns the lists of X_k, Z_k and Y_k for k = 1..iters (Y also k = 0).
    """
    C = np.asarray(C, dtype=np.float64)
    Y = np.asarray(Y0, dtype=np.float64).copy()
    Xs, Zs, Ys = [], [], [Y.copy()]
    for _ in range(iters):
        X = np.maximum(Y - rho * C, 0.0)
        Z = project_marginals(2.0 * X - Y, p, q)
        Y = Y + Z - X
        Xs.append(X)
        Zs.append(Z)
        Ys.append(Y.copy())
    return Xs, Zs, Ys


def lp_optimum(C, p, q):
    """Exact optimal value (and plan) of eq. ot:dist via SciPy's HiGHS LP solver."""
    from scipy.optimize import linprog

    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    rows = np.zeros((m, m * n))
    for i in range(m):
        rows[i, i * n:(i + 1) * n] = 1.0
    cols = np.zeros((n, m * n))
    for j in range(n):
        cols[j, j::n] = 1.0
    A = np.vstack([rows, cols])
    b = np.concatenate([p, q])
    res = linprog(C.ravel(), A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(f"HiGHS failed: {res.message}")
    return float(res.fun), res.x.reshape(m, n)


def lp_primal_dual(C, p, q):
    """Exact primal-dual optimum (X*, mu*, nu*, value) of eq. ot:dist via HiGHS.

    mu*, nu* are the multipliers of the row and column constraints (HiGHS reports the
    sensitivity of the optimal value to the right-hand side), i.e. a solution of the dual
    max p^T mu + q^T nu s.t. mu_i + nu_j <= C_ij.  Callers check dual feasibility and strong
    duality themselves before using them.
    """
    from scipy.optimize import linprog

    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    rows = np.zeros((m, m * n))
    for i in range(m):
        rows[i, i * n:(i + 1) * n] = 1.0
    cols = np.zeros((n, m * n))
    for j in range(n):
        cols[j, j::n] = 1.0
    res = linprog(C.ravel(), A_eq=np.vstack([rows, cols]), b_eq=np.concatenate([p, q]), bounds=(0, None),
                  method="highs")
    if res.status != 0:
        raise RuntimeError(f"HiGHS failed: {res.message}")
    y = np.asarray(res.eqlin.marginals, dtype=np.float64)
    return res.x.reshape(m, n), y[:m].copy(), y[m:].copy(), float(res.fun)


def fixed_point_from_pair(X, mu, nu, rho):
    """Lemma opt-rel (Appendix A.2): a primal-dual optimum (X*, mu*, nu*) gives the fixed
    point Y* = X* + rho (mu* e^T + f nu*^T) of the DR operator T of eq. dr:operator:T."""
    return np.asarray(X, dtype=np.float64) + rho * (np.asarray(mu)[:, None] + np.asarray(nu)[None, :])


def permutation_optimum(C):
    """min over permutations sigma of (1/n) sum_i C[i, sigma(i)] (uniform marginals, m = n)."""
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    best = np.inf
    for perm in itertools.permutations(range(n)):
        best = min(best, C[np.arange(n), perm].sum())
    return best / n


def nw_corner_1d(x, y, p, q):
    """Optimal plan for 1-D points under a convex cost (the monotone rearrangement).

    Sort both supports, then fill the plan north-west-corner style: the mass
    of the i-th smallest source goes to the smallest targets with capacity
    left.  Returns the plan in the original index order.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ix = np.argsort(x, kind="stable")
    iy = np.argsort(y, kind="stable")
    a = np.asarray(p, dtype=np.float64)[ix].copy()
    b = np.asarray(q, dtype=np.float64)[iy].copy()
    P = np.zeros((len(x), len(y)))
    i = j = 0
    while i < len(a) and j < len(b):
        t = min(a[i], b[j])
        P[ix[i], iy[j]] += t
        a[i] -= t
        b[j] -= t
        if a[i] <= b[j]:
            i += 1
        else:
            j += 1
    return P


def plan_stats(C, p, q, X, mu, nu):
    """Sec. 3.1 stopping quantities of a primal-dual pair, in FP64."""
    C = np.asarray(C, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    r = X.sum(axis=1) - p
    s = X.sum(axis=0) - q
    primal = float((C * X).sum())
    dual = float(p @ mu + q @ nu)
    viol = np.maximum(mu[:, None] + nu[None, :] - C, 0.0)
    return dict(primal=primal, dual=dual, gap=abs(primal - dual),
                res_l1=float(np.abs(r).sum() + np.abs(s).sum()),
                res_l2=float(np.sqrt((r * r).sum() + (s * s).sum())),
                dual_res=float(np.sqrt((viol * viol).sum())),
                nnz=int((X > 0).sum()))
