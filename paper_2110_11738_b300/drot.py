"""Python binding of the C ABI in include/drot.h (argument marshalling only).

Every step of a solve runs in the CUDA library ``lib/libdrot_b300.so``; this
module converts torch tensors (or NumPy arrays, for the host-buffer path) to
pointers and sizes and returns the C result struct as a dict.  There is no
fallback: if the library is missing or no GPU is present the calls raise.

The entry points keep the C names: ``drot_create``, ``drot_solve``,
``drot_solve_batched``, ``drot_destroy``; :class:`Solver` wraps a handle.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

# drot_status values (include/drot.h)
DROT_OK = 0
DROT_ERR_INVALID_ARG = 1
DROT_ERR_MARGINALS = 2
DROT_ERR_OOM = 3
DROT_ERR_CUDA = 4
DROT_NOT_CONVERGED = 5
DROT_ERR_TIMEOUT = 6
DROT_ERR_NONFINITE = 7
DROT_ERR_TOO_LARGE = 8

STATUS_NAMES = {
    DROT_OK: "DROT_OK", DROT_ERR_INVALID_ARG: "DROT_ERR_INVALID_ARG", DROT_ERR_MARGINALS: "DROT_ERR_MARGINALS",
    DROT_ERR_OOM: "DROT_ERR_OOM", DROT_ERR_CUDA: "DROT_ERR_CUDA", DROT_NOT_CONVERGED: "DROT_NOT_CONVERGED",
    DROT_ERR_TIMEOUT: "DROT_ERR_TIMEOUT", DROT_ERR_NONFINITE: "DROT_ERR_NONFINITE",
    DROT_ERR_TOO_LARGE: "DROT_ERR_TOO_LARGE",
}

# Every symbol include/drot.h declares.
EXPORTED = ("drot_config_default", "drot_create", "drot_solve", "drot_solve_f64", "drot_solve_batched", "drot_destroy",
            "drot_get_profile", "drot_reset_profile", "drot_status_string", "drot_last_error",
            "drot_solve_static", "drot_mlp_create", "drot_mlp_destroy", "drot_mlp_set_params",
            "drot_mlp_get_params", "drot_mlp_features", "drot_mlp_forward", "drot_mlp_train_step",
            "drot_mlp_warm_start")

MLP_FEATURES = 64
MLP_WIDTH = 256
MLP_PARAMS = 256 * 64 + 256 + 2 * (256 * 256 + 256) + 256 + 1


class DrotConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("stop_rule", ctypes.c_int),
                ("rho0", ctypes.c_double), ("graph_iters", ctypes.c_int), ("tile_k", ctypes.c_int),
                ("grid_ctas", ctypes.c_int), ("profile", ctypes.c_int), ("step_variant", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("autotune", ctypes.c_int), ("persistent", ctypes.c_int),
                ("c_skip", ctypes.c_int), ("cluster", ctypes.c_int), ("trace", ctypes.c_void_p),
                ("trace_len", ctypes.c_int64), ("wait_limit", ctypes.c_int64), ("serpentine", ctypes.c_int),
                ("batch_narrow", ctypes.c_int)]


class DrotResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("primal_obj", ctypes.c_double), ("dual_obj", ctypes.c_double),
                ("gap", ctypes.c_double), ("res_l1", ctypes.c_double), ("res_l2", ctypes.c_double),
                ("dual_res", ctypes.c_double), ("nnz", ctypes.c_int64), ("status", ctypes.c_int32),
                ("seconds", ctypes.c_double)]


class DrotProblem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("C", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("q", ctypes.c_void_p), ("X", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("nu", ctypes.c_void_p), ("rho", ctypes.c_double)]


class DrotProfile(ctypes.Structure):
    _fields_ = [("step_ms_total", ctypes.c_double), ("step_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("tile_k", ctypes.c_int32), ("grid_ctas", ctypes.c_int32), ("col_tiles", ctypes.c_int32),
                ("graph_iters", ctypes.c_int32), ("step_variant", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("finish_ms_total", ctypes.c_double), ("iter_ms_total", ctypes.c_double)]


class DrotError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the solver library (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"solver library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.drot_config_default.restype = None
    lib.drot_config_default.argtypes = [ctypes.POINTER(DrotConfig)]
    lib.drot_create.restype = ctypes.c_int
    lib.drot_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(DrotConfig)]
    lib.drot_destroy.restype = ctypes.c_int
    lib.drot_destroy.argtypes = [vp]
    lib.drot_solve.restype = ctypes.c_int
    lib.drot_solve.argtypes = [vp, i64, i64, vp, i64, vp, vp, ctypes.c_double, ctypes.c_double, i64, vp, vp, vp,
                               ctypes.c_int, ctypes.POINTER(DrotResult)]
    lib.drot_solve_f64.restype = ctypes.c_int
    lib.drot_solve_f64.argtypes = list(lib.drot_solve.argtypes)
    lib.drot_solve_batched.restype = ctypes.c_int
    lib.drot_solve_batched.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(DrotProblem), ctypes.c_double, i64,
                                       ctypes.c_int, ctypes.POINTER(DrotResult)]
    lib.drot_get_profile.restype = ctypes.c_int
    lib.drot_get_profile.argtypes = [vp, ctypes.POINTER(DrotProfile)]
    lib.drot_reset_profile.restype = ctypes.c_int
    lib.drot_reset_profile.argtypes = [vp]
    lib.drot_status_string.restype = ctypes.c_char_p
    lib.drot_status_string.argtypes = [ctypes.c_int]
    lib.drot_last_error.restype = ctypes.c_char_p
    lib.drot_last_error.argtypes = [vp]
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.drot_mlp_create.restype = ctypes.c_int
    lib.drot_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.drot_mlp_destroy.restype = ctypes.c_int
    lib.drot_mlp_destroy.argtypes = [vp]
    lib.drot_mlp_set_params.restype = ctypes.c_int
    lib.drot_mlp_set_params.argtypes = [vp, f32p]
    lib.drot_mlp_get_params.restype = ctypes.c_int
    lib.drot_mlp_get_params.argtypes = [vp, f32p]
    lib.drot_mlp_features.restype = ctypes.c_int
    lib.drot_mlp_features.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, i64]
    lib.drot_mlp_forward.restype = ctypes.c_int
    lib.drot_mlp_forward.argtypes = [vp, i64, vp, vp]
    lib.drot_mlp_train_step.restype = ctypes.c_int
    lib.drot_mlp_train_step.argtypes = [vp, i64, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_float, ctypes.c_int,
                                        f32p, f32p]
    lib.drot_mlp_warm_start.restype = ctypes.c_int
    lib.drot_mlp_warm_start.argtypes = [vp, i64, i64, vp, vp, vp, vp, ctypes.c_double, vp, i64, vp, vp, vp]
    lib.drot_solve_static.restype = ctypes.c_int
    lib.drot_solve_static.argtypes = [i64, i64, vp, i64, vp, vp, ctypes.c_double, ctypes.c_double, i64, vp, vp, vp,
                                      ctypes.c_int, vp, ctypes.POINTER(DrotResult)]
    _lib = lib
    return lib


def _result_dict(r: DrotResult) -> dict:
    return dict(iters=int(r.iters), primal_obj=r.primal_obj, dual_obj=r.dual_obj, gap=r.gap, res_l1=r.res_l1,
                res_l2=r.res_l2, dual_res=r.dual_res, nnz=int(r.nnz), status=int(r.status),
                status_name=STATUS_NAMES.get(int(r.status), str(r.status)), seconds=r.seconds)


# ---------------------------------------------------------------- C-named entry points

STOP_GAP = 1
STOP_RES_L1 = 2
STOP_DUAL_RES = 4


def drot_create(device: int = 0, stream: Optional[int] = None, stop_rule: int = STOP_GAP | STOP_RES_L1,
                rho0: float = 2.0, graph_iters: int = 0, tile_k: int = 0, grid_ctas: int = 0,
                profile: bool = False, step_variant: int = 0, deterministic: bool = False,
                autotune: bool = False, persistent: bool = False, c_skip: bool = False,
                cluster: int = 0, trace=None, wait_limit: int = 0, serpentine: int = 0,
                batch_narrow: int = 0) -> int:
    """Create a solver handle; returns the opaque handle as an int.  ``trace``: optional float64
    CUDA tensor of 2 * L entries that receives <C, X_k> and the l1 residual of iterations 1 .. L
    of every solve (the caller keeps it alive while the handle is used).  ``serpentine``: 1 or 0
    (default) alternates the direction of the fused-step passes so that each starts on what the
    previous one left in L2; -1 runs every pass forwards.  ``cluster``: 0 chooses the on-chip
    schemes automatically (one cluster for small problems, grid-resident from 2e6 entries where the
    rows fit), 1 always streams, 2 requires the cluster, 3 the grid-resident solve.  ``batch_narrow`` (batched solves): 1
    always, -1 never, 0 (default) automatically sends tiles of at most 256 columns to the kernel
    that packs rows."""
    lib = load()
    cfg = DrotConfig()
    lib.drot_config_default(ctypes.byref(cfg))
    cfg.device = int(device)
    cfg.stream = int(stream) if stream else None
    cfg.stop_rule = int(stop_rule)
    cfg.rho0 = float(rho0)
    cfg.graph_iters = int(graph_iters)
    cfg.tile_k = int(tile_k)
    cfg.grid_ctas = int(grid_ctas)
    cfg.profile = int(bool(profile))
    cfg.step_variant = int(step_variant)
    cfg.deterministic = int(bool(deterministic))
    cfg.autotune = int(bool(autotune))
    cfg.persistent = int(bool(persistent))
    cfg.c_skip = int(bool(c_skip))
    cfg.cluster = int(cluster)
    cfg.wait_limit = int(wait_limit)
    cfg.serpentine = int(serpentine)
    cfg.batch_narrow = int(batch_narrow)
    if trace is not None:
        cfg.trace = _ptr(trace)
        cfg.trace_len = int(trace.numel()) // 2
    h = ctypes.c_void_p()
    st = lib.drot_create(ctypes.byref(h), ctypes.byref(cfg))
    if st != DROT_OK:
        raise DrotError(st, lib.drot_status_string(st).decode())
    return h.value


def drot_destroy(handle: int) -> None:
    load().drot_destroy(ctypes.c_void_p(handle))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _is_f64(x) -> bool:
    return str(x.dtype) in ("float64", "torch.float64")


def _ld_of(C) -> int:
    if isinstance(C, np.ndarray):
        return C.strides[0] // C.itemsize
    return C.stride(0)


def drot_solve(handle: int, C, p, q, rho: float = 0.0, tol: float = 1e-6, max_iter: int = 1_000_000,
               X=None, mu=None, nu=None, warm: bool = False, m: Optional[int] = None,
               n: Optional[int] = None, check: bool = True) -> dict:
    """Call drot_solve on torch CUDA tensors (device path) or NumPy arrays (host path).

    C and X: float32, shape (m, ld) or a row-strided (m, n) view, unit column
    stride; p, q, mu, nu: float64.  X, mu, nu are written in place.  ``n``
    defaults to C.shape[1].  float64 C and X call drot_solve_f64 instead.
    """
    lib = load()
    m = int(C.shape[0]) if m is None else int(m)
    n = int(C.shape[1]) if n is None else int(n)
    ld = _ld_of(C)
    if X is not None and _ld_of(X) != ld:
        raise ValueError("C and X must share the row pitch")
    res = DrotResult()
    entry = lib.drot_solve_f64 if _is_f64(C) else lib.drot_solve
    if X is not None and _is_f64(X) != _is_f64(C):
        raise ValueError("C and X must have the same dtype")
    st = entry(ctypes.c_void_p(handle), m, n, ctypes.c_void_p(_ptr(C)), ld, ctypes.c_void_p(_ptr(p)),
                        ctypes.c_void_p(_ptr(q)), float(rho), float(tol), int(max_iter),
                        ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(mu)), ctypes.c_void_p(_ptr(nu)),
                        int(bool(warm)), ctypes.byref(res))
    out = _result_dict(res)
    out["status"] = int(st)
    out["status_name"] = STATUS_NAMES.get(int(st), str(st))
    if check and st not in (DROT_OK, DROT_NOT_CONVERGED):
        raise DrotError(st, lib.drot_last_error(ctypes.c_void_p(handle)).decode())
    return out


def drot_solve_batched(handle: int, problems: Sequence[dict], tol: float = 1e-6, max_iter: int = 1_000_000,
                       warm: bool = False, check: bool = True) -> list:
    """Call drot_solve_batched; each problem is a dict with C, p, q, X, mu, nu (and optional rho, n)."""
    lib = load()
    B = len(problems)
    arr = (DrotProblem * max(B, 1))()
    for b, pr in enumerate(problems):
        C = pr["C"]
        arr[b].m = int(C.shape[0])
        arr[b].n = int(pr.get("n", C.shape[1]))
        arr[b].ld = _ld_of(C)
        arr[b].C = _ptr(C)
        arr[b].p = _ptr(pr["p"])
        arr[b].q = _ptr(pr["q"])
        arr[b].X = _ptr(pr["X"])
        arr[b].mu = _ptr(pr["mu"])
        arr[b].nu = _ptr(pr["nu"])
        arr[b].rho = float(pr.get("rho", 0.0))
    res = (DrotResult * max(B, 1))()
    st = lib.drot_solve_batched(ctypes.c_void_p(handle), B, arr, float(tol), int(max_iter), int(bool(warm)), res)
    if check and st not in (DROT_OK, DROT_NOT_CONVERGED):
        raise DrotError(st, lib.drot_last_error(ctypes.c_void_p(handle)).decode())
    return [_result_dict(res[b]) for b in range(B)]


def drot_solve_static(C, p, q, rho: float = 0.0, tol: float = 1e-6, max_iter: int = 1_000_000, X=None, mu=None,
                      nu=None, warm: bool = False, n: Optional[int] = None, stream: Optional[int] = None) -> dict:
    """Call drot_solve_static: the handle-free solve that allocates no device memory.

    For callers that cannot allocate GPU memory when they solve (see include/drot.h).  All
    buffers must be CUDA tensors on the current device; X, mu, nu are written in place.
    Returns the result dict; "status" holds the drot_status (DROT_ERR_TOO_LARGE when the
    problem does not fit the library's fixed 16 MiB workspace).
    """
    lib = load()
    m = int(C.shape[0])
    n = int(C.shape[1]) if n is None else int(n)
    ld = _ld_of(C)
    if X is not None and _ld_of(X) != ld:
        raise ValueError("C and X must share the row pitch")
    res = DrotResult()
    st = lib.drot_solve_static(m, n, ctypes.c_void_p(_ptr(C)), ld, ctypes.c_void_p(_ptr(p)),
                               ctypes.c_void_p(_ptr(q)), float(rho), float(tol), int(max_iter),
                               ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(mu)), ctypes.c_void_p(_ptr(nu)),
                               int(bool(warm)), ctypes.c_void_p(stream or 0), ctypes.byref(res))
    out = _result_dict(res)
    out["status"] = int(st)
    out["status_name"] = STATUS_NAMES.get(int(st), str(st))
    return out


def drot_get_profile(handle: int) -> dict:
    lib = load()
    pr = DrotProfile()
    st = lib.drot_get_profile(ctypes.c_void_p(handle), ctypes.byref(pr))
    if st != DROT_OK:
        raise DrotError(st, "drot_get_profile")
    return {name: getattr(pr, name) for name, _ in DrotProfile._fields_}


def drot_reset_profile(handle: int) -> None:
    load().drot_reset_profile(ctypes.c_void_p(handle))


# ---------------------------------------------------------------- convenience wrapper

class Solver:
    """A solver handle bound to one GPU.  Use as a context manager or call close()."""

    def __init__(self, device: int = 0, **cfg):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the DROT solver needs a CUDA device")
        self.device = int(device)
        self._trace = cfg.get("trace")  # the handle writes into it: keep it alive
        self.handle = drot_create(device=self.device, **cfg)

    def close(self):
        if self.handle:
            drot_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, C, p, q, rho: float = 0.0, tol: float = 1e-6, max_iter: int = 1_000_000, X=None, mu=None,
              nu=None, warm: bool = False, n: Optional[int] = None, check: bool = True) -> dict:
        """Solve on device tensors; allocates X, mu, nu when not given.  Returns the result dict
        with the output tensors under "X", "mu", "nu"."""
        import torch

        dev = torch.device("cuda", self.device)
        m = int(C.shape[0])
        n = int(C.shape[1]) if n is None else int(n)
        if X is None:
            ld = _ld_of(C)
            X = torch.empty((m, ld), dtype=C.dtype, device=dev)[:, :n]
        if mu is None:
            mu = torch.zeros(m, dtype=torch.float64, device=dev)
        if nu is None:
            nu = torch.zeros(n, dtype=torch.float64, device=dev)
        torch.cuda.current_stream(dev).synchronize()
        out = drot_solve(self.handle, C, p, q, rho=rho, tol=tol, max_iter=max_iter, X=X, mu=mu, nu=nu, warm=warm,
                         n=n, check=check)
        out.update(X=X, mu=mu, nu=nu)
        return out

    def solve_batched(self, problems, tol: float = 1e-6, max_iter: int = 1_000_000, warm: bool = False,
                      check: bool = True) -> list:
        import torch

        torch.cuda.current_stream(self.device).synchronize()
        return drot_solve_batched(self.handle, problems, tol=tol, max_iter=max_iter, warm=warm, check=check)

    def profile(self) -> dict:
        return drot_get_profile(self.handle)

    def reset_profile(self) -> None:
        drot_reset_profile(self.handle)


def padded_matrix(A, ld: Optional[int] = None, device=None, dtype=None):
    """Copy a (m, n) matrix into a (m, ld) float32 (or ``dtype``) tensor with 16-byte aligned rows;
    returns the (m, n) view (row stride ld) that drot_solve (drot_solve_f64 for float64) accepts."""
    import torch

    dtype = torch.float32 if dtype is None else dtype
    A = torch.as_tensor(A, dtype=dtype)
    m, n = A.shape
    vec = 16 // A.element_size()
    ld = (n + vec - 1) // vec * vec if ld is None else int(ld)
    buf = torch.zeros((m, ld), dtype=dtype, device=device if device is not None else A.device)
    buf[:, :n] = A.to(buf.device)
    return buf[:, :n]


# ---------------------------------------------------------------- learned warm start

class Mlp:
    """The warm-start network (drot_mlp_* in include/drot.h) on one GPU.

    Feature matrices are torch.bfloat16 CUDA tensors of shape (rows, MLP_FEATURES) with
    rows a multiple of 64; targets, weights are float32, seg int32 (-1 marks padding rows).
    """

    def __init__(self, device: int = 0, params: Optional[np.ndarray] = None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the warm-start network needs a CUDA device")
        self.lib = load()
        self.device = int(device)
        h = ctypes.c_void_p()
        st = self.lib.drot_mlp_create(ctypes.byref(h), self.device)
        if st != DROT_OK:
            raise DrotError(st, "drot_mlp_create")
        self.handle = h.value
        if params is not None:
            self.set_params(params)

    def close(self):
        if self.handle:
            self.lib.drot_mlp_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != DROT_OK:
            raise DrotError(st, what)

    def set_params(self, params: np.ndarray) -> None:
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        assert a.size == MLP_PARAMS
        self._check(self.lib.drot_mlp_set_params(ctypes.c_void_p(self.handle),
                                                 a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "set_params")

    def get_params(self) -> np.ndarray:
        a = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(self.lib.drot_mlp_get_params(ctypes.c_void_p(self.handle),
                                                 a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "get_params")
        return a

    def features(self, xs, yt, p, q, feat, row0: int = 0) -> None:
        m, n = int(xs.shape[0]), int(yt.shape[0])
        self._check(self.lib.drot_mlp_features(ctypes.c_void_p(self.handle), m, n, ctypes.c_void_p(_ptr(xs)),
                                               ctypes.c_void_p(_ptr(yt)), ctypes.c_void_p(_ptr(p)),
                                               ctypes.c_void_p(_ptr(q)), ctypes.c_void_p(_ptr(feat)), int(row0)),
                    "features")

    def forward(self, feat, out) -> None:
        self._check(self.lib.drot_mlp_forward(ctypes.c_void_p(self.handle), int(feat.shape[0]),
                                              ctypes.c_void_p(_ptr(feat)), ctypes.c_void_p(_ptr(out))), "forward")

    def train_step(self, feat, target, weight, seg, nseg: int, lr: float, update: bool = True,
                   want_grad: bool = False):
        loss = ctypes.c_float(0.0)
        grad = np.zeros(MLP_PARAMS, dtype=np.float32) if want_grad else None
        st = self.lib.drot_mlp_train_step(ctypes.c_void_p(self.handle), int(feat.shape[0]),
                                          ctypes.c_void_p(_ptr(feat)), ctypes.c_void_p(_ptr(target)),
                                          ctypes.c_void_p(_ptr(weight)), ctypes.c_void_p(_ptr(seg)), int(nseg),
                                          float(lr), int(bool(update)), ctypes.byref(loss),
                                          grad.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
                                          if grad is not None else None)
        self._check(st, "train_step")
        return (loss.value, grad) if want_grad else loss.value

    def warm_start(self, xs, yt, p, q, cost_scale: float, C, X, mu, nu) -> None:
        m, n = int(xs.shape[0]), int(yt.shape[0])
        st = self.lib.drot_mlp_warm_start(ctypes.c_void_p(self.handle), m, n, ctypes.c_void_p(_ptr(xs)),
                                          ctypes.c_void_p(_ptr(yt)), ctypes.c_void_p(_ptr(p)),
                                          ctypes.c_void_p(_ptr(q)), float(cost_scale), ctypes.c_void_p(_ptr(C)),
                                          _ld_of(C), ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(mu)),
                                          ctypes.c_void_p(_ptr(nu)))
        self._check(st, "warm_start")
