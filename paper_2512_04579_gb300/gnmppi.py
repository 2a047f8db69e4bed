"""Thin ctypes binding of the GN-MPPI C ABI (``include/gnmppi.h``).

Argument marshalling only: every step of the solver runs in ``libgnmppi.so``.
The functions carry the C names; arrays are numpy arrays (host memory,
``mem=MEM_HOST``) or CUDA torch tensors / raw device pointers (``mem=MEM_DEVICE``).
Loading fails loudly when the library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgnmppi.so")

OK, E_ARG, E_CUDA, E_NOT_PD, E_NONFINITE, E_TIMEOUT, E_NOMEM = 0, -1, -2, -3, -4, -5, -6
DYN_PENDULUM, DYN_CHAIN, DYN_LINEAR, DYN_ROSENBROCK, DYN_RASTRIGIN, DYN_HEAVISIDE = 0, 1, 2, 3, 4, 5
PREC_FP64, PREC_FP32, PREC_BF16 = 0, 1, 2
JAC_LSQ, JAC_SIGMA, JAC_AUTO = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
SAMPLE_RANDOM, SAMPLE_SIGMA = 0, 1
METHOD_GN, METHOD_MPPI = 0, 1

EXPORTS = ["gnmppi_create", "gnmppi_layout", "gnmppi_solve", "gnmppi_solve_masked", "gnmppi_step", "gnmppi_cost", "gnmppi_debug_read",
           "gnmppi_phase_times", "gnmppi_phase_name", "gnmppi_softmin_noalloc", "gnmppi_launch_count",
           "gnmppi_destroy", "gnmppi_last_error", "gnmppi_status_string", "gnmppi_version", "gnmppi_mlp_create",
           "gnmppi_mlp_num_params", "gnmppi_mlp_set_params", "gnmppi_mlp_get_params", "gnmppi_mlp_set_normalization",
           "gnmppi_mlp_forward", "gnmppi_mlp_loss_grad", "gnmppi_mlp_train_step", "gnmppi_mlp_warm_start",
           "gnmppi_mlp_destroy", "gnmppi_mlp_last_error", "gnmppi_autotune", "gnmppi_tune_set", "gnmppi_solve_async", "gnmppi_solve_wait",
           "gnmppi_tune_report", "gnmppi_debug_inject", "gnmppi_mlp_get_state", "gnmppi_mlp_set_state",
           "gnmppi_check_count"]


class Problem(C.Structure):
    _fields_ = [("dynamics", C.c_int32), ("nx", C.c_int32), ("nu", C.c_int32), ("N", C.c_int32), ("M", C.c_int32),
                ("n_lin", C.c_int32), ("dt", C.c_double), ("params", C.c_double * 8),
                ("lin", C.POINTER(C.c_double)), ("K", C.c_int32), ("iterations", C.c_int32), ("L", C.c_int32),
                ("precision", C.c_int32), ("jac_mode", C.c_int32), ("antithetic", C.c_int32),
                ("monotone", C.c_int32), ("ir_steps", C.c_int32), ("lam", C.c_double), ("sigma0", C.c_double),
                ("beta", C.c_double), ("gamma", C.c_double), ("tau", C.c_double), ("seed", C.c_uint64),
                ("sampling", C.c_int32), ("method", C.c_int32), ("first_instance", C.c_int32), ("pad0", C.c_int32)]


class InstanceShape(C.Structure):
    _fields_ = [("N", C.c_int32), ("M", C.c_int32), ("K", C.c_int32), ("pad", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("C_initial", C.c_double), ("C_prev", C.c_double), ("C_final", C.c_double),
                ("sigma_final", C.c_double),
                ("iterations", C.c_int32), ("status", C.c_int32), ("n_masked", C.c_int32),
                ("chol_retries", C.c_int32)]


class IterReport(C.Structure):
    _fields_ = [("C_nom", C.c_double), ("C_new", C.c_double), ("alpha", C.c_double), ("lambda_used", C.c_double),
                ("c_min", C.c_double), ("sum_w", C.c_double), ("sum_w2", C.c_double), ("ess", C.c_double),
                ("pr_norm", C.c_double), ("step_norm", C.c_double), ("j_star", C.c_int32),
                ("n_masked", C.c_int32), ("jac_mode_used", C.c_int32), ("status", C.c_int32),
                ("chol_retries", C.c_int32), ("pad", C.c_int32)]


_lib = None


def load(path: str | None = None):
    """Load libgnmppi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgnmppi.so not found at {path}; run __graft_entry__.build() first")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.gnmppi_create.argtypes = [C.POINTER(Problem), C.c_int32, C.POINTER(InstanceShape), vp, C.POINTER(vp)]
    L.gnmppi_layout.argtypes = [vp, vp, vp, vp]
    L.gnmppi_solve.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
    L.gnmppi_solve_masked.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp, vp]
    L.gnmppi_solve_masked.restype = C.c_int32
    L.gnmppi_step.argtypes = [vp, C.c_int32, vp, vp, vp, vp, C.c_int32, vp]
    L.gnmppi_cost.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
    L.gnmppi_debug_read.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int64, C.POINTER(C.c_int64)]
    L.gnmppi_phase_times.argtypes = [vp, C.c_int32, vp, C.c_int32, C.POINTER(C.c_int32)]
    L.gnmppi_phase_times.restype = C.c_int32
    L.gnmppi_phase_name.argtypes = [C.c_int32]
    L.gnmppi_phase_name.restype = C.c_char_p
    L.gnmppi_softmin_noalloc.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_double, vp, vp, vp, C.c_char_p,
                                         C.c_int32]
    L.gnmppi_softmin_noalloc.restype = C.c_int32
    L.gnmppi_launch_count.argtypes = [vp]
    L.gnmppi_launch_count.restype = C.c_int64
    L.gnmppi_check_count.argtypes = []
    L.gnmppi_check_count.restype = C.c_int64
    L.gnmppi_destroy.argtypes = [vp]
    L.gnmppi_destroy.restype = None
    L.gnmppi_last_error.argtypes = [vp]
    L.gnmppi_last_error.restype = C.c_char_p
    L.gnmppi_status_string.argtypes = [C.c_int32]
    L.gnmppi_status_string.restype = C.c_char_p
    L.gnmppi_version.restype = C.c_int32
    L.gnmppi_solve_async.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
    L.gnmppi_solve_async.restype = C.c_int32
    L.gnmppi_solve_wait.argtypes = [vp, vp]
    L.gnmppi_solve_wait.restype = C.c_int32
    L.gnmppi_autotune.argtypes = [vp, C.c_int32, vp, vp, vp, vp, C.c_int32]
    L.gnmppi_autotune.restype = C.c_int32
    L.gnmppi_tune_set.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
    L.gnmppi_tune_set.restype = C.c_int32
    L.gnmppi_tune_report.argtypes = [vp, C.c_char_p, C.c_int32]
    L.gnmppi_debug_inject.restype = C.c_int32
    L.gnmppi_debug_inject.argtypes = [vp, C.c_int32, C.c_int32]
    L.gnmppi_tune_report.restype = C.c_int32
    for f in ("gnmppi_create", "gnmppi_layout", "gnmppi_solve", "gnmppi_step", "gnmppi_cost", "gnmppi_debug_read"):
        getattr(L, f).restype = C.c_int32
    L.gnmppi_mlp_create.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int32, vp,
                                    C.POINTER(vp)]
    L.gnmppi_mlp_num_params.argtypes = [vp]
    L.gnmppi_mlp_num_params.restype = C.c_int64
    L.gnmppi_mlp_set_params.argtypes = [vp, C.c_int32, vp, C.c_int64]
    L.gnmppi_mlp_get_params.argtypes = [vp, C.c_int32, vp, C.c_int64]
    L.gnmppi_mlp_set_normalization.argtypes = [vp, vp, vp, C.c_double]
    L.gnmppi_mlp_get_state.argtypes = [vp, C.c_int32, vp, vp, vp, C.c_int64, C.POINTER(C.c_int32)]
    L.gnmppi_mlp_set_state.argtypes = [vp, C.c_int32, vp, vp, vp, C.c_int64, C.c_int32]
    L.gnmppi_mlp_forward.argtypes = [vp, C.c_int32, vp, C.c_int32, vp]
    L.gnmppi_mlp_loss_grad.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, vp, vp]
    L.gnmppi_mlp_train_step.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_double, vp]
    L.gnmppi_mlp_warm_start.argtypes = [vp, C.c_int32, vp, C.c_int32, C.c_double, C.c_double, vp, vp]
    L.gnmppi_mlp_destroy.argtypes = [vp]
    L.gnmppi_mlp_destroy.restype = None
    L.gnmppi_mlp_last_error.argtypes = [vp]
    L.gnmppi_mlp_last_error.restype = C.c_char_p
    for f in ("gnmppi_mlp_create", "gnmppi_mlp_set_params", "gnmppi_mlp_get_params", "gnmppi_mlp_set_normalization",
              "gnmppi_mlp_forward", "gnmppi_mlp_loss_grad", "gnmppi_mlp_train_step", "gnmppi_mlp_warm_start",
              "gnmppi_mlp_get_state", "gnmppi_mlp_set_state"):
        getattr(L, f).restype = C.c_int32
    _lib = L
    return L


class GnmppiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "arrays must be contiguous float64"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous() and str(a.dtype) == "torch.float64", "tensors must be contiguous float64"
        return a.data_ptr()
    return int(a)


def make_problem(dynamics: int, *, N: int, K: int, iterations: int = 20, nx: int = 0, nu: int = 0, M: int = 0,
                 dt: float = 0.0, params=(), lin=None, L: int = 16, precision: int = PREC_FP64,
                 jac_mode: int = JAC_AUTO, antithetic: bool = True, monotone: bool = False, ir_steps: int = 1,
                 lam: float = 1e-3, sigma0: float = 0.5, beta: float = 0.7, gamma: float = 0.5, tau: float = 1.0,
                 seed: int = 0, sampling: int = 0, method: int = 0, first_instance: int = 0) -> Problem:
    p = Problem()
    p.dynamics, p.nx, p.nu, p.N, p.M = dynamics, nx, nu, N, M
    p.dt = dt
    for i, v in enumerate(params):
        p.params[i] = v
    if lin is not None:
        arr = np.ascontiguousarray(lin, dtype=np.float64)
        p._lin_keep = arr
        p.lin = arr.ctypes.data_as(C.POINTER(C.c_double))
        p.n_lin = arr.size
    p.K, p.iterations, p.L = K, iterations, L
    p.precision, p.jac_mode, p.antithetic, p.monotone, p.ir_steps = precision, jac_mode, int(antithetic), \
        int(monotone), ir_steps
    p.lam, p.sigma0, p.beta, p.gamma, p.tau, p.seed = lam, sigma0, beta, gamma, tau, seed
    p.sampling, p.method = sampling, method
    p.first_instance = first_instance
    return p


def pendulum_problem(u_friction: float = 0.0, **kw) -> Problem:
    """Pendulum swing-up: g=9.81, l=1, m=1, b=0.1, RK4 dt=0.05; u_friction > 0
    adds dead-zone friction at the input (Setting V.ii)."""
    kw.setdefault("N", 50)
    kw.setdefault("dt", 0.05)
    kw.setdefault("params", (9.81, 1.0, 1.0, 0.1, u_friction))
    return make_problem(DYN_PENDULUM, nx=2, nu=1, **kw)


def chain_problem(M: int = 10, u_friction: float = 0.0, **kw) -> Problem:
    """Hanging chain: mass 0.1, k=10, k3=1, damping 0.05, gravity 9.81, RK4 dt=0.02;
    u_friction > 0 adds dead-zone friction per force component (Setting V.ii)."""
    kw.setdefault("N", 100)
    kw.setdefault("dt", 0.02)
    kw.setdefault("params", (0.1, 10.0, 1.0, 0.05, 9.81, u_friction))
    return make_problem(DYN_CHAIN, nx=4 * (M - 1), nu=2, M=M, **kw)


def testfun_problem(name: str, **kw) -> Problem:
    """The static test problems of Sec. 5 (N = 1): "rosenbrock", "rastrigin", "heaviside"."""
    dyn = {"rosenbrock": DYN_ROSENBROCK, "rastrigin": DYN_RASTRIGIN, "heaviside": DYN_HEAVISIDE}[name]
    kw.setdefault("N", 1)
    return make_problem(dyn, nx=1, nu=1 if dyn == DYN_HEAVISIDE else 2, **kw)


def linear_problem(A, B, wq, wr, wqN, **kw) -> Problem:
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    lin = np.concatenate([A.ravel(), B.ravel(), np.asarray(wq, float), np.asarray(wr, float),
                          np.asarray(wqN, float)])
    return make_problem(DYN_LINEAR, nx=B.shape[0], nu=B.shape[1], lin=lin, **kw)


# ---------------------------------------------------------------------------
# C entry points under their own names


def gnmppi_version() -> int:
    return int(load().gnmppi_version())


def gnmppi_status_string(st: int) -> str:
    return load().gnmppi_status_string(st).decode()


def gnmppi_last_error(h=None) -> str:
    return load().gnmppi_last_error(h).decode()


def gnmppi_create(problem: Problem, batch: int, shapes=None, stream=None):
    L = load()
    arr = None
    if shapes is not None:
        arr = (InstanceShape * batch)()
        for i, (N, M, K) in enumerate(shapes):
            arr[i].N, arr[i].M, arr[i].K = int(N), int(M), int(K)
    h = C.c_void_p()
    st = L.gnmppi_create(C.byref(problem), batch, arr, stream, C.byref(h))
    if st != OK:
        raise GnmppiError(st, f"gnmppi_create: {gnmppi_last_error(None)}")
    return h


def gnmppi_destroy(h) -> None:
    load().gnmppi_destroy(h)


def gnmppi_layout(h, batch: int):
    x0 = np.zeros(batch + 1, np.int64)
    xr = np.zeros(batch + 1, np.int64)
    U = np.zeros(batch + 1, np.int64)
    st = load().gnmppi_layout(h, x0.ctypes.data, xr.ctypes.data, U.ctypes.data)
    if st != OK:
        raise GnmppiError(st, "gnmppi_layout")
    return x0, xr, U


def _check(h, st, name):
    if st not in (OK, E_NOT_PD, E_NONFINITE):
        raise GnmppiError(st, f"{name}: {gnmppi_last_error(h)}")
    return st


def gnmppi_solve(h, mem, x0, xref, U, sigma=None, batch: int | None = None):
    rep = (Report * batch)() if batch else None
    st = load().gnmppi_solve(h, mem, _ptr(x0), _ptr(xref), _ptr(U), _ptr(sigma), rep)
    _check(h, st, "gnmppi_solve")
    return st, rep


def gnmppi_autotune(h, mem, x0, xref, U, sigma=None, reps: int = 3) -> dict:
    """Pick the handle's launch configuration by timing (see the C header);
    returns the report as a dict."""
    st = load().gnmppi_autotune(h, mem, _ptr(x0), _ptr(xref), _ptr(U), _ptr(sigma), reps)
    _check(h, st, "gnmppi_autotune")
    return gnmppi_tune_report(h)


def gnmppi_tune_set(h, branches: int, solve_nt: int, contract_mt: int = 0):
    st = load().gnmppi_tune_set(h, branches, solve_nt, contract_mt)
    _check(h, st, "gnmppi_tune_set")


INJECT_OFF, INJECT_LSQ_BREAKDOWN, INJECT_NOT_PD, INJECT_TC_TIMEOUT = 0, 1, 2, 3


def gnmppi_debug_inject(h, kind: int, iteration: int = 0):
    st = load().gnmppi_debug_inject(h, kind, iteration)
    _check(h, st, "gnmppi_debug_inject")


def gnmppi_tune_report(h) -> dict:
    import json

    buf = C.create_string_buffer(8192)
    st = load().gnmppi_tune_report(h, buf, len(buf))
    _check(h, st, "gnmppi_tune_report")
    return json.loads(buf.value.decode())


def gnmppi_solve_async(h, mem, x0, xref, U, sigma=None, active=None):
    """Enqueue a solve and return (see gnmppi_solve_wait); keep U alive until then."""
    act = None
    if active is not None:
        act = np.ascontiguousarray(active, dtype=np.int32)
    st = load().gnmppi_solve_async(h, mem, _ptr(x0), _ptr(xref), _ptr(U), _ptr(sigma),
                                   None if act is None else act.ctypes.data)
    _check(h, st, "gnmppi_solve_async")
    return st


def gnmppi_solve_wait(h, batch: int | None = None):
    rep = (Report * batch)() if batch else None
    st = load().gnmppi_solve_wait(h, rep)
    _check(h, st, "gnmppi_solve_wait")
    return st, rep


def gnmppi_solve_masked(h, mem, x0, xref, U, sigma, active, batch: int):
    rep = (Report * batch)()
    act = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
    st = load().gnmppi_solve_masked(h, mem, _ptr(x0), _ptr(xref), _ptr(U), _ptr(sigma),
                                    None if act is None else act.ctypes.data, rep)
    _check(h, st, "gnmppi_solve_masked")
    return st, rep


def gnmppi_step(h, mem, x0, xref, U, sigma, iteration: int, batch: int | None = None):
    rep = (IterReport * batch)() if batch else None
    st = load().gnmppi_step(h, mem, _ptr(x0), _ptr(xref), _ptr(U), _ptr(sigma), iteration, rep)
    _check(h, st, "gnmppi_step")
    return st, rep


def gnmppi_cost(h, mem, x0, xref, U, C_out):
    st = load().gnmppi_cost(h, mem, _ptr(x0), _ptr(xref), _ptr(U), _ptr(C_out))
    _check(h, st, "gnmppi_cost")
    return st


def gnmppi_debug_read(h, what: int, inst: int, count: int) -> np.ndarray:
    out = np.zeros(count)
    w = C.c_int64()
    st = load().gnmppi_debug_read(h, what, inst, out.ctypes.data, count, C.byref(w))
    if st != OK:
        raise GnmppiError(st, f"gnmppi_debug_read: {gnmppi_last_error(h)}")
    return out[: w.value]


def gnmppi_phase_times(h, iteration: int = 0) -> dict:
    ms = np.zeros(16)
    n = C.c_int32()
    st = load().gnmppi_phase_times(h, iteration, ms.ctypes.data, 16, C.byref(n))
    if st != OK:
        raise GnmppiError(st, f"gnmppi_phase_times: {gnmppi_last_error(h)}")
    return {gnmppi_phase_name(i): float(ms[i]) for i in range(n.value)}


def gnmppi_phase_name(i: int):
    v = load().gnmppi_phase_name(i)
    return v.decode() if v else None


def gnmppi_softmin_noalloc(C_dev, W_dev, count: int, n: int, antithetic: bool, tau: float, mppi_dev, stats_dev,
                           stream=None):
    """Softmin weights and MPPI mean perturbation of one sample set; device
    pointers in and out, no device allocation.  Returns (status, error text)."""
    buf = C.create_string_buffer(256)
    st = load().gnmppi_softmin_noalloc(_ptr(C_dev), _ptr(W_dev), count, n, int(antithetic), tau, _ptr(mppi_dev),
                                       _ptr(stats_dev), stream, buf, 256)
    return int(st), buf.value.decode()


def gnmppi_launch_count(h) -> int:
    return int(load().gnmppi_launch_count(h))


DEBUG = {"dR": 0, "W": 1, "C": 2, "e": 3, "PS": 4, "A": 5, "g": 6, "delta": 7, "Cline": 8, "r": 9, "mppi": 10, "S2": 11}


@dataclass
class Solver:
    """Convenience owner of a handle (host numpy arrays)."""

    problem: Problem
    batch: int = 1
    shapes: list | None = None

    def __post_init__(self):
        self.h = gnmppi_create(self.problem, self.batch, self.shapes)
        self.off_x0, self.off_xref, self.off_U = gnmppi_layout(self.h, self.batch)

    def close(self):
        if self.h is not None:
            gnmppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, x0, xref, U0, sigma=None):
        U = np.array(U0, dtype=np.float64, copy=True).ravel()
        st, rep = gnmppi_solve(self.h, MEM_HOST, np.ascontiguousarray(x0, float).ravel(),
                               None if xref is None else np.ascontiguousarray(xref, float).ravel(), U,
                               None if sigma is None else np.ascontiguousarray(sigma, float).ravel(), self.batch)
        return st, U, rep

    def step(self, x0, xref, U, sigma, iteration):
        U = np.array(U, dtype=np.float64, copy=True).ravel()
        st, rep = gnmppi_step(self.h, MEM_HOST, np.ascontiguousarray(x0, float).ravel(),
                              None if xref is None else np.ascontiguousarray(xref, float).ravel(), U,
                              np.ascontiguousarray(sigma, float).ravel(), iteration, self.batch)
        return st, U, rep

    def cost(self, x0, xref, U):
        out = np.zeros(self.batch)
        gnmppi_cost(self.h, MEM_HOST, np.ascontiguousarray(x0, float).ravel(),
                    None if xref is None else np.ascontiguousarray(xref, float).ravel(),
                    np.ascontiguousarray(U, float).ravel(), out)
        return out

    def debug(self, name: str, inst: int = 0, count: int = 1 << 26) -> np.ndarray:
        return gnmppi_debug_read(self.h, DEBUG[name], inst, count)


# ---------------------------------------------------------------------------
# learned warm start


class Mlp:
    """Owner of a gnmppi_mlp_t handle; arrays are host numpy (MEM_HOST) or
    CUDA torch tensors (MEM_DEVICE)."""

    def __init__(self, dims, nu=2, weights_bf16=True, max_batch=4096, stream=None):
        L = load()
        self.dims = list(dims)
        self.nu = nu
        self.nmu = dims[-1] // (nu + 1) * nu
        arr = (C.c_int32 * len(dims))(*dims)
        h = C.c_void_p()
        st = L.gnmppi_mlp_create(len(dims) - 1, arr, nu, int(weights_bf16), max_batch, stream, C.byref(h))
        if st != OK:
            raise GnmppiError(st, "gnmppi_mlp_create: " + L.gnmppi_mlp_last_error(None).decode())
        self.h = h
        self.np = int(L.gnmppi_mlp_num_params(h))

    def _chk(self, st, name):
        if st != OK:
            raise GnmppiError(st, f"{name}: " + load().gnmppi_mlp_last_error(self.h).decode())

    def close(self):
        if self.h is not None:
            load().gnmppi_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, mem=MEM_HOST):
        self._chk(load().gnmppi_mlp_set_params(self.h, mem, _ptr(params), self.np), "gnmppi_mlp_set_params")

    def get_params(self):
        out = np.zeros(self.np)
        self._chk(load().gnmppi_mlp_get_params(self.h, MEM_HOST, out.ctypes.data, self.np), "gnmppi_mlp_get_params")
        return out

    def get_state(self):
        """(params, Adam first moments, second moments, step count)."""
        p, m1, m2 = np.zeros(self.np), np.zeros(self.np), np.zeros(self.np)
        step = C.c_int32()
        self._chk(load().gnmppi_mlp_get_state(self.h, MEM_HOST, p.ctypes.data, m1.ctypes.data, m2.ctypes.data,
                                               self.np, C.byref(step)), "gnmppi_mlp_get_state")
        return p, m1, m2, int(step.value)

    def set_state(self, params, m1, m2, step):
        arrs = [np.ascontiguousarray(a, float) for a in (params, m1, m2)]
        self._chk(load().gnmppi_mlp_set_state(self.h, MEM_HOST, *(a.ctypes.data for a in arrs), self.np, int(step)),
                  "gnmppi_mlp_set_state")

    def set_normalization(self, x_mean, x_std, y_scale):
        xm = np.ascontiguousarray(x_mean, float)
        xs = np.ascontiguousarray(x_std, float)
        self._chk(load().gnmppi_mlp_set_normalization(self.h, xm.ctypes.data, xs.ctypes.data, float(y_scale)),
                  "gnmppi_mlp_set_normalization")

    def forward(self, X):
        X = np.ascontiguousarray(X, float)
        Y = np.zeros((X.shape[0], self.dims[-1]))
        self._chk(load().gnmppi_mlp_forward(self.h, MEM_HOST, X.ctypes.data, X.shape[0], Y.ctypes.data),
                  "gnmppi_mlp_forward")
        return Y

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(X, float)
        T = np.ascontiguousarray(T, float)
        g = np.zeros(self.np)
        loss = C.c_double()
        self._chk(load().gnmppi_mlp_loss_grad(self.h, MEM_HOST, X.ctypes.data, T.ctypes.data, X.shape[0],
                                               C.byref(loss), g.ctypes.data), "gnmppi_mlp_loss_grad")
        return loss.value, g

    def train_step(self, X, T, B, lr, mem=MEM_DEVICE):
        loss = C.c_double()
        self._chk(load().gnmppi_mlp_train_step(self.h, mem, _ptr(X), _ptr(T), B, lr, C.byref(loss)),
                  "gnmppi_mlp_train_step")
        return loss.value

    def warm_start(self, X, B, U0, sigma, sigma_min=1e-300, sigma_max=1e300, mem=MEM_DEVICE):
        self._chk(load().gnmppi_mlp_warm_start(self.h, mem, _ptr(X), B, sigma_min, sigma_max, _ptr(U0), _ptr(sigma)),
                  "gnmppi_mlp_warm_start")
