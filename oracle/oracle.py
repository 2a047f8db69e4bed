"""Python access to the plain FP64 CPU oracle (``gnmppi_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It builds
and loads ``liboracle.so`` from ``gnmppi_oracle.c`` with gcc and exposes its
routines on numpy arrays.  It imports nothing from the CUDA package.

Every routine follows the paper (arXiv 2512.04579): the simulator and cost
(Sec. 2, Eq. 1-4), softmin weights (Sec. 3, Eq. 3-5), the Gaussian-smoothing
Jacobian (Sec. 4.1, Eq. 7), the GGN step (Sec. 4.2, Eq. 9), the line search
and covariance shrink (Algorithm 1, Eq. 10-11) and Method A (Sec. 5).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gnmppi_oracle.c")
MLP_SRC = os.path.join(HERE, "mlp_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

DYN = {"pendulum": 0, "chain": 1, "linear": 2, "rosenbrock": 3, "rastrigin": 4, "heaviside": 5, "lincont": 6}
JAC = {"lsq": 0, "sigma": 1, "auto": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so x86 and Arm agree)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(MLP_SRC), os.path.getmtime(os.path.join(HERE, "gnmppi_oracle.h"))
    ):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
             "-o", tmp, SRC, MLP_SRC, "-lm"]
        )
        os.replace(tmp, LIB)
    return LIB


class OrcModel(C.Structure):
    _fields_ = [("dyn", C.c_int32), ("nx", C.c_int32), ("nu", C.c_int32), ("N", C.c_int32),
                ("M", C.c_int32), ("pad0", C.c_int32), ("dt", C.c_double), ("params", C.c_double * 8),
                ("lin", C.POINTER(C.c_double))]


class OrcOptions(C.Structure):
    _fields_ = [("K", C.c_int32), ("iterations", C.c_int32), ("L", C.c_int32), ("jac_mode", C.c_int32),
                ("antithetic", C.c_int32), ("monotone", C.c_int32), ("threads", C.c_int32),
                ("ir_steps", C.c_int32), ("lam", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("tau", C.c_double), ("seed", C.c_uint64), ("sampling", C.c_int32), ("method", C.c_int32),
                ("break_it", C.c_int32), ("break_kind", C.c_int32)]


_DP = C.POINTER(C.c_double)


class OrcRecord(C.Structure):
    _fields_ = [("C_nom", C.c_double), ("C_new", C.c_double), ("alpha", C.c_double), ("lambda_used", C.c_double),
                ("c_min", C.c_double), ("sum_w", C.c_double), ("sum_w2", C.c_double), ("ess", C.c_double),
                ("grad_norm", C.c_double), ("step_norm", C.c_double), ("j_star", C.c_int32),
                ("n_masked", C.c_int32), ("jac_mode_used", C.c_int32), ("status", C.c_int32),
                ("chol_retries", C.c_int32), ("pad", C.c_int32), ("delta", _DP), ("C_line", _DP),
                ("mppi_dir", _DP), ("C_samp", _DP), ("J", _DP), ("dR", _DP), ("W", _DP), ("r", _DP)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_nR.restype = C.c_int32
        L.orc_n.restype = C.c_int32
        L.orc_uniform53.restype = C.c_double
        L.orc_uniform53.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_cost.restype = C.c_double
        L.orc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int32, _DP]
        L.orc_iteration.argtypes = [C.POINTER(OrcModel), C.POINTER(OrcOptions), _DP, _DP, _DP, _DP, C.c_uint32,
                                    C.c_uint32, C.POINTER(OrcRecord)]
        L.orc_solve.argtypes = [C.POINTER(OrcModel), C.POINTER(OrcOptions), _DP, _DP, _DP, _DP, C.c_uint32,
                                C.POINTER(OrcRecord), _DP, _DP]
        L.orc_method_a.argtypes = [C.POINTER(OrcModel), _DP, _DP, _DP, C.c_int32, C.c_double, C.c_double,
                                   C.c_double, _DP, C.POINTER(C.c_int32)]
        L.orc_softmin.argtypes = [C.c_int32, _DP, C.c_void_p, C.c_double, _DP, _DP]
        L.orc_cholesky.argtypes = [C.c_int32, _DP]
        L.orc_chol_solve.argtypes = [C.c_int32, _DP, _DP]
        IP = C.POINTER(C.c_int32)
        L.mlo_num_params.restype = C.c_int64
        L.mlo_num_params.argtypes = [C.c_int32, IP]
        L.mlo_forward.argtypes = [C.c_int32, IP, _DP, _DP, _DP, C.c_int32, _DP, _DP]
        L.mlo_loss_grad.restype = C.c_double
        L.mlo_loss_grad.argtypes = [C.c_int32, IP, _DP, _DP, _DP, C.c_int32, _DP, _DP, C.c_int32, _DP]
        L.mlo_adam.argtypes = [C.c_int64, _DP, _DP, _DP, _DP, C.c_int32, C.c_double, C.c_double, C.c_double,
                               C.c_double]
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


@dataclass
class Model:
    """A problem definition: dynamics, horizon and constants (Sec. 2)."""

    dyn: str
    nx: int
    nu: int
    N: int
    dt: float = 0.0
    M: int = 0
    params: tuple = ()
    lin: np.ndarray | None = None
    _keep: list = field(default_factory=list, repr=False)

    @property
    def n(self) -> int:
        return self.N * self.nu

    def c(self) -> OrcModel:
        m = OrcModel()
        m.dyn, m.nx, m.nu, m.N, m.M = DYN[self.dyn], self.nx, self.nu, self.N, self.M
        m.dt = self.dt
        for i, v in enumerate(self.params):
            m.params[i] = v
        if self.lin is not None:
            arr = np.ascontiguousarray(self.lin, dtype=np.float64)
            self._keep.append(arr)
            m.lin = _p(arr)
        return m

    @property
    def nR(self) -> int:
        return int(lib().orc_nR(C.byref(self.c())))


def pendulum(N=50, dt=0.05, g=9.81, l=1.0, m=1.0, b=0.1, u_friction=0.0) -> Model:
    """u_friction > 0: dead-zone friction at the input (Setting V.ii of Sec. 5)."""
    return Model("pendulum", 2, 1, N, dt=dt, params=(g, l, m, b, u_friction))


def chain(M=10, N=100, dt=0.02, mass=0.1, k=10.0, k3=1.0, damping=0.05, gravity=9.81, u_friction=0.0) -> Model:
    """u_friction > 0: dead-zone friction at the input, per component (Setting V.ii of Sec. 5)."""
    return Model("chain", 4 * (M - 1), 2, N, dt=dt, M=M, params=(mass, k, k3, damping, gravity, u_friction))


def linear(A, B, wq, wr, wqN, N) -> Model:
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    nx, nu = B.shape
    lin = np.concatenate([A.ravel(), B.ravel(), np.asarray(wq, float), np.asarray(wr, float),
                          np.asarray(wqN, float)])
    return Model("linear", nx, nu, N, lin=lin)


def lincont(A, B, dt) -> Model:
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    nx, nu = B.shape
    lin = np.concatenate([A.ravel(), B.ravel()])
    return Model("lincont", nx, nu, 1, dt=dt, lin=lin)


def testfun(name: str) -> Model:
    nu = 1 if name == "heaviside" else 2
    return Model(name, 0, nu, 1)


@dataclass
class Options:
    """Algorithm 1's inputs plus the readings the paper leaves open."""

    K: int = 256
    iterations: int = 20
    L: int = 16
    jac_mode: str = "auto"
    antithetic: bool = True
    monotone: bool = False
    threads: int = 1
    ir_steps: int = 1
    lam: float = 1e-3
    beta: float = 0.7
    gamma: float = 0.5
    tau: float = 1.0
    seed: int = 0
    sampling: str = "random"  # "random" (Method D) or "sigma" (sigma points, Method E)
    method: str = "gn"  # "gn" (Algorithm 1) or "mppi" (the MPPI step of Eq. 5, Method C)
    # test hook: at iteration break_it make the LSQ form break down ("s": S has
    # no Cholesky factor; "system": the damped LSQ system has none)
    break_it: int = -1
    break_kind: str = "none"

    def c(self) -> OrcOptions:
        o = OrcOptions()
        o.K, o.iterations, o.L = self.K, self.iterations, self.L
        o.jac_mode = JAC[self.jac_mode]
        o.antithetic, o.monotone, o.threads, o.ir_steps = int(self.antithetic), int(self.monotone), self.threads, \
            self.ir_steps
        o.lam, o.beta, o.gamma, o.tau, o.seed = self.lam, self.beta, self.gamma, self.tau, self.seed
        o.sampling = {"random": 0, "sigma": 1}[self.sampling]
        o.method = {"gn": 0, "mppi": 1}[self.method]
        o.break_it = self.break_it
        o.break_kind = {"none": 0, "s": 1, "system": 2}[self.break_kind]
        return o

    def pairs(self, n: int) -> int:
        """Sample pairs (antithetic) or samples per iteration for n unknowns."""
        if self.sampling == "sigma":
            return n
        return self.K // 2 if self.antithetic else self.K


# ---------------------------------------------------------------------------
# thin wrappers


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform53(hi: int, lo: int) -> float:
    return float(lib().orc_uniform53(hi, lo))


def normals(seed: int, inst: int, it: int, m: int, n: int) -> np.ndarray:
    z = np.zeros(n)
    lib().orc_normals(seed, inst, it, m, n, _p(z))
    return z


def deriv(model: Model, x, u) -> np.ndarray:
    x = np.ascontiguousarray(x, float)
    u = np.ascontiguousarray(u, float)
    out = np.zeros(model.nx)
    lib().orc_deriv(C.byref(model.c()), _p(x), _p(u), _p(out))
    return out


def rk4_step(model: Model, x, u) -> np.ndarray:
    x = np.ascontiguousarray(x, float)
    u = np.ascontiguousarray(u, float)
    out = np.zeros(model.nx)
    lib().orc_rk4_step(C.byref(model.c()), _p(x), _p(u), _p(out))
    return out


def rollout(model: Model, x0, U) -> np.ndarray:
    x0 = np.ascontiguousarray(x0, float)
    U = np.ascontiguousarray(U, float)
    X = np.zeros((model.N + 1) * model.nx)
    st = lib().orc_rollout(C.byref(model.c()), _p(x0), _p(U), _p(X))
    assert st == 0
    return X.reshape(model.N + 1, model.nx)


def _xref(model, xref):
    if xref is None:
        xref = np.zeros(max(1, 2 * (model.M - 1)))
    return np.ascontiguousarray(xref, float)


def residual(model: Model, x0, xref, U) -> np.ndarray:
    x0 = np.ascontiguousarray(x0 if x0 is not None else np.zeros(max(1, model.nx)), float)
    U = np.ascontiguousarray(U, float)
    R = np.zeros(model.nR)
    st = lib().orc_residual(C.byref(model.c()), _p(x0), _p(_xref(model, xref)), _p(U), _p(R))
    assert st == 0
    return R


def cost(model: Model, x0, xref, U) -> float:
    x0 = np.ascontiguousarray(x0 if x0 is not None else np.zeros(max(1, model.nx)), float)
    U = np.ascontiguousarray(U, float)
    return float(lib().orc_cost(C.byref(model.c()), _p(x0), _p(_xref(model, xref)), _p(U)))


def softmin(Cs, tau=1.0, valid=None):
    Cs = np.ascontiguousarray(Cs, float)
    w = np.zeros_like(Cs)
    st = np.zeros(4)
    v = None
    if valid is not None:
        v = np.ascontiguousarray(valid, np.uint8)
    lib().orc_softmin(len(Cs), _p(Cs), v.ctypes.data_as(C.c_void_p) if v is not None else None, tau, _p(w), _p(st))
    return w, {"c_min": st[0], "sum_w": st[1], "sum_w2": st[2], "ess": st[3]}


def cholesky(A) -> tuple[int, np.ndarray]:
    A = np.array(A, float, order="C", copy=True)
    st = lib().orc_cholesky(A.shape[0], _p(A))
    return int(st), A


def chol_solve(Lf, b) -> np.ndarray:
    Lf = np.ascontiguousarray(Lf, float)
    x = np.array(b, float, copy=True)
    lib().orc_chol_solve(Lf.shape[0], _p(Lf), _p(x))
    return x


@dataclass
class Iter:
    """Outputs of one Algorithm-1 iteration."""

    status: int
    U_next: np.ndarray
    C_nom: float
    C_new: float
    alpha: float
    j_star: int
    lambda_used: float
    delta: np.ndarray
    C_line: np.ndarray
    mppi_dir: np.ndarray
    C_samp: np.ndarray
    c_min: float
    sum_w: float
    sum_w2: float
    ess: float
    n_masked: int
    jac_mode_used: int
    chol_retries: int
    grad_norm: float
    J: np.ndarray | None = None
    dR: np.ndarray | None = None
    W: np.ndarray | None = None
    r: np.ndarray | None = None


def _rec(model: Model, opt: Options, want_big: bool):
    n, nR = model.n, model.nR
    Kp = opt.pairs(n)
    nl = opt.L + (1 if opt.monotone else 0)
    bufs = {"delta": np.zeros(n), "C_line": np.zeros(nl), "mppi_dir": np.zeros(n),
            "C_samp": np.zeros(2 * Kp if opt.antithetic else Kp)}
    if want_big:
        bufs.update({"J": np.zeros((nR, n)), "dR": np.zeros((Kp, nR)), "W": np.zeros((Kp, n)), "r": np.zeros(nR)})
    rec = OrcRecord()
    for k, v in bufs.items():
        setattr(rec, k, _p(v))
    return rec, bufs


def _to_iter(rec, bufs, U) -> Iter:
    return Iter(status=rec.status, U_next=U.copy(), C_nom=rec.C_nom, C_new=rec.C_new, alpha=rec.alpha,
                j_star=rec.j_star, lambda_used=rec.lambda_used, delta=bufs["delta"].copy(),
                C_line=bufs["C_line"].copy(), mppi_dir=bufs["mppi_dir"].copy(), C_samp=bufs["C_samp"].copy(),
                c_min=rec.c_min, sum_w=rec.sum_w, sum_w2=rec.sum_w2, ess=rec.ess, n_masked=rec.n_masked,
                jac_mode_used=rec.jac_mode_used, chol_retries=rec.chol_retries, grad_norm=rec.grad_norm,
                J=bufs.get("J"), dR=bufs.get("dR"), W=bufs.get("W"), r=bufs.get("r"))


def iteration(model: Model, opt: Options, x0, xref, U, s, inst=0, it=0, want_big=False) -> Iter:
    """One Algorithm-1 iteration at (U, s); returns its outputs (U is not modified)."""
    x0 = np.ascontiguousarray(x0 if x0 is not None else np.zeros(max(1, model.nx)), float)
    U = np.array(U, float, copy=True)
    s = np.ascontiguousarray(np.broadcast_to(np.asarray(s, float), (model.n,)), float)
    rec, bufs = _rec(model, opt, want_big)
    st = lib().orc_iteration(C.byref(model.c()), C.byref(opt.c()), _p(x0), _p(_xref(model, xref)), _p(U), _p(s),
                             inst, it, C.byref(rec))
    if st != 0 and rec.status == 0:  # rejected before the record was written
        rec.status = st
    return _to_iter(rec, bufs, U)


def solve(model: Model, opt: Options, x0, xref, U0, s0, inst=0):
    """Algorithm 1 from U0; returns (status, U_K, U history, cost history, per-iteration records)."""
    x0 = np.ascontiguousarray(x0 if x0 is not None else np.zeros(max(1, model.nx)), float)
    U = np.array(U0, float, copy=True)
    s0 = np.ascontiguousarray(np.broadcast_to(np.asarray(s0, float), (model.n,)), float)
    T = opt.iterations
    recs = (OrcRecord * T)()
    keep = []
    for t in range(T):
        r, b = _rec(model, opt, False)
        recs[t] = r
        keep.append(b)
    Uh = np.zeros((T + 1, model.n))
    Ch = np.zeros(T + 1)
    st = lib().orc_solve(C.byref(model.c()), C.byref(opt.c()), _p(x0), _p(_xref(model, xref)), _p(U), _p(s0), inst,
                         recs, _p(Uh), _p(Ch))
    its = [_to_iter(recs[t], keep[t], Uh[t + 1]) for t in range(T)]
    return int(st), U, Uh, Ch, its


def method_a(model: Model, x0, xref, U0, max_iter=200, eps=6e-6, lam=1e-10, gtol=1e-10):
    """Method A (central-FD GGN, Sec. 5) polish; returns (status, U, C, iterations)."""
    x0 = np.ascontiguousarray(x0 if x0 is not None else np.zeros(max(1, model.nx)), float)
    U = np.array(U0, float, copy=True)
    c = C.c_double()
    it = C.c_int32()
    st = lib().orc_method_a(C.byref(model.c()), _p(x0), _p(_xref(model, xref)), _p(U), max_iter, eps, lam, gtol,
                            C.byref(c), C.byref(it))
    return int(st), U, float(c.value), int(it.value)


# ---------------------------------------------------------------------------
# learned warm start: FP64 MLP (mlp_oracle.c)


def _dims(dims):
    return (C.c_int32 * len(dims))(*dims)


def mlp_num_params(dims) -> int:
    return int(lib().mlo_num_params(len(dims) - 1, _dims(dims)))


def mlp_forward(dims, params, x_mean, x_std, X) -> np.ndarray:
    X = np.ascontiguousarray(X, float)
    B = X.shape[0]
    out = np.zeros((B, dims[-1]))
    lib().mlo_forward(len(dims) - 1, _dims(dims), _p(np.ascontiguousarray(params, float)),
                      _p(np.ascontiguousarray(x_mean, float)), _p(np.ascontiguousarray(x_std, float)), B, _p(X),
                      _p(out))
    return out


def mlp_loss_grad(dims, params, x_mean, x_std, X, T, nu):
    X = np.ascontiguousarray(X, float)
    T = np.ascontiguousarray(T, float)
    g = np.zeros(mlp_num_params(dims))
    loss = lib().mlo_loss_grad(len(dims) - 1, _dims(dims), _p(np.ascontiguousarray(params, float)),
                               _p(np.ascontiguousarray(x_mean, float)), _p(np.ascontiguousarray(x_std, float)),
                               X.shape[0], _p(X), _p(T), nu, _p(g))
    return float(loss), g


def mlp_adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays."""
    lib().mlo_adam(params.size, _p(params), _p(np.ascontiguousarray(grad, float)), _p(m), _p(v), t, lr, b1, b2, eps)
