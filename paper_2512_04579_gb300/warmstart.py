"""Learned warm start for GN-MPPI on the hanging chain (M = 10, N = 100).

Orchestration only -- every computation (the solves that generate the
training targets, the network's training and inference, the warm-started
and fallback solves, the FP64 cost checks) runs in libgnmppi.so through its
C ABI.

  * make_dataset: plain GN-MPPI solves (K = 2048, 30 iterations, FP32 mode)
    of seeded initial states around the rest state, all for one target;
  * train: Gaussian-NLL training of the MLP 36 -> 256 -> 256 -> 256 -> 300
    (mu: 200 controls, s: 100 per-step log sampling scales), Adam;
  * LearnedSolver: warm start (U_0 = mu, sigma = exp(s) clamped to
    [SIGMA_MIN, SIGMA_MAX]) -> GN-MPPI with
    K = 512 and 5 iterations -> instances whose last iteration still changed
    the cost by more than `tol` (relative) continue with plain GN-MPPI
    (K = 2048, 30 iterations) from the warm result.

Command line:  python -m paper_2512_04579_gb300.warmstart --train N --epochs E --out FILE
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import gnmppi as G
from . import inputs as I

M, N, NU = 10, 100, 2
NX, NMU = 4 * (M - 1), N * NU
DIMS = [NX, 256, 256, 256, NMU + N]
# Warm-start sampling scale range.  The network's NLL scale is its own fitting
# error, far below what a Jacobian estimate from FP32 rollouts resolves; the
# floor keeps the smoothing scale where that estimate is accurate, the ceiling
# is the cold-start scale.
SIGMA_MIN, SIGMA_MAX = 0.05, 0.2
SEED = I.BASE_SEED + 3
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "chain_m10_warmstart.npz")


def _torch():
    import torch

    return torch


def chain_problem(K, T, precision=G.PREC_FP32, sigma0=0.2):
    return G.chain_problem(M=M, N=N, K=K, iterations=T, lam=1e-3, sigma0=sigma0, seed=SEED, precision=precision)


def solve_chunks(x0, target, K=2048, T=30, chunk=2048, precision=G.PREC_FP32, stream=None):
    """Plain GN-MPPI (cold start U_0 = 0) of many instances, `chunk` per handle."""
    torch = _torch()
    n = x0.shape[0]
    out = np.zeros((n, NMU))
    dt = torch.tensor(np.tile(target, (min(chunk, n), 1)).ravel(), dtype=torch.float64, device="cuda")
    h = None
    hb = 0
    for s in range(0, n, chunk):
        b = min(chunk, n - s)
        if h is None or hb != b:
            if h is not None:
                G.gnmppi_destroy(h)
            h = G.gnmppi_create(chain_problem(K, T, precision), b, None, stream)
            hb = b
        dx = torch.tensor(x0[s:s + b].ravel(), dtype=torch.float64, device="cuda")
        dU = torch.zeros(b * NMU, dtype=torch.float64, device="cuda")
        G.gnmppi_solve(h, G.MEM_DEVICE, dx, dt[: b * 2 * (M - 1)], dU, None)
        out[s:s + b] = dU.view(b, NMU).cpu().numpy()
    if h is not None:
        G.gnmppi_destroy(h)
    return out


def make_dataset(n, chunk=2048, stream_id=I.TRAIN_STREAM):
    x0, target = I.chain_fixed_target_states(SEED, n, M, I.WARM_PHI, stream=stream_id)
    U = solve_chunks(x0, target, chunk=chunk)
    return x0, U


def init_params(seed=0, sigma0=0.2, y_scale=1.0):
    """Uniform(-1/sqrt(d_in), 1/sqrt(d_in)) weights, zero biases; the log-scale
    outputs start at log(sigma0 / y_scale) (the cold-start sampling scale)."""
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(1, len(DIMS)):
        a = 1.0 / math.sqrt(DIMS[l - 1])
        W = rng.uniform(-a, a, size=(DIMS[l], DIMS[l - 1]))
        b = np.zeros(DIMS[l])
        if l == len(DIMS) - 1:
            W[NMU:] *= 0.1
            b[NMU:] = math.log(sigma0 / y_scale)
        ps += [W.ravel(), b]
    return np.concatenate(ps)


def train(X, U, epochs=30, batch=1024, lr=1e-3, seed=0, bf16=True, stream=None, log=None):
    """Train the warm-start network; returns (Mlp, meta, loss history)."""
    torch = _torch()
    x_mean = X.mean(0)
    x_std = X.std(0) + 1e-12
    y_scale = float(U.std())
    m = G.Mlp(DIMS, nu=NU, weights_bf16=bf16, max_batch=max(batch, 4096), stream=stream)
    m.set_params(init_params(seed, y_scale=y_scale))
    m.set_normalization(x_mean, x_std, y_scale)
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    dT = torch.tensor(U / y_scale, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(seed + 1)
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n), device="cuda")
        tot = 0.0
        steps = 0
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / max(1, epochs)))  # cosine schedule
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            xb = dX.index_select(0, idx).contiguous()
            tb = dT.index_select(0, idx).contiguous()
            tot += m.train_step(xb, tb, batch, lr_ep)
            steps += 1
        hist.append(tot / max(1, steps))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    meta = {"x_mean": x_mean, "x_std": x_std, "y_scale": y_scale}
    return m, meta, hist


def save(m, meta, path=WEIGHTS, **extra):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, dims=np.array(DIMS), params=m.get_params(), x_mean=meta["x_mean"], x_std=meta["x_std"],
             y_scale=meta["y_scale"], **extra)


def load(path=WEIGHTS, bf16=True, max_batch=4096, stream=None):
    z = np.load(path)
    m = G.Mlp(list(z["dims"]), nu=NU, weights_bf16=bf16, max_batch=max_batch, stream=stream)
    m.set_params(z["params"])
    m.set_normalization(z["x_mean"], z["x_std"], float(z["y_scale"]))
    return m


class LearnedSolver:
    """Warm-started GN-MPPI with plain GN-MPPI as the fallback, for a batch of
    instances of one size (device-resident inputs).  An instance whose last
    warm-started iteration still lowered its cost by more than `tol`
    (relative), or whose cost is not finite, continues from the warm-started
    controls with the plain settings for the rest of the plain iteration
    budget (T_plain - T iterations)."""

    def __init__(self, mlp, batch, K=512, T=5, K_plain=2048, T_plain=30, tol=1e-6, precision=G.PREC_FP32,
                 stream=None):
        self.mlp, self.batch, self.tol = mlp, batch, tol
        self.h_warm = G.gnmppi_create(chain_problem(K, T, precision), batch, None, stream)
        self.h_plain = G.gnmppi_create(chain_problem(K_plain, max(1, T_plain - T), precision), batch, None, stream)
        # the fallback runs the few instances the warm start left unconverged
        # (the others are masked off): one SM and 16 warps per Cholesky
        G.gnmppi_tune_set(self.h_plain, 1, 512)
        torch = _torch()
        self.U0 = torch.zeros(batch * NMU, dtype=torch.float64, device="cuda")
        self.sig = torch.zeros(batch * NMU, dtype=torch.float64, device="cuda")

    def close(self):
        for h in (self.h_warm, self.h_plain):
            if h is not None:
                G.gnmppi_destroy(h)
        self.h_warm = self.h_plain = None

    def solve(self, dx0, dtgt, dU):
        """dU (out): solutions.  Returns the number of instances that fell back."""
        self.mlp.warm_start(dx0, self.batch, dU, self.sig, SIGMA_MIN, SIGMA_MAX)
        st, rep = G.gnmppi_solve(self.h_warm, G.MEM_DEVICE, dx0, dtgt, dU, self.sig, self.batch)
        active = np.array([0 if (math.isfinite(r.C_final) and abs(r.C_prev - r.C_final) <= self.tol * abs(r.C_final))
                           else 1 for r in rep], dtype=np.int32)
        nfb = int(active.sum())
        if nfb:
            G.gnmppi_solve_masked(self.h_plain, G.MEM_DEVICE, dx0, dtgt, dU, None, active, self.batch)
        return nfb


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200000, help="training solves")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--chunk", type=int, default=2048)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    from . import build as B

    B.build()
    G.load()
    t0 = time.time()
    X, U = make_dataset(args.train, chunk=args.chunk)
    t1 = time.time()
    print(f"dataset: {args.train} plain GN-MPPI solves in {t1 - t0:.1f} s", flush=True)
    m, meta, hist = train(X, U, epochs=args.epochs, batch=args.batch, lr=args.lr, log=print)
    t2 = time.time()
    print(f"training: {args.epochs} epochs in {t2 - t1:.1f} s, final loss {hist[-1]:.4f}", flush=True)
    save(m, meta, args.out, train_solves=args.train, epochs=args.epochs, loss=np.array(hist),
         data_seconds=t1 - t0, train_seconds=t2 - t1)
    m.close()
    print("saved", args.out)


if __name__ == "__main__":
    main()
