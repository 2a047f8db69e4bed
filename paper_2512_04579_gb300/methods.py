"""Method comparison on the GPU in the manner of the paper's Table 1 (Sec. 5):
iterations until each method reaches the problem's optimum, for

  Method C  deterministic MPPI (the step of Eq. 5 taken whole),
  Method D  GN-MPPI with random antithetic samples (Algorithm 1),
  Method E  GN-MPPI with the sigma-point Dirac mixture,

on Problems I-IV of Sec. 5 (Rosenbrock, Rastrigin, Heaviside, the linear
double integrator), the pendulum swing-up (with and without dead-zone
friction, Setting V.ii) and the chain (M = 10, N = 100).  Methods C and D use
K = 2048 samples (the paper: 2000, antithetic).  Converged: the cost within
`tol` of the optimum (absolute for Problems I-III, whose optimum is 0;
relative to the best cost any method reached otherwise).

Orchestration only; every iteration runs in libgnmppi.so (one gnmppi_step per
iteration, so the cost history can be read after each).

  python -m paper_2512_04579_gb300.methods [--iters 200] [--tol 1e-6]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import gnmppi as G
from . import inputs as I


def problems():
    """(name, problem factory(sampling, method, K, T), x0, xref, U0, sigma0, zero optimum)."""
    h = 0.1
    A = np.array([[1.0, h], [0.0, 1.0]])
    B = np.array([[h * h / 2], [h]])
    wq, wr, wqN = math.sqrt(2.0) * np.ones(2), math.sqrt(2 * 0.01) * np.ones(1), math.sqrt(2 * 10.0) * np.ones(2)
    px0 = I.pendulum_x0(I.BASE_SEED, 1)[0]
    cx0, ctg = I.chain_instances(I.BASE_SEED + 1, 1, 10)
    out = []
    for name, U0, s0 in (("rosenbrock", (0.0, 0.0), 0.5), ("rastrigin", (1.9, 1.7), 1.0),
                         ("heaviside", (0.5,), 0.5)):
        out.append((f"{name}", lambda smp, meth, K, T, name=name, s0=s0: G.testfun_problem(
            name, K=K, iterations=T, lam=1e-3, sigma0=s0, sampling=smp, method=meth, seed=I.BASE_SEED),
                    np.zeros(1), None, np.array(U0, float), s0, True))
    out.append(("lq (Problem IV)", lambda smp, meth, K, T: G.linear_problem(
        A, B, wq, wr, wqN, N=50, K=K, iterations=T, lam=1e-3, sigma0=0.5, sampling=smp, method=meth,
        seed=I.BASE_SEED), np.array([1.0, 0.0]), None, np.zeros(50), 0.5, False))
    out.append(("pendulum", lambda smp, meth, K, T: G.pendulum_problem(
        N=50, K=K, iterations=T, lam=1e-3, sigma0=0.5, sampling=smp, method=meth, seed=I.BASE_SEED),
        px0, None, np.zeros(50), 0.5, False))
    out.append(("pendulum, friction 0.5 (V.ii)", lambda smp, meth, K, T: G.pendulum_problem(
        u_friction=0.5, N=50, K=K, iterations=T, lam=1e-3, sigma0=0.5, sampling=smp, method=meth,
        seed=I.BASE_SEED), px0, None, np.zeros(50), 0.5, False))
    out.append(("chain M=10", lambda smp, meth, K, T: G.chain_problem(
        M=10, N=100, K=K, iterations=T, lam=1e-3, sigma0=0.2, sampling=smp, method=meth, seed=I.BASE_SEED + 1),
        cx0[0], ctg[0], np.zeros(200), 0.2, False))
    return out


METHODS = (("C", G.SAMPLE_RANDOM, G.METHOD_MPPI), ("D", G.SAMPLE_RANDOM, G.METHOD_GN),
           ("E", G.SAMPLE_SIGMA, G.METHOD_GN))


def history(factory, x0, xref, U0, s0, sampling, method, iters, K=2048):
    """Cost after every iteration (FP64 mode, gnmppi_step per iteration)."""
    prob = factory(sampling, method, K, iters)
    s = G.Solver(prob, 1)
    U = U0.copy()
    sig = np.full(U.size, s0)
    sb = math.sqrt(prob.beta)
    C = [float(s.cost(x0, xref, U)[0])]
    try:
        for k in range(iters):
            st, U, rep = s.step(x0, xref, U, sig, k)
            if st != 0 or not math.isfinite(rep[0].C_new):
                break
            C.append(float(rep[0].C_new))
            sig = sig * sb
    finally:
        s.close()
    return np.array(C)


def first_within(C, target):
    hit = np.nonzero(C <= target)[0]
    return int(hit[0]) if hit.size else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--tol", type=float, default=1e-6)
    args = ap.parse_args()
    from . import build as B

    B.build()
    G.load()
    rows = []
    for name, factory, x0, xref, U0, s0, zero_opt in problems():
        hist = {m: history(factory, x0, xref, U0, s0, smp, meth, args.iters) for m, smp, meth in METHODS}
        best = min(float(np.min(h)) for h in hist.values())
        target = args.tol if zero_opt else best * (1 + args.tol)
        row = {"problem": name, "optimum": 0.0 if zero_opt else best, "target": target}
        for m in hist:
            row[m] = {"iterations": first_within(hist[m], target), "final_cost": float(hist[m][-1]),
                      "C0": float(hist[m][0])}
        rows.append(row)
        print(json.dumps(row), flush=True)
    print("| problem | C: iterations | D: iterations | E: iterations |")
    print("|---|---:|---:|---:|")
    for r in rows:
        cells = [str(r[m]["iterations"]) if r[m]["iterations"] is not None else f"> {args.iters}" for m in "CDE"]
        print(f"| {r['problem']} | " + " | ".join(cells) + " |")


if __name__ == "__main__":
    main()
