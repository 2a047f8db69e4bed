"""High-dimensional scaling sweep of one GN-MPPI iteration on the GPU.

Chains of M in {16, 32, 64} masses (nx = 4(M-1) up to 252, nu = 2, N = 200,
n = N nu = 400 unknowns, nR = 200 (2(M-1) + 2) + 2(M-1) residual rows) with
K in {4096, 16384, 65536} samples.  For every (M, K) the sweep times the
kernels of one Algorithm-1 iteration with CUDA events (gnmppi_phase_times)
on a batch sized to fit the device, and reports throughput and roofline
fractions: rollouts against the FP32 pipe (152 SMs x 128 lanes x 2 flop x
clock), the contraction against HBM bandwidth (its operands are streamed
once), the FP64 Cholesky against the FP64 pipe (2 DFMA per clock per SM).

Orchestration only; every kernel runs in libgnmppi.so.

  python -m paper_2512_04579_gb300.sweep [--prec bf16|fp32|fp64] [--budget-gb 60]
  python -m paper_2512_04579_gb300.sweep --gap --prec bf16   (cost gap vs the FP64 mode)
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import gnmppi as G
from . import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def chain_flops_per_step(F: int) -> int:
    """FP32 flops of one RK4 step of an F-free-mass chain plus its residual
    rows (FMA = 2): 4 right-hand sides of 25F + 2, 52F for the RK4
    combinations, 6 per residual row (2F + 2 rows)."""
    return 4 * (25 * F + 2) + 52 * F + 6 * (2 * F + 2)


def peaks():
    try:
        p = json.load(open(os.path.join(os.path.dirname(HERE), "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        p = {}
    clk = float(p.get("sm_max_mhz", 2070.0)) * 1e6
    return {"fp32_tflops": 152 * 128 * 2 * clk / 1e12, "fp64_tflops": 152 * 2 * 2 * clk / 1e12,
            "hbm_gbs": float(p.get("hbm_gbs", 6764.7))}


def batch_for(M, N, K, esz, budget_gb):
    F = M - 1
    nR = N * (2 * F + 2) + 2 * F
    n = 2 * N
    per = (nR + n) * (K // 2) * esz + n * (nR + n) * 4 + 3 * n * n * 8 + 16 * nR * 4
    return max(1, min(256, int(budget_gb * 1e9 // per))), nR, n


def run_point(M, K, prec, N=200, budget_gb=60.0, iters=3, seed=I.BASE_SEED + 4):
    import torch

    # bytes per stored dR / W entry: the BF16 mode keeps a head and a remainder plane
    esz = {G.PREC_BF16: 4, G.PREC_FP32: 4, G.PREC_FP64: 8}[prec]
    B, nR, n = batch_for(M, N, K, esz, budget_gb)
    x0, tgt = I.chain_instances(seed, B, M)
    prob = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    h = G.gnmppi_create(prob, B)
    dx = torch.tensor(x0.ravel(), dtype=torch.float64, device="cuda")
    dt = torch.tensor(tgt.ravel(), dtype=torch.float64, device="cuda")
    dU = torch.zeros(B * n, dtype=torch.float64, device="cuda")
    sig = torch.full((B * n,), 0.2, dtype=torch.float64, device="cuda")
    G.gnmppi_step(h, G.MEM_DEVICE, dx, dt, dU, sig, 0)
    ph = None
    for it in range(iters):
        p = G.gnmppi_phase_times(h, it + 1)
        ph = p if ph is None else {k: min(ph[k], p[k]) for k in p}
    G.gnmppi_destroy(h)
    pk = peaks()
    F = M - 1
    flops_roll = B * K * N * chain_flops_per_step(F)
    bytes_contract = B * ((nR + n) * (K // 2) * esz + n * (nR + n) * 4)
    flops_chol = B * n ** 3 / 3
    it_ms = sum(ph.values())
    return {
        "M": M, "K": K, "N": N, "n": n, "nR": nR, "batch": B,
        "precision": {G.PREC_BF16: "bf16", G.PREC_FP32: "fp32", G.PREC_FP64: "fp64"}[prec],
        "ms_per_iteration": it_ms, "instance_iterations_per_s": B / (it_ms / 1e3), "phases_ms": ph,
        "rollout_tflops": flops_roll / (ph["samples"] / 1e3) / 1e12,
        "rollout_frac_fp32": flops_roll / (ph["samples"] / 1e3) / 1e12 / pk["fp32_tflops"],
        "contract_gbs": bytes_contract / (ph["contract"] / 1e3) / 1e9,
        "contract_frac_hbm": bytes_contract / (ph["contract"] / 1e3) / 1e9 / pk["hbm_gbs"],
        "solve_frac_fp64": flops_chol / (ph["solve"] / 1e3) / 1e12 / pk["fp64_tflops"],
    }


def run_gap(M, K, prec, N=200, batch=4, T=10, seed=I.BASE_SEED + 4):
    """Cost gap of a reduced-precision solve against the FP64 reference mode:
    the same instances, seeds and Philox noise, T iterations in each mode; the
    final costs are re-evaluated in FP64.  gap = (C_prec - C_fp64) / C_fp64."""
    import torch

    x0, tgt = I.chain_instances(seed, batch, M)
    dx = torch.tensor(x0.ravel(), dtype=torch.float64, device="cuda")
    dt = torch.tensor(tgt.ravel(), dtype=torch.float64, device="cuda")
    out = {}
    for name, pr in (("fp64", G.PREC_FP64), ("prec", prec)):
        prob = G.chain_problem(M=M, N=N, K=K, iterations=T, lam=1e-3, sigma0=0.2, seed=seed, precision=pr)
        h = G.gnmppi_create(prob, batch)
        dU = torch.zeros(batch * 2 * N, dtype=torch.float64, device="cuda")
        G.gnmppi_solve(h, G.MEM_DEVICE, dx, dt, dU, None)
        C = torch.empty(batch, dtype=torch.float64, device="cuda")
        G.gnmppi_cost(h, G.MEM_DEVICE, dx, dt, dU, C)
        out[name] = C.cpu().numpy()
        G.gnmppi_destroy(h)
    g = (out["prec"] - out["fp64"]) / out["fp64"]
    return {"M": M, "K": K, "N": N, "batch": batch, "iterations": T,
            "precision": {G.PREC_BF16: "bf16", G.PREC_FP32: "fp32"}[prec],
            "C_fp64": out["fp64"].tolist(), "C_prec": out["prec"].tolist(),
            "gap_median": float(np.median(g)), "gap_max_abs": float(np.max(np.abs(g)))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--budget-gb", type=float, default=60.0)
    ap.add_argument("--M", type=int, nargs="*", default=[16, 32, 64])
    ap.add_argument("--K", type=int, nargs="*", default=[4096, 16384, 65536])
    ap.add_argument("--gap", action="store_true",
                    help="cost gap of --prec solves against the FP64 reference mode instead of timings")
    ap.add_argument("--gap-batch", type=int, default=4)
    ap.add_argument("--gap-iters", type=int, default=10)
    args = ap.parse_args()
    from . import build as B

    B.build()
    G.load()
    prec = {"bf16": G.PREC_BF16, "fp32": G.PREC_FP32, "fp64": G.PREC_FP64}[args.prec]
    for M in args.M:
        for K in args.K:
            if args.gap:
                print(json.dumps(run_gap(M, K, prec, batch=args.gap_batch, T=args.gap_iters)), flush=True)
            else:
                print(json.dumps(run_point(M, K, prec, budget_gb=args.budget_gb)), flush=True)


if __name__ == "__main__":
    main()
