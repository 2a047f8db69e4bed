"""Benchmark: OCP solves per second to a 1e-6 relative cost gap, GN-MPPI on GB300.

Workload: a batch of seeded chain OCPs (M=10 masses, N=100, nu=2, K=2048
samples, 30 Algorithm-1 iterations, sigma0 0.2, lambda 1e-3), FP32 rollouts
with an FP64 Cholesky (the library's FP32 mode), all instances in one handle
and one CUDA graph per solve.  A step = one batched solve of every instance.
An instance counts as solved when the FP64 re-evaluation of its final cost is
within 1e-6 (relative) of its reference optimum C*, which the FP64 CPU oracle
wrote to tests/golden/chain_m10_cstar.txt.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gnmppi|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle,
as it stands, on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, K, T, SIGMA0, LAM = 10, 100, 2048, 30, 0.2, 1e-3
GAP = 1e-6
METRIC = "OCP solves/s to 1e-6 rel. cost gap"
CSTAR = os.path.join(ROOT, "tests", "golden", "chain_m10_cstar.txt")
CSTAR_FIXED = os.path.join(ROOT, "tests", "golden", "chain_m10_fixed_cstar.txt")
CSTAR_UNEVEN = os.path.join(ROOT, "tests", "golden", "chain_uneven_cstar.txt")
CSTAR_PEND = os.path.join(ROOT, "tests", "golden", "pendulum_cstar.txt")
WORKLOAD = "chain M=10 N=100 nu=2 K=2048 T=30 sigma0=0.2 lambda=1e-3"
PREC, PREC_NAME = 2, "bf16x3"  # the library's BF16 mode (GNMPPI_PREC_BF16)
DTYPE = "f32 rollouts, bf16 head+remainder contractions (3 passes, f32 accumulate), f64 Cholesky"


# DRAM read + write of one k_samples launch of the default workload (256 instances), from one
# full-size ncu capture of this command (one-pass metrics); null for other batch sizes.
K_SAMPLES_TRAFFIC_B256 = 2.4886e9


def load_cstar(path=CSTAR):
    rows = np.loadtxt(path, comments="#")
    return rows[:, 0].astype(int), rows[:, 1], rows[:, 2]


def uneven_arm(args, dev, stream):
    """The uneven batch: 1024 chain instances with M ~ U{4..16}, N ~ U{40..160},
    K ~ U{512..4096} in one handle and one CUDA graph per solve, FP32 rollouts,
    BF16 contraction, FP64 Cholesky; solved against the oracle's optima."""
    import torch

    from paper_2512_04579_gb300 import gnmppi as G
    from paper_2512_04579_gb300 import inputs as I

    seed = I.BASE_SEED + 2
    B = 1024
    Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, B)
    shapes = [(int(Ns[b]), int(Ms[b]), int(Ks[b])) for b in range(B)]
    prob = G.chain_problem(M=int(Ms[0]), N=int(Ns[0]), K=int(Ks[0]), iterations=T, lam=LAM, sigma0=SIGMA0, seed=seed,
                           precision=G.PREC_BF16)
    h = G.gnmppi_create(prob, B, shapes, stream.cuda_stream)
    dx = torch.tensor(np.concatenate(x0s), dtype=torch.float64, device=dev)
    dt = torch.tensor(np.concatenate(tgts), dtype=torch.float64, device=dev)
    nU = int(sum(2 * n for n in Ns))
    dU = torch.zeros(nU, dtype=torch.float64, device=dev)

    def once():
        dU.zero_()
        G.gnmppi_solve(h, G.MEM_DEVICE, dx, dt, dU, None)

    tune = G.gnmppi_autotune(h, G.MEM_DEVICE, dx, dt, dU)  # launch configuration, before the warm-up
    for _ in range(max(1, args.warmup)):
        once()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel times of one more iteration on the solve's final state (before
    # gnmppi_cost, which reloads the inputs and resets the per-instance state)
    phases = G.gnmppi_phase_times(h, T)
    C = torch.empty(B, dtype=torch.float64, device=dev)
    G.gnmppi_cost(h, G.MEM_DEVICE, dx, dt, dU, C)
    G.gnmppi_destroy(h)
    out = {"workload": "%d chain instances, M~U{4..16}, N~U{40..160}, K~U{512,1024,2048,4096}, BF16 contraction" % B,
           "ms_per_batch": ms, "instances_per_s": B / (ms / 1e3), "phases_ms_per_iteration": phases,
           "launch_config": tune}
    if os.path.exists(CSTAR_UNEVEN):
        _, _, Cs = load_cstar(CSTAR_UNEVEN)
        g = (C.cpu().numpy()[: len(Cs)] - Cs) / Cs
        solved = int(np.sum(g <= GAP))
        out.update({"solved": solved, "checked": len(Cs), "gap_median": float(np.median(g)),
                    "solves_per_s": solved / len(Cs) * B / (ms / 1e3)})
    else:
        out["solved"] = None
    return out


def pendulum_arm(args, dev, stream):
    """The pendulum swing-up (N=50, K=256, sigma0 0.5, lambda 1e-3, 20
    iterations, FP64 mode), one instance per handle and solve as the
    configuration states it, on the held-out initial states whose reference
    optima the oracle wrote to tests/golden/pendulum_cstar.txt (its 20-iteration
    solve polished by Method A).  Reports solves/s to the 1e-6 gap (honestly
    0 when 20 iterations do not reach the optimum), the latency per solve, and
    the same instances batched in one handle."""
    import torch

    from paper_2512_04579_gb300 import gnmppi as G
    from paper_2512_04579_gb300 import inputs as I

    if not os.path.exists(CSTAR_PEND):
        return {"unavailable": "no pendulum reference optima"}
    _, C_gn, Cs = load_cstar(CSTAR_PEND)
    B = len(Cs)
    seed = I.BASE_SEED
    x0 = I.pendulum_x0(seed, B)
    dx = torch.tensor(x0.ravel(), dtype=torch.float64, device=dev)
    C = torch.empty(1, dtype=torch.float64, device=dev)
    Cfin = np.zeros(B)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    hs = [G.gnmppi_create(G.pendulum_problem(N=50, K=256, iterations=20, lam=LAM, sigma0=0.5, seed=seed,
                                             first_instance=b), 1, None, stream.cuda_stream) for b in range(B)]
    dU = torch.zeros(50, dtype=torch.float64, device=dev)
    for b in range(min(B, 3)):  # warm-up (graph capture)
        G.gnmppi_solve(hs[b], G.MEM_DEVICE, dx[2 * b: 2 * b + 2], None, dU, None)
    t_ms = 0.0
    for b in range(B):
        dU.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        G.gnmppi_solve(hs[b], G.MEM_DEVICE, dx[2 * b: 2 * b + 2], None, dU, None)
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms += e0.elapsed_time(e1)
        G.gnmppi_cost(hs[b], G.MEM_DEVICE, dx[2 * b: 2 * b + 2], None, dU, C)
        Cfin[b] = float(C.item())
    for h in hs:
        G.gnmppi_destroy(h)
    ms = t_ms / B
    g = (Cfin - Cs) / Cs
    solved = int(np.sum(g <= GAP))
    # the same instances in one handle
    hb = G.gnmppi_create(G.pendulum_problem(N=50, K=256, iterations=20, lam=LAM, sigma0=0.5, seed=seed), B, None,
                         stream.cuda_stream)
    dUb = torch.zeros(B * 50, dtype=torch.float64, device=dev)
    G.gnmppi_solve(hb, G.MEM_DEVICE, dx, None, dUb, None)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, args.steps)):
        dUb.zero_()
        G.gnmppi_solve(hb, G.MEM_DEVICE, dx, None, dUb, None)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / max(1, args.steps)
    G.gnmppi_destroy(hb)
    return {"workload": "pendulum swing-up N=50 K=256 sigma0=0.5 lambda=1e-3 T=20, FP64, %d held-out x0" % B,
            "solves_per_s": solved / (ms / 1e3), "solved": solved, "instances": B, "ms_per_solve": ms,
            "gap_median": float(np.median(g)), "gap_min": float(np.min(g)),
            "oracle_gap_median": float(np.median((C_gn - Cs) / Cs)),
            "batched": {"ms_per_batch": ms_b, "instance_solves_per_s": B / (ms_b / 1e3)},
            "note": "20 iterations of Method D do not reach the swing-up optimum (the oracle's own solve neither); "
                    "the GPU's FP64 solve follows the oracle's"}


def learned_eval(args, dev, stream, B, steps):
    """Learned warm start and plain GN-MPPI on the first B held-out initial
    states of the warm-start workload; returns times and the FP64
    re-evaluated final costs of both."""
    import torch

    from paper_2512_04579_gb300 import gnmppi as G
    from paper_2512_04579_gb300 import inputs as I
    from paper_2512_04579_gb300 import warmstart as W

    x0, tg = I.chain_fixed_target_states(W.SEED, B, W.M, I.WARM_PHI, stream=I.EVAL_STREAM)
    dx = torch.tensor(x0.ravel(), dtype=torch.float64, device=dev)
    dt = torch.tensor(np.tile(tg, (B, 1)).ravel(), dtype=torch.float64, device=dev)
    mlp = W.load(W.WEIGHTS, max_batch=B, stream=stream.cuda_stream)
    ls = W.LearnedSolver(mlp, B, stream=stream.cuda_stream)
    hp = G.gnmppi_create(W.chain_problem(2048, 30), B, None, stream.cuda_stream)
    Cout = torch.empty(B, dtype=torch.float64, device=dev)

    def cost_of(dU):
        G.gnmppi_cost(hp, G.MEM_DEVICE, dx, dt, dU, Cout)
        return Cout.cpu().numpy().copy()

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = None
        for _ in range(steps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out

    dU = torch.zeros(B * W.NMU, dtype=torch.float64, device=dev)
    ms_l, nfb = timed(lambda: ls.solve(dx, dt, dU))
    C_l = cost_of(dU)
    dP = torch.zeros_like(dU)

    def plain_once():
        dP.zero_()
        G.gnmppi_solve(hp, G.MEM_DEVICE, dx, dt, dP, None)

    ms_p, _ = timed(plain_once)
    C_p = cost_of(dP)
    ls.close()
    mlp.close()
    G.gnmppi_destroy(hp)
    return ms_l, int(nfb), C_l, ms_p, C_p


def learned_arm(args, dev, stream):
    """Batched + learned warm start vs plain GN-MPPI on the warm-start workload
    (one chain target).  Learned: MLP warm start -> GN-MPPI K=512, 5
    iterations -> plain GN-MPPI (K=2048, 30 iterations) from there for
    instances whose last iteration still moved the cost by more than 1e-6
    (relative).  Plain: cold start, K=2048, 30 iterations.
      * 256 held-out initial states with the oracle's optima C*;
      * 4096 held-out initial states (the first 256 are the ones above),
        measured against the better of the two methods' final costs, since the
        oracle's optima of all 4096 are out of reach on the host."""
    from paper_2512_04579_gb300 import warmstart as W

    if not os.path.exists(W.WEIGHTS):
        return {"unavailable": "no trained warm-start weights"}
    _, _, Cs = load_cstar(CSTAR_FIXED)
    B = len(Cs)
    ms_l, nfb, C_l, ms_p, C_p = learned_eval(args, dev, stream, B, args.steps)
    g_l = (C_l - Cs) / Cs
    g_p = (C_p - Cs) / Cs
    s_l, s_p = int(np.sum(g_l <= GAP)), int(np.sum(g_p <= GAP))
    z = np.load(W.WEIGHTS)
    out = {"workload": "chain M=10 N=100, one target (phi=3pi/32), %d held-out initial states" % B,
           "learned_solves_per_s": s_l / (ms_l / 1e3), "learned_ms_per_batch": ms_l, "learned_solved": s_l,
           "learned_fallbacks": nfb, "learned_gap_median": float(np.median(g_l)),
           "plain_solves_per_s": s_p / (ms_p / 1e3), "plain_ms_per_batch": ms_p, "plain_solved": s_p,
           "plain_gap_median": float(np.median(g_p)), "speedup": (s_l / ms_l) / max(1e-30, s_p / ms_p),
           "network": "36-256-256-256-300 GELU, BF16 weights, trained on %d plain solves" % int(z["train_solves"])}
    if args.learned_eval > 0:
        B4 = args.learned_eval
        ms_l, nfb, C_l, ms_p, C_p = learned_eval(args, dev, stream, B4, max(1, min(args.steps, 2)))
        Cb = np.minimum(C_l, C_p)
        s_l = int(np.sum((C_l - Cb) / Cb <= GAP))
        s_p = int(np.sum((C_p - Cb) / Cb <= GAP))
        out["heldout"] = {
            "instances": B4, "reference": "per instance, the better of the two methods' FP64 re-evaluated final costs",
            "learned_solves_per_s": s_l / (ms_l / 1e3), "learned_ms_per_batch": ms_l, "learned_solved": s_l,
            "learned_fallbacks": nfb, "plain_solves_per_s": s_p / (ms_p / 1e3), "plain_ms_per_batch": ms_p,
            "plain_solved": s_p, "speedup": (s_l / ms_l) / max(1e-30, s_p / ms_p)}
    return out


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def partition(batch, rank, world):
    """Contiguous instance range [lo, hi) of rank r.  Instances are
    independent, so the ranks split one batch with no data-path exchange; a
    rank's handle gets first_instance = lo, so every instance draws the noise
    stream it draws in the unsplit batch and the ranks together compute
    exactly the one-GPU batch (strong scaling: the total work is fixed)."""
    q, r = divmod(batch, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def gather_rows(local, batch, world, device):
    """Per-instance rows ([hi - lo, w] on each rank) of every rank, in
    instance order, on every rank: the final gather of U and of the costs.
    Ranks with fewer rows pad to the largest share for the all-gather."""
    if world <= 1:
        return local
    import torch
    import torch.distributed as dist

    cnt = -(-batch // world)
    buf = torch.zeros((cnt,) + tuple(local.shape[1:]), dtype=local.dtype, device=device)
    buf[: local.shape[0]] = local.to(device)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    rows = []
    for r in range(world):
        lo, hi = partition(batch, r, world)
        rows.append(parts[r][: hi - lo])
    return torch.cat(rows)


def reduce_over_ranks(ms, solved, world, device):
    """The job's time is the slowest rank's (max over ranks) and its work the
    instances solved on all ranks (sum); returns both, unchanged for one
    rank."""
    if world <= 1:
        return ms, solved
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(solved)], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(s.item()))


class Clocks:
    """nvidia-smi sampler for SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            out, _ = self.p.communicate(timeout=5)
            for line in out.strip().splitlines():
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    self.rows.append(f)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if num(r[1])]
        mx = [num(r[2]) for r in self.rows if num(r[2])]
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def chain_flops_per_step(F: int) -> int:
    """Algorithmic FP32 flops of one RK4 step of the F-free-mass chain plus its
    residual rows (FMA = 2): 4 right-hand sides of 25F + 2, 52F for the RK4
    combinations, 6 per residual row (2F + 2 rows)."""
    return 4 * (25 * F + 2) + 52 * F + 6 * (2 * F + 2)


def run_gnmppi(args):
    import torch

    from paper_2512_04579_gb300 import build as B
    from paper_2512_04579_gb300 import gnmppi as G
    from paper_2512_04579_gb300 import inputs as I

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or not os.path.exists(B.OUT):
        B.build()
    if world > 1:
        dist.barrier()
    G.load()

    idx, C_gn_oracle, Cstar_all = load_cstar()
    batch = len(idx) if args.batch <= 0 else min(args.batch, len(idx))
    Cstar_all = Cstar_all[:batch]
    seed = I.BASE_SEED + 1
    x0, tgt = I.chain_instances(seed, len(idx), M)
    lo, hi = partition(batch, rank, world)  # this rank's instances
    nb = hi - lo
    x0, tgt, Cstar = x0[lo:hi], tgt[lo:hi], Cstar_all[lo:hi]
    stream = torch.cuda.current_stream(dev)
    prob = G.chain_problem(M=M, N=N, K=K, iterations=T, lam=LAM, sigma0=SIGMA0, seed=seed, precision=PREC,
                           first_instance=lo)
    h = G.gnmppi_create(prob, nb, None, stream.cuda_stream)
    d_x0 = torch.tensor(x0.ravel(), dtype=torch.float64, device=dev)
    d_tgt = torch.tensor(tgt.ravel(), dtype=torch.float64, device=dev)
    d_U0 = torch.zeros(nb * N * 2, dtype=torch.float64, device=dev)
    d_U = torch.empty_like(d_U0)

    def one_step():
        d_U.copy_(d_U0)
        G.gnmppi_solve(h, G.MEM_DEVICE, d_x0, d_tgt, d_U, None)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = G.gnmppi_launch_count(h)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = G.gnmppi_launch_count(h) - launches0
    # per-kernel CUDA-event times of one more iteration on the solve's final
    # state (before gnmppi_cost, which reloads the inputs and resets the state)
    phases = G.gnmppi_phase_times(h, T)
    # FP64 re-evaluation of the final costs, outside the timed region, and the
    # final gather of every rank's U and costs
    Cfin = torch.empty(nb, dtype=torch.float64, device=dev)
    G.gnmppi_cost(h, G.MEM_DEVICE, d_x0, d_tgt, d_U, Cfin)
    U_all = gather_rows(d_U.view(nb, N * 2), batch, world, dev)
    C_all = gather_rows(Cfin.view(nb, 1), batch, world, dev).view(-1).cpu().numpy()
    assert U_all.shape[0] == batch and C_all.shape[0] == batch
    gap = (C_all - Cstar_all) / Cstar_all
    solved = int(np.sum(gap <= GAP))
    ms, _ = reduce_over_ranks(ms, 0, world, dev)
    ms_step = ms / args.steps
    value = solved / (ms_step / 1e3)

    F = M - 1
    roll_flops = nb * (K) * (N * chain_flops_per_step(F))  # K rollouts of N steps each
    t_roll = phases["samples"] / 1e3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s at the maximum SM clock
    achieved = roll_flops / t_roll / 1e12
    G.gnmppi_destroy(h)

    # end to end through the C ABI with host buffers: the copies of x0, the
    # targets and U0 in and of U out are inside every timed step
    prob_e = G.chain_problem(M=M, N=N, K=K, iterations=T, lam=LAM, sigma0=SIGMA0, seed=seed, precision=PREC,
                             first_instance=lo)
    he = G.gnmppi_create(prob_e, nb, None, stream.cuda_stream)
    hx0 = torch.tensor(x0.ravel(), dtype=torch.float64).pin_memory()
    htg = torch.tensor(tgt.ravel(), dtype=torch.float64).pin_memory()
    hU = torch.zeros(nb * N * 2, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        hU.zero_()
        G.gnmppi_solve(he, G.MEM_HOST, hx0, htg, hU, None)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hU.zero_()
        G.gnmppi_solve(he, G.MEM_HOST, hx0, htg, hU, None)
    e2e_s = (time.perf_counter() - t0) / args.steps
    Ce = np.zeros(nb)
    G.gnmppi_cost(he, G.MEM_HOST, hx0.numpy(), htg.numpy(), hU.numpy(), Ce)
    G.gnmppi_destroy(he)
    e2e_s, e2e_solved = reduce_over_ranks(e2e_s, int(np.sum((Ce - Cstar) / Cstar <= GAP)), world, dev)
    e2e = {"value": e2e_solved / e2e_s, "unit": "solves/s", "steps": args.steps,
           "h2d_bytes_per_step": int(8 * (batch * 4 * F + batch * 2 * F + batch * N * 2)),
           "d2h_bytes_per_step": int(8 * batch * N * 2)}

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": DTYPE, "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD + f" batch={batch}", "batch": batch, "precision": PREC_NAME,
                   "parallelism": f"instances split over {world} GPUs" if world > 1 else "single GPU",
                   "l2": "working set per iteration > L2 (dR alone %.1f GB)" % (batch * (2 * F + 2) * N * K / 2 * 4 / 1e9)},
        "solved": solved, "solved_fraction": solved / batch, "gap_median": float(np.median(gap)),
        "gap_max": float(np.max(gap)),
        "phases_ms_per_iteration": phases,
        "roofline": {"kernel": "k_samples (RK4 rollouts + residual/cost/dR/W)", "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": K_SAMPLES_TRAFFIC_B256 if nb == 256 else None,
                     "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size k_samples "
                                     "launch at 256 instances, bytes per launch",
                     "peak_note": "FP32 152 SMs x 128 lanes x 2 flop/FMA at the %.0f MHz maximum SM clock" % sm_max},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    if rank == 0:
        out["plain"] = plain_arm(args, dev, stream, prob, d_x0, d_tgt, Cstar)
        out["learned"] = learned_arm(args, dev, stream)
        out["pendulum"] = pendulum_arm(args, dev, stream)
        if not args.no_uneven:
            out["uneven"] = uneven_arm(args, dev, stream)
        out["cpu_baseline"] = cpu_baseline(args)
        if args.cpu_configs:
            out["cpu_configs"] = cpu_configs(args)
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def plain_arm(args, dev, stream, prob, d_x0, d_tgt, Cstar):
    """Plain GN-MPPI: one instance per handle and graph launch, in sequence,
    same kernels (the first instances of this rank's share)."""
    import torch

    from paper_2512_04579_gb300 import gnmppi as G

    F = M - 1
    nplain = min(args.plain, len(Cstar))
    p1 = G.chain_problem(M=M, N=N, K=K, iterations=T, lam=LAM, sigma0=SIGMA0, seed=prob.seed, precision=PREC,
                         first_instance=prob.first_instance)
    hp = G.gnmppi_create(p1, 1, None, stream.cuda_stream)
    pU = torch.zeros(N * 2, dtype=torch.float64, device=dev)
    pC = torch.empty(1, dtype=torch.float64, device=dev)
    G.gnmppi_solve(hp, G.MEM_DEVICE, d_x0[: 4 * F], d_tgt[: 2 * F], pU, None)
    torch.cuda.synchronize()
    p_solved = 0
    p0 = torch.cuda.Event(enable_timing=True)
    p1e = torch.cuda.Event(enable_timing=True)
    p_ms = 0.0
    for b in range(nplain):
        pU.zero_()
        p0.record(stream)
        G.gnmppi_solve(hp, G.MEM_DEVICE, d_x0[b * 4 * F:(b + 1) * 4 * F], d_tgt[b * 2 * F:(b + 1) * 2 * F], pU, None)
        p1e.record(stream)
        G.gnmppi_cost(hp, G.MEM_DEVICE, d_x0[b * 4 * F:(b + 1) * 4 * F], d_tgt[b * 2 * F:(b + 1) * 2 * F], pU, pC)
        torch.cuda.synchronize()
        p_ms += p0.elapsed_time(p1e)
        p_solved += int((float(pC.item()) - Cstar[b]) / Cstar[b] <= GAP)
    plain_ms = p_ms / max(1, nplain)
    G.gnmppi_destroy(hp)
    return {"solves_per_s": (p_solved / max(1, nplain)) * 1e3 / plain_ms, "ms_per_solve": plain_ms,
            "instances": nplain, "solved": p_solved,
            "note": "one instance per handle and graph launch, in sequence, same kernels"}


def oracle_iteration_seconds(threads: int, iters: int, b: int = 0):
    from oracle import oracle as O
    from paper_2512_04579_gb300 import inputs as I

    O.build()
    seed = I.BASE_SEED + 1
    x0, tgt = I.chain_instances(seed, 256, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=iters, lam=LAM, seed=seed, threads=threads)
    t0 = time.perf_counter()
    O.solve(m, opt, x0[b], tgt[b], np.zeros(m.n), SIGMA0, inst=b)
    return (time.perf_counter() - t0) / iters


def cpu_baseline(args):
    cores = os.cpu_count() or 1
    iters = max(1, args.cpu_iters)
    t_it = oracle_iteration_seconds(cores, iters)
    t_1 = oracle_iteration_seconds(1, 1)  # the same on one thread, one iteration
    _, C_gn, Cs = load_cstar()
    frac = float(np.mean((C_gn - Cs) / Cs <= GAP))
    return {"value": frac / (t_it * T), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"1 instance, {iters} of {T} iterations, {cores} OpenMP threads over samples; "
                      f"scaled by T and by the oracle's own solved fraction {frac:.3f}",
            "one_thread": {"value": frac / (t_1 * T), "unit": "solves/s", "cores": 1,
                           "sample": f"1 instance, 1 of {T} iterations, one thread"}}


def cpu_configs(args):
    """The oracle, as it stands, on this host's cores for the other
    configurations (bounded samples, scaled, each stated): the pendulum
    swing-up (one 20-iteration solve), the uneven batch (one iteration of 8 of
    its 1024 instances, scaled to the batch and 30 iterations) and the
    high-dimensional sweep (one iteration of one instance at K = 4096 per
    chain size, scaled linearly in K: rollouts and the P / S sums are linear
    in the sample count, the K-independent Jacobian / GGN work is a few %)."""
    from oracle import oracle as O
    from paper_2512_04579_gb300 import inputs as I

    O.build()
    cores = os.cpu_count() or 1
    out = {"cores": cores, "kind": "oracle"}
    # pendulum swing-up, FP64, N=50, K=256, 20 iterations
    seed = I.BASE_SEED
    x0 = I.pendulum_x0(seed, 1)[0]
    m = O.pendulum(N=50)
    res = {}
    for th in (1, cores):
        t0 = time.perf_counter()
        O.solve(m, O.Options(K=256, iterations=20, lam=LAM, seed=seed, threads=th), x0, None, np.zeros(m.n), 0.5)
        res[th] = time.perf_counter() - t0
    out["pendulum"] = {"instance_solves_per_s_1thread": 1.0 / res[1], f"instance_solves_per_s_{cores}threads":
                       1.0 / res[cores], "solves_per_s_to_gap": 0.0,
                       "sample": "one 20-iteration solve of instance 0; none of the oracle's solves reach the 1e-6 gap"}
    # uneven batch: one iteration of 8 instances
    seed = I.BASE_SEED + 2
    Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, 1024)
    ts = []
    for b in range(8):
        mb = O.chain(M=int(Ms[b]), N=int(Ns[b]))
        t0 = time.perf_counter()
        O.iteration(mb, O.Options(K=int(Ks[b]), lam=LAM, seed=seed, threads=cores), x0s[b], tgts[b], np.zeros(mb.n),
                    SIGMA0, inst=b)
        ts.append(time.perf_counter() - t0)
    t_inst = float(np.mean(ts)) * T  # one 30-iteration solve of an average instance
    _, C_gn, Cs = load_cstar(CSTAR_UNEVEN)
    frac = float(np.mean((C_gn - Cs) / Cs <= GAP))
    out["uneven"] = {"solves_per_s": frac / t_inst, "instance_solves_per_s": 1.0 / t_inst,
                     "sample": f"one iteration of instances 0-7 of the 1024, {cores} threads over samples; scaled by "
                               f"30 iterations and the oracle's own solved fraction {frac:.3f}"}
    # sweep: chain M in {16, 32, 64}, N = 200, one iteration at K = 4096
    sw = []
    seed = I.BASE_SEED + 4
    for Mc in (16, 32, 64):
        xs, tg = I.chain_instances(seed, 1, Mc)
        mc = O.chain(M=Mc, N=200)
        t0 = time.perf_counter()
        O.iteration(mc, O.Options(K=4096, lam=LAM, seed=seed, threads=cores), xs[0], tg[0], np.zeros(mc.n), SIGMA0)
        t = time.perf_counter() - t0
        sw.append({"M": Mc, "N": 200, "K": 4096, "s_per_instance_iteration": t,
                   "scaled": {str(Kc): t * Kc / 4096 for Kc in (4096, 16384, 65536)},
                   "instance_iterations_per_s": {str(Kc): 4096 / (t * Kc) for Kc in (4096, 16384, 65536)}})
    out["sweep"] = {"points": sw, "sample": f"one iteration of one instance at K = 4096, {cores} threads over "
                                            "samples; K = 16384 and 65536 scaled linearly in K"}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_iteration_seconds(cores, 1)
    ts = [oracle_iteration_seconds(cores, 1, b=i % 4) for i in range(args.steps)]
    t_it = float(np.mean(ts))
    _, C_gn, Cs = load_cstar()
    frac = float(np.mean((C_gn - Cs) / Cs <= GAP))
    value = frac / (t_it * T)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
           "config": {"workload": WORKLOAD + " (one instance per step, one iteration)", "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step one of {T} iterations of one instance; solves/s = solved "
                                      f"fraction {frac:.3f} / ({T} x mean iteration time)"},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gnmppi", choices=["gnmppi", "reference"])
    ap.add_argument("--batch", type=int, default=0, help="instances (default: every instance with a stored C*)")
    ap.add_argument("--plain", type=int, default=8, help="instances for the one-at-a-time plain arm")
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven-batch arm")
    ap.add_argument("--learned-eval", type=int, default=4096,
                    help="held-out instances of the second learned-warm-start evaluation (0: skip)")
    ap.add_argument("--cpu-configs", action="store_true",
                    help="also time the oracle on the pendulum, uneven-batch and sweep configurations")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gnmppi(args)


if __name__ == "__main__":
    main()
