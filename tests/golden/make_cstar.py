"""Write the reference optima C* of the chain benchmark instances.

Calls only the FP64 CPU oracle.  Two seeded workloads (chain M=10, N=100,
K=2048, 30 iterations, sigma0 0.2, lambda 1e-3):
  chain_m10        targets rotated by phi ~ U(pi/16, pi/8), seed 2512045790 + 1
  chain_m10_fixed  one target (phi = 3 pi / 32), held-out initial states of the
                   warm-start evaluation stream, seed 2512045790 + 3
  chain_uneven     per-instance M ~ U{4..16}, N ~ U{40..160}, K ~ U{512..4096}
                   (inputs.uneven_chain_instances), seed 2512045790 + 2
  pendulum         the swing-up of configuration 0: x0 ~ U([-0.5, 0.5]^2),
                   N=50, K=256, sigma0 0.5, lambda 1e-3, 20 iterations,
                   seed 2512045790 + 0 (instance b draws noise stream b)
For each instance b:
  C_gn  = cost after the oracle's 30-iteration GN-MPPI solve (Algorithm 1),
  C*    = cost after polishing that solution with Method A (central-FD GGN,
          Sec. 5) until the FD gradient falls below 1e-10 or no step helps.
Output: <workload>_cstar.txt (one line per instance: b C_gn C*).

Usage: python tests/golden/make_cstar.py [batch] [processes] [workload]
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

M, N, K, T, SIGMA0, LAM = 10, 100, 2048, 30, 0.2, 1e-3


def instances(workload, batch):
    """(seed, x0 [batch][nx], targets [batch][2(M-1)]) of a workload."""
    import numpy as np

    from paper_2512_04579_gb300 import inputs as I

    if workload == "chain_m10":
        seed = I.BASE_SEED + 1
        x0, tgt = I.chain_instances(seed, batch, M)
        return seed, x0, tgt
    seed = I.BASE_SEED + 3
    x0, t = I.chain_fixed_target_states(seed, batch, M, I.WARM_PHI, stream=I.EVAL_STREAM)
    return seed, x0, np.tile(t, (batch, 1))


def one(args):
    import numpy as np

    from oracle import oracle as O
    from paper_2512_04579_gb300 import inputs as I

    b, workload = args
    if workload == "pendulum":
        seed = I.BASE_SEED
        x0 = I.pendulum_x0(seed, BATCH)
        m = O.pendulum(N=50)
        opt = O.Options(K=256, iterations=20, lam=LAM, seed=seed, threads=1)
        st, U, Uh, Ch, its = O.solve(m, opt, x0[b], None, np.zeros(m.n), 0.5, inst=b)
        stA, UA, CA, itA = O.method_a(m, x0[b], None, U.copy(), max_iter=300, lam=LAM)
        return b, Ch[-1], min(CA, Ch[-1])
    if workload == "chain_uneven":
        seed = I.BASE_SEED + 2
        Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, BATCH)
        m = O.chain(M=int(Ms[b]), N=int(Ns[b]))
        opt = O.Options(K=int(Ks[b]), iterations=T, lam=LAM, seed=seed, threads=1)
        st, U, Uh, Ch, its = O.solve(m, opt, x0s[b], tgts[b], np.zeros(m.n), SIGMA0, inst=b)
        stA, UA, CA, itA = O.method_a(m, x0s[b], tgts[b], U.copy(), max_iter=300, lam=LAM)
        return b, Ch[-1], min(CA, Ch[-1])
    seed, x0, tgt = instances(workload, BATCH)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=T, lam=LAM, seed=seed, threads=1)
    st, U, Uh, Ch, its = O.solve(m, opt, x0[b], tgt[b], np.zeros(m.n), SIGMA0, inst=b)
    stA, UA, CA, itA = O.method_a(m, x0[b], tgt[b], U.copy(), max_iter=300, lam=LAM)
    return b, Ch[-1], min(CA, Ch[-1])


BATCH = int(sys.argv[1]) if len(sys.argv) > 1 else 256

if __name__ == "__main__":
    procs = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count()
    workload = sys.argv[3] if len(sys.argv) > 3 else "chain_m10"
    from oracle import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        rows = sorted(pool.map(one, [(b, workload) for b in range(BATCH)], chunksize=1))
    out = os.path.join(HERE, f"{workload}_cstar.txt")
    seed_note = {"chain_m10": "2512045790+1", "chain_m10_fixed": "2512045790+3 (fixed target, eval stream)",
                 "chain_uneven": "2512045790+2 (per-instance M, N, K)", "pendulum": "2512045790+0"}[workload]
    if workload == "pendulum":
        head = "pendulum swing-up N=50 K=256 T=20 sigma0=0.5"
    elif workload == "chain_uneven":
        head = f"chain M, N, K per instance (inputs.uneven_chain_instances) T={T} sigma0={SIGMA0}"
    else:
        head = f"chain M={M} N={N} K={K} T={T} sigma0={SIGMA0}"
    with open(out, "w") as f:
        f.write(f"# {workload}: {head} lambda={LAM} seed={seed_note} batch={BATCH}\n")
        f.write("# written by tests/golden/make_cstar.py from the FP64 oracle: b C_gn C_star\n")
        for b, cg, cs in rows:
            f.write(f"{b} {cg:.17g} {cs:.17g}\n")
    print("wrote", out)
