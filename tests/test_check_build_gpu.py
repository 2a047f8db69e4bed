"""The bounds-check build (libgnmppi_check.so, compiled with -DGNMPPI_CHECK):
every checked store of the hot kernels -- rollout emission (dR, W, sample
costs), line-search residuals, the tensor-core contraction, Gram and MLP
epilogues, the step and the update -- tests its index against the
instance's block and counts (and skips) any that falls outside, without a
trap.  Small cases of every kernel family run in a subprocess against each
library: the check build must count no offence and give the normal build's
results bitwise.  (A memory checker is not available on this machine; this is
its stand-in for the library's own indexing.)"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I
G.load(sys.argv[1])
out = {}
seed = I.BASE_SEED
x0 = I.pendulum_x0(seed, 1)[0]
s = G.Solver(G.pendulum_problem(N=20, K=64, iterations=3, lam=1e-3, sigma0=0.5, seed=seed), 1)
out["pendulum_fp64"] = s.solve(x0, None, np.zeros(20))[1].tolist()
s.close()
for name, M, N, K, prec in (("chain_fp32", 6, 20, 256, G.PREC_FP32), ("chain_bf16", 6, 20, 256, G.PREC_BF16),
                            ("chain_group_bf16", 20, 10, 96, G.PREC_BF16), ("chain_group_fp64", 20, 8, 64, G.PREC_FP64)):
    xs, tg = I.chain_instances(seed + M, 2, M)
    s = G.Solver(G.chain_problem(M=M, N=N, K=K, iterations=3, lam=1e-3, sigma0=0.2, seed=seed, precision=prec), 2)
    out[name] = s.solve(xs, tg, np.zeros(2 * 2 * N))[1].tolist()
    s.close()
shapes = [(20, 4, 64), (33, 6, 130), (12, 3, 200)]
xs, tgs = [], []
for i, (N, M, K) in enumerate(shapes):
    a, b = I.chain_instances(seed + 40 + i, 1, M)
    xs.append(a[0]); tgs.append(b[0])
s = G.Solver(G.chain_problem(M=4, N=20, K=64, iterations=2, lam=1e-3, sigma0=0.2, seed=seed,
                             precision=G.PREC_FP32), 3, shapes=shapes)
out["uneven_fp32"] = s.solve(np.concatenate(xs), np.concatenate(tgs), np.zeros(sum(2 * N for N, _, _ in shapes)))[1].tolist()
s.close()
dims = [8, 48, 40, 30]
rng = np.random.default_rng(0)
ps = []
for l in range(1, len(dims)):
    ps += [rng.normal(0, 0.3, size=dims[l] * dims[l - 1]), rng.normal(0, 0.1, size=dims[l])]
X = rng.normal(size=(70, 8)); T = rng.normal(size=(70, 20))
m = G.Mlp(dims, nu=2, weights_bf16=True, max_batch=128)
m.set_params(np.concatenate(ps)); m.set_normalization(X.mean(0), X.std(0), 1.0)
out["mlp_forward"] = m.forward(X).ravel().tolist()
out["mlp_grad"] = m.loss_grad(X, T)[1].tolist()
m.close()
out["offences"] = int(G.load().gnmppi_check_count())
print(json.dumps(out))
"""


def _run(lib_path):
    r = subprocess.run([sys.executable, "-c", CASES, lib_path, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_check_build_counts_no_out_of_range_store_and_matches_the_normal_build():
    from paper_2512_04579_gb300 import build as B

    normal = _run(B.build())
    checked = _run(B.build(check=True))
    assert normal["offences"] == -1  # the normal build has no checks
    assert checked["offences"] == 0
    for k, v in normal.items():
        if k != "offences":
            assert checked[k] == v, k
