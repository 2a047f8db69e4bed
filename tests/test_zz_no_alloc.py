"""The allocation-free softmin entry point against the solver's own softmin.

gnmppi_softmin_noalloc is for callers that cannot allocate device memory when
they call in (a real-time controller with a fixed per-cycle latency budget, or
a host that grants a fixed memory budget up front).  Its scratch is a fixed
device array shared by every call; this test checks two calls in a row -- the
second on a different sample set, so stale scratch from the first call would
show -- against the weights statistics and weighted mean perturbation that
gnmppi_step reports for the same samples, within the FP64 parity tolerance.
"""
import numpy as np
import pytest

from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _step_outputs(K, seed, it):
    """One FP64 Algorithm-1 iteration through the existing entry point."""
    N = 50
    x0 = I.pendulum_x0(seed, 1)[0]
    s = G.Solver(G.pendulum_problem(N=N, K=K, iterations=1, lam=1e-3, sigma0=0.5, seed=seed, tau=2.0), 1)
    st, U, rep = s.step(x0, None, np.zeros(N), np.full(N, 0.5), it)
    assert st == 0
    out = dict(C=s.debug("C"), W=s.debug("W"), mppi=s.debug("mppi"), rep=rep[0], n=N, Kp=K // 2)
    s.close()
    return out


def test_softmin_noalloc_matches_step_on_two_calls_in_a_row():
    import torch

    from paper_2512_04579_gb300 import build as B

    B.build()
    G.load()
    ref = [_step_outputs(512, 3, 0), _step_outputs(128, 4, 1)]  # larger set first, then a smaller one
    for r in ref:
        C = torch.tensor(r["C"], dtype=torch.float64, device="cuda")
        W = torch.tensor(r["W"], dtype=torch.float64, device="cuda")
        mppi = torch.full((r["n"],), np.nan, dtype=torch.float64, device="cuda")
        stats = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
        st, msg = G.gnmppi_softmin_noalloc(C, W, r["Kp"], r["n"], True, 2.0, mppi, stats,
                                           torch.cuda.current_stream().cuda_stream)
        assert st == G.OK, msg
        torch.cuda.synchronize()
        m = mppi.cpu().numpy()
        sv = stats.cpu().numpy()
        assert np.linalg.norm(m - r["mppi"]) <= TOL * np.linalg.norm(r["mppi"])
        rep = r["rep"]
        np.testing.assert_allclose(sv, [rep.c_min, rep.sum_w, rep.sum_w2, rep.ess], rtol=TOL)


def test_softmin_noalloc_rejects_counts_beyond_its_scratch():
    import torch

    from paper_2512_04579_gb300 import build as B

    B.build()
    G.load()
    C = torch.zeros(2, dtype=torch.float64, device="cuda")
    st, msg = G.gnmppi_softmin_noalloc(C, C, 65537, 1, True, 1.0, C, C)
    assert st == G.E_ARG and "65536" in msg
