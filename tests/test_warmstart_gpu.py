"""What the learned warm start gains: an MLP trained (on the GPU, by the
library's own kernels) on 16384 plain GN-MPPI solutions of one chain target
warm-starts held-out instances so that GN-MPPI with K = 512 and 5 iterations
lands much closer to the plain solution (K = 2048, 30 iterations, the
reference of the cost gap) than the same budget from a cold start."""
import numpy as np
import pytest

from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_2512_04579_gb300 import build as B
    from paper_2512_04579_gb300 import warmstart as W

    B.build()
    G.load()
    X, U = W.make_dataset(16384, chunk=4096)
    m, meta, hist = W.train(X, U, epochs=100, batch=512, lr=2e-3)
    yield m, hist
    m.close()


def _costs(h, dx, dt, dU, batch):
    import torch

    C = torch.empty(batch, dtype=torch.float64, device="cuda")
    G.gnmppi_cost(h, G.MEM_DEVICE, dx, dt, dU, C)
    return C.cpu().numpy()


def test_training_loss_decreases(trained):
    m, hist = trained
    assert hist[-1] < hist[0] - 1.0


def test_warm_start_beats_cold_start_at_equal_budget(trained):
    import torch

    from paper_2512_04579_gb300 import warmstart as W

    m, _ = trained
    B = 64
    x0, tgt = I.chain_fixed_target_states(W.SEED, B, W.M, I.WARM_PHI, stream=I.EVAL_STREAM)
    dx = torch.tensor(x0.ravel(), dtype=torch.float64, device="cuda")
    dt = torch.tensor(np.tile(tgt, (B, 1)).ravel(), dtype=torch.float64, device="cuda")
    # reference: plain GN-MPPI, cold start, K = 2048, 30 iterations
    hp = G.gnmppi_create(W.chain_problem(2048, 30), B)
    Up = torch.zeros(B * W.NMU, dtype=torch.float64, device="cuda")
    G.gnmppi_solve(hp, G.MEM_DEVICE, dx, dt, Up, None)
    Cref = _costs(hp, dx, dt, Up, B)
    # cold start with the warm-start budget: K = 512, 5 iterations
    hc = G.gnmppi_create(W.chain_problem(512, 5), B)
    Uc = torch.zeros(B * W.NMU, dtype=torch.float64, device="cuda")
    G.gnmppi_solve(hc, G.MEM_DEVICE, dx, dt, Uc, None)
    Cc = _costs(hp, dx, dt, Uc, B)
    # warm start, same budget
    Uw = torch.zeros(B * W.NMU, dtype=torch.float64, device="cuda")
    sig = torch.zeros(B * W.NMU, dtype=torch.float64, device="cuda")
    m.warm_start(dx, B, Uw, sig, W.SIGMA_MIN, W.SIGMA_MAX)
    G.gnmppi_solve(hc, G.MEM_DEVICE, dx, dt, Uw, sig)
    Cw = _costs(hp, dx, dt, Uw, B)
    G.gnmppi_destroy(hp)
    G.gnmppi_destroy(hc)
    gap_cold = np.median((Cc - Cref) / Cref)
    gap_warm = np.median((Cw - Cref) / Cref)
    print(f"median gap to plain GN-MPPI: cold {gap_cold:.3e}, warm {gap_warm:.3e}")
    assert gap_warm < 0.1 * gap_cold
    assert gap_warm < 1e-6


def test_learned_solver_with_fallback_matches_plain(trained):
    import torch

    from paper_2512_04579_gb300 import warmstart as W

    m, _ = trained
    B = 64
    x0, tgt = I.chain_fixed_target_states(W.SEED, B, W.M, I.WARM_PHI, stream=I.EVAL_STREAM)
    dx = torch.tensor(x0.ravel(), dtype=torch.float64, device="cuda")
    dt = torch.tensor(np.tile(tgt, (B, 1)).ravel(), dtype=torch.float64, device="cuda")
    hp = G.gnmppi_create(W.chain_problem(2048, 30), B)
    Up = torch.zeros(B * W.NMU, dtype=torch.float64, device="cuda")
    G.gnmppi_solve(hp, G.MEM_DEVICE, dx, dt, Up, None)
    Cref = _costs(hp, dx, dt, Up, B)
    ls = W.LearnedSolver(m, B)
    Ul = torch.zeros(B * W.NMU, dtype=torch.float64, device="cuda")
    nfb = ls.solve(dx, dt, Ul)
    ls.close()
    Cl = _costs(hp, dx, dt, Ul, B)
    G.gnmppi_destroy(hp)
    gap = (Cl - Cref) / Cref
    print(f"fallback {nfb}/{B}, median gap {np.median(gap):.3e}, max {gap.max():.3e}")
    assert np.median(gap) < 1e-6
