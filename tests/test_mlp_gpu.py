"""The learned warm start's CUDA kernels (through the C ABI) against the FP64
oracle: forward pass, Gaussian-NLL loss and gradient, one Adam step, and the
warm-start outputs.  FP32 weights: 1e-5 / 1e-4; BF16 weights: 2e-2."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_04579_gb300 import gnmppi as G

pytestmark = pytest.mark.gpu

DIMS = [8, 48, 40, 30]  # n_mu = 20, nu = 2: 10 per-step scales; 48 > 32 and 40 span ragged GEMM tiles


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2512_04579_gb300 import build as B

    B.build()
    return G.load()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _setup(seed=0, B=70):
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(1, len(DIMS)):
        ps.append(rng.normal(0, 1.0 / math.sqrt(DIMS[l - 1]), size=DIMS[l] * DIMS[l - 1]))
        ps.append(rng.normal(0, 0.1, size=DIMS[l]))
    params = np.concatenate(ps)
    X = rng.normal(1.0, 2.0, size=(B, DIMS[0]))
    T = rng.normal(0, 1.0, size=(B, 20))
    xm = X.mean(0)
    xs = X.std(0)
    return params, X, T, xm, xs


@pytest.mark.parametrize("bf16,tol", [(False, 1e-5), (True, 2e-2)])
def test_forward_matches_oracle(bf16, tol):
    params, X, T, xm, xs = _setup()
    m = G.Mlp(DIMS, nu=2, weights_bf16=bf16, max_batch=128)
    m.set_params(params)
    m.set_normalization(xm, xs, 1.0)
    Y = m.forward(X)
    m.close()
    assert rel(Y, O.mlp_forward(DIMS, params, xm, xs, X)) < tol


@pytest.mark.parametrize("bf16,tol", [(False, 1e-4), (True, 3e-2)])
def test_loss_and_gradient_match_oracle(bf16, tol):
    params, X, T, xm, xs = _setup(1)
    m = G.Mlp(DIMS, nu=2, weights_bf16=bf16, max_batch=128)
    m.set_params(params)
    m.set_normalization(xm, xs, 1.0)
    loss, g = m.loss_grad(X, T)
    m.close()
    lo, go = O.mlp_loss_grad(DIMS, params, xm, xs, X, T, 2)
    assert loss == pytest.approx(lo, rel=tol)
    assert rel(g, go) < tol


def test_adam_step_matches_oracle():
    import torch

    params, X, T, xm, xs = _setup(2)
    m = G.Mlp(DIMS, nu=2, weights_bf16=False, max_batch=128)
    m.set_params(params)
    m.set_normalization(xm, xs, 1.0)
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    dT = torch.tensor(T, dtype=torch.float64, device="cuda")
    for _ in range(3):
        m.train_step(dX, dT, X.shape[0], 1e-2)
    p_gpu = m.get_params()
    m.close()
    p = params.copy()
    mo = np.zeros_like(p)
    vo = np.zeros_like(p)
    for t in range(1, 4):
        _, g = O.mlp_loss_grad(DIMS, p, xm, xs, X, T, 2)
        O.mlp_adam(p, g, mo, vo, t, lr=1e-2)
    # FP32 parameters: compare the moves, which are O(lr)
    assert rel(p_gpu - params, p - params) < 1e-3


def test_warm_start_scales_outputs():
    import torch

    params, X, T, xm, xs = _setup(3, B=16)
    m = G.Mlp(DIMS, nu=2, weights_bf16=False, max_batch=128)
    m.set_params(params)
    m.set_normalization(xm, xs, 2.5)
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    U0 = torch.zeros((16, 20), dtype=torch.float64, device="cuda")
    sig = torch.zeros((16, 20), dtype=torch.float64, device="cuda")
    m.warm_start(dX, 16, U0, sig)
    m.close()
    Y = O.mlp_forward(DIMS, params, xm, xs, X)
    assert rel(U0.cpu().numpy(), 2.5 * Y[:, :20]) < 1e-5
    assert rel(sig.cpu().numpy(), 2.5 * np.exp(np.repeat(Y[:, 20:], 2, axis=1))) < 1e-5


def test_training_reduces_loss():
    """A few hundred Adam steps on a learnable map lower the loss."""
    import torch

    rng = np.random.default_rng(4)
    X = rng.normal(size=(512, 8))
    A = rng.normal(size=(8, 20)) / 3
    T = np.tanh(X @ A)
    params, _, _, _, _ = _setup(5)
    m = G.Mlp(DIMS, nu=2, weights_bf16=True, max_batch=512)
    m.set_params(params)
    m.set_normalization(X.mean(0), X.std(0), 1.0)
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    dT = torch.tensor(T, dtype=torch.float64, device="cuda")
    first = m.train_step(dX, dT, 512, 3e-3)
    for _ in range(400):
        last = m.train_step(dX, dT, 512, 3e-3)
    m.close()
    assert last < first - 2.0


# ------------------------------------------------ the production network ---
FULL = [36, 256, 256, 256, 300]  # the warm-start network: n_mu = 200, 100 per-step scales


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), as the library rounds its weights."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)


def _full_setup(seed, B):
    rng = np.random.default_rng(seed)
    ps, wmask = [], []
    for l in range(1, len(FULL)):
        ps.append(rng.normal(0, 1.0 / math.sqrt(FULL[l - 1]), size=FULL[l] * FULL[l - 1]))
        wmask.append(np.ones(FULL[l] * FULL[l - 1], bool))
        ps.append(rng.normal(0, 0.1, size=FULL[l]))
        wmask.append(np.zeros(FULL[l], bool))
    params, wmask = np.concatenate(ps), np.concatenate(wmask)
    X = rng.normal(1.0, 2.0, size=(B, FULL[0]))
    T = rng.normal(0, 1.0, size=(B, 200))
    return params, wmask, X, T, X.mean(0), X.std(0)


@pytest.mark.parametrize("bf16", [False, True])
def test_full_width_network_matches_oracle(bf16):
    """36-256-256-256-300 at batch 1024 (8 x 2-3 tiles of 128 x 128 per
    product, K up to 1024 in the weight gradients): forward outputs, loss and
    every gradient entry against the FP64 oracle.  With BF16 weights the
    oracle is evaluated at the same BF16-rounded weight matrices (biases stay
    FP32), the products the library forms, so both modes are held to the
    FP32-level accuracy of the three-pass BF16 products: operands carry
    2^-17 relative, the dropped remainder x remainder term 2^-18."""
    B = 1024
    params, wmask, X, T, xm, xs = _full_setup(11, B)
    ref = np.where(wmask, bf16_round(params), params) if bf16 else params
    m = G.Mlp(FULL, nu=2, weights_bf16=bf16, max_batch=B)
    m.set_params(params)
    m.set_normalization(xm, xs, 1.0)
    Y = m.forward(X)
    loss, g = m.loss_grad(X, T)
    m.close()
    Yo = O.mlp_forward(FULL, ref, xm, xs, X)
    lo, go = O.mlp_loss_grad(FULL, ref, xm, xs, X, T, 2)
    assert rel(Y, Yo) < 3e-5
    assert np.max(np.abs(Y - Yo)) < 1e-4 * np.max(np.abs(Yo))
    assert loss == pytest.approx(lo, rel=3e-5)
    assert rel(g, go) < 3e-4
    # per layer: every weight and bias block, so that a stale or missing
    # tile of any product fails
    off = 0
    for l in range(1, len(FULL)):
        for size in (FULL[l] * FULL[l - 1], FULL[l]):
            blk = slice(off, off + size)
            assert rel(g[blk], go[blk]) < 3e-4, (l, size)
            off += size


def test_full_width_training_step_matches_oracle():
    """Two Adam steps of the production network on a 1024 batch, FP32
    weights, against the oracle's Adam on its own gradients."""
    import torch

    B = 1024
    params, wmask, X, T, xm, xs = _full_setup(12, B)
    m = G.Mlp(FULL, nu=2, weights_bf16=False, max_batch=B)
    m.set_params(params)
    m.set_normalization(xm, xs, 1.0)
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    dT = torch.tensor(T, dtype=torch.float64, device="cuda")
    for _ in range(2):
        m.train_step(dX, dT, B, 1e-3)
    p_gpu = m.get_params()
    m.close()
    p = params.copy()
    mo, vo = np.zeros_like(p), np.zeros_like(p)
    g1 = None
    for t in range(1, 3):
        _, gr = O.mlp_loss_grad(FULL, p, xm, xs, X, T, 2)
        g1 = gr if g1 is None else g1
        O.mlp_adam(p, gr, mo, vo, t, lr=1e-3)
    # Adam's first moves are ~lr sign(g): an entry whose gradient is near zero
    # flips with any rounding of g.  Where |g| is at least 1 % of its RMS (some
    # 300 times the gradient error measured above) the moves must agree.
    sure = np.abs(g1) >= 1e-2 * np.sqrt(np.mean(g1 ** 2))
    assert sure.mean() > 0.95
    assert rel((p_gpu - params)[sure], (p - params)[sure]) < 1e-3


def test_training_resumes_exactly_from_a_saved_state():
    """Three Adam steps, save (parameters, both moments, step count), two more
    steps; a fresh handle given the saved state and the same two steps ends
    bitwise at the same parameters and moments."""
    import torch

    params, X, T, xm, xs = _setup(6)
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    dT = torch.tensor(T, dtype=torch.float64, device="cuda")
    a = G.Mlp(DIMS, nu=2, weights_bf16=True, max_batch=128)
    a.set_params(params)
    a.set_normalization(xm, xs, 1.0)
    for _ in range(3):
        a.train_step(dX, dT, X.shape[0], 1e-2)
    saved = a.get_state()
    assert saved[3] == 3
    for _ in range(2):
        a.train_step(dX, dT, X.shape[0], 1e-2)
    end_a = a.get_state()
    a.close()
    b = G.Mlp(DIMS, nu=2, weights_bf16=True, max_batch=128)
    b.set_normalization(xm, xs, 1.0)
    b.set_state(*saved)
    for _ in range(2):
        b.train_step(dX, dT, X.shape[0], 1e-2)
    end_b = b.get_state()
    b.close()
    for x, y in zip(end_a[:3], end_b[:3]):
        assert np.array_equal(x, y)
    assert end_a[3] == end_b[3] == 5
    # set_params, unlike set_state, starts a new optimisation (moments reset)
    assert not np.array_equal(saved[1], np.zeros_like(saved[1]))
