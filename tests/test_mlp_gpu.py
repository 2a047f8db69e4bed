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
