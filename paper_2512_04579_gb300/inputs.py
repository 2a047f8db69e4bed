"""Seeded synthetic inputs for the GN-MPPI workloads.

This module only draws problem data (initial states, targets, per-instance
sizes) with numpy's counter-based Philox generator.  It holds none of the
method's arithmetic, so the CUDA library's callers and the CPU oracle's tests
take their inputs from the same place.

Workloads (all synthetic; the paper measures on no dataset):
  * pendulum swing-up: x0 ~ U([-0.5, 0.5]^2);
  * chain of M point masses hanging in a vertical plane (mass 0 fixed at
    the origin): rest state = static hanging equilibrium; target = the rest
    positions rotated about mass 0 by phi ~ U(pi/16, pi/8); x0 = rest state
    + N(0, 0.05^2) on every entry (positions and velocities);
  * uneven batches: M ~ U{4..16}, N ~ U{40..160}, K ~ U{512,1024,2048,4096}.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2512045790
CHAIN_DEFAULTS = dict(mass=0.1, k=10.0, k3=1.0, damping=0.05, gravity=9.81)
PHI_RANGE = (np.pi / 16, np.pi / 8)
WARM_PHI = 3 * np.pi / 32  # the one target of the warm-start workload
TRAIN_STREAM, EVAL_STREAM = 0, 1  # initial-state streams of its training and evaluation sets


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1), counter=int(stream)))


def pendulum_x0(seed: int, batch: int) -> np.ndarray:
    """(batch, 2) initial states [theta, omega] ~ U([-0.5, 0.5]^2)."""
    return rng(seed, 1).uniform(-0.5, 0.5, size=(batch, 2))


def chain_rest_positions(M: int, mass=0.1, k=10.0, k3=1.0, gravity=9.81, **_) -> np.ndarray:
    """(M-1, 2) static hanging equilibrium of the free masses.

    Link j (between masses j-1 and j) carries the weight of masses j..M-1,
    T_j = (M - j) mass gravity, and stretches by the real root d_j of
    k d + k3 d^3 = T_j beyond the rest length 1/(M-1); the chain hangs
    straight down from the fixed mass 0 at the origin.
    """
    l0 = 1.0 / (M - 1)
    p = np.zeros((M - 1, 2))
    y = 0.0
    for j in range(1, M):
        T = (M - j) * mass * gravity
        if k3 != 0.0:
            roots = np.roots([k3, 0.0, k, -T])
            d = float(np.real(roots[np.argmin(np.abs(np.imag(roots)))]))
        else:
            d = T / k
        y -= l0 + d
        p[j - 1] = (0.0, y)
    return p


def chain_rest_state(M: int, **params) -> np.ndarray:
    q = dict(CHAIN_DEFAULTS, **params)
    return np.concatenate([chain_rest_positions(M, **q).ravel(), np.zeros(2 * (M - 1))])


def chain_target(M: int, phi: float, **params) -> np.ndarray:
    """Rest positions rotated about mass 0 by phi, flattened (2(M-1),)."""
    q = dict(CHAIN_DEFAULTS, **params)
    p = chain_rest_positions(M, **q)
    c, s = np.cos(phi), np.sin(phi)
    R = np.array([[c, -s], [s, c]])
    return (p @ R.T).ravel()


def chain_instances(seed: int, batch: int, M: int, stream: int = 0, x0_std: float = 0.05, **params):
    """x0 (batch, 4(M-1)) and targets (batch, 2(M-1)) for `batch` chain instances."""
    g = rng(seed, 2 + 16 * stream)
    phi = g.uniform(PHI_RANGE[0], PHI_RANGE[1], size=batch)
    rest = chain_rest_state(M, **params)
    x0 = rest[None, :] + g.normal(0.0, x0_std, size=(batch, rest.size))
    tgt = np.stack([chain_target(M, p, **params) for p in phi])
    return x0, tgt


def stream_rng(seed: int, stream: int) -> np.random.Generator:
    """Philox stream whose counter starts with the stream id in its third word,
    so streams of one key never overlap."""
    return np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1),
                                                counter=np.array([0, 0, int(stream) + 1, 0], dtype=np.uint64)))


def chain_fixed_target_states(seed: int, batch: int, M: int, phi: float, stream: int = 0, x0_std: float = 0.05,
                              **params):
    """Initial states around the rest state for one fixed target (warm-start
    workload); training and evaluation sets come from disjoint streams."""
    g = stream_rng(seed, stream)
    rest = chain_rest_state(M, **params)
    return rest[None, :] + g.normal(0.0, x0_std, size=(batch, rest.size)), chain_target(M, phi, **params)


def uneven_batch(seed: int, batch: int, M_range=(4, 16), N_range=(40, 160), K_choices=(512, 1024, 2048, 4096)):
    """Per-instance (M, N, K) of an uneven batch."""
    g = rng(seed, 4)
    M = g.integers(M_range[0], M_range[1] + 1, size=batch)
    N = g.integers(N_range[0], N_range[1] + 1, size=batch)
    K = np.asarray(K_choices)[g.integers(0, len(K_choices), size=batch)]
    return M, N, K


def uneven_chain_instances(seed: int, batch: int):
    """Uneven batch of chain instances: per instance (M, N, K), x0 = rest state
    + N(0, 0.05^2) and a target rotated by phi ~ U(pi/16, pi/8), each instance
    from its own Philox stream."""
    M, N, K = uneven_batch(seed, batch)
    x0s, tgts = [], []
    for b in range(batch):
        g = stream_rng(seed, 1000 + b)
        phi = g.uniform(PHI_RANGE[0], PHI_RANGE[1])
        rest = chain_rest_state(int(M[b]))
        x0s.append(rest + g.normal(0.0, 0.05, size=rest.size))
        tgts.append(chain_target(int(M[b]), phi))
    return M, N, K, x0s, tgts
