"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments before touching the device."""
import os
import re

import numpy as np
import pytest

from paper_2512_04579_gb300 import build as B
from paper_2512_04579_gb300 import gnmppi as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "gnmppi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gnmppi_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert "gnmppi_create" in names and "gnmppi_solve" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(G.EXPORTS)


def test_version_and_status_strings(lib):
    assert G.gnmppi_version() == 100
    assert G.gnmppi_status_string(G.E_NOT_PD) == "GNMPPI_E_NOT_PD"
    assert G.gnmppi_status_string(12345) == "GNMPPI_E_UNKNOWN"


def _bad(**kw):
    base = dict(N=10, K=16, iterations=2)
    base.update(kw)
    return G.pendulum_problem(**base)


@pytest.mark.parametrize("kw,msg", [
    (dict(K=15), "K must be"),
    (dict(L=0), "L must be"),
    (dict(L=64), "L must be"),
    (dict(gamma=1.0), "gamma"),
    (dict(beta=0.0), "beta"),
    (dict(tau=0.0), "tau"),
    (dict(lam=-1.0), "lambda"),
    (dict(sigma0=0.0), "sigma0"),
    (dict(N=0), "N must be"),
    (dict(precision=7), "precision"),
    (dict(jac_mode=9), "jac_mode"),
    (dict(ir_steps=11), "ir_steps"),
])
def test_invalid_problems_are_rejected_before_any_device_call(lib, kw, msg):
    with pytest.raises(G.GnmppiError) as ei:
        G.gnmppi_create(_bad(**kw), 1)
    assert ei.value.status == G.E_ARG
    assert msg in G.gnmppi_last_error(None)


def test_chain_mass_count_and_linear_sizes_are_checked(lib):
    with pytest.raises(G.GnmppiError) as ei:
        G.gnmppi_create(G.chain_problem(M=70, N=10, K=16), 1)
    assert ei.value.status == G.E_ARG
    with pytest.raises(G.GnmppiError) as ei:  # group-per-rollout chains need antithetic pairs
        G.gnmppi_create(G.chain_problem(M=30, N=10, K=16, antithetic=False), 1)
    assert ei.value.status == G.E_ARG
    p = G.linear_problem(np.eye(3), np.ones((3, 1)), np.ones(3), np.ones(1), np.ones(3), N=5, K=16)
    with pytest.raises(G.GnmppiError) as ei:
        G.gnmppi_create(p, 1)
    assert ei.value.status == G.E_ARG
    with pytest.raises(G.GnmppiError) as ei:
        G.gnmppi_create(_bad(), 0)
    assert ei.value.status == G.E_ARG


def test_uneven_shapes_are_validated(lib):
    with pytest.raises(G.GnmppiError) as ei:
        G.gnmppi_create(G.chain_problem(M=5, N=10, K=16), 2, shapes=[(10, 5, 16), (10, 5, 17)])
    assert ei.value.status == G.E_ARG


def test_valid_problem_without_gpu_reports_cuda_error(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.GnmppiError) as ei:
        G.gnmppi_create(_bad(), 1)
    assert ei.value.status == G.E_CUDA
    assert "no CUDA device" in G.gnmppi_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.gnmppi_solve(None, 0, None, None, None, None, None) == G.E_ARG
    assert lib.gnmppi_step(None, 0, None, None, None, None, 0, None) == G.E_ARG
    assert lib.gnmppi_cost(None, 0, None, None, None, None) == G.E_ARG
    assert lib.gnmppi_launch_count(None) == 0
    assert lib.gnmppi_debug_inject(None, 1, 0) == G.E_ARG
    lib.gnmppi_destroy(None)
