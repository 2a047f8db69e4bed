"""Failure handling on the GPU, injected from the host (gnmppi_debug_inject):
no test faults, traps or hangs the GPU.

* The LSQ-breakdown reading of Eq. 9 (which assumes B_GGN > 0): a forced
  breakdown takes the printed Monte Carlo form for that iteration and the rest
  of the solve, exactly like the oracle with the same breakdown forced.
* Damping retries that run out end the instance with GNMPPI_E_NOT_PD.
* A bounded tensor-core wait that runs out (a barrier nothing completes)
  returns GNMPPI_E_TIMEOUT, the kernels wind down, and the same handle then
  solves exactly as a fresh one.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2512_04579_gb300 import build as B

    B.build()
    return G.load()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300)


def _problem():
    seed = 41
    M, N, K = 4, 10, 64  # n = 20, K' = 32 >= n: the LSQ form
    x0, tgt = I.chain_instances(seed, 1, M)
    return M, N, K, seed, x0[0], tgt[0]


def test_injected_lsq_breakdown_takes_the_printed_form_for_the_rest_of_the_solve():
    M, N, K, seed, x0, tgt = _problem()
    T, b = 6, 2
    m = O.chain(M=M, N=N)
    st, Uo, Uh, Ch, its = O.solve(m, O.Options(K=K, iterations=T, seed=seed, break_it=b, break_kind="system"), x0,
                                  tgt, np.zeros(m.n), 0.2)
    assert st == 0 and [it.jac_mode_used for it in its] == [0] * b + [1] * (T - b)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=T, lam=1e-3, sigma0=0.2, seed=seed)
    s = G.Solver(gp, 1)
    try:
        G.gnmppi_debug_inject(s.h, G.INJECT_LSQ_BREAKDOWN, b)
        stg, U, rep = s.solve(x0, tgt, np.zeros(m.n))
        assert stg == 0 and rep[0].status == 0 and rep[0].iterations == T
        assert rel(U, Uo) < 1e-9
        assert rep[0].C_final == pytest.approx(Ch[-1], rel=1e-10)
        # one step at the oracle's iterate U_b: the printed form, the oracle's step
        stg, Ug, r = s.step(x0, tgt, Uh[b], np.full(m.n, 0.2 * 0.7 ** (b / 2)), b)
        assert r[0].jac_mode_used == 1 and r[0].status == 0
        assert rel(s.debug("delta"), its[b].delta) < 1e-9
        # off again: the LSQ form
        G.gnmppi_debug_inject(s.h, G.INJECT_OFF, 0)
        stg, Ug, r = s.step(x0, tgt, Uh[b], np.full(m.n, 0.2 * 0.7 ** (b / 2)), b)
        assert r[0].jac_mode_used == 0
    finally:
        s.close()


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32, G.PREC_BF16])
def test_injected_breakdown_of_every_system_ends_with_not_pd(prec):
    M, N, K, seed, x0, tgt = _problem()
    gp = G.chain_problem(M=M, N=N, K=K, iterations=4, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 2)
    x2, t2 = np.concatenate([x0, x0]), np.concatenate([tgt, tgt])
    try:
        G.gnmppi_debug_inject(s.h, G.INJECT_NOT_PD, 0)
        st, U, rep = s.step(x2, t2, np.zeros(2 * 2 * N), np.full(2 * 2 * N, 0.2), 0)
        assert st == G.E_NOT_PD
        assert all(r.status == G.E_NOT_PD and r.chol_retries == 7 for r in rep)
        assert np.array_equal(U, np.zeros(2 * 2 * N))  # no step taken
        # a solve stops those instances at the injected iteration
        G.gnmppi_debug_inject(s.h, G.INJECT_NOT_PD, 2)
        st, U, rep = s.solve(x2, t2, np.zeros(2 * 2 * N))
        assert st == G.E_NOT_PD and all(r.status == G.E_NOT_PD and r.iterations == 2 for r in rep)
        G.gnmppi_debug_inject(s.h, G.INJECT_OFF, 0)
        st, U, rep = s.solve(x2, t2, np.zeros(2 * 2 * N))
        assert st == 0 and all(r.status == 0 and r.iterations == 4 for r in rep)
    finally:
        s.close()


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
def test_tensor_core_wait_that_runs_out_returns_timeout_and_the_handle_recovers(prec):
    seed = 12
    M, N, K = 6, 75, 1400  # several contraction tiles and ragged edges
    x0, tgt = I.chain_instances(seed, 2, M)
    n = 2 * N
    gp = G.chain_problem(M=M, N=N, K=K, iterations=3, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    ref = G.Solver(gp, 2)
    st, Uref, rref = ref.solve(x0, tgt, np.zeros(2 * n))
    ref.close()
    assert st == 0
    s = G.Solver(gp, 2)
    try:
        G.gnmppi_debug_inject(s.h, G.INJECT_TC_TIMEOUT, 0)
        with pytest.raises(G.GnmppiError) as e:
            s.step(x0, tgt, np.zeros(2 * n), np.full(2 * n, 0.2), 0)
        assert e.value.status == G.E_TIMEOUT
        G.gnmppi_debug_inject(s.h, G.INJECT_TC_TIMEOUT, 1)  # inside a graph-captured solve
        with pytest.raises(G.GnmppiError) as e:
            s.solve(x0, tgt, np.zeros(2 * n))
        assert e.value.status == G.E_TIMEOUT
        G.gnmppi_debug_inject(s.h, G.INJECT_OFF, 0)
        st, U, rep = s.solve(x0, tgt, np.zeros(2 * n))
        assert st == 0
        assert np.array_equal(U, Uref)
        assert [r.C_final for r in rep] == [r.C_final for r in rref]
    finally:
        s.close()


def test_timeout_injection_needs_the_tensor_core_path():
    M, N, K, seed, x0, tgt = _problem()
    s = G.Solver(G.chain_problem(M=M, N=N, K=K, iterations=1, seed=seed), 1)
    try:
        with pytest.raises(G.GnmppiError):
            G.gnmppi_debug_inject(s.h, G.INJECT_TC_TIMEOUT, 0)
        with pytest.raises(G.GnmppiError):
            G.gnmppi_debug_inject(s.h, 7, 0)
    finally:
        s.close()
