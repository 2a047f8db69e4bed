"""Pins for the FP64 CPU oracle: each test checks it against something other than
itself -- published known-answer values, closed forms, textbook/library
routines, brute force on tiny inputs, or invariants -- so that a dropped term,
a wrong sign or index, or a transposed operand fails at least one of them.

CPU only (no GPU marker).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_04579_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ---
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t, 16) for t in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox(ctr, key).tolist() == out


def test_uniform53_range_and_order():
    assert O.uniform53(0, 0) == 2.0 ** -54
    assert O.uniform53(0xFFFFFFFF, 0xFFFFFFFF) <= 1.0
    vals = [O.uniform53(h, l) for h, l in [(0, 0), (0, 1 << 11), (1, 0), (1 << 31, 0), (0xFFFFFFFF, 0)]]
    assert all(a < b for a, b in zip(vals, vals[1:]))
    # 53 bits: consecutive codes differ by exactly 2^-53
    assert O.uniform53(5, 7 << 11) - O.uniform53(5, 6 << 11) == 2.0 ** -53


def test_normals_are_standard_normal():
    from scipy import stats

    z = np.concatenate([O.normals(123, 0, it, m, 100) for it in range(4) for m in range(500)])
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the cos/sin halves of one Box-Muller pair are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.02
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.1


def test_noise_streams_are_distinct_and_reproducible():
    a = O.normals(7, 0, 0, 0, 16)
    assert np.array_equal(a, O.normals(7, 0, 0, 0, 16))
    for args in [(8, 0, 0, 0), (7, 1, 0, 0), (7, 0, 1, 0), (7, 0, 0, 1)]:
        assert not np.allclose(a, O.normals(*args, 16))
    # a prefix of a longer draw is the shorter draw (counter = j/2)
    assert np.array_equal(O.normals(7, 0, 0, 0, 5), a[:5])


# ------------------------------------------------------------------ RK4 ---
def test_rk4_equals_fourth_order_taylor_map_on_linear_ode():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(4, 4))
    B = rng.normal(size=(4, 2))
    h = 0.05
    m = O.lincont(A, B, h)
    x = rng.normal(size=4)
    u = rng.normal(size=2)
    Phi = sum(np.linalg.matrix_power(h * A, i) / math.factorial(i) for i in range(5))
    Gam = sum(h ** i * np.linalg.matrix_power(A, i - 1) / math.factorial(i) for i in range(1, 5)) @ B
    np.testing.assert_allclose(O.rk4_step(m, x, u), Phi @ x + Gam @ u, rtol=1e-13, atol=1e-13)


def _pendulum_end_state(dt, T=2.0):
    m = O.pendulum(N=int(round(T / dt)), dt=dt, b=0.0)
    return O.rollout(m, [2.0, 0.0], np.zeros(m.n))[-1]


def test_pendulum_global_error_is_fourth_order():
    # RK4's global error shrinks by 2^4 when the step halves (reference: h/64)
    ref = _pendulum_end_state(0.05 / 64)
    e1 = np.linalg.norm(_pendulum_end_state(0.05) - ref)
    e2 = np.linalg.norm(_pendulum_end_state(0.025) - ref)
    assert 12.0 < e1 / e2 < 20.0
    # and energy is conserved up to that error
    x = _pendulum_end_state(0.025)
    assert abs(0.5 * x[1] ** 2 - 9.81 * math.cos(x[0]) + 9.81 * math.cos(2.0)) < 1e-4


def test_pendulum_rhs_terms():
    m = O.pendulum(g=9.81, l=2.0, m=3.0, b=0.7)
    xd = O.deriv(m, [0.3, -1.2], [0.9])
    assert xd[0] == -1.2
    assert xd[1] == pytest.approx(-(9.81 / 2.0) * math.sin(0.3) + 0.7 * 1.2 + 0.9 / (3.0 * 4.0), rel=1e-14)


def _chain_potential(p, M, k, k3):
    prev = np.zeros(2)
    V = 0.0
    l0 = 1.0 / (M - 1)
    for i in range(M - 1):
        d = np.linalg.norm(p[i] - prev) - l0
        V += 0.5 * k * d * d + 0.25 * k3 * d ** 4
        prev = p[i]
    return V


def test_chain_spring_forces_are_minus_gradient_of_potential():
    M, mass, k, k3 = 6, 0.1, 10.0, 1.0
    m = O.chain(M=M, mass=mass, k=k, k3=k3, damping=0.0, gravity=0.0)
    rng = np.random.default_rng(1)
    p = I.chain_rest_positions(M, gravity=0.0) + rng.normal(0, 0.05, size=(M - 1, 2))
    x = np.concatenate([p.ravel(), np.zeros(2 * (M - 1))])
    acc = O.deriv(m, x, np.zeros(2))[2 * (M - 1):]
    h = 1e-6
    grad = np.zeros(2 * (M - 1))
    for j in range(2 * (M - 1)):
        e = np.zeros(2 * (M - 1))
        e[j] = h
        grad[j] = (_chain_potential((p.ravel() + e).reshape(-1, 2), M, k, k3)
                   - _chain_potential((p.ravel() - e).reshape(-1, 2), M, k, k3)) / (2 * h)
    np.testing.assert_allclose(acc, -grad / mass, rtol=1e-6, atol=1e-7)


def test_chain_damping_control_gravity_terms():
    M, mass, c, g = 4, 0.2, 0.3, 9.81
    m = O.chain(M=M, mass=mass, damping=c, gravity=g)
    rest = I.chain_rest_state(M, mass=mass, gravity=g)
    v = np.arange(1, 2 * (M - 1) + 1, dtype=float) * 0.1
    x = rest.copy()
    x[2 * (M - 1):] = v
    u = np.array([0.5, -0.25])
    xd = O.deriv(m, x, u)
    np.testing.assert_array_equal(xd[:2 * (M - 1)], v)  # p' = v
    expect = -c * v / mass
    expect[-2:] += u / mass  # force on the last mass only
    np.testing.assert_allclose(xd[2 * (M - 1):], expect, rtol=1e-9, atol=1e-9)  # hanging equilibrium cancels g


def test_chain_single_link_closed_form():
    # one free mass stretched by d along x: a = -(k d + k3 d^3)/m, no gravity
    m = O.chain(M=2, mass=0.1, k=10.0, k3=1.0, damping=0.0, gravity=0.0)
    d = 0.3
    xd = O.deriv(m, [1.0 + d, 0.0, 0.0, 0.0], [0.0, 0.0])
    assert xd[2] == pytest.approx(-(10.0 * d + d ** 3) / 0.1, rel=1e-14)
    assert xd[3] == 0.0


def test_chain_rotated_rest_state_is_static_without_gravity():
    M = 10
    m = O.chain(M=M, N=100, gravity=0.0)
    tgt = I.chain_target(M, 0.5, gravity=0.0)
    x0 = np.concatenate([tgt, np.zeros(2 * (M - 1))])
    X = O.rollout(m, x0, np.zeros(m.n))
    assert np.abs(X - x0[None, :]).max() < 1e-12


def test_chain_hanging_rest_state_is_static():
    M = 10
    m = O.chain(M=M, N=50)
    x0 = I.chain_rest_state(M)
    X = O.rollout(m, x0, np.zeros(m.n))
    assert np.abs(X - x0[None, :]).max() < 1e-9


def test_chain_global_error_is_fourth_order_and_energy_conserved():
    M = 5

    def end(dt):
        m = O.chain(M=M, N=int(round(1.0 / dt)), dt=dt, damping=0.0, gravity=0.0)
        x0 = I.chain_rest_state(M, gravity=0.0) + np.r_[np.zeros(2 * (M - 1)), 0.3 * np.ones(2 * (M - 1))]
        return x0, O.rollout(m, x0, np.zeros(m.n))[-1]

    x0, ref = end(0.02 / 64)
    e1 = np.linalg.norm(end(0.02)[1] - ref)
    e2 = np.linalg.norm(end(0.01)[1] - ref)
    assert 12.0 < e1 / e2 < 20.0

    def E(x):
        p = x[:2 * (M - 1)].reshape(-1, 2)
        v = x[2 * (M - 1):]
        return 0.5 * 0.1 * v @ v + _chain_potential(p, M, 10.0, 1.0)

    assert abs(E(ref) - E(x0)) < 1e-9 * E(x0)


# ------------------------------------------------------------ residuals ---
def test_pendulum_residual_layout_at_upright_equilibrium():
    m = O.pendulum()
    R = O.residual(m, [math.pi, 0.0], None, np.zeros(m.n))
    assert R.shape == (3 * 50 + 2,)
    assert np.abs(R).max() < 1e-12  # upright rest, zero input: every row vanishes
    U = np.zeros(m.n)
    U[7] = 2.0
    R = O.residual(m, [math.pi, 0.0], None, U)
    assert R[3 * 7 + 2] == pytest.approx(0.2)  # 0.1 u_k row of stage k
    assert np.abs(R[: 3 * 7 + 2]).max() < 1e-12  # stages before k untouched (causality)


def test_pendulum_terminal_weights():
    m = O.pendulum(N=1, b=0.0)
    x0 = np.array([0.1, 0.2])
    R = O.residual(m, x0, None, [0.0])
    xN = O.rollout(m, x0, [0.0])[-1]
    np.testing.assert_allclose(R, [0.1 - math.pi, 0.02, 0.0, 10 * (xN[0] - math.pi), 10 * xN[1]], rtol=1e-14)


def test_chain_residual_layout():
    M, N = 5, 3
    m = O.chain(M=M, N=N)
    x0 = I.chain_rest_state(M)
    tgt = I.chain_target(M, 0.2)
    U = np.arange(N * 2, dtype=float)
    R = O.residual(m, x0, tgt, U)
    assert R.shape == (N * (2 * (M - 1) + 2) + 2 * (M - 1),)
    np.testing.assert_allclose(R[: 2 * (M - 1)], x0[: 2 * (M - 1)] - tgt)
    np.testing.assert_allclose(R[2 * (M - 1): 2 * (M - 1) + 2], 0.1 * U[:2])
    X = O.rollout(m, x0, U)
    np.testing.assert_allclose(R[-2 * (M - 1):], X[-1, : 2 * (M - 1)] - tgt)


def test_cost_is_half_squared_residual_norm_and_matches_problem_objectives():
    m = O.testfun("rosenbrock")
    for u in [(0.0, 0.0), (1.0, 1.0), (-0.7, 2.3)]:
        assert O.cost(m, None, None, u) == pytest.approx((1 - u[0]) ** 2 + 100 * (u[1] - u[0] ** 2) ** 2, rel=1e-13,
                                                         abs=1e-15)
    m = O.testfun("rastrigin")
    for u in [(1.9, 1.7), (0.0, 0.0), (0.5, -0.25)]:
        f = 10 + u[0] ** 2 - 5 * math.cos(2 * math.pi * u[0]) + u[1] ** 2 - 5 * math.cos(2 * math.pi * u[1])
        assert O.cost(m, None, None, u) == pytest.approx(f, rel=1e-12, abs=1e-12)
    m = O.testfun("heaviside")
    assert O.cost(m, None, None, [0.5]) == 0.5 and O.cost(m, None, None, [-1e-9]) == 0.0


# ----------------------------------------------------------- Jacobian -----
def _lq_problem(N=50):
    h = 0.1
    A = np.array([[1.0, h], [0.0, 1.0]])
    B = np.array([[h * h / 2], [h]])
    wq = np.sqrt(2.0) * np.ones(2)
    wr = np.sqrt(2 * 0.01) * np.ones(1)
    wqN = np.sqrt(2 * 10.0) * np.ones(2)
    return O.linear(A, B, wq, wr, wqN, N), A, B, wq, wr, wqN


def _lq_affine_map(A, B, wq, wr, wqN, N, x0):
    """R(U) = G U + h by explicit stage-by-stage construction."""
    nx, nu = B.shape
    rows_G, rows_h = [], []
    Phi = np.eye(nx)
    Gx = np.zeros((nx, N * nu))  # x_k = Phi x0 + Gx U
    for k in range(N):
        rows_G.append(wq[:, None] * Gx)
        rows_h.append(wq * (Phi @ x0))
        Ru = np.zeros((nu, N * nu))
        Ru[:, k * nu:(k + 1) * nu] = np.diag(wr)
        rows_G.append(Ru)
        rows_h.append(np.zeros(nu))
        Gx = A @ Gx
        Gx[:, k * nu:(k + 1) * nu] += B
        Phi = A @ Phi
    rows_G.append(wqN[:, None] * Gx)
    rows_h.append(wqN * (Phi @ x0))
    return np.vstack(rows_G), np.concatenate(rows_h)


def test_linear_residual_matches_affine_map():
    m, A, B, wq, wr, wqN = _lq_problem(N=12)
    x0 = np.array([1.0, 0.0])
    G, h = _lq_affine_map(A, B, wq, wr, wqN, 12, x0)
    U = np.random.default_rng(3).normal(size=12)
    np.testing.assert_allclose(O.residual(m, x0, None, U), G @ U + h, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("antithetic,K", [(True, 2 * 24), (False, 24)])
def test_lsq_jacobian_is_exact_for_affine_residual(antithetic, K):
    N = 20  # n = 20
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, _ = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    it = O.iteration(m, O.Options(K=K, antithetic=antithetic, jac_mode="lsq", seed=11), x0, None,
                     np.random.default_rng(4).normal(size=N), 0.3, want_big=True)
    assert it.jac_mode_used == 0
    np.testing.assert_allclose(it.J, G, rtol=0, atol=1e-10 * np.abs(G).max())


def test_sigma_jacobian_is_the_printed_monte_carlo_form():
    N = 10
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, _ = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    s = 0.3
    it = O.iteration(m, O.Options(K=64, jac_mode="sigma", seed=5), x0, None, np.zeros(N), s, want_big=True)
    # for affine R, dR_m = G W_m, so J = G (sum W W^T) / (K' s^2)
    S = it.W.T @ it.W
    np.testing.assert_allclose(it.J, G @ S / (32 * s * s), rtol=1e-10, atol=1e-12)


def test_antithetic_lsq_jacobian_exact_for_quadratic_rosenbrock():
    m = O.testfun("rosenbrock")
    u = np.array([0.3, -0.2])
    it = O.iteration(m, O.Options(K=8, jac_mode="lsq", seed=2), None, None, u, 0.4, want_big=True)
    Jex = np.array([[-math.sqrt(2), 0.0], [-2 * math.sqrt(200) * u[0], math.sqrt(200)]])
    np.testing.assert_allclose(it.J, Jex, rtol=1e-12, atol=1e-12)


def test_heaviside_smoothed_jacobian_matches_stein_closed_form_within_lemma1_bound():
    # E[H(u+w) w]/sigma^2 = phi(u/sigma)/sigma for w ~ N(0, sigma^2) (Eq. 7, Fig. 2)
    from scipy import stats

    m = O.testfun("heaviside")
    u, s = 0.3, 0.5
    K = 4000
    est = []
    for seed in range(20):
        it = O.iteration(m, O.Options(K=K, jac_mode="sigma", seed=seed), None, None, [u], s, want_big=True)
        est.append(it.J[0, 0])
    exact = stats.norm.pdf(u / s) / s
    # Lemma 1: E|mean - mu| <= sqrt(var)/sqrt(K'); per-pair var of dR w / s^2 from the draws
    w = np.linspace(-6, 6, 200001) * s
    dens = stats.norm.pdf(w, scale=s)
    x = 0.5 * ((u + w >= 0).astype(float) - (u - w >= 0).astype(float)) * w / s ** 2
    var = np.trapezoid(x * x * dens, w) - np.trapezoid(x * dens, w) ** 2
    bound = math.sqrt(var / (K // 2))
    errs = np.abs(np.array(est) - exact)
    assert errs.mean() <= 1.5 * bound
    assert abs(np.mean(est) - exact) <= 4 * bound / math.sqrt(len(est))


# -------------------------------------------------------------- GGN step ---
def test_one_ggn_step_reaches_batch_least_squares_solution_on_lq():
    N = 50
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, h = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    Ustar = np.linalg.lstsq(G, -h, rcond=None)[0]
    it = O.iteration(m, O.Options(K=2 * 64, jac_mode="lsq", lam=0.0, seed=3), x0, None, np.zeros(N), 0.5)
    assert it.j_star == 0 and it.alpha == 1.0
    np.testing.assert_allclose(it.U_next, Ustar, rtol=1e-7, atol=1e-9)


def test_damped_ggn_step_matches_closed_form():
    N = 30
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, h = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    U0 = np.random.default_rng(9).normal(size=N)
    lam = 0.7
    d = -np.linalg.solve(G.T @ G + lam * np.eye(N), G.T @ (G @ U0 + h))
    it = O.iteration(m, O.Options(K=2 * 40, jac_mode="lsq", lam=lam, seed=4), x0, None, U0, 0.5)
    np.testing.assert_allclose(it.delta, d, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(it.grad_norm, np.linalg.norm(G.T @ (G @ U0 + h)), rtol=1e-9)


def test_cholesky_and_solve_match_lapack():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(40, 40))
    A = X @ X.T + 0.1 * np.eye(40)
    st, Lf = O.cholesky(A)
    assert st == 0
    np.testing.assert_allclose(Lf, np.linalg.cholesky(A), rtol=1e-11, atol=1e-12)
    b = rng.normal(size=40)
    x = O.chol_solve(Lf, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    backward = np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x))
    assert backward < 40 * np.finfo(float).eps * 10
    st, _ = O.cholesky(A - 10 * np.eye(40) * np.abs(np.linalg.eigvalsh(A)).max())
    assert st == -3


# --------------------------------------------------------------- softmin ---
def test_softmin_matches_brute_force_and_is_shift_invariant():
    import mpmath

    Cs = np.array([3.0, 1.25, 7.5, 1.2500001, 40.0])
    tau = 0.8
    w, st = O.softmin(Cs, tau)
    mp = [mpmath.e ** (-mpmath.mpf(c) / tau) for c in Cs]
    tot = sum(mp)
    np.testing.assert_allclose(w / st["sum_w"], [float(v / tot) for v in mp], rtol=1e-14)
    ess = float(tot ** 2 / sum(v * v for v in mp))
    assert st["ess"] == pytest.approx(ess, rel=1e-13)
    w2, st2 = O.softmin(Cs + 1000.0, tau)
    np.testing.assert_allclose(w2, w, rtol=1e-12)  # equal up to the rounding of C + 1000
    w3, _ = O.softmin(Cs, tau, valid=[1, 0, 1, 1, 1])
    assert w3[1] == 0.0 and w3[3] == 1.0  # shifted by the smallest valid cost


def test_mppi_direction_is_weighted_mean_of_perturbations():
    # Eq. 3 on a tiny sample set: sum w_i W_i / sum w_i over +W and -W
    import mpmath

    m = O.testfun("rosenbrock")
    it = O.iteration(m, O.Options(K=6, tau=2.0, seed=8), None, None, [0.1, 0.4], 0.3, want_big=True)
    num = [mpmath.mpf(0), mpmath.mpf(0)]
    den = mpmath.mpf(0)
    for p in range(3):
        for sgn, c in ((1, it.C_samp[2 * p]), (-1, it.C_samp[2 * p + 1])):
            wgt = mpmath.e ** (-mpmath.mpf(c) / 2.0)
            den += wgt
            for j in range(2):
                num[j] += wgt * sgn * mpmath.mpf(it.W[p, j])
    np.testing.assert_allclose(it.mppi_dir, [float(v / den) for v in num], rtol=1e-12)


# ---------------------------------------------------------- line search ---
def test_line_search_picks_first_minimiser_over_step_set():
    # Heaviside (Problem III): every step that crosses 0 costs 0 -> ties -> smallest j
    m = O.testfun("heaviside")
    it = O.iteration(m, O.Options(K=200, jac_mode="sigma", L=16, lam=1e-3, seed=1), None, None, [0.5], 0.5)
    assert it.C_line.min() == 0.0
    assert it.j_star == int(np.argmin(it.C_line))  # first occurrence
    assert it.alpha == 0.5 ** it.j_star
    assert it.U_next[0] == pytest.approx(0.5 + it.alpha * it.delta[0])


def test_monotone_option_adds_zero_step():
    m = O.testfun("rosenbrock")
    it = O.iteration(m, O.Options(K=8, L=4, monotone=True, lam=1e3, seed=1), None, None, [1.0, 1.0], 0.1)
    assert len(it.C_line) == 5 and it.C_line[4] == it.C_nom


def test_nonfinite_samples_are_masked():
    # Rastrigin residual sqrt(5 - 5 cos) is finite everywhere; Heaviside too; use a pendulum with huge sigma
    m = O.pendulum(N=5)
    it = O.iteration(m, O.Options(K=16, seed=0), [0.1, 0.0], None, np.zeros(5), 1e200)
    assert it.n_masked > 0 or it.status != 0


# --------------------------------------------------------- whole solves ---
def test_gn_mppi_solves_lq_problem_iv():
    N = 50
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, h = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    Ustar = np.linalg.lstsq(G, -h, rcond=None)[0]
    Cstar = 0.5 * np.sum((G @ Ustar + h) ** 2)
    st, U, Uh, Ch, its = O.solve(m, O.Options(K=128, iterations=3, lam=1e-8, seed=2), x0, None, np.zeros(N), 0.5)
    assert st == 0
    assert Ch[1] <= Cstar * (1 + 1e-10)


def test_method_a_solves_lq_in_one_step():
    N = 20
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, h = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    Ustar = np.linalg.lstsq(G, -h, rcond=None)[0]
    st, U, C, its = O.method_a(m, x0, None, np.zeros(N))
    np.testing.assert_allclose(U, Ustar, rtol=1e-7, atol=1e-8)


def test_gn_mppi_on_rosenbrock_reaches_optimum():
    # Problem I: optimum U* = (1, 1), C* = 0 (Table 1: Method D converges)
    m = O.testfun("rosenbrock")
    st, U, Uh, Ch, its = O.solve(m, O.Options(K=2000, iterations=40, lam=1e-6, seed=3), None, None, [0.0, 0.0],
                                 0.5)
    np.testing.assert_allclose(U, [1.0, 1.0], atol=1e-6)


def test_gn_mppi_on_chain_converges_to_method_a_optimum():
    M, N = 4, 20
    m = O.chain(M=M, N=N)
    x0, tgt = I.chain_instances(5, 1, M)
    st, U, Uh, Ch, its = O.solve(m, O.Options(K=256, iterations=15, seed=1), x0[0], tgt[0], np.zeros(m.n), 0.2)
    stA, UA, CA, itA = O.method_a(m, x0[0], tgt[0], np.zeros(m.n))
    assert (Ch[-1] - CA) / CA < 1e-8
    assert np.all(np.diff(Ch[5:]) <= 1e-9 * CA)  # monotone once converging


def test_covariance_shrinks_by_sqrt_beta():
    # iteration k uses s_k = s_0 beta^(k/2): the drawn W of iteration 2 is beta x that of a fresh draw
    m = O.testfun("rosenbrock")
    opt = O.Options(K=4, iterations=3, beta=0.36, seed=9)
    st, U, Uh, Ch, its = O.solve(m, opt, None, None, [0.2, 0.1], 0.5)
    it2 = O.iteration(m, opt, None, None, Uh[2], 0.5 * 0.36, it=2, want_big=True)
    np.testing.assert_allclose(it2.delta, its[2].delta, rtol=1e-12)


# ------------------------------------------- Method E: sigma points (Sec. 5) ---
def test_sigma_point_jacobian_exact_for_quadratic_rosenbrock():
    """The symmetric sigma points +-sqrt(n) s_i e_i turn the smoothed Jacobian of
    Eq. 7 into central differences, exact for a quadratic residual at any step."""
    m = O.testfun("rosenbrock")
    u = np.array([0.3, -0.2])
    it = O.iteration(m, O.Options(K=2, sampling="sigma", seed=2), None, None, u, np.array([0.4, 0.7]),
                     want_big=True)
    assert it.status == 0 and it.W.shape == (2, 2)
    Jex = np.array([[-math.sqrt(2), 0.0], [-2 * math.sqrt(200) * u[0], math.sqrt(200)]])
    np.testing.assert_allclose(it.J, Jex, rtol=1e-12, atol=1e-12)


def test_sigma_point_jacobian_is_central_differences_with_step_sqrt_n_sigma():
    """Nonlinear pendulum: column i of the Dirac-mixture Jacobian equals
    (R(U + h_i e_i) - R(U - h_i e_i)) / (2 h_i) with h_i = sqrt(n) s_i,
    evaluated here directly from the residual; the perturbations are
    W_i = h_i e_i and the softmin sees all 2n costs."""
    N = 10
    m = O.pendulum(N=N)
    n = m.n
    x0 = np.array([0.3, -0.1])
    rng = np.random.default_rng(4)
    U = rng.normal(0, 0.5, n)
    s = 0.05 + 0.1 * rng.random(n)
    it = O.iteration(m, O.Options(K=999, sampling="sigma", seed=9), x0, None, U, s, want_big=True)
    assert it.status == 0
    h = math.sqrt(n) * s
    np.testing.assert_allclose(it.W, np.diag(h), rtol=1e-15, atol=0)
    Jcd = np.empty((m.nR, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = h[i]
        Jcd[:, i] = (O.residual(m, x0, None, U + e) - O.residual(m, x0, None, U - e)) / (2 * h[i])
    np.testing.assert_allclose(it.J, Jcd, rtol=1e-10, atol=1e-12)
    assert len(it.C_samp) == 2 * n


def test_sigma_points_require_antithetic_pairs():
    m = O.testfun("rosenbrock")
    it = O.iteration(m, O.Options(K=8, sampling="sigma", antithetic=False), None, None, [0.1, 0.2], 0.3)
    assert it.status == -1  # ORC_E_ARG


# ---------------------------------------------- Method C: MPPI step (Sec. 3) ---
def test_mppi_step_matches_the_tilted_gaussian_mean_on_a_quadratic_cost():
    """For C(U) = 1/2 ||G U + h||^2 (Problem IV's affine residual) the MPPI step
    of Eq. 3 has the closed form (Sigma^-1 + H/tau)^-1 (H/tau)(U* - U), H = G^T G,
    U* the least-squares minimiser; the empirical step of Eq. 5 over 2e5
    antithetic pairs must agree within Monte Carlo error, and the iterate takes
    the step whole (alpha = 1)."""
    N = 4
    m, A, B, wq, wr, wqN = _lq_problem(N=N)
    x0 = np.array([1.0, 0.0])
    G, hv = _lq_affine_map(A, B, wq, wr, wqN, N, x0)
    H = G.T @ G
    Ustar = np.linalg.lstsq(G, -hv, rcond=None)[0]
    U = np.array([0.4, -0.2, 0.1, 0.3])
    sig, tau = 0.3, 1.0
    exact = np.linalg.solve(np.eye(N) / sig ** 2 + H / tau, (H / tau) @ (Ustar - U))
    it = O.iteration(m, O.Options(K=400000, method="mppi", tau=tau, seed=12, threads=8), x0, None, U, sig)
    assert it.status == 0 and it.alpha == 1.0 and it.j_star == 0
    np.testing.assert_allclose(it.delta, it.mppi_dir, rtol=0, atol=0)
    assert np.linalg.norm(it.delta - exact) <= 1e-2 * np.linalg.norm(exact)
    np.testing.assert_allclose(it.U_next, U + it.delta, rtol=0, atol=1e-15)
    assert it.C_new == pytest.approx(O.cost(m, x0, None, U + it.delta), rel=1e-14)


# ------------------------------------- Setting V.ii: dead-zone friction ---
def test_dead_zone_friction_zeroes_exactly_the_small_controls():
    """u_apply = 0 where |u| <= u_f, u elsewhere (per component): the rollout
    with friction equals the frictionless rollout of the thresholded controls,
    and controls inside the dead zone act like no control at all."""
    uf = 0.3
    for fric, plain, U in (
        (O.pendulum(N=12, u_friction=uf), O.pendulum(N=12), np.linspace(-0.6, 0.6, 12)),
        (O.chain(M=4, N=6, u_friction=uf), O.chain(M=4, N=6), np.linspace(-0.9, 0.7, 12)),
    ):
        x0 = np.linspace(0.05, 0.4, fric.nx)
        Ua = np.where(np.abs(U) <= uf, 0.0, U)
        assert np.any(Ua == 0.0) and np.any(Ua != 0.0)
        np.testing.assert_array_equal(O.rollout(fric, x0, U), O.rollout(plain, x0, Ua))
        small = np.clip(U, -uf, uf)
        np.testing.assert_array_equal(O.rollout(fric, x0, small), O.rollout(plain, x0, np.zeros_like(U)))
        # the residual still penalises the decision variable: 0.1 u rows differ
        assert not np.array_equal(O.residual(fric, x0, np.zeros(2 * (fric.M - 1)) if fric.M else None, small),
                                  O.residual(plain, x0, np.zeros(2 * (fric.M - 1)) if fric.M else None,
                                             np.zeros_like(U)))


# ------------------------------------------- LSQ breakdown (Eq. 9, B > 0) ---
# Eq. 9 assumes a positive definite B_GGN.  The oracle's reading: when the
# LSQ form J = P S^-1 breaks down (S without a Cholesky factor, or the damped
# LSQ system without one at every damping), the iteration takes the printed
# Monte Carlo form J = P Sigma^-1 / K', and so does the rest of the solve.
# The breakdown is forced through the oracle's test hook, so both branches and
# the sticky rule are pinned on any input: against a direct call in the
# printed form (a different code path through the same arithmetic), and
# against the LSQ iteration it replaces (which must differ).
def _breakdown_problem():
    seed = 41
    M, N, K = 4, 10, 64  # n = 20, K' = 32 >= n: AUTO takes the LSQ form
    x0, tgt = I.chain_instances(seed, 1, M)
    return O.chain(M=M, N=N), x0[0], tgt[0], K, seed


@pytest.mark.parametrize("kind", ["s", "system"])
def test_lsq_breakdown_takes_the_printed_form(kind):
    m, x0, tgt, K, seed = _breakdown_problem()
    U = np.random.default_rng(3).normal(0.0, 0.2, size=m.n)
    lsq = O.iteration(m, O.Options(K=K, seed=seed), x0, tgt, U, 0.2, it=1)
    sig = O.iteration(m, O.Options(K=K, seed=seed, jac_mode="sigma"), x0, tgt, U, 0.2, it=1)
    brk = O.iteration(m, O.Options(K=K, seed=seed, break_it=1, break_kind=kind), x0, tgt, U, 0.2, it=1)
    other_it = O.iteration(m, O.Options(K=K, seed=seed, break_it=1, break_kind=kind), x0, tgt, U, 0.2, it=2)
    lsq2 = O.iteration(m, O.Options(K=K, seed=seed), x0, tgt, U, 0.2, it=2)
    assert lsq.status == sig.status == brk.status == 0
    assert lsq.jac_mode_used == 0 and sig.jac_mode_used == 1 and brk.jac_mode_used == 1
    assert np.array_equal(brk.delta, sig.delta) and np.array_equal(brk.U_next, sig.U_next)
    assert brk.C_new == sig.C_new and brk.j_star == sig.j_star
    assert np.linalg.norm(brk.delta - lsq.delta) > 1e-3 * np.linalg.norm(lsq.delta)
    # the hook acts at its own iteration only
    assert other_it.jac_mode_used == 0 and np.array_equal(other_it.delta, lsq2.delta)


def test_lsq_breakdown_is_sticky_for_the_rest_of_the_solve():
    m, x0, tgt, K, seed = _breakdown_problem()
    T, b = 6, 2
    opt = O.Options(K=K, iterations=T, seed=seed, break_it=b, break_kind="system")
    st, U, Uh, Ch, its = O.solve(m, opt, x0, tgt, np.zeros(m.n), 0.2)
    assert st == 0
    assert [it.jac_mode_used for it in its] == [0] * b + [1] * (T - b)
    # the same path step by step: LSQ before the breakdown, the printed form from it on
    s = np.full(m.n, 0.2)
    Uk = np.zeros(m.n)
    for k in range(T):
        jm = "auto" if k < b else "sigma"
        ref = O.iteration(m, O.Options(K=K, seed=seed, jac_mode=jm), x0, tgt, Uk, s, it=k)
        assert np.array_equal(Uh[k + 1], ref.U_next), k
        Uk = ref.U_next
        s = s * math.sqrt(0.7)
    # without the sticky rule iteration b + 1 would return to LSQ
    free = O.iteration(m, O.Options(K=K, seed=seed), x0, tgt, Uh[b + 1], s * 0 + 0.2 * math.sqrt(0.7) ** (b + 1),
                       it=b + 1)
    assert free.jac_mode_used == 0
