"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle
on the same seeded inputs.

FP64 mode: relative 1e-10 (normwise for vectors) per Algorithm-1 iteration,
with the oracle's iterate U_k fed to both sides so that the comparison never
drifts; the step delta (and U_{k+1}) within max(1e-10, 4 kappa_2 u) of the
damped normal equations, the forward-error bound of a backward-stable solve.
Reduced-precision modes (FP32 rollouts; tensor-core contractions of
FP32-level accuracy): 1e-4 relative on every cost -- nominal, per sample,
line search, after each step, converged.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLRED = 1e-4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2512_04579_gb300 import build as B

    B.build()
    return G.load()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def sigmas(s0, beta, T, n):
    s = np.full(n, float(s0))
    out = []
    sb = math.sqrt(beta)
    for _ in range(T):
        out.append(s.copy())
        s = s * sb
    return out


U64 = np.finfo(float).eps / 2  # unit roundoff of FP64
U32 = float(np.finfo(np.float32).eps) / 2  # unit roundoff of FP32


def step_tol(big, it, tol):
    """Normwise tolerance for the GGN step.  Both sides solve the damped normal
    equations (J^T J + lambda I) delta = -J^T r (Eq. 9; the GPU in the scaled
    form with delta = S y) by a backward-stable FP64 solve with refinement, so
    each side's forward error is bounded by kappa_2(J^T J + lambda I) times the
    unit roundoff; 4 kappa u covers both.  Never below tol."""
    H = big.J.T @ big.J + it.lambda_used * np.eye(big.J.shape[1])
    return max(tol, 4.0 * np.linalg.cond(H) * U64)


def check_iteration(rep, Ug, it, C_ref, tol, tie=1e-12, tol_step=None, c_scale=0.0):
    """Compare one GPU iteration report with an oracle record.  c_scale: the
    cost scale of the problem (its initial cost); costs near a zero minimum
    carry rounding at that scale (the residual terms cancel), so cost
    comparisons get an absolute floor tol * c_scale."""
    tol_step = tol if tol_step is None else tol_step
    assert rep.status == it.status == 0
    assert rep.C_nom == pytest.approx(it.C_nom, rel=tol, abs=tol * c_scale)
    if rep.j_star != it.j_star:
        # a tie between two step lengths: both must give the same cost
        assert abs(it.C_line[rep.j_star] - it.C_line[it.j_star]) <= tie * abs(C_ref)
    else:
        assert rel(Ug, it.U_next) < tol_step
    assert rep.C_new == pytest.approx(it.C_new, rel=tol, abs=tol * c_scale)


def per_iteration_parity(model, gprob, opt, x0, xref, U0, s0, T, tol=TOL64, sample_check=True):
    st, Uend, Uh, Ch, its = O.solve(model, opt, x0, xref, U0, s0)
    assert st == 0
    ss = sigmas(s0, opt.beta, T, model.n)
    solver = G.Solver(gprob, 1)
    try:
        for k in range(T):
            stg, Ug, rep = solver.step(x0, xref, Uh[k], ss[k], k)
            r = rep[0]
            it = its[k]
            big = O.iteration(model, opt, x0, xref, Uh[k], ss[k], it=k, want_big=True)
            tol_d = step_tol(big, it, tol)
            check_iteration(r, Ug, it, Ch[k], tol, tol_step=tol_d, c_scale=abs(Ch[0]))
            d = solver.debug("delta")
            assert rel(d, it.delta) < tol_d, f"iteration {k}: delta"
            np.testing.assert_allclose(solver.debug("Cline"), it.C_line[: opt.L], rtol=tol, atol=tol * abs(Ch[0]))
            assert r.c_min == pytest.approx(it.c_min, rel=tol)
            assert r.ess == pytest.approx(it.ess, rel=1e-8)
            assert r.n_masked == it.n_masked
            assert rel(solver.debug("mppi"), it.mppi_dir) < 1e-8
            if sample_check and k in (0, T - 1):
                Kp = big.W.shape[0]
                dR = solver.debug("dR").reshape(model.nR, Kp)
                W = solver.debug("W").reshape(model.n, Kp)
                assert rel(dR, big.dR.T) < tol
                assert rel(W, big.W.T) < 1e-13
                np.testing.assert_allclose(solver.debug("C"), big.C_samp, rtol=1e-12)
                assert rel(solver.debug("e"), big.dR @ big.r) < tol
    finally:
        solver.close()
    return its


# ----------------------------------------------------------------- FP64 mode
def test_fp64_pendulum_swingup_per_iteration():
    """Pendulum swing-up, N=50, K=256, sigma 0.5, lambda 1e-3, 20 iterations."""
    seed = I.BASE_SEED
    x0 = I.pendulum_x0(seed, 1)[0]
    m = O.pendulum()
    opt = O.Options(K=256, iterations=20, lam=1e-3, seed=seed)
    gp = G.pendulum_problem(N=50, K=256, iterations=20, lam=1e-3, sigma0=0.5, seed=seed)
    per_iteration_parity(m, gp, opt, x0, None, np.zeros(m.n), 0.5, 20)


def test_fp64_chain_ragged_sizes_per_iteration():
    """Chain M=5, N=30 (n=60, nR=308), K=300 (150 pairs: 64+64+22), 6 iterations."""
    seed = I.BASE_SEED + 11
    M, N, K = 5, 30, 300
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=6, lam=1e-3, seed=seed)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=6, lam=1e-3, sigma0=0.2, seed=seed)
    per_iteration_parity(m, gp, opt, x0[0], tgt[0], np.zeros(m.n), 0.2, 6)


def test_fp64_sigma_mode_when_samples_are_fewer_than_unknowns():
    """K' = 20 pairs < n = 60: AUTO picks the printed Monte Carlo form (SIGMA)."""
    seed = 5
    M, N, K = 4, 30, 40
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=3, lam=1e-2, seed=seed)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=3, lam=1e-2, sigma0=0.2, seed=seed)
    its = per_iteration_parity(m, gp, opt, x0[0], tgt[0], np.zeros(m.n), 0.2, 3)
    assert all(it.jac_mode_used == 1 for it in its)


def test_fp64_one_sided_and_monotone_options():
    seed = 9
    x0 = I.pendulum_x0(seed, 1)[0]
    m = O.pendulum(N=25)
    opt = O.Options(K=80, iterations=3, lam=1e-3, antithetic=False, monotone=True, seed=seed)
    gp = G.pendulum_problem(N=25, K=80, iterations=3, lam=1e-3, sigma0=0.4, antithetic=False, monotone=True,
                            seed=seed)
    per_iteration_parity(m, gp, opt, x0, None, np.zeros(m.n), 0.4, 3)


def _lq(N):
    h = 0.1
    A = np.array([[1.0, h], [0.0, 1.0]])
    B = np.array([[h * h / 2], [h]])
    wq = np.sqrt(2.0) * np.ones(2)
    wr = np.sqrt(0.02) * np.ones(1)
    wqN = np.sqrt(20.0) * np.ones(2)
    return A, B, wq, wr, wqN


def test_fp64_lq_single_newton_step_reaches_closed_form():
    """Problem IV: one GGN step with lambda = 0 reaches the batch least-squares solution."""
    N = 50
    A, B, wq, wr, wqN = _lq(N)
    x0 = np.array([1.0, 0.0])
    m = O.linear(A, B, wq, wr, wqN, N)
    # closed form from the oracle-independent affine map R(U) = G U + h
    Gm = np.zeros((m.nR, N))
    h0 = O.residual(m, x0, None, np.zeros(N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        Gm[:, j] = O.residual(m, x0, None, e) - h0
    Ustar = np.linalg.lstsq(Gm, -h0, rcond=None)[0]
    gp = G.linear_problem(A, B, wq, wr, wqN, N=N, K=128, iterations=1, lam=0.0, sigma0=0.5, seed=3)
    s = G.Solver(gp, 1)
    st, U, rep = s.step(x0, None, np.zeros(N), np.full(N, 0.5), 0)
    s.close()
    assert st == 0 and rep[0].j_star == 0
    assert rel(U, Ustar) < 1e-8


def test_fp64_uneven_batch_matches_per_instance_oracle():
    """Three chain instances of different M, N, K in one handle."""
    seed = 21
    shapes = [(20, 4, 64), (33, 6, 130), (12, 3, 200)]
    x0s, tgts, U0s = [], [], []
    for i, (N, M, K) in enumerate(shapes):
        x0, tg = I.chain_instances(seed + i, 1, M)
        x0s.append(x0[0])
        tgts.append(tg[0])
        U0s.append(np.zeros(N * 2))
    gp = G.chain_problem(M=4, N=20, K=64, iterations=2, lam=1e-3, sigma0=0.2, seed=seed)
    s = G.Solver(gp, 3, shapes=shapes)
    sig = [np.full(N * 2, 0.2) for (N, M, K) in shapes]
    st, U, rep = s.step(np.concatenate(x0s), np.concatenate(tgts), np.concatenate(U0s), np.concatenate(sig), 0)
    assert st == 0
    for i, (N, M, K) in enumerate(shapes):
        m = O.chain(M=M, N=N)
        it = O.iteration(m, O.Options(K=K, lam=1e-3, seed=seed), x0s[i], tgts[i], U0s[i], 0.2, inst=i, it=0)
        Ui = U[s.off_U[i]: s.off_U[i + 1]]
        check_iteration(rep[i], Ui, it, it.C_nom, TOL64)
        assert rel(s.debug("delta", i), it.delta) < TOL64
    s.close()


def test_fp64_whole_solve_graph_matches_oracle():
    """gnmppi_solve (one CUDA graph) over 8 iterations vs the oracle's solve."""
    seed = 33
    M, N, K = 4, 20, 128
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=8, lam=1e-3, seed=seed)
    st, Uo, Uh, Ch, its = O.solve(m, opt, x0[0], tgt[0], np.zeros(m.n), 0.2)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=8, lam=1e-3, sigma0=0.2, seed=seed)
    s = G.Solver(gp, 1)
    stg, U, rep = s.solve(x0[0], tgt[0], np.zeros(m.n))
    assert stg == 0 and rep[0].iterations == 8
    assert rep[0].C_final == pytest.approx(Ch[-1], rel=TOL64)
    assert rel(U, Uo) < 1e-9
    assert rep[0].sigma_final == pytest.approx(0.2 * math.sqrt(0.7) ** 8, rel=1e-14)
    # a second solve on the same handle replays the graph and gives the same answer
    stg2, U2, rep2 = s.solve(x0[0], tgt[0], np.zeros(m.n))
    assert np.array_equal(U, U2)
    s.close()


def test_fp64_cost_reevaluation():
    seed = 4
    M, N = 10, 100
    x0, tgt = I.chain_instances(seed, 3, M)
    rng = np.random.default_rng(1)
    U = rng.normal(0, 0.3, size=(3, N * 2))
    gp = G.chain_problem(M=M, N=N, K=64, iterations=1, precision=G.PREC_FP32, seed=seed)
    s = G.Solver(gp, 3)
    C = s.cost(x0, tgt, U)
    s.close()
    m = O.chain(M=M, N=N)
    for b in range(3):
        assert C[b] == pytest.approx(O.cost(m, x0[b], tgt[b], U[b]), rel=1e-12)


def test_nonfinite_samples_are_dropped_like_the_oracle():
    seed = 0
    m = O.pendulum(N=5)
    x0 = np.array([0.1, 0.0])
    it = O.iteration(m, O.Options(K=16, seed=seed), x0, None, np.zeros(5), 1e200)
    gp = G.pendulum_problem(N=5, K=16, iterations=1, sigma0=1.0, seed=seed)
    s = G.Solver(gp, 1)
    st, U, rep = s.step(x0, None, np.zeros(5), np.full(5, 1e200), 0)
    s.close()
    assert rep[0].n_masked == it.n_masked
    assert rep[0].status == it.status


# -------------------------------------------------------- reduced precision
@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
def test_reduced_precision_chain_full_size_iteration(prec):
    """Chain M=10, N=100 (n=200, nR=2018), K=2048, sigma 0.2: one iteration at
    full size against the FP64 oracle, costs within 1e-4."""
    seed = I.BASE_SEED + 1
    M, N, K = 10, 100, 2048
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=1, lam=1e-3, seed=seed, threads=8)
    it = O.iteration(m, opt, x0[0], tgt[0], np.zeros(m.n), 0.2)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 1)
    st, U, rep = s.step(x0[0], tgt[0], np.zeros(m.n), np.full(m.n, 0.2), 0)
    Cs = s.debug("C")
    s.close()
    assert st == 0
    assert rep[0].C_nom == pytest.approx(it.C_nom, rel=TOLRED)
    np.testing.assert_allclose(Cs, it.C_samp, rtol=TOLRED)
    assert rep[0].j_star == it.j_star
    assert rep[0].C_new == pytest.approx(it.C_new, rel=TOLRED)
    # U_0 = 0, so U_1 = alpha* delta on both sides: the steps agree
    assert rel(U, it.U_next) < 1e-2


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
def test_reduced_precision_chain_solve_cost(prec):
    """Chain M=6, N=40, K=512, 10 iterations: final cost within 1e-4 of the oracle's."""
    seed = 77
    M, N, K, T = 6, 40, 512, 10
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    st, Uo, Uh, Ch, its = O.solve(m, O.Options(K=K, iterations=T, lam=1e-3, seed=seed, threads=8), x0[0], tgt[0],
                                  np.zeros(m.n), 0.2)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=T, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 1)
    stg, U, rep = s.solve(x0[0], tgt[0], np.zeros(m.n))
    C = s.cost(x0[0], tgt[0], U)[0]
    s.close()
    assert stg == 0
    assert C == pytest.approx(Ch[-1], rel=TOLRED)
    assert O.cost(m, x0[0], tgt[0], U) == pytest.approx(C, rel=1e-12)


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
def test_reduced_precision_per_iteration_full_size(prec):
    """Chain M=10, N=100 (n=200, nR=2018), K=2048: four Algorithm-1
    iterations along the oracle's own trajectory (its U_k and sampling scale
    fed to both sides, so nothing drifts): nominal, sample and line-search
    costs and the cost after each step within 1e-4."""
    seed = I.BASE_SEED + 1
    M, N, K, T = 10, 100, 2048, 4
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=T, lam=1e-3, seed=seed, threads=16)
    st, Uo, Uh, Ch, its = O.solve(m, opt, x0[0], tgt[0], np.zeros(m.n), 0.2)
    assert st == 0
    ss = sigmas(0.2, opt.beta, T, m.n)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 1)
    try:
        for k in range(T):
            stg, Ug, rep = s.step(x0[0], tgt[0], Uh[k], ss[k], k)
            r, it = rep[0], its[k]
            assert stg == 0 and r.status == 0
            assert r.C_nom == pytest.approx(it.C_nom, rel=TOLRED)
            np.testing.assert_allclose(s.debug("C"), it.C_samp, rtol=TOLRED)
            np.testing.assert_allclose(s.debug("Cline"), it.C_line[: opt.L], rtol=TOLRED)
            assert r.C_new == pytest.approx(it.C_new, rel=TOLRED), k
    finally:
        s.close()


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
def test_reduced_precision_full_size_solves_reach_the_reference_optima(prec):
    """The benchmark problem at full size: chain M=10, N=100, K=2048,
    30 iterations, 8 instances in one handle and one CUDA graph.  Every final
    FP64 re-evaluated cost is within 1e-4 of the oracle's own 30-iteration
    solve, and within 1e-6 of the reference optimum C* (the oracle's solve
    polished by Method A) wherever the oracle's solve is."""
    rows = np.loadtxt(os.path.join(GOLDEN, "chain_m10_cstar.txt"), comments="#")
    B = 8
    seed = I.BASE_SEED + 1
    x0, tgt = I.chain_instances(seed, len(rows), 10)
    gp = G.chain_problem(M=10, N=100, K=2048, iterations=30, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, B)
    try:
        st, U, rep = s.solve(x0[:B], tgt[:B], np.zeros(B * 200))
        C = s.cost(x0[:B], tgt[:B], U)
    finally:
        s.close()
    assert st == 0 and all(r.status == 0 and r.iterations == 30 for r in rep)
    Cgn, Cs = rows[:B, 1], rows[:B, 2]
    np.testing.assert_allclose(C, Cgn, rtol=TOLRED)
    reached = (Cgn - Cs) / Cs <= 1e-6
    assert reached.sum() >= B - 1
    assert np.all((C - Cs)[reached] / Cs[reached] <= 1e-6)


@pytest.mark.parametrize("prec,tol", [(G.PREC_FP32, 1e-4), (G.PREC_BF16, 1e-4)])
def test_tensor_core_contraction_matches_oracle(prec, tol):
    """[P^T | S] from the tcgen05 contraction (FP32 mode: three TF32 passes
    over head/remainder splits of the FP32 operands; BF16 mode: head +
    remainder BF16 operands in three passes; FP32 accumulation) against the
    oracle's P = sum dR W^T and S = sum W W^T, at sizes spanning several
    tiles with ragged edges (n = 150, nR + n = 1130, K' = 700 pairs, padded
    to 704): normwise against the oracle, and entry by entry against the
    FP64 products of the operands the GPU holds.  Each entry is a dot product
    over the K' pairs, so its rounding error is bounded by a multiple of
    sum_m |dR_m,i| |W_m,j| (and |W_m,i| |W_m,k| for S): the TF32 split leaves
    ~2^-21 relative per product, the BF16 head + remainder pair 2^-17 per
    operand (the dropped remainder x remainder term 2^-18), and the FP32
    accumulation over 704 terms adds at most ~4e-5 of that sum.  A stale,
    missing or misplaced tile leaves an O(|P|) error, about 1/sqrt(K') of the
    bound's scale here, so it fails."""
    seed = 12
    M, N, K = 6, 75, 1400
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    big = O.iteration(m, O.Options(K=K, lam=1e-3, seed=seed, threads=8), x0[0], tgt[0], np.zeros(m.n), 0.2,
                      want_big=True)
    P = big.dR.T @ big.W  # nR x n
    S = big.W.T @ big.W
    gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 1)
    s.step(x0[0], tgt[0], np.zeros(m.n), np.full(m.n, 0.2), 0)
    PS = s.debug("PS").reshape(m.n, m.nR + m.n)
    A = s.debug("A").reshape(m.n, m.n)
    Kp = K // 2
    dRg = s.debug("dR").reshape(m.nR, Kp)
    Wg = s.debug("W").reshape(m.n, Kp)
    s.close()
    assert rel(PS[:, : m.nR], P.T) < tol
    assert rel(PS[:, m.nR:], S) < tol
    # entry by entry against the GPU's own operands
    ent = 1e-4
    for got, ref, bound in ((PS[:, : m.nR], Wg @ dRg.T, np.abs(Wg) @ np.abs(dRg).T),
                            (PS[:, m.nR:], Wg @ Wg.T, np.abs(Wg) @ np.abs(Wg).T)):
        assert np.all(np.abs(got - ref) <= ent * bound)
    # Gram A = P^T P on the tensor cores (three TF32 passes): its error is that of P
    assert rel(A, P.T @ P) < 2 * tol
    assert np.allclose(A, A.T, rtol=1e-5, atol=1e-5 * np.abs(A).max())


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
@pytest.mark.parametrize("M,N,K", [(6, 75, 1400), (4, 150, 640), (3, 260, 1056), (10, 120, 512), (16, 150, 640)])
def test_tensor_core_gram_matches_its_definition(prec, M, N, K):
    """A = P^T P and S2 = S S^T of Eq. 9 from the tcgen05 Gram kernel (head/
    remainder split in shared memory: TF32 in the FP32 mode, BF16 in the BF16
    mode; three passes, FP32 accumulation) against the same products formed
    in FP64 from the [P^T | S] the GPU holds,
    at n = 150, 300 and 520: one and two 128-row sub-tiles on the diagonal,
    off-diagonal tiles, lower blocks stored transposed, ragged edges; and at
    nR = 2418 and 4830 (n = 240, 300), where A is summed over 2048-column
    chunks in FP64 (two and three chunks, the last one ragged).  Every entry
    must be written (a stale or missing block fails the entrywise bound) and
    A symmetric."""
    seed = 31
    n = 2 * N
    x0, tgt = I.chain_instances(seed, 1, M)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 1)
    s.step(x0[0], tgt[0], np.zeros(n), np.full(n, 0.2), 0)
    PS = s.debug("PS")
    nR = PS.size // n - n
    PS = PS.reshape(n, nR + n)
    A = s.debug("A").reshape(n, n)
    S2 = s.debug("S2").reshape(n, n)
    s.close()
    assert K // 2 >= n  # LSQ mode: S2 is formed
    Pt, S = PS[:, :nR], PS[:, nR:]
    for got, ref in ((A, Pt @ Pt.T), (S2, S @ S.T)):
        # Each entry is a dot product of two rows: its rounding error is
        # bounded by a multiple of |row_i| |row_j| = sqrt(ref_ii ref_jj)
        # (Cauchy-Schwarz).  The split itself leaves ~2^-22 (TF32) or ~2^-16
        # (BF16, the dropped remainder x remainder term, of random sign) per
        # product; the tensor core's FP32 accumulation over nR = 1206-1566
        # terms measures ~2e-5 of that scale here, so 1e-4 bounds it while a
        # stale or missing block (an O(1) error) fails.
        d = np.sqrt(np.diag(ref))
        assert rel(got, ref) < 5e-5
        assert np.all(np.abs(got - ref) <= 1e-4 * np.outer(d, d))
    assert np.all(np.abs(A - A.T) <= 1e-4 * np.outer(np.sqrt(np.diag(A)), np.sqrt(np.diag(A))))
    # The FP32 accumulators are widened to FP64 exactly (on the integer pipe):
    # every entry of an unchunked product is an FP32 value, so a misplaced
    # fraction bit (which the 1e-4 bound above cannot see) fails here.  A
    # chunked A is a FP64 sum of such values.
    for got in ((A, S2) if nR <= 2048 else (S2,)):
        assert np.array_equal(got.astype(np.float32).astype(np.float64), got)
    # The remainder passes take effect: the head-only product hi hi^T (hi =
    # [P^T] rounded to TF32 or BF16, the one pass a dropped remainder would
    # leave) has a different, larger error, and the GPU's error is
    # uncorrelated with it.
    u = Pt.astype(np.float32).view(np.uint32).astype(np.uint64)
    if prec == G.PREC_BF16:  # round to nearest even on the 16 kept bits
        hi = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)
    else:
        hi = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32).astype(np.float64)
    Aref = Pt @ Pt.T
    d = np.sqrt(np.diag(Aref))
    e_gpu = (A - Aref) / np.outer(d, d)
    e_head = (hi @ hi.T - Aref) / np.outer(d, d)
    # (a TF32 head-only product's random rounding averages down over long
    # sums, below the FP32 accumulation error, so the size comparison is made
    # where the head's rounding dominates: BF16, or short sums)
    if prec == G.PREC_BF16 or nR <= 2048:
        assert np.sqrt(np.mean(e_gpu ** 2)) < 0.5 * np.sqrt(np.mean(e_head ** 2))
    assert abs(np.sum(e_gpu * e_head)) < 0.3 * np.sqrt(np.sum(e_gpu ** 2) * np.sum(e_head ** 2))


@pytest.mark.parametrize("M,N,K", [(20, 15, 200), (40, 10, 96), (65, 6, 64)])
def test_fp64_group_rollout_chains_per_iteration(M, N, K):
    """Chains of 19, 39 and 64 free masses: a group of 4 or 8 lanes per rollout
    (placeholder masses in the last lane for 19 and 39), ragged pair blocks."""
    seed = 100 + M
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=K, iterations=2, lam=1e-2, seed=seed, threads=8)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=2, lam=1e-2, sigma0=0.2, seed=seed)
    per_iteration_parity(m, gp, opt, x0[0], tgt[0], np.zeros(m.n), 0.2, 2)


def test_group_rollout_cost_and_uneven_mix():
    """FP64 cost of long chains and a batch that mixes thread- and group-per-rollout sizes."""
    seed = 55
    shapes = [(12, 8, 64), (10, 33, 96), (8, 61, 64)]
    x0s, tgts = [], []
    for i, (N, M, K) in enumerate(shapes):
        x0, tg = I.chain_instances(seed + i, 1, M)
        x0s.append(x0[0])
        tgts.append(tg[0])
    gp = G.chain_problem(M=8, N=12, K=64, iterations=1, lam=1e-2, sigma0=0.2, seed=seed, precision=G.PREC_FP32)
    s = G.Solver(gp, 3, shapes=shapes)
    rng = np.random.default_rng(0)
    Us = [rng.normal(0, 0.3, size=N * 2) for (N, M, K) in shapes]
    C = s.cost(np.concatenate(x0s), np.concatenate(tgts), np.concatenate(Us))
    for i, (N, M, K) in enumerate(shapes):
        assert C[i] == pytest.approx(O.cost(O.chain(M=M, N=N), x0s[i], tgts[i], Us[i]), rel=1e-12)
    sig = np.concatenate([np.full(N * 2, 0.2) for (N, M, K) in shapes])
    st, U, rep = s.step(np.concatenate(x0s), np.concatenate(tgts), np.zeros(sum(N * 2 for N, _, _ in shapes)), sig, 0)
    for i, (N, M, K) in enumerate(shapes):
        it = O.iteration(O.chain(M=M, N=N), O.Options(K=K, lam=1e-2, seed=seed), x0s[i], tgts[i], np.zeros(N * 2),
                         0.2, inst=i, it=0)
        assert rep[i].C_nom == pytest.approx(it.C_nom, rel=TOLRED)
        np.testing.assert_allclose(s.debug("C", i), it.C_samp, rtol=TOLRED)
    s.close()


_SWEEP_ORACLE = {}
# (M, N, K, seed): the benchmark problem, then the high-dimensional sweep's sizes
_STEP_SIZES = [(10, 100, 2048, I.BASE_SEED + 1), (32, 200, 4096, 32), (64, 200, 4096, 64)]


def _sweep_oracle(M, N, K, seed):
    """The oracle's first iteration of a chain at U = 0, cached per size."""
    key = (M, N, K, seed)
    if key not in _SWEEP_ORACLE:
        x0, tgt = I.chain_instances(seed, 1, M)
        m = O.chain(M=M, N=N)
        it = O.iteration(m, O.Options(K=K, lam=1e-3, seed=seed, threads=16), x0[0], tgt[0], np.zeros(m.n), 0.2,
                         want_big=True)
        _SWEEP_ORACLE[key] = (m, x0[0], tgt[0], it)
    return _SWEEP_ORACLE[key]


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16])
@pytest.mark.parametrize("M,N,K,seed", _STEP_SIZES)
def test_reduced_precision_iteration_at_sweep_sizes(M, N, K, seed, prec):
    """One iteration against the oracle at the benchmark size (chain M = 10,
    N = 100, K = 2048) and the high-dimensional sweep's sizes (M = 32 / 64,
    nx = 124 / 252, N = 200, n = 400, nR = 12862 / 25726, K = 4096; group-per-
    rollout kernels).  Every sample cost and the nominal cost within 1e-4; dR
    within 1e-4 normwise (the FP32 group model keeps positions relative to the
    initial state); the cost after the step within 1e-4 as well (the Gram sums
    P^T P over at most 2048 columns per FP32 accumulator and adds the chunks
    in FP64: with one accumulator over nR = 12862 rows its rounding moved
    this step's cost by 2.4e-4 at M = 32).  Prints the measured deviations
    and, for reference, 4 kappa(J^T J + lambda I) u_FP32 (pytest -s)."""
    m, x0, tgt, it = _sweep_oracle(M, N, K, seed)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
    s = G.Solver(gp, 1)
    st, U, rep = s.step(x0, tgt, np.zeros(m.n), np.full(m.n, 0.2), 0)
    Cs = s.debug("C")
    dR = s.debug("dR").reshape(m.nR, K // 2)
    s.close()
    assert st == 0
    assert rep[0].C_nom == pytest.approx(it.C_nom, rel=TOLRED)
    np.testing.assert_allclose(Cs, it.C_samp, rtol=TOLRED)
    e_dR = rel(dR, it.dR.T)
    assert e_dR < TOLRED
    H = it.J.T @ it.J + it.lambda_used * np.eye(m.n)
    kap = np.linalg.cond(H)
    e_new = abs(rep[0].C_new - it.C_new) / it.C_new
    print(f"\nchain M={M} N={N} K={K} prec={prec}: dR {e_dR:.2e}, samples max "
          f"{np.max(np.abs(Cs - it.C_samp) / np.abs(it.C_samp)):.2e}, C_new {e_new:.2e}, "
          f"kappa(J^T J + lambda I) {kap:.3e}, bound {max(TOLRED, 4 * kap * U32):.2e}")
    assert rep[0].C_new < rep[0].C_nom and it.C_new < it.C_nom
    assert e_new <= TOLRED


def test_reduced_precision_indefinite_lsq_system_takes_the_diagonal_shift():
    """The same near-singular draw without injection.  The FP64 mode factors
    the damped LSQ system at once, like the oracle.  In the reduced modes the
    tensor-core Gram's rounding (~1e-5 of sqrt(A_ii A_jj)) can leave
    P^T P + lambda S^2 indefinite when S is this ill-conditioned; the retry
    then adds tau diag(A) (tau = 1e-5, 1e-4, 1e-3) at the stated lambda
    before it raises lambda, so the step stays in the LSQ form at lambda =
    1e-3 and close to the oracle's (the shift perturbs the system by at most
    1e-3 of its diagonal)."""
    seed = I.BASE_SEED + 77
    Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, 24)
    b = 23
    M, N, K = int(Ms[b]), int(Ns[b]), int(Ks[b])
    m = O.chain(M=M, N=N)
    ref = O.iteration(m, O.Options(K=K, lam=1e-3, seed=seed, threads=8), x0s[b], tgts[b], np.zeros(m.n), 0.2,
                      inst=0, it=0)
    assert ref.status == 0 and ref.jac_mode_used == 0 and ref.chol_retries == 0
    for prec in (G.PREC_FP64, G.PREC_FP32, G.PREC_BF16):
        gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
        s = G.Solver(gp, 1)
        st, U, rep = s.step(x0s[b], tgts[b], np.zeros(m.n), np.full(m.n, 0.2), 0)
        s.close()
        r = rep[0]
        print(f"\nprec={prec}: retries {r.chol_retries}, lambda {r.lambda_used:.1e}, jac_mode {r.jac_mode_used}, "
              f"C_new {r.C_new:.9e} vs oracle {ref.C_new:.9e} ({abs(r.C_new - ref.C_new) / ref.C_nom:.2e} of C_nom)")
        assert st == 0 and r.status == 0 and r.jac_mode_used == 0
        if prec == G.PREC_FP64:
            assert r.chol_retries == 0
            assert r.C_new == pytest.approx(ref.C_new, rel=2e-6)
        else:
            assert r.chol_retries <= 3 and r.lambda_used == 1e-3
            assert r.C_new < r.C_nom
            assert abs(r.C_new - ref.C_new) <= 1e-3 * ref.C_nom


def test_reduced_precision_lsq_breakdown_takes_the_printed_form():
    """K' = 256 pairs barely above n = 246: S is nearly singular (kappa(S)
    ~ 5.6e3), the case the LSQ-breakdown reading of Eq. 9 exists for.  With
    the breakdown forced at iteration 0 (host-side injection, and the
    oracle's hook) every precision takes the printed Monte Carlo form
    J = P Sigma^-1 / K' (jac_mode_used 1) and agrees with the oracle run with
    the same breakdown; without it the FP64 mode solves the LSQ system, like
    the oracle in AUTO mode."""
    seed = I.BASE_SEED + 77
    Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, 24)
    b = 23
    M, N, K = int(Ms[b]), int(Ns[b]), int(Ks[b])
    assert (M, N, K) == (8, 123, 512)
    m = O.chain(M=M, N=N)
    it_brk = O.iteration(m, O.Options(K=K, lam=1e-3, seed=seed, break_it=0, break_kind="system", threads=8), x0s[b],
                         tgts[b], np.zeros(m.n), 0.2, inst=0, it=0, want_big=True)
    it_auto = O.iteration(m, O.Options(K=K, lam=1e-3, seed=seed, threads=8), x0s[b], tgts[b], np.zeros(m.n), 0.2,
                          inst=0, it=0)
    assert it_brk.status == 0 and it_auto.status == 0
    assert it_brk.jac_mode_used == 1 and it_auto.jac_mode_used == 0
    for prec, inject in ((G.PREC_FP64, True), (G.PREC_FP32, True), (G.PREC_BF16, True), (G.PREC_FP64, False)):
        ref = it_brk if inject else it_auto
        gp = G.chain_problem(M=M, N=N, K=K, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, precision=prec)
        s = G.Solver(gp, 1)
        if inject:
            G.gnmppi_debug_inject(s.h, G.INJECT_LSQ_BREAKDOWN, 0)
        st, U, rep = s.step(x0s[b], tgts[b], np.zeros(m.n), np.full(m.n, 0.2), 0)
        s.close()
        assert st == 0 and rep[0].status == 0
        assert rep[0].jac_mode_used == ref.jac_mode_used
        assert rep[0].C_nom == pytest.approx(ref.C_nom, rel=TOLRED)
        assert rep[0].C_new < rep[0].C_nom
        if prec == G.PREC_FP64 and inject:
            assert rep[0].C_new == pytest.approx(ref.C_new, rel=TOL64)
        elif prec == G.PREC_FP64:
            # the scaled system (P^T P + lambda S^2) y = -b has kappa up to
            # kappa(S)^2 kappa(J^T J + lambda I) ~ 3e7 * 470 here, so the step,
            # and the cost after it, agree to ~kappa u = 1.6e-6
            assert rep[0].C_new == pytest.approx(ref.C_new, rel=2e-6)
        else:
            # the printed form's system is ill-conditioned for this draw: the
            # FP32 rounding of the rollouts that form J moves the step by up to
            # kappa(J^T J + lambda I) u_FP32 (the forward-error bound of the
            # FP64 tests with FP32's unit roundoff), and the cost after it with it
            H = ref.J.T @ ref.J + ref.lambda_used * np.eye(m.n)
            assert rep[0].C_new == pytest.approx(ref.C_new, rel=max(TOLRED, 4.0 * np.linalg.cond(H) * U32))


# ------------------------------------------- Methods E and C (Sec. 5, Sec. 3)
def test_fp64_method_e_sigma_points_pendulum_per_iteration():
    """Method E: the n = 50 sigma-point pairs +-sqrt(n) s_i e_i instead of
    Philox draws (K ignored), per-iteration FP64 parity with the oracle."""
    seed = I.BASE_SEED + 5
    x0 = I.pendulum_x0(seed, 1)[0]
    m = O.pendulum()
    opt = O.Options(K=2, iterations=8, lam=1e-3, seed=seed, sampling="sigma")
    gp = G.pendulum_problem(N=50, K=2, iterations=8, lam=1e-3, sigma0=0.5, seed=seed, sampling=G.SAMPLE_SIGMA)
    its = per_iteration_parity(m, gp, opt, x0, None, np.zeros(m.n), 0.5, 8)
    assert all(it.jac_mode_used == 0 for it in its)


def test_fp64_method_e_sigma_points_chain_per_iteration():
    """Method E on a chain, M = 5, N = 30 (n = 60 pairs, 8 rows of 4 lanes ragged)."""
    seed = I.BASE_SEED + 6
    M, N = 5, 30
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    opt = O.Options(K=2, iterations=4, lam=1e-3, seed=seed, sampling="sigma")
    gp = G.chain_problem(M=M, N=N, K=2, iterations=4, lam=1e-3, sigma0=0.2, seed=seed, sampling=G.SAMPLE_SIGMA)
    per_iteration_parity(m, gp, opt, x0[0], tgt[0], np.zeros(m.n), 0.2, 4)


def test_fp64_method_c_mppi_step_pendulum_per_iteration():
    """Method C: the MPPI step of Eq. 5 taken whole (alpha = 1), per-iteration
    FP64 parity with the oracle (same samples as Method D)."""
    seed = I.BASE_SEED + 7
    x0 = I.pendulum_x0(seed, 1)[0]
    m = O.pendulum()
    opt = O.Options(K=256, iterations=6, L=1, lam=1e-3, seed=seed, method="mppi")
    gp = G.pendulum_problem(N=50, K=256, iterations=6, lam=1e-3, sigma0=0.5, seed=seed, method=G.METHOD_MPPI)
    its = per_iteration_parity(m, gp, opt, x0, None, np.zeros(m.n), 0.5, 6)
    assert all(it.alpha == 1.0 and it.jac_mode_used == -1 for it in its)


def test_method_e_reduced_precision_and_group_chain():
    """Method E in FP32 mode on a 40-mass chain (group-per-rollout kernel): the
    sample costs and the step's cost against the FP64 oracle."""
    seed = I.BASE_SEED + 8
    M, N = 40, 12
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N)
    it = O.iteration(m, O.Options(K=2, lam=1e-3, seed=seed, sampling="sigma"), x0[0], tgt[0], np.zeros(m.n), 0.2)
    gp = G.chain_problem(M=M, N=N, K=2, iterations=1, lam=1e-3, sigma0=0.2, seed=seed, sampling=G.SAMPLE_SIGMA,
                         precision=G.PREC_FP32)
    s = G.Solver(gp, 1)
    st, U, rep = s.step(x0[0], tgt[0], np.zeros(m.n), np.full(m.n, 0.2), 0)
    Cs = s.debug("C")
    s.close()
    assert st == 0
    np.testing.assert_allclose(Cs, it.C_samp, rtol=TOLRED)
    assert rep[0].C_new == pytest.approx(it.C_new, rel=TOLRED)


# -------------------------------------------- the test problems of Sec. 5 ----
@pytest.mark.parametrize("name,U0,s0,sampling,method,K,T", [
    ("rosenbrock", (0.0, 0.0), 0.5, "random", "gn", 64, 10),     # Problem I, Method D
    ("rosenbrock", (0.0, 0.0), 0.5, "sigma", "gn", 2, 10),       # Problem I, Method E
    ("rastrigin", (1.9, 1.7), 1.0, "sigma", "gn", 2, 10),        # Problem II, Method E
    ("rastrigin", (1.9, 1.7), 1.0, "random", "mppi", 512, 6),    # Problem II, Method C
    ("heaviside", (0.5,), 0.5, "random", "gn", 256, 5),          # Problem III, Method D
])
def test_fp64_test_problems_per_iteration(name, U0, s0, sampling, method, K, T):
    """Problems I-III (static residuals, N = 1) through the batched kernels,
    per-iteration FP64 parity with the oracle, from the paper's initial guesses."""
    seed = I.BASE_SEED + 9
    m = O.testfun(name)
    L = 1 if method == "mppi" else 16
    opt = O.Options(K=K, iterations=T, L=L, lam=1e-3, seed=seed, sampling=sampling, method=method)
    gp = G.testfun_problem(name, K=K, iterations=T, lam=1e-3, sigma0=s0, seed=seed,
                           sampling=G.SAMPLE_SIGMA if sampling == "sigma" else G.SAMPLE_RANDOM,
                           method=G.METHOD_MPPI if method == "mppi" else G.METHOD_GN)
    per_iteration_parity(m, gp, opt, np.zeros(1), None, np.array(U0, float), s0, T)


# ------------------------------------- Setting V.ii: dead-zone friction ---
def test_fp64_dead_zone_friction_pendulum_per_iteration():
    """Pendulum swing-up with dead-zone friction u_f = 0.5 at the input
    (nonsmooth in U), per-iteration FP64 parity with the oracle."""
    seed = I.BASE_SEED + 10
    x0 = I.pendulum_x0(seed, 1)[0]
    m = O.pendulum(u_friction=0.5)
    opt = O.Options(K=256, iterations=10, lam=1e-3, seed=seed)
    gp = G.pendulum_problem(u_friction=0.5, N=50, K=256, iterations=10, lam=1e-3, sigma0=0.5, seed=seed)
    per_iteration_parity(m, gp, opt, x0, None, np.zeros(m.n), 0.5, 10)


def test_fp64_dead_zone_friction_chain_per_iteration():
    """Chain M = 5, N = 30 with dead-zone friction u_f = 0.2 per force component."""
    seed = I.BASE_SEED + 12
    M, N, K = 5, 30, 256
    x0, tgt = I.chain_instances(seed, 1, M)
    m = O.chain(M=M, N=N, u_friction=0.2)
    opt = O.Options(K=K, iterations=4, lam=1e-3, seed=seed)
    gp = G.chain_problem(M=M, u_friction=0.2, N=N, K=K, iterations=4, lam=1e-3, sigma0=0.2, seed=seed)
    per_iteration_parity(m, gp, opt, x0[0], tgt[0], np.zeros(m.n), 0.2, 4)


def test_async_solves_on_two_streams_match_blocking_solves():
    """gnmppi_solve_async + gnmppi_solve_wait on two handles and two streams,
    in flight together, give bitwise the blocking gnmppi_solve results; a
    second async call before the wait and a wait with nothing in flight are
    rejected."""
    import torch

    seed = I.BASE_SEED + 13
    M, N, K, B = 6, 20, 256, 8
    x0, tgt = I.chain_instances(seed, 2 * B, M)
    gp = G.chain_problem(M=M, N=N, K=K, iterations=5, lam=1e-3, sigma0=0.2, seed=seed, precision=G.PREC_FP32)
    dev = torch.device("cuda")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hs = [G.gnmppi_create(gp, B, None, s.cuda_stream) for s in streams]
    try:
        xs = [torch.tensor(x0[i * B:(i + 1) * B].ravel(), dtype=torch.float64, device=dev) for i in range(2)]
        ts = [torch.tensor(tgt[i * B:(i + 1) * B].ravel(), dtype=torch.float64, device=dev) for i in range(2)]
        ref = []
        for h, x, t in zip(hs, xs, ts):
            U = torch.zeros(B * 2 * N, dtype=torch.float64, device=dev)
            st, rep = G.gnmppi_solve(h, G.MEM_DEVICE, x, t, U, None, B)
            ref.append((U.cpu().numpy(), [r.C_final for r in rep]))
        Us = [torch.zeros(B * 2 * N, dtype=torch.float64, device=dev) for _ in range(2)]
        torch.cuda.synchronize()
        for h, x, t, U in zip(hs, xs, ts, Us):
            G.gnmppi_solve_async(h, G.MEM_DEVICE, x, t, U, None)
        with pytest.raises(G.GnmppiError):
            G.gnmppi_solve_async(hs[0], G.MEM_DEVICE, xs[0], ts[0], Us[0], None)
        for i, h in enumerate(hs):
            st, rep = G.gnmppi_solve_wait(h, B)
            assert st == 0
            assert np.array_equal(Us[i].cpu().numpy(), ref[i][0])
            assert [r.C_final for r in rep] == ref[i][1]
        with pytest.raises(G.GnmppiError):
            G.gnmppi_solve_wait(hs[0], B)
    finally:
        for h in hs:
            G.gnmppi_destroy(h)


def test_split_batch_with_first_instance_matches_the_unsplit_batch():
    """A batch split into contiguous ranges over several handles (as the
    multi-GPU benchmark splits it over ranks), each handle given its range's
    first instance, draws the same noise and gives bitwise the same solves as
    the unsplit batch."""
    seed = I.BASE_SEED + 14
    M, N, K, B = 6, 20, 256, 8
    x0, tgt = I.chain_instances(seed, B, M)
    n = 2 * N
    ref = G.Solver(G.chain_problem(M=M, N=N, K=K, iterations=4, lam=1e-3, sigma0=0.2, seed=seed,
                                   precision=G.PREC_BF16), B)
    st, U_all, rep_all = ref.solve(x0, tgt, np.zeros(B * n))
    ref.close()
    assert st == 0
    for lo, hi in ((0, 3), (3, 8)):
        s = G.Solver(G.chain_problem(M=M, N=N, K=K, iterations=4, lam=1e-3, sigma0=0.2, seed=seed,
                                     precision=G.PREC_BF16, first_instance=lo), hi - lo)
        st, U, rep = s.solve(x0[lo:hi], tgt[lo:hi], np.zeros((hi - lo) * n))
        s.close()
        assert st == 0
        assert np.array_equal(U, U_all[lo * n: hi * n])
        assert [r.C_final for r in rep] == [r.C_final for r in rep_all[lo:hi]]
    # without the offset the second range draws other noise
    s = G.Solver(G.chain_problem(M=M, N=N, K=K, iterations=4, lam=1e-3, sigma0=0.2, seed=seed,
                                 precision=G.PREC_BF16), 5)
    st, U, rep = s.solve(x0[3:8], tgt[3:8], np.zeros(5 * n))
    s.close()
    assert not np.array_equal(U, U_all[3 * n: 8 * n])
