/*
 * gnmppi_oracle.c -- plain FP64 CPU oracle for Gauss-Newton accelerated MPPI.
 *
 * TEST INFRASTRUCTURE ONLY (see gnmppi_oracle.h): loaded by the tests, the
 * smoke check and the benchmark's CPU-baseline leg, never by the product.
 *
 * Every routine follows the paper (Homburger, Baumgaertner, Diehl, Reuter,
 * "Gauss-Newton accelerated MPPI Control", arXiv 2512.04579) step by step,
 * in FP64, with textbook loops and no blocking or fusion:
 *   - simulator X = F(x0, U) and cost C = sum L_k + E            (Sec. 2, Eq. 1-2)
 *   - convex-over-unknown C = Phi(R(U)), Phi = 0.5 ||R||^2        (Sec. 2, Eq. 4)
 *   - softmin sample weights and the weighted mean perturbation    (Sec. 3, Eq. 3-5)
 *   - Gaussian-smoothing Jacobian E[R(U+W) W^T] Sigma^-1            (Sec. 4.1, Eq. 7)
 *   - GGN step -B^-1 grad with B = J^T J                            (Sec. 4.2, Eq. 9)
 *   - step-length set {gamma^j}, argmin line search, Sigma <- beta Sigma
 *                                                                  (Algorithm 1, Eq. 10-11)
 *   - Method A (GGN with a central finite-difference Jacobian)      (Sec. 5) for C*.
 * Readings taken where the paper is silent (the regression form of the
 * Jacobian, the damping lambda, beta, gamma, L, tau, the dynamics of the
 * synthetic workloads) are stated at each routine.
 *
 * Built with -ffp-contract=off so that x86 and Arm hosts round identically.
 */
#include "gnmppi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC 2011).            */
/* ------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { /* key schedule: Weyl increments between rounds */
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    philox_round(c, k);
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* 53 random bits from two words, mapped into the open interval (0, 1]:
 * u = (hi * 2^21 + lo / 2^11) * 2^-53 + 2^-54. */
double orc_uniform53(uint32_t hi, uint32_t lo) {
  const uint64_t x = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return (double)x * 0x1p-53 + 0x1p-54;
}

/* The noise stream.  Normal z_j, j < n, of sample m at iteration `it` of
 * instance `inst`: Philox counter (j/2, m, it, inst*16 + 0), key = seed;
 * Box-Muller on the two uniforms of the four output words gives
 * z_{2q} = r cos(2 pi u2), z_{2q+1} = r sin(2 pi u2), r = sqrt(-2 ln u1). */
void orc_normals(uint64_t seed, uint32_t inst, uint32_t it, uint32_t m, int32_t n, double* z) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int32_t q = 0; 2 * q < n; ++q) {
    const uint32_t ctr[4] = {(uint32_t)q, m, it, (inst << 4) | 0u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const double u1 = orc_uniform53(w[0], w[1]);
    const double u2 = orc_uniform53(w[2], w[3]);
    const double rad = sqrt(-2.0 * log(u1));
    const double t = 6.283185307179586 * u2;
    z[2 * q] = rad * cos(t);
    if (2 * q + 1 < n) z[2 * q + 1] = rad * sin(t);
  }
}

/* ------------------------------------------------------------------ */
/* Models: dimensions, dynamics, residuals.                            */
/* ------------------------------------------------------------------ */
int32_t orc_n(const orc_model* m) { return m->N * m->nu; }

int32_t orc_nR(const orc_model* m) {
  switch (m->dyn) {
    case ORC_DYN_PENDULUM: return 3 * m->N + 2;
    case ORC_DYN_CHAIN: return m->N * (2 * (m->M - 1) + 2) + 2 * (m->M - 1);
    case ORC_DYN_LINEAR: return m->N * (m->nx + m->nu) + m->nx;
    case ORC_DYN_ROSENBROCK: return 2;
    case ORC_DYN_RASTRIGIN: return 4;
    case ORC_DYN_HEAVISIDE: return 1;
    default: return -1;
  }
}

/* Continuous-time right-hand sides x' = f(x, u).
 *  Pendulum (x = [theta, omega]):  theta'' = -(g/l) sin theta - b omega + u/(m l^2).
 *  Chain: masses 0..M-1, mass 0 fixed at the origin, free masses 1..M-1 with
 *    state [p_1..p_{M-1}, v_1..v_{M-1}] (2-D each).  Link i joins masses i-1
 *    and i: d = |p_i - p_{i-1}| - l0, tension f = k d + k3 d^3, force -f e on
 *    mass i and +f e on mass i-1 (e the unit vector from i-1 to i), rest
 *    length l0 = 1/(M-1), viscous damping -c v_i, control force u on mass
 *    M-1, gravity g along -y (the chain hangs in a vertical plane).
 *    params = {mass, k, k3, c, g}. */
void orc_deriv(const orc_model* m, const double* x, const double* u, double* xdot) {
  if (m->dyn == ORC_DYN_PENDULUM) {
    const double g = m->params[0], l = m->params[1], ms = m->params[2], b = m->params[3];
    xdot[0] = x[1];
    xdot[1] = -(g / l) * sin(x[0]) - b * x[1] + u[0] / (ms * l * l);
    return;
  }
  if (m->dyn == ORC_DYN_CHAIN) {
    const int F = m->M - 1; /* free masses */
    const double mass = m->params[0], k = m->params[1], k3 = m->params[2], c = m->params[3];
    const double l0 = 1.0 / (double)F;
    const double* p = x;
    const double* v = x + 2 * F;
    double* pd = xdot;
    double* vd = xdot + 2 * F;
    for (int i = 0; i < F; ++i) {
      pd[2 * i] = v[2 * i];
      pd[2 * i + 1] = v[2 * i + 1];
      vd[2 * i] = -c * v[2 * i];
      vd[2 * i + 1] = -c * v[2 * i + 1];
    }
    for (int i = 1; i <= F; ++i) { /* link between mass i-1 and mass i */
      const double px0 = (i == 1) ? 0.0 : p[2 * (i - 2)];
      const double py0 = (i == 1) ? 0.0 : p[2 * (i - 2) + 1];
      const double dx = p[2 * (i - 1)] - px0;
      const double dy = p[2 * (i - 1) + 1] - py0;
      const double len = sqrt(dx * dx + dy * dy);
      const double d = len - l0;
      const double f = k * d + k3 * d * d * d;
      const double fx = f * dx / len, fy = f * dy / len;
      vd[2 * (i - 1)] -= fx;
      vd[2 * (i - 1) + 1] -= fy;
      if (i >= 2) {
        vd[2 * (i - 2)] += fx;
        vd[2 * (i - 2) + 1] += fy;
      }
    }
    vd[2 * (F - 1)] += u[0];
    vd[2 * (F - 1) + 1] += u[1];
    for (int i = 0; i < 2 * F; ++i) vd[i] /= mass;
    for (int i = 0; i < F; ++i) vd[2 * i + 1] -= m->params[4]; /* gravity along -y */
    return;
  }
  if (m->dyn == ORC_DYN_LINCONT) {
    const int nx = m->nx, nu = m->nu;
    const double* A = m->lin;
    const double* B = m->lin + nx * nx;
    for (int i = 0; i < nx; ++i) {
      double s = 0.0;
      for (int j = 0; j < nx; ++j) s += A[i * nx + j] * x[j];
      for (int j = 0; j < nu; ++j) s += B[i * nu + j] * u[j];
      xdot[i] = s;
    }
  }
}

/* One step of the classical explicit Runge-Kutta method of order 4 with the
 * control held constant over the step (the discretisation Sec. 5 names). */
void orc_rk4_step(const orc_model* m, const double* x, const double* u, double* xn) {
  const int nx = m->nx;
  const double h = m->dt;
  double k1[256], k2[256], k3[256], k4[256], t[256];
  orc_deriv(m, x, u, k1);
  for (int i = 0; i < nx; ++i) t[i] = x[i] + 0.5 * h * k1[i];
  orc_deriv(m, t, u, k2);
  for (int i = 0; i < nx; ++i) t[i] = x[i] + 0.5 * h * k2[i];
  orc_deriv(m, t, u, k3);
  for (int i = 0; i < nx; ++i) t[i] = x[i] + h * k3[i];
  orc_deriv(m, t, u, k4);
  for (int i = 0; i < nx; ++i) xn[i] = x[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* X = F(x0, U), Eq. 1: X holds x_0 .. x_N, (N+1)*nx values. */
int32_t orc_rollout(const orc_model* m, const double* x0, const double* U, double* X) {
  const int nx = m->nx, nu = m->nu, N = m->N;
  if (nx <= 0 || nx > 256) return ORC_E_ARG;
  memcpy(X, x0, sizeof(double) * nx);
  for (int k = 0; k < N; ++k) {
    const double* xk = X + k * nx;
    double* xk1 = X + (k + 1) * nx;
    const double* uk = U + k * nu;
    if (m->dyn == ORC_DYN_LINEAR) {
      const double* A = m->lin;
      const double* B = m->lin + nx * nx;
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int j = 0; j < nx; ++j) s += A[i * nx + j] * xk[j];
        for (int j = 0; j < nu; ++j) s += B[i * nu + j] * uk[j];
        xk1[i] = s;
      }
    } else {
      /* Setting V.ii (Sec. 5): dead-zone friction at the input of the dynamics,
       * u_apply = 0 where |u| <= u_friction (per component; u_friction = 0: off) */
      const double uf = (m->dyn == ORC_DYN_PENDULUM) ? m->params[4] : (m->dyn == ORC_DYN_CHAIN ? m->params[5] : 0.0);
      double ua[8];
      for (int j = 0; j < nu && j < 8; ++j) ua[j] = (uf > 0.0 && fabs(uk[j]) <= uf) ? 0.0 : uk[j];
      orc_rk4_step(m, xk, nu <= 8 ? ua : uk, xk1);
    }
  }
  return ORC_OK;
}

/* Inner function R(x0, U) of the convex-over-unknown cost (Eq. 4), with
 * outer function Phi(R) = 0.5 ||R||^2 throughout.
 *  Pendulum: stage k < N: [theta_k - pi, 0.1 omega_k, 0.1 u_k];
 *            terminal [10 (theta_N - pi), 10 omega_N].
 *  Chain:    stage k < N: [p_{i,k} - p*_i (i = 1..M-1), 0.1 u_k];
 *            terminal [p_{i,N} - p*_i];  xref holds p*.
 *  Linear:   stage k < N: [wq .* x_k, wr .* u_k]; terminal wqN .* x_N.
 *  Rosenbrock (Problem I):  [sqrt2 (1 - u1), sqrt200 (u2 - u1^2)].
 *  Rastrigin (Problem II):  sqrt2 [u1, u2, sqrt(5 - 5cos 2pi u1), sqrt(5 - 5cos 2pi u2)]
 *            (the paper's R with Phi = ||R||^2, rescaled so Phi = 0.5||R||^2).
 *  Heaviside (Problem III): [H(u)], H(u) = 1 for u >= 0, else 0. */
int32_t orc_residual(const orc_model* m, const double* x0, const double* xref, const double* U, double* R) {
  const int nx = m->nx, nu = m->nu, N = m->N;
  if (m->dyn == ORC_DYN_ROSENBROCK) {
    R[0] = sqrt(2.0) * (1.0 - U[0]);
    R[1] = sqrt(200.0) * (U[1] - U[0] * U[0]);
    return ORC_OK;
  }
  if (m->dyn == ORC_DYN_RASTRIGIN) {
    const double pi = 3.141592653589793;
    R[0] = sqrt(2.0) * U[0];
    R[1] = sqrt(2.0) * U[1];
    R[2] = sqrt(2.0) * sqrt(5.0 - 5.0 * cos(2.0 * pi * U[0]));
    R[3] = sqrt(2.0) * sqrt(5.0 - 5.0 * cos(2.0 * pi * U[1]));
    return ORC_OK;
  }
  if (m->dyn == ORC_DYN_HEAVISIDE) {
    R[0] = (U[0] >= 0.0) ? 1.0 : 0.0;
    return ORC_OK;
  }
  double* X = (double*)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nx);
  if (!X) return ORC_E_ARG;
  int32_t st = orc_rollout(m, x0, U, X);
  if (st != ORC_OK) {
    free(X);
    return st;
  }
  int row = 0;
  if (m->dyn == ORC_DYN_PENDULUM) {
    const double pi = 3.141592653589793;
    for (int k = 0; k < N; ++k) {
      R[row++] = X[k * 2] - pi;
      R[row++] = 0.1 * X[k * 2 + 1];
      R[row++] = 0.1 * U[k];
    }
    R[row++] = 10.0 * (X[N * 2] - pi);
    R[row++] = 10.0 * X[N * 2 + 1];
  } else if (m->dyn == ORC_DYN_CHAIN) {
    const int F = m->M - 1;
    for (int k = 0; k <= N; ++k) {
      const double* xk = X + k * nx;
      for (int i = 0; i < 2 * F; ++i) R[row++] = xk[i] - xref[i];
      if (k < N)
        for (int j = 0; j < nu; ++j) R[row++] = 0.1 * U[k * nu + j];
    }
  } else if (m->dyn == ORC_DYN_LINEAR) {
    const double* wq = m->lin + nx * nx + nx * nu;
    const double* wr = wq + nx;
    const double* wqN = wr + nu;
    for (int k = 0; k < N; ++k) {
      for (int i = 0; i < nx; ++i) R[row++] = wq[i] * X[k * nx + i];
      for (int j = 0; j < nu; ++j) R[row++] = wr[j] * U[k * nu + j];
    }
    for (int i = 0; i < nx; ++i) R[row++] = wqN[i] * X[N * nx + i];
  } else {
    free(X);
    return ORC_E_ARG;
  }
  free(X);
  return ORC_OK;
}

/* C(U) = Phi(R(U)) = 0.5 ||R(U)||^2  (Eq. 2 and Eq. 4). */
double orc_cost(const orc_model* m, const double* x0, const double* xref, const double* U) {
  const int nR = orc_nR(m);
  double* R = (double*)malloc(sizeof(double) * (size_t)nR);
  orc_residual(m, x0, xref, U, R);
  double s = 0.0;
  for (int i = 0; i < nR; ++i) s += R[i] * R[i];
  free(R);
  return 0.5 * s;
}

/* ------------------------------------------------------------------ */
/* Softmin weights of Eq. 5, omega = exp(-C / tau), evaluated after the */
/* exact shift by min C.  stats = {min C, sum w, sum w^2, ESS}.         */
/* ------------------------------------------------------------------ */
int32_t orc_softmin(int32_t count, const double* C, const uint8_t* valid, double tau, double* w, double* stats) {
  double cmin = INFINITY;
  for (int i = 0; i < count; ++i)
    if (!valid || valid[i])
      if (C[i] < cmin) cmin = C[i];
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < count; ++i) {
    double wi = 0.0;
    if ((!valid || valid[i]) && isfinite(cmin)) wi = exp(-(C[i] - cmin) / tau);
    w[i] = wi;
    s1 += wi;
    s2 += wi * wi;
  }
  stats[0] = cmin;
  stats[1] = s1;
  stats[2] = s2;
  stats[3] = (s2 > 0.0) ? s1 * s1 / s2 : 0.0;
  return isfinite(cmin) ? ORC_OK : ORC_E_NONFINITE;
}

/* ------------------------------------------------------------------ */
/* Dense linear algebra (textbook).                                    */
/* ------------------------------------------------------------------ */
/* In-place Cholesky A = L L^T (row-major, lower triangle overwritten).  */
int32_t orc_cholesky(int32_t n, double* A) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0) || !isfinite(d)) return ORC_E_NOT_PD;
    const double ljj = sqrt(d);
    A[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / ljj;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
  return ORC_OK;
}

/* Solve L L^T x = b in place (forward then backward substitution). */
void orc_chol_solve(int32_t n, const double* Lf, double* b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= Lf[i * n + k] * b[k];
    b[i] = s / Lf[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= Lf[k * n + i] * b[k];
    b[i] = s / Lf[i * n + i];
  }
}

/* Solve (G + lambda I) x = rhs with Cholesky and `ir` steps of iterative
 * refinement; on a non-positive pivot lambda grows tenfold (at most six
 * times).  Returns the number of increases, or ORC_E_NOT_PD. */
static int32_t damped_solve(int n, const double* G, double lambda, const double* rhs, int ir, double* x,
                            double* lambda_used) {
  double* H = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* Lf = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* res = (double*)malloc(sizeof(double) * (size_t)n);
  int retries = 0;
  int32_t st = ORC_E_NOT_PD;
  for (; retries <= 6; ++retries) {
    for (int i = 0; i < n * n; ++i) H[i] = G[i];
    for (int i = 0; i < n; ++i) H[i * n + i] += lambda;
    memcpy(Lf, H, sizeof(double) * (size_t)n * (size_t)n);
    if (orc_cholesky(n, Lf) == ORC_OK) {
      st = ORC_OK;
      break;
    }
    lambda *= 10.0;
  }
  if (st == ORC_OK) {
    memcpy(x, rhs, sizeof(double) * (size_t)n);
    orc_chol_solve(n, Lf, x);
    for (int t = 0; t < ir; ++t) {
      for (int i = 0; i < n; ++i) {
        double s = rhs[i];
        for (int j = 0; j < n; ++j) s -= H[i * n + j] * x[j];
        res[i] = s;
      }
      orc_chol_solve(n, Lf, res);
      for (int i = 0; i < n; ++i) x[i] += res[i];
    }
  }
  *lambda_used = lambda;
  free(H);
  free(Lf);
  free(res);
  return st == ORC_OK ? retries : ORC_E_NOT_PD;
}

static int all_finite(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/* ------------------------------------------------------------------ */
/* One iteration of Algorithm 1 (Method D: random sampling of Eq. 7).   */
/* ------------------------------------------------------------------ */
/*
 * s holds the per-component standard deviation, Sigma_k = diag(s^2).
 *  1. nominal residual r = R(U_k) and cost C_nom;
 *  2. perturbations W_m = s .* z_m from the noise stream; antithetic pairs
 *     evaluate R(U_k + W_m) and R(U_k - W_m), one-sided samples R(U_k + W_m);
 *     samples with a non-finite residual are dropped (their pair with them);
 *  3. softmin weights over all evaluated sample costs (Eq. 5), the weighted
 *     mean perturbation (Eq. 3) and the effective sample size -- reported,
 *     not used by the GGN step (Algorithm 1 does not use them);
 *  4. Jacobian of the smoothed residual (Eq. 7).  With dR_m = (R+ - R-)/2
 *     (antithetic) or R(U+W_m) - r (one-sided, baseline subtracted),
 *     P = sum_m dR_m W_m^T and S = sum_m W_m W_m^T:
 *       SIGMA (the printed Monte Carlo form):  J = P Sigma^-1 / K'
 *       LSQ   (regression form: Sigma replaced by the sample second moment
 *              S/K' of the drawn W; exact for affine R):  J = P S^-1
 *       AUTO:  LSQ when the drawn W can have full column rank (K' >= n),
 *              SIGMA otherwise;
 *  5. GGN step (Eq. 9) with Phi = 0.5||R||^2, so grad Phi = R and
 *     hess Phi = I:  (J^T J + lambda I) delta = -J^T r, solved by Cholesky
 *     with iterative refinement.  Eq. 9 assumes B = J^T J positive definite;
 *     when the LSQ system has no Cholesky factor at any of the damping
 *     retries (a draw with K' barely above n leaves S nearly singular), the
 *     iteration takes the SIGMA form instead (reported as jac_mode_used);
 *  6. line search (Eq. 11) over A = {gamma^j, j < L} (plus 0 if monotone):
 *     alpha* = argmin C(U_k + alpha delta), ties to the smallest j;
 *  7. U_{k+1} = U_k + alpha* delta (Eq. 10).  The covariance shrink is
 *     applied by the caller (orc_solve).
 */
int32_t orc_iteration(const orc_model* m, const orc_options* o, const double* x0, const double* xref,
                      double* U, const double* s, uint32_t inst, uint32_t it, orc_record* rec) {
  const int n = orc_n(m), nR = orc_nR(m);
  const int sigma_pts = o->sampling == ORC_SAMPLE_SIGMA;
  if (n <= 0 || nR <= 0 || (o->K <= 0 && !sigma_pts) || o->L <= 0) return ORC_E_ARG;
  const int anti = o->antithetic ? 1 : 0;
  if (sigma_pts && !anti) return ORC_E_ARG;
  /* pairs (antithetic) or samples; the sigma points are the n pairs +-sqrt(n) s_i e_i */
  const int Kp = sigma_pts ? n : (anti ? o->K / 2 : o->K);
  if (Kp <= 0) return ORC_E_ARG;
  const int mppi_step = o->method == ORC_METHOD_MPPI;
  const int Lc = mppi_step ? 1 : o->L; /* MPPI takes its step whole: alpha = 1 */
  const int mono = mppi_step ? 0 : o->monotone;
  const int nsamp = anti ? 2 * Kp : Kp;

  double* r = (double*)calloc((size_t)nR, sizeof(double));
  double* W = (double*)calloc((size_t)Kp * n, sizeof(double));
  double* dR = (double*)calloc((size_t)Kp * nR, sizeof(double));
  double* Cs = (double*)calloc((size_t)nsamp, sizeof(double));
  uint8_t* valid = (uint8_t*)calloc((size_t)nsamp, 1);
  double* P = (double*)calloc((size_t)nR * n, sizeof(double));
  double* S = (double*)calloc((size_t)n * n, sizeof(double));
  double* J = (double*)calloc((size_t)nR * n, sizeof(double));
  double* G = (double*)calloc((size_t)n * n, sizeof(double));
  double* g = (double*)calloc((size_t)n, sizeof(double));
  double* delta = (double*)calloc((size_t)n, sizeof(double));
  double* wts = (double*)calloc((size_t)nsamp, sizeof(double));
  int32_t status = ORC_OK;

  /* 1. nominal residual */
  orc_residual(m, x0, xref, U, r);
  double C_nom = 0.0;
  for (int i = 0; i < nR; ++i) C_nom += r[i] * r[i];
  C_nom *= 0.5;

  /* 2. sample rollouts, independent over m */
  int threads = o->threads > 0 ? o->threads : 1;
  (void)threads;
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads)
  for (int mi = 0; mi < Kp; ++mi) {
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* Up = (double*)malloc(sizeof(double) * (size_t)n);
    double* Rp = (double*)malloc(sizeof(double) * (size_t)nR);
    double* Rm = (double*)malloc(sizeof(double) * (size_t)nR);
    if (sigma_pts) {
      for (int j = 0; j < n; ++j) z[j] = (j == mi) ? sqrt((double)n) : 0.0;
    } else {
      orc_normals(o->seed, inst, it, (uint32_t)mi, n, z);
    }
    double* Wm = W + (size_t)mi * n;
    for (int j = 0; j < n; ++j) Wm[j] = s[j] * z[j];
    for (int j = 0; j < n; ++j) Up[j] = U[j] + Wm[j];
    orc_residual(m, x0, xref, Up, Rp);
    double cp = 0.0;
    for (int i = 0; i < nR; ++i) cp += Rp[i] * Rp[i];
    cp *= 0.5;
    double* dRm = dR + (size_t)mi * nR;
    if (anti) {
      for (int j = 0; j < n; ++j) Up[j] = U[j] - Wm[j];
      orc_residual(m, x0, xref, Up, Rm);
      double cm = 0.0;
      for (int i = 0; i < nR; ++i) cm += Rm[i] * Rm[i];
      cm *= 0.5;
      Cs[2 * mi] = cp;
      Cs[2 * mi + 1] = cm;
      const int ok = all_finite(Rp, nR) && all_finite(Rm, nR) && isfinite(cp) && isfinite(cm);
      valid[2 * mi] = valid[2 * mi + 1] = (uint8_t)ok;
      for (int i = 0; i < nR; ++i) dRm[i] = ok ? 0.5 * (Rp[i] - Rm[i]) : 0.0;
    } else {
      Cs[mi] = cp;
      const int ok = all_finite(Rp, nR) && isfinite(cp);
      valid[mi] = (uint8_t)ok;
      for (int i = 0; i < nR; ++i) dRm[i] = ok ? Rp[i] - r[i] : 0.0;
    }
    free(z);
    free(Up);
    free(Rp);
    free(Rm);
  }
  int n_masked = 0, Keff = 0;
  for (int mi = 0; mi < Kp; ++mi) {
    const int ok = anti ? valid[2 * mi] : valid[mi];
    if (!ok) {
      ++n_masked;
      for (int j = 0; j < n; ++j) W[(size_t)mi * n + j] = 0.0; /* dropped from P and S */
    } else {
      ++Keff;
    }
  }

  /* 3. softmin diagnostics over every evaluated sample cost */
  double st4[4] = {0, 0, 0, 0};
  orc_softmin(nsamp, Cs, valid, o->tau, wts, st4);
  double* mppi = (double*)calloc((size_t)n, sizeof(double));
  if (st4[1] > 0.0) {
    for (int mi = 0; mi < Kp; ++mi) {
      const double* Wm = W + (size_t)mi * n;
      const double wsum = anti ? (wts[2 * mi] - wts[2 * mi + 1]) : wts[mi];
      for (int j = 0; j < n; ++j) mppi[j] += wsum * Wm[j];
    }
    for (int j = 0; j < n; ++j) mppi[j] /= st4[1];
  }
  if (rec && rec->mppi_dir) memcpy(rec->mppi_dir, mppi, sizeof(double) * (size_t)n);

  /* 4. P = sum dR_m W_m^T, S = sum W_m W_m^T (sums in sample order);
   *    the MPPI step (Method C) needs neither */
  for (int mi = 0; mi < (mppi_step ? 0 : Kp); ++mi) {
    const double* Wm = W + (size_t)mi * n;
    const double* dRm = dR + (size_t)mi * nR;
    for (int i = 0; i < nR; ++i) {
      const double a = dRm[i];
      for (int j = 0; j < n; ++j) P[(size_t)i * n + j] += a * Wm[j];
    }
    for (int i = 0; i < n; ++i) {
      const double a = Wm[i];
      for (int j = 0; j < n; ++j) S[(size_t)i * n + j] += a * Wm[j];
    }
  }
  int jm = mppi_step ? -1 : o->jac_mode; /* -1: no Jacobian (MPPI step) */
  if (jm == ORC_JAC_AUTO) jm = (Kp >= n) ? ORC_JAC_LSQ : ORC_JAC_SIGMA;
  if (Keff == 0) status = ORC_E_NONFINITE;
  if (status == ORC_OK && jm == ORC_JAC_LSQ) {
    /* J = P S^-1, i.e. S J^T = P^T: one Cholesky solve per row of P */
    double* Sf = (double*)malloc(sizeof(double) * (size_t)n * n);
    memcpy(Sf, S, sizeof(double) * (size_t)n * n);
    const int s_broken = o->break_kind == ORC_BREAK_S && (int32_t)it == o->break_it;
    if (!s_broken && orc_cholesky(n, Sf) == ORC_OK) {
      for (int i = 0; i < nR; ++i) {
        double* Ji = J + (size_t)i * n;
        memcpy(Ji, P + (size_t)i * n, sizeof(double) * (size_t)n);
        orc_chol_solve(n, Sf, Ji);
      }
    } else {
      jm = ORC_JAC_SIGMA; /* rank-deficient draw: fall back to the printed form */
    }
    free(Sf);
  }
  if (status == ORC_OK && jm == ORC_JAC_SIGMA) {
    for (int i = 0; i < nR; ++i)
      for (int j = 0; j < n; ++j) J[(size_t)i * n + j] = P[(size_t)i * n + j] / ((double)Keff * s[j] * s[j]);
  }

  /* 5. GGN step: G = J^T J, g = J^T r, (G + lambda I) delta = -g; an LSQ
   *    system without a Cholesky factor at any damping falls back to SIGMA */
  double lambda_used = o->lambda;
  int retries = 0;
  for (int pass = 0; status == ORC_OK && !mppi_step && pass < 2; ++pass) {
    if (pass == 1) {
      if (retries >= 0 || jm != ORC_JAC_LSQ) break;
      jm = ORC_JAC_SIGMA;
      for (int i = 0; i < nR; ++i)
        for (int j = 0; j < n; ++j) J[(size_t)i * n + j] = P[(size_t)i * n + j] / ((double)Keff * s[j] * s[j]);
    }
    for (int a = 0; a < n; ++a) {
      for (int b = 0; b < n; ++b) {
        double acc = 0.0;
        for (int i = 0; i < nR; ++i) acc += J[(size_t)i * n + a] * J[(size_t)i * n + b];
        G[a * n + b] = acc;
      }
      double acc = 0.0;
      for (int i = 0; i < nR; ++i) acc += J[(size_t)i * n + a] * r[i];
      g[a] = acc;
    }
    double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) rhs[j] = -g[j];
    retries = damped_solve(n, G, o->lambda, rhs, o->ir_steps, delta, &lambda_used);
    if (pass == 0 && jm == ORC_JAC_LSQ && o->break_kind == ORC_BREAK_SYSTEM && (int32_t)it == o->break_it)
      retries = ORC_E_NOT_PD; /* test hook: the LSQ system has no factor */
    free(rhs);
  }
  if (status == ORC_OK && retries < 0) status = ORC_E_NOT_PD;
  if (status == ORC_OK && mppi_step) memcpy(delta, mppi, sizeof(double) * (size_t)n); /* Eq. 5 step */

  /* 6. line search over {gamma^j}; alpha_{j+1} = alpha_j * gamma (MPPI: alpha = 1 only) */
  const int nl = Lc + (mono ? 1 : 0);
  double* Cl = (double*)malloc(sizeof(double) * (size_t)nl);
  int jstar = -1;
  double alpha_star = 0.0, C_new = C_nom;
  if (status == ORC_OK) {
    double* Ut = (double*)malloc(sizeof(double) * (size_t)n);
    double alpha = 1.0;
    for (int j = 0; j < Lc; ++j) {
      for (int i = 0; i < n; ++i) Ut[i] = U[i] + alpha * delta[i];
      Cl[j] = orc_cost(m, x0, xref, Ut);
      alpha *= o->gamma;
    }
    if (mono) Cl[Lc] = C_nom;
    double best = INFINITY;
    alpha = 1.0;
    for (int j = 0; j < nl; ++j) {
      const double aj = (j < Lc) ? alpha : 0.0;
      if (Cl[j] < best) { /* strict: ties keep the smaller j */
        best = Cl[j];
        jstar = j;
        alpha_star = aj;
      }
      if (j < Lc) alpha *= o->gamma;
    }
    if (jstar < 0) { /* every candidate non-finite */
      status = ORC_E_NONFINITE;
      alpha_star = 0.0;
    } else {
      C_new = best;
    }
    /* 7. update */
    for (int i = 0; i < n; ++i) U[i] = U[i] + alpha_star * delta[i];
    free(Ut);
  }

  if (rec) {
    double gn = 0.0, dn = 0.0;
    for (int j = 0; j < n; ++j) {
      gn += g[j] * g[j];
      dn += delta[j] * delta[j];
    }
    rec->C_nom = C_nom;
    rec->C_new = C_new;
    rec->alpha = alpha_star;
    rec->lambda_used = lambda_used;
    rec->c_min = st4[0];
    rec->sum_w = st4[1];
    rec->sum_w2 = st4[2];
    rec->ess = st4[3];
    rec->grad_norm = sqrt(gn);
    rec->step_norm = sqrt(dn);
    rec->j_star = jstar;
    rec->n_masked = n_masked;
    rec->jac_mode_used = jm;
    rec->status = status;
    rec->chol_retries = retries < 0 ? 7 : retries;
    if (rec->delta) memcpy(rec->delta, delta, sizeof(double) * (size_t)n);
    if (rec->C_line) memcpy(rec->C_line, Cl, sizeof(double) * (size_t)nl);
    if (rec->C_samp) memcpy(rec->C_samp, Cs, sizeof(double) * (size_t)nsamp);
    if (rec->J) memcpy(rec->J, J, sizeof(double) * (size_t)nR * n);
    if (rec->dR) memcpy(rec->dR, dR, sizeof(double) * (size_t)Kp * nR);
    if (rec->W) memcpy(rec->W, W, sizeof(double) * (size_t)Kp * n);
    if (rec->r) memcpy(rec->r, r, sizeof(double) * (size_t)nR);
  }
  free(Cl);
  free(r);
  free(W);
  free(dR);
  free(Cs);
  free(valid);
  free(P);
  free(S);
  free(J);
  free(G);
  free(g);
  free(delta);
  free(wts);
  free(mppi);
  return status;
}

/* Algorithm 1: `iterations` GN-MPPI iterations from U (in: U_0, out: U_K),
 * with Sigma_{k+1} = beta Sigma_k, i.e. s <- sqrt(beta) s.  recs, U_hist
 * ((iterations+1)*n) and C_hist (iterations+1) are optional. */
int32_t orc_solve(const orc_model* m, const orc_options* o, const double* x0, const double* xref, double* U,
                  const double* s0, uint32_t inst, orc_record* recs, double* U_hist, double* C_hist) {
  const int n = orc_n(m);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(s, s0, sizeof(double) * (size_t)n);
  const double sb = sqrt(o->beta);
  int32_t st = ORC_OK;
  if (U_hist) memcpy(U_hist, U, sizeof(double) * (size_t)n);
  if (C_hist) C_hist[0] = orc_cost(m, x0, xref, U);
  /* once the LSQ form breaks down (orc_iteration fell back to SIGMA), the
   * rest of the solve uses SIGMA: K' and n, which cause it, do not change */
  orc_options oo = *o;
  const int Kp = o->sampling == ORC_SAMPLE_SIGMA ? n : (o->antithetic ? o->K / 2 : o->K);
  const int lsq_chosen = o->method == ORC_METHOD_GN &&
                         (o->jac_mode == ORC_JAC_LSQ || (o->jac_mode == ORC_JAC_AUTO && Kp >= n));
  for (int it = 0; it < o->iterations; ++it) {
    orc_record local;
    memset(&local, 0, sizeof(local));
    orc_record* rec = recs ? &recs[it] : &local;
    st = orc_iteration(m, &oo, x0, xref, U, s, inst, (uint32_t)it, rec);
    if (lsq_chosen && rec->jac_mode_used == ORC_JAC_SIGMA) oo.jac_mode = ORC_JAC_SIGMA;
    if (U_hist) memcpy(U_hist + (size_t)(it + 1) * n, U, sizeof(double) * (size_t)n);
    if (C_hist) C_hist[it + 1] = rec->C_new;
    if (st != ORC_OK) break;
    for (int j = 0; j < n; ++j) s[j] *= sb;
  }
  free(s);
  return st;
}

/* Method A of Sec. 5: GGN with a central finite-difference Jacobian,
 * used here only to polish the reference optimum C*.  Step h_j = eps *
 * max(1, |U_j|); the step-length set is {2^-j, j < 30} plus 0, so the cost
 * never increases; stops when alpha = 0 wins, or ||J^T r|| < gtol. */
int32_t orc_method_a(const orc_model* m, const double* x0, const double* xref, double* U, int32_t max_iter,
                     double eps, double lambda, double gtol, double* C_out, int32_t* iters_out) {
  const int n = orc_n(m), nR = orc_nR(m);
  double* r = (double*)malloc(sizeof(double) * (size_t)nR);
  double* Rp = (double*)malloc(sizeof(double) * (size_t)nR);
  double* Rm = (double*)malloc(sizeof(double) * (size_t)nR);
  double* J = (double*)malloc(sizeof(double) * (size_t)nR * n);
  double* G = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* Ut = (double*)malloc(sizeof(double) * (size_t)n);
  int it = 0;
  int32_t st = ORC_OK;
  double C = orc_cost(m, x0, xref, U);
  for (; it < max_iter; ++it) {
    orc_residual(m, x0, xref, U, r);
    for (int j = 0; j < n; ++j) {
      const double h = eps * (fabs(U[j]) > 1.0 ? fabs(U[j]) : 1.0);
      memcpy(Ut, U, sizeof(double) * (size_t)n);
      Ut[j] = U[j] + h;
      orc_residual(m, x0, xref, Ut, Rp);
      Ut[j] = U[j] - h;
      orc_residual(m, x0, xref, Ut, Rm);
      for (int i = 0; i < nR; ++i) J[(size_t)i * n + j] = (Rp[i] - Rm[i]) / (2.0 * h);
    }
    double gn = 0.0;
    for (int a = 0; a < n; ++a) {
      for (int b = 0; b < n; ++b) {
        double acc = 0.0;
        for (int i = 0; i < nR; ++i) acc += J[(size_t)i * n + a] * J[(size_t)i * n + b];
        G[a * n + b] = acc;
      }
      double acc = 0.0;
      for (int i = 0; i < nR; ++i) acc += J[(size_t)i * n + a] * r[i];
      rhs[a] = -acc;
      gn += acc * acc;
    }
    if (sqrt(gn) < gtol) break;
    double lu;
    if (damped_solve(n, G, lambda, rhs, 2, d, &lu) < 0) {
      st = ORC_E_NOT_PD;
      break;
    }
    double best = C, alpha = 1.0, abest = 0.0;
    for (int j = 0; j < 30; ++j) {
      for (int i = 0; i < n; ++i) Ut[i] = U[i] + alpha * d[i];
      const double c = orc_cost(m, x0, xref, Ut);
      if (c < best) {
        best = c;
        abest = alpha;
      }
      alpha *= 0.5;
    }
    if (abest == 0.0) break;
    for (int i = 0; i < n; ++i) U[i] = U[i] + abest * d[i];
    C = best;
  }
  if (C_out) *C_out = C;
  if (iters_out) *iters_out = it;
  free(r);
  free(Rp);
  free(Rm);
  free(J);
  free(G);
  free(rhs);
  free(d);
  free(Ut);
  return st;
}
