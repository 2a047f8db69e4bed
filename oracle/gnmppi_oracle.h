/*
 * gnmppi_oracle.h -- plain FP64 CPU oracle for Gauss-Newton accelerated MPPI.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library
 * against the method as the paper defines it.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never does.  It shares no code, header, table or helper with the CUDA
 * library: its Philox generator, Box-Muller transform, dynamics, residuals,
 * Jacobian estimator, Cholesky factorisation and line search are written
 * here, from their published definitions, a second time.
 *
 * Notation (paper -> this file):  samples M -> K (antithetic pairs K' = K/2),
 * iterations -> iterations, MPPI temperature lambda_k -> tau, step-length set
 * size -> L, horizon N, control dim nu, state dim nx, n = N*nu, residual
 * dimension nR, Levenberg damping of the GGN system -> lambda.
 */
#ifndef GNMPPI_ORACLE_H
#define GNMPPI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_DYN_PENDULUM = 0,   /* pendulum swing-up, RK4 */
  ORC_DYN_CHAIN = 1,      /* planar chain of point masses, RK4 */
  ORC_DYN_LINEAR = 2,     /* discrete x+ = A x + B u, quadratic residual */
  ORC_DYN_ROSENBROCK = 3, /* Problem I  (Sec. 5) */
  ORC_DYN_RASTRIGIN = 4,  /* Problem II (Sec. 5) */
  ORC_DYN_HEAVISIDE = 5,  /* Problem III (Sec. 5) */
  ORC_DYN_LINCONT = 6     /* continuous x' = A x + B u under RK4 (pin only) */
};

enum { ORC_JAC_LSQ = 0, ORC_JAC_SIGMA = 1, ORC_JAC_AUTO = 2 };
/* perturbations: random Philox normals (Method D) or the symmetric sigma
 * points +-sqrt(n) s_i e_i of a Dirac mixture (Method E, Sec. 5) */
enum { ORC_SAMPLE_RANDOM = 0, ORC_SAMPLE_SIGMA = 1 };
/* step: Gauss-Newton (Algorithm 1) or the deterministic MPPI step of Eq. 3/5
 * (Method C, Sec. 3) */
enum { ORC_METHOD_GN = 0, ORC_METHOD_MPPI = 1 };

enum {
  ORC_OK = 0,
  ORC_E_ARG = -1,
  ORC_E_NOT_PD = -3,
  ORC_E_NONFINITE = -4
};

/* Problem definition.  `lin` points at the linear model's data
 * (A nx*nx, B nx*nu row-major, then wq nx, wr nu, wqN nx); NULL otherwise.
 * params: pendulum {g, l, m, b}; chain {mass, k, k3, damping, gravity}. */
typedef struct {
  int32_t dyn, nx, nu, N, M, pad0;
  double dt;
  double params[8];
  const double* lin;
} orc_model;

typedef struct {
  int32_t K;          /* samples per iteration (antithetic: K/2 pairs)      */
  int32_t iterations; /* Algorithm 1 outer iterations                       */
  int32_t L;          /* number of step lengths gamma^j, j < L              */
  int32_t jac_mode;   /* ORC_JAC_*                                          */
  int32_t antithetic; /* 1: pairs +W,-W; 0: one-sided with baseline         */
  int32_t monotone;   /* 1: alpha = 0 joins the step-length set             */
  int32_t threads;    /* OpenMP threads for the sample rollouts             */
  int32_t ir_steps;   /* iterative-refinement steps after the Cholesky solve*/
  double lambda;      /* damping of (J^T J + lambda I)                      */
  double beta;        /* covariance shrink Sigma <- beta Sigma              */
  double gamma;       /* step-length ratio                                  */
  double tau;         /* softmin temperature                                */
  uint64_t seed;
  int32_t sampling;   /* ORC_SAMPLE_*; sigma points need antithetic, K = 2n */
  int32_t method;     /* ORC_METHOD_*                                       */
  /* Test hook (off when break_kind is 0): at iteration break_it the LSQ
   * form is made to break down as if S had no Cholesky factor (kind 1) or
   * the damped LSQ system had none at any damping (kind 2), so that the
   * tests can pin the fallback to the printed form on any input. */
  int32_t break_it, break_kind;
} orc_options;

enum { ORC_BREAK_NONE = 0, ORC_BREAK_S = 1, ORC_BREAK_SYSTEM = 2 };

/* One Algorithm-1 iteration's outputs.  Array pointers are optional. */
typedef struct {
  double C_nom, C_new, alpha, lambda_used;
  double c_min, sum_w, sum_w2, ess;
  double grad_norm, step_norm;
  int32_t j_star, n_masked, jac_mode_used, status, chol_retries, pad;
  double* delta;    /* n   : GGN step                                      */
  double* C_line;   /* L(+1 if monotone): line-search costs                */
  double* mppi_dir; /* n   : softmin-weighted mean perturbation (Eq. 3)    */
  double* C_samp;   /* K   : sample costs (antithetic: C+ then C- per pair)*/
  double* J;        /* nR*n: Jacobian estimate, row-major                  */
  double* dR;       /* K'*nR: residual differences per pair/sample         */
  double* W;        /* K'*n : perturbations per pair/sample                */
  double* r;        /* nR  : nominal residual R(U_k)                       */
} orc_record;

int32_t orc_nR(const orc_model* m);
int32_t orc_n(const orc_model* m);

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform53(uint32_t hi, uint32_t lo);
/* z[0..n) for (seed, instance, iteration, sample) -- the noise stream. */
void orc_normals(uint64_t seed, uint32_t inst, uint32_t it, uint32_t m, int32_t n, double* z);

void orc_deriv(const orc_model* m, const double* x, const double* u, double* xdot);
void orc_rk4_step(const orc_model* m, const double* x, const double* u, double* xn);
int32_t orc_rollout(const orc_model* m, const double* x0, const double* U, double* X);
int32_t orc_residual(const orc_model* m, const double* x0, const double* xref, const double* U, double* R);
double orc_cost(const orc_model* m, const double* x0, const double* xref, const double* U);

int32_t orc_softmin(int32_t count, const double* C, const uint8_t* valid, double tau, double* w, double* stats);
int32_t orc_cholesky(int32_t n, double* A);
void orc_chol_solve(int32_t n, const double* Lf, double* b);

int32_t orc_iteration(const orc_model* m, const orc_options* o, const double* x0, const double* xref,
                      double* U, const double* s, uint32_t inst, uint32_t it, orc_record* rec);
int32_t orc_solve(const orc_model* m, const orc_options* o, const double* x0, const double* xref, double* U,
                  const double* s0, uint32_t inst, orc_record* recs, double* U_hist, double* C_hist);
int32_t orc_method_a(const orc_model* m, const double* x0, const double* xref, double* U, int32_t max_iter,
                     double eps, double lambda, double gtol, double* C_out, int32_t* iters_out);

#ifdef __cplusplus
}
#endif
#endif
