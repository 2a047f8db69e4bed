/*
 * gnmppi.h -- C ABI of the GB300 (sm_103a) Gauss-Newton accelerated MPPI solver.
 *
 * The solver implements Algorithm 1 of Homburger, Baumgaertner, Diehl, Reuter,
 * "Gauss-Newton accelerated MPPI Control" (arXiv 2512.04579), Method D (random
 * sampling of the Gaussian-smoothing Jacobian, Eq. 7), batched over many
 * independent optimal control problems (Eq. 2-3) on one GPU.  Per iteration:
 * Philox noise, antithetic RK4 rollouts with fused residual / cost / softmin
 * reductions, the Jacobian-reconstruction contraction, the GGN system of Eq. 9
 * with a Levenberg damping lambda, an FP64 Cholesky solve with iterative
 * refinement, the parallel line search of Eq. 11 and the covariance shrink.
 *
 * Conventions for every entry point:
 *   - Arrays are plain pointers.  `mem` says whether they are host
 *     (GNMPPI_MEM_HOST) or device (GNMPPI_MEM_DEVICE) memory; the caller
 *     owns them and keeps them valid until the call returns (calls are
 *     synchronous with respect to the handle's stream).
 *   - Per-instance arrays are packed instance after instance; the offset of
 *     instance b is given by gnmppi_layout().  Element type is double.
 *   - No exception crosses the ABI.  Each call returns a gnmppi_status; the
 *     text of the last error of a handle is available from
 *     gnmppi_last_error().  A handle is used from one host thread at a time.
 *   - All device work is issued on the handle's stream (the one passed to
 *     gnmppi_create, or a stream the handle creates when NULL).
 */
#ifndef GNMPPI_H
#define GNMPPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gnmppi_s* gnmppi_t;

typedef enum {
  GNMPPI_OK = 0,
  GNMPPI_E_ARG = -1,       /* invalid argument (null pointer, size, mode)         */
  GNMPPI_E_CUDA = -2,      /* CUDA runtime error, or no usable GPU                */
  GNMPPI_E_NOT_PD = -3,    /* GGN matrix not positive definite after 6 retries   */
  GNMPPI_E_NONFINITE = -4, /* every sample or every line-search cost non-finite  */
  GNMPPI_E_TIMEOUT = -5,   /* a bounded device wait ran out                      */
  GNMPPI_E_NOMEM = -6      /* device allocation failed                           */
} gnmppi_status;

/* Dynamics (Sec. 2: the black-box simulator X = F(x0, U) and residual R). */
enum {
  GNMPPI_DYN_PENDULUM = 0, /* x=[theta,omega]; theta''=-(g/l)sin(theta)-b*omega+u/(m l^2); RK4.
                              Residual stage k: [theta_k-pi, 0.1 omega_k, 0.1 u_k];
                              terminal [10(theta_N-pi), 10 omega_N].  params {g,l,m,b,u_f}:
                              u_f > 0 adds dead-zone friction at the input (Setting
                              V.ii): u_apply = 0 where |u| <= u_f; the residual keeps u. */
  GNMPPI_DYN_CHAIN = 1,    /* M point masses in a vertical plane, mass 0 fixed at the origin,
                              link tension k d + k3 d^3 (rest length 1/(M-1)), damping -c v,
                              gravity -g y, force control on mass M-1; RK4.  Residual stage k:
                              [p_{1..M-1,k} - p*, 0.1 u_k]; terminal p_{.,N} - p*.
                              xref = p* (2(M-1) values).  params {mass,k,k3,c,g,u_f}
                              (u_f: dead-zone friction per force component, as above). */
  GNMPPI_DYN_LINEAR = 2,   /* x+ = A x + B u (discrete); residual stage k [wq.*x_k, wr.*u_k],
                              terminal wqN.*x_N.  lin = {A (nx*nx), B (nx*nu), wq, wr, wqN}. */
  /* The static test problems of Sec. 5: N = 1, R depends on U alone; x0 is one
     ignored value per instance, xref unused, dt unused. */
  GNMPPI_DYN_ROSENBROCK = 3, /* Problem I, nu = 2: [sqrt2 (1 - u1), sqrt200 (u2 - u1^2)]   */
  GNMPPI_DYN_RASTRIGIN = 4,  /* Problem II, nu = 2: sqrt2 [u1, u2, sqrt(5 - 5cos 2pi u1),
                                sqrt(5 - 5cos 2pi u2)] (the paper's R, scaled for 0.5||R||^2) */
  GNMPPI_DYN_HEAVISIDE = 5   /* Problem III, nu = 1: [H(u)], H(u) = 1 for u >= 0 else 0     */
};

/* Arithmetic of the hot path. */
enum {
  GNMPPI_PREC_FP64 = 0, /* every step in FP64 (parity mode)                               */
  GNMPPI_PREC_FP32 = 1, /* FP32 rollouts with compensated cost sums; contraction and Gram
                           on the tensor cores from three TF32 passes over FP32 operands
                           split into head and remainder (FP32-level accuracy, FP32
                           accumulation; the Gram's sum over the residual rows in chunks
                           of 2048, added in FP64); FP64 Cholesky with iterative
                           refinement.  An
                           LSQ system that does not factor is retried with 1e-5, 1e-4,
                           1e-3 of diag(P^T P) added before lambda grows (the Gram's
                           rounding can leave it indefinite when K' is close to n)       */
  GNMPPI_PREC_BF16 = 2  /* as FP32, but the contraction's and the Gram's FP32 operands are
                           split into a BF16 head and a BF16 remainder (in shared memory;
                           the contraction's W rows once by the rollouts, which keep a split
                           copy of W) and multiplied by three BF16 passes (head x head + head
                           x remainder + remainder x head, FP32 accumulation; 16 significant
                           bits per operand)                                               */
};

/* Jacobian estimator (Eq. 7).  dR_m = (R(U+W_m) - R(U-W_m))/2 (antithetic) or
 * R(U+W_m) - R(U) (one-sided); P = sum dR_m W_m^T, S = sum W_m W_m^T over K' pairs.
 *   SIGMA: J = P Sigma^-1 / K'  (the printed Monte Carlo form)
 *   LSQ:   J = P S^-1           (regression form; exact for affine R once K' >= n)
 *   AUTO:  LSQ when K' >= n, otherwise SIGMA. */
enum { GNMPPI_JAC_LSQ = 0, GNMPPI_JAC_SIGMA = 1, GNMPPI_JAC_AUTO = 2 };

enum { GNMPPI_MEM_HOST = 0, GNMPPI_MEM_DEVICE = 1 };

/* Perturbations of the Jacobian estimate (Eq. 7, Sec. 5).
 *   RANDOM: W_m = s .* z_m, z_m from Philox4x32-10 + Box-Muller (Method D).
 *   SIGMA:  the symmetric sigma points of a Dirac mixture, W_m = sqrt(n) s_m e_m
 *           for m < n (K' = n antithetic pairs, K ignored; antithetic required)
 *           (Method E).  J is then central differences with step sqrt(n) s_m. */
enum { GNMPPI_SAMPLE_RANDOM = 0, GNMPPI_SAMPLE_SIGMA = 1 };

/* Step of an iteration.
 *   GN:   Algorithm 1, the damped GGN step with a line search (Eq. 9-11).
 *   MPPI: the deterministic MPPI step of Eq. 3, estimated by Eq. 5 over the
 *         same samples and taken whole (alpha = 1, no line search, no
 *         contraction or Cholesky) (Method C, Sec. 3). */
enum { GNMPPI_METHOD_GN = 0, GNMPPI_METHOD_MPPI = 1 };

/* Problem and Algorithm-1 options shared by every instance of a handle. */
typedef struct {
  int32_t dynamics;   /* GNMPPI_DYN_*                                              */
  int32_t nx, nu, N;  /* state dim, control dim, horizon (defaults per instance)   */
  int32_t M;          /* chain masses (chain only)                                 */
  int32_t n_lin;      /* number of doubles in lin (linear only)                    */
  double dt;          /* RK4 step                                                  */
  double params[8];   /* model constants, see GNMPPI_DYN_*                         */
  const double* lin;  /* host pointer, copied by gnmppi_create; may be NULL        */
  int32_t K;          /* samples per iteration; antithetic: K/2 pairs              */
  int32_t iterations; /* Algorithm 1 iterations per gnmppi_solve                   */
  int32_t L;          /* line-search set {gamma^j : j < L} (Eq. 11)                */
  int32_t precision;  /* GNMPPI_PREC_*                                             */
  int32_t jac_mode;   /* GNMPPI_JAC_*                                              */
  int32_t antithetic; /* 1: +-W pairs (default); 0: one-sided, baseline-subtracted */
  int32_t monotone;   /* 1: alpha = 0 joins the line-search set                    */
  int32_t ir_steps;   /* iterative-refinement steps after the Cholesky solve       */
  double lambda;      /* damping of (J^T J + lambda I) (Eq. 9)                     */
  double sigma0;      /* initial sampling std, Sigma_0 = sigma0^2 I                */
  double beta;        /* covariance shrink Sigma <- beta Sigma (Algorithm 1)       */
  double gamma;       /* step-length ratio in (0, 1)                               */
  double tau;         /* softmin temperature of the sample weights (Eq. 5)         */
  uint64_t seed;      /* Philox key of the noise stream                            */
  int32_t sampling;   /* GNMPPI_SAMPLE_* (0: random, Method D)                     */
  int32_t method;     /* GNMPPI_METHOD_* (0: Gauss-Newton, Algorithm 1)            */
  int32_t first_instance; /* noise stream of instance b is that of instance
                             first_instance + b (>= 0; 0: its position), so a batch
                             split into contiguous ranges over several handles or
                             GPUs, each given its range's first index, draws exactly
                             the noise of the unsplit batch                       */
  int32_t pad0;
} gnmppi_problem;

/* Per-instance shape of an uneven batch; fields <= 0 take the problem's value. */
typedef struct {
  int32_t N, M, K, pad;
} gnmppi_instance_shape;

/* Per-instance result of gnmppi_solve. */
typedef struct {
  double C_initial;  /* C(U_0)                                        */
  double C_prev;     /* C(U_{T-1}), the cost before the last iteration */
  double C_final;    /* C(U_T) from the last line search              */
  double sigma_final;/* sampling std scale after the last shrink      */
  int32_t iterations;/* iterations run                                */
  int32_t status;    /* gnmppi_status of this instance                */
  int32_t n_masked;  /* non-finite sample pairs dropped, all iterations*/
  int32_t chol_retries; /* damping increases, all iterations          */
} gnmppi_report;

/* Per-instance outputs of one Algorithm-1 iteration (gnmppi_step). */
typedef struct {
  double C_nom;      /* C(U_k)                                          */
  double C_new;      /* C(U_k + alpha* delta)                           */
  double alpha;      /* selected step length                            */
  double lambda_used;/* damping after retries                           */
  double c_min, sum_w, sum_w2, ess; /* softmin statistics (Eq. 5)       */
  double pr_norm;    /* ||P^T r|| (gradient up to the metric S^-1)       */
  double step_norm;  /* ||delta||                                       */
  int32_t j_star;    /* index of alpha* in the step-length set          */
  int32_t n_masked;  /* non-finite sample pairs dropped                 */
  int32_t jac_mode_used;
  int32_t status;
  int32_t chol_retries;
  int32_t pad;
} gnmppi_iter_report;

/* Create a solver for `batch` instances (batch >= 1).  `shapes` (nullable, host,
 * batch entries) gives per-instance N, M, K for an uneven batch.  `cuda_stream`
 * is a cudaStream_t or NULL.  Allocates all device workspace; *out receives the
 * handle (NULL on failure).  Errors: E_ARG (bad sizes, modes, K odd with
 * antithetic sampling, chain M outside 2..65, one-sided sampling with M > 17), E_CUDA (no
 * GPU), E_NOMEM.  Chains of up to 17 masses roll out one thread per sample; longer
 * chains (up to 65 masses) use a group of 4 or 8 lanes per sample. */
gnmppi_status gnmppi_create(const gnmppi_problem* p, int32_t batch, const gnmppi_instance_shape* shapes,
                            void* cuda_stream, gnmppi_t* out);

/* Packed-array offsets (host arrays of batch+1 int64 each, nullable): x0 (nx per
 * instance), xref (2(M-1) per chain instance, 1 otherwise), U (N*nu per instance). */
gnmppi_status gnmppi_layout(gnmppi_t h, int64_t* x0_off, int64_t* xref_off, int64_t* U_off);

/* Algorithm 1: problem->iterations iterations from U_0 for every instance.
 * x0, xref: inputs; U: in U_0, out U_T; sigma (nullable): per-instance,
 * per-component initial std packed like U (NULL: problem->sigma0).  rep
 * (nullable, host, batch entries) receives per-instance reports.  Returns the
 * worst instance status (E_NOT_PD / E_NONFINITE), or OK. */
gnmppi_status gnmppi_solve(gnmppi_t h, int32_t mem, const double* x0, const double* xref, double* U,
                           const double* sigma, gnmppi_report* rep);

/* gnmppi_solve restricted to the instances with active[b] != 0 (host array
 * of batch int32, nullable = all): the others are skipped by every kernel,
 * keep their U unchanged and report status OK with 0 iterations. */
gnmppi_status gnmppi_solve_masked(gnmppi_t h, int32_t mem, const double* x0, const double* xref, double* U,
                                  const double* sigma, const int32_t* active, gnmppi_report* rep);

/* gnmppi_solve_masked in two halves, so that the host (or another handle on
 * another stream) works while this handle's solve runs.  gnmppi_solve_async
 * enqueues the input copies, the solve's CUDA graph and the copy of U back on
 * the handle's stream and returns; U must stay valid until the matching
 * gnmppi_solve_wait.  With mem = HOST and pageable U the copy back blocks until
 * it is done (pinned U keeps the call asynchronous).  gnmppi_solve_wait blocks
 * until that solve has finished and fills rep like gnmppi_solve.  One solve in
 * flight per handle.  Errors: E_ARG for a second async call before the wait,
 * or a wait with nothing in flight; otherwise as gnmppi_solve. */
gnmppi_status gnmppi_solve_async(gnmppi_t h, int32_t mem, const double* x0, const double* xref, double* U,
                                 const double* sigma, const int32_t* active);
gnmppi_status gnmppi_solve_wait(gnmppi_t h, gnmppi_report* rep);

/* One Algorithm-1 iteration with index `iteration` (it selects the Philox
 * stream) at the given U (in/out: U_k -> U_{k+1}) and per-component std sigma
 * (packed like U, not modified).  rep (nullable, host, batch entries). */
gnmppi_status gnmppi_step(gnmppi_t h, int32_t mem, const double* x0, const double* xref, double* U,
                          const double* sigma, int32_t iteration, gnmppi_iter_report* rep);

/* FP64 re-evaluation of C(U) = 0.5 ||R(U)||^2 (Eq. 2, 4) for every instance;
 * C: batch doubles in `mem` memory. */
gnmppi_status gnmppi_cost(gnmppi_t h, int32_t mem, const double* x0, const double* xref, const double* U,
                          double* C);

/* Copy an internal buffer of instance `inst` from the last gnmppi_step or
 * gnmppi_solve iteration to host memory as doubles, for verification.
 * what: 0 dR [nR][K'], 1 W [n][K'], 2 sample costs [K'][2] (one-sided: [K]), 3 e = dR r [K'],
 * 4 [P^T | S] [n][nR+n], 5 A = P^T P [n][n], 6 g = P^T r [n], 7 delta [n],
 * 8 line-search costs [L(+1)], 9 nominal residual r [nR], 10 MPPI direction [n],
 * 11 S2 = S S^T [n][n] (formed for instances in LSQ mode only).
 * count: capacity of host_out in doubles; the number written is returned in
 * *written.  Errors: E_ARG for unknown `what` or too small a buffer. */
gnmppi_status gnmppi_debug_read(gnmppi_t h, int32_t what, int32_t inst, double* host_out, int64_t count,
                                int64_t* written);

/* Time the kernels of one Algorithm-1 iteration (index `iteration`) on the
 * handle's current device state -- the state the last gnmppi_solve or
 * gnmppi_step left -- with CUDA events on the handle's stream between phases.
 * The iteration runs for real (it updates the device iterate; no covariance
 * shrink).  ms (host, cap doubles) receives per-phase milliseconds in the
 * order of gnmppi_phase_name(); *nphase the number of phases.  Errors: E_ARG
 * if cap is smaller than the number of phases. */
gnmppi_status gnmppi_phase_times(gnmppi_t h, int32_t iteration, double* ms, int32_t cap, int32_t* nphase);

/* Name of phase i of gnmppi_phase_times ("samples", "softmin", "contract",
 * "gram", "s2", "solve", "line", "update"), or NULL.  With the tensor-core
 * path S2 is formed inside the "gram" phase and "s2" stays empty. */
const char* gnmppi_phase_name(int32_t i);

/* Autotuner of the batched launch (the paper has no counterpart: it concerns
 * how Algorithm 1 is scheduled over many instances, not what it computes).
 * Times, on this handle's instances and the caller's inputs (same arguments
 * and memory kinds as gnmppi_solve; U and sigma are read only), the candidate
 * launch configurations and keeps the fastest:
 *   - branches: how many concurrent CUDA-graph branches carry the per-size
 *     rollout groups (sample rollouts and line search), 1, 2, 4 or 8;
 *   - solve_nt: threads per Cholesky CTA, 512 (one per SM), 256 (two) or 128
 *     (four); without tuning 512 when the batch fits one instance per SM, else 256.
 * reps: timed repetitions per candidate (<= 0: 3), after one warm-up.  The
 * choice is cached for the process under a signature of the device, the
 * model, the precision and the multiset of instance shapes; when the
 * environment variable GNMPPI_TUNE_FILE names a file, cached choices are read
 * from it and new ones appended ("signature branches solve_nt" lines).  A
 * cached choice is applied without timing.  The iterates do not depend on the
 * configuration (the arithmetic of every kernel is unchanged); only the
 * reported norms |b| and |delta|, block-wide sums, may round differently.  The next
 * gnmppi_solve recaptures its CUDA graph.  Errors: as gnmppi_solve. */
gnmppi_status gnmppi_autotune(gnmppi_t h, int32_t mem, const double* x0, const double* xref, const double* U,
                              const double* sigma, int32_t reps);

/* Set the launch configuration by hand: branches 1..8; solve_nt 128, 256 or
 * 512; contract_mt the BF16-mode contraction tile, 2 (256 [dR; W] rows per
 * CTA, one CTA per SM), 1 (128 rows, two CTAs per SM) or 0 (unchanged).
 * None of them changes a result bit.  Errors: E_ARG for values out of range. */
gnmppi_status gnmppi_tune_set(gnmppi_t h, int32_t branches, int32_t solve_nt, int32_t contract_mt);

/* The handle's launch configuration as a JSON object (source "default",
 * "set", "cache" or "timed"; the timed candidates when tuned), NUL-terminated
 * into buf (host, cap bytes).  Errors: E_ARG if cap is too small. */
gnmppi_status gnmppi_tune_report(gnmppi_t h, char* buf, int32_t cap);

/* Failure injection for tests (the paper has no counterpart: it exercises the
 * library's handling of failures that Eq. 9's assumption B_GGN > 0 and the
 * bounded device waits leave open, without faulting the GPU).  At Algorithm-1
 * iteration `iteration` of every later gnmppi_step / gnmppi_solve on h:
 *   kind 1: every LSQ system's Cholesky factorisation is treated as failed at
 *           all dampings, so the iteration takes the printed form J = P Sigma^-1 / K'
 *           (jac_mode_used 1) and the rest of the solve stays in it;
 *   kind 2: every system of the iteration fails (the damping retries run out),
 *           so the instances end with status GNMPPI_E_NOT_PD;
 *   kind 3: in the tensor-core contraction every CTA first waits on a barrier
 *           that nothing completes; the wait gives up after 20 ms, the kernel
 *           winds down and the call returns GNMPPI_E_TIMEOUT (FP32 and BF16
 *           modes only);
 *   kind 0: off.
 * The arithmetic of every kernel is otherwise unchanged; the next solve
 * recaptures its CUDA graph.  Errors: E_ARG for an unknown kind, or kind 3
 * on an FP64 handle. */
gnmppi_status gnmppi_debug_inject(gnmppi_t h, int32_t kind, int32_t iteration);

/* Softmin weights exp(-(C - min C)/tau) and the weighted mean perturbation
 * sum w_i W_i / sum w_i of one sample set, computed without any device
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory when they call in -- a real-time
 * controller whose per-cycle latency budget has no room for cudaMalloc /
 * cudaFree (unbounded latency; cudaFree synchronises the device), or a host
 * that grants the library a fixed memory budget up front and forbids later
 * allocation.
 *   C      device, count doubles (one-sided) or 2*count doubles (antithetic:
 *          C[2m] = C(U + W_m), C[2m+1] = C(U - W_m)); non-finite pairs get
 *          weight 0.
 *   W      device, [n][count] doubles, sample-contiguous rows of exactly
 *          count entries with no padding (the layout of gnmppi_debug_read
 *          buffer 1; a solver handle's internal W, whose rows are padded and
 *          stored in the handle's precision, is not this layout).
 *   mppi   device, n doubles out; stats device, 4 doubles out:
 *          {min C, sum w, sum w^2, effective sample size}.
 *   cuda_stream  cudaStream_t or NULL; the call is asynchronous on it.
 *   err    optional host buffer of err_len bytes for the error text.
 * Scratch: one double per sample pair in a fixed device array of 65536
 * entries (512 KB) that every GPU loading the library holds until exit; count
 * above 65536 is rejected with E_ARG.  The first call on a device is a set-up
 * call: it looks up that array's device address (cudaGetSymbolAddress) with
 * the device current, and under lazy module loading (the CUDA default) that
 * lookup also loads the library's device code onto the device, which the
 * driver allocates for; make that first call before any stream capture and
 * outside the allocation-free phase (a warm-up call).  The address is kept
 * for the life of the process, so resetting the device (cudaDeviceReset)
 * after the first call is not supported.  Every call on a device shares the
 * array, so calls that overlap on the GPU race: serialise them (one stream,
 * or synchronise between calls).  No cudaMalloc, cudaFree or other
 * allocating routine is called. */
gnmppi_status gnmppi_softmin_noalloc(const double* C, const double* W, int32_t count, int32_t n,
                                     int32_t antithetic, double tau, double* mppi, double* stats,
                                     void* cuda_stream, char* err, int32_t err_len);

/* ---------------------------------------------------------------------------
 * Learned warm start.  A multilayer perceptron maps an initial state x0 to a
 * nominal control sequence mu (U_0 of Algorithm 1) and one log sampling scale
 * s_k per control step (Sigma_0 = diag(exp(2 s_k))).  The paper cites learned
 * sampling distributions as prior art (Sec. 1); the network is trained on
 * solutions of plain GN-MPPI by minimising the Gaussian negative
 * log-likelihood  (1/B) sum_b sum_j [ (t_j - mu_j)^2 exp(-2 s_{j/nu}) / 2 + s_{j/nu} ]
 * with Adam (Kingma & Ba, 2015).  Architecture: h_0 = (x0 - x_mean) / x_std,
 * hidden layers h_l = GELU(W_l h_{l-1} + b_l), linear output y = W_L h + b_L,
 * mu = y[0 : n_mu], s = y[n_mu : n_mu + n_mu/nu].  Parameters are flat, per
 * layer W_l [d_l][d_{l-1}] row-major then b_l [d_l].  Arrays are doubles in
 * `mem` memory; B <= max_batch.
 * ------------------------------------------------------------------------- */
typedef struct gnmppi_mlp_s* gnmppi_mlp_t;

/* dims: nlayers + 1 widths (input ... output); the output width must be
 * n_mu + n_mu/nu.  weights_bf16: forward and input-gradient products use
 * BF16-rounded weights (FP32 master weights, FP32 accumulation).  Parameters
 * start at zero; set them with gnmppi_mlp_set_params.  E_ARG on bad sizes,
 * E_CUDA without a GPU. */
gnmppi_status gnmppi_mlp_create(int32_t nlayers, const int32_t* dims, int32_t nu, int32_t weights_bf16,
                                int32_t max_batch, void* cuda_stream, gnmppi_mlp_t* out);
int64_t gnmppi_mlp_num_params(gnmppi_mlp_t m);
/* Copy parameters in (resets the Adam moments and step count) or out. */
gnmppi_status gnmppi_mlp_set_params(gnmppi_mlp_t m, int32_t mem, const double* params, int64_t count);
gnmppi_status gnmppi_mlp_get_params(gnmppi_mlp_t m, int32_t mem, double* params, int64_t count);
/* Training checkpoint (the paper has no counterpart; the network itself is
 * prior art, Sec. 1): the FP32 master parameters, Adam's first and second
 * moments (count doubles each, in `mem` memory) and the step count.  Setting
 * a state saved by get_state makes later train_step calls continue exactly
 * where the saved handle would have (the state is held in FP32, so a round
 * trip through doubles is exact).  Errors: E_ARG on NULL arrays, a count that
 * is not the parameter count, or a negative step. */
gnmppi_status gnmppi_mlp_get_state(gnmppi_mlp_t m, int32_t mem, double* params, double* m1, double* m2, int64_t count,
                                   int32_t* step);
gnmppi_status gnmppi_mlp_set_state(gnmppi_mlp_t m, int32_t mem, const double* params, const double* m1,
                                   const double* m2, int64_t count, int32_t step);
/* Input normalisation (host arrays of d_0) and the output scale: the network
 * is trained on the optimal controls divided by y_scale and warm-starts with U_0 = y_scale mu,
 * sigma = y_scale exp(s). */
gnmppi_status gnmppi_mlp_set_normalization(gnmppi_mlp_t m, const double* x_mean, const double* x_std, double y_scale);
/* Raw network outputs Y [B][d_L] for inputs X [B][d_0]. */
gnmppi_status gnmppi_mlp_forward(gnmppi_mlp_t m, int32_t mem, const double* X, int32_t B, double* Y);
/* Mean loss (host double, nullable) and its gradient (grad: n_params doubles
 * in `mem` memory, nullable) for inputs X [B][d_0] and targets T [B][n_mu]. */
gnmppi_status gnmppi_mlp_loss_grad(gnmppi_mlp_t m, int32_t mem, const double* X, const double* T, int32_t B,
                                   double* loss, double* grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on one minibatch; loss
 * (host, nullable) receives the minibatch loss before the step. */
gnmppi_status gnmppi_mlp_train_step(gnmppi_mlp_t m, int32_t mem, const double* X, const double* T, int32_t B,
                                    double lr, double* loss);
/* Warm start for B states: U0 [B][n_mu] and per-component sigma [B][n_mu]
 * (both laid out like gnmppi_solve's U and sigma for a uniform batch).  The
 * sampling scale is clamped to [sigma_min, sigma_max]: the network's scale is
 * its uncertainty about U*, which can fall below what a finite-difference
 * Jacobian from FP32 rollouts resolves. */
gnmppi_status gnmppi_mlp_warm_start(gnmppi_mlp_t m, int32_t mem, const double* X, int32_t B, double sigma_min,
                                    double sigma_max, double* U0, double* sigma);
void gnmppi_mlp_destroy(gnmppi_mlp_t m);
const char* gnmppi_mlp_last_error(gnmppi_mlp_t m);

/* Number of kernels the library launched on this handle since creation. */
int64_t gnmppi_launch_count(gnmppi_t h);

/* Bounds-check build (the paper has no counterpart; a stand-in for a memory
 * checker): in a library compiled with -DGNMPPI_CHECK (libgnmppi_check.so)
 * the hot kernels' global stores check their index against the instance's
 * block and skip, and count, any that fall outside.  Returns the number of
 * such stores since the last call on the current device (synchronising it)
 * and clears the counters; -1 in the normal build, -2 on a CUDA error. */
int64_t gnmppi_check_count(void);

/* Release the handle and all its device memory.  NULL is ignored. */
void gnmppi_destroy(gnmppi_t h);

/* Text of the last error on h (static string for h == NULL). */
const char* gnmppi_last_error(gnmppi_t h);

/* Name of a status code. */
const char* gnmppi_status_string(int32_t status);

/* ABI version (major*10000 + minor*100 + patch). */
int32_t gnmppi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GNMPPI_H */
