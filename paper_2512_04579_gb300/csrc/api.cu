// api.cu -- host side of the GN-MPPI C ABI (include/gnmppi.h): argument
// validation, workspace layout in HBM, the per-iteration launch sequence of
// Algorithm 1 (arXiv 2512.04579) and its capture into one CUDA graph per solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <array>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gnmppi.h"
#include "launch.cuh"
#include "solver_kernels.cuh"
#include "tc_contract.cuh"

using namespace gnm;

namespace {

struct Group {
  int key = 0;
  Launchers fn{};
  std::vector<int> insts;
  std::vector<int2> bmap;
  int* d_list = nullptr;
  int2* d_bmap = nullptr;
  int smem = 0;
  double work = 0.0;  // rollout steps x state size, for the branch assignment
  int branch = 0;
};

constexpr int kMaxBranches = 8;

// Launch configuration picked by the autotuner (or the defaults).
struct TuneCfg {
  int branches = 1;   // concurrent graph branches for the per-size rollout groups
  int solve_nt = 256; // threads per k_solve CTA (512: one CTA per SM, 256: two, 128: four)
  int contract_mt = 2; // BF16 contraction tile: A sub-tiles per CTA (2: one CTA per SM, 1: two)
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct gnmppi_s {
  gnmppi_problem p{};
  int batch = 0;
  int nmax = 0;  // largest horizon N of the instances
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<InstDesc> desc;
  InstDesc* d_desc = nullptr;
  InstState* d_st = nullptr;
  Consts cs{};
  // workspace
  double *d_x0 = nullptr, *d_xref = nullptr, *d_U = nullptr, *d_s = nullptr, *d_g = nullptr, *d_mppi = nullptr;
  double *d_delta = nullptr, *d_y = nullptr, *d_C = nullptr, *d_e = nullptr, *d_A = nullptr;
  double *d_S2 = nullptr, *d_H = nullptr, *d_Cl = nullptr, *d_Cout = nullptr, *d_lin = nullptr, *d_Lg = nullptr;
  int64_t* d_oL = nullptr;
  void *d_dR = nullptr, *d_W = nullptr, *d_P = nullptr, *d_r = nullptr, *d_RL = nullptr;
  uint32_t* d_W2 = nullptr;  // BF16 mode: W split into BF16 head and remainder (the contraction's B rows)
  int64_t n_x0 = 0, n_xref = 0, n_U = 0, n_dR = 0, n_W = 0, n_C = 0, n_P = 0, n_nn = 0, n_R = 0, n_RL = 0, n_L = 0;
  size_t szT = 8, szS = 8, szA = 8;
  int4* d_tiles[3] = {nullptr, nullptr, nullptr};
  int ntiles[3] = {0, 0, 0};
  std::vector<Group> groups;
  int* d_all = nullptr;  // 0..batch-1
  std::vector<int> order;  // k_solve instance order
  int* d_order = nullptr;
  int solve_smem = 0;
  bool use_tc = false;
  // concurrency of the rollout groups and the solve CTA shape
  TuneCfg tune{};
  std::string tune_report;
  // asynchronous solve: per-instance states (and the initial ones of a
  // masked solve) and the tensor-core error word pass through pinned host memory
  InstState* h_st = nullptr;
  InstState* h_init = nullptr;
  int* h_err = nullptr;
  // test injection (gnmppi_debug_inject): kind 3 = tensor-core wait at iteration inj_it
  int inj_tc = 0;
  cudaEvent_t ev_done = nullptr;
  bool pending = false;
  cudaStream_t aux[kMaxBranches] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxBranches] = {};
  // the softmin's graph branch beside the contraction and Gram
  cudaStream_t side = nullptr;
  cudaEvent_t ev_side_fork = nullptr, ev_side_join = nullptr;
  TcPlan tc{};
  // graph of one Algorithm-1 solve
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_nodes = 0;
  int64_t launches = 0;
  std::vector<void*> allocs;
  std::string err;
};

static thread_local std::string g_create_err;  // errors raised before a handle exists

static void assign_branches(gnmppi_t h, int nb);
static void set_branches(gnmppi_t h, int nb) {
  h->tune.branches = std::max(1, std::min(nb, kMaxBranches));
  assign_branches(h, h->tune.branches);
}

static gnmppi_status fail(gnmppi_t h, gnmppi_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_err = buf;
  return st;
}

#define CK(call)                                                                                       \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return fail(h, GNMPPI_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                            \
  } while (0)

#define CKL()                                                                                          \
  do {                                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                                               \
    if (e_ != cudaSuccess) return fail(h, GNMPPI_E_CUDA, "launch: %s (%s:%d)", cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                            \
  } while (0)

template <typename P>
static gnmppi_status dalloc(gnmppi_t h, P** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, GNMPPI_E_NOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back((void*)*ptr);
  e = cudaMemsetAsync(*ptr, 0, bytes, h->stream);
  if (e != cudaSuccess) return fail(h, GNMPPI_E_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
  return GNMPPI_OK;
}

static bool get_launchers(int prec, int dyn, int key, Launchers* o) {
  // both reduced modes roll out and store dR / W in FP32; they differ in the
  // tensor-core format of the contraction only
  if (dyn == kChain && key > kMaxChainF) return prec == kFP64 ? group_launchers_f64(key, o) : group_launchers_f32(key, o);
  return prec == kFP64 ? launchers_f64(dyn, key, o) : launchers_f32(dyn, key, o);
}

static gnmppi_status validate(const gnmppi_problem* p, int32_t batch, const gnmppi_instance_shape* shapes) {
  if (!p) return fail(nullptr, GNMPPI_E_ARG, "problem is NULL");
  if (batch < 1) return fail(nullptr, GNMPPI_E_ARG, "batch must be >= 1");
  if (p->dynamics < 0 || p->dynamics > 5) return fail(nullptr, GNMPPI_E_ARG, "unknown dynamics");
  if (p->precision < 0 || p->precision > 2) return fail(nullptr, GNMPPI_E_ARG, "unknown precision");
  if (p->jac_mode < 0 || p->jac_mode > 2) return fail(nullptr, GNMPPI_E_ARG, "unknown jac_mode");
  if (p->L < 1 || p->L > kMaxL) return fail(nullptr, GNMPPI_E_ARG, "L must be in 1..%d", kMaxL);
  if (!(p->gamma > 0.0 && p->gamma < 1.0)) return fail(nullptr, GNMPPI_E_ARG, "gamma must be in (0,1)");
  if (!(p->beta > 0.0 && p->beta <= 1.0)) return fail(nullptr, GNMPPI_E_ARG, "beta must be in (0,1]");
  if (!(p->tau > 0.0)) return fail(nullptr, GNMPPI_E_ARG, "tau must be > 0");
  if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) return fail(nullptr, GNMPPI_E_ARG, "lambda must be >= 0");
  if (!(p->sigma0 > 0.0) || !std::isfinite(p->sigma0)) return fail(nullptr, GNMPPI_E_ARG, "sigma0 must be > 0");
  if (p->iterations < 0) return fail(nullptr, GNMPPI_E_ARG, "iterations must be >= 0");
  if (p->ir_steps < 0 || p->ir_steps > 10) return fail(nullptr, GNMPPI_E_ARG, "ir_steps must be in 0..10");
  if ((p->dynamics == GNMPPI_DYN_PENDULUM || p->dynamics == GNMPPI_DYN_CHAIN) && !(p->dt > 0.0))
    return fail(nullptr, GNMPPI_E_ARG, "dt must be > 0");
  if (p->sampling != GNMPPI_SAMPLE_RANDOM && p->sampling != GNMPPI_SAMPLE_SIGMA)
    return fail(nullptr, GNMPPI_E_ARG, "unknown sampling");
  if (p->sampling == GNMPPI_SAMPLE_SIGMA && !p->antithetic)
    return fail(nullptr, GNMPPI_E_ARG, "sigma points need antithetic pairs");
  if (p->method != GNMPPI_METHOD_GN && p->method != GNMPPI_METHOD_MPPI)
    return fail(nullptr, GNMPPI_E_ARG, "unknown method");
  if (p->first_instance < 0 || (int64_t)p->first_instance + batch > (1 << 28))
    return fail(nullptr, GNMPPI_E_ARG, "first_instance + batch must be in 0..2^28 (noise-stream counter)");
  if (p->dynamics == GNMPPI_DYN_LINEAR) {
    const int nx = p->nx, nu = p->nu;
    const int key = nx * 16 + nu;
    if (!(key == 2 * 16 + 1 || key == 2 * 16 + 2 || key == 4 * 16 + 1 || key == 4 * 16 + 2 || key == 16 + 1))
      return fail(nullptr, GNMPPI_E_ARG, "linear (nx, nu) must be one of (1,1) (2,1) (2,2) (4,1) (4,2)");
    if (!p->lin || p->n_lin != nx * nx + nx * nu + nx + nu + nx)
      return fail(nullptr, GNMPPI_E_ARG, "linear model needs lin with nx*nx + nx*nu + 2nx + nu doubles");
  }
  for (int b = 0; b < batch; ++b) {
    const int N = (shapes && shapes[b].N > 0) ? shapes[b].N : p->N;
    const int M = (shapes && shapes[b].M > 0) ? shapes[b].M : p->M;
    const bool testfun = p->dynamics >= GNMPPI_DYN_ROSENBROCK;
    if (testfun && ((shapes && shapes[b].N > 0) ? shapes[b].N : p->N) != 1)
      return fail(nullptr, GNMPPI_E_ARG, "instance %d: the test problems have N = 1", b);
    const int nu_b = p->dynamics == GNMPPI_DYN_CHAIN ? 2
                     : p->dynamics == GNMPPI_DYN_PENDULUM ? 1
                     : p->dynamics == GNMPPI_DYN_HEAVISIDE ? 1
                     : testfun ? 2 : p->nu;
    const int K = p->sampling == GNMPPI_SAMPLE_SIGMA ? 2 * N * nu_b
                                                      : ((shapes && shapes[b].K > 0) ? shapes[b].K : p->K);
    if (N < 1 || N > 100000) return fail(nullptr, GNMPPI_E_ARG, "instance %d: N must be in 1..100000", b);
    if (K < 1 || (p->antithetic && (K % 2 != 0 || K < 2)))
      return fail(nullptr, GNMPPI_E_ARG, "instance %d: K must be >= 1 (even and >= 2 with antithetic pairs)", b);
    if (p->dynamics == GNMPPI_DYN_CHAIN && (M < 2 || M > kMaxChainGroupF + 1))
      return fail(nullptr, GNMPPI_E_ARG, "instance %d: chain M must be in 2..%d", b, kMaxChainGroupF + 1);
    if (p->dynamics == GNMPPI_DYN_CHAIN && M > kMaxChainF + 1 && !p->antithetic)
      return fail(nullptr, GNMPPI_E_ARG, "instance %d: chains of more than %d masses need antithetic sampling", b,
                  kMaxChainF + 1);
    if (K > (1 << 26)) return fail(nullptr, GNMPPI_E_ARG, "instance %d: K too large", b);
  }
  return GNMPPI_OK;
}

extern "C" int32_t gnmppi_version(void) { return 100; }

extern "C" const char* gnmppi_status_string(int32_t s) {
  switch (s) {
    case GNMPPI_OK: return "GNMPPI_OK";
    case GNMPPI_E_ARG: return "GNMPPI_E_ARG";
    case GNMPPI_E_CUDA: return "GNMPPI_E_CUDA";
    case GNMPPI_E_NOT_PD: return "GNMPPI_E_NOT_PD";
    case GNMPPI_E_NONFINITE: return "GNMPPI_E_NONFINITE";
    case GNMPPI_E_TIMEOUT: return "GNMPPI_E_TIMEOUT";
    case GNMPPI_E_NOMEM: return "GNMPPI_E_NOMEM";
    default: return "GNMPPI_E_UNKNOWN";
  }
}

extern "C" const char* gnmppi_last_error(gnmppi_t h) {
  static thread_local char buf[512];
  snprintf(buf, sizeof(buf), "%s", h ? h->err.c_str() : g_create_err.c_str());
  return buf;
}

extern "C" void gnmppi_destroy(gnmppi_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (int i = 0; i < kMaxBranches; ++i) {
    if (h->aux[i]) cudaStreamDestroy(h->aux[i]);
    if (h->ev_join[i]) cudaEventDestroy(h->ev_join[i]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_side_fork) cudaEventDestroy(h->ev_side_fork);
  if (h->ev_side_join) cudaEventDestroy(h->ev_side_join);
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_init) cudaFreeHost(h->h_init);
  if (h->h_err) cudaFreeHost(h->h_err);
  for (void* p : h->allocs) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

extern "C" int64_t gnmppi_launch_count(gnmppi_t h) { return h ? h->launches : 0; }

namespace gnm {
GNM_CHECK_ACCESSOR(check_count_api)
}

extern "C" int64_t gnmppi_check_count(void) {
#ifdef GNMPPI_CHECK
  if (cudaDeviceSynchronize() != cudaSuccess) return -2;
  int64_t n = 0;
  for (unsigned int c : {check_count_rollout_f32(), check_count_rollout_f64(), check_count_group_f32(),
                         check_count_group_f64(), check_count_api(), check_count_tc(), check_count_mlp()}) {
    if (c == 0xffffffffu) return -2;
    n += c;
  }
  return n;
#else
  return -1;
#endif
}

static gnmppi_status build(gnmppi_t h, const gnmppi_instance_shape* shapes) {
  const gnmppi_problem& p = h->p;
  const int prec = p.precision;
  h->szT = prec == kFP64 ? 8 : 4;
  h->szS = prec == kFP64 ? 8 : 4;
  h->szA = prec == kFP64 ? 8 : 4;
  const int anti = p.antithetic ? 1 : 0;
  // per-instance layout
  h->desc.resize(h->batch);
  int64_t oX = 0, oR = 0, oU = 0, odR = 0, oW = 0, oC = 0, oP = 0, onn = 0, orr = 0, orl = 0, oL = 0;
  std::vector<int64_t> offL(h->batch, 0);
  for (int b = 0; b < h->batch; ++b) {
    InstDesc d{};
    d.N = (shapes && shapes[b].N > 0) ? shapes[b].N : p.N;
    const int K = (shapes && shapes[b].K > 0) ? shapes[b].K : p.K;
    if (p.dynamics == GNMPPI_DYN_CHAIN) {
      d.M = (shapes && shapes[b].M > 0) ? shapes[b].M : p.M;
      d.F = d.M - 1;
      d.nx = 4 * d.F;
      d.nu = 2;
      d.rps = 2 * d.F + 2;
      d.nR = d.N * d.rps + 2 * d.F;
      d.nref = 2 * d.F;
    } else if (p.dynamics == GNMPPI_DYN_PENDULUM) {
      d.nx = 2;
      d.nu = 1;
      d.rps = 3;
      d.nR = 3 * d.N + 2;
      d.nref = 1;
    } else if (p.dynamics >= GNMPPI_DYN_ROSENBROCK) {  // static test problems: one stage, no state
      d.nx = 1;
      d.nu = p.dynamics == GNMPPI_DYN_HEAVISIDE ? 1 : 2;
      d.rps = p.dynamics == GNMPPI_DYN_ROSENBROCK ? 2 : (p.dynamics == GNMPPI_DYN_RASTRIGIN ? 4 : 1);
      d.nR = d.N * d.rps;
      d.nref = 1;
    } else {
      d.nx = p.nx;
      d.nu = p.nu;
      d.rps = p.nx + p.nu;
      d.nR = d.N * d.rps + p.nx;
      d.nref = 1;
    }
    d.n = d.N * d.nu;
    d.Kp = p.sampling == GNMPPI_SAMPLE_SIGMA ? d.n : (anti ? K / 2 : K);  // sigma points: n pairs
    d.ldK = (int)round_up(d.Kp, kPadK);
    d.sP = (int)round_up(d.nR, 32);  // S columns start 16-byte aligned (TMA operand of S S^T)
    d.ldP = (int)round_up(d.sP + d.n, 8);
    if (p.jac_mode == GNMPPI_JAC_LSQ) d.lsq = 1;
    else if (p.jac_mode == GNMPPI_JAC_SIGMA) d.lsq = 0;
    else d.lsq = d.Kp >= d.n ? 1 : 0;
    d.o_x0 = oX; oX += d.nx;
    d.o_xref = oR; oR += d.nref;
    d.o_U = oU; oU += d.n;
    // dR and W of an instance form one [nR + n][ldK] block (W rows last), so a
    // single TMA tensor map covers both contraction operands
    d.o_dR = odR;
    d.o_W = odR + (int64_t)d.nR * d.ldK;
    odR += (int64_t)(d.nR + d.n) * d.ldK;
    d.o_W2 = oW;  // the BF16 mode's split W copy, [n][ldK] words
    oW += (int64_t)d.n * d.ldK;
    d.o_C = oC; oC += 2 * (int64_t)d.Kp;
    d.o_P = oP; oP += (int64_t)d.n * d.ldP;
    d.o_nn = onn; onn += (int64_t)d.n * d.n;
    d.o_R = orr; orr += d.nR;
    d.o_RL = orl; orl += (int64_t)p.L * d.nR;
    h->desc[b] = d;
    h->nmax = std::max(h->nmax, d.N);
  }
  // k_solve keeps rhs, x, res, 1/diag and the float split of y (5 n doubles)
  // in shared memory; the packed factor plus the inverted diagonal blocks,
  // and the packed copy of the system, live in global scratch (o_L).
  int n_all_max = 0;
  for (auto& d : h->desc) n_all_max = std::max(n_all_max, d.n);
  for (int b = 0; b < h->batch; ++b) {
    const int n = h->desc[b].n;
    offL[b] = oL;
    oL += (int64_t)n * (n + 1) / 2 + (int64_t)((n + 15) / 16) * 256;
    oL = (oL + 31) / 32 * 32;  // 256-byte aligned per instance
  }
  h->solve_smem = (int)(8 * (int64_t)5 * n_all_max);
  // solve order: largest systems first (longest-processing-time scheduling)
  h->order.resize(h->batch);
  for (int b = 0; b < h->batch; ++b) h->order[b] = b;
  std::stable_sort(h->order.begin(), h->order.end(),
                   [&](int x, int y) { return h->desc[x].n > h->desc[y].n; });
  h->n_x0 = oX; h->n_xref = oR; h->n_U = oU; h->n_dR = odR; h->n_W = oW; h->n_C = oC; h->n_P = oP;
  h->n_nn = onn; h->n_R = orr; h->n_RL = orl; h->n_L = oL;

  gnmppi_status st;
#define AL(ptr, bytes) if ((st = dalloc(h, &(ptr), (bytes))) != GNMPPI_OK) return st
  AL(h->d_desc, sizeof(InstDesc) * h->batch);
  AL(h->d_st, sizeof(InstState) * h->batch);
  AL(h->d_x0, 8 * h->n_x0);
  AL(h->d_xref, 8 * h->n_xref);
  AL(h->d_U, 8 * h->n_U);
  AL(h->d_s, 8 * h->n_U);
  AL(h->d_g, 8 * h->n_U);
  AL(h->d_mppi, 8 * h->n_U);
  AL(h->d_delta, 8 * h->n_U);
  AL(h->d_y, 8 * h->n_U);
  AL(h->d_e, 8 * (h->n_C / 2));
  AL(h->d_C, 8 * h->n_C);
  AL(h->d_A, 8 * h->n_nn);
  AL(h->d_S2, 8 * h->n_nn);
  AL(h->d_H, 8 * h->n_L);
  AL(h->d_Cl, 8 * (int64_t)h->batch * (kMaxL + 1));
  AL(h->d_Cout, 8 * (int64_t)h->batch);
  AL(h->d_dR, h->szS * h->n_dR);
  h->d_W = h->d_dR;
  if (p.precision == kBF16) AL(h->d_W2, 4 * h->n_W);
  AL(h->d_P, h->szA * h->n_P);
  AL(h->d_r, h->szT * h->n_R);
  AL(h->d_RL, h->szT * h->n_RL);
  AL(h->d_Lg, 8 * h->n_L);
  AL(h->d_oL, 8 * (int64_t)h->batch);
  AL(h->d_order, 4 * (int64_t)h->batch);
  AL(h->d_all, 4 * (int64_t)h->batch);
  if (p.dynamics == GNMPPI_DYN_LINEAR) {
    AL(h->d_lin, 8 * (int64_t)p.n_lin);
    CK(cudaMemcpyAsync(h->d_lin, p.lin, 8 * (size_t)p.n_lin, cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaMemcpyAsync(h->d_desc, h->desc.data(), sizeof(InstDesc) * h->batch, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_oL, offL.data(), 8 * (size_t)h->batch, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_order, h->order.data(), 4 * (size_t)h->batch, cudaMemcpyHostToDevice, h->stream));
  std::vector<int> all(h->batch);
  for (int b = 0; b < h->batch; ++b) all[b] = b;
  CK(cudaMemcpyAsync(h->d_all, all.data(), 4 * (size_t)h->batch, cudaMemcpyHostToDevice, h->stream));

  // rollout groups: one kernel instantiation per distinct model size
  std::map<int, int> gidx;
  for (int b = 0; b < h->batch; ++b) {
    const InstDesc& d = h->desc[b];
    int key = 0;
    if (p.dynamics == GNMPPI_DYN_CHAIN) key = d.F;
    if (p.dynamics == GNMPPI_DYN_LINEAR) key = d.nx * 16 + d.nu;
    auto it = gidx.find(key);
    if (it == gidx.end()) {
      Group g;
      g.key = key;
      if (!get_launchers(prec, p.dynamics, key, &g.fn)) return fail(h, GNMPPI_E_ARG, "no kernel for model key %d", key);
      gidx[key] = (int)h->groups.size();
      h->groups.push_back(g);
      it = gidx.find(key);
    }
    Group& g = h->groups[it->second];
    g.insts.push_back(b);
    g.work += (double)d.Kp * d.N * (d.nx + 2);
    const int per = g.fn.pairs_per_block ? g.fn.pairs_per_block : (anti ? kPairsPerBlock : kSamplesPerBlock);
    for (int c = 0; c < (d.Kp + per - 1) / per; ++c) g.bmap.push_back(make_int2(b, c));
    // group kernels stage r and the targets interleaved: (N + 1) stages of 2 slots + 2 words
    const int64_t words = g.fn.slots ? 2 * d.n + (int64_t)(d.N + 1) * (2 * g.fn.slots + 2) + 2 * g.fn.slots
                                     : 2 * d.n + d.nR + d.nref;
    g.smem = std::max(g.smem, (int)(h->szT * words));
  }
  // concurrency: streams and events for up to kMaxBranches graph branches
  for (int i = 0; i < kMaxBranches; ++i) {
    CK(cudaStreamCreateWithFlags(&h->aux[i], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming));
  }
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_side_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_side_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
  CK(cudaMallocHost((void**)&h->h_st, sizeof(InstState) * h->batch));
  CK(cudaMallocHost((void**)&h->h_init, sizeof(InstState) * h->batch));
  CK(cudaMallocHost((void**)&h->h_err, sizeof(int)));
  *h->h_err = 0;
  for (auto& g : h->groups) {
    CK(g.fn.prepare(g.smem));
    AL(g.d_list, 4 * g.insts.size());
    AL(g.d_bmap, sizeof(int2) * g.bmap.size());
    CK(cudaMemcpyAsync(g.d_list, g.insts.data(), 4 * g.insts.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(g.d_bmap, g.bmap.data(), sizeof(int2) * g.bmap.size(), cudaMemcpyHostToDevice, h->stream));
  }
  // GEMM tile maps (64 x 64 tiles)
  std::vector<int4> tl[3];
  for (int b = 0; b < h->batch; ++b) {
    const InstDesc& d = h->desc[b];
    const int tm = (d.n + 63) / 64;
    for (int i = 0; i < tm; ++i) {
      for (int j = 0; j < (d.nR + d.n + 63) / 64; ++j) tl[0].push_back(make_int4(b, i, j, 0));
      for (int j = 0; j < tm; ++j) {
        tl[1].push_back(make_int4(b, i, j, 0));
        if (d.lsq) tl[2].push_back(make_int4(b, i, j, 0));
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    h->ntiles[k] = (int)tl[k].size();
    AL(h->d_tiles[k], sizeof(int4) * std::max<size_t>(1, tl[k].size()));
    if (!tl[k].empty())
      CK(cudaMemcpyAsync(h->d_tiles[k], tl[k].data(), sizeof(int4) * tl[k].size(), cudaMemcpyHostToDevice, h->stream));
  }
#undef AL
  // constants
  Consts& c = h->cs;
  c.dt = p.dt;
  for (int i = 0; i < 8; ++i) c.params[i] = p.params[i];
  c.lambda = p.lambda;
  c.beta_sqrt = std::sqrt(p.beta);
  c.gamma = p.gamma;
  c.tau = p.tau;
  c.seed = p.seed;
  c.L = p.L;
  c.monotone = p.monotone ? 1 : 0;
  c.ir_steps = p.ir_steps;
  c.antithetic = anti;
  c.sampling = p.sampling;
  c.inst_base = p.first_instance;
  c.u_friction = p.dynamics == GNMPPI_DYN_PENDULUM ? p.params[4] : (p.dynamics == GNMPPI_DYN_CHAIN ? p.params[5] : 0.0);
  c.nx_lin = p.nx;
  c.nu_lin = p.nu;
  c.lin = h->d_lin;
  // tensor-core contraction (three TF32 passes, or three BF16 passes, over FP32 operands)
  h->use_tc = prec != kFP64;
  if (h->use_tc) {
    st = tc_plan_create(h->desc, h->d_dR, h->d_W2, h->d_P, prec == kBF16 ? 1 : 0, h->stream, &h->tc, h->err);
    for (void* q : h->tc.allocs) h->allocs.push_back(q);
    if (st != GNMPPI_OK) return st;
  }
  // the Cholesky kernel: vectors only in shared memory, one (512 threads), two
  // (256) or four (128) CTAs per SM, the rest of the carveout left to L1 (which
  // caches the factor's panels)
  {
    int dev = 0, optin = 0, smsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    if (h->solve_smem + 1024 > optin) return fail(h, GNMPPI_E_ARG, "N*nu too large for the solver");
    const int pct2 = std::min(100, (int)(100.0 * 2 * (h->solve_smem + 2048) / std::max(1, smsm)) + 5);
    const int pct4 = std::min(100, (int)(100.0 * 4 * (h->solve_smem + 2048) / std::max(1, smsm)) + 5);
    const int pct1 = std::min(100, (int)(100.0 * (h->solve_smem + 2048) / std::max(1, smsm)) + 5);
    if (prec == kFP64) {
      CK(cudaFuncSetAttribute(k_solve<double, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->solve_smem));
      CK(cudaFuncSetAttribute(k_solve<double, 512>, cudaFuncAttributePreferredSharedMemoryCarveout, pct1));
      CK(cudaFuncSetAttribute(k_solve<double, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->solve_smem));
      CK(cudaFuncSetAttribute(k_solve<double, 256>, cudaFuncAttributePreferredSharedMemoryCarveout, pct2));
      CK(cudaFuncSetAttribute(k_solve<double, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->solve_smem));
      CK(cudaFuncSetAttribute(k_solve<double, 128>, cudaFuncAttributePreferredSharedMemoryCarveout, pct4));
    } else {
      CK(cudaFuncSetAttribute(k_solve<float, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->solve_smem));
      CK(cudaFuncSetAttribute(k_solve<float, 512>, cudaFuncAttributePreferredSharedMemoryCarveout, pct1));
      CK(cudaFuncSetAttribute(k_solve<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->solve_smem));
      CK(cudaFuncSetAttribute(k_solve<float, 256>, cudaFuncAttributePreferredSharedMemoryCarveout, pct2));
      CK(cudaFuncSetAttribute(k_solve<float, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->solve_smem));
      CK(cudaFuncSetAttribute(k_solve<float, 128>, cudaFuncAttributePreferredSharedMemoryCarveout, pct4));
    }
  }
  // default launch configuration (the autotuner may replace it): a batch no
  // larger than the SM count gets one SM per instance, and then 16 warps per
  // Cholesky shorten its serial steps; larger batches pair instances per SM
  {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    h->tune.solve_nt = h->batch <= nsm ? 512 : 256;
  }
  set_branches(h, std::min<int>(4, (int)h->groups.size()));
  CK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_create(const gnmppi_problem* p, int32_t batch, const gnmppi_instance_shape* shapes,
                                       void* cuda_stream, gnmppi_t* out) {
  if (!out) {
    g_create_err = "out is NULL";
    return GNMPPI_E_ARG;
  }
  *out = nullptr;
  gnmppi_status st = validate(p, batch, shapes);
  if (st != GNMPPI_OK) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_create_err = "no CUDA device available";
    return GNMPPI_E_CUDA;
  }
  gnmppi_t h = new gnmppi_s();
  h->p = *p;
  h->p.lin = nullptr;
  h->batch = batch;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      g_create_err = "cudaStreamCreate failed";
      delete h;
      return GNMPPI_E_CUDA;
    }
    h->own_stream = true;
  }
  h->p = *p;
  if (h->p.method == GNMPPI_METHOD_MPPI) {  // the MPPI step is taken whole: one step length, alpha = 1
    h->p.L = 1;
    h->p.monotone = 0;
  }
  st = build(h, shapes);
  h->p.lin = nullptr;
  if (st != GNMPPI_OK) {
    g_create_err = h->err;
    gnmppi_destroy(h);
    return st;
  }
  *out = h;
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_layout(gnmppi_t h, int64_t* x0_off, int64_t* xref_off, int64_t* U_off) {
  if (!h) return GNMPPI_E_ARG;
  for (int b = 0; b <= h->batch; ++b) {
    const bool end = b == h->batch;
    if (x0_off) x0_off[b] = end ? h->n_x0 : h->desc[b].o_x0;
    if (xref_off) xref_off[b] = end ? h->n_xref : h->desc[b].o_xref;
    if (U_off) U_off[b] = end ? h->n_U : h->desc[b].o_U;
  }
  return GNMPPI_OK;
}

// ----------------------------------------------------------------- launches
static RollArgs roll_args(gnmppi_t h, uint32_t it) {
  RollArgs a{};
  a.inst = h->d_desc;
  a.st = h->d_st;
  a.cs = h->cs;
  a.x0 = h->d_x0;
  a.xref = h->d_xref;
  a.U = h->d_U;
  a.s = h->d_s;
  a.delta = h->d_delta;
  a.r = h->d_r;
  a.dR = h->d_dR;
  a.W = h->d_W;
  a.W2 = h->d_W2;
  a.C = h->d_C;
  a.e = h->d_e;
  a.RL = h->d_RL;
  a.Cl = h->d_Cl;
  a.Cout = h->d_Cout;
  a.it = it;
  a.nmax = h->nmax;
  return a;
}

static SolveArgs solve_args(gnmppi_t h, int shrink) {
  SolveArgs a{};
  a.inst = h->d_desc;
  a.st = h->d_st;
  a.cs = h->cs;
  a.U = h->d_U;
  a.s = h->d_s;
  a.g = h->d_g;
  a.mppi = h->d_mppi;
  a.delta = h->d_delta;
  a.y = h->d_y;
  a.C = h->d_C;
  a.e = h->d_e;
  a.W = h->d_W;
  a.P = h->d_P;
  a.A = h->d_A;
  a.S2 = h->d_S2;
  a.H = h->d_H;
  a.Lg = h->d_Lg;
  a.o_L = h->d_oL;
  a.r = h->d_r;
  a.RL = h->d_RL;
  a.Cl = h->d_Cl;
  a.shrink = shrink;
  a.order = h->d_order;
  return a;
}

// Assign the rollout groups to nb branches, heaviest first to the least
// loaded branch (longest-processing-time rule).
static void assign_branches(gnmppi_t h, int nb) {
  std::vector<int> idx(h->groups.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return h->groups[x].work > h->groups[y].work; });
  std::vector<double> load(std::max(1, nb), 0.0);
  for (int gi : idx) {
    const int bi = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    h->groups[gi].branch = bi;
    load[bi] += h->groups[gi].work;
  }
}

// Launch fn(group, stream) for every rollout group: on the handle's stream, or
// forked over tune.branches streams and joined back (also inside a capture,
// where the fork and join become graph edges).
template <class Fn>
static gnmppi_status for_groups(gnmppi_t h, Fn&& fn) {
  const int nb = std::min<int>(h->tune.branches, (int)h->groups.size());
  if (nb <= 1) {
    for (auto& g : h->groups) {
      gnmppi_status st = fn(g, h->stream);
      if (st != GNMPPI_OK) return st;
    }
    return GNMPPI_OK;
  }
  CK(cudaEventRecord(h->ev_fork, h->stream));
  for (int i = 0; i < nb; ++i) CK(cudaStreamWaitEvent(h->aux[i], h->ev_fork, 0));
  for (auto& g : h->groups) {
    gnmppi_status st = fn(g, h->aux[g.branch]);
    if (st != GNMPPI_OK) return st;
  }
  for (int i = 0; i < nb; ++i) {
    CK(cudaEventRecord(h->ev_join[i], h->aux[i]));
    CK(cudaStreamWaitEvent(h->stream, h->ev_join[i], 0));
  }
  return GNMPPI_OK;
}

static gnmppi_status launch_nominal(gnmppi_t h) {
  return for_groups(h, [&](Group& g, cudaStream_t s) -> gnmppi_status {
    RollArgs a = roll_args(h, 0);
    a.list = g.d_list;
    a.count = (int)g.insts.size();
    a.mode = 1;
    g.fn.line(a, a.count, s);
    CKL();
    h->launches++;
    return GNMPPI_OK;
  });
}

static const char* kPhaseNames[] = {"samples", "softmin", "contract", "gram", "s2", "solve", "line", "update"};
constexpr int kNumPhases = 8;

constexpr unsigned kAllPhases = (1u << kNumPhases) - 1;

// ev (nullable): kNumPhases + 1 events recorded before the first phase and
// after each phase.  mask: the phases to launch (bit i = kPhaseNames[i]);
// the autotuner times single phases this way.
template <typename S, typename TA, typename TC, typename T>
static gnmppi_status launch_iteration_t(gnmppi_t h, uint32_t it, int shrink, cudaEvent_t* ev, unsigned mask) {
#define MARK(i) \
  if (ev) CK(cudaEventRecord(ev[i], h->stream))
#define ON(i) (mask & (1u << (i)))
  MARK(0);
  if (ON(0)) {
    gnmppi_status st = for_groups(h, [&](Group& g, cudaStream_t s) -> gnmppi_status {
      RollArgs a = roll_args(h, it);
      a.bmap = g.d_bmap;
      g.fn.samples(a, (int)g.bmap.size(), g.smem, s);
      CKL();
      h->launches++;
      return GNMPPI_OK;
    });
    if (st != GNMPPI_OK) return st;
  }
  MARK(1);
  SolveArgs sa = solve_args(h, shrink);
  sa.it = it;
  // Method C needs no Jacobian: no contraction, Gram or Cholesky
  const bool gn = h->p.method == GNMPPI_METHOD_GN;
  if (!gn) mask &= ~((1u << 2) | (1u << 3) | (1u << 4));
  // The softmin (weights, b = W^T e, the MPPI direction) and the contraction
  // and Gram read the rollouts' outputs and write disjoint arrays, and only
  // the solve reads both: outside phase timing the softmin runs on a graph
  // branch of its own beside the contraction (0.75 ms less per 30-iteration
  // solve of 256 chain instances, M = 10; forcing the largest shared-memory
  // carveout on it, or forking it beside the Gram instead, gained less or lost).
  // (Its one write that the contraction and Gram read, status -4 when every
  // sample of an instance is non-finite, only decides whether they skip an
  // instance that the solve skips anyway.)
  const bool side = !ev && ON(1) && ON(2);
  if (ON(1)) {
    cudaStream_t ss = h->stream;
    if (side) {
      CK(cudaEventRecord(h->ev_side_fork, h->stream));
      CK(cudaStreamWaitEvent(h->side, h->ev_side_fork, 0));
      ss = h->side;
    }
    k_softmin_wvec<S, TC><<<h->batch * kSoftminSplit, 256, 0, ss>>>(sa);
    CKL();
    h->launches++;
    if (side) CK(cudaEventRecord(h->ev_side_join, h->side));
  }
  MARK(2);
  GemmArgs ga{h->d_desc, h->d_st, nullptr, h->d_dR, h->d_W, h->d_P, h->d_A, h->d_S2};
  if (ON(2)) {
    if (h->use_tc) {
      const int inject = h->inj_tc && (int32_t)it == h->cs.inj_it;
      CK(tc_contract_launch(h->tc, h->d_st, reinterpret_cast<float*>(h->d_P), h->stream, inject,
                            h->tune.contract_mt));
      h->launches++;
    } else {
      ga.tiles = h->d_tiles[0];
      k_gemm_nt<kContract, S, TC, TA><<<h->ntiles[0], 256, 0, h->stream>>>(ga);
      CKL();
      h->launches++;
    }
  }
  MARK(3);
  if (ON(3)) {
    if (h->use_tc) {
      CK(tc_gram_launch(h->tc, h->d_st, h->d_A, h->d_S2, h->stream));
      h->launches += h->tc.nred > 0 ? 2 : 1;  // the chunk sum is a second launch
    } else {
      ga.tiles = h->d_tiles[1];
      k_gemm_nt<kGram, TA, TC, double><<<h->ntiles[1], 256, 0, h->stream>>>(ga);
      CKL();
      h->launches++;
    }
  }
  MARK(4);
  if (ON(4) && !h->use_tc && h->ntiles[2] > 0) {  // the tensor-core Gram launch already formed S2
    ga.tiles = h->d_tiles[2];
    k_gemm_nt<kS2, TA, TC, double><<<h->ntiles[2], 256, 0, h->stream>>>(ga);
    CKL();
    h->launches++;
  }
  if (side) CK(cudaStreamWaitEvent(h->stream, h->ev_side_join, 0));
  MARK(5);
  if (ON(5)) {
    if (!gn) k_mppi_step<<<h->batch, 256, 0, h->stream>>>(sa);
    else if (h->tune.solve_nt == 128) k_solve<TA, 128><<<h->batch, 128, h->solve_smem, h->stream>>>(sa);
    else if (h->tune.solve_nt == 512) k_solve<TA, 512><<<h->batch, 512, h->solve_smem, h->stream>>>(sa);
    else k_solve<TA, 256><<<h->batch, 256, h->solve_smem, h->stream>>>(sa);
    CKL();
    h->launches++;
  }
  MARK(6);
  if (ON(6)) {
    gnmppi_status st = for_groups(h, [&](Group& g, cudaStream_t s) -> gnmppi_status {
      RollArgs a = roll_args(h, it);
      a.list = g.d_list;
      a.count = (int)g.insts.size();
      a.ncand = h->p.L;
      a.mode = 0;
      g.fn.line(a, a.count * h->p.L, s);
      CKL();
      h->launches++;
      return GNMPPI_OK;
    });
    if (st != GNMPPI_OK) return st;
  }
  MARK(7);
  if (ON(7)) {
    k_update<T><<<h->batch, 128, 0, h->stream>>>(sa);
    CKL();
    h->launches++;
  }
  MARK(8);
#undef ON
#undef MARK
  return GNMPPI_OK;
}

static gnmppi_status launch_iteration(gnmppi_t h, uint32_t it, int shrink, cudaEvent_t* ev = nullptr,
                                      unsigned mask = kAllPhases) {
  switch (h->p.precision) {
    case kFP64: return launch_iteration_t<double, double, double, double>(h, it, shrink, ev, mask);
    case kFP32: return launch_iteration_t<float, float, float, float>(h, it, shrink, ev, mask);
    default: return launch_iteration_t<float, float, float, float>(h, it, shrink, ev, mask);
  }
}

extern "C" const char* gnmppi_phase_name(int32_t i) { return (i >= 0 && i < kNumPhases) ? kPhaseNames[i] : nullptr; }

extern "C" gnmppi_status gnmppi_phase_times(gnmppi_t h, int32_t iteration, double* ms, int32_t cap, int32_t* nphase) {
  if (!h) return GNMPPI_E_ARG;
  if (!ms || cap < kNumPhases) return fail(h, GNMPPI_E_ARG, "ms needs %d entries", kNumPhases);
  if (iteration < 0) return fail(h, GNMPPI_E_ARG, "iteration must be >= 0");
  cudaEvent_t ev[kNumPhases + 1];
  for (int i = 0; i <= kNumPhases; ++i) CK(cudaEventCreate(&ev[i]));
  gnmppi_status st = launch_iteration(h, (uint32_t)iteration, 0, ev);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (st == GNMPPI_OK && e == cudaSuccess) {
    for (int i = 0; i < kNumPhases; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] = t;
    }
  }
  for (int i = 0; i <= kNumPhases; ++i) cudaEventDestroy(ev[i]);
  if (st != GNMPPI_OK) return st;
  if (e != cudaSuccess) return fail(h, GNMPPI_E_CUDA, "phase timing: %s", cudaGetErrorString(e));
  if (nphase) *nphase = kNumPhases;
  return GNMPPI_OK;
}

static gnmppi_status load_inputs(gnmppi_t h, int32_t mem, const double* x0, const double* xref, const double* U,
                                 const double* sigma) {
  if (!x0 || !U) return fail(h, GNMPPI_E_ARG, "x0 and U must not be NULL");
  if (h->p.dynamics == GNMPPI_DYN_CHAIN && !xref) return fail(h, GNMPPI_E_ARG, "chain needs xref");
  if (mem != GNMPPI_MEM_HOST && mem != GNMPPI_MEM_DEVICE) return fail(h, GNMPPI_E_ARG, "mem must be HOST or DEVICE");
  const cudaMemcpyKind k = mem == GNMPPI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->d_x0, x0, 8 * h->n_x0, k, h->stream));
  if (xref) CK(cudaMemcpyAsync(h->d_xref, xref, 8 * h->n_xref, k, h->stream));
  CK(cudaMemcpyAsync(h->d_U, U, 8 * h->n_U, k, h->stream));
  if (sigma) {
    CK(cudaMemcpyAsync(h->d_s, sigma, 8 * h->n_U, k, h->stream));
  } else {
    const int64_t blocks = std::min<int64_t>(1024, (h->n_U + 255) / 256);
    k_fill<<<(int)std::max<int64_t>(1, blocks), 256, 0, h->stream>>>(h->d_s, h->n_U, h->p.sigma0);
    CKL();
    h->launches++;
  }
  CK(cudaMemsetAsync(h->d_st, 0, sizeof(InstState) * h->batch, h->stream));
  return GNMPPI_OK;
}

// The tensor-core error word (a bounded device wait ran out): copied to
// pinned host memory and cleared on the stream, after the work it covers;
// read by check_timeout once the stream has passed that point.
static gnmppi_status fetch_timeout(gnmppi_t h) {
  if (!h->use_tc) return GNMPPI_OK;
  CK(cudaMemcpyAsync(h->h_err, h->tc.d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemsetAsync(h->tc.d_err, 0, sizeof(int), h->stream));
  return GNMPPI_OK;
}

static gnmppi_status check_timeout(gnmppi_t h) {
  if (!h->use_tc) return GNMPPI_OK;
  if (*h->h_err) {
    *h->h_err = 0;
    return fail(h, GNMPPI_E_TIMEOUT, "a bounded wait in the tensor-core contraction ran out");
  }
  return GNMPPI_OK;
}

static gnmppi_status worst_status(const std::vector<InstState>& s) {
  int w = 0;
  for (auto& x : s)
    if (x.status < 0 && (w == 0 || x.status < w)) w = x.status;
  return (gnmppi_status)w;
}

// Inactive instances carry this status: every kernel skips them.
constexpr int32_t kInactive = 1;

extern "C" gnmppi_status gnmppi_solve_async(gnmppi_t h, int32_t mem, const double* x0, const double* xref,
                                            double* U, const double* sigma, const int32_t* active) {
  if (!h) return GNMPPI_E_ARG;
  if (h->pending) return fail(h, GNMPPI_E_ARG, "a solve is already in flight on this handle");
  gnmppi_status st = load_inputs(h, mem, x0, xref, U, sigma);
  if (st != GNMPPI_OK) return st;
  if (active) {
    // staged in the handle's pinned buffer: the previous solve's copy of it
    // has completed (gnmppi_solve_wait synchronised), so no wait is needed here
    memset(h->h_init, 0, sizeof(InstState) * h->batch);
    for (int b = 0; b < h->batch; ++b) h->h_init[b].status = active[b] ? 0 : kInactive;
    CK(cudaMemcpyAsync(h->d_st, h->h_init, sizeof(InstState) * h->batch, cudaMemcpyHostToDevice, h->stream));
  }
  // one CUDA graph per handle: the nominal rollout and every Algorithm-1 iteration
  if (!h->gexec) {
    cudaGraph_t graph;
    const int64_t before = h->launches;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    gnmppi_status cst = launch_nominal(h);
    for (int it = 0; cst == GNMPPI_OK && it < h->p.iterations; ++it) cst = launch_iteration(h, (uint32_t)it, 1);
    cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (cst != GNMPPI_OK) return cst;
    if (ce != cudaSuccess) return fail(h, GNMPPI_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      h->gexec = nullptr;
      return fail(h, GNMPPI_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    h->graph_nodes = h->launches - before;
    h->launches = before;
  }
  CK(cudaGraphLaunch(h->gexec, h->stream));
  h->launches += h->graph_nodes;
  k_sigma_end<<<(h->batch + 127) / 128, 128, 0, h->stream>>>(h->d_desc, h->d_st, h->d_s, h->batch);
  CKL();
  h->launches++;
  const cudaMemcpyKind k = mem == GNMPPI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(U, h->d_U, 8 * h->n_U, k, h->stream));
  CK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(InstState) * h->batch, cudaMemcpyDeviceToHost, h->stream));
  gnmppi_status fst = fetch_timeout(h);
  if (fst != GNMPPI_OK) return fst;
  CK(cudaEventRecord(h->ev_done, h->stream));
  h->pending = true;
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_solve_wait(gnmppi_t h, gnmppi_report* rep) {
  if (!h) return GNMPPI_E_ARG;
  if (!h->pending) return fail(h, GNMPPI_E_ARG, "no solve in flight on this handle");
  h->pending = false;
  gnmppi_status st;
  CK(cudaEventSynchronize(h->ev_done));
  if ((st = check_timeout(h)) != GNMPPI_OK) return st;
  std::vector<InstState> s(h->h_st, h->h_st + h->batch);
  if (rep) {
    for (int b = 0; b < h->batch; ++b) {
      rep[b].C_final = s[b].C_nom;
      rep[b].C_initial = s[b].C_init;
      rep[b].C_prev = s[b].iters > 0 ? s[b].C_start : s[b].C_nom;
      rep[b].sigma_final = s[b].sigma_end;
      rep[b].iterations = s[b].iters;
      rep[b].status = s[b].status == kInactive ? 0 : s[b].status;
      rep[b].n_masked = s[b].total_masked;
      rep[b].chol_retries = s[b].total_retries;
    }
  }
  return worst_status(s);
}

extern "C" gnmppi_status gnmppi_solve_masked(gnmppi_t h, int32_t mem, const double* x0, const double* xref,
                                             double* U, const double* sigma, const int32_t* active,
                                             gnmppi_report* rep) {
  gnmppi_status st = gnmppi_solve_async(h, mem, x0, xref, U, sigma, active);
  if (st != GNMPPI_OK) return st;
  return gnmppi_solve_wait(h, rep);
}

extern "C" gnmppi_status gnmppi_solve(gnmppi_t h, int32_t mem, const double* x0, const double* xref, double* U,
                                      const double* sigma, gnmppi_report* rep) {
  return gnmppi_solve_masked(h, mem, x0, xref, U, sigma, nullptr, rep);
}

extern "C" gnmppi_status gnmppi_step(gnmppi_t h, int32_t mem, const double* x0, const double* xref, double* U,
                                     const double* sigma, int32_t iteration, gnmppi_iter_report* rep) {
  if (!h) return GNMPPI_E_ARG;
  if (iteration < 0) return fail(h, GNMPPI_E_ARG, "iteration must be >= 0");
  gnmppi_status st = load_inputs(h, mem, x0, xref, U, sigma);
  if (st != GNMPPI_OK) return st;
  st = launch_nominal(h);
  if (st != GNMPPI_OK) return st;
  st = launch_iteration(h, (uint32_t)iteration, 0);
  if (st != GNMPPI_OK) return st;
  const cudaMemcpyKind k = mem == GNMPPI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(U, h->d_U, 8 * h->n_U, k, h->stream));
  std::vector<InstState> s(h->batch);
  CK(cudaMemcpyAsync(s.data(), h->d_st, sizeof(InstState) * h->batch, cudaMemcpyDeviceToHost, h->stream));
  if ((st = fetch_timeout(h)) != GNMPPI_OK) return st;
  CK(cudaStreamSynchronize(h->stream));
  if ((st = check_timeout(h)) != GNMPPI_OK) return st;
  if (rep) {
    for (int b = 0; b < h->batch; ++b) {
      gnmppi_iter_report& r = rep[b];
      const InstState& x = s[b];
      r.C_nom = x.iters > 0 ? x.C_start : x.C_nom;
      r.C_new = x.C_new;
      r.alpha = x.alpha;
      r.lambda_used = x.lambda_used;
      r.c_min = x.c_min;
      r.sum_w = x.sum_w;
      r.sum_w2 = x.sum_w2;
      r.ess = x.ess;
      r.pr_norm = x.pr_norm;
      r.step_norm = x.step_norm;
      r.j_star = x.j_star;
      r.n_masked = x.n_masked;
      r.jac_mode_used = x.jac_mode_used;
      r.status = x.status;
      r.chol_retries = x.chol_retries;
      r.pad = 0;
    }
  }
  return worst_status(s);
}

extern "C" gnmppi_status gnmppi_cost(gnmppi_t h, int32_t mem, const double* x0, const double* xref, const double* U,
                                     double* C) {
  if (!h) return GNMPPI_E_ARG;
  if (!C) return fail(h, GNMPPI_E_ARG, "C must not be NULL");
  gnmppi_status st = load_inputs(h, mem, x0, xref, U, nullptr);
  if (st != GNMPPI_OK) return st;
  for (auto& g : h->groups) {
    RollArgs a = roll_args(h, 0);
    a.list = g.d_list;
    a.count = (int)g.insts.size();
    a.mode = 2;
    g.fn.cost64(a, a.count, h->stream);
    CKL();
    h->launches++;
  }
  const cudaMemcpyKind k = mem == GNMPPI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(C, h->d_Cout, 8 * (size_t)h->batch, k, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}

// ------------------------------------------------------------ verification
template <typename X>
static void widen(const void* src, double* dst, int64_t count) {
  const X* s = reinterpret_cast<const X*>(src);
  for (int64_t i = 0; i < count; ++i) dst[i] = (double)s[i];
}

static gnmppi_status read_typed(gnmppi_t h, const void* dptr, size_t esz, int kind, int64_t count, double* out) {
  std::vector<unsigned char> tmp((size_t)count * esz);
  CK(cudaMemcpy(tmp.data(), dptr, tmp.size(), cudaMemcpyDeviceToHost));
  if (esz == 8) widen<double>(tmp.data(), out, count);
  else widen<float>(tmp.data(), out, count);
  (void)kind;
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_debug_read(gnmppi_t h, int32_t what, int32_t inst, double* host_out, int64_t count,
                                           int64_t* written) {
  if (!h) return GNMPPI_E_ARG;
  if (inst < 0 || inst >= h->batch) return fail(h, GNMPPI_E_ARG, "instance out of range");
  if (!host_out) return fail(h, GNMPPI_E_ARG, "host_out is NULL");
  CK(cudaStreamSynchronize(h->stream));
  const InstDesc& d = h->desc[inst];
  int64_t need = 0;
  gnmppi_status st = GNMPPI_OK;
  auto rows = [&](const unsigned char* base, size_t esz, int64_t nrows, int64_t ld, int64_t ncols) -> gnmppi_status {
    need = nrows * ncols;
    if (count < need) return fail(h, GNMPPI_E_ARG, "buffer too small: need %lld doubles", (long long)need);
    std::vector<double> row(ld);
    for (int64_t r = 0; r < nrows; ++r) {
      gnmppi_status s2 = read_typed(h, base + (size_t)r * ld * esz, esz, 0, ncols, host_out + r * ncols);
      if (s2 != GNMPPI_OK) return s2;
    }
    return GNMPPI_OK;
  };
  const unsigned char* dR = (const unsigned char*)h->d_dR + h->szS * d.o_dR;
  const unsigned char* W = (const unsigned char*)h->d_W + h->szS * d.o_W;
  const unsigned char* P = (const unsigned char*)h->d_P + h->szA * d.o_P;
  switch (what) {
    case 0: st = rows(dR, h->szS, d.nR, d.ldK, d.Kp); break;
    case 1: st = rows(W, h->szS, d.n, d.ldK, d.Kp); break;
    case 2: {
      const int64_t nc = h->p.antithetic ? 2 * (int64_t)d.Kp : d.Kp;
      st = rows((const unsigned char*)(h->d_C + d.o_C), 8, 1, nc, nc);
      break;
    }
    case 3: st = rows((const unsigned char*)(h->d_e + d.o_C / 2), 8, 1, d.Kp, d.Kp); break;
    case 4: {  // rows [P^T | S] without the alignment gap between the two parts
      need = (int64_t)d.n * (d.nR + d.n);
      if (count < need) return fail(h, GNMPPI_E_ARG, "buffer too small: need %lld doubles", (long long)need);
      for (int64_t r = 0; r < d.n && st == GNMPPI_OK; ++r) {
        double* o = host_out + r * (d.nR + d.n);
        st = read_typed(h, P + (size_t)r * d.ldP * h->szA, h->szA, 0, d.nR, o);
        if (st == GNMPPI_OK) st = read_typed(h, P + ((size_t)r * d.ldP + d.sP) * h->szA, h->szA, 0, d.n, o + d.nR);
      }
      break;
    }
    case 5: st = rows((const unsigned char*)(h->d_A + d.o_nn), 8, d.n, d.n, d.n); break;
    case 6: st = rows((const unsigned char*)(h->d_g + d.o_U), 8, 1, d.n, d.n); break;
    case 7: st = rows((const unsigned char*)(h->d_delta + d.o_U), 8, 1, d.n, d.n); break;
    case 8: st = rows((const unsigned char*)(h->d_Cl + (int64_t)inst * (kMaxL + 1)), 8, 1, h->p.L, h->p.L); break;
    case 9: st = rows((const unsigned char*)h->d_r + h->szT * d.o_R, h->szT, 1, d.nR, d.nR); break;
    case 10: st = rows((const unsigned char*)(h->d_mppi + d.o_U), 8, 1, d.n, d.n); break;
    case 11: st = rows((const unsigned char*)(h->d_S2 + d.o_nn), 8, d.n, d.n, d.n); break;
    default: return fail(h, GNMPPI_E_ARG, "unknown buffer %d", what);
  }
  if (written) *written = (st == GNMPPI_OK) ? need : 0;
  return st;
}

// ---------------------------------------------------------------- autotuner
// Picks the launch configuration of a handle by timing the candidates on its
// own instances and inputs: the number of concurrent graph branches for the
// per-size rollout groups (samples and line search), the k_solve CTA shape and,
// in BF16 mode, the contraction tile.  Choices are cached per process under a
// signature of the device, the model and the multiset of instance shapes, and
// appended to the text file named by GNMPPI_TUNE_FILE (one "signature branches
// solve_nt contract_mt" line per entry), which later processes read back.
namespace {

std::mutex g_tune_mu;
std::map<std::string, TuneCfg> g_tune_cache;
bool g_tune_file_read = false;

std::string tune_signature(gnmppi_t h) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string name = prop.name;
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  std::vector<std::array<int, 4>> sh;
  sh.reserve(h->desc.size());
  for (auto& d : h->desc) sh.push_back({d.n, d.nR, d.Kp, d.nx});
  std::sort(sh.begin(), sh.end());
  uint64_t f = 1469598103934665603ull;  // FNV-1a over the sorted shapes
  for (auto& a : sh)
    for (int v : a) {
      for (int byte = 0; byte < 4; ++byte) {
        f ^= (uint64_t)((uint32_t)v >> (8 * byte)) & 0xffu;
        f *= 1099511628211ull;
      }
    }
  char buf[320];
  snprintf(buf, sizeof(buf), "%s/sm%d/dyn%d/prec%d/anti%d/L%d/meth%d/B%d/%016llx", name.c_str(),
           prop.multiProcessorCount, h->p.dynamics, h->p.precision, h->p.antithetic ? 1 : 0, h->p.L, h->p.method,
           h->batch, (unsigned long long)f);
  return buf;
}

void read_tune_file() {  // under g_tune_mu
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = getenv("GNMPPI_TUNE_FILE");
  if (!path || !*path) return;
  FILE* fp = fopen(path, "r");
  if (!fp) return;
  char line[512], sig[320];
  while (fgets(line, sizeof(line), fp)) {
    int nb = 0, nt = 0, mt = 2;
    const int got = sscanf(line, "%319s %d %d %d", sig, &nb, &nt, &mt);  // lines without the tile field: 2
    if (got >= 3 && nb >= 1 && nb <= kMaxBranches && (nt == 128 || nt == 256 || nt == 512) && (mt == 1 || mt == 2))
      g_tune_cache[sig] = TuneCfg{nb, nt, mt};
  }
  fclose(fp);
}

void append_tune_file(const std::string& sig, const TuneCfg& c) {  // under g_tune_mu
  const char* path = getenv("GNMPPI_TUNE_FILE");
  if (!path || !*path) return;
  FILE* fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d %d\n", sig.c_str(), c.branches, c.solve_nt, c.contract_mt);
  fclose(fp);
}

}  // namespace

static void drop_graph(gnmppi_t h) {
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
}

// Minimum over reps of the device time of the masked phases of iteration 0.
static gnmppi_status time_phases(gnmppi_t h, unsigned mask, int reps, double* best_ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  gnmppi_status st = GNMPPI_OK;
  for (int r = 0; r <= reps && st == GNMPPI_OK; ++r) {  // r = 0 warms up
    cudaEventRecord(e0, h->stream);
    st = launch_iteration(h, 0, 0, nullptr, mask);
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(h, GNMPPI_E_CUDA, "autotune timing failed");
    float ms = 0.f;
    if (st == GNMPPI_OK && r > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = best;
  return st;
}

extern "C" gnmppi_status gnmppi_tune_set(gnmppi_t h, int32_t branches, int32_t solve_nt, int32_t contract_mt) {
  if (!h) return GNMPPI_E_ARG;
  if (branches < 1 || branches > kMaxBranches) return fail(h, GNMPPI_E_ARG, "branches must be in 1..%d", kMaxBranches);
  if (solve_nt != 128 && solve_nt != 256 && solve_nt != 512)
    return fail(h, GNMPPI_E_ARG, "solve_nt must be 128, 256 or 512");
  if (contract_mt != 0 && contract_mt != 1 && contract_mt != 2)
    return fail(h, GNMPPI_E_ARG, "contract_mt must be 0 (keep), 1 or 2");
  set_branches(h, branches);
  h->tune.solve_nt = solve_nt;
  if (contract_mt) h->tune.contract_mt = contract_mt;
  drop_graph(h);
  char buf[192];
  snprintf(buf, sizeof(buf), "{\"source\": \"set\", \"branches\": %d, \"solve_nt\": %d, \"contract_mt\": %d}",
           h->tune.branches, h->tune.solve_nt, h->tune.contract_mt);
  h->tune_report = buf;
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_autotune(gnmppi_t h, int32_t mem, const double* x0, const double* xref,
                                         const double* U, const double* sigma, int32_t reps) {
  if (!h) return GNMPPI_E_ARG;
  if (reps <= 0) reps = 3;
  const std::string sig = tune_signature(h);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_tune_file();
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      set_branches(h, it->second.branches);
      h->tune.solve_nt = it->second.solve_nt;
      h->tune.contract_mt = it->second.contract_mt;
      drop_graph(h);
      char buf[512];
      snprintf(buf, sizeof(buf),
               "{\"source\": \"cache\", \"signature\": \"%s\", \"branches\": %d, \"solve_nt\": %d, \"contract_mt\": %d}",
               sig.c_str(), h->tune.branches, h->tune.solve_nt, h->tune.contract_mt);
      h->tune_report = buf;
      return GNMPPI_OK;
    }
  }
  // every intermediate of iteration 0 from the caller's inputs, then timings
  gnmppi_status st = load_inputs(h, mem, x0, xref, U, sigma);
  if (st != GNMPPI_OK) return st;
  st = launch_nominal(h);
  if (st != GNMPPI_OK) return st;
  st = launch_iteration(h, 0, 0, nullptr, kAllPhases & ~(1u << 7));  // everything but the update
  if (st != GNMPPI_OK) return st;
  CK(cudaStreamSynchronize(h->stream));
  std::string rows;
  char buf[256];
  // 1. concurrent branches for the rollout groups (samples + line search)
  const int ng = (int)h->groups.size();
  int best_nb = 1;
  if (ng > 1) {
    double best = 1e300;
    for (int nb : {1, 2, 4, 8}) {
      if (nb > 1 && nb / 2 >= ng) break;
      set_branches(h, nb);
      double ms = 0.0;
      st = time_phases(h, (1u << 0) | (1u << 6), reps, &ms);
      if (st != GNMPPI_OK) return st;
      snprintf(buf, sizeof(buf), "%s{\"branches\": %d, \"ms\": %.4f}", rows.empty() ? "" : ", ", nb, ms);
      rows += buf;
      if (ms < best * 0.98) {  // keep fewer branches unless more win clearly
        best = ms;
        best_nb = nb;
      }
    }
  }
  set_branches(h, best_nb);
  // 2. k_solve CTA shape
  int best_nt = 256;
  {
    double best = 1e300;
    for (int nt : {256, 128, 512}) {
      h->tune.solve_nt = nt;
      double ms = 0.0;
      st = time_phases(h, 1u << 5, reps, &ms);
      if (st != GNMPPI_OK) return st;
      snprintf(buf, sizeof(buf), "%s{\"solve_nt\": %d, \"ms\": %.4f}", rows.empty() ? "" : ", ", nt, ms);
      rows += buf;
      if (ms < best * 0.98) {
        best = ms;
        best_nt = nt;
      }
    }
  }
  h->tune.solve_nt = best_nt;
  // 3. BF16 contraction tile: two 128-row A sub-tiles per CTA (one CTA per
  //    SM) or one (two CTAs per SM)
  int best_mt = 2;
  if (h->use_tc && h->p.precision == kBF16) {
    double best = 1e300;
    for (int mt : {2, 1}) {
      h->tune.contract_mt = mt;
      double ms = 0.0;
      st = time_phases(h, 1u << 2, reps, &ms);
      if (st != GNMPPI_OK) return st;
      snprintf(buf, sizeof(buf), "%s{\"contract_mt\": %d, \"ms\": %.4f}", rows.empty() ? "" : ", ", mt, ms);
      rows += buf;
      if (ms < best * 0.98) {
        best = ms;
        best_mt = mt;
      }
    }
  }
  h->tune.contract_mt = best_mt;
  if ((st = fetch_timeout(h)) != GNMPPI_OK) return st;
  CK(cudaStreamSynchronize(h->stream));
  st = check_timeout(h);
  if (st != GNMPPI_OK) return st;
  drop_graph(h);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[sig] = h->tune;
    append_tune_file(sig, h->tune);
  }
  h->tune_report = std::string("{\"source\": \"timed\", \"signature\": \"") + sig + "\", \"branches\": " +
                   std::to_string(h->tune.branches) + ", \"solve_nt\": " + std::to_string(h->tune.solve_nt) +
                   ", \"contract_mt\": " + std::to_string(h->tune.contract_mt) + ", \"candidates\": [" + rows + "]}";
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_debug_inject(gnmppi_t h, int32_t kind, int32_t iteration) {
  if (!h) return GNMPPI_E_ARG;
  if (kind < 0 || kind > 3) return fail(h, GNMPPI_E_ARG, "unknown injection kind %d", (int)kind);
  if (kind == 3 && !h->use_tc) return fail(h, GNMPPI_E_ARG, "the FP64 mode has no tensor-core waits");
  h->cs.inj_kind = (kind == 1 || kind == 2) ? kind : 0;
  h->inj_tc = kind == 3 ? 1 : 0;
  h->cs.inj_it = kind == 0 ? -1 : iteration;
  drop_graph(h);  // the captured graph holds the old kernel arguments
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_tune_report(gnmppi_t h, char* buf, int32_t cap) {
  if (!h || !buf || cap <= 0) return GNMPPI_E_ARG;
  std::string r = h->tune_report;
  if (r.empty()) {
    char b[160];
    snprintf(b, sizeof(b), "{\"source\": \"default\", \"branches\": %d, \"solve_nt\": %d, \"contract_mt\": %d}",
             h->tune.branches, h->tune.solve_nt, h->tune.contract_mt);
    r = b;
  }
  if ((int32_t)r.size() + 1 > cap) return fail(h, GNMPPI_E_ARG, "report needs %d bytes", (int)r.size() + 1);
  memcpy(buf, r.c_str(), r.size() + 1);
  return GNMPPI_OK;
}
