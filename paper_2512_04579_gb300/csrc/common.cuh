// common.cuh -- device-side building blocks of the GN-MPPI library: instance
// descriptors, the Philox4x32-10 noise stream with Box-Muller, compensated
// sums, and the dynamics / residual models (Sec. 2, Eq. 1-4 of arXiv
// 2512.04579).  Internal; not part of the C ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gnm {

// ---------------------------------------------------------------------------
// Bounds-check build.  Compiled with -DGNMPPI_CHECK (libgnmppi_check.so), the
// hot kernels' global stores pass their index and the extent of the
// instance's block (or of the output array) through GNM_IN(i, n): an index
// outside [0, n) is counted in this translation unit's offence counter and
// the store is skipped, so a wrong index shows up as a count instead of a
// memory fault (no trap).  gnmppi_check_count() collects the counters.  In
// the normal build GNM_IN(i, n) is `true` and costs nothing.
#ifdef GNMPPI_CHECK
static __device__ unsigned int g_check_offences;
__device__ __forceinline__ bool gnm_in(int64_t i, int64_t n) {
  if (i >= 0 && i < n) return true;
  atomicAdd(&g_check_offences, 1u);
  return false;
}
#define GNM_IN(i, n) ::gnm::gnm_in((int64_t)(i), (int64_t)(n))
// Host side: returns and clears this translation unit's counter.
#define GNM_CHECK_ACCESSOR(name)                                               \
  unsigned int name() {                                                        \
    unsigned int v = 0, z = 0;                                                 \
    if (cudaMemcpyFromSymbol(&v, g_check_offences, sizeof(v)) != cudaSuccess) \
      return 0xffffffffu;                                                      \
    cudaMemcpyToSymbol(g_check_offences, &z, sizeof(z));                       \
    return v;                                                                  \
  }
#else
#define GNM_IN(i, n) true
#define GNM_CHECK_ACCESSOR(name) \
  unsigned int name() { return 0; }
#endif
// one accessor per translation unit that holds kernels
unsigned int check_count_rollout_f32();
unsigned int check_count_rollout_f64();
unsigned int check_count_group_f32();
unsigned int check_count_group_f64();
unsigned int check_count_api();
unsigned int check_count_tc();
unsigned int check_count_mlp();

constexpr int kPairsPerBlock = 64;   // antithetic pairs per rollout CTA (2 lanes each)
constexpr int kSamplesPerBlock = 128;  // one-sided samples per rollout CTA
constexpr int kPadK = 64;            // sample-dimension padding of dR / W rows
constexpr int kMaxL = 32;            // largest line-search set
constexpr int kMaxChainF = 16;       // free masses handled by the thread-per-rollout chain kernels
constexpr int kMaxChainGroupF = 64;  // free masses handled by the group-per-rollout chain kernels

enum Dyn { kPendulum = 0, kChain = 1, kLinear = 2, kRosenbrock = 3, kRastrigin = 4, kHeaviside = 5 };
enum Prec { kFP64 = 0, kFP32 = 1, kBF16 = 2 };

// Per-instance sizes and offsets into the packed workspace arrays.
struct InstDesc {
  int32_t N, M, F, nx, nu, n, nR, rps;  // rps: residual rows per stage
  int32_t Kp;                           // antithetic pairs, or one-sided samples
  int32_t ldK;                          // padded row length of dR / W (multiple of kPadK)
  int32_t ldP;                          // row length of [P^T | S] (sP + n, padded; columns nR..sP unused)
  int32_t lsq;                          // 1: J = P S^-1, 0: J = P Sigma^-1 / K'
  int32_t nref;                         // entries of xref
  int32_t sP;                           // column of S in a [P^T | S] row: nR rounded up to 32 (16-byte aligned)
  int64_t o_x0, o_xref, o_U;            // packed double arrays (x0; xref; U, s, delta, g, ...)
  int64_t o_dR, o_W;                    // dR [nR][ldK], W [n][ldK] (storage type)
  int64_t o_W2;                         // BF16 mode: W split into BF16 head and remainder, [n][ldK] words
  int64_t o_C;                          // sample costs [Kp][2] (double), e and weights [Kp]
  int64_t o_P;                          // [P^T | S]  [n][ldP] (accumulation type)
  int64_t o_nn;                         // n*n double arrays (A, S2, H)
  int64_t o_R;                          // residual r [nR] (scalar type)
  int64_t o_RL;                         // line-search residuals [L][nR] (scalar type)
};

// Per-instance solver state carried across kernels of one iteration.
struct InstState {
  double C_nom;        // C(U_k) of the current iterate
  double C_start;      // C(U_k) at the start of the last completed iteration
  double C_init;       // C(U_0) from the nominal rollout
  double lambda_used;
  double c_min, sum_w, sum_w2, ess, pr_norm, step_norm;
  double C_new, alpha;
  int32_t n_masked, status, chol_retries, j_star;
  int32_t jac_mode_used, total_masked, total_retries, iters;
  int32_t lsq_broken;  // the LSQ system broke down earlier in this solve
  int32_t pad;
  double sigma_end;    // first sampling-scale component after the solve (report)
};

// Problem-wide constants.
struct Consts {
  double dt, params[8];
  double lambda, beta_sqrt, gamma, tau;
  uint64_t seed;
  int32_t L, monotone, ir_steps, antithetic;
  int32_t nx_lin, nu_lin;
  const double* lin;  // device copy of the linear model data
  int32_t sampling;   // 0: Philox normals (Method D), 1: sigma points sqrt(n) e_m (Method E)
  int32_t pad;
  double u_friction;  // dead-zone friction at the input of the dynamics (0: off)
  // test injection (gnmppi_debug_inject): at iteration inj_it, kind 1 makes
  // the LSQ system fail its factorisation at every damping, kind 2 every
  // system of the iteration (0: off)
  int32_t inj_kind, inj_it;
  int32_t inst_base;  // noise-stream index of the handle's first instance
  int32_t pad2;
};

// Setting V.ii of Sec. 5: dead-zone friction at the input of the dynamics,
// u_apply = 0 where |u| <= u_friction (per component), u otherwise; the
// residual still penalises the decision variable u.  uf is the threshold in
// the arithmetic type, taken once per kernel by friction_threshold (negative:
// off), so the per-step test stays off GB300's FP64 pipe in FP32 kernels.
template <typename T>
__device__ __forceinline__ T friction_threshold(const Consts& cs) {
  return cs.u_friction > 0.0 ? (T)cs.u_friction : (T)-1;
}
template <typename T, int NU>
__device__ __forceinline__ void dead_zone(const T* u, T* ua, T uf) {
#pragma unroll
  for (int c = 0; c < NU; ++c) ua[c] = (fabs(u[c]) <= uf) ? (T)0 : u[c];
}

// ------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011) and the noise stream
// ------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Counter layout of the noise stream: (q, sample, iteration, instance*16 + 0),
// key = seed; normals 2q and 2q+1 of the sample's perturbation come from one call.
__device__ __forceinline__ uint4 noise_words(uint64_t seed, uint32_t inst, uint32_t it, uint32_t m, uint32_t q) {
  return philox4x32_10(make_uint4(q, m, it, inst << 4), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Box-Muller in FP64 on 53-bit uniforms u = (hi*2^21 + lo/2^11) 2^-53 + 2^-54.
__device__ __forceinline__ void box_muller(uint4 w, double& z0, double& z1) {
  const uint64_t a = ((uint64_t)w.x << 21) | (uint64_t)(w.y >> 11);
  const uint64_t b = ((uint64_t)w.z << 21) | (uint64_t)(w.w >> 11);
  const double u1 = (double)a * 0x1p-53 + 0x1p-54;
  const double u2 = (double)b * 0x1p-53 + 0x1p-54;
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincos(6.283185307179586 * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

// The same transform in FP32: the uniforms are formed from the same 53 bits
// to FP32 relative accuracy, and cos/sin(2 pi u2) use the exact-argument
// sincospi.
__device__ __forceinline__ void box_muller(uint4 w, float& z0, float& z1) {
  const float u1 = fmaf((float)w.x, 0x1p-32f, fmaf((float)(w.y >> 11), 0x1p-53f, 0x1p-54f));
  const float u2 = fmaf((float)w.z, 0x1p-32f, fmaf((float)(w.w >> 11), 0x1p-53f, 0x1p-54f));
  const float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

// ------------------------------------------------------------------------
// Accumulators: plain in FP64; in FP32 a Neumaier-compensated sum, so that
// costs and dot products over thousands of rows keep FP32-level relative error.
// ------------------------------------------------------------------------
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// One dR / W slot in the storage type (FP64 in the FP64 mode, FP32 otherwise).
__device__ __forceinline__ void put(double* p, double v) { *p = v; }
__device__ __forceinline__ void put(float* p, float v) { *p = v; }

// Sample m of row j of the BF16 mode's split copy of W: the BF16 head of w
// (round to nearest even) and the BF16 rounding of its remainder w - head,
// laid out per 16 samples as 16 heads then 16 remainders (one 64-byte row of
// the contraction's BF16 operand for that k-block).  row: the copy's row j,
// ldK words = 2 ldK BF16 slots.  The same arithmetic as the contraction's
// in-place split of FP32 W rows.
__device__ __forceinline__ void put_w2(uint16_t* row, int m, float w) {
  const __nv_bfloat16 h = __float2bfloat16_rn(w);
  const __nv_bfloat16 l = __float2bfloat16_rn(w - __bfloat162float(h));
  const int i = (m >> 4) * 32 + (m & 15);
  row[i] = __bfloat16_as_ushort(h);
  row[i + 16] = __bfloat16_as_ushort(l);
}

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }

// ------------------------------------------------------------------------
// Models.  Each provides NX, NU, RPS (rows per stage), RT (terminal rows),
// step(x, u) (one RK4 / discrete step in place), stage(x, u, emit) and
// terminal(x, emit), where emit(row, value) receives residual rows in order.
// ------------------------------------------------------------------------
template <typename T>
struct Pendulum {
  static constexpr int NX = 2, NU = 1, RPS = 3, RT = 2;
  T g_l, b, inv_ml2, h, h2, h6;
  __device__ Pendulum(const Consts& c) {
    g_l = (T)(c.params[0] / c.params[1]);
    b = (T)c.params[3];
    inv_ml2 = (T)(1.0 / (c.params[2] * c.params[1] * c.params[1]));
    h = (T)c.dt;
    h2 = (T)(0.5 * c.dt);
    h6 = (T)(c.dt / 6.0);
  }
  __device__ __forceinline__ void f(const T* x, const T* u, T* d) const {
    d[0] = x[1];
    d[1] = -g_l * sin(x[0]) - b * x[1] + u[0] * inv_ml2;
  }
  __device__ __forceinline__ void step(T* x, const T* u) const {
    T k[2], t[2], a[2];
    f(x, u, k);
#pragma unroll
    for (int i = 0; i < 2; ++i) { a[i] = k[i]; t[i] = x[i] + h2 * k[i]; }
    f(t, u, k);
#pragma unroll
    for (int i = 0; i < 2; ++i) { a[i] = a[i] + (T)2 * k[i]; t[i] = x[i] + h2 * k[i]; }
    f(t, u, k);
#pragma unroll
    for (int i = 0; i < 2; ++i) { a[i] = a[i] + (T)2 * k[i]; t[i] = x[i] + h * k[i]; }
    f(t, u, k);
#pragma unroll
    for (int i = 0; i < 2; ++i) x[i] = x[i] + h6 * (a[i] + k[i]);
  }
  template <class E>
  __device__ __forceinline__ void stage(const T* x, const T* u, E& emit) const {
    emit(0, x[0] - (T)3.141592653589793);
    emit(1, (T)0.1 * x[1]);
    emit(2, (T)0.1 * u[0]);
  }
  template <class E>
  __device__ __forceinline__ void terminal(const T* x, E& emit) const {
    emit(0, (T)10 * (x[0] - (T)3.141592653589793));
    emit(1, (T)10 * x[1]);
  }
};

// Chain of F = M-1 free point masses: state [p_1..p_F, v_1..v_F] (2-D each).
template <typename T, int F>
struct Chain {
  static constexpr int NX = 4 * F, NU = 2, RPS = 2 * F + 2, RT = 2 * F;
  T mass_inv, k, k3, c, g, l0, h, h2, h6;
  const T* pref;  // target positions p* (2F), staged by the kernel
  __device__ Chain(const Consts& cs) {
    mass_inv = (T)(1.0 / cs.params[0]);
    k = (T)cs.params[1];
    k3 = (T)cs.params[2];
    c = (T)cs.params[3];
    g = (T)cs.params[4];
    l0 = (T)(1.0 / (double)F);
    h = (T)cs.dt;
    h2 = (T)(0.5 * cs.dt);
    h6 = (T)(cs.dt / 6.0);
    pref = nullptr;
  }
  // Accelerations at state s: link i (masses i-1, i) pulls with tension
  // k d + k3 d^3 along its direction; damping -c v; force u on the last mass;
  // gravity -g along y.  FP32 uses one rsqrt per link; FP64 keeps sqrt and a
  // division.
  __device__ __forceinline__ void accel(const T* s, const T* u, T* acc) const {
    const T* v = s + 2 * F;
#pragma unroll
    for (int i = 0; i < 2 * F; ++i) acc[i] = -c * v[i];
#pragma unroll
    for (int i = 1; i <= F; ++i) {
      const T px0 = (i == 1) ? (T)0 : s[2 * (i - 2)];
      const T py0 = (i == 1) ? (T)0 : s[2 * (i - 2) + 1];
      const T dx = s[2 * (i - 1)] - px0;
      const T dy = s[2 * (i - 1) + 1] - py0;
      const T q = dx * dx + dy * dy;
      T fx, fy;
      if constexpr (sizeof(T) == 4) {
        const T rinv = rsqrtf(q);
        const T dd = q * rinv - l0;
        const T fr = (k * dd + k3 * dd * dd * dd) * rinv;
        fx = fr * dx;
        fy = fr * dy;
      } else {
        const T len = sqrt(q);
        const T dd = len - l0;
        const T fm = k * dd + k3 * dd * dd * dd;
        fx = fm * dx / len;
        fy = fm * dy / len;
      }
      acc[2 * (i - 1)] -= fx;
      acc[2 * (i - 1) + 1] -= fy;
      if (i >= 2) {
        acc[2 * (i - 2)] += fx;
        acc[2 * (i - 2) + 1] += fy;
      }
    }
    acc[2 * (F - 1)] += u[0];
    acc[2 * (F - 1) + 1] += u[1];
#pragma unroll
    for (int i = 0; i < 2 * F; ++i) acc[i] = acc[i] * mass_inv;
#pragma unroll
    for (int i = 0; i < F; ++i) acc[2 * i + 1] -= g;
  }
  // Classical RK4; the position rates are the stage velocities, so only the
  // 2F accelerations are materialised per stage.
  __device__ __forceinline__ void step(T* x, const T* u) const {
    constexpr int H = 2 * F;
    T a[NX], t[NX], acc[H];
    accel(x, u, acc);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      a[i] = x[H + i];
      a[H + i] = acc[i];
      t[i] = x[i] + h2 * x[H + i];
      t[H + i] = x[H + i] + h2 * acc[i];
    }
    accel(t, u, acc);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      a[i] = a[i] + (T)2 * t[H + i];
      a[H + i] = a[H + i] + (T)2 * acc[i];
      t[i] = x[i] + h2 * t[H + i];
      t[H + i] = x[H + i] + h2 * acc[i];
    }
    accel(t, u, acc);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      a[i] = a[i] + (T)2 * t[H + i];
      a[H + i] = a[H + i] + (T)2 * acc[i];
      t[i] = x[i] + h * t[H + i];
      t[H + i] = x[H + i] + h * acc[i];
    }
    accel(t, u, acc);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      x[i] = x[i] + h6 * (a[i] + t[H + i]);
      x[H + i] = x[H + i] + h6 * (a[H + i] + acc[i]);
    }
  }
  template <class E>
  __device__ __forceinline__ void stage(const T* x, const T* u, E& emit) const {
#pragma unroll
    for (int i = 0; i < 2 * F; ++i) emit(i, x[i] - pref[i]);
    emit(2 * F, (T)0.1 * u[0]);
    emit(2 * F + 1, (T)0.1 * u[1]);
  }
  template <class E>
  __device__ __forceinline__ void terminal(const T* x, E& emit) const {
#pragma unroll
    for (int i = 0; i < 2 * F; ++i) emit(i, x[i] - pref[i]);
  }
};

// FP32 chain on paired FP32 instructions: a mass's position, velocity and
// acceleration are float2, updated with FFMA2 / FADD2 / FMUL2 (sm_100+); 1/m
// is folded into the spring, damping and control constants.  The state array
// keeps the scalar layout [p_1..p_F, v_1..v_F] (x, y interleaved) and must be
// 8-byte aligned.
template <int F>
struct Chain<float, F> {
  static constexpr int NX = 4 * F, NU = 2, RPS = 2 * F + 2, RT = 2 * F;
  float mass_inv, k, k3, l0, h, h2, h6, km, k3m;
  float2 cneg, grav, two, hh2, hh, hh6, mneg1;
  const float* pref;
  __device__ Chain(const Consts& cs) {
    mass_inv = (float)(1.0 / cs.params[0]);
    k = (float)cs.params[1];
    k3 = (float)cs.params[2];
    km = (float)(cs.params[1] / cs.params[0]);
    k3m = (float)(cs.params[2] / cs.params[0]);
    const float cm = (float)(-cs.params[3] / cs.params[0]);
    cneg = make_float2(cm, cm);
    grav = make_float2(0.f, (float)(-cs.params[4]));
    l0 = (float)(1.0 / (double)F);
    h = (float)cs.dt;
    h2 = (float)(0.5 * cs.dt);
    h6 = (float)(cs.dt / 6.0);
    two = make_float2(2.f, 2.f);
    hh2 = make_float2(h2, h2);
    hh = make_float2(h, h);
    hh6 = make_float2(h6, h6);
    mneg1 = make_float2(-1.f, -1.f);
    pref = nullptr;
  }
  // acc = (-c v + link forces + u on the last mass) / m - g y
  __device__ __forceinline__ void accel(const float2* p, const float2* v, float2 um, float2* acc) const {
#pragma unroll
    for (int i = 0; i < F; ++i) acc[i] = __ffma2_rn(v[i], cneg, grav);
    acc[F - 1] = __fadd2_rn(acc[F - 1], um);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      const float2 d = (i == 0) ? p[0] : __ffma2_rn(p[i - 1], mneg1, p[i]);
      const float q = fmaf(d.x, d.x, d.y * d.y);
      const float rinv = rsqrtf(q);
      const float dd = fmaf(q, rinv, -l0);
      const float t = fmaf(k3m * dd, dd, km) * dd;
      const float fr = t * rinv;  // (k d + k3 d^3) / (m |d|): the link pulls mass i back, mass i-1 on
      acc[i] = __ffma2_rn(make_float2(-fr, -fr), d, acc[i]);
      if (i > 0) acc[i - 1] = __ffma2_rn(make_float2(fr, fr), d, acc[i - 1]);
    }
  }
  __device__ __forceinline__ void step(float* xs, const float* u) const {
    float2* p = reinterpret_cast<float2*>(xs);
    float2* v = p + F;
    const float2 um = make_float2(u[0] * mass_inv, u[1] * mass_inv);
    float2 ap[F], av[F], tp[F], tv[F], acc[F];
    accel(p, v, um, acc);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      ap[i] = v[i];
      av[i] = acc[i];
      tp[i] = __ffma2_rn(hh2, v[i], p[i]);
      tv[i] = __ffma2_rn(hh2, acc[i], v[i]);
    }
    accel(tp, tv, um, acc);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      ap[i] = __ffma2_rn(two, tv[i], ap[i]);
      av[i] = __ffma2_rn(two, acc[i], av[i]);
      tp[i] = __ffma2_rn(hh2, tv[i], p[i]);
      tv[i] = __ffma2_rn(hh2, acc[i], v[i]);
    }
    accel(tp, tv, um, acc);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      ap[i] = __ffma2_rn(two, tv[i], ap[i]);
      av[i] = __ffma2_rn(two, acc[i], av[i]);
      tp[i] = __ffma2_rn(hh, tv[i], p[i]);
      tv[i] = __ffma2_rn(hh, acc[i], v[i]);
    }
    accel(tp, tv, um, acc);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      p[i] = __ffma2_rn(hh6, __fadd2_rn(ap[i], tv[i]), p[i]);
      v[i] = __ffma2_rn(hh6, __fadd2_rn(av[i], acc[i]), v[i]);
    }
  }
  // residual rows come in (x, y) pairs; pref is 8-byte aligned (shared memory
  // at an even float offset, or an alignas(8) local array)
  template <class E>
  __device__ __forceinline__ void stage(const float* x, const float* u, E& emit) const {
    const float2* pr = reinterpret_cast<const float2*>(pref);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      const float2 q = pr[i];
      emit.pair(2 * i, x[2 * i] - q.x, x[2 * i + 1] - q.y);
    }
    emit.pair(2 * F, 0.1f * u[0], 0.1f * u[1]);
  }
  template <class E>
  __device__ __forceinline__ void terminal(const float* x, E& emit) const {
    const float2* pr = reinterpret_cast<const float2*>(pref);
#pragma unroll
    for (int i = 0; i < F; ++i) {
      const float2 q = pr[i];
      emit.pair(2 * i, x[2 * i] - q.x, x[2 * i + 1] - q.y);
    }
  }
};

// The static test problems of Sec. 5 as one-stage models (N = 1, the state is
// one ignored value, no terminal rows), residual R(u) with Phi = 0.5 ||R||^2:
//   3 Rosenbrock (Problem I):  [sqrt2 (1 - u1), sqrt200 (u2 - u1^2)]
//   4 Rastrigin (Problem II):  sqrt2 [u1, u2, sqrt(5 - 5 cos 2pi u1), sqrt(5 - 5 cos 2pi u2)]
//                              (the paper's R for Phi = ||R||^2, rescaled by sqrt2)
//   5 Heaviside (Problem III): [H(u)], H(u) = 1 for u >= 0, else 0
template <typename T, int KIND>
struct TestFun {
  static constexpr int NX = 1, NU = (KIND == kHeaviside) ? 1 : 2;
  static constexpr int RPS = (KIND == kRosenbrock) ? 2 : ((KIND == kRastrigin) ? 4 : 1), RT = 0;
  __device__ TestFun(const Consts&) {}
  __device__ __forceinline__ void step(T*, const T*) const {}
  template <class E>
  __device__ __forceinline__ void stage(const T*, const T* u, E& emit) const {
    const T r2 = (T)1.4142135623730951;  // sqrt(2)
    if (KIND == kRosenbrock) {
      emit(0, r2 * ((T)1 - u[0]));
      emit(1, (T)14.142135623730951 * (u[1] - u[0] * u[0]));  // sqrt(200)
    } else if (KIND == kRastrigin) {
      const T tp = (T)6.283185307179586;  // 2 pi
      emit(0, r2 * u[0]);
      emit(1, r2 * u[1]);
      emit(2, r2 * sqrt((T)5 - (T)5 * cos(tp * u[0])));
      emit(3, r2 * sqrt((T)5 - (T)5 * cos(tp * u[1])));
    } else {
      emit(0, u[0] >= (T)0 ? (T)1 : (T)0);
    }
  }
  template <class E>
  __device__ __forceinline__ void terminal(const T*, E&) const {}
};

// Discrete linear model x+ = A x + B u with diagonal residual weights.
template <typename T, int NXv, int NUv>
struct Linear {
  static constexpr int NX = NXv, NU = NUv, RPS = NXv + NUv, RT = NXv;
  const double* lin;  // A (NX*NX), B (NX*NU), wq, wr, wqN
  __device__ Linear(const Consts& cs) : lin(cs.lin) {}
  __device__ __forceinline__ void step(T* x, const T* u) const {
    T y[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      T s = (T)0;
#pragma unroll
      for (int j = 0; j < NX; ++j) s += (T)lin[i * NX + j] * x[j];
#pragma unroll
      for (int j = 0; j < NU; ++j) s += (T)lin[NX * NX + i * NU + j] * u[j];
      y[i] = s;
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = y[i];
  }
  template <class E>
  __device__ __forceinline__ void stage(const T* x, const T* u, E& emit) const {
    const double* wq = lin + NX * NX + NX * NU;
#pragma unroll
    for (int i = 0; i < NX; ++i) emit(i, (T)wq[i] * x[i]);
#pragma unroll
    for (int j = 0; j < NU; ++j) emit(NX + j, (T)wq[NX + j] * u[j]);
  }
  template <class E>
  __device__ __forceinline__ void terminal(const T* x, E& emit) const {
    const double* wqN = lin + NX * NX + NX * NU + NX + NU;
#pragma unroll
    for (int i = 0; i < NX; ++i) emit(i, (T)wqN[i] * x[i]);
  }
};

}  // namespace gnm
