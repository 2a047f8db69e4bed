// rollout_group.cuh -- chain rollouts with a group of G lanes per rollout, for
// chains too long for one thread's registers (F = M - 1 free masses up to
// G * FL).  Lane l of a group owns masses l*FL + 1 .. l*FL + FL (1-based;
// masses beyond F are inert placeholders with zero state).  Per right-hand
// side evaluation a lane needs the position of the mass just before its first
// one (shuffle up) and the link just after its last one (its vector and force
// scale, shuffle down); shuffles are width-G so groups never mix.  The two rollouts
// of an antithetic pair are two adjacent groups (partner lane = lane ^ G).
// Same outputs as k_samples / k_line (rollout.cuh): dR, W, sample costs and
// e = dR . r; line-search residuals and costs.
#pragma once
#include "rollout.cuh"

namespace gnm {

// FX > 0: the chain has exactly FX free masses, known at compile time, so
// that the "slot holds a real mass" and "slot holds the forced mass" tests
// fold to constants for every slot but the last lanes' (FX = 0: F at run time).
template <typename T, int FL, int G, int FX = 0>
struct ChainGroup {
  static constexpr int NXL = 4 * FL;  // lane-local state: p (2FL), v (2FL)
  static constexpr bool kRelative = false;  // positions are absolute
  T mass_inv, k, k3, c, g, l0, h, h2, h6;
  int F, lg;
  unsigned mask;  // lanes that execute this group's shuffles together
  const T* pref;  // target positions: global row indexed (pref_local false) or lane-local (2FL)
  bool pref_local;
  __device__ ChainGroup(const Consts& cs, int F_, int lg_, unsigned mask_)
      : F(F_), lg(lg_), mask(mask_), pref(nullptr), pref_local(false) {
    mass_inv = (T)(1.0 / cs.params[0]);
    k = (T)cs.params[1];
    k3 = (T)cs.params[2];
    c = (T)cs.params[3];
    g = (T)cs.params[4];
    l0 = (T)(1.0 / (double)F_);
    h = (T)cs.dt;
    h2 = (T)(0.5 * cs.dt);
    h6 = (T)(cs.dt / 6.0);
  }
  __device__ __forceinline__ int mass(int j) const { return lg * FL + j + 1; }  // 1-based global index
  // slot j of this lane holds a real mass / the mass the control force acts on
  __device__ __forceinline__ bool real(int j) const { return (FX > 0 && j + 1 + (G - 1) * FL <= FX) || mass(j) <= F; }
  __device__ __forceinline__ bool ctrl(int j) const {
    return FX > 0 ? (j == (FX - 1) % FL && lg == (FX - 1) / FL) : mass(j) == F;
  }
  __device__ __forceinline__ void set_reference(const double*) {}
  __device__ __forceinline__ void accel(const T* s, const T* u, T* acc) const {
    const T* v = s + 2 * FL;
    // position of the mass before this lane's first one (origin for lane 0)
    T pxp = __shfl_up_sync(mask, s[2 * (FL - 1)], 1, G);
    T pyp = __shfl_up_sync(mask, s[2 * (FL - 1) + 1], 1, G);
    if (lg == 0) pxp = pyp = (T)0;
    T fx[FL], fy[FL];
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      const T px0 = (j == 0) ? pxp : s[2 * (j - 1)];
      const T py0 = (j == 0) ? pyp : s[2 * (j - 1) + 1];
      const T dx = s[2 * j] - px0;
      const T dy = s[2 * j + 1] - py0;
      const bool real = this->real(j);
      const T q = real ? dx * dx + dy * dy : (T)1;
      if constexpr (sizeof(T) == 4) {
        const T rinv = rsqrtf(q);
        const T dd = q * rinv - l0;
        const T fr = real ? (k * dd + k3 * dd * dd * dd) * rinv : (T)0;
        fx[j] = fr * dx;
        fy[j] = fr * dy;
      } else {
        const T len = sqrt(q);
        const T dd = len - l0;
        const T fm = real ? k * dd + k3 * dd * dd * dd : (T)0;
        fx[j] = fm * dx / len;
        fy[j] = fm * dy / len;
      }
    }
    // force of the link after this lane's last mass (first link of the next lane)
    T fxn = __shfl_down_sync(mask, fx[0], 1, G);
    T fyn = __shfl_down_sync(mask, fy[0], 1, G);
    if (lg == G - 1) fxn = fyn = (T)0;
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      const T nx = (j + 1 < FL) ? fx[j + 1] : fxn;
      const T ny = (j + 1 < FL) ? fy[j + 1] : fyn;
      T ax = -c * v[2 * j] - fx[j] + nx;
      T ay = -c * v[2 * j + 1] - fy[j] + ny;
      if (ctrl(j)) {
        ax += u[0];
        ay += u[1];
      }
      const bool real = this->real(j);
      acc[2 * j] = real ? ax * mass_inv : (T)0;
      acc[2 * j + 1] = real ? ay * mass_inv - g : (T)0;
    }
  }
  __device__ __forceinline__ void step(T* x, const T* u) const {
    constexpr int H = 2 * FL;
    T a[NXL], t[NXL], acc[H];
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
  // Residual rows of this lane at a stage (its masses' position errors; lane
  // 0 also the two control rows at 2F, 2F+1) or at the terminal state, as
  // (x, y) row pairs.  Every lane calls emit.pair(slot, row, v_x, v_y, valid)
  // the same FL + 1 times (slot j < FL: the lane's mass j; slot FL: the
  // controls), so emitters may shuffle; slots that belong to no row of this
  // lane come with valid false.  The target positions are read from pref
  // either lane-local (pref[2j], [2j+1]) or from the group-interleaved layout
  // (pref already offset by 2 lg; mass slot j at pref[2Gj], [2Gj+1]).
  template <class E>
  __device__ __forceinline__ void rows(const T* x, const T* u, bool terminal, E& emit) const {
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      const int i = mass(j);
      const bool real = this->real(j);
      const int r0 = real ? 2 * (i - 1) : 0;
      const T px = pref_local ? pref[2 * j] : pref[2 * G * j];
      const T py = pref_local ? pref[2 * j + 1] : pref[2 * G * j + 1];
      emit.pair(j, r0, x[2 * j] - px, x[2 * j + 1] - py, real);
    }
    const bool urow = !terminal && lg == 0;
    emit.pair(FL, 2 * F, (T)0.1 * u[0], (T)0.1 * u[1], urow);
  }
};

// FP32 group chain on paired FP32 instructions (FFMA2 / FADD2 / FMUL2),
// 1/m folded into the constants; same interface and layout as above, except
// that positions are kept relative to the instance's initial positions (the
// reference): a hanging chain of M masses is some 3M m long, so absolute FP32
// positions carry ~3M u m of rounding and every link vector would be the
// difference of two large numbers.  Here a link vector is its reference
// vector (formed in FP64, rounded once) plus the difference of two small
// deviations, and the residual rows use the target's offset from the
// reference.  Mathematically the same dynamics and residuals.
template <int FL, int G, int FX>
struct ChainGroup<float, FL, G, FX> {
  static constexpr int NXL = 4 * FL;
  static constexpr bool kRelative = true;
  float mass_inv, l0, km, k3m;
  float2 cneg, grav, two, hh2, hh, hh6, mneg1;
  float2 dref[FL];  // reference link vectors ending at this lane's masses
  int F, lg;
  unsigned mask;
  const float* pref;
  bool pref_local;
  __device__ ChainGroup(const Consts& cs, int F_, int lg_, unsigned mask_)
      : F(F_), lg(lg_), mask(mask_), pref(nullptr), pref_local(false) {
    mass_inv = (float)(1.0 / cs.params[0]);
    km = (float)(cs.params[1] / cs.params[0]);
    k3m = (float)(cs.params[2] / cs.params[0]);
    const float cm = (float)(-cs.params[3] / cs.params[0]);
    cneg = make_float2(cm, cm);
    grav = make_float2(0.f, (float)(-cs.params[4]));
    l0 = (float)(1.0 / (double)F_);
    const float h = (float)cs.dt, h2 = (float)(0.5 * cs.dt), h6 = (float)(cs.dt / 6.0);
    two = make_float2(2.f, 2.f);
    hh2 = make_float2(h2, h2);
    hh = make_float2(h, h);
    hh6 = make_float2(h6, h6);
    mneg1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int j = 0; j < FL; ++j) dref[j] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ int mass(int j) const { return lg * FL + j + 1; }
  // slot j of this lane holds a real mass / the mass the control force acts on
  __device__ __forceinline__ bool real(int j) const { return (FX > 0 && j + 1 + (G - 1) * FL <= FX) || mass(j) <= F; }
  __device__ __forceinline__ bool ctrl(int j) const {
    return FX > 0 ? (j == (FX - 1) % FL && lg == (FX - 1) / FL) : mass(j) == F;
  }
  // Reference link vectors from the initial positions x0p (FP64, packed
  // [p_1 .. p_F]); mass 0 is fixed at the origin.
  __device__ __forceinline__ void set_reference(const double* x0p) {
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      const int i = mass(j);
      if (i <= F) {
        const double bx = i > 1 ? x0p[2 * (i - 2)] : 0.0, by = i > 1 ? x0p[2 * (i - 2) + 1] : 0.0;
        dref[j] = make_float2((float)(x0p[2 * (i - 1)] - bx), (float)(x0p[2 * (i - 1) + 1] - by));
      }
    }
  }
  __device__ __forceinline__ void accel(const float2* p, const float2* v, float2 um, float2* acc) const {
    float2 prev;
    prev.x = __shfl_up_sync(mask, p[FL - 1].x, 1, G);
    prev.y = __shfl_up_sync(mask, p[FL - 1].y, 1, G);
    if (lg == 0) prev = make_float2(0.f, 0.f);
    // link j of this lane ends at its mass j: d_j and fr_j with the force
    // fr_j d_j pulling mass j back and the mass before it on
    float2 d[FL];
    float fr[FL];
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      d[j] = __fadd2_rn(__ffma2_rn((j == 0) ? prev : p[j - 1], mneg1, p[j]), dref[j]);
      const bool real = this->real(j);
      const float q = real ? fmaf(d[j].x, d[j].x, d[j].y * d[j].y) : 1.f;
      const float rinv = rsqrtf(q);
      const float dd = fmaf(q, rinv, -l0);
      fr[j] = real ? fmaf(k3m * dd, dd, km) * dd * rinv : 0.f;
    }
    // the next lane's first link (the one after this lane's last mass)
    float2 dn;
    dn.x = __shfl_down_sync(mask, d[0].x, 1, G);
    dn.y = __shfl_down_sync(mask, d[0].y, 1, G);
    float frn = __shfl_down_sync(mask, fr[0], 1, G);
    if (lg == G - 1) frn = 0.f;
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      float2 a = __ffma2_rn(v[j], cneg, grav);
      a = __ffma2_rn(make_float2(-fr[j], -fr[j]), d[j], a);
      const float fo = (j + 1 < FL) ? fr[j + 1] : frn;
      a = __ffma2_rn(make_float2(fo, fo), (j + 1 < FL) ? d[j + 1] : dn, a);
      if (ctrl(j)) a = __fadd2_rn(a, um);
      acc[j] = real(j) ? a : make_float2(0.f, 0.f);
    }
  }
  __device__ __forceinline__ void step(float* xs, const float* u) const {
    float2* p = reinterpret_cast<float2*>(xs);
    float2* v = p + FL;
    const float2 um = make_float2(u[0] * mass_inv, u[1] * mass_inv);
    float2 ap[FL], av[FL], tp[FL], tv[FL], acc[FL];
    accel(p, v, um, acc);
#pragma unroll
    for (int i = 0; i < FL; ++i) {
      ap[i] = v[i];
      av[i] = acc[i];
      tp[i] = __ffma2_rn(hh2, v[i], p[i]);
      tv[i] = __ffma2_rn(hh2, acc[i], v[i]);
    }
    accel(tp, tv, um, acc);
#pragma unroll
    for (int i = 0; i < FL; ++i) {
      ap[i] = __ffma2_rn(two, tv[i], ap[i]);
      av[i] = __ffma2_rn(two, acc[i], av[i]);
      tp[i] = __ffma2_rn(hh2, tv[i], p[i]);
      tv[i] = __ffma2_rn(hh2, acc[i], v[i]);
    }
    accel(tp, tv, um, acc);
#pragma unroll
    for (int i = 0; i < FL; ++i) {
      ap[i] = __ffma2_rn(two, tv[i], ap[i]);
      av[i] = __ffma2_rn(two, acc[i], av[i]);
      tp[i] = __ffma2_rn(hh, tv[i], p[i]);
      tv[i] = __ffma2_rn(hh, acc[i], v[i]);
    }
    accel(tp, tv, um, acc);
#pragma unroll
    for (int i = 0; i < FL; ++i) {
      p[i] = __ffma2_rn(hh6, __fadd2_rn(ap[i], tv[i]), p[i]);
      v[i] = __ffma2_rn(hh6, __fadd2_rn(av[i], acc[i]), v[i]);
    }
  }
  template <class E>
  __device__ __forceinline__ void rows(const float* x, const float* u, bool terminal, E& emit) const {
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      const int i = mass(j);
      const bool real = this->real(j);
      const int r0 = real ? 2 * (i - 1) : 0;
      const float px = pref_local ? pref[2 * j] : pref[2 * G * j];
      const float py = pref_local ? pref[2 * j + 1] : pref[2 * G * j + 1];
      emit.pair(j, r0, x[2 * j] - px, x[2 * j + 1] - py, real);
    }
    const bool urow = !terminal && lg == 0;
    emit.pair(FL, 2 * F, 0.1f * u[0], 0.1f * u[1], urow);
  }
};

template <typename T>
__device__ __forceinline__ T group_sum(T v, int G, unsigned mask) {
  for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// k_samples for groups.  Every lane of a group emits its rows in the same
// order and the partner group emits the same rows, so the difference is taken
// row by row with one xor-shuffle per emitted row.
template <typename T, typename S, int FL, int G, int FX = 0>
__global__ void __launch_bounds__(256, 2) k_samples_group(RollArgs a) {
  constexpr int PAIRS = 256 / (2 * G);
  const int2 bm = a.bmap[blockIdx.x];
  const InstDesc I = a.inst[bm.x];
  if (a.st[bm.x].status != 0) return;
  // Shared: U, s (n each), then the nominal residual and the target positions
  // in a group-interleaved layout, so that the 2G lanes of a pair read 2G
  // consecutive words (lane lg's mass slot j at [2G j + 2 lg], the controls
  // after the SL mass slots of a stage):
  //   sR[k RS + 2G j + 2 lg + c] = r[k rps + 2 (lg FL + j) + c],
  //   sR[k RS + 2 SL + c]        = r[k rps + 2F + c],   sRef likewise, zero-padded.
  constexpr int SL = G * FL;      // mass slots of a rollout group
  constexpr int RS = 2 * SL + 2;  // interleaved words per stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sS = sU + I.n;
  T* sR = sS + I.n;
  T* sRef = sR + (int64_t)(I.N + 1) * RS;
  const T* rg = reinterpret_cast<const T*>(a.r) + I.o_R;
  const int rps = 2 * I.F + 2;
  for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
    sU[j] = (T)a.U[I.o_U + j];
    sS[j] = (T)a.s[I.o_U + j];
  }
  for (int idx = threadIdx.x; idx < I.nR; idx += blockDim.x) {
    const int k = idx / rps, i = idx - k * rps, q = i >> 1;
    const int w = i < 2 * I.F ? (q % FL) * 2 * G + 2 * (q / FL) + (i & 1) : 2 * SL + (i - 2 * I.F);
    sR[k * RS + w] = rg[idx];
  }
  // targets (FP32 model: their offsets from the initial positions)
  constexpr bool REL = ChainGroup<T, FL, G, FX>::kRelative;
  for (int idx = threadIdx.x; idx < 2 * SL; idx += blockDim.x) {
    const int q = idx >> 1;
    sRef[(q % FL) * 2 * G + 2 * (q / FL) + (idx & 1)] =
        q < I.F ? (T)(a.xref[I.o_xref + idx] - (REL ? a.x0[I.o_x0 + idx] : 0.0)) : (T)0;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const bool plus = (lane & G) == 0;
  const int m = bm.y * PAIRS + (int)(threadIdx.x / (2 * G));
  const bool active = m < I.Kp;
  const T sign = plus ? (T)1 : (T)-1;
  // every lane of a block works on one instance with one horizon, so whole
  // warps stay converged and shuffles use the full mask
  ChainGroup<T, FL, G, FX> md(a.cs, I.F, lg, 0xffffffffu);
  const T uf_t = friction_threshold<T>(a.cs);
  md.pref = sRef + 2 * lg;
  md.set_reference(a.x0 + I.o_x0);
  alignas(16) T x[4 * FL];
#pragma unroll
  for (int j = 0; j < FL; ++j) {
    const int i = md.mass(j);
    const bool real = i <= I.F;
    const bool pos = real && !REL;  // FP32: deviations from the initial positions start at 0
    x[2 * j] = pos ? (T)a.x0[I.o_x0 + 2 * (i - 1)] : (T)0;
    x[2 * j + 1] = pos ? (T)a.x0[I.o_x0 + 2 * (i - 1) + 1] : (T)0;
    x[2 * FL + 2 * j] = real ? (T)a.x0[I.o_x0 + 2 * I.F + 2 * (i - 1)] : (T)0;
    x[2 * FL + 2 * j + 1] = real ? (T)a.x0[I.o_x0 + 2 * I.F + 2 * (i - 1) + 1] : (T)0;
  }
  S* dR = reinterpret_cast<S*>(a.dR) + I.o_dR;
  S* Wm = reinterpret_cast<S*>(a.W) + I.o_W;
  uint32_t* W2b = a.W2 ? a.W2 + I.o_W2 : nullptr;
  Acc<T> cost, eacc;
  const uint32_t mm = active ? (uint32_t)m : 0u;
  // Per-row difference emitter: the + group owns row r0 and the - group row
  // r0 + 1 of each (x, y) pair, so both halves of the rollout pair store one
  // difference per pair of rows (e is then the sum of both halves' partial
  // sums).  csum and esum are plain per-stage partial sums, folded into the
  // compensated accumulators once per stage.  Every lane shuffles.
  struct Em {
    S* dR;
    const T* r;  // interleaved nominal residual at the stage's first word
    int ldK, m, base, own_w, ctl_w;
    int nrows;   // rows of dR (bounds-check build)
    bool active, plus;
    T sign, csum, esum;
    __device__ __forceinline__ void pair(int slot, int r0, T v0, T v1, bool valid) {
      const T give = plus ? v1 : v0;  // the row the other half owns
      const T got = __shfl_xor_sync(0xffffffffu, give, G);
      if (!valid) return;
      csum += v0 * v0;
      csum += v1 * v1;
      const T own = plus ? v0 : v1;
      const int row = base + r0 + (plus ? 0 : 1);
      const T d = sign * (own - got) * (T)0.5;
      if (active && GNM_IN(row, nrows)) put(dR + (int64_t)row * ldK + m, d);
      esum += d * r[slot < FL ? 2 * G * slot + own_w : ctl_w];
    }
  } em{dR, sR, I.ldK, m, 0, 2 * lg + (plus ? 0 : 1), 2 * SL + (plus ? 0 : 1), I.nR, active, plus, sign, (T)0, (T)0};
  // The 2G lanes of a pair draw the normals of 2G consecutive steps at once
  // (lane l of the pair: Philox call q = k + l) and hand them round by shuffle.
  // Sigma points (Method E): pair m perturbs control m alone, by sqrt(n) s_m.
  const int pl = lane & (2 * G - 1);
  const bool sigma_pts = a.cs.sampling != 0;
  const T sqrtn = sqrt((T)I.n);
  T na0 = (T)0, na1 = (T)0;
  for (int k = 0; k < I.N; ++k) {
    T z0, z1;
    if (sigma_pts) {
      z0 = (2 * k == m) ? sqrtn : (T)0;
      z1 = (2 * k + 1 == m) ? sqrtn : (T)0;
    } else {
      if (k % (2 * G) == 0)
        box_muller(noise_words(a.cs.seed, (uint32_t)(bm.x + a.cs.inst_base), a.it, mm, (uint32_t)(k + pl)), na0, na1);
      z0 = __shfl_sync(0xffffffffu, na0, k % (2 * G), 2 * G);
      z1 = __shfl_sync(0xffffffffu, na1, k % (2 * G), 2 * G);
    }
    const T w0 = sS[2 * k] * z0, w1 = sS[2 * k + 1] * z1;
    const T u[2] = {sU[2 * k] + sign * w0, sU[2 * k + 1] + sign * w1};
    if (active && plus && lg == 0 && GNM_IN(2 * k + 1, I.n)) {
      put_w(Wm, W2b, I.ldK, 2 * k, m, w0);
      put_w(Wm, W2b, I.ldK, 2 * k + 1, m, w1);
    }
    em.base = k * rps;
    em.r = sR + k * RS;
    em.csum = (T)0;
    em.esum = (T)0;
    md.rows(x, u, false, em);
    cost.add(em.csum);
    eacc.add(em.esum);
    {
      T ua[2];
      dead_zone<T, 2>(u, ua, uf_t);
      md.step(x, ua);
    }
  }
  em.base = I.N * rps;
  em.r = sR + I.N * RS;
  em.csum = (T)0;
  em.esum = (T)0;
  {
    const T u0[2] = {(T)0, (T)0};
    md.rows(x, u0, true, em);
  }
  cost.add(em.csum);
  eacc.add(em.esum);
  // reduce over the group; exchange with the partner group
  const double Cself = 0.5 * group_sum(cost.value(), G, 0xffffffffu);
  double ev = group_sum(eacc.value(), G, 0xffffffffu);
  const double Cother = __shfl_xor_sync(0xffffffffu, Cself, G);
  const double evo = __shfl_xor_sync(0xffffffffu, ev, G);  // every lane shuffles
  ev = ev + evo;  // the two halves of the pair each hold half of the rows' terms
  const bool ok = isfinite(Cself) && isfinite(Cother) && isfinite(ev);
  if (active && lg == 0 && GNM_IN(m, I.Kp)) {
    a.C[I.o_C + 2 * m + (plus ? 0 : 1)] = Cself;
    if (plus) a.e[I.o_C / 2 + m] = ok ? ev : 0.0;
  }
  if (active && plus && !ok) {  // dropped pair: its columns leave P and S
    const int rows = I.N * rps + 2 * I.F;
    for (int row = lg; row < rows; row += G) put(dR + (int64_t)row * I.ldK + m, (T)0);
    for (int j = lg; j < I.n; j += G) put_w(Wm, W2b, I.ldK, j, m, (T)0);
  }
}

// Line search / nominal / FP64 cost for groups: one group per (instance, candidate).
template <typename T, int FL, int G, int FX = 0>
__global__ void __launch_bounds__(256) k_line_group(RollArgs a) {
  const int gid = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
  const int lg = threadIdx.x & (G - 1);
  const int ncand = a.mode == 0 ? a.ncand : 1;
  const bool valid = gid < a.count * ncand;
  const int b = a.list[valid ? gid / ncand : 0];
  const int j = valid ? gid % ncand : 0;
  const InstDesc I = a.inst[b];
  // whole groups leave together (lanes of a group share gid and b)
  if (!valid) return;
  if (a.mode != 2 && a.st[b].status != 0) return;
  double alpha = 0.0;
  if (a.mode == 0) {
    alpha = 1.0;
    for (int q = 0; q < j; ++q) alpha *= a.cs.gamma;
  }
  // groups of one warp may run different instances (different horizons):
  // every shuffle is confined to this group's lanes
  const unsigned gmask = ((G == 32) ? 0xffffffffu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
  ChainGroup<T, FL, G, FX> md(a.cs, I.F, lg, gmask);
  const T uf_t = friction_threshold<T>(a.cs);
  // targets and initial positions: the FP32 model keeps positions relative
  // to the initial ones (and the targets as offsets from them)
  constexpr bool REL = ChainGroup<T, FL, G, FX>::kRelative;
  T ref[2 * FL];
#pragma unroll
  for (int q = 0; q < FL; ++q) {
    const int i = md.mass(q);
    const bool real = i <= I.F;
    const int o = 2 * (i - 1);
    ref[2 * q] = real ? (T)(a.xref[I.o_xref + o] - (REL ? a.x0[I.o_x0 + o] : 0.0)) : (T)0;
    ref[2 * q + 1] = real ? (T)(a.xref[I.o_xref + o + 1] - (REL ? a.x0[I.o_x0 + o + 1] : 0.0)) : (T)0;
  }
  md.pref = ref;
  md.pref_local = true;
  md.set_reference(a.x0 + I.o_x0);
  alignas(16) T x[4 * FL];
#pragma unroll
  for (int q = 0; q < FL; ++q) {
    const int i = md.mass(q);
    const bool real = i <= I.F;
    const bool pos = real && !REL;
    x[2 * q] = pos ? (T)a.x0[I.o_x0 + 2 * (i - 1)] : (T)0;
    x[2 * q + 1] = pos ? (T)a.x0[I.o_x0 + 2 * (i - 1) + 1] : (T)0;
    x[2 * FL + 2 * q] = real ? (T)a.x0[I.o_x0 + 2 * I.F + 2 * (i - 1)] : (T)0;
    x[2 * FL + 2 * q + 1] = real ? (T)a.x0[I.o_x0 + 2 * I.F + 2 * (i - 1) + 1] : (T)0;
  }
  T* out = nullptr;
  if (a.mode == 0) out = reinterpret_cast<T*>(a.RL) + I.o_RL + (int64_t)j * I.nR;
  if (a.mode == 1) out = const_cast<T*>(reinterpret_cast<const T*>(a.r)) + I.o_R;
  struct Em {
    T* out;
    int base;
    T csum;
    int nrows;  // rows of the residual (bounds-check build)
    __device__ __forceinline__ void operator()(int row_local, T v, bool valid) {
      if (!valid) return;
      csum += v * v;
      if (out && GNM_IN(base + row_local, nrows)) out[base + row_local] = v;
    }
    __device__ __forceinline__ void pair(int, int r0, T v0, T v1, bool valid) {
      (*this)(r0, v0, valid);
      (*this)(r0 + 1, v1, valid);
    }
  } em{out, 0, (T)0, I.nR};
  Acc<T> cost;
  const double* U = a.U + I.o_U;
  const double* D = a.delta + I.o_U;
  const int rps = 2 * I.F + 2;
  // Staged controls (FP32 candidates): the group's lanes form U + alpha delta
  // for steps lg, lg + G, ... in FP64 once, so the FP64 work of a warp
  // instruction covers G steps instead of one (GB300's FP64 pipe issues one
  // instruction per warp per 64 cycles whatever the active lanes).
  extern __shared__ __align__(16) unsigned char line_smem[];
  float2* su = reinterpret_cast<float2*>(line_smem) + (int64_t)(threadIdx.x / G) * a.nmax;
  if (a.pre) {
    for (int k = lg; k < I.N; k += G) {
      const double v0 = (a.mode == 0) ? U[2 * k] + alpha * D[2 * k] : U[2 * k];
      const double v1 = (a.mode == 0) ? U[2 * k + 1] + alpha * D[2 * k + 1] : U[2 * k + 1];
      su[k] = make_float2((float)v0, (float)v1);
    }
    __syncwarp(gmask);
  }
  for (int k = 0; k < I.N; ++k) {
    T u[2];
    if (a.pre) {
      const float2 v = su[k];
      u[0] = (T)v.x;
      u[1] = (T)v.y;
    } else {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int q = 2 * k + c;
        u[c] = (a.mode == 0) ? (T)(U[q] + alpha * D[q]) : (T)U[q];
      }
    }
    em.base = k * rps;
    em.csum = (T)0;
    md.rows(x, u, false, em);
    cost.add(em.csum);
    {
      T ua[2];
      dead_zone<T, 2>(u, ua, uf_t);
      md.step(x, ua);
    }
  }
  em.base = I.N * rps;
  em.csum = (T)0;
  {
    const T u0[2] = {(T)0, (T)0};
    md.rows(x, u0, true, em);
  }
  cost.add(em.csum);
  const double C = 0.5 * group_sum(cost.value(), G, gmask);
  if (lg == 0) {
    if (a.mode == 0) a.Cl[(int64_t)b * (kMaxL + 1) + j] = C;
    if (a.mode == 1) {
      a.st[b].C_nom = C;
      a.st[b].C_init = C;
    }
    if (a.mode == 2) a.Cout[b] = C;
  }
}

}  // namespace gnm
