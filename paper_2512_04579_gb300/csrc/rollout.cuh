// rollout.cuh -- batched RK4 rollouts of the GN-MPPI hot path (arXiv 2512.04579):
//   * k_samples: the K perturbed rollouts of one Algorithm-1 iteration (Sec. 4.1,
//     Eq. 7 sampled as in Method D, antithetic pairs as in Sec. 5), with the
//     residual, cost and Jacobian-reconstruction operands fused into the rollout:
//     each pair writes dR_m = (R(U+W_m) - R(U-W_m))/2 and W_m column-wise into
//     sample-contiguous rows, its two costs C = 0.5||R||^2 (Eq. 2, 4) and
//     e_m = dR_m . r (so that P^T r = W^T e needs no second pass over dR);
//   * k_line: the L step-length candidates of the line search (Eq. 11), the
//     nominal rollout R(U_k), and FP64 cost re-evaluation.
// One thread per rollout; the two rollouts of an antithetic pair sit in
// adjacent lanes and exchange residual rows with one shuffle.  States stay in
// registers (the models are compile-time sized), controls and sampling scales
// are staged through shared memory.  Internal; instantiated per precision.
#pragma once
#include "common.cuh"

namespace gnm {

struct RollArgs {
  const InstDesc* inst;
  InstState* st;
  Consts cs;
  const double* x0;
  const double* xref;
  const double* U;
  const double* s;
  const double* delta;
  const void* r;      // nominal residual [nR] per instance (scalar type)
  void* dR;           // [nR][ldK] storage type
  void* W;            // [n][ldK]  storage type
  uint32_t* W2;       // BF16 mode: W's head/remainder copy [n][ldK] words (else null)
  double* C;          // [Kp][2]
  double* e;          // [Kp]
  void* RL;           // [L][nR] scalar type
  double* Cl;         // [kMaxL + 1] per instance
  double* Cout;       // cost output (mode 2)
  const int2* bmap;   // sample blocks: (instance, chunk)
  const int* list;    // instances of this launch (line / nominal / cost)
  int count;          // entries of list
  int ncand;          // candidates per instance (line search)
  uint32_t it;        // iteration index of the noise stream
  int mode;           // k_line: 0 line search, 1 nominal, 2 FP64 cost only
  int nmax;           // largest horizon N of the handle's instances
  int pre;            // k_line_group: controls staged in dynamic shared memory
                      // (candidates of the CTA x nmax float2), else formed per step
};

// Sample m of W row j, and in the BF16 mode (W2b not null) its split copy.
template <typename S, typename V>
__device__ __forceinline__ void put_w(S* Wm, uint32_t* W2b, int ldK, int j, int m, V w) {
  put(Wm + (int64_t)j * ldK + m, (S)w);
  if constexpr (sizeof(S) == 4) {
    if (W2b) put_w2(reinterpret_cast<uint16_t*>(W2b + (int64_t)j * ldK), m, (float)w);
  }
}

// Models that read a per-instance reference (the chain's target positions)
// get it from a caller-staged copy in the scalar type.
template <class Model>
struct RefSize {
  static constexpr int value = 0;
};
template <typename T, int F>
struct RefSize<Chain<T, F>> {
  static constexpr int value = 2 * F;
};
template <class Model, typename T>
__device__ __forceinline__ void bind_model(Model&, const T*) {}
template <typename T, int F>
__device__ __forceinline__ void bind_model(Chain<T, F>& m, const T* ref) {
  m.pref = ref;
}

template <typename T>
struct StageSum {
  T s = (T)0;
};

// Emitter for the sample kernel: antithetic difference across the pair lanes,
// dR written and e = dR . r accumulated by the lane whose parity matches the
// row.  csum and esum are plain per-stage partial sums, folded into the
// compensated totals once per stage; dR addresses advance by one row of ldK.
template <typename T, typename S, bool ANTI>
struct SampleEmit {
  S* col;        // this sample's column of dR at the stage's first row
  const T* r;    // nominal residual at the stage's first row
  int ldK, par;
  int row0, nrows;  // first row of the stage, rows of dR (bounds-check build)
  bool active;
  T sign, csum, esum;
  __device__ __forceinline__ void operator()(int i, T v) {
    csum += v * v;
    if (ANTI) {
      const T vo = __shfl_xor_sync(0xffffffffu, v, 1);
      if (par == (i & 1)) {
        const T d = sign * (v - vo) * (T)0.5;
        if (active && GNM_IN(row0 + i, nrows)) put(col + (int64_t)i * ldK, d);
        esum += d * r[i];
      }
    } else {
      const T d = v - r[i];
      if (active && GNM_IN(row0 + i, nrows)) put(col + (int64_t)i * ldK, d);
      esum += d * r[i];
    }
  }
  // Rows i and i + 1 (i even) at once: with antithetic pairs each lane of the
  // pair owns one of the two rows (row i + par), so the difference, the dR
  // store and the e update run once per lane without a divergent branch.
  // Same arithmetic, same order per lane as two calls of operator().
  __device__ __forceinline__ void pair(int i, T v0, T v1) {
    if (ANTI) {
      csum += v0 * v0;
      csum += v1 * v1;
      const T give = par ? v0 : v1;  // the row the partner owns
      const T own = par ? v1 : v0;
      const T got = __shfl_xor_sync(0xffffffffu, give, 1);
      const T d = sign * (own - got) * (T)0.5;
      const int row = i + par;
      if (active && GNM_IN(row0 + row, nrows)) put(col + (int64_t)row * ldK, d);
      esum += d * r[row];
    } else {
      (*this)(i, v0);
      (*this)(i + 1, v1);
    }
  }
};

template <class Model, typename T, typename S, bool ANTI>
__global__ void __launch_bounds__(128) k_samples(RollArgs a) {
  constexpr int NX = Model::NX, NU = Model::NU;
  const int2 bm = a.bmap[blockIdx.x];
  const InstDesc I = a.inst[bm.x];
  if (a.st[bm.x].status != 0) return;
  // shared: U, s (n each), the nominal residual r (nR) and the reference, in T
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sS = sU + I.n;
  T* sR = sS + I.n;
  T* sRef = sR + I.nR;
  const T* rg = reinterpret_cast<const T*>(a.r) + I.o_R;
  for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
    sU[j] = (T)a.U[I.o_U + j];
    sS[j] = (T)a.s[I.o_U + j];
  }
  for (int j = threadIdx.x; j < I.nR; j += blockDim.x) sR[j] = rg[j];
  for (int j = threadIdx.x; j < RefSize<Model>::value; j += blockDim.x) sRef[j] = (T)a.xref[I.o_xref + j];
  __syncthreads();

  const int per_block = ANTI ? kPairsPerBlock : kSamplesPerBlock;
  const int local = ANTI ? (threadIdx.x >> 1) : threadIdx.x;
  const int m = bm.y * per_block + local;
  const bool active = m < I.Kp;
  const int par = ANTI ? (threadIdx.x & 1) : 0;
  const T sign = par ? (T)-1 : (T)1;

  Model md(a.cs);
  const T uf_t = friction_threshold<T>(a.cs);
  bind_model(md, (const T*)sRef);
  alignas(16) T x[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) x[i] = (T)a.x0[I.o_x0 + i];

  S* dR = reinterpret_cast<S*>(a.dR) + I.o_dR + m;  // this sample's column
  S* Wm = reinterpret_cast<S*>(a.W) + I.o_W;
  uint32_t* W2b = a.W2 ? a.W2 + I.o_W2 : nullptr;
  Acc<T> cost, eacc;
  SampleEmit<T, S, ANTI> em{dR, sR, I.ldK, par, 0, I.nR, active, sign, (T)0, (T)0};
  const uint32_t mm = active ? (uint32_t)m : 0u;
  const int64_t stage_stride = (int64_t)Model::RPS * I.ldK;
  // Two controls per step (nu = 2) with antithetic pairs: the normals of steps
  // k and k+1 come from Philox calls q = k and q = k + 1; each lane of the pair
  // draws one of the two and the partner's arrives by shuffle.
  constexpr bool SHARE = ANTI && NU == 2;
  // Sigma points (Method E): pair m perturbs control m alone, by sqrt(n) s_m.
  const bool sigma_pts = ANTI && a.cs.sampling != 0;
  const T sqrtn = sqrt((T)I.n);
  int qc = -1;
  T z0 = (T)0, z1 = (T)0, y0 = (T)0, y1 = (T)0;
  for (int k = 0; k < I.N; ++k) {
    T u[NU];
    if (sigma_pts) {
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        const int j = k * NU + c;
        const T w = (j == m) ? sS[j] * sqrtn : (T)0;
        u[c] = sU[j] + sign * w;
        if (active && par == 0 && GNM_IN(j, I.n)) put_w(Wm, W2b, I.ldK, j, m, w);
      }
    } else if (SHARE) {
      if ((k & 1) == 0) {
        T a0, a1;
        box_muller(noise_words(a.cs.seed, (uint32_t)(bm.x + a.cs.inst_base), a.it, mm, (uint32_t)(k + par)), a0, a1);
        const T b0 = __shfl_xor_sync(0xffffffffu, a0, 1);
        const T b1 = __shfl_xor_sync(0xffffffffu, a1, 1);
        z0 = par ? b0 : a0;
        z1 = par ? b1 : a1;
        y0 = par ? a0 : b0;
        y1 = par ? a1 : b1;
      } else {
        z0 = y0;
        z1 = y1;
      }
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        const int j = k * NU + c;
        const T w = sS[j] * (c ? z1 : z0);
        u[c] = sU[j] + sign * w;
        if (active && par == c && GNM_IN(j, I.n)) put_w(Wm, W2b, I.ldK, j, m, w);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        const int j = k * NU + c;
        const int q = j >> 1;
        if (q != qc) {
          box_muller(noise_words(a.cs.seed, (uint32_t)(bm.x + a.cs.inst_base), a.it, mm, (uint32_t)q), z0, z1);
          qc = q;
        }
        const T w = sS[j] * ((j & 1) ? z1 : z0);
        u[c] = sU[j] + sign * w;
        if (active && par == (ANTI ? (j & 1) : 0) && GNM_IN(j, I.n)) put_w(Wm, W2b, I.ldK, j, m, w);
      }
    }
    em.col = dR + k * stage_stride;
    em.r = sR + k * Model::RPS;
    em.row0 = k * Model::RPS;
    em.csum = (T)0;
    em.esum = (T)0;
    md.stage(x, u, em);
    cost.add(em.csum);
    eacc.add(em.esum);
    {
      T ua[Model::NU];
      dead_zone<T, Model::NU>(u, ua, uf_t);
      md.step(x, ua);
    }
  }
  em.col = dR + I.N * stage_stride;
  em.r = sR + I.N * Model::RPS;
  em.row0 = I.N * Model::RPS;
  em.csum = (T)0;
  em.esum = (T)0;
  md.terminal(x, em);
  cost.add(em.csum);
  eacc.add(em.esum);
  dR -= m;

  const double Cself = 0.5 * cost.value();
  double ev = eacc.value();
  double Cother = Cself;
  if (ANTI) {
    Cother = __shfl_xor_sync(0xffffffffu, Cself, 1);
    ev += __shfl_xor_sync(0xffffffffu, ev, 1);
  }
  const bool ok = isfinite(Cself) && isfinite(Cother) && isfinite(ev);
  if (active && GNM_IN(m, I.Kp)) {
    a.C[I.o_C + (ANTI ? 2 * m + par : m)] = Cself;
    if (par == 0) a.e[I.o_C / 2 + m] = ok ? ev : 0.0;
    if (!ok) {  // dropped pair: its columns leave P and S
      const int rows = I.N * Model::RPS + Model::RT;
      for (int row = par; row < rows; row += (ANTI ? 2 : 1)) put(dR + (int64_t)row * I.ldK + m, (T)0);
      for (int j = par; j < I.n; j += (ANTI ? 2 : 1)) put_w(Wm, W2b, I.ldK, j, m, (T)0);
    }
  }
}

template <typename T>
struct LineEmit {
  T* out;  // nullptr: cost only
  int base;
  T csum;
  int nrows;  // rows of the residual (bounds-check build)
  __device__ __forceinline__ void operator()(int i, T v) {
    csum += v * v;
    if (out && GNM_IN(base + i, nrows)) out[base + i] = v;
  }
  __device__ __forceinline__ void pair(int i, T v0, T v1) {
    (*this)(i, v0);
    (*this)(i + 1, v1);
  }
};

// One thread per (instance, candidate).  mode 0: candidate j rolls out
// U + gamma^j delta; mode 1: the nominal U; mode 2: the nominal U in FP64 into
// Cout.  Instances whose status is not OK are skipped.
template <class Model, typename T>
__global__ void __launch_bounds__(128) k_line(RollArgs a) {
  constexpr int NX = Model::NX, NU = Model::NU;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ncand = a.mode == 0 ? a.ncand : 1;
  if (t >= a.count * ncand) return;
  const int b = a.list[t / ncand];
  const int j = t % ncand;
  const InstDesc I = a.inst[b];
  if (a.mode != 2 && a.st[b].status != 0) return;
  double alpha = 0.0;
  if (a.mode == 0) {
    alpha = 1.0;
    for (int q = 0; q < j; ++q) alpha *= a.cs.gamma;
  }
  Model md(a.cs);
  const T uf_t = friction_threshold<T>(a.cs);
  alignas(8) T ref[RefSize<Model>::value > 0 ? RefSize<Model>::value : 1];  // read as float2 pairs
#pragma unroll
  for (int i = 0; i < RefSize<Model>::value; ++i) ref[i] = (T)a.xref[I.o_xref + i];
  bind_model(md, (const T*)ref);
  alignas(16) T x[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) x[i] = (T)a.x0[I.o_x0 + i];
  T* out = nullptr;
  if (a.mode == 0) out = reinterpret_cast<T*>(a.RL) + I.o_RL + (int64_t)j * I.nR;
  if (a.mode == 1) out = const_cast<T*>(reinterpret_cast<const T*>(a.r)) + I.o_R;
  LineEmit<T> em{out, 0, (T)0, I.nR};
  Acc<T> cost;
  const double* U = a.U + I.o_U;
  const double* D = a.delta + I.o_U;
  for (int k = 0; k < I.N; ++k) {
    T u[NU];
#pragma unroll
    for (int c = 0; c < NU; ++c) {
      const int q = k * NU + c;
      u[c] = (a.mode == 0) ? (T)(U[q] + alpha * D[q]) : (T)U[q];
    }
    em.base = k * Model::RPS;
    em.csum = (T)0;
    md.stage(x, u, em);
    cost.add(em.csum);
    {
      T ua[Model::NU];
      dead_zone<T, Model::NU>(u, ua, uf_t);
      md.step(x, ua);
    }
  }
  em.base = I.N * Model::RPS;
  em.csum = (T)0;
  md.terminal(x, em);
  cost.add(em.csum);
  const double C = 0.5 * cost.value();
  if (a.mode == 0) a.Cl[(int64_t)b * (kMaxL + 1) + j] = C;
  if (a.mode == 1) {
    a.st[b].C_nom = C;
    a.st[b].C_init = C;
  }
  if (a.mode == 2) a.Cout[b] = C;
}

}  // namespace gnm
