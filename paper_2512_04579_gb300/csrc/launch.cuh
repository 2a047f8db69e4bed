// launch.cuh -- host-side launch table of the model-templated rollout kernels.
// Internal; one table per rollout precision (rollout_{f64,f32}.cu).
#pragma once
#include "rollout_group.cuh"

namespace gnm {

struct Launchers {
  cudaError_t (*prepare)(int smem);  // opt the sample kernel into `smem` bytes of shared memory
  void (*samples)(const RollArgs&, int nblocks, int smem, cudaStream_t);
  void (*line)(const RollArgs&, int ncand_total, cudaStream_t);   // one rollout per candidate
  void (*cost64)(const RollArgs&, int ncand_total, cudaStream_t);
  int pairs_per_block = 0;     // antithetic pairs per sample CTA (0: use the thread-per-rollout defaults)
  int antithetic_only = 0;     // group kernels support antithetic sampling only
  int slots = 0;               // group kernels: mass slots G * FL of the interleaved shared layout
};

// key: chain -> free masses F; linear -> nx * 16 + nu; pendulum -> 0.
bool launchers_f64(int dyn, int key, Launchers* out);
bool launchers_f32(int dyn, int key, Launchers* out);
// chains of 17..64 free masses: a group of 4 or 8 lanes per rollout
bool group_launchers_f64(int F, Launchers* out);
bool group_launchers_f32(int F, Launchers* out);

template <class Model, typename T, typename S>
void launch_samples(const RollArgs& a, int nb, int smem, cudaStream_t s) {
  if (a.cs.antithetic)
    k_samples<Model, T, S, true><<<nb, 128, smem, s>>>(a);
  else
    k_samples<Model, T, S, false><<<nb, 128, smem, s>>>(a);
}
template <class Model, typename T, typename S>
cudaError_t prepare_samples(int smem) {
  cudaError_t e = cudaFuncSetAttribute(k_samples<Model, T, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_samples<Model, T, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <class Model, typename T>
void launch_line(const RollArgs& a, int nthreads, cudaStream_t s) {
  if (nthreads > 0) k_line<Model, T><<<(nthreads + 127) / 128, 128, 0, s>>>(a);
}

template <class M32, class M64, typename T, typename S>
void fill(Launchers* o) {
  o->prepare = &prepare_samples<M32, T, S>;
  o->samples = &launch_samples<M32, T, S>;
  o->line = &launch_line<M32, T>;
  o->cost64 = &launch_line<M64, double>;
}

// Line search and FP64 cost of a chain with a group of G lanes per candidate
// rollout: one rollout per thread leaves a few warps per SM running a long
// serial chain of RK4 steps; split over G lanes, each lane's chain is ~G times
// shorter (same rows and costs, see k_line_group).  Measured at 256 chain
// instances (16 candidates each): M = 10 0.18 / 0.127 / 0.096 / 0.105 ms with
// 1 / 4 / 8 / 16 lanes per candidate, M = 16 0.152 / 0.094 / 0.107 ms with 4 / 8 / 16.
template <typename T, int FL, int G, int FX = 0>
void launch_line_group(const RollArgs& a, int ncand_total, cudaStream_t s) {
  const long lanes = (long)ncand_total * G;
  if (lanes <= 0) return;
  // FP32 candidates stage their controls U + alpha delta (formed in FP64,
  // lane-parallel over the steps) in shared memory when they fit the default
  // 48 KB; longer horizons form them per step
  RollArgs b = a;
  const size_t smem = (size_t)(256 / G) * (size_t)a.nmax * sizeof(float2);
  b.pre = (sizeof(T) == 4 && a.mode != 2 && smem <= 48 * 1024) ? 1 : 0;
  k_line_group<T, FL, G, FX><<<(unsigned)((lanes + 255) / 256), 256, b.pre ? smem : 0, s>>>(b);
}
template <typename T, typename S, int F>
void fill_chain(Launchers* o) {
  fill<Chain<T, F>, Chain<double, F>, T, S>(o);
  if constexpr (F >= 5) {
    constexpr int G = 8, FL = (F + G - 1) / G;
    o->line = &launch_line_group<T, FL, G>;
    o->cost64 = &launch_line_group<double, FL, G>;
  }
}

#define GNM_DEFINE_LAUNCHERS(NAME, T, S)                                              \
  bool NAME(int dyn, int key, Launchers* o) {                                         \
    switch (dyn) {                                                                    \
      case kPendulum:                                                                 \
        fill<Pendulum<T>, Pendulum<double>, T, S>(o);                                 \
        return true;                                                                  \
      case kChain:                                                                    \
        switch (key) {                                                                \
          GNM_CHAIN_CASE(T, S, 1) GNM_CHAIN_CASE(T, S, 2) GNM_CHAIN_CASE(T, S, 3)     \
          GNM_CHAIN_CASE(T, S, 4) GNM_CHAIN_CASE(T, S, 5) GNM_CHAIN_CASE(T, S, 6)     \
          GNM_CHAIN_CASE(T, S, 7) GNM_CHAIN_CASE(T, S, 8) GNM_CHAIN_CASE(T, S, 9)     \
          GNM_CHAIN_CASE(T, S, 10) GNM_CHAIN_CASE(T, S, 11) GNM_CHAIN_CASE(T, S, 12)  \
          GNM_CHAIN_CASE(T, S, 13) GNM_CHAIN_CASE(T, S, 14) GNM_CHAIN_CASE(T, S, 15)  \
          GNM_CHAIN_CASE(T, S, 16)                                                    \
          default: return false;                                                      \
        }                                                                             \
      case kRosenbrock:                                                               \
        fill<TestFun<T, kRosenbrock>, TestFun<double, kRosenbrock>, T, S>(o);         \
        return true;                                                                  \
      case kRastrigin:                                                                \
        fill<TestFun<T, kRastrigin>, TestFun<double, kRastrigin>, T, S>(o);           \
        return true;                                                                  \
      case kHeaviside:                                                                \
        fill<TestFun<T, kHeaviside>, TestFun<double, kHeaviside>, T, S>(o);           \
        return true;                                                                  \
      case kLinear:                                                                   \
        switch (key) {                                                                \
          GNM_LIN_CASE(T, S, 2, 1) GNM_LIN_CASE(T, S, 2, 2) GNM_LIN_CASE(T, S, 4, 1)  \
          GNM_LIN_CASE(T, S, 4, 2) GNM_LIN_CASE(T, S, 1, 1)                           \
          default: return false;                                                      \
        }                                                                             \
      default:                                                                        \
        return false;                                                                 \
    }                                                                                 \
  }
#define GNM_CHAIN_CASE(T, S, F) \
  case F:                       \
    fill_chain<T, S, F>(o);     \
    return true;
#define GNM_LIN_CASE(T, S, X, U) \
  case X * 16 + U:               \
    fill<Linear<T, X, U>, Linear<double, X, U>, T, S>(o); \
    return true;

}  // namespace gnm
