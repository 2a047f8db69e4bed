// Group-per-rollout chain kernels (FP32).
#include "launch.cuh"
#include "rollout_group.cuh"

namespace gnm {
namespace {
template <typename T, typename S, int FL, int G, int FX>
cudaError_t prep(int smem) {
  return cudaFuncSetAttribute(k_samples_group<T, S, FL, G, FX>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <typename T, typename S, int FL, int G, int FX>
void samp(const RollArgs& a, int nb, int smem, cudaStream_t s) {
  k_samples_group<T, S, FL, G, FX><<<nb, 256, smem, s>>>(a);
}
// FX: the exact free-mass count when the kernel is specialised for it, else 0
template <typename T, typename S, int FL, int G, int FX = 0>
void fill_group(Launchers* o) {
  o->prepare = &prep<T, S, FL, G, FX>;
  o->samples = &samp<T, S, FL, G, FX>;
  o->line = &launch_line_group<T, FL, G, FX>;
  o->cost64 = &launch_line_group<double, FL, G, FX>;
  o->pairs_per_block = 256 / (2 * G);
  o->antithetic_only = 1;
  o->slots = G * FL;
}
}  // namespace

bool group_launchers_f32(int F, Launchers* o) {
  const int G = F <= 32 ? 4 : 8;
  const int FL = (F + G - 1) / G;
  if (F < 17 || F > 64) return false;
  // The chains of 32 and 64 masses.  M = 32: the mass count compiled in
  // (42.5 -> 33.4 ms for 256 instances at N = 200, K = 4096).  M = 64: the
  // sample rollouts stay generic (93.5 ms there; compiled in, 123 ms with
  // eight lanes per rollout and 98 ms with sixteen, though both ran faster
  // than generic at 32 instances).  The line search, one group per candidate,
  // spreads each rollout over twice the lanes of the sample kernel (its launch
  // has only L candidates per instance to run in parallel).
  if (F == 31) {
    fill_group<float, float, 8, 4, 31>(o);
    o->line = &launch_line_group<float, 4, 8, 31>;
    o->cost64 = &launch_line_group<double, 4, 8, 31>;
    return true;
  }
  if (F == 63) {
    fill_group<float, float, 8, 8>(o);
    o->line = &launch_line_group<float, 4, 16, 63>;
    o->cost64 = &launch_line_group<double, 4, 16, 63>;
    return true;
  }
  switch (G * 16 + FL) {
    case 4 * 16 + 5: fill_group<float, float, 5, 4>(o); return true;
    case 4 * 16 + 6: fill_group<float, float, 6, 4>(o); return true;
    case 4 * 16 + 7: fill_group<float, float, 7, 4>(o); return true;
    case 4 * 16 + 8: fill_group<float, float, 8, 4>(o); return true;
    case 8 * 16 + 5: fill_group<float, float, 5, 8>(o); return true;
    case 8 * 16 + 6: fill_group<float, float, 6, 8>(o); return true;
    case 8 * 16 + 7: fill_group<float, float, 7, 8>(o); return true;
    case 8 * 16 + 8: fill_group<float, float, 8, 8>(o); return true;
    default: return false;
  }
}

GNM_CHECK_ACCESSOR(check_count_group_f32)

}  // namespace gnm
