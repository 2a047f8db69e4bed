// Group-per-rollout chain kernels (FP64).
#include "launch.cuh"
#include "rollout_group.cuh"

namespace gnm {
namespace {
template <typename T, typename S, int FL, int G>
cudaError_t prep(int smem) {
  return cudaFuncSetAttribute(k_samples_group<T, S, FL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <typename T, typename S, int FL, int G>
void samp(const RollArgs& a, int nb, int smem, cudaStream_t s) {
  k_samples_group<T, S, FL, G><<<nb, 256, smem, s>>>(a);
}
template <typename T, typename S, int FL, int G>
void fill_group(Launchers* o) {
  o->prepare = &prep<T, S, FL, G>;
  o->samples = &samp<T, S, FL, G>;
  o->line = &launch_line_group<T, FL, G>;
  o->cost64 = &launch_line_group<double, FL, G>;
  o->pairs_per_block = 256 / (2 * G);
  o->antithetic_only = 1;
  o->slots = G * FL;
}
}  // namespace

bool group_launchers_f64(int F, Launchers* o) {
  const int G = F <= 32 ? 4 : 8;
  const int FL = (F + G - 1) / G;
  if (F < 17 || F > 64) return false;
  switch (G * 16 + FL) {
    case 4 * 16 + 5: fill_group<double, double, 5, 4>(o); return true;
    case 4 * 16 + 6: fill_group<double, double, 6, 4>(o); return true;
    case 4 * 16 + 7: fill_group<double, double, 7, 4>(o); return true;
    case 4 * 16 + 8: fill_group<double, double, 8, 4>(o); return true;
    case 8 * 16 + 5: fill_group<double, double, 5, 8>(o); return true;
    case 8 * 16 + 6: fill_group<double, double, 6, 8>(o); return true;
    case 8 * 16 + 7: fill_group<double, double, 7, 8>(o); return true;
    case 8 * 16 + 8: fill_group<double, double, 8, 8>(o); return true;
    default: return false;
  }
}

GNM_CHECK_ACCESSOR(check_count_group_f64)

}  // namespace gnm
