// FP32 instantiation of the rollout kernels (FP32 storage of dR and W).
#include "launch.cuh"
namespace gnm {
GNM_DEFINE_LAUNCHERS(launchers_f32, float, float)
GNM_CHECK_ACCESSOR(check_count_rollout_f32)
}
