// FP64 instantiation of the rollout kernels (parity mode).
#include "launch.cuh"
namespace gnm {
GNM_DEFINE_LAUNCHERS(launchers_f64, double, double)
GNM_CHECK_ACCESSOR(check_count_rollout_f64)
}
