// FP32 rollouts with BF16 storage of dR and W (tensor-core contraction operands).
#include "launch.cuh"
namespace gnm {
GNM_DEFINE_LAUNCHERS(launchers_bf16, float, __nv_bfloat16)
}
