// tc_contract.cuh -- host interface of the tensor-core Jacobian-reconstruction
// contraction (Eq. 7 of arXiv 2512.04579): [P^T | S] = W^T [dR | W] per
// instance on tcgen05 (BF16 or TF32 operands, FP32 accumulation in TMEM),
// operands staged by TMA.  Internal.
#pragma once
#include <cuda.h>

#include <string>
#include <vector>

#include "../../include/gnmppi.h"
#include "common.cuh"

namespace gnm {

struct TcPlan {
  CUtensorMap* d_maps = nullptr;  // one tensor map per instance over its [dR; W] block
  int4* d_tiles = nullptr;        // (instance, m tile, n tile, -)
  int ntiles = 0;
  int smem = 0;
  int bf16 = 1;
  int* d_err = nullptr;           // set to 1 when a bounded wait ran out
  std::vector<void*> allocs;
};

// dRW: the combined per-instance [nR + n][ldK] operand block (storage type
// BF16 when bf16, FP32 otherwise).  Builds tensor maps and the tile list.
gnmppi_status tc_plan_create(const std::vector<InstDesc>& desc, void* dRW, int bf16, cudaStream_t stream,
                             TcPlan* plan, std::string& err);

// P: FP32 [P^T | S] output.  Returns the launch error, if any.
cudaError_t tc_contract_launch(const TcPlan& plan, const InstDesc* d_desc, const InstState* d_st, float* P,
                               cudaStream_t stream);

}  // namespace gnm
