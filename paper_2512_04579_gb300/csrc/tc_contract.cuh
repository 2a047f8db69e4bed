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

// One batched NT GEMM per instance: D[i][j] = sum_k A[i][k] B[j][k] with A
// rows a_row0.., B rows b_row0.. of tensor map `map` (and, for the three-pass
// TF32 split, remainder rows lo_off further down), k from column x0 over nkb
// k-blocks; the output goes to the launch's first (out_sel 0) or second array.
struct TcJob {
  int32_t inst, map;
  int32_t a_row0, b_row0, lo_off;
  int32_t M, Nc, nkb;
  int64_t out_off;
  int32_t ldc, x0, out_sel, pad;
};

struct TcPlan {
  CUtensorMap* d_maps = nullptr;  // [contraction maps (one per instance); Gram maps]
  TcJob* d_jobs = nullptr;        // same order as the maps
  int4* d_tiles_c = nullptr;      // (job, m tile, n tile, -) of the contraction
  int4* d_tiles_g = nullptr;      // ... of the Gram product
  int2* d_rows = nullptr;         // (instance, row) of the TF32 split
  float* d_G = nullptr;           // Gram operands [Ph; Pl] per instance (P^T columns, then S columns)
  int64_t* d_goff = nullptr;
  int* d_gld = nullptr;
  int ntiles_c = 0, ntiles_g = 0, nrows = 0;
  int smem = 0;
  int bf16 = 1;
  int* d_err = nullptr;           // set to 1 when a bounded wait ran out
  std::vector<void*> allocs;
};

// dRW: the combined per-instance [nR + n][ldK] operand block (BF16 when bf16,
// FP32 otherwise); P: the FP32 [P^T | S] array.  Builds tensor maps, jobs and
// tile lists, and allocates the Gram operand blocks.
gnmppi_status tc_plan_create(const std::vector<InstDesc>& desc, void* dRW, void* P, int bf16, cudaStream_t stream,
                             TcPlan* plan, std::string& err);

// [P^T | S] = W^T [dR | W] into P (FP32).
cudaError_t tc_contract_launch(const TcPlan& plan, const InstState* d_st, float* P, cudaStream_t stream);

// A = P^T P and, for instances in LSQ mode, S2 = S S^T (FP64 outputs) from
// three TF32 passes over the split of [P^T | S], in one launch.
cudaError_t tc_gram_launch(const TcPlan& plan, const InstDesc* d_desc, const InstState* d_st, const float* P, double* A,
                           double* S2, cudaStream_t stream);

}  // namespace gnm
