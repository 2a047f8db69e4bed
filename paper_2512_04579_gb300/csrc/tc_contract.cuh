// tc_contract.cuh -- host interface of the tensor-core Jacobian-reconstruction
// contraction (Eq. 7 of arXiv 2512.04579): [P^T | S] = W^T [dR | W] per
// instance on tcgen05 from FP32 operands staged by TMA and split in shared
// memory into TF32 or BF16 head + remainder parts (three passes, FP32
// accumulation in TMEM).  Internal.
#pragma once
#include <cuda.h>

#include <string>
#include <vector>

#include "../../include/gnmppi.h"
#include "common.cuh"

namespace gnm {

// One batched NT GEMM per instance: D[i][j] = sum_k A[i][k] B[j][k] with A
// rows a_row0.., B rows b_row0.. of tensor map `map`, k from column x0 over
// nkb k-blocks, M x Nc outputs with row stride ldc from out_off of the
// launch's first (out_sel 0: A, or the contraction's [P^T | S]), second (1:
// S2) or chunk array (2: one column chunk of a chunked Gram); output columns >= ccut are
// stored cgap further right (the S block of [P^T | S] starts aligned).
struct TcJob {
  int32_t inst, map;
  int32_t map2, pad0;  // BF16-mode contraction: tensor map of the split W copy (the B rows)
  int32_t a_row0, b_row0;
  int32_t M, Nc, nkb, x0;
  int64_t out_off;
  int32_t ldc, out_sel;
  int32_t ccut, cgap;
};

// One instance whose Gram A = P^T P runs in column chunks: A (at out_off,
// nn = n^2 entries) = sum over the chunks of part[part_off + c nn + i].
struct GramRed {
  int64_t out_off, part_off;
  int64_t nn;
  int32_t chunks, inst;
};

// Columns of P^T summed by one FP32 accumulator of the Gram; longer sums are
// split into chunks whose FP32 results are added with a compensated sum (the
// tensor core's FP32 accumulation error grows with the number of steps).
constexpr int kGramChunkCols = 2048;

struct TcPlan {
  CUtensorMap* d_maps = nullptr;  // per instance: contraction [dR; W]; then P^T columns; then S columns
  TcJob* d_jobs = nullptr;        // same order as the maps (contraction, Gram, S2)
  int4* d_tiles_c = nullptr;      // (job, m tile, n tile, sub-tiles) of the contraction
  int4* d_tiles_c1 = nullptr;     // the same with one A sub-tile per tile (BF16 mode)
  int4* d_tiles_g = nullptr;      // (job, first row, first column, sub-tiles | 4 diagonal) of the Gram products
  int ntiles_c = 0, ntiles_c1 = 0, ntiles_g = 0;
  int smem = 0, smem1 = 0;
  int bf16 = 1;
  float* d_part = nullptr;        // FP32 chunk results of the chunked Grams
  GramRed* d_red = nullptr;       // one record per chunked instance
  int nred = 0;
  int* d_err = nullptr;           // set to 1 when a bounded wait ran out
  std::vector<void*> allocs;
};

// dRW: the combined per-instance FP32 [nR + n][ldK] operand block; W2 (BF16
// mode): W split into BF16 head and remainder by the rollouts, [n][ldK]
// words per instance at InstDesc::o_W2; P: the FP32 [P^T | S] array (S from
// column sP on); bf16 selects the contraction's BF16 passes (otherwise TF32).
// Builds tensor maps, jobs and tile lists.
gnmppi_status tc_plan_create(const std::vector<InstDesc>& desc, void* dRW, const uint32_t* W2, void* P, int bf16,
                             cudaStream_t stream, TcPlan* plan, std::string& err);

// [P^T | S] = W^T [dR | W] into P (FP32).  inject != 0 (tests only): every
// CTA's first MMA-side wait is on a barrier that nothing completes, so it
// runs out after 20 ms, sets the error word and the CTA winds down.
// mt (BF16 mode): A sub-tiles per CTA, 2 (one CTA per SM) or 1 (two per SM).
cudaError_t tc_contract_launch(const TcPlan& plan, const InstState* d_st, float* P, cudaStream_t stream, int inject,
                               int mt);

// A = P^T P and, for instances in LSQ mode, S2 = S S^T (FP64 outputs) from
// three passes over [P^T | S] split in shared memory (BF16 head + remainder
// in BF16 mode, TF32 otherwise), in one launch; where nR exceeds
// kGramChunkCols, A is formed per column chunk and a second launch adds the
// chunks (compensated, into FP64).
cudaError_t tc_gram_launch(const TcPlan& plan, const InstState* d_st, double* A, double* S2, cudaStream_t stream);

}  // namespace gnm
