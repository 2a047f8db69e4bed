// tc_contract.cu -- Jacobian-reconstruction contraction on the sm_103a tensor
// cores.  For every instance: D = W^T [dR | W]^T-rows, i.e.
//   P^T[i][j] = sum_m W_m[i] dR_m[j]   (P = sum_m dR_m W_m^T, Eq. 7 of arXiv 2512.04579)
//   S[i][k]   = sum_m W_m[i] W_m[k]
// with the sample index m as the reduction dimension.  dR and W of an instance
// are stored as one [nR + n][ldK] block (sample-contiguous rows), so one TMA
// tensor map per instance covers both operands: the A tile is rows nR + i of
// the block, the B tile rows j.  One CTA computes a 128 x 256 output tile:
//   warp 0 lane 0  issues TMA loads into a 4-stage shared-memory ring,
//   warp 1 lane 0  issues tcgen05.mma (M=128, N=256, K=16 BF16 / K=8 TF32)
//                  into a 256-column TMEM accumulator,
//   warps 0-3      read TMEM back (tcgen05.ld 32x32b) and store FP32 rows.
// Every mbarrier wait is bounded by the global timer; a wait that runs out
// sets the plan's error word and the CTA winds down without a trap.
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_contract.cuh"

namespace gnm {

namespace {

constexpr int BM = 128, BN = 256, STAGES = 4;
constexpr int ROW_BYTES = 128;  // one k-block of a row: 64 BF16 or 32 FP32 values
constexpr int A_BYTES = BM * ROW_BYTES;
constexpr int B_BYTES = BN * ROW_BYTES;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity; gives up after WAIT_NS or when
// another role of the CTA has aborted (check_abort).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort, bool check_abort) {
  const unsigned long long t0 = gtimer();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(a, parity)) return true;
    if (check_abort && *abort) return false;
    if ((i & 255u) == 255u && gtimer() - t0 > WAIT_NS) return false;
  }
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, uint32_t mbar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(mbar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16 for
// kind::f16, 2 = TF32 for kind::tf32), both K-major, N >> 3 and M >> 4.
template <bool BF16>
__device__ __forceinline__ uint32_t idesc() {
  const uint32_t fmt = BF16 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define GNM_R32(x) "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]), \
                   "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]),       \
                   "=r"(x[15]), "=r"(x[16]), "=r"(x[17]), "=r"(x[18]), "=r"(x[19]), "=r"(x[20]), "=r"(x[21]),     \
                   "=r"(x[22]), "=r"(x[23]), "=r"(x[24]), "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]),     \
                   "=r"(x[29]), "=r"(x[30]), "=r"(x[31])

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : GNM_R32(v)
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool BF16>
__global__ void __launch_bounds__(128, 1) k_contract_tc(const CUtensorMap* __restrict__ maps,
                                                        const InstDesc* __restrict__ inst,
                                                        const InstState* __restrict__ st,
                                                        const int4* __restrict__ tiles, float* __restrict__ P,
                                                        int* __restrict__ err) {
  constexpr int KBLK = BF16 ? 64 : 32;   // elements per k-block
  constexpr int KSTEP = BF16 ? 16 : 8;   // elements per MMA
  constexpr int NSUB = KBLK / KSTEP;     // MMAs per k-block (4)
  const int4 tl = tiles[blockIdx.x];
  const int b = tl.x;
  if (st[b].status != 0) return;  // uniform over the CTA, before any allocation
  const InstDesc I = inst[b];
  const int nkb = I.ldK / KBLK;
  const CUtensorMap* map = maps + b;

  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  // bars[0..S): full, bars[S..2S): empty, bars[2S]: done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * STAGES + 1; ++s) mbar_init(su32(bars + s), 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t done = su32(bars + 2 * STAGES);

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(su32(bars + STAGES + s), (round - 1) & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      const uint32_t full = su32(bars + s);
      mbar_expect_tx(full, STAGE_BYTES);
      const uint32_t a_dst = su32(base + s * STAGE_BYTES);
      const uint32_t b_dst = a_dst + A_BYTES;
      const int x = kb * KBLK;
      tma_load(a_dst, map, full, x, I.nR + tl.y * BM);
      tma_load(b_dst, map, full, x, tl.z * BN);
      tma_load(b_dst + BM * ROW_BYTES, map, full, x, tl.z * BN + BM);
      ++issued;
    }
    // every copy this thread issued has landed before the CTA may exit
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(su32(bars + kb % STAGES), (kb / STAGES) & 1, abort, false);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t id = idesc<BF16>();
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (!mbar_wait(su32(bars + s), round & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = su32(base + s * STAGE_BYTES);
      const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
      for (int k = 0; k < NSUB; ++k)
        mma<BF16>(tmem, sdesc(a0 + k * 32), sdesc(b0 + k * 32), id, (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(su32(bars + STAGES + s));  // frees the stage once these MMAs have read it
    }
    mma_commit(done);  // accumulator complete (or every issued MMA retired, on abort)
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> global (rows of P^T | S)
  const bool ok = mbar_wait(done, 0, abort, false);
  tc_fence_after();
  // tcgen05.ld is warp-collective: the whole warp takes the same branch
  if (__all_sync(0xffffffffu, ok && !*abort)) {
    const int row = tl.y * BM + warp * 32 + lane;
    const int ncols = I.nR + I.n;
    float* out = P + I.o_P + (int64_t)row * I.ldP;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
      const int col0 = tl.z * BN + c * 32;
      if (row < I.n) {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (col0 + q < ncols) out[col0 + q] = __uint_as_float(v[q]);
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

gnmppi_status tc_plan_create(const std::vector<InstDesc>& desc, void* dRW, int bf16, cudaStream_t stream,
                             TcPlan* plan, std::string& err) {
  plan->bf16 = bf16;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    err = "cuTensorMapEncodeTiled is not available";
    return GNMPPI_E_CUDA;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const size_t esz = bf16 ? 2 : 4;
  const int kblk = bf16 ? 64 : 32;
  std::vector<CUtensorMap> maps(desc.size());
  std::vector<int4> tiles;
  for (size_t b = 0; b < desc.size(); ++b) {
    const InstDesc& d = desc[b];
    if (d.ldK % kblk != 0) {
      err = "sample padding is not a multiple of the k-block";
      return GNMPPI_E_ARG;
    }
    char* gaddr = reinterpret_cast<char*>(dRW) + esz * (size_t)d.o_dR;
    cuuint64_t dims[2] = {(cuuint64_t)d.ldK, (cuuint64_t)(d.nR + d.n)};
    cuuint64_t strides[1] = {(cuuint64_t)d.ldK * esz};
    cuuint32_t box[2] = {(cuuint32_t)kblk, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[b], bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, gaddr,
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled failed for instance " + std::to_string(b) + " (code " + std::to_string((int)r) + ")";
      return GNMPPI_E_CUDA;
    }
    for (int i = 0; i < (d.n + BM - 1) / BM; ++i)
      for (int j = 0; j < (d.nR + d.n + BN - 1) / BN; ++j) tiles.push_back(make_int4((int)b, i, j, 0));
  }
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    plan->allocs.push_back(*p);
    return true;
  };
  if (!alloc((void**)&plan->d_maps, sizeof(CUtensorMap) * maps.size()) ||
      !alloc((void**)&plan->d_tiles, sizeof(int4) * std::max<size_t>(1, tiles.size())) ||
      !alloc((void**)&plan->d_err, sizeof(int))) {
    err = "cudaMalloc failed for the tensor-core plan";
    return GNMPPI_E_NOMEM;
  }
  plan->ntiles = (int)tiles.size();
  if (cudaMemcpyAsync(plan->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(plan->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, stream) !=
          cudaSuccess ||
      cudaMemsetAsync(plan->d_err, 0, sizeof(int), stream) != cudaSuccess) {
    err = "copying the tensor-core plan failed";
    return GNMPPI_E_CUDA;
  }
  plan->smem = STAGES * STAGE_BYTES + 1024 + 256;
  cudaError_t e = bf16 ? cudaFuncSetAttribute(k_contract_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              plan->smem)
                       : cudaFuncSetAttribute(k_contract_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              plan->smem);
  if (e != cudaSuccess) {
    err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return GNMPPI_E_CUDA;
  }
  return GNMPPI_OK;
}

cudaError_t tc_contract_launch(const TcPlan& plan, const InstDesc* d_desc, const InstState* d_st, float* P,
                               cudaStream_t stream) {
  if (plan.ntiles == 0) return cudaSuccess;
  if (plan.bf16)
    k_contract_tc<true><<<plan.ntiles, 128, plan.smem, stream>>>(plan.d_maps, d_desc, d_st, plan.d_tiles, P, plan.d_err);
  else
    k_contract_tc<false><<<plan.ntiles, 128, plan.smem, stream>>>(plan.d_maps, d_desc, d_st, plan.d_tiles, P,
                                                                 plan.d_err);
  return cudaGetLastError();
}

}  // namespace gnm
