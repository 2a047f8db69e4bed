// tc_contract.cu -- batched NT GEMMs on the sm_103a tensor cores:
//  (1) the Jacobian-reconstruction contraction; for every instance
//      D = W^T [dR | W]^T-rows, i.e.
//   P^T[i][j] = sum_m W_m[i] dR_m[j]   (P = sum_m dR_m W_m^T, Eq. 7 of arXiv 2512.04579)
//   S[i][k]   = sum_m W_m[i] W_m[k]
// with the sample index m as the reduction dimension.  dR and W of an instance
// are stored as one [nR + n][ldK] block (sample-contiguous rows), so one TMA
// tensor map per instance covers both operands: the A tile is rows nR + i of
// the block, the B tile rows j.  One CTA computes a (128 or 256) x 256 output
// tile -- two 128-row sub-tiles when the instance has more than 128 unknowns,
// so that each B tile is streamed from L2 once for both:
//   warp 0 lane 0  issues TMA loads into a 3-stage shared-memory ring,
//   warp 1 lane 0  issues tcgen05.mma (M=128, N <= 256, K=16 BF16 / K=8 TF32)
//                  per sub-tile into its own 256-column TMEM accumulator,
//   warps 0-3      read TMEM back (tcgen05.ld 32x32b) and store FP32 rows.
//  (2) the Gram product A = P^T P of Eq. 9 in FP32-level accuracy from three
//      TF32 passes, A ~ Ph Ph^T + Ph Pl^T + Pl Ph^T with P^T = Ph + Pl split into
//      a TF32 head and its FP32 remainder (k_split_tf32 writes [Ph; Pl] rows;
//      one 128 x 256 tile per CTA, a 2-stage ring of head + remainder blocks),
//      and in the same launch S2 = S S^T for the scaled LSQ system: the S
//      columns sit in the same split rows from a 32-aligned column on.
// Both use the same kernel, driven by per-instance job descriptors.
// Every mbarrier wait is bounded by the global timer; a wait that runs out
// sets the plan's error word and the CTA winds down without a trap.
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_contract.cuh"

namespace gnm {

namespace {

constexpr int BM = 128, BN = 256;
constexpr int ROW_BYTES = 128;  // one k-block of a row: 64 BF16 or 32 FP32 values
constexpr int A_BYTES = BM * ROW_BYTES;
constexpr int B_BYTES = BN * ROW_BYTES;
constexpr int RING_BYTES = 4 * (A_BYTES + B_BYTES);  // 192 KB of operand ring
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
// n_mma: the tile's MMA width, a multiple of 16 in [16, BN] (narrower for the
// last column tile of a job, so no MMA work goes to columns that are dropped).
template <bool BF16>
__device__ __forceinline__ uint32_t idesc(int n_mma) {
  const uint32_t fmt = BF16 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n_mma >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
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

// D[i][j] = sum_k A[i][k] B[j][k] for one 128 x 256 tile of one job.  SPLIT3:
// A and B each have a head block and a remainder block lo_off rows below, and
// the tile accumulates head*head + head*rem + rem*head.
template <bool BF16, bool SPLIT3, typename TOut>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const CUtensorMap* __restrict__ maps, const TcJob* __restrict__ jobs,
                                                    const InstState* __restrict__ st, const int4* __restrict__ tiles,
                                                    TOut* __restrict__ D, TOut* __restrict__ D2,
                                                    int* __restrict__ err) {
  constexpr int KBLK = BF16 ? 64 : 32;   // elements per k-block
  constexpr int KSTEP = BF16 ? 16 : 8;   // elements per MMA
  constexpr int NSUB = KBLK / KSTEP;     // MMAs per k-block and operand pair (4)
  constexpr int PARTS = SPLIT3 ? 2 : 1;  // head (+ remainder) blocks per operand
  constexpr int MTMAX = SPLIT3 ? 1 : 2;  // 128-row sub-tiles of A per tile (each its own accumulator)
  constexpr int STAGE_BYTES = PARTS * (MTMAX * A_BYTES + B_BYTES);
  constexpr int STAGES = RING_BYTES / STAGE_BYTES;
  constexpr uint32_t TCOLS = MTMAX * TMEM_COLS;
  const int4 tl = tiles[blockIdx.x];
  const TcJob J = jobs[tl.x];
  // tl.w: sub-tiles of this tile (1, or 2 when the job has more than 128 rows),
  // so every B tile is streamed once for up to 256 output rows
  const int mt = SPLIT3 ? 1 : tl.w;
  const int row_org = tl.y * mt * BM;
  const uint32_t tx_bytes = (uint32_t)(PARTS * (mt * A_BYTES + B_BYTES));
  if (st[J.inst].status != 0) return;  // uniform over the CTA, before any allocation
  const int nkb = J.nkb;
  const CUtensorMap* map = maps + J.map;

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
                 "r"(TCOLS)
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
      mbar_expect_tx(full, tx_bytes);
      const uint32_t a_dst = su32(base + s * STAGE_BYTES);
      const uint32_t b_dst = a_dst + PARTS * MTMAX * A_BYTES;
      const int x = J.x0 + kb * KBLK;
#pragma unroll
      for (int p = 0; p < PARTS; ++p) {
        const int off = p * J.lo_off;
        for (int q = 0; q < mt; ++q)
          tma_load(a_dst + (p * MTMAX + q) * A_BYTES, map, full, x, J.a_row0 + off + row_org + q * BM);
        tma_load(b_dst + p * B_BYTES, map, full, x, J.b_row0 + off + tl.z * BN);
        tma_load(b_dst + p * B_BYTES + BM * ROW_BYTES, map, full, x, J.b_row0 + off + tl.z * BN + BM);
      }
      ++issued;
    }
    // every copy this thread issued has landed before the CTA may exit
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(su32(bars + kb % STAGES), (kb / STAGES) & 1, abort, false);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const int ncols = min(BN, J.Nc - tl.z * BN);  // columns of this tile that are kept
    const uint32_t id = idesc<BF16>(min(BN, (ncols + 15) / 16 * 16));
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (!mbar_wait(su32(bars + s), round & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = su32(base + s * STAGE_BYTES);
      const uint32_t b0 = a0 + PARTS * MTMAX * A_BYTES;
#pragma unroll
      for (int k = 0; k < NSUB; ++k) {
        // sub-tile q accumulates into TMEM columns [256 q, 256 q + 256)
        for (int q = 0; q < mt; ++q)
          mma<BF16>(tmem + (uint32_t)(q * TMEM_COLS), sdesc(a0 + q * A_BYTES + k * 32), sdesc(b0 + k * 32), id,
                    (kb > 0 || k > 0) ? 1u : 0u);
        if (SPLIT3) {
          mma<BF16>(tmem, sdesc(a0 + k * 32), sdesc(b0 + B_BYTES + k * 32), id, 1u);
          mma<BF16>(tmem, sdesc(a0 + A_BYTES + k * 32), sdesc(b0 + k * 32), id, 1u);
        }
      }
      mma_commit(su32(bars + STAGES + s));  // frees the stage once these MMAs have read it
    }
    mma_commit(done);  // accumulator complete (or every issued MMA retired, on abort)
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> shared -> coalesced rows of D
  // Once `done` fires every stage has been consumed, so the operand ring is
  // free: each warp transposes its 32 x 32 slices through a padded staging
  // block and writes whole rows (lane = column) instead of one column of 32
  // rows per store.
  const bool ok = mbar_wait(done, 0, abort, false);
  tc_fence_after();
  // tcgen05.ld is warp-collective: the whole warp takes the same branch
  if (__all_sync(0xffffffffu, ok && !*abort)) {
    TOut* stg = reinterpret_cast<TOut*>(base) + warp * 32 * 33;
    TOut* out = (J.out_sel ? D2 : D) + J.out_off;
#pragma unroll 1
    for (int sub = 0; sub < mt; ++sub) {
    const int row0 = row_org + sub * BM + warp * 32;
#pragma unroll 1
    for (int c = 0; c < BN / 32 && tl.z * BN + c * 32 < J.Nc; ++c) {  // uniform: kept 32-column chunks
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sub * TMEM_COLS + c * 32), v);
#pragma unroll
      for (int q = 0; q < 32; ++q) stg[lane * 33 + q] = (TOut)__uint_as_float(v[q]);
      __syncwarp();
      const int col = tl.z * BN + c * 32 + lane;
      if (col < J.Nc) {
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr)
          if (row0 + rr < J.M) out[(int64_t)(row0 + rr) * J.ldc + col] = stg[rr * 33 + lane];
      }
      __syncwarp();
    }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

// [Ph; Pl] rows of the Gram operand: Ph = [P^T | S] rounded to TF32
// (cvt.rna), Pl = [P^T | S] - Ph (exact in FP32).  The P^T columns go to
// [0, nR), the S columns (LSQ mode) to [nRp, nRp + n) with nRp = nR rounded
// up to a k-block; the gap stays zero.  One CTA per instance row.
__global__ void __launch_bounds__(256) k_split_tf32(const InstDesc* __restrict__ inst, const InstState* __restrict__ st,
                                                    const int2* __restrict__ rows, const float* __restrict__ P,
                                                    float* __restrict__ G, const int64_t* __restrict__ g_off,
                                                    const int* __restrict__ g_ld) {
  const int2 rb = rows[blockIdx.x];  // (instance, row)
  if (st[rb.x].status != 0) return;
  const InstDesc I = inst[rb.x];
  const float* src = P + I.o_P + (int64_t)rb.y * I.ldP;
  float* hi = G + g_off[rb.x] + (int64_t)rb.y * g_ld[rb.x];
  float* lo = hi + (int64_t)I.n * g_ld[rb.x];
  const int nRp = (I.nR + 31) / 32 * 32;
  const int ncol = I.nR + (I.lsq ? I.n : 0);
  for (int k = threadIdx.x; k < ncol; k += blockDim.x) {
    const float x = src[k];
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float hf = __uint_as_float(h);
    const int c = k < I.nR ? k : nRp + (k - I.nR);
    hi[c] = hf;
    lo[c] = x - hf;
  }
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 get_encode(std::string& err) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    err = "cuTensorMapEncodeTiled is not available";
    return nullptr;
  }
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

// Rank-2 tensor map over rows of `cols` elements (row stride ld elements),
// box = one 128-byte k-block x 128 rows, 128-byte swizzle, zero fill outside.
static bool encode_rows(PFN_cuTensorMapEncodeTiled_v12000 encode, CUtensorMap* m, void* gaddr, bool bf16, int64_t cols,
                        int64_t ld, int64_t rows) {
  const size_t esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
  cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / esz), (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  return encode(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, gaddr, dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename P>
static bool plan_alloc(TcPlan* plan, P** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) return false;
  plan->allocs.push_back((void*)*p);
  return true;
}

gnmppi_status tc_plan_create(const std::vector<InstDesc>& desc, void* dRW, void* P, int bf16, cudaStream_t stream,
                             TcPlan* plan, std::string& err) {
  plan->bf16 = bf16;
  auto encode = get_encode(err);
  if (!encode) return GNMPPI_E_CUDA;
  const size_t esz = bf16 ? 2 : 4;
  const int kblk = bf16 ? 64 : 32;
  const int nb = (int)desc.size();
  // Gram operand blocks [Ph; Pl], rows of ldG = nR rounded to 32 floats plus,
  // in LSQ mode, n rounded to 32 floats for the S columns
  std::vector<int64_t> g_off(nb);
  std::vector<int> g_ld(nb);
  int64_t g_total = 0;
  for (int b = 0; b < nb; ++b) {
    g_ld[b] = (int)((desc[b].nR + 31) / 32 * 32) + (desc[b].lsq ? (int)((desc[b].n + 31) / 32 * 32) : 0);
    g_off[b] = g_total;
    g_total += 2 * (int64_t)desc[b].n * g_ld[b];
  }
  if (!plan_alloc(plan, &plan->d_G, 4 * (size_t)std::max<int64_t>(g_total, 4))) {
    err = "cudaMalloc failed for the Gram operands";
    return GNMPPI_E_NOMEM;
  }
  std::vector<CUtensorMap> maps(2 * (size_t)nb);
  std::vector<TcJob> jobs(3 * (size_t)nb);
  std::vector<int4> tc, tg;
  std::vector<int2> rows;
  for (int b = 0; b < nb; ++b) {
    const InstDesc& d = desc[b];
    if (d.ldK % kblk != 0) {
      err = "sample padding is not a multiple of the k-block";
      return GNMPPI_E_ARG;
    }
    // contraction: one map over the instance's [dR; W] block
    if (!encode_rows(encode, &maps[b], reinterpret_cast<char*>(dRW) + esz * (size_t)d.o_dR, bf16, d.ldK, d.ldK,
                     d.nR + d.n)) {
      err = "cuTensorMapEncodeTiled failed (contraction, instance " + std::to_string(b) + ")";
      return GNMPPI_E_CUDA;
    }
    TcJob& jc = jobs[b];
    jc.inst = b;
    jc.map = b;
    jc.a_row0 = d.nR;
    jc.b_row0 = 0;
    jc.lo_off = 0;
    jc.M = d.n;
    jc.Nc = d.nR + d.n;
    jc.nkb = d.ldK / kblk;
    jc.out_off = d.o_P;
    jc.ldc = d.ldP;
    jc.x0 = 0;
    jc.out_sel = 0;
    const int mt = d.n > BM ? 2 : 1;  // up to 256 rows per tile: each B tile streamed once
    for (int i = 0; i < (d.n + mt * BM - 1) / (mt * BM); ++i)
      for (int j = 0; j < (d.nR + d.n + BN - 1) / BN; ++j) tc.push_back(make_int4(b, i, j, mt));
    // Gram: one FP32 map over [Ph; Pl] (2n rows, ldG columns)
    if (!encode_rows(encode, &maps[nb + b], plan->d_G + g_off[b], false, g_ld[b], g_ld[b], 2 * (int64_t)d.n)) {
      err = "cuTensorMapEncodeTiled failed (Gram, instance " + std::to_string(b) + ")";
      return GNMPPI_E_CUDA;
    }
    TcJob& jg = jobs[nb + b];
    jg.inst = b;
    jg.map = nb + b;
    jg.a_row0 = 0;
    jg.b_row0 = 0;
    jg.lo_off = d.n;
    jg.M = d.n;
    jg.Nc = d.n;
    jg.nkb = (d.nR + 31) / 32;
    jg.out_off = d.o_nn;
    jg.ldc = d.n;
    jg.x0 = 0;
    jg.out_sel = 0;
    for (int i = 0; i < (d.n + BM - 1) / BM; ++i)
      for (int j = 0; j < (d.n + BN - 1) / BN; ++j) tg.push_back(make_int4(nb + b, i, j, 1));
    // S2 = S S^T over the S columns of the same split rows (LSQ mode)
    TcJob& js = jobs[2 * nb + b];
    js = jg;
    js.x0 = (d.nR + 31) / 32 * 32;
    js.nkb = (d.n + 31) / 32;
    js.out_sel = 1;
    if (d.lsq)
      for (int i = 0; i < (d.n + BM - 1) / BM; ++i)
        for (int j = 0; j < (d.n + BN - 1) / BN; ++j) tg.push_back(make_int4(2 * nb + b, i, j, 1));
    for (int r = 0; r < d.n; ++r) rows.push_back(make_int2(b, r));
  }
  if (!plan_alloc(plan, &plan->d_maps, sizeof(CUtensorMap) * maps.size()) ||
      !plan_alloc(plan, &plan->d_jobs, sizeof(TcJob) * jobs.size()) ||
      !plan_alloc(plan, &plan->d_tiles_c, sizeof(int4) * std::max<size_t>(1, tc.size())) ||
      !plan_alloc(plan, &plan->d_tiles_g, sizeof(int4) * std::max<size_t>(1, tg.size())) ||
      !plan_alloc(plan, &plan->d_rows, sizeof(int2) * std::max<size_t>(1, rows.size())) ||
      !plan_alloc(plan, &plan->d_goff, sizeof(int64_t) * (size_t)nb) ||
      !plan_alloc(plan, &plan->d_gld, sizeof(int) * (size_t)nb) || !plan_alloc(plan, &plan->d_err, sizeof(int))) {
    err = "cudaMalloc failed for the tensor-core plan";
    return GNMPPI_E_NOMEM;
  }
  plan->ntiles_c = (int)tc.size();
  plan->ntiles_g = (int)tg.size();
  plan->nrows = (int)rows.size();
  bool ok = cudaMemcpyAsync(plan->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                            stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_jobs, jobs.data(), sizeof(TcJob) * jobs.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_tiles_c, tc.data(), sizeof(int4) * tc.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_tiles_g, tg.data(), sizeof(int4) * tg.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_rows, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_goff, g_off.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_gld, g_ld.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, stream) == cudaSuccess;
  ok = ok && cudaMemsetAsync(plan->d_G, 0, 4 * (size_t)std::max<int64_t>(g_total, 4), stream) == cudaSuccess;
  ok = ok && cudaMemsetAsync(plan->d_err, 0, sizeof(int), stream) == cudaSuccess;
  if (!ok) {
    err = "copying the tensor-core plan failed";
    return GNMPPI_E_CUDA;
  }
  plan->smem = RING_BYTES + 1024 + 256;
  cudaError_t e = bf16 ? cudaFuncSetAttribute(k_gemm_tc<true, false, float>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem)
                       : cudaFuncSetAttribute(k_gemm_tc<false, false, float>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gemm_tc<false, true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem);
  if (e != cudaSuccess) {
    err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return GNMPPI_E_CUDA;
  }
  (void)P;
  return GNMPPI_OK;
}

cudaError_t tc_contract_launch(const TcPlan& plan, const InstState* d_st, float* P, cudaStream_t stream) {
  if (plan.ntiles_c == 0) return cudaSuccess;
  if (plan.bf16)
    k_gemm_tc<true, false, float><<<plan.ntiles_c, 128, plan.smem, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                             plan.d_tiles_c, P, P, plan.d_err);
  else
    k_gemm_tc<false, false, float><<<plan.ntiles_c, 128, plan.smem, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                              plan.d_tiles_c, P, P, plan.d_err);
  return cudaGetLastError();
}

cudaError_t tc_gram_launch(const TcPlan& plan, const InstDesc* d_desc, const InstState* d_st, const float* P, double* A,
                           double* S2, cudaStream_t stream) {
  if (plan.ntiles_g == 0) return cudaSuccess;
  k_split_tf32<<<plan.nrows, 256, 0, stream>>>(d_desc, d_st, plan.d_rows, P, plan.d_G, plan.d_goff, plan.d_gld);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gemm_tc<false, true, double><<<plan.ntiles_g, 128, plan.smem, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                            plan.d_tiles_g, A, S2, plan.d_err);
  return cudaGetLastError();
}

}  // namespace gnm
