// tc_contract.cu -- batched NT GEMMs on the sm_103a tensor cores:
//  (1) the Jacobian-reconstruction contraction; for every instance
//      D = W^T [dR | W]^T-rows, i.e.
//   P^T[i][j] = sum_m W_m[i] dR_m[j]   (P = sum_m dR_m W_m^T, Eq. 7 of arXiv 2512.04579)
//   S[i][k]   = sum_m W_m[i] W_m[k]
// with the sample index m as the reduction dimension.  dR and W of an instance
// are stored as one [nR + n][ldK] block (sample-contiguous rows), so one TMA
// tensor map per instance covers both operands.  Both reduced-precision modes
// keep FP32-level accuracy (a single TF32 or BF16 pass does not: its operand
// rounding moves the Gauss-Newton step, and the cost after it, by up to
// 1e-3 / 1e-2 at 10^4 residual rows):
//    BF16 mode (k_contract_tc): one CTA computes the products of up to 256
//      rows of the [dR; W] block (two 128-row sub-tiles, each with its own
//      256-column TMEM accumulator) with up to 256 W rows, from three
//      kind::f16 passes per product:
//        warp 0 lane 0  issues TMA loads of 16-value k-blocks into a 6-stage
//                       ring: the FP32 [dR; W] rows, and the W rows from the
//                       rollouts' BF16 head/remainder copy of W,
//        warps 2-5      rewrite each landed FP32 row in place as a BF16
//                       [head | remainder] row (each thread its own rows),
//        warp 1 lane 0  issues tcgen05.mma (M=128, N = the W rows, K=16) per
//                       sub-tile,
//        warps 0-3      read TMEM back (tcgen05.ld 32x32b, one lane per
//                       [P^T | S] column) and store 32 consecutive columns
//                       per warp store (the S columns from column sP on);
//    FP32 mode: the three-pass TF32 kernel of (2) on the FP32 [dR; W] block.
//  (2) k_gram_tc: the Gram product A = P^T P of Eq. 9 in FP32-level accuracy
//      from three passes, A ~ Ph Ph^T + Ph Pl^T + Pl Ph^T with every FP32
//      operand x split into a head h and its remainder x - h, and in the same
//      launch S2 = S S^T for the scaled LSQ system.  FP32 mode: TF32 heads
//      h = rna(x) (remainder exact in FP32), 32-value k-blocks, the remainder
//      beside the head.  BF16 mode: BF16 head and remainder written in place
//      as a [head | remainder] row per 16-value k-block, as in (1), one
//      128-row sub-tile per CTA and two CTAs per SM.  TMA
//      streams the FP32 rows of [P^T | S] straight from the contraction's
//      output; warps 2-5 split each landed stage in shared memory before the
//      MMAs read it.  A
//      diagonal tile takes its A sub-tiles from its own B rows (the operand is
//      the same matrix), each sub-tile's MMAs stop at the diagonal, and the
//      strictly lower 32 x 32 blocks are also stored transposed, so every
//      entry of the symmetric output is written once.
// Every mbarrier wait is bounded by the global timer; a wait that runs out
// sets the plan's error word and the CTA winds down without a trap.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "tc_contract.cuh"
#include "tc_ptx.cuh"

namespace gnm {

namespace {

constexpr int BM = 128, BN = 256;
constexpr int ROW_BYTES = 128;  // one k-block of an FP32 row: 32 values
constexpr int KBLK_F32 = 32;    // Gram and three-pass TF32 k-block (128-byte rows, 128-byte swizzle)
constexpr int KBLK_BF16 = 16;   // BF16-mode contraction k-block (64-byte rows, 64-byte swizzle)
constexpr int A_BYTES = BM * ROW_BYTES;
constexpr int B_BYTES = BN * ROW_BYTES;
constexpr int RING_BYTES = 4 * (A_BYTES + B_BYTES);  // 192 KB of operand ring (every kernel here)
constexpr int TMEM_COLS = 256;

// BF16 heads of two adjacent FP32 values (round to nearest even) and the
// BF16 roundings of their remainders x - head (exact in FP32), each pair
// packed as the 32-bit word a K-major row holds (first value in the low half).
__device__ __forceinline__ void bf16_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Row `row` of a landed 64-byte-swizzled TMA box at p (16 FP32 values, one
// contraction k-block) rewritten in place as a 64-byte BF16 row [16 heads |
// 16 remainders] with the same swizzle (16-byte chunk j of the row at chunk
// j ^ ((row >> 1) & 3)).  The row's four chunks are read before any is
// written and no other row's bytes are touched, so each thread splits its
// own rows without waiting for the others.
__device__ __forceinline__ void split_row_sw64(unsigned char* p, int row) {
  unsigned char* r = p + row * 64;
  const int sw = (row >> 1) & 3;
  float v[16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float4 q = *reinterpret_cast<const float4*>(r + ((c ^ sw) << 4));
    v[4 * c] = q.x;
    v[4 * c + 1] = q.y;
    v[4 * c + 2] = q.z;
    v[4 * c + 3] = q.w;
  }
  uint4 H0, L0, H1, L1;  // heads of values 0-7 and 8-15, remainders likewise
  bf16_split2(v[0], v[1], H0.x, L0.x);
  bf16_split2(v[2], v[3], H0.y, L0.y);
  bf16_split2(v[4], v[5], H0.z, L0.z);
  bf16_split2(v[6], v[7], H0.w, L0.w);
  bf16_split2(v[8], v[9], H1.x, L1.x);
  bf16_split2(v[10], v[11], H1.y, L1.y);
  bf16_split2(v[12], v[13], H1.z, L1.z);
  bf16_split2(v[14], v[15], H1.w, L1.w);
  *reinterpret_cast<uint4*>(r + ((0 ^ sw) << 4)) = H0;
  *reinterpret_cast<uint4*>(r + ((1 ^ sw) << 4)) = H1;
  *reinterpret_cast<uint4*>(r + ((2 ^ sw) << 4)) = L0;
  *reinterpret_cast<uint4*>(r + ((3 ^ sw) << 4)) = L1;
}

// One (128 or 256) x (up to 256) tile of the BF16 mode's contraction: the A
// side is rows a_row0 + i of the instance's [dR; W] block (i < Nc, the
// columns of [P^T | S]), the B side its W rows b_row0 + j (j < M = n), and
// D[i][j] = sum_k A[i][k] B[j][k] is stored transposed, into row j and column
// i of [P^T | S] (columns >= ccut cgap further right): one TMEM lane per
// output column i, so each warp store writes 32 consecutive columns.  TMA
// lands k-blocks of 16 values (64-byte rows, 64-byte swizzle): the FP32 rows
// of up to two 128-row A sub-tiles, which four splitter warps rewrite in
// place as BF16 [head | remainder] rows, and 256 B rows from the rollouts'
// BF16 copy of W, which arrive in that layout already (split once per
// iteration instead of once per tile).  Each product is formed from three
// BF16 MMAs of K = 16 (head x head, head x remainder, remainder x head, the
// remainders 32 bytes into the rows), which keeps FP32-level accuracy (the
// dropped remainder x remainder term is ~2^-18 relative).  192 threads: warp
// 0 lane 0 TMA, warp 1 lane 0 MMA, warps 2-5 split; warps 0-3 read TMEM back.
//
// MT: A sub-tiles per CTA.  MT = 2: 256 A rows, a 6-stage ring of 32 KB, one
// CTA per SM; MT = 1: 128 A rows, a 4-stage ring of 24 KB (96 KB), two CTAs per
// SM, whose pipelines hide each other's load latency (the W rows are then read
// twice as often, from L2).  Same products, same accumulation order per output.
constexpr int kContractThreads = 192;
template <int MT>
__global__ void __launch_bounds__(kContractThreads, 3 - MT) k_contract_tc(const CUtensorMap* __restrict__ maps,
                                                                    const TcJob* __restrict__ jobs,
                                                                    const InstState* __restrict__ st,
                                                                    const int4* __restrict__ tiles,
                                                                    float* __restrict__ D, int* __restrict__ err,
                                                                    int inject) {
  constexpr int KBLK = KBLK_BF16;            // FP32 values per k-block (one 64-byte row)
  constexpr int TILE = BM * 64;              // one landed 128-row box (8 KB)
  constexpr int STAGE_BYTES = (MT + 2) * TILE;  // A sub-tiles, then 256 B rows
  constexpr int STAGES = (MT == 2 ? RING_BYTES : RING_BYTES / 2) / STAGE_BYTES;
  constexpr int SPLITTERS = kContractThreads - 64;
  constexpr uint32_t TCOLS = MT * TMEM_COLS;
  const int4 tl = tiles[blockIdx.x];
  const TcJob J = jobs[tl.x];
  // tl.y: block of MT x 128 A rows, tl.z: block of 256 B rows, tl.w: A sub-tiles (1 or 2)
  const int mt = tl.w;
  const int row_org = tl.y * MT * BM;
  const uint32_t tx_bytes = (uint32_t)((mt + 2) * TILE);
  if (st[J.inst].status != 0) return;  // uniform over the CTA, before any allocation
  const int nkb = J.nkb;
  const CUtensorMap* map = maps + J.map;
  const CUtensorMap* map2 = maps + J.map2;

  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  // bars[0..S): full (TMA landed), [S..2S): split (rows rewritten),
  // [2S..3S): empty (MMAs done with the stage), [3S]: done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(su32(bars + s), 1);
      mbar_init(su32(bars + STAGES + s), SPLITTERS);
      mbar_init(su32(bars + 2 * STAGES + s), 1);
    }
    mbar_init(su32(bars + 3 * STAGES), 1);
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
  const uint32_t done = su32(bars + 3 * STAGES);
  // stage layout: A sub-tile 0, [A sub-tile 1,] B rows 0-127, B rows 128-255 (8 KB each)

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map2) : "memory");
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(su32(bars + 2 * STAGES + s), (round - 1) & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      const uint32_t full = su32(bars + s);
      mbar_expect_tx(full, tx_bytes);
      const uint32_t a_dst = su32(base + s * STAGE_BYTES);
      const uint32_t b_dst = a_dst + MT * TILE;
      const int x = J.x0 + kb * KBLK;
      for (int q = 0; q < mt; ++q) tma_load(a_dst + q * TILE, map, full, x, J.a_row0 + row_org + q * BM);
      // the B rows land already split (the rollouts' BF16 W copy, rows 0..n)
      tma_load(b_dst, map2, full, x, tl.z * BN);
      tma_load(b_dst + TILE, map2, full, x, tl.z * BN + BM);
      ++issued;
    }
    // every copy this thread issued has landed before the CTA may exit
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(su32(bars + kb % STAGES), (kb / STAGES) & 1, abort, false);
  } else if (warp >= 2) {
    // ---------------- splitters: thread t owns row t of every 128-row box
    const int t = threadIdx.x - 64;
    bool alive = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (!mbar_wait(su32(bars + s), round & 1, abort, true)) {
        alive = false;
        break;
      }
      unsigned char* sb = base + s * STAGE_BYTES;
      for (int q = 0; q < mt; ++q) split_row_sw64(sb + q * TILE, t);
      // the generic-proxy writes become visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bars + STAGES + s)) : "memory");
    }
    if (!alive) {
      *abort = 1;
      atomicExch(err, 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const int ncols = min(BN, J.M - tl.z * BN);  // W rows of this tile
    const uint32_t id = idesc<true>(min(BN, (ncols + 15) / 16 * 16));
    if (inject && !mbar_wait(su32(bars + 2 * STAGES), 0, abort, true, INJECT_WAIT_NS)) {
      *abort = 1;
      atomicExch(err, 1);
    }
    for (int kb = 0; kb < nkb && !*abort; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (!mbar_wait(su32(bars + STAGES + s), round & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = su32(base + s * STAGE_BYTES);
      const uint32_t bh = a0 + MT * TILE, bl = bh + 32;
      // sub-tile q accumulates into TMEM columns [256 q, 256 q + 256)
      for (int q = 0; q < mt; ++q) {
        const uint32_t d = tmem + (uint32_t)(q * TMEM_COLS);
        const uint32_t ah = a0 + q * TILE, al = ah + 32;
        mma<true>(d, sdesc<true>(ah), sdesc<true>(bh), id, kb > 0 ? 1u : 0u);
        mma<true>(d, sdesc<true>(ah), sdesc<true>(bl), id, 1u);
        mma<true>(d, sdesc<true>(al), sdesc<true>(bh), id, 1u);
      }
      mma_commit(su32(bars + 2 * STAGES + s));  // frees the stage once these MMAs have read it
    }
    mma_commit(done);  // accumulator complete (or every issued MMA retired, on abort)
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> rows of [P^T | S]
  // Lane l of warp w holds A row i = row_org + 128 sub + 32 w + l, i.e.
  // output column i; a 32-column TMEM load gives it 32 consecutive output
  // rows j, and each store of the warp covers 32 consecutive columns.
  const bool ok = mbar_wait(done, 0, abort, false);
  tc_fence_after();
  // tcgen05.ld is warp-collective: the whole warp takes the same branch
  if (warp >= 4) {
    // no TMEM lanes of their own
  } else if (__all_sync(0xffffffffu, ok && !*abort)) {
    float* out = D + J.out_off;
    const int jn = min(BN, J.M - tl.z * BN);  // output rows of this tile
#pragma unroll 1
    for (int sub = 0; sub < mt; ++sub) {
      const int i = row_org + sub * BM + warp * 32 + lane;
      const bool live = i < J.Nc;
      const int colw = i < J.ccut ? i : i + J.cgap;
#pragma unroll 1
      for (int c = 0; c * 32 < jn; ++c) {  // uniform over the warp
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sub * TMEM_COLS + c * 32), v);
        const int j0 = tl.z * BN + c * 32;
        if (live) {
#pragma unroll 8
          for (int jj = 0; jj < 32; ++jj)
            if (c * 32 + jj < jn && GNM_IN((int64_t)(j0 + jj) * J.ldc + colw, (int64_t)J.M * J.ldc))
              out[(int64_t)(j0 + jj) * J.ldc + colw] = __uint_as_float(v[jj]);
        }
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

// TF32 head of x: rounded to 10 mantissa bits, to nearest with ties away
// from zero, on the bit pattern (adding half a TF32 unit to the magnitude
// bits carries into the kept bits, the exponent included), then the 13 low
// bits cleared.  Integer pipe work; the remainder x - head is exact in FP32.
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// FP32 bit pattern u widened to the FP64 value it encodes, on the integer
// pipe (GB300's FP64 pipe retires one warp instruction per ~19 cycles per SM,
// so a conversion per output entry there would dominate the Gram's
// epilogue).  IEEE 754 binary32 -> binary64: the sign stays, a normal
// exponent is rebiased by 1023 - 127 = 896, the 23 fraction bits become the
// top of the 52 (the low 3 of them land in the low word's top 3 bits);
// zeros, infinities and NaNs keep their class; subnormals (rare here) take
// the hardware conversion.
__device__ __forceinline__ double widen_f32(uint32_t u) {
  const uint32_t a = u & 0x7FFFFFFFu, sgn = u & 0x80000000u;
  uint32_t hi;
  if (a >= 0x7F800000u) hi = sgn | 0x7FF00000u | ((a & 0x007FFFFFu) >> 3);
  else if (a >= 0x00800000u) hi = sgn | ((a >> 3) + (896u << 20));
  else if (a == 0u) hi = sgn;
  else return (double)__uint_as_float(u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// Splits `n4` float4 of a landed operand block in place: head (TF32) at p,
// remainder at p + delta bytes.  Same positions in both blocks, so the
// 128-byte swizzle of the TMA layout carries over.
__device__ __forceinline__ void split_block(unsigned char* p, int delta, int n4, int t, int nt) {
#pragma unroll 4
  for (int i = t; i < n4; i += nt) {
    float4* hp = reinterpret_cast<float4*>(p) + i;
    const float4 x = *hp;
    float4 h, l;
    h.x = tf32_head(x.x);
    h.y = tf32_head(x.y);
    h.z = tf32_head(x.z);
    h.w = tf32_head(x.w);
    l.x = x.x - h.x;
    l.y = x.y - h.y;
    l.z = x.z - h.z;
    l.w = x.w - h.w;
    *hp = h;
    *reinterpret_cast<float4*>(p + delta + (size_t)i * 16) = l;
  }
}

// One warp's store of a staged 32 x 32 block (stg[r * 33 + c], row r of the
// block in TMEM lane row0 + r, column col_org + 32 c0 + c) into out with row
// stride ldc: the rows, and with mirror also the transposed block.
template <typename T>
__device__ __forceinline__ void store_block(T* out, const T* stg, const TcJob& J, int lane, int row0, int cbase,
                                            bool mirror) {
  const int col = cbase + lane;
  if (col < J.Nc) {
    const int colw = col < J.ccut ? col : col + J.cgap;
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr)
      if (row0 + rr < J.M && GNM_IN((int64_t)(row0 + rr) * J.ldc + colw, (int64_t)J.M * J.ldc))
        out[(int64_t)(row0 + rr) * J.ldc + colw] = stg[rr * 33 + lane];
  }
  if (mirror) {
    const int rowt = row0 + lane;
    if (rowt < J.M) {
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        const int colt = cbase + rr;
        if (colt < J.Nc && GNM_IN((int64_t)colt * J.ldc + rowt, (int64_t)J.M * J.ldc))
          out[(int64_t)colt * J.ldc + rowt] = stg[lane * 33 + rr];
      }
    }
  }
}

// Gram tile of one job: output rows tl.y.., columns tl.z.. (the B rows),
// tl.w = sub-tiles (1 or 2) | 4 if the tile sits on the diagonal.  Per stage
// (one 32-column k-block): B head and remainder (256 rows), and for an
// off-diagonal tile A head and remainder (128 rows).  192 threads: warp 0
// lane 0 TMA, warp 1 lane 0 MMA, warps 2-5 split; warps 0-3 read TMEM back.
// CONTRACT: the same three-pass product for the FP32 mode's contraction
// [P^T | S] = W^T [dR | W] (off-diagonal tiles only, A rows a_row0 + i and B
// rows b_row0 + j of the instance's FP32 [dR; W] map), FP32 output into out0
// with the S columns moved to sP; otherwise A = out0 or S2 in FP64.
constexpr int kGramThreads = 192;
// BF (the BF16 mode's Gram, CONTRACT false only): k-blocks of 16 FP32 values
// (64-byte rows, 64-byte swizzle) split in place row by row into BF16
// [head | remainder] rows, three kind::f16 passes; B rows and (off the
// diagonal) A rows only, no separate remainder area.  Every tile has one
// 128-row sub-tile (256 TMEM columns) and a 96 KB ring (up to 8 stages), so
// two CTAs share an SM and each hides the other's pipeline latency: a
// diagonal tile with two sub-tiles runs as two CTAs (tl.w bit 3 marks the
// second), the first loading only the 128 B rows its MMAs read.  Same
// products in the same order per output as one CTA per diagonal tile
// (0.266 -> 0.215 ms per launch at 256 instances of n = 200).  12 diagonal
// stages of 16 KB in a 192 KB ring measured slower (0.92 against 0.84 ms for
// 64 instances of M = 32).
template <bool CONTRACT, bool BF = false>
__global__ void __launch_bounds__(kGramThreads, BF ? 2 : 1) k_gram_tc(const CUtensorMap* __restrict__ maps, const TcJob* __restrict__ jobs,
                                                    const InstState* __restrict__ st, const int4* __restrict__ tiles,
                                                    void* __restrict__ out0, double* __restrict__ S2,
                                                    float* __restrict__ part,
                                                    int* __restrict__ err, int inject) {
  using TO = typename std::conditional<CONTRACT, float, double>::type;
  static_assert(!(CONTRACT && BF), "the BF16 contraction is k_contract_tc");
  // FP32 elements per k-block; MMAs (TF32 K = 8, BF16 K = 16) per k-block
  constexpr int KBLK = BF ? KBLK_BF16 : 32, NSUB = BF ? 1 : 4;
  constexpr int RB = BF ? 64 : ROW_BYTES;  // bytes of one landed row of a k-block
  constexpr int SPLITTERS = kGramThreads - 64;  // warps 2-5
  constexpr int MAXST = BF ? 8 : 3;
  const int4 tl = tiles[blockIdx.x];
  const TcJob J = jobs[tl.x];
  const int mt = tl.w & 3;
  const bool diag = (tl.w & 4) != 0;
  const int q0 = (tl.w >> 3) & 1;  // BF16: the diagonal tile's second sub-tile alone
  const int row_org = tl.y, col_org = tl.z;
  const int kept = min(BN, J.Nc - col_org);  // output columns of this tile = B rows
  const int kept_b = diag ? min(kept, BM * (q0 + mt)) : kept;  // B rows the MMAs read
  const int nbox = kept_b > BM ? 2 : 1;      // 128-row TMA boxes of B
  // TF32: B head, B remainder (256 rows each) [, A head, A remainder];
  // BF16: 256 B rows [, 128 A rows], each split in place
  constexpr int RING = BF ? RING_BYTES / 2 : RING_BYTES;  // BF16: two CTAs per SM
  const int stage_bytes = BF ? (diag ? nbox * BM * RB : (BN + BM) * RB) : (diag ? 2 * B_BYTES : 2 * (B_BYTES + A_BYTES));
  const int stages = min(MAXST, RING / stage_bytes);  // TF32: 3 (diagonal) or 2; BF16: 8
  const int a_off = BF ? BN * RB : 2 * B_BYTES;              // A rows of an off-diagonal stage
  const uint32_t tx_bytes = (uint32_t)(nbox * BM * RB + (diag ? 0 : BM * RB));
  const uint32_t tcols = mt == 2 ? 2 * TMEM_COLS : TMEM_COLS;
  if (st[J.inst].status != 0) return;  // uniform over the CTA, before any allocation
  const int nkb = J.nkb;
  const CUtensorMap* map = maps + J.map;

  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + RING);
  // bars[0..3): full (TMA landed), [3..6): split (heads and remainders
  // written), [6..9): empty (MMAs done with the stage), [9]: done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * MAXST + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXST; ++s) {
      mbar_init(su32(bars + s), 1);
      mbar_init(su32(bars + MAXST + s), SPLITTERS);
      mbar_init(su32(bars + 2 * MAXST + s), 1);
    }
    mbar_init(su32(bars + 3 * MAXST), 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t done = su32(bars + 3 * MAXST);
  // stage layout: B head [0, 32K), B remainder [32K, 64K), A head, A remainder (off-diagonal)

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % stages, round = kb / stages;
      if (kb >= stages && !mbar_wait(su32(bars + 2 * MAXST + s), (round - 1) & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      const uint32_t full = su32(bars + s);
      mbar_expect_tx(full, tx_bytes);
      const uint32_t b_dst = su32(base + s * stage_bytes);
      const int x = J.x0 + kb * KBLK;
      for (int q = 0; q < nbox; ++q) tma_load(b_dst + q * BM * RB, map, full, x, J.b_row0 + col_org + q * BM);
      if (!diag) tma_load(b_dst + a_off, map, full, x, J.a_row0 + row_org);
      ++issued;
    }
    for (int kb = (issued > stages ? issued - stages : 0); kb < issued; ++kb)
      mbar_wait(su32(bars + kb % stages), (kb / stages) & 1, abort, false);
  } else if (warp >= 2) {
    // ---------------- splitters: head in place, remainder beside it
    const int t = threadIdx.x - 64;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % stages, round = kb / stages;
      if (!mbar_wait(su32(bars + s), round & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      unsigned char* sb = base + s * stage_bytes;
      if constexpr (BF) {
        for (int q = 0; q < nbox; ++q) split_row_sw64(sb, t + q * BM);
        if (!diag) split_row_sw64(sb + a_off, t);
      } else {
        split_block(sb, B_BYTES, nbox * A_BYTES / 16, t, SPLITTERS);
        if (!diag) split_block(sb + 2 * B_BYTES, A_BYTES, A_BYTES / 16, t, SPLITTERS);
      }
      // the generic-proxy writes become visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bars + MAXST + s)) : "memory");
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: three passes (TF32 or BF16) per sub-tile
    uint32_t id[2];
    for (int q = 0; q < 2; ++q) {
      const int need = diag ? min(kept, BM * (q0 + q + 1)) : kept;  // columns up to the diagonal
      id[q] = idesc<BF>(min(BN, (need + 15) / 16 * 16));
    }
    if (inject && !mbar_wait(su32(bars + 2 * MAXST), 0, abort, true, INJECT_WAIT_NS)) {
      *abort = 1;
      atomicExch(err, 1);
    }
    for (int kb = 0; kb < nkb && !*abort; ++kb) {
      const int s = kb % stages, round = kb / stages;
      if (!mbar_wait(su32(bars + MAXST + s), round & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      if constexpr (BF) {
        // [head | remainder] rows: the remainders 32 bytes into each row
        const uint32_t bh = su32(base + s * stage_bytes), bl = bh + 32;
        for (int q = 0; q < mt; ++q) {
          // diagonal: A sub-tile q is B rows [128 q, 128 q + 128)
          const uint32_t ah = diag ? bh + (q0 + q) * BM * RB : bh + a_off, al = ah + 32;
          const uint32_t d = tmem + (uint32_t)(q * TMEM_COLS);
          mma<true>(d, sdesc<true>(ah), sdesc<true>(bh), id[q], kb > 0 ? 1u : 0u);
          mma<true>(d, sdesc<true>(ah), sdesc<true>(bl), id[q], 1u);
          mma<true>(d, sdesc<true>(al), sdesc<true>(bh), id[q], 1u);
        }
      } else {
        const uint32_t bh = su32(base + s * stage_bytes), bl = bh + B_BYTES;
#pragma unroll
        for (int k = 0; k < NSUB; ++k) {
          for (int q = 0; q < mt; ++q) {
            // diagonal: A sub-tile q is B rows [128 q, 128 q + 128)
            const uint32_t ah = diag ? bh + q * A_BYTES : bh + 2 * B_BYTES;
            const uint32_t al = diag ? bl + q * A_BYTES : bh + 2 * B_BYTES + A_BYTES;
            const uint32_t d = tmem + (uint32_t)(q * TMEM_COLS);
            mma<false>(d, sdesc(ah + k * 32), sdesc(bh + k * 32), id[q], (kb > 0 || k > 0) ? 1u : 0u);
            mma<false>(d, sdesc(ah + k * 32), sdesc(bl + k * 32), id[q], 1u);
            mma<false>(d, sdesc(al + k * 32), sdesc(bh + k * 32), id[q], 1u);
          }
        }
      }
      mma_commit(su32(bars + 2 * MAXST + s));
    }
    mma_commit(done);
  }
  __syncwarp();

  // ---------------- epilogue: rows of D, and the transposes of the blocks
  // strictly below the diagonal (whose mirror images no tile computes);
  // warps 0-3, one per 32 TMEM lanes
  const bool ok = mbar_wait(done, 0, abort, false);
  tc_fence_after();
  if (warp >= 4) {
    // no TMEM lanes of their own
  } else if (__all_sync(0xffffffffu, ok && !*abort)) {
    TO* stg = reinterpret_cast<TO*>(base) + warp * 32 * 33;
    TO* out = (CONTRACT ? reinterpret_cast<TO*>(out0)
                        : reinterpret_cast<TO*>(J.out_sel ? S2 : reinterpret_cast<double*>(out0))) + J.out_off;
    // a chunk of a chunked Gram keeps its FP32 accumulators as they are
    const bool fpart = !CONTRACT && J.out_sel == 2;
    float* stgf = reinterpret_cast<float*>(base) + warp * 32 * 33;
    float* outf = fpart ? part + J.out_off : nullptr;
#pragma unroll 1
    for (int sub = 0; sub < mt; ++sub) {
      const int row0 = row_org + (q0 + sub) * BM + warp * 32;
      const int cend = diag ? min(kept, BM * (q0 + sub + 1)) : kept;
#pragma unroll 1
      for (int c = 0; c * 32 < cend; ++c) {  // uniform over the warp
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sub * TMEM_COLS + c * 32), v);
        // strictly lower block of the symmetric Gram: its transpose is stored
        // too (the contraction's output is rectangular and has no mirror image)
        const bool mirror = !CONTRACT && (!diag || c < 4 * (q0 + sub));
        if (fpart) {
#pragma unroll
          for (int q = 0; q < 32; ++q) stgf[lane * 33 + q] = __uint_as_float(v[q]);
          __syncwarp();
          store_block(outf, stgf, J, lane, row0, col_org + c * 32, mirror);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            if constexpr (CONTRACT) stg[lane * 33 + q] = __uint_as_float(v[q]);
            else stg[lane * 33 + q] = widen_f32(v[q]);
          }
          __syncwarp();
          store_block(out, stg, J, lane, row0, col_org + c * 32, mirror);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

}  // namespace

// A of the instances whose Gram runs in column chunks: the sum, in chunk
// order, of the chunks' FP32 tile results (the reduction over nR split so
// that no FP32 accumulator sums more than kGramChunkCols columns).  The sum
// runs in FP32 with Knuth's TwoSum collecting every addition's rounding
// error in a second word, and hi + lo, both widened exactly, is added once
// in FP64: the result is the chunks' sum to well below an FP32 ulp, with one
// FP64 instruction per entry (GB300's FP64 pipe is slow).  Instances whose
// status is not OK are skipped (their chunk tiles did not run).
__global__ void __launch_bounds__(256) k_gram_reduce(const GramRed* __restrict__ red, const InstState* __restrict__ st,
                                                     const float* __restrict__ part, double* __restrict__ A) {
  const GramRed r = red[blockIdx.y];
  if (st[r.inst].status != 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < r.nn; i += (int64_t)gridDim.x * blockDim.x) {
    const float* p = part + r.part_off + i;
    float hi = p[0], lo = 0.f;
    for (int c = 1; c < r.chunks; ++c) {
      const float x = p[(int64_t)c * r.nn];
      const float t = __fadd_rn(hi, x);
      const float z = __fsub_rn(t, hi);
      lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(x, z)));
      hi = t;
    }
    A[r.out_off + i] = widen_f32(__float_as_uint(hi)) + widen_f32(__float_as_uint(lo));
  }
}

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

// Rank-2 FP32 tensor map over rows of `cols` elements (row stride ld
// elements), box = one 128-byte k-block x 128 rows, 128-byte swizzle, zero
// fill outside.
// FP32 rows [rows x cols] with row stride ld (elements), boxes of 128 rows x
// kblk values: kblk = 32 with the 128-byte swizzle (Gram, three-pass TF32
// contraction), kblk = 16 with the 64-byte swizzle (BF16-mode contraction).
static bool encode_rows(PFN_cuTensorMapEncodeTiled_v12000 encode, CUtensorMap* m, void* gaddr, int64_t cols, int64_t ld,
                        int64_t rows, int kblk = KBLK_F32) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)kblk, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, gaddr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                kblk == KBLK_BF16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename P>
static bool plan_alloc(TcPlan* plan, P** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) return false;
  plan->allocs.push_back((void*)*p);
  return true;
}

// Gram tiles of an n x n symmetric output: per 256-column block J the
// diagonal tile (rows = columns, one or two 128-row sub-tiles; with split,
// two one-sub-tile tiles, the second marked by bit 3), then the 128-row
// off-diagonal tiles below it.
static void gram_tiles(int job, int n, std::vector<int4>& out, bool split) {
  for (int J = 0; J * BN < n; ++J) {
    const int r0 = J * BN;
    if (split && n - r0 > BM) {
      out.push_back(make_int4(job, r0, r0, 1 | 4));
      out.push_back(make_int4(job, r0, r0, 1 | 4 | 8));
    } else {
      out.push_back(make_int4(job, r0, r0, (n - r0 > BM ? 2 : 1) | 4));
    }
    for (int i = r0 + BN; i < n; i += BM) out.push_back(make_int4(job, i, r0, 1));
  }
}

gnmppi_status tc_plan_create(const std::vector<InstDesc>& desc, void* dRW, const uint32_t* W2, void* P, int bf16,
                             cudaStream_t stream, TcPlan* plan, std::string& err) {
  plan->bf16 = bf16;
  auto encode = get_encode(err);
  if (!encode) return GNMPPI_E_CUDA;
  const int kblk = KBLK_F32;
  const int nb = (int)desc.size();
  if (bf16 && !W2) {
    err = "the BF16 contraction needs the split W copy";
    return GNMPPI_E_ARG;
  }
  std::vector<CUtensorMap> maps(4 * (size_t)nb);
  std::vector<TcJob> jobs(3 * (size_t)nb);
  std::vector<int4> tc, tc1, tg, ts;
  std::vector<TcJob> chunk_jobs;  // appended after the 3 nb fixed jobs
  std::vector<GramRed> red;
  int64_t part_elems = 0;
  for (int b = 0; b < nb; ++b) {
    const InstDesc& d = desc[b];
    if (d.ldK % kblk != 0) {
      err = "sample padding is not a multiple of the k-block";
      return GNMPPI_E_ARG;
    }
    if (d.sP % 32 != 0 || d.ldP % 4 != 0 || d.o_P % 4 != 0) {
      err = "[P^T | S] rows are not 16-byte aligned";
      return GNMPPI_E_ARG;
    }
    // contraction: one FP32 map over the instance's [dR; W] block
    if (!encode_rows(encode, &maps[b], reinterpret_cast<char*>(dRW) + 4 * (size_t)d.o_dR, d.ldK, d.ldK,
                     d.nR + d.n, bf16 ? KBLK_BF16 : KBLK_F32)) {
      err = "cuTensorMapEncodeTiled failed (contraction, instance " + std::to_string(b) + ")";
      return GNMPPI_E_CUDA;
    }
    // BF16 mode: the B rows come from the rollouts' split W copy
    if (bf16 && !encode_rows(encode, &maps[3 * nb + b], const_cast<uint32_t*>(W2) + d.o_W2, d.ldK, d.ldK, d.n,
                             KBLK_BF16)) {
      err = "cuTensorMapEncodeTiled failed (split W, instance " + std::to_string(b) + ")";
      return GNMPPI_E_CUDA;
    }
    TcJob& jc = jobs[b];
    jc = TcJob{};
    jc.inst = b;
    jc.map = b;
    jc.map2 = 3 * nb + b;
    // BF16 kernel: A side = the [dR; W] rows, B side = the W rows; three-pass
    // TF32 kernel: A side = the W rows, B side = the [dR; W] rows
    jc.a_row0 = bf16 ? 0 : d.nR;
    jc.b_row0 = bf16 ? d.nR : 0;
    jc.M = d.n;
    jc.Nc = d.nR + d.n;
    jc.nkb = d.ldK / (bf16 ? KBLK_BF16 : KBLK_F32);
    jc.x0 = 0;
    jc.out_off = d.o_P;
    jc.ldc = d.ldP;
    jc.ccut = d.nR;          // S columns of the output ...
    jc.cgap = d.sP - d.nR;   // ... start at sP
    if (bf16) {
      // (job, block of 256 [dR; W] rows, block of 256 W rows, A sub-tiles);
      // the W blocks of a row block adjacent (its A rows read once from HBM);
      // and the same with one 128-row A sub-tile per tile
      for (int i = 0; i * 2 * BM < d.nR + d.n; ++i)
        for (int j = 0; j * BN < d.n; ++j)
          tc.push_back(make_int4(b, i, j, d.nR + d.n - i * 2 * BM > BM ? 2 : 1));
      for (int i = 0; i * BM < d.nR + d.n; ++i)
        for (int j = 0; j * BN < d.n; ++j) tc1.push_back(make_int4(b, i, j, 1));
    } else {
      // three-pass TF32 kernel: (job, first row, first column, 1), the row
      // tiles of a column block adjacent so that its B rows are read from L2
      for (int j = 0; j < d.nR + d.n; j += BN)
        for (int i = 0; i < d.n; i += BM) tc.push_back(make_int4(b, i, j, 1));
    }
    // Gram: FP32 maps over the P^T columns (nR) and the S columns (n) of [P^T | S]
    float* Pb = reinterpret_cast<float*>(P) + d.o_P;
    const int gk = bf16 ? KBLK_BF16 : KBLK_F32;  // the BF16 mode's Gram: BF16 passes too
    if (!encode_rows(encode, &maps[nb + b], Pb, d.nR, d.ldP, d.n, gk) ||
        !encode_rows(encode, &maps[2 * nb + b], Pb + d.sP, d.n, d.ldP, d.n, gk)) {
      err = "cuTensorMapEncodeTiled failed (Gram, instance " + std::to_string(b) + ")";
      return GNMPPI_E_CUDA;
    }
    TcJob& jg = jobs[nb + b];
    jg = TcJob{};
    jg.inst = b;
    jg.map = nb + b;
    jg.M = d.n;
    jg.Nc = d.n;
    jg.nkb = (d.nR + gk - 1) / gk;
    jg.out_off = d.o_nn;
    jg.ldc = d.n;
    jg.ccut = d.n;
    // nR beyond kGramChunkCols: one job per column chunk into the FP64 chunk
    // buffer, added up by k_gram_reduce
    const int gchunk = kGramChunkCols / gk;
    const int nchunks = (jg.nkb + gchunk - 1) / gchunk;
    if (nchunks <= 1) {
      gram_tiles(nb + b, d.n, tg, bf16 != 0);
    } else {
      const int64_t nn = (int64_t)d.n * d.n;
      for (int c = 0; c < nchunks; ++c) {
        TcJob jc2 = jg;
        jc2.x0 = c * gchunk * gk;
        jc2.nkb = std::min(gchunk, jg.nkb - c * gchunk);
        jc2.out_sel = 2;
        jc2.out_off = part_elems + c * nn;
        chunk_jobs.push_back(jc2);
        gram_tiles(3 * nb + (int)chunk_jobs.size() - 1, d.n, tg, bf16 != 0);
      }
      red.push_back(GramRed{d.o_nn, part_elems, nn, nchunks, b});
      part_elems += nchunks * nn;
    }
    // S2 = S S^T over the S columns (LSQ mode)
    TcJob& js = jobs[2 * nb + b];
    js = jg;
    js.map = 2 * nb + b;
    js.nkb = (d.n + gk - 1) / gk;
    js.out_sel = 1;
    if (d.lsq) gram_tiles(2 * nb + b, d.n, ts, bf16 != 0);
  }
  // longest first, so that the short tiles (the S2 products, small
  // instances) fill the SMs that the last long ones leave idle.  Gram tiles
  // by k-blocks x sub-tiles x kept columns; contraction tiles by their
  // instance's k-blocks x sub-tiles only, so that the column tiles of an
  // instance, which share its W rows in L2, stay adjacent.
  jobs.insert(jobs.end(), chunk_jobs.begin(), chunk_jobs.end());
  tg.insert(tg.end(), ts.begin(), ts.end());
  auto gram_work = [&](const int4& t) {
    const TcJob& j = jobs[t.x];
    return (int64_t)j.nkb * (t.w & 3) * std::min(BN, j.Nc - t.z);
  };
  auto contract_work = [&](const int4& t) { return (int64_t)jobs[t.x].nkb * (bf16 ? t.w : 1); };
  std::stable_sort(tc.begin(), tc.end(),
                   [&](const int4& a, const int4& b) { return contract_work(a) > contract_work(b); });
  std::stable_sort(tc1.begin(), tc1.end(),
                   [&](const int4& a, const int4& b) { return contract_work(a) > contract_work(b); });
  std::stable_sort(tg.begin(), tg.end(), [&](const int4& a, const int4& b) { return gram_work(a) > gram_work(b); });
  if (!plan_alloc(plan, &plan->d_maps, sizeof(CUtensorMap) * maps.size()) ||
      !plan_alloc(plan, &plan->d_jobs, sizeof(TcJob) * jobs.size()) ||
      !plan_alloc(plan, &plan->d_tiles_c, sizeof(int4) * std::max<size_t>(1, tc.size())) ||
      !plan_alloc(plan, &plan->d_tiles_c1, sizeof(int4) * std::max<size_t>(1, tc1.size())) ||
      !plan_alloc(plan, &plan->d_tiles_g, sizeof(int4) * std::max<size_t>(1, tg.size())) ||
      (part_elems > 0 && !plan_alloc(plan, &plan->d_part, sizeof(float) * (size_t)part_elems)) ||
      (!red.empty() && !plan_alloc(plan, &plan->d_red, sizeof(GramRed) * red.size())) ||
      !plan_alloc(plan, &plan->d_err, sizeof(int))) {
    err = "cudaMalloc failed for the tensor-core plan";
    return GNMPPI_E_NOMEM;
  }
  plan->ntiles_c = (int)tc.size();
  plan->ntiles_c1 = (int)tc1.size();
  plan->ntiles_g = (int)tg.size();
  plan->nred = (int)red.size();
  bool ok = cudaMemcpyAsync(plan->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                            stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_jobs, jobs.data(), sizeof(TcJob) * jobs.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_tiles_c, tc.data(), sizeof(int4) * tc.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  if (!tc1.empty())
    ok = ok && cudaMemcpyAsync(plan->d_tiles_c1, tc1.data(), sizeof(int4) * tc1.size(), cudaMemcpyHostToDevice,
                               stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(plan->d_tiles_g, tg.data(), sizeof(int4) * tg.size(), cudaMemcpyHostToDevice, stream) ==
                 cudaSuccess;
  if (!red.empty())
    ok = ok && cudaMemcpyAsync(plan->d_red, red.data(), sizeof(GramRed) * red.size(), cudaMemcpyHostToDevice,
                               stream) == cudaSuccess;
  ok = ok && cudaMemsetAsync(plan->d_err, 0, sizeof(int), stream) == cudaSuccess;
  if (!ok) {
    err = "copying the tensor-core plan failed";
    return GNMPPI_E_CUDA;
  }
  // the host vectors are temporaries
  if (cudaStreamSynchronize(stream) != cudaSuccess) {
    err = "copying the tensor-core plan failed";
    return GNMPPI_E_CUDA;
  }
  plan->smem = RING_BYTES + 1024 + 256;
  plan->smem1 = RING_BYTES / 2 + 1024 + 256;
  cudaError_t e = bf16 ? cudaFuncSetAttribute(k_contract_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem)
                       : cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem);
  if (e == cudaSuccess && bf16)
    e = cudaFuncSetAttribute(k_contract_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem1);
  if (e == cudaSuccess)
    e = bf16 ? cudaFuncSetAttribute(k_gram_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem1)
             : cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem);
  if (e != cudaSuccess) {
    err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return GNMPPI_E_CUDA;
  }
  return GNMPPI_OK;
}

cudaError_t tc_contract_launch(const TcPlan& plan, const InstState* d_st, float* P, cudaStream_t stream, int inject,
                               int mt) {
  if (plan.ntiles_c == 0) return cudaSuccess;
  if (plan.bf16 && mt == 1)
    k_contract_tc<1><<<plan.ntiles_c1, kContractThreads, plan.smem1, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                               plan.d_tiles_c1, P, plan.d_err, inject);
  else if (plan.bf16)
    k_contract_tc<2><<<plan.ntiles_c, kContractThreads, plan.smem, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                             plan.d_tiles_c, P, plan.d_err, inject);
  else
    k_gram_tc<true><<<plan.ntiles_c, kGramThreads, plan.smem, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                        plan.d_tiles_c, P, nullptr, nullptr, plan.d_err,
                                                                        inject);
  return cudaGetLastError();
}

cudaError_t tc_gram_launch(const TcPlan& plan, const InstState* d_st, double* A, double* S2, cudaStream_t stream) {
  if (plan.ntiles_g == 0) return cudaSuccess;
  if (plan.bf16)
    k_gram_tc<false, true><<<plan.ntiles_g, kGramThreads, plan.smem1, stream>>>(
        plan.d_maps, plan.d_jobs, d_st, plan.d_tiles_g, A, S2, plan.d_part, plan.d_err, 0);
  else
    k_gram_tc<false><<<plan.ntiles_g, kGramThreads, plan.smem, stream>>>(plan.d_maps, plan.d_jobs, d_st,
                                                                          plan.d_tiles_g, A, S2, plan.d_part,
                                                                          plan.d_err, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && plan.nred > 0) {
    k_gram_reduce<<<dim3(32, plan.nred), 256, 0, stream>>>(plan.d_red, d_st, plan.d_part, A);
    e = cudaGetLastError();
  }
  return e;
}

GNM_CHECK_ACCESSOR(check_count_tc)

}  // namespace gnm
