// chol.cuh -- FP64 Cholesky factorisation and triangular solves of one n x n
// symmetric positive definite system per CTA of 128, 256 or 512 threads, for
// the damped Gauss-Newton step of GN-MPPI (arXiv 2512.04579, Sec. 4, the
// normal equations of Eq. 9 with damping).
//
// Shaped by the GB300 FP64 pipe: one warp issues at most one FP64 instruction
// per 64 cycles whatever its active lanes, and the SM retires one FP64 warp
// instruction per 19 cycles once four or more warps feed it.  So the work is
// kept on full warps, serial chains are short, and the latency-bound
// diagonal-block step runs on one warp while the others carry the trailing
// update (look-ahead by one panel).
//
// Storage: the lower factor is packed by rows in global memory (element
// (i, j), j <= i, at i (i + 1) / 2 + j) and stays L2/L1 resident; the inverse
// of every CNB x CNB diagonal block is kept row-major (CNB x CNB, zero upper
// part) for the panel and substitution steps.
#pragma once
#include <cstdint>

namespace gnm {

constexpr int CNB = 16;  // panel width
constexpr int CNB2 = CNB * CNB;

__device__ __forceinline__ int64_t pk(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }  // j <= i

// Factor the nb x nb diagonal block at (p0, p0) (already reduced by every
// earlier panel) with one warp: lane r keeps row r of the block in registers.
// Writes the factor in place, invd[p0 + r] = 1 / L[r][r] and Yp = the block's
// inverse (row-major, zeros above the diagonal).  Returns false, uniformly
// over the warp, on a pivot that is not positive and finite.
__device__ __noinline__ bool diag_factor(double* L, double* invd, double* Yp, int p0, int nb) {
  const int lane = threadIdx.x & 31;
  double a[CNB];
#pragma unroll
  for (int c = 0; c < CNB; ++c) a[c] = (lane < nb && c <= lane) ? L[pk(p0 + lane, p0 + c)] : 0.0;
  bool ok = true;
  double rinv = 0.0;
#pragma unroll
  for (int c = 0; c < CNB; ++c) {
    if (c < nb) {
      const double d = __shfl_sync(0xffffffffu, a[c], c);  // pivot, already reduced
      ok = ok && (d > 0.0) && isfinite(d);
      const double rj = rsqrt(d);
      if (lane == c) rinv = rj;
      // column c: L[c][c] = d rj (lane c holds d), L[r][c] = a[r][c] rj below it
      a[c] = (lane >= c) ? a[c] * rj : a[c];
      // rank-1 update of the rows below: a[r][k] -= L[r][c] L[k][c], c < k <= r
#pragma unroll
      for (int k = c + 1; k < CNB; ++k) {
        const double lkc = __shfl_sync(0xffffffffu, a[c], k);
        if (lane >= k) a[k] = fma(-a[c], lkc, a[k]);
      }
    }
  }
  if (lane < nb) {
#pragma unroll
    for (int c = 0; c < CNB; ++c)
      if (c <= lane) L[pk(p0 + lane, p0 + c)] = a[c];
    invd[p0 + lane] = rinv;
  }
  // inverse of the block, column j = lane: y_i = (delta_ij - sum_{q<i} L[i][q] y_q) / L[i][i]
  double y[CNB];
#pragma unroll
  for (int i = 0; i < CNB; ++i) {
    y[i] = 0.0;
    if (i < nb) {
      double s = (lane == i) ? 1.0 : 0.0;
#pragma unroll
      for (int q = 0; q < i; ++q) s = fma(-__shfl_sync(0xffffffffu, a[q], i), y[q], s);
      y[i] = s * __shfl_sync(0xffffffffu, rinv, i);
    }
  }
  if (lane < nb) {
#pragma unroll
    for (int i = 0; i < CNB; ++i)
      if (i < nb) Yp[i * CNB + lane] = y[i];
  }
  return ok;
}

// Panel rows below the diagonal block at p0: L21 = A21 L11^-T, i.e.
// v_c = sum_{q <= c} a_q Y[c][q] with Y = L11^-1.  Called by every thread of
// the CTA (4, 8 or 16 warps).  Short panels split each row's 16 outputs over R = 2
// or 4 warps (a warp-uniform residue class of c) so that their FP64 work
// still reaches all four sub-partitions of the SM.
__device__ __forceinline__ void panel_rows(double* L, const double* Yp, int n, int p0, int nb) {
  const int r0 = p0 + nb, m = n - r0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  if (m > 16 * nwarp) {
    for (int i = r0 + (int)threadIdx.x; i < n; i += (int)blockDim.x) {
      double* Li = L + pk(i, p0);
      double a[CNB];
#pragma unroll
      for (int q = 0; q < CNB; ++q) a[q] = (q < nb) ? Li[q] : 0.0;
#pragma unroll
      for (int c = 0; c < CNB; ++c) {
        if (c < nb) {
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q <= c; ++q) acc = fma(a[q], Yp[c * CNB + q], acc);
          Li[c] = acc;
        }
      }
    }
    return;
  }
  // m <= 16 nwarp: one row per thread group; every thread reads its row before any writes
  const int R = (m > 8 * nwarp) ? 2 : 4;
  const int j = warp % R;
  const int i = r0 + (warp / R) * 32 + lane;
  const bool has = (m > 0) && (i < n);
  double a[CNB];
#pragma unroll
  for (int q = 0; q < CNB; ++q) a[q] = (has && q < nb) ? L[pk(has ? i : 0, p0) + q] : 0.0;
  __syncthreads();
  if (has) {
    double* Li = L + pk(i, p0);
#pragma unroll
    for (int c = 0; c < CNB; ++c) {
      if (c % R == j && c < nb) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q <= c; ++q) acc = fma(a[q], Yp[c * CNB + q], acc);
        Li[c] = acc;
      }
    }
  }
}

// One TS x TS tile of the rank-nb update by the panel at p0:
// L[i][k] -= sum_c L[i][p0 + c] L[k][p0 + c] for i in [i0, i0 + TS),
// k in [k0, k0 + TS), k <= i, i < n, k < kend.
template <int TS>
__device__ __forceinline__ void rank_tile(double* L, int n, int p0, int nb, int i0, int k0, int kend) {
  double acc[TS][TS];
#pragma unroll
  for (int p = 0; p < TS; ++p)
#pragma unroll
    for (int q = 0; q < TS; ++q) acc[p][q] = 0.0;
  const double* ra[TS];
  const double* rb[TS];
#pragma unroll
  for (int p = 0; p < TS; ++p) {
    ra[p] = L + pk(min(i0 + p, n - 1), p0);
    rb[p] = L + pk(min(k0 + p, n - 1), p0);
  }
#pragma unroll 4
  for (int c = 0; c < nb; ++c) {
    double av[TS], bv[TS];
#pragma unroll
    for (int p = 0; p < TS; ++p) {
      av[p] = ra[p][c];
      bv[p] = rb[p][c];
    }
#pragma unroll
    for (int p = 0; p < TS; ++p)
#pragma unroll
      for (int q = 0; q < TS; ++q) acc[p][q] = fma(av[p], bv[q], acc[p][q]);
  }
#pragma unroll
  for (int p = 0; p < TS; ++p)
#pragma unroll
    for (int q = 0; q < TS; ++q) {
      const int i = i0 + p, k = k0 + q;
      if (i < n && k < kend && k <= i) L[pk(i, k)] -= acc[p][q];
    }
}

// Update of the next block column [q0, q0 + nbq) (rows q0..n-1) by the panel
// at p0, in 2 x 2 tiles over threads t = 0..nt-1.
__device__ __forceinline__ void next_column_update(double* L, int n, int p0, int nb, int q0, int nbq, int t, int nt) {
  const int nI = (n - q0 + 1) / 2, nK = (nbq + 1) / 2;
  for (int u = t; u < nI * nK; u += nt) {
    const int I = u / nK, K = u - I * nK;
    if (K > I) continue;  // entirely above the diagonal
    rank_tile<2>(L, n, p0, nb, q0 + 2 * I, q0 + 2 * K, q0 + nbq);
  }
}

// Update of the trailing lower triangle [r1, n) x [r1, n) by the panel at p0,
// in 4 x 4 tiles over threads t = 0..nt-1.
__device__ __forceinline__ void trailing_update(double* L, int n, int p0, int nb, int r1, int t, int nt) {
  const int m = n - r1;
  if (m <= 0) return;
  const int T = (m + 3) / 4, ntile = T * (T + 1) / 2;
  for (int u = t; u < ntile; u += nt) {
    int I = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= u) ++I;
    while (I * (I + 1) / 2 > u) --I;
    const int K = u - I * (I + 1) / 2;
    rank_tile<4>(L, n, p0, nb, r1 + 4 * I, r1 + 4 * K, n);
  }
}

// Right-looking blocked Cholesky of the packed lower matrix in L, in place,
// with look-ahead: per panel p, (1) all warps form the panel rows, (2) all
// warps reduce the next block column, (3) warp 0 factors the next diagonal
// block (and inverts it) while the other warps reduce the rest of the
// trailing matrix.  invd[i] = 1 / L[i][i]; Y holds the inverted diagonal
// blocks (CNB2 doubles per panel).  Returns false, uniformly over the CTA, on
// a pivot that is not positive and finite.  128, 256 or 512 threads.
__device__ bool chol_factor(double* L, double* invd, double* Y, int n, int* fail) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = (n + CNB - 1) / CNB;
  if (tid == 0) *fail = 0;
  __syncthreads();
  if (warp == 0) {
    const bool ok = diag_factor(L, invd, Y, 0, min(CNB, n));
    if (!ok && lane == 0) *fail = 1;
  }
  __syncthreads();
  if (*fail) return false;
  for (int p = 0; p < np; ++p) {
    const int p0 = p * CNB, nb = min(CNB, n - p0);
    panel_rows(L, Y + (int64_t)p * CNB2, n, p0, nb);
    __syncthreads();
    if (p + 1 < np) {
      const int q0 = p0 + nb, nbq = min(CNB, n - q0);
      next_column_update(L, n, p0, nb, q0, nbq, tid, (int)blockDim.x);
      __syncthreads();
      if (warp == 0) {
        const bool ok = diag_factor(L, invd, Y + (int64_t)(p + 1) * CNB2, q0, nbq);
        if (!ok && lane == 0) *fail = 1;
      } else {
        trailing_update(L, n, p0, nb, q0 + nbq, tid - 32, (int)blockDim.x - 32);
      }
      __syncthreads();
      if (*fail) return false;
    }
  }
  return true;
}

// Solve L z = x in place (x in shared memory): per panel, warp 0 applies the
// inverted diagonal block, then every thread reduces one row below it.
__device__ void chol_forward(const double* L, const double* Y, double* x, int n) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __syncthreads();
  for (int p0 = 0; p0 < n; p0 += CNB) {
    const int nb = min(CNB, n - p0);
    const double* Yp = Y + (int64_t)(p0 / CNB) * CNB2;
    if (warp == 0) {
      double acc = 0.0;
      if (lane < nb)
        for (int c = 0; c < nb; ++c) acc = fma(Yp[lane * CNB + c], x[p0 + c], acc);
      __syncwarp();
      if (lane < nb) x[p0 + lane] = acc;
    }
    __syncthreads();
    for (int i = p0 + nb + tid; i < n; i += (int)blockDim.x) {
      const double* Li = L + pk(i, p0);
      double s = 0.0;
      for (int c = 0; c < nb; ++c) s = fma(Li[c], x[p0 + c], s);
      x[i] -= s;
    }
    __syncthreads();
  }
}

// Solve L^T x = z in place (x in shared memory), panels in reverse order.
__device__ void chol_backward(const double* L, const double* Y, double* x, int n) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __syncthreads();
  const int last = ((n - 1) / CNB) * CNB;
  for (int p0 = last; p0 >= 0; p0 -= CNB) {
    const int nb = min(CNB, n - p0);
    const double* Yp = Y + (int64_t)(p0 / CNB) * CNB2;
    if (warp == 0) {
      double acc = 0.0;
      if (lane < nb)
        for (int r = 0; r < nb; ++r) acc = fma(Yp[r * CNB + lane], x[p0 + r], acc);
      __syncwarp();
      if (lane < nb) x[p0 + lane] = acc;
    }
    __syncthreads();
    for (int i = tid; i < p0; i += (int)blockDim.x) {
      double s = 0.0;
      for (int c = 0; c < nb; ++c) s = fma(L[pk(p0 + c, i)], x[p0 + c], s);
      x[i] -= s;
    }
    __syncthreads();
  }
}

}  // namespace gnm
