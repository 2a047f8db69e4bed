// solver_kernels.cuh -- the per-iteration linear-algebra kernels of GN-MPPI
// (arXiv 2512.04579, Algorithm 1):
//   * k_softmin_wvec: softmin weights of the sample costs (Eq. 5) with the
//     min shift, their sums and effective sample size, the weighted mean
//     perturbation of Eq. 3, and b = P^T r = W^T e (the GGN gradient, Eq. 9,
//     up to the metric S^-1);
//   * k_gemm_nt: SIMT batched C = A B^T with the reduction dimension contiguous
//     in both operands, used for the contraction [P^T | S] = W^T [dR | W]
//     (Eq. 7), the Gram A = P^T P and S^2 in FP64/FP32 modes;
//   * k_solve: (A + lambda S_used^2) y = -b by Cholesky in FP64 with iterative
//     refinement and tenfold damping retries, delta = S_used y, which equals
//     the damped GGN step (J^T J + lambda I) delta = -J^T r for J = P S_used^-1;
//   * k_update: argmin of the line search (Eq. 11), U += alpha* delta (Eq. 10),
//     r <- R(U_{k+1}) and the covariance shrink Sigma <- beta Sigma.
// Internal; instantiated once in solver.cu.
#pragma once
#include "common.cuh"

namespace gnm {

struct SolveArgs {
  const InstDesc* inst;
  InstState* st;
  Consts cs;
  double* U;
  double* s;
  double* g;       // b = P^T r [n]
  double* mppi;    // weighted mean perturbation [n]
  double* delta;   // [n]
  double* y;       // [n] scratch
  double* wt;      // [Kp] softmin weight differences
  const double* C; // [Kp][2]
  const double* e; // [Kp]
  const void* W;   // [n][ldK] storage type
  const void* P;   // [n][ldP] accumulation type
  double* A;       // [n][n]
  double* S2;      // [n][n]
  double* H;       // [n][n]
  double* Lg;      // global Cholesky scratch (packed lower) for large n, or nullptr
  const int64_t* o_L;  // per-instance offsets into Lg
  void* r;         // nominal residual [nR] scalar type
  const void* RL;  // [L][nR]
  double* Cl;      // [kMaxL+1]
  int shrink;      // apply the covariance shrink after the update
  int smem_n_max;  // largest n whose packed factor fits in shared memory
};

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide reductions for 256 threads (8 warps).
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}
__device__ __forceinline__ double block_min(double v, double* red) {
  v = warp_min(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = INFINITY;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmin(t, red[i]);
  return t;
}

// One CTA (256 threads) per instance.
template <typename S, typename TA>
__global__ void __launch_bounds__(256) k_softmin_wvec(SolveArgs a) {
  const int b = blockIdx.x;
  const InstDesc I = a.inst[b];
  if (a.st[b].status != 0) return;
  __shared__ double red[32];
  const bool anti = a.cs.antithetic != 0;
  const double* C = a.C + I.o_C;
  const double* e = a.e + I.o_C / 2;
  double* wt = a.wt + I.o_C / 2;
  // 1. minimum over the finite sample costs; pairs with a non-finite cost are dropped
  double cmin = INFINITY;
  int masked = 0;
  for (int m = threadIdx.x; m < I.Kp; m += blockDim.x) {
    const double c0 = C[anti ? 2 * m : m];
    const double c1 = anti ? C[2 * m + 1] : c0;
    const bool ok = isfinite(c0) && isfinite(c1);
    if (ok) cmin = fmin(cmin, fmin(c0, c1));
    masked += ok ? 0 : 1;
  }
  cmin = block_min(cmin, red);
  const int nmask = (int)block_sum((double)masked, red);
  // 2. weights exp(-(C - cmin)/tau) (Eq. 5), their sums, and w+ - w- per pair
  double s1 = 0.0, s2 = 0.0;
  const double itau = 1.0 / a.cs.tau;
  for (int m = threadIdx.x; m < I.Kp; m += blockDim.x) {
    const double c0 = C[anti ? 2 * m : m];
    const double c1 = anti ? C[2 * m + 1] : c0;
    const bool ok = isfinite(c0) && isfinite(c1) && isfinite(cmin);
    const double w0 = ok ? exp(-(c0 - cmin) * itau) : 0.0;
    const double w1 = (ok && anti) ? exp(-(c1 - cmin) * itau) : 0.0;
    s1 += w0 + w1;
    s2 += w0 * w0 + w1 * w1;
    wt[m] = w0 - w1;
  }
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  __syncthreads();  // wt visible to every warp
  // 3. rows of W: b_j = sum_m W[j][m] e_m, mppi_j = sum_m W[j][m] wt_m / sum w
  const S* W = reinterpret_cast<const S*>(a.W) + I.o_W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double gsq = 0.0;
  for (int j = warp; j < I.n; j += nw) {
    const S* row = W + (int64_t)j * I.ldK;
    TA ag = (TA)0, am = (TA)0;
    for (int m = lane; m < I.Kp; m += 32) {
      const TA w = (TA)to_d(row[m]);
      ag += w * (TA)e[m];
      am += w * (TA)wt[m];
    }
    const double G = warp_sum((double)ag);
    const double Mp = warp_sum((double)am);
    if (lane == 0) {
      a.g[I.o_U + j] = G;
      a.mppi[I.o_U + j] = s1 > 0.0 ? Mp / s1 : 0.0;
      gsq += G * G;
    }
  }
  gsq = block_sum(gsq, red);
  if (threadIdx.x == 0) {
    InstState& s = a.st[b];
    s.c_min = cmin;
    s.sum_w = s1;
    s.sum_w2 = s2;
    s.ess = s2 > 0.0 ? s1 * s1 / s2 : 0.0;
    s.n_masked = nmask;
    s.pr_norm = sqrt(gsq);
    if (nmask >= I.Kp) s.status = -4;  // every sample non-finite
  }
}

// ------------------------------------------------------------- SIMT GEMM
enum GemmKind { kContract = 0, kGram = 1, kS2 = 2 };

struct GemmArgs {
  const InstDesc* inst;
  const InstState* st;
  const int4* tiles;  // (instance, tile row, tile col, -)
  const void* dR;
  const void* W;
  void* P;
  double* A;
  double* S2;
};

// C[i][j] = sum_k A[i][k] B[j][k], 64x64 tile per CTA, 4x4 per thread.
template <GemmKind KIND, typename TIn, typename TC, typename TOut>
__global__ void __launch_bounds__(256) k_gemm_nt(GemmArgs g) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ TC As[BK][BM + 1];
  __shared__ TC Bs[BK][BN + 1];
  const int4 tl = g.tiles[blockIdx.x];
  const int b = tl.x;
  if (g.st[b].status != 0) return;
  const InstDesc I = g.inst[b];
  int Mr, Nc, Kd;
  const TIn* Abase;
  const TIn* B1;
  const TIn* B2;
  int64_t lda, ldb;
  int nb1;
  TOut* Cbase;
  int64_t ldc;
  if (KIND == kContract) {
    Mr = I.n; Nc = I.nR + I.n; Kd = I.Kp;
    Abase = reinterpret_cast<const TIn*>(g.W) + I.o_W; lda = I.ldK;
    B1 = reinterpret_cast<const TIn*>(g.dR) + I.o_dR; nb1 = I.nR;
    B2 = reinterpret_cast<const TIn*>(g.W) + I.o_W; ldb = I.ldK;
    Cbase = reinterpret_cast<TOut*>(g.P) + I.o_P; ldc = I.ldP;
  } else if (KIND == kGram) {
    Mr = I.n; Nc = I.n; Kd = I.nR;
    Abase = reinterpret_cast<const TIn*>(g.P) + I.o_P; lda = I.ldP;
    B1 = Abase; nb1 = I.n; B2 = Abase; ldb = I.ldP;
    Cbase = reinterpret_cast<TOut*>(g.A) + I.o_nn; ldc = I.n;
  } else {
    Mr = I.n; Nc = I.n; Kd = I.n;
    Abase = reinterpret_cast<const TIn*>(g.P) + I.o_P + I.nR; lda = I.ldP;
    B1 = Abase; nb1 = I.n; B2 = Abase; ldb = I.ldP;
    Cbase = reinterpret_cast<TOut*>(g.S2) + I.o_nn; ldc = I.n;
  }
  const int i0 = tl.y * BM, j0 = tl.z * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  TC acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = (TC)0;
  const int lr = threadIdx.x >> 2, lk = (threadIdx.x & 3) * 4;
  for (int k0 = 0; k0 < Kd; k0 += BK) {
    {
      const int i = i0 + lr;
      const TIn* ar = Abase + (int64_t)i * lda;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + lk + q;
        As[lk + q][lr] = (i < Mr && k < Kd) ? (TC)to_d(ar[k]) : (TC)0;
      }
      const int j = j0 + lr;
      const TIn* br = (j < nb1) ? B1 + (int64_t)j * ldb : B2 + (int64_t)(j - nb1) * ldb;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + lk + q;
        Bs[lk + q][lr] = (j < Nc && k < Kd) ? (TC)to_d(br[k]) : (TC)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TC av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + ty * 4 + p;
    if (i >= Mr) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx * 4 + q;
      if (j < Nc) Cbase[(int64_t)i * ldc + j] = (TOut)acc[p][q];
    }
  }
}

// ----------------------------------------------------------- Cholesky solve
__device__ __forceinline__ int64_t pk(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }  // j <= i

constexpr int CNB = 16;  // Cholesky panel width

// Blocked right-looking Cholesky of a packed lower matrix, in place (256
// threads): per panel of CNB columns, warp 0 factors the diagonal block,
// every thread solves one panel row against it, and the trailing lower
// triangle is updated in 4 x 4 register tiles (two DFMAs per shared-memory
// load).  Returns false, uniformly across the CTA, on a non-positive pivot.
__device__ bool chol_blocked(double* L, double* invd, int n, int* fail) {
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const double* inv = nullptr;  // reciprocals of the current panel's diagonal
  if (tid == 0) *fail = 0;
  __syncthreads();
  for (int p0 = 0; p0 < n; p0 += CNB) {
    const int nb = min(CNB, n - p0);
    inv = invd + p0;
    if (warp == 0) {
      for (int c = 0; c < nb; ++c) {
        const int pc = p0 + c;
        const double d = L[pk(pc, pc)];
        const double rj = rsqrt(d);
        const double ljj = d * rj;
        __syncwarp();
        if (lane == 0) {
          L[pk(pc, pc)] = ljj;
          invd[pc] = rj;
          if (!(d > 0.0) || !isfinite(d)) *fail = 1;
        }
        if (lane > c && lane < nb) L[pk(p0 + lane, pc)] *= rj;
        __syncwarp();
        if (lane > c && lane < nb) {
          const double lrc = L[pk(p0 + lane, pc)];
          for (int k = c + 1; k <= lane; ++k) L[pk(p0 + lane, p0 + k)] -= lrc * L[pk(p0 + k, pc)];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (*fail) return false;
    // panel rows: L21 = A21 L11^-T, one row per thread
    for (int i = p0 + nb + tid; i < n; i += nt) {
      double* Li = L + pk(i, p0);
      double v[CNB];
#pragma unroll
      for (int c = 0; c < CNB; ++c) v[c] = (c < nb) ? Li[c] : 0.0;
#pragma unroll
      for (int c = 0; c < CNB; ++c) {
        if (c < nb) {
          double sacc = v[c];
          const double* Lc = L + pk(p0 + c, p0);
#pragma unroll
          for (int q = 0; q < CNB; ++q)
            if (q < c) sacc -= v[q] * Lc[q];
          v[c] = sacc * inv[c];
        }
      }
#pragma unroll
      for (int c = 0; c < CNB; ++c)
        if (c < nb) Li[c] = v[c];
    }
    __syncthreads();
    // trailing update A22 -= L21 L21^T on the lower triangle, 4 x 4 tiles
    const int r0 = p0 + nb, m = n - r0;
    if (m > 0) {
      const int Tt = (m + 3) / 4, ntile = Tt * (Tt + 1) / 2;
      for (int t = tid; t < ntile; t += nt) {
        int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((I + 1) * (I + 2) / 2 <= t) ++I;
        while (I * (I + 1) / 2 > t) --I;
        const int Kt = t - I * (I + 1) / 2;
        const int i0 = r0 + 4 * I, k0 = r0 + 4 * Kt;
        double acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
        const double* ra[4];
        const double* rb[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          ra[p] = L + pk(min(i0 + p, n - 1), p0);
          rb[p] = L + pk(min(k0 + p, n - 1), p0);
        }
        for (int c = 0; c < nb; ++c) {
          double a[4], b[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            a[p] = ra[p][c];
            b[p] = rb[p][c];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = i0 + p, k = k0 + q;
            if (i < n && k <= i) L[pk(i, k)] -= acc[p][q];
          }
      }
    }
    __syncthreads();
  }
  return true;
}

// Solve L L^T x = x in place (packed lower L, invd = 1 / diag(L)), blocked
// like the factorisation.
__device__ void chol_subst(const double* L, const double* invd, double* x, int n) {
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  __syncthreads();
  // forward: L z = x
  for (int p0 = 0; p0 < n; p0 += CNB) {
    const int nb = min(CNB, n - p0);
    if (warp == 0) {
      for (int c = 0; c < nb; ++c) {
        double zc = x[p0 + c];
        __syncwarp();
        zc *= invd[p0 + c];
        if (lane == 0) x[p0 + c] = zc;
        if (lane > c && lane < nb) x[p0 + lane] -= L[pk(p0 + lane, p0 + c)] * zc;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = p0 + nb + tid; i < n; i += nt) {
      const double* Li = L + pk(i, p0);
      double sacc = 0.0;
      for (int c = 0; c < nb; ++c) sacc += Li[c] * x[p0 + c];
      x[i] -= sacc;
    }
    __syncthreads();
  }
  // backward: L^T x = z
  const int last = ((n - 1) / CNB) * CNB;
  for (int p0 = last; p0 >= 0; p0 -= CNB) {
    const int nb = min(CNB, n - p0);
    if (warp == 0) {
      for (int c = nb - 1; c >= 0; --c) {
        double xc = x[p0 + c];
        __syncwarp();
        xc *= invd[p0 + c];
        if (lane == 0) x[p0 + c] = xc;
        if (lane < c) x[p0 + lane] -= L[pk(p0 + c, p0 + lane)] * xc;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < p0; i += nt) {
      double sacc = 0.0;
      for (int c = 0; c < nb; ++c) sacc += L[pk(p0 + c, i)] * x[p0 + c];
      x[i] -= sacc;
    }
    __syncthreads();
  }
}

// One CTA (256 threads) per instance.  Packed lower factor in shared memory
// when n <= smem_n_max, otherwise in the global scratch.
template <typename TA>
__global__ void __launch_bounds__(256) k_solve(SolveArgs a) {
  const int b = blockIdx.x;
  InstState& st = a.st[b];
  if (st.status != 0) return;
  const InstDesc I = a.inst[b];
  const int n = I.n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* vec = reinterpret_cast<double*>(smem_raw);  // rhs, x, res, 1/diag(L)
  double* rhs = vec;
  double* x = vec + n;
  double* res = vec + 2 * n;
  double* invd = vec + 3 * n;
  double* L = (n <= a.smem_n_max) ? vec + 4 * n : a.Lg + a.o_L[b];
  __shared__ int fail;
  const double* A = a.A + I.o_nn;
  const double* S2 = a.S2 + I.o_nn;
  double* H = a.H + I.o_nn;
  const TA* P = reinterpret_cast<const TA*>(a.P) + I.o_P;
  const double* s = a.s + I.o_U;
  const double Keff = (double)(I.Kp - st.n_masked);
  for (int j = threadIdx.x; j < n; j += blockDim.x) rhs[j] = -a.g[I.o_U + j];
  double lam = a.cs.lambda;
  int retries = 0;
  bool ok = false;
  for (; retries <= 6; ++retries) {
    // H = A + lam * S_used^2
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const int r = i / n, c = i - r * n;
      double t;
      if (I.lsq) {
        t = S2[i];
      } else {
        const double sc = Keff * s[r] * s[r];
        t = (r == c) ? sc * sc : 0.0;
      }
      H[i] = A[i] + lam * t;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      for (int c = 0; c <= r; ++c) L[pk(r, c)] = H[(int64_t)r * n + c];
    __syncthreads();
    if (chol_blocked(L, invd, n, &fail)) {
      ok = true;
      break;
    }
    lam *= 10.0;
    __syncthreads();
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      st.status = -3;
      st.chol_retries = 7;
      st.lambda_used = lam;
    }
    return;
  }
  // y = H^-1 rhs with iterative refinement (residual in FP64 against H)
  for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = rhs[j];
  __syncthreads();
  chol_subst(L, invd, x, n);
  for (int t = 0; t < a.cs.ir_steps; ++t) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < n; i += 8) {
      double acc = 0.0;
      for (int c = lane; c < n; c += 32) acc += H[(int64_t)i * n + c] * x[c];
      acc = warp_sum(acc);
      if (lane == 0) res[i] = rhs[i] - acc;
    }
    __syncthreads();
    chol_subst(L, invd, res, n);
    for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] += res[j];
    __syncthreads();
  }
  // delta = S_used y
  double dsq = 0.0;
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < n; i += 8) {
      double acc = 0.0;
      if (I.lsq) {
        const TA* Srow = P + (int64_t)i * I.ldP + I.nR;
        for (int c = lane; c < n; c += 32) acc += (double)Srow[c] * x[c];
        acc = warp_sum(acc);
      } else {
        acc = Keff * s[i] * s[i] * x[i];
      }
      if (lane == 0) {
        a.delta[I.o_U + i] = acc;
        a.y[I.o_U + i] = x[i];
        dsq += acc * acc;
      }
    }
  }
  __shared__ double red[32];
  dsq = block_sum(dsq, red);
  if (threadIdx.x == 0) {
    st.chol_retries = retries;
    st.lambda_used = lam;
    st.step_norm = sqrt(dsq);
    st.jac_mode_used = I.lsq ? 0 : 1;
  }
}

// One CTA (128 threads) per instance: line-search argmin (ties to the smallest
// j; alpha = 0 last when monotone), U += alpha* delta, r <- R(U + alpha* delta),
// and, in Algorithm-1 solves, s <- sqrt(beta) s.
template <typename T>
__global__ void __launch_bounds__(128) k_update(SolveArgs a) {
  const int b = blockIdx.x;
  InstState& st = a.st[b];
  if (st.status != 0) return;
  const InstDesc I = a.inst[b];
  __shared__ int js;
  __shared__ double alpha_s, cnew_s;
  if (threadIdx.x == 0) {
    const double* Cl = a.Cl + (int64_t)b * (kMaxL + 1);
    double best = INFINITY, al = 1.0, ab = 0.0;
    int jb = -1;
    for (int j = 0; j < a.cs.L; ++j) {
      if (Cl[j] < best) {
        best = Cl[j];
        jb = j;
        ab = al;
      }
      al *= a.cs.gamma;
    }
    if (a.cs.monotone && st.C_nom < best) {
      best = st.C_nom;
      jb = a.cs.L;
      ab = 0.0;
    }
    js = jb;
    alpha_s = ab;
    cnew_s = best;
    if (jb < 0) st.status = -4;
  }
  __syncthreads();
  if (js < 0) return;
  const double al = alpha_s;
  for (int i = threadIdx.x; i < I.n; i += blockDim.x) {
    a.U[I.o_U + i] = a.U[I.o_U + i] + al * a.delta[I.o_U + i];
    if (a.shrink) a.s[I.o_U + i] *= a.cs.beta_sqrt;
  }
  if (js < a.cs.L) {
    T* r = reinterpret_cast<T*>(a.r) + I.o_R;
    const T* src = reinterpret_cast<const T*>(a.RL) + I.o_RL + (int64_t)js * I.nR;
    for (int i = threadIdx.x; i < I.nR; i += blockDim.x) r[i] = src[i];
  }
  if (threadIdx.x == 0) {
    st.C_start = st.C_nom;
    st.C_new = cnew_s;
    st.C_nom = cnew_s;
    st.alpha = al;
    st.j_star = js;
    st.total_masked += st.n_masked;
    st.total_retries += st.chol_retries;
    st.iters += 1;
  }
}

}  // namespace gnm
