// mlp.cu -- the learned warm start: a small MLP that maps an initial state to
// a nominal control sequence mu (U_0 of Algorithm 1) and one log sampling
// scale per control step (Sigma_0), trained on solutions of plain GN-MPPI with
// a Gaussian negative log-likelihood.  Training and inference run in these
// kernels.  Every product -- forward, input gradient, weight gradient -- is a
// tcgen05 GEMM on the sm_103a tensor cores: its operands are stored as a BF16
// head plane and a BF16 remainder plane (K-major rows, loaded by TMA), each
// product is formed from three BF16 passes (head x head + head x remainder +
// remainder x head, FP32 accumulation in TMEM, FP32-level accuracy), and the
// epilogue fuses the bias, GELU (keeping the pre-activation) or the GELU'
// factor of the layer below.  Weights optionally rounded to BF16 (their
// remainder plane is then zero) for the forward and input-gradient products.
// Then the loss and its output gradient, column sums for the bias gradients,
// and Adam with bias correction.  Parameter layout per layer: W [d_out][d_in]
// row-major, then b [d_out].
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gnmppi.h"
#include "common.cuh"
#include "tc_ptx.cuh"

namespace gnm {
namespace {

constexpr int kMaxLayers = 8;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// One product C[i][j] = sum_k A[i][k] B[j][k] (i < M, j < N, k < K) with the
// epilogue `mode`: 0 acc + bias[j]; 1 Z = acc + bias[j], C = GELU(Z);
// 2 acc * GELU'(Zprev); 3 acc.  C, Z and Zprev share the row stride ldc.
struct MlpTc {
  float* C;
  int64_t ldc;
  int M, N, K;
  const float* bias;
  float* Z;
  const float* Zprev;
  int mode;
};

constexpr int kTcBox = 128 * 128;           // one 128-row x 64-value BF16 box (128-byte rows), 16 KB
constexpr int kTcStage = 4 * kTcBox;         // A head, A remainder, B head, B remainder
constexpr int kTcStages = 3;
constexpr int kTcSmem = kTcStages * kTcStage + 1024 + 256;

// 128 x 128 output tile per CTA.  Warp 0 lane 0 issues the TMA loads of the
// four operand boxes of a 64-value k-block into a 3-stage ring, warp 1 lane 0
// the three BF16 passes (M = N = 128, K = 16 per MMA) into one TMEM
// accumulator, warps 0-3 read it back (one TMEM lane per output row) and
// store through a padded shared-memory transpose, whole rows per warp store.
// Every wait is bounded; a wait that runs out sets *err and the CTA winds down.
__global__ void __launch_bounds__(128, 1) k_mlp_tc(const __grid_constant__ CUtensorMap ah,
                                                   const __grid_constant__ CUtensorMap al,
                                                   const __grid_constant__ CUtensorMap bh,
                                                   const __grid_constant__ CUtensorMap bl, MlpTc g,
                                                   int* __restrict__ err) {
  const int i0 = blockIdx.y * 128, j0 = blockIdx.x * 128;
  const int nkb = (g.K + 63) / 64;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTcStages * kTcStage);
  // bars[0..3): full, [3..6): empty, [6]: done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * kTcStages + 1; ++s) mbar_init(su32(bars + s), 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t done = su32(bars + 2 * kTcStages);

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kTcStages, round = kb / kTcStages;
      if (kb >= kTcStages && !mbar_wait(su32(bars + kTcStages + s), (round - 1) & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      const uint32_t full = su32(bars + s);
      mbar_expect_tx(full, (uint32_t)kTcStage);
      const uint32_t d = su32(base + s * kTcStage);
      tma_load(d, &ah, full, kb * 64, i0);
      tma_load(d + kTcBox, &al, full, kb * 64, i0);
      tma_load(d + 2 * kTcBox, &bh, full, kb * 64, j0);
      tma_load(d + 3 * kTcBox, &bl, full, kb * 64, j0);
      ++issued;
    }
    for (int kb = (issued > kTcStages ? issued - kTcStages : 0); kb < issued; ++kb)
      mbar_wait(su32(bars + kb % kTcStages), (kb / kTcStages) & 1, abort, false);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t id = idesc<true>(min(128, (g.N - j0 + 15) / 16 * 16));
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kTcStages, round = kb / kTcStages;
      if (!mbar_wait(su32(bars + s), round & 1, abort, true)) {
        *abort = 1;
        atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = su32(base + s * kTcStage);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t xa = a0 + k * 32, xb = a0 + 2 * kTcBox + k * 32;
        mma<true>(tmem, sdesc(xa), sdesc(xb), id, (kb > 0 || k > 0) ? 1u : 0u);
        mma<true>(tmem, sdesc(xa), sdesc(xb + kTcBox), id, 1u);
        mma<true>(tmem, sdesc(xa + kTcBox), sdesc(xb), id, 1u);
      }
      mma_commit(su32(bars + kTcStages + s));
    }
    mma_commit(done);
  }
  __syncwarp();

  const bool ok = mbar_wait(done, 0, abort, false);
  tc_fence_after();
  if (__all_sync(0xffffffffu, ok && !*abort)) {
    float* stg = reinterpret_cast<float*>(base) + warp * 32 * 33;
    const int row0 = i0 + warp * 32;
#pragma unroll 1
    for (int c = 0; c < 4 && j0 + c * 32 < g.N; ++c) {  // uniform over the warp
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
#pragma unroll
      for (int q = 0; q < 32; ++q) stg[lane * 33 + q] = __uint_as_float(v[q]);
      __syncwarp();
      const int j = j0 + c * 32 + lane;
      if (j < g.N) {
        const float bj = (g.mode <= 1) ? g.bias[j] : 0.f;
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const int i = row0 + rr;
          if (i >= g.M) break;
          const int64_t o = (int64_t)i * g.ldc + j;
          if (!GNM_IN(o, (int64_t)g.M * g.ldc)) continue;
          float x = stg[rr * 33 + lane];
          if (g.mode == 0) {
            x += bj;
          } else if (g.mode == 1) {
            x += bj;
            g.Z[o] = x;
            x = gelu_f(x);
          } else if (g.mode == 2) {
            x *= gelu_df(g.Zprev[o]);
          }
          g.C[o] = x;
        }
      }
      __syncwarp();
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  }
}

// BF16 head / remainder planes of an FP32 [rows][cols] array (row stride
// lds): hi[r ld + c] = bf16(x), lo[r ld + c] = bf16(x - hi) (0 when zero_lo,
// for BF16-exact weights), and, when hiT is not NULL, the same planes of the
// transpose, hiT[c ldt + r].  32 x 32 tiles through shared memory keep both
// the row and the transposed stores coalesced; block (32, 8).
__global__ void __launch_bounds__(256) k_planes(const float* __restrict__ src, int rows, int cols, int64_t lds,
                                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                                int64_t ld, __nv_bfloat16* __restrict__ hiT,
                                                __nv_bfloat16* __restrict__ loT, int64_t ldt, int zero_lo) {
  __shared__ __nv_bfloat16 sh[32][33], sl[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int rr = threadIdx.y; rr < 32; rr += 8) {
    const int r = r0 + rr, c = c0 + threadIdx.x;
    __nv_bfloat16 h = __float2bfloat16_rn(0.f), l = h;
    if (r < rows && c < cols) {
      const float x = src[(int64_t)r * lds + c];
      h = __float2bfloat16_rn(x);
      l = zero_lo ? __float2bfloat16_rn(0.f) : __float2bfloat16_rn(x - __bfloat162float(h));
      hi[(int64_t)r * ld + c] = h;
      lo[(int64_t)r * ld + c] = l;
    }
    sh[rr][threadIdx.x] = h;
    sl[rr][threadIdx.x] = l;
  }
  if (!hiT) return;  // uniform
  __syncthreads();
  for (int cc = threadIdx.y; cc < 32; cc += 8) {
    const int c = c0 + cc, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      hiT[(int64_t)c * ldt + r] = sh[threadIdx.x][cc];
      loT[(int64_t)c * ldt + r] = sl[threadIdx.x][cc];
    }
  }
}

// h0 = (x - mean) / std in FP32, x given in FP64.
__global__ void k_mlp_input(const double* X, int B, int d0, const float* mean, const float* stdv, float* H) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * d0) return;
  const int i = (int)(t % d0);
  H[t] = ((float)X[t] - mean[i]) / stdv[i];
}

// Per-sample Gaussian NLL and dL/dy (one thread per sample).
__global__ void k_mlp_nll(const float* Y, int B, int dL, int nmu, int nu, const double* T, float* dY, double* loss_b) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* y = Y + (int64_t)b * dL;
  float* dy = dY + (int64_t)b * dL;
  const double* t = T + (int64_t)b * nmu;
  const float invB = 1.0f / (float)B;
  double L = 0.0;
  for (int k = 0; nu * k < nmu; ++k) dy[nmu + k] = 0.f;
  for (int j = 0; j < nmu; ++j) {
    const int k = j / nu;
    const float s = y[nmu + k];
    const float e = (float)t[j] - y[j];
    const float w = expf(-2.0f * s);
    L += 0.5 * (double)e * (double)e * (double)w + (double)s;
    dy[j] = -e * w * invB;
    dy[nmu + k] += (1.0f - e * e * w) * invB;
  }
  loss_b[b] = L;
}

// Deterministic sum of n doubles into out[0] (one block).
__global__ void k_sum(const double* x, int n, double scale, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// gb[j] = sum_b dZ[b][j]
__global__ void k_colsum(const float* dZ, int B, int N, float* gb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * N + j];
  gb[j] = s;
}

__global__ void k_adam(int64_t np, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
}

__global__ void k_d2f(const double* x, int64_t n, float* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
__global__ void k_f2d(const float* x, int64_t n, double* y, double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i] * scale;
}

// U0 = y_scale * mu, sigma_j = clamp(y_scale * exp(s_{j / nu}), lo, hi)
__global__ void k_warm(const float* Y, int B, int dL, int nmu, int nu, float yscale, double lo, double hi, double* U0,
                       double* sig) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * nmu) return;
  const int b = (int)(t / nmu), j = (int)(t % nmu);
  const float* y = Y + (int64_t)b * dL;
  U0[t] = (double)(yscale * y[j]);
  sig[t] = fmin(hi, fmax(lo, (double)(yscale * expf(y[nmu + j / nu]))));
}

}  // namespace
GNM_CHECK_ACCESSOR(check_count_mlp)
}  // namespace gnm

using namespace gnm;

struct gnmppi_mlp_s {
  int L = 0;
  int dims[kMaxLayers + 1] = {0};
  int nu = 1, nmu = 0, bf16 = 0, max_batch = 0;
  int64_t np = 0;
  int64_t off[kMaxLayers + 1] = {0};  // parameter offset of layer l (1-based)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *xmean = nullptr, *xstd = nullptr;
  float yscale = 1.f;
  float* H[kMaxLayers + 1] = {nullptr};  // activations (H[0] = normalised input)
  float* Z[kMaxLayers + 1] = {nullptr};  // pre-activations
  float *dA = nullptr, *dB = nullptr;    // gradient ping-pong buffers
  // BF16 head / remainder planes of the tensor-core operands: activations
  // H_l [B][ldh l] and their transposes [d_l][ldb] (l < L), weights W_l
  // [d_l][ldh l-1] and their transposes [d_{l-1}][ldh l], output gradients
  // dZ [B][ldd] and their transposes [d][ldb]
  __nv_bfloat16 *Hh[kMaxLayers + 1] = {nullptr}, *Hl[kMaxLayers + 1] = {nullptr};
  __nv_bfloat16 *HTh[kMaxLayers + 1] = {nullptr}, *HTl[kMaxLayers + 1] = {nullptr};
  __nv_bfloat16 *Wh[kMaxLayers + 1] = {nullptr}, *Wl[kMaxLayers + 1] = {nullptr};
  __nv_bfloat16 *WTh[kMaxLayers + 1] = {nullptr}, *WTl[kMaxLayers + 1] = {nullptr};
  __nv_bfloat16 *dZh = nullptr, *dZl = nullptr, *dZTh = nullptr, *dZTl = nullptr;
  int64_t ldh[kMaxLayers + 1] = {0};
  int64_t ldb = 0, ldd = 0;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  int* d_err = nullptr;  // a bounded wait of the tensor-core GEMM ran out
  int* h_err = nullptr;  // pinned copy
  double *loss_b = nullptr, *loss = nullptr;
  int t = 0;
  std::vector<void*> allocs;
  std::string err;
};

static thread_local char g_mlp_err[512];

static gnmppi_status mfail(gnmppi_mlp_t h, gnmppi_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else snprintf(g_mlp_err, sizeof(g_mlp_err), "%s", buf);
  return st;
}

#define MCK(call)                                                                                             \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess) return mfail(h, GNMPPI_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
  } while (0)
#define MCKL() MCK(cudaGetLastError())

template <typename P>
static gnmppi_status malloc_(gnmppi_mlp_t h, P** ptr, size_t bytes) {
  if (cudaMalloc((void**)ptr, bytes < 16 ? 16 : bytes) != cudaSuccess) {
    cudaGetLastError();
    return mfail(h, GNMPPI_E_NOMEM, "cudaMalloc(%zu) failed", bytes);
  }
  h->allocs.push_back((void*)*ptr);
  MCK(cudaMemsetAsync(*ptr, 0, bytes < 16 ? 16 : bytes, h->stream));
  return GNMPPI_OK;
}

extern "C" const char* gnmppi_mlp_last_error(gnmppi_mlp_t h) { return h ? h->err.c_str() : g_mlp_err; }

extern "C" void gnmppi_mlp_destroy(gnmppi_mlp_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* q : h->allocs) cudaFree(q);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

extern "C" gnmppi_status gnmppi_mlp_create(int32_t nlayers, const int32_t* dims, int32_t nu, int32_t weights_bf16,
                                           int32_t max_batch, void* cuda_stream, gnmppi_mlp_t* out) {
  if (!out || !dims) return mfail(nullptr, GNMPPI_E_ARG, "dims and out must not be NULL");
  *out = nullptr;
  if (nlayers < 1 || nlayers > kMaxLayers) return mfail(nullptr, GNMPPI_E_ARG, "nlayers must be in 1..%d", kMaxLayers);
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] < 1 || dims[l] > 65536) return mfail(nullptr, GNMPPI_E_ARG, "layer widths must be in 1..65536");
  if (nu < 1 || dims[nlayers] % (nu + 1) != 0)
    return mfail(nullptr, GNMPPI_E_ARG, "output width must be n_mu + n_mu/nu (a multiple of nu + 1)");
  if (max_batch < 1) return mfail(nullptr, GNMPPI_E_ARG, "max_batch must be >= 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return mfail(nullptr, GNMPPI_E_CUDA, "no CUDA device available");
  }
  gnmppi_mlp_t h = new gnmppi_mlp_s();
  h->L = nlayers;
  for (int l = 0; l <= nlayers; ++l) h->dims[l] = dims[l];
  h->nu = nu;
  h->nmu = dims[nlayers] / (nu + 1) * nu;
  h->bf16 = weights_bf16 ? 1 : 0;
  h->max_batch = max_batch;
  int64_t np = 0;
  for (int l = 1; l <= nlayers; ++l) {
    h->off[l] = np;
    np += (int64_t)dims[l] * dims[l - 1] + dims[l];
  }
  h->np = np;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return mfail(nullptr, GNMPPI_E_CUDA, "cudaStreamCreate failed");
    }
    h->own_stream = true;
  }
  gnmppi_status st;
#define MA(ptr, bytes)                                          \
  if ((st = malloc_(h, &(ptr), (bytes))) != GNMPPI_OK) {        \
    snprintf(g_mlp_err, sizeof(g_mlp_err), "%s", h->err.c_str()); \
    gnmppi_mlp_destroy(h);                                      \
    return st;                                                  \
  }
  MA(h->p, 4 * np);
  MA(h->g, 4 * np);
  MA(h->m, 4 * np);
  MA(h->v, 4 * np);
  MA(h->xmean, 4 * (size_t)dims[0]);
  MA(h->xstd, 4 * (size_t)dims[0]);
  int maxd = 0;
  for (int l = 0; l <= nlayers; ++l) {
    MA(h->H[l], 4 * (size_t)max_batch * dims[l]);
    MA(h->Z[l], 4 * (size_t)max_batch * dims[l]);
    maxd = dims[l] > maxd ? dims[l] : maxd;
  }
  MA(h->dA, 4 * (size_t)max_batch * maxd);
  MA(h->dB, 4 * (size_t)max_batch * maxd);
  // BF16 operand planes; row strides rounded up to 8 values (16 bytes, the TMA stride rule)
  auto r8 = [](int64_t x) { return (x + 7) / 8 * 8; };
  h->ldb = r8(max_batch);
  h->ldd = r8(maxd);
  for (int l = 0; l <= nlayers; ++l) h->ldh[l] = r8(dims[l]);
  for (int l = 0; l < nlayers; ++l) {
    MA(h->Hh[l], 2 * (size_t)max_batch * h->ldh[l]);
    MA(h->Hl[l], 2 * (size_t)max_batch * h->ldh[l]);
    MA(h->HTh[l], 2 * (size_t)dims[l] * h->ldb);
    MA(h->HTl[l], 2 * (size_t)dims[l] * h->ldb);
  }
  for (int l = 1; l <= nlayers; ++l) {
    MA(h->Wh[l], 2 * (size_t)dims[l] * h->ldh[l - 1]);
    MA(h->Wl[l], 2 * (size_t)dims[l] * h->ldh[l - 1]);
    MA(h->WTh[l], 2 * (size_t)dims[l - 1] * h->ldh[l]);
    MA(h->WTl[l], 2 * (size_t)dims[l - 1] * h->ldh[l]);
  }
  MA(h->dZh, 2 * (size_t)max_batch * h->ldd);
  MA(h->dZl, 2 * (size_t)max_batch * h->ldd);
  MA(h->dZTh, 2 * (size_t)maxd * h->ldb);
  MA(h->dZTl, 2 * (size_t)maxd * h->ldb);
  MA(h->d_err, sizeof(int));
  MA(h->loss_b, 8 * (size_t)max_batch);
  MA(h->loss, 8);
#undef MA
  {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn ||
        cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      gnmppi_mlp_destroy(h);
      return mfail(nullptr, GNMPPI_E_CUDA, "tensor-core GEMM set-up failed (cuTensorMapEncodeTiled, shared memory)");
    }
    h->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    *h->h_err = 0;
  }
  std::vector<float> one(dims[0], 1.f);
  if (cudaMemcpyAsync(h->xstd, one.data(), 4 * one.size(), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    gnmppi_mlp_destroy(h);
    return mfail(nullptr, GNMPPI_E_CUDA, "initialising the MLP failed");
  }
  *out = h;
  return GNMPPI_OK;
}

extern "C" int64_t gnmppi_mlp_num_params(gnmppi_mlp_t h) { return h ? h->np : 0; }

static gnmppi_status refresh_weights(gnmppi_mlp_t h);

static gnmppi_status to_device_f(gnmppi_mlp_t h, int32_t mem, const double* src, int64_t n, float* dst) {
  const double* dsrc = src;
  double* tmp = nullptr;
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMallocAsync((void**)&tmp, 8 * (size_t)n, h->stream));
    MCK(cudaMemcpyAsync(tmp, src, 8 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    dsrc = tmp;
  }
  k_d2f<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(dsrc, n, dst);
  MCKL();
  if (tmp) MCK(cudaFreeAsync(tmp, h->stream));
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_set_params(gnmppi_mlp_t h, int32_t mem, const double* params, int64_t count) {
  if (!h || !params) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (count != h->np) return mfail(h, GNMPPI_E_ARG, "expected %lld parameters", (long long)h->np);
  gnmppi_status st = to_device_f(h, mem, params, count, h->p);
  if (st != GNMPPI_OK) return st;
  if ((st = refresh_weights(h)) != GNMPPI_OK) return st;
  MCK(cudaMemsetAsync(h->m, 0, 4 * (size_t)h->np, h->stream));
  MCK(cudaMemsetAsync(h->v, 0, 4 * (size_t)h->np, h->stream));
  h->t = 0;
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_get_params(gnmppi_mlp_t h, int32_t mem, double* params, int64_t count) {
  if (!h || !params) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (count != h->np) return mfail(h, GNMPPI_E_ARG, "expected %lld parameters", (long long)h->np);
  double* dst = params;
  if (mem == GNMPPI_MEM_HOST) MCK(cudaMallocAsync((void**)&dst, 8 * (size_t)count, h->stream));
  k_f2d<<<(unsigned)((count + 255) / 256), 256, 0, h->stream>>>(h->p, count, dst, 1.0);
  MCKL();
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMemcpyAsync(params, dst, 8 * (size_t)count, cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaFreeAsync(dst, h->stream));
  }
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}

// Copy an FP32 device array out as doubles into `mem` memory.
static gnmppi_status out_f(gnmppi_mlp_t h, int32_t mem, const float* src, int64_t n, double* dst_user) {
  double* dst = dst_user;
  if (mem == GNMPPI_MEM_HOST) MCK(cudaMallocAsync((void**)&dst, 8 * (size_t)n, h->stream));
  k_f2d<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(src, n, dst, 1.0);
  MCKL();
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMemcpyAsync(dst_user, dst, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaFreeAsync(dst, h->stream));
  }
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_get_state(gnmppi_mlp_t h, int32_t mem, double* params, double* m1, double* m2,
                                              int64_t count, int32_t* step) {
  if (!h || !params || !m1 || !m2 || !step) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (count != h->np) return mfail(h, GNMPPI_E_ARG, "expected %lld parameters", (long long)h->np);
  gnmppi_status st;
  if ((st = out_f(h, mem, h->p, count, params)) != GNMPPI_OK) return st;
  if ((st = out_f(h, mem, h->m, count, m1)) != GNMPPI_OK) return st;
  if ((st = out_f(h, mem, h->v, count, m2)) != GNMPPI_OK) return st;
  MCK(cudaStreamSynchronize(h->stream));
  *step = h->t;
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_set_state(gnmppi_mlp_t h, int32_t mem, const double* params, const double* m1,
                                              const double* m2, int64_t count, int32_t step) {
  if (!h || !params || !m1 || !m2) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (count != h->np) return mfail(h, GNMPPI_E_ARG, "expected %lld parameters", (long long)h->np);
  if (step < 0) return mfail(h, GNMPPI_E_ARG, "step must be >= 0");
  gnmppi_status st;
  if ((st = to_device_f(h, mem, params, count, h->p)) != GNMPPI_OK) return st;
  if ((st = to_device_f(h, mem, m1, count, h->m)) != GNMPPI_OK) return st;
  if ((st = to_device_f(h, mem, m2, count, h->v)) != GNMPPI_OK) return st;
  if ((st = refresh_weights(h)) != GNMPPI_OK) return st;
  MCK(cudaStreamSynchronize(h->stream));
  h->t = step;
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_set_normalization(gnmppi_mlp_t h, const double* x_mean, const double* x_std,
                                                      double y_scale) {
  if (!h || !x_mean || !x_std) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (!(y_scale > 0.0)) return mfail(h, GNMPPI_E_ARG, "y_scale must be > 0");
  std::vector<float> m(h->dims[0]), s(h->dims[0]);
  for (int i = 0; i < h->dims[0]; ++i) {
    if (!(x_std[i] > 0.0)) return mfail(h, GNMPPI_E_ARG, "x_std must be > 0");
    m[i] = (float)x_mean[i];
    s[i] = (float)x_std[i];
  }
  MCK(cudaMemcpyAsync(h->xmean, m.data(), 4 * m.size(), cudaMemcpyHostToDevice, h->stream));
  MCK(cudaMemcpyAsync(h->xstd, s.data(), 4 * s.size(), cudaMemcpyHostToDevice, h->stream));
  MCK(cudaStreamSynchronize(h->stream));
  h->yscale = (float)y_scale;
  return GNMPPI_OK;
}

// K-major BF16 plane [rows][ld] as a TMA operand: boxes of 64 values x 128
// rows, 128-byte swizzle, zero fill outside the `cols` x `rows` extent.
static bool encode_plane(gnmppi_mlp_t h, CUtensorMap* m, const __nv_bfloat16* p, int64_t cols, int64_t rows,
                         int64_t ld) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  return h->encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A B^T on the tensor cores: A [M][K] (planes Ah, Al, row stride lda),
// B [N][K] (planes Bh, Bl, row stride ldb); g carries C, the epilogue and M, N, K.
static gnmppi_status tc_gemm(gnmppi_mlp_t h, const __nv_bfloat16* Ah, const __nv_bfloat16* Al, int64_t lda,
                             const __nv_bfloat16* Bh, const __nv_bfloat16* Bl, int64_t ldb, MlpTc g) {
  CUtensorMap m[4];
  if (!encode_plane(h, &m[0], Ah, g.K, g.M, lda) || !encode_plane(h, &m[1], Al, g.K, g.M, lda) ||
      !encode_plane(h, &m[2], Bh, g.K, g.N, ldb) || !encode_plane(h, &m[3], Bl, g.K, g.N, ldb))
    return mfail(h, GNMPPI_E_CUDA, "cuTensorMapEncodeTiled failed (MLP operand)");
  dim3 grid((unsigned)((g.N + 127) / 128), (unsigned)((g.M + 127) / 128));
  k_mlp_tc<<<grid, 128, kTcSmem, h->stream>>>(m[0], m[1], m[2], m[3], g, h->d_err);
  MCKL();
  return GNMPPI_OK;
}

// Head / remainder planes (and, with hiT, those of the transpose) of an FP32 array.
static gnmppi_status planes(gnmppi_mlp_t h, const float* src, int rows, int cols, int64_t lds, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, int64_t ld, __nv_bfloat16* hiT, __nv_bfloat16* loT, int64_t ldt,
                            int zero_lo) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  k_planes<<<grid, dim3(32, 8), 0, h->stream>>>(src, rows, cols, lds, hi, lo, ld, hiT, loT, ldt, zero_lo);
  MCKL();
  return GNMPPI_OK;
}

// Weight planes W_l and W_l^T from the FP32 master parameters (the
// remainder plane is zero when the products use BF16-rounded weights).
static gnmppi_status refresh_weights(gnmppi_mlp_t h) {
  for (int l = 1; l <= h->L; ++l) {
    const int din = h->dims[l - 1], dout = h->dims[l];
    gnmppi_status st = planes(h, h->p + h->off[l], dout, din, din, h->Wh[l], h->Wl[l], h->ldh[l - 1], h->WTh[l],
                              h->WTl[l], h->ldh[l], h->bf16);
    if (st != GNMPPI_OK) return st;
  }
  return GNMPPI_OK;
}

// The tensor-core error word: copied to pinned memory and cleared on the
// stream (before the caller's final synchronisation), then checked.
static gnmppi_status fetch_err(gnmppi_mlp_t h) {
  MCK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MCK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  return GNMPPI_OK;
}
static gnmppi_status check_err(gnmppi_mlp_t h) {
  if (*h->h_err) {
    *h->h_err = 0;
    return mfail(h, GNMPPI_E_TIMEOUT, "a bounded wait in the MLP's tensor-core GEMM ran out");
  }
  return GNMPPI_OK;
}
static gnmppi_status finish(gnmppi_mlp_t h) {
  gnmppi_status st = fetch_err(h);
  if (st != GNMPPI_OK) return st;
  MCK(cudaStreamSynchronize(h->stream));
  return check_err(h);
}

// Forward pass of B samples already in device memory (FP64), outputs in H[L];
// `train` also writes the transposed activation planes the weight gradients use.
static gnmppi_status forward(gnmppi_mlp_t h, const double* dX, int B, bool train) {
  const int d0 = h->dims[0];
  k_mlp_input<<<(unsigned)(((int64_t)B * d0 + 255) / 256), 256, 0, h->stream>>>(dX, B, d0, h->xmean, h->xstd, h->H[0]);
  MCKL();
  gnmppi_status st = planes(h, h->H[0], B, d0, d0, h->Hh[0], h->Hl[0], h->ldh[0], train ? h->HTh[0] : nullptr,
                            h->HTl[0], h->ldb, 0);
  if (st != GNMPPI_OK) return st;
  for (int l = 1; l <= h->L; ++l) {
    const int din = h->dims[l - 1], dout = h->dims[l];
    MlpTc g{};
    g.C = h->H[l];
    g.ldc = dout;
    g.M = B;
    g.N = dout;
    g.K = din;
    g.bias = h->p + h->off[l] + (int64_t)dout * din;
    g.Z = h->Z[l];
    g.mode = (l < h->L) ? 1 : 0;
    if ((st = tc_gemm(h, h->Hh[l - 1], h->Hl[l - 1], h->ldh[l - 1], h->Wh[l], h->Wl[l], h->ldh[l - 1], g)) !=
        GNMPPI_OK)
      return st;
    if (l < h->L &&
        (st = planes(h, h->H[l], B, dout, dout, h->Hh[l], h->Hl[l], h->ldh[l], train ? h->HTh[l] : nullptr,
                     h->HTl[l], h->ldb, 0)) != GNMPPI_OK)
      return st;
  }
  return GNMPPI_OK;
}

// Loss and gradient of B samples (device FP64 inputs) into h->g and h->loss.
static gnmppi_status loss_grad(gnmppi_mlp_t h, const double* dX, const double* dT, int B) {
  gnmppi_status st = forward(h, dX, B, true);
  if (st != GNMPPI_OK) return st;
  const int L = h->L, dL = h->dims[L];
  k_mlp_nll<<<(B + 127) / 128, 128, 0, h->stream>>>(h->H[L], B, dL, h->nmu, h->nu, dT, h->dA, h->loss_b);
  MCKL();
  k_sum<<<1, 256, 0, h->stream>>>(h->loss_b, B, 1.0 / B, h->loss);
  MCKL();
  float* dz = h->dA;  // dL/dz of layer l
  float* other = h->dB;
  if ((st = planes(h, dz, B, dL, dL, h->dZh, h->dZl, h->ldd, h->dZTh, h->dZTl, h->ldb, 0)) != GNMPPI_OK) return st;
  for (int l = L; l >= 1; --l) {
    const int din = h->dims[l - 1], dout = h->dims[l];
    // gW[o][i] = sum_b dz[b][o] h_{l-1}[b][i]: the transposed planes, K = B
    MlpTc gw{};
    gw.C = h->g + h->off[l];
    gw.ldc = din;
    gw.M = dout;
    gw.N = din;
    gw.K = B;
    gw.mode = 3;
    if ((st = tc_gemm(h, h->dZTh, h->dZTl, h->ldb, h->HTh[l - 1], h->HTl[l - 1], h->ldb, gw)) != GNMPPI_OK) return st;
    k_colsum<<<(dout + 127) / 128, 128, 0, h->stream>>>(dz, B, dout, h->g + h->off[l] + (int64_t)dout * din);
    MCKL();
    if (l > 1) {
      // dz_{l-1}[b][i] = (sum_o dz[b][o] W[o][i]) * GELU'(z_{l-1}[b][i])
      MlpTc gx{};
      gx.C = other;
      gx.ldc = din;
      gx.M = B;
      gx.N = din;
      gx.K = dout;
      gx.Zprev = h->Z[l - 1];
      gx.mode = 2;
      if ((st = tc_gemm(h, h->dZh, h->dZl, h->ldd, h->WTh[l], h->WTl[l], h->ldh[l], gx)) != GNMPPI_OK) return st;
      if ((st = planes(h, other, B, din, din, h->dZh, h->dZl, h->ldd, h->dZTh, h->dZTl, h->ldb, 0)) != GNMPPI_OK)
        return st;
      float* tmp = dz;
      dz = other;
      other = tmp;
    }
  }
  return GNMPPI_OK;
}

static gnmppi_status stage_in(gnmppi_mlp_t h, int32_t mem, const double* src, int64_t n, const double** dptr,
                              double** tmp) {
  *tmp = nullptr;
  *dptr = src;
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMallocAsync((void**)tmp, 8 * (size_t)(n > 0 ? n : 1), h->stream));
    MCK(cudaMemcpyAsync(*tmp, src, 8 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    *dptr = *tmp;
  }
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_forward(gnmppi_mlp_t h, int32_t mem, const double* X, int32_t B, double* Y) {
  if (!h || !X || !Y) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (B < 1 || B > h->max_batch) return mfail(h, GNMPPI_E_ARG, "B must be in 1..%d", h->max_batch);
  const double* dX;
  double* tx;
  gnmppi_status st = stage_in(h, mem, X, (int64_t)B * h->dims[0], &dX, &tx);
  if (st != GNMPPI_OK) return st;
  if ((st = forward(h, dX, B, false)) != GNMPPI_OK) return st;
  const int64_t n = (int64_t)B * h->dims[h->L];
  double* dY = Y;
  if (mem == GNMPPI_MEM_HOST) MCK(cudaMallocAsync((void**)&dY, 8 * (size_t)n, h->stream));
  k_f2d<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->H[h->L], n, dY, 1.0);
  MCKL();
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMemcpyAsync(Y, dY, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaFreeAsync(dY, h->stream));
  }
  if (tx) MCK(cudaFreeAsync(tx, h->stream));
  return finish(h);
}

extern "C" gnmppi_status gnmppi_mlp_loss_grad(gnmppi_mlp_t h, int32_t mem, const double* X, const double* T,
                                              int32_t B, double* loss, double* grad) {
  if (!h || !X || !T) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (B < 1 || B > h->max_batch) return mfail(h, GNMPPI_E_ARG, "B must be in 1..%d", h->max_batch);
  const double *dX, *dT;
  double *tx, *tt;
  gnmppi_status st = stage_in(h, mem, X, (int64_t)B * h->dims[0], &dX, &tx);
  if (st == GNMPPI_OK) st = stage_in(h, mem, T, (int64_t)B * h->nmu, &dT, &tt);
  if (st != GNMPPI_OK) return st;
  if ((st = loss_grad(h, dX, dT, B)) != GNMPPI_OK) return st;
  if (grad) {
    double* dg = grad;
    if (mem == GNMPPI_MEM_HOST) MCK(cudaMallocAsync((void**)&dg, 8 * (size_t)h->np, h->stream));
    k_f2d<<<(unsigned)((h->np + 255) / 256), 256, 0, h->stream>>>(h->g, h->np, dg, 1.0);
    MCKL();
    if (mem == GNMPPI_MEM_HOST) {
      MCK(cudaMemcpyAsync(grad, dg, 8 * (size_t)h->np, cudaMemcpyDeviceToHost, h->stream));
      MCK(cudaFreeAsync(dg, h->stream));
    }
  }
  if (loss) MCK(cudaMemcpyAsync(loss, h->loss, 8, cudaMemcpyDeviceToHost, h->stream));
  if (tx) MCK(cudaFreeAsync(tx, h->stream));
  if (tt) MCK(cudaFreeAsync(tt, h->stream));
  return finish(h);
}

extern "C" gnmppi_status gnmppi_mlp_train_step(gnmppi_mlp_t h, int32_t mem, const double* X, const double* T,
                                               int32_t B, double lr, double* loss) {
  if (!h || !X || !T) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (B < 1 || B > h->max_batch) return mfail(h, GNMPPI_E_ARG, "B must be in 1..%d", h->max_batch);
  if (!(lr > 0.0)) return mfail(h, GNMPPI_E_ARG, "lr must be > 0");
  const double *dX, *dT;
  double *tx, *tt;
  gnmppi_status st = stage_in(h, mem, X, (int64_t)B * h->dims[0], &dX, &tx);
  if (st == GNMPPI_OK) st = stage_in(h, mem, T, (int64_t)B * h->nmu, &dT, &tt);
  if (st != GNMPPI_OK) return st;
  if ((st = loss_grad(h, dX, dT, B)) != GNMPPI_OK) return st;
  h->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, h->t)), c2 = (float)(1.0 - std::pow(b2, h->t));
  k_adam<<<(unsigned)((h->np + 255) / 256), 256, 0, h->stream>>>(h->np, h->p, h->g, h->m, h->v, (float)lr, (float)b1,
                                                                 (float)b2, 1e-8f, c1, c2);
  MCKL();
  if ((st = refresh_weights(h)) != GNMPPI_OK) return st;
  if (loss) MCK(cudaMemcpyAsync(loss, h->loss, 8, cudaMemcpyDeviceToHost, h->stream));
  if (tx) MCK(cudaFreeAsync(tx, h->stream));
  if (tt) MCK(cudaFreeAsync(tt, h->stream));
  return finish(h);
}

extern "C" gnmppi_status gnmppi_mlp_warm_start(gnmppi_mlp_t h, int32_t mem, const double* X, int32_t B,
                                               double sigma_min, double sigma_max, double* U0, double* sigma) {
  if (!h || !X || !U0 || !sigma) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (!(sigma_min > 0.0) || !(sigma_max >= sigma_min)) return mfail(h, GNMPPI_E_ARG, "need 0 < sigma_min <= sigma_max");
  if (B < 1 || B > h->max_batch) return mfail(h, GNMPPI_E_ARG, "B must be in 1..%d", h->max_batch);
  const double* dX;
  double* tx;
  gnmppi_status st = stage_in(h, mem, X, (int64_t)B * h->dims[0], &dX, &tx);
  if (st != GNMPPI_OK) return st;
  if ((st = forward(h, dX, B, false)) != GNMPPI_OK) return st;
  const int64_t n = (int64_t)B * h->nmu;
  double *dU = U0, *dS = sigma;
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMallocAsync((void**)&dU, 8 * (size_t)n, h->stream));
    MCK(cudaMallocAsync((void**)&dS, 8 * (size_t)n, h->stream));
  }
  k_warm<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->H[h->L], B, h->dims[h->L], h->nmu, h->nu, h->yscale,
                                                             sigma_min, sigma_max, dU, dS);
  MCKL();
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMemcpyAsync(U0, dU, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaMemcpyAsync(sigma, dS, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaFreeAsync(dU, h->stream));
    MCK(cudaFreeAsync(dS, h->stream));
  }
  if (tx) MCK(cudaFreeAsync(tx, h->stream));
  return finish(h);
}
