// mlp.cu -- the learned warm start: a small MLP that maps an initial state to
// a nominal control sequence mu (U_0 of Algorithm 1) and one log sampling
// scale per control step (Sigma_0), trained on solutions of plain GN-MPPI with
// a Gaussian negative log-likelihood.  Training and inference run in these
// kernels: strided SIMT GEMMs with fused bias / GELU / GELU' epilogues (FP32
// accumulation; weights optionally rounded to BF16 for the forward and
// input-gradient products), the loss and its output gradient, column sums for
// the bias gradients, and Adam with bias correction.  Parameter layout per
// layer: W [d_out][d_in] row-major, then b [d_out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gnmppi.h"

namespace {

constexpr int kMaxLayers = 8;

struct MlpGemm {
  // C[i][j] = sum_k A[i * a_i + k * a_k] * B[j * b_j + k * b_k]
  const float* A;
  int64_t a_i, a_k;
  const void* B;
  int64_t b_j, b_k;
  float* C;
  int64_t ldc;
  int M, N, K;
  const float* bias;   // [N] (modes 0, 1)
  float* Z;            // pre-activations out (mode 1)
  const float* Zprev;  // [M][ldc] pre-activations of the layer below (mode 2)
  int mode;            // 0: acc + bias; 1: GELU(acc + bias), Z = acc + bias; 2: acc * GELU'(Zprev); 3: acc
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}
__device__ __forceinline__ float ldw(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ldw(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

template <typename TB>
__global__ void __launch_bounds__(256) k_mlp_gemm(MlpGemm g) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const TB* Bp = reinterpret_cast<const TB*>(g.B);
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      const int i = i0 + r, k = k0 + kk;
      As[kk][r] = (i < g.M && k < g.K) ? g.A[(int64_t)i * g.a_i + (int64_t)k * g.a_k] : 0.f;
      const int j = j0 + r;
      Bs[kk][r] = (j < g.N && k < g.K) ? ldw(Bp, (int64_t)j * g.b_j + (int64_t)k * g.b_k) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + ty * 4 + p;
    if (i >= g.M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx * 4 + q;
      if (j >= g.N) continue;
      const int64_t o = (int64_t)i * g.ldc + j;
      float v = acc[p][q];
      if (g.mode == 0) {
        v += g.bias[j];
      } else if (g.mode == 1) {
        v += g.bias[j];
        g.Z[o] = v;
        v = gelu_f(v);
      } else if (g.mode == 2) {
        v *= gelu_df(g.Zprev[o]);
      }
      g.C[o] = v;
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
                       float c1, float c2, __nv_bfloat16* pb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (pb) pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_d2f(const double* x, int64_t n, float* y, __nv_bfloat16* yb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = (float)x[i];
  if (yb) yb[i] = __float2bfloat16_rn((float)x[i]);
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

struct gnmppi_mlp_s {
  int L = 0;
  int dims[kMaxLayers + 1] = {0};
  int nu = 1, nmu = 0, bf16 = 0, max_batch = 0;
  int64_t np = 0;
  int64_t off[kMaxLayers + 1] = {0};  // parameter offset of layer l (1-based)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* pb = nullptr;
  float *xmean = nullptr, *xstd = nullptr;
  float yscale = 1.f;
  float* H[kMaxLayers + 1] = {nullptr};  // activations (H[0] = normalised input)
  float* Z[kMaxLayers + 1] = {nullptr};  // pre-activations
  float *dA = nullptr, *dB = nullptr;    // gradient ping-pong buffers
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
  MA(h->pb, 2 * np);
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
  MA(h->loss_b, 8 * (size_t)max_batch);
  MA(h->loss, 8);
#undef MA
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

static gnmppi_status to_device_f(gnmppi_mlp_t h, int32_t mem, const double* src, int64_t n, float* dst,
                                 __nv_bfloat16* dstb) {
  const double* dsrc = src;
  double* tmp = nullptr;
  if (mem == GNMPPI_MEM_HOST) {
    MCK(cudaMallocAsync((void**)&tmp, 8 * (size_t)n, h->stream));
    MCK(cudaMemcpyAsync(tmp, src, 8 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    dsrc = tmp;
  }
  k_d2f<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(dsrc, n, dst, dstb);
  MCKL();
  if (tmp) MCK(cudaFreeAsync(tmp, h->stream));
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}

extern "C" gnmppi_status gnmppi_mlp_set_params(gnmppi_mlp_t h, int32_t mem, const double* params, int64_t count) {
  if (!h || !params) return mfail(h, GNMPPI_E_ARG, "NULL argument");
  if (count != h->np) return mfail(h, GNMPPI_E_ARG, "expected %lld parameters", (long long)h->np);
  gnmppi_status st = to_device_f(h, mem, params, count, h->p, h->pb);
  if (st != GNMPPI_OK) return st;
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

static void gemm(gnmppi_mlp_t h, const MlpGemm& g, bool weights_b) {
  dim3 grid((g.N + 63) / 64, (g.M + 63) / 64);
  if (weights_b && h->bf16)
    k_mlp_gemm<__nv_bfloat16><<<grid, 256, 0, h->stream>>>(g);
  else
    k_mlp_gemm<float><<<grid, 256, 0, h->stream>>>(g);
}

// Forward pass of B samples already in device memory (FP64), outputs in H[L].
static gnmppi_status forward(gnmppi_mlp_t h, const double* dX, int B) {
  const int d0 = h->dims[0];
  k_mlp_input<<<(unsigned)(((int64_t)B * d0 + 255) / 256), 256, 0, h->stream>>>(dX, B, d0, h->xmean, h->xstd, h->H[0]);
  MCKL();
  for (int l = 1; l <= h->L; ++l) {
    const int din = h->dims[l - 1], dout = h->dims[l];
    MlpGemm g{};
    g.A = h->H[l - 1];
    g.a_i = din;
    g.a_k = 1;
    g.B = h->bf16 ? (const void*)(h->pb + h->off[l]) : (const void*)(h->p + h->off[l]);
    g.b_j = din;
    g.b_k = 1;
    g.C = h->H[l];
    g.ldc = dout;
    g.M = B;
    g.N = dout;
    g.K = din;
    g.bias = h->p + h->off[l] + (int64_t)dout * din;
    g.Z = h->Z[l];
    g.mode = (l < h->L) ? 1 : 0;
    gemm(h, g, true);
    MCKL();
  }
  return GNMPPI_OK;
}

// Loss and gradient of B samples (device FP64 inputs) into h->g and h->loss.
static gnmppi_status loss_grad(gnmppi_mlp_t h, const double* dX, const double* dT, int B) {
  gnmppi_status st = forward(h, dX, B);
  if (st != GNMPPI_OK) return st;
  const int L = h->L, dL = h->dims[L];
  k_mlp_nll<<<(B + 127) / 128, 128, 0, h->stream>>>(h->H[L], B, dL, h->nmu, h->nu, dT, h->dA, h->loss_b);
  MCKL();
  k_sum<<<1, 256, 0, h->stream>>>(h->loss_b, B, 1.0 / B, h->loss);
  MCKL();
  float* dz = h->dA;  // dL/dz of layer l
  float* other = h->dB;
  for (int l = L; l >= 1; --l) {
    const int din = h->dims[l - 1], dout = h->dims[l];
    // gW[o][i] = sum_b dz[b][o] h_{l-1}[b][i]
    MlpGemm gw{};
    gw.A = dz;
    gw.a_i = 1;
    gw.a_k = dout;
    gw.B = h->H[l - 1];
    gw.b_j = 1;
    gw.b_k = din;
    gw.C = h->g + h->off[l];
    gw.ldc = din;
    gw.M = dout;
    gw.N = din;
    gw.K = B;
    gw.mode = 3;
    gemm(h, gw, false);
    MCKL();
    k_colsum<<<(dout + 127) / 128, 128, 0, h->stream>>>(dz, B, dout, h->g + h->off[l] + (int64_t)dout * din);
    MCKL();
    if (l > 1) {
      // dz_{l-1}[b][i] = (sum_o dz[b][o] W[o][i]) * GELU'(z_{l-1}[b][i])
      MlpGemm gx{};
      gx.A = dz;
      gx.a_i = dout;
      gx.a_k = 1;
      gx.B = h->bf16 ? (const void*)(h->pb + h->off[l]) : (const void*)(h->p + h->off[l]);
      gx.b_j = 1;
      gx.b_k = din;
      gx.C = other;
      gx.ldc = din;
      gx.M = B;
      gx.N = din;
      gx.K = dout;
      gx.Zprev = h->Z[l - 1];
      gx.mode = 2;
      gemm(h, gx, true);
      MCKL();
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
  if ((st = forward(h, dX, B)) != GNMPPI_OK) return st;
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
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
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
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
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
                                                                 (float)b2, 1e-8f, c1, c2, h->pb);
  MCKL();
  if (loss) MCK(cudaMemcpyAsync(loss, h->loss, 8, cudaMemcpyDeviceToHost, h->stream));
  if (tx) MCK(cudaFreeAsync(tx, h->stream));
  if (tt) MCK(cudaFreeAsync(tt, h->stream));
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
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
  if ((st = forward(h, dX, B)) != GNMPPI_OK) return st;
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
  MCK(cudaStreamSynchronize(h->stream));
  return GNMPPI_OK;
}
