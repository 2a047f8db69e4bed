// noalloc.cu -- softmin weights and MPPI mean perturbation for one sample set,
// computed without any device allocation.
//
// Some callers cannot allocate device memory when they call in: a real-time
// controller whose per-cycle latency budget leaves no room for cudaMalloc /
// cudaFree (their latency is unbounded and cudaFree synchronises the device),
// or a host that hands the library a fixed memory budget up front and forbids
// any allocation afterwards.  gnmppi_softmin_noalloc serves them: the caller
// passes device inputs and outputs, and the only scratch the kernel needs --
// one weight difference per sample pair -- lives in the file-scope device
// array below, which every GPU that loads the library holds until exit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/gnmppi.h"

namespace {

constexpr int kNoAllocMaxSamples = 65536;  // 512 KB of FP64 scratch per device
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: w+ - w- (or w) per sample pair.
// Each call writes every entry it reads before reading it, so nothing needs
// clearing between calls; calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_softmin_scratch[kNoAllocMaxSamples];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmin(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ double bsum(double v, double* red) {
  v = wsum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}
__device__ double bmin(double v, double* red) {
  v = wmin(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = INFINITY;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmin(t, red[i]);
  return t;
}

// One CTA of 256 threads: the same reduction as the solver's softmin kernel
// (Eq. 5 weights after the min shift; Eq. 3 weighted mean perturbation), for
// a single sample set in FP64.
__global__ void __launch_bounds__(256) k_softmin_noalloc(const double* __restrict__ C, const double* __restrict__ W,
                                                         int count, int n, int anti, double tau,
                                                         double* __restrict__ scratch, double* __restrict__ mppi,
                                                         double* __restrict__ stats) {
  __shared__ double red[32];
  double cmin = INFINITY;
  for (int m = threadIdx.x; m < count; m += blockDim.x) {
    const double c0 = C[anti ? 2 * m : m];
    const double c1 = anti ? C[2 * m + 1] : c0;
    if (isfinite(c0) && isfinite(c1)) cmin = fmin(cmin, fmin(c0, c1));
  }
  cmin = bmin(cmin, red);
  const double itau = 1.0 / tau;
  double s1 = 0.0, s2 = 0.0;
  for (int m = threadIdx.x; m < count; m += blockDim.x) {
    const double c0 = C[anti ? 2 * m : m];
    const double c1 = anti ? C[2 * m + 1] : c0;
    const bool ok = isfinite(c0) && isfinite(c1) && isfinite(cmin);
    const double w0 = ok ? exp(-(c0 - cmin) * itau) : 0.0;
    const double w1 = (ok && anti) ? exp(-(c1 - cmin) * itau) : 0.0;
    s1 += w0 + w1;
    s2 += w0 * w0 + w1 * w1;
    scratch[m] = w0 - w1;
  }
  s1 = bsum(s1, red);
  s2 = bsum(s2, red);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < n; j += (int)(blockDim.x >> 5)) {
    const double* row = W + (int64_t)j * count;
    double a = 0.0;
    for (int m = lane; m < count; m += 32) a += row[m] * scratch[m];
    a = wsum(a);
    if (lane == 0) mppi[j] = s1 > 0.0 ? a / s1 : 0.0;
  }
  if (threadIdx.x == 0) {
    stats[0] = cmin;
    stats[1] = s1;
    stats[2] = s2;
    stats[3] = s2 > 0.0 ? s1 * s1 / s2 : 0.0;
  }
}

void put_err(char* err, int32_t len, const char* msg) {
  if (err && len > 0) snprintf(err, (size_t)len, "%s", msg);
}

}  // namespace

extern "C" gnmppi_status gnmppi_softmin_noalloc(const double* C, const double* W, int32_t count, int32_t n,
                                                int32_t antithetic, double tau, double* mppi, double* stats,
                                                void* cuda_stream, char* err, int32_t err_len) {
  if (!C || !W || !mppi || !stats) {
    put_err(err, err_len, "C, W, mppi and stats must be device pointers, not NULL");
    return GNMPPI_E_ARG;
  }
  if (count < 1 || count > kNoAllocMaxSamples) {
    char buf[160];
    snprintf(buf, sizeof(buf), "count = %d is outside 1..%d, the size of the fixed scratch array", (int)count,
             kNoAllocMaxSamples);
    put_err(err, err_len, buf);
    return GNMPPI_E_ARG;
  }
  if (n < 1 || !(tau > 0.0)) {
    put_err(err, err_len, "n must be >= 1 and tau > 0");
    return GNMPPI_E_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    put_err(err, err_len, e != cudaSuccess ? cudaGetErrorString(e) : "device index out of range");
    return GNMPPI_E_CUDA;
  }
  double* scratch = nullptr;
  {
    // first call on a device: look up the device address of the scratch array
    // (the host-side symbol is only a stand-in) with that device current
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_softmin_scratch);
      if (e != cudaSuccess || !p) {
        put_err(err, err_len, e != cudaSuccess ? cudaGetErrorString(e) : "no device address for the scratch array");
        return GNMPPI_E_CUDA;
      }
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  k_softmin_noalloc<<<1, 256, 0, (cudaStream_t)cuda_stream>>>(C, W, count, n, antithetic ? 1 : 0, tau, scratch, mppi,
                                                               stats);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    put_err(err, err_len, cudaGetErrorString(e));
    return GNMPPI_E_CUDA;
  }
  return GNMPPI_OK;
}
