// hfx_energy_noalloc: the exchange energy E = sum_{mu nu} P_{mu nu} K_{mu nu} with no
// device allocation at all.
//
// Why it exists: some callers cannot let a library call cudaMalloc -- host programs that
// hand all device memory out of their own pool or run under a fixed device-memory budget,
// and latency-critical loops where an allocation would synchronise the device.  This
// entry point therefore keeps its scratch (one compensated partial sum per matrix row)
// in a fixed device array that is part of the loaded library image.
//
// The scratch is a file-scope __device__ array.  Host code cannot use its name as a
// device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first call on a
// device should come before any stream capture.  The cache is per device ordinal, for the
// runtime's primary context: a cudaDeviceReset later in the process would leave it stale.  Every call on a device shares the
// array: calls whose kernels overlap on the GPU race on it and must be ordered by the
// caller (e.g. issued on one stream).  The array keeps the previous call's contents;
// each call writes every row partial it later reads, so nothing has to be cleared.
#include <mutex>
#include <string>

#include "hfx.h"

namespace hfx {
void set_global_error(const std::string& msg);
}

// (sum, compensation) per row, HFX_NOALLOC_MAX_N rows: 256 KiB per device
static __device__ __align__(256) double g_noalloc_rows[2 * HFX_NOALLOC_MAX_N];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_rows_ptr[kMaxDevices] = {};

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// One block per row: compensated sum of P_ij K_ij over the row.
__global__ void k_noalloc_rows(int n, int ld, const double* __restrict__ P, const double* __restrict__ K,
                               double* __restrict__ rows) {
  __shared__ double ss[128], cc[128];
  const int i = blockIdx.x;
  double s = 0.0, c = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double e;
    two_sum(s, P[(size_t)i * ld + j] * K[(size_t)i * ld + j], s, e);
    c += e;
  }
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + w], ss[threadIdx.x], e);
      cc[threadIdx.x] += cc[threadIdx.x + w] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rows[2 * i] = ss[0];
    rows[2 * i + 1] = cc[0];
  }
}

// One block: compensated sum of the n row partials.
__global__ void k_noalloc_final(int n, const double* __restrict__ rows, double* __restrict__ out) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double e;
    two_sum(s, rows[2 * i], s, e);
    c += e + rows[2 * i + 1];
  }
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + w], ss[threadIdx.x], e);
      cc[threadIdx.x] += cc[threadIdx.x + w] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = ss[0] + cc[0];
}

}  // namespace

extern "C" int hfx_energy_noalloc(const double* P_dev, const double* K_dev, int n, int ld, double* E_dev,
                                  void* stream) {
  if (!P_dev || !K_dev || !E_dev) {
    hfx::set_global_error("hfx_energy_noalloc: NULL pointer");
    return HFX_ERR_ARG;
  }
  if (n < 1 || n > HFX_NOALLOC_MAX_N || ld < n) {
    hfx::set_global_error("hfx_energy_noalloc: n must be in 1.." + std::to_string(HFX_NOALLOC_MAX_N) +
                          " (the size of the fixed scratch array) and ld >= n; got n=" + std::to_string(n) +
                          ", ld=" + std::to_string(ld));
    return HFX_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    hfx::set_global_error(std::string("hfx_energy_noalloc: no usable CUDA device: ") + cudaGetErrorString(e));
    return HFX_ERR_CUDA;
  }
  double* rows = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_rows_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_rows);
      if (e != cudaSuccess || !p) {
        hfx::set_global_error(std::string("hfx_energy_noalloc: cudaGetSymbolAddress failed: ") +
                              cudaGetErrorString(e));
        return HFX_ERR_CUDA;
      }
      g_rows_ptr[dev] = (double*)p;
    }
    rows = g_rows_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_rows<<<n, 128, 0, s>>>(n, ld, P_dev, K_dev, rows);
  k_noalloc_final<<<1, 256, 0, s>>>(n, rows, E_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    hfx::set_global_error(std::string("hfx_energy_noalloc: launch failed: ") + cudaGetErrorString(e));
    return HFX_ERR_CUDA;
  }
  return HFX_OK;
}
