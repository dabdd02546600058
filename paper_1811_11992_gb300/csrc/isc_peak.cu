// Measured FMA throughput of this GPU in FP64 and FP32: the ALU roof that the
// FP64 kernels of the Newton step are reported against (on GB300 the FP64 pipe
// is narrow, so an FP64 kernel above ~0.18 flop per HBM byte is bound by it,
// not by HBM). A register-resident loop of independent FMA chains, enough
// warps to cover the pipe latency, timed with CUDA events, best of five runs.
#include <cuda_runtime.h>

#include "isc_internal.cuh"

namespace isc {
namespace {

constexpr int CHAINS = 8;       // independent accumulators per thread
constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_loop(int iters, T b, T c, T* out) {
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  // b and c are run-time values, so the loop cannot be folded; one store per
  // thread keeps it live
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FMA/s of one precision: best of `runs` timed launches after one warm-up
template <typename T>
int measure(int sms, int iters, double* fma_per_s) {
  const int blocks = sms * PEAK_BLOCKS_PER_SM;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * PEAK_THREADS) != cudaSuccess) return ISC_ERR_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = ISC_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = ISC_ERR_CUDA;
  double best = 0.0;
  // b slightly below one and c small keep every chain finite and normal
  const T b = T(0.999999), c = T(1e-6);
  for (int run = 0; run < 6 && st == ISC_OK; ++run) {
    cudaEventRecord(e0);
    k_fma_loop<T><<<blocks, PEAK_THREADS>>>(iters, b, c, out);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      st = ISC_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double fmas = (double)blocks * PEAK_THREADS * CHAINS * iters;
    if (run > 0 && ms > 0.f) best = fmas / (ms * 1e-3) > best ? fmas / (ms * 1e-3) : best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  *fma_per_s = best;
  return st;
}

}  // namespace
}  // namespace isc

extern "C" int isc_measure_fma_rates(double* fp64_gflops, double* fp32_gflops) {
  using namespace isc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ISC_ERR_CUDA;
  if (fp64_gflops) {
    double r = 0.0;
    // ~10 G FMA: about 17 ms at GB300's FP64 rate
    const int st = measure<double>(sms, 4096, &r);
    if (st != ISC_OK) return st;
    *fp64_gflops = 2.0 * r * 1e-9;
  }
  if (fp32_gflops) {
    double r = 0.0;
    const int st = measure<float>(sms, 65536, &r);
    if (st != ISC_OK) return st;
    *fp32_gflops = 2.0 * r * 1e-9;
  }
  return ISC_OK;
}
