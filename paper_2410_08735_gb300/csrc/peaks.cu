// FMA-throughput probe: the FP32 and FP64 fused multiply-add peaks of the GPU the library runs on, the
// denominators of the roofline fractions of its ALU-bound kernels (the fused sweeps).  Every thread runs
// eight independent FMA chains (enough instruction-level parallelism to cover the pipe latency at full
// occupancy), the grid covers every SM several times over, and the launch is timed with CUDA events.
#include <algorithm>

#include "internal.h"

namespace rte {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T a, T b, int iters, T* sink) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = a + (T)(threadIdx.x & 7) + (T)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], b, a);
    }
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  // never true for the arguments the host passes; keeps the chains alive
  if (s == (T)-1.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int fma_peak_t(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  RTE_CHECK_CUDA(cudaGetDevice(&dev));
  RTE_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  cudaEvent_t e0, e1;
  RTE_CHECK_CUDA(cudaEventCreate(&e0));
  RTE_CHECK_CUDA(cudaEventCreate(&e1));
  // a + b x stays bounded (|b| < 1), never reaches -1 from the positive start values
  const T a = (T)0.25, b = (T)0.5;
  float best = 1e30f;
  int rc = RTE_OK;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_peak<T><<<blocks, threads, 0, st>>>(a, b, iters, nullptr);
    count_launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      set_error(std::string("fma peak probe: ") + cudaGetErrorString(e));
      rc = RTE_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);   // the first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RTE_OK) return rc;
  const double flops = 2.0 * 8 * 4 * (double)iters * threads * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return RTE_OK;
}

}  // namespace rte

extern "C" int rte_fma_peak(int dtype, double* tflops, void* stream) {
  RTE_ARG(tflops, "null pointer");
  RTE_ARG(dtype == RTE_F64 || dtype == RTE_F32, "dtype must be RTE_F64 or RTE_F32");
  // FP64 runs far fewer iterations: its pipe is a small fraction of the FP32 rate on this GPU
  if (dtype == RTE_F32) return rte::fma_peak_t<float>(4096, tflops, (cudaStream_t)stream);
  return rte::fma_peak_t<double>(128, tflops, (cudaStream_t)stream);
}
