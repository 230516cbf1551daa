// Arithmetic-rate probe: the FMA throughput of this GPU in FP64 and FP32, measured by a
// kernel of independent fused multiply-add chains.  The FP64 operator kernels (SpMV,
// assembly, Arnoldi) are bound by GB300's narrow FP64 pipe rather than by memory, and this
// figure is the roofline they are reported against.
#include "common.h"

namespace gdsw {

template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T b, T c) {
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = T(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps every chain live
}

template <typename T>
static double run_probe(int iters) {
  constexpr int kChains = 8;
  int dev = 0, sms = 0;
  GDSW_CUDA(cudaGetDevice(&dev));
  GDSW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  GDSW_CUDA(cudaMalloc(&out, sizeof(T) * size_t(blocks) * threads));
  cudaEvent_t e0, e1;
  GDSW_CUDA(cudaEventCreate(&e0));
  GDSW_CUDA(cudaEventCreate(&e1));
  const T b = T(0.999999), c = T(1e-7);
  k_fma_probe<T, kChains><<<blocks, threads>>>(out, iters / 8, b, c);  // warm-up
  check_launch("k_fma_probe");
  GDSW_CUDA(cudaEventRecord(e0));
  k_fma_probe<T, kChains><<<blocks, threads>>>(out, iters, b, c);
  GDSW_CUDA(cudaEventRecord(e1));
  GDSW_CUDA(cudaEventSynchronize(e1));
  check_launch("k_fma_probe");
  float ms = 0;
  GDSW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 2.0 * kChains * double(iters) * blocks * threads;
  return flops / (double(ms) * 1e-3) / 1e12;
}

}  // namespace gdsw

extern "C" int gdsw_probe_fma(int32_t precision, double* tflops) {
  using namespace gdsw;
  if (!tflops || (precision != GDSW_FP64 && precision != GDSW_FP32)) return GDSW_ERR_INVALID_ARG;
  try {
    *tflops = precision == GDSW_FP64 ? run_probe<double>(1 << 14) : run_probe<float>(1 << 16);
    return GDSW_OK;
  } catch (const gdsw::Error& e) {
    return e.code;
  } catch (...) {
    return GDSW_ERR_CUDA;
  }
}
