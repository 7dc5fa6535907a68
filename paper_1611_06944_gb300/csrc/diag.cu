// Measured arithmetic peak of this GPU: the rate of fused multiply-adds of one
// precision when every SM runs long chains of independent FMAs and nothing else.
// It is the denominator of the roofline of the FP64 operator, which is bound by
// the FP64 pipe rather than by memory (a property of the machine, not a step of
// the method).
#include "hdcr_internal.cuh"

namespace hdcr {

constexpr int FMA_THREADS = 256;
constexpr int FMA_CHAINS = 8;     // independent chains per thread (covers the FMA latency)
constexpr int FMA_ITERS = 4096;   // FMAs per chain

static __device__ double g_fma_sink[2];

template <typename R>
__global__ void __launch_bounds__(FMA_THREADS) fma_rate_kernel(R b, R c, R guard) {
  R a[FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) a[i] = (R)(threadIdx.x + i) * (R)1e-3;
#pragma unroll 4
  for (int it = 0; it < FMA_ITERS; ++it)
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) a[i] = fma(a[i], b, c);
  R s = (R)0;
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) s += a[i];
  if (s == guard) g_fma_sink[0] = (double)s;  // never true for the guard passed; keeps the chains live
}

template <typename R>
static int fma_rate(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  HDCR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // 64 warps per SM
  cudaEvent_t e0, e1;
  HDCR_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(cudaErrorMemoryAllocation, "cudaEventCreate");
  }
  // b slightly below 1 and c small keep the chains finite
  const R b = (R)0.999999, c = (R)1e-6, guard = (R)-12345.0;
  fma_rate_kernel<R><<<blocks, FMA_THREADS, 0, st>>>(b, c, guard);  // warm-up
  count_launch();
  constexpr int reps = 5;
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r) {
    fma_rate_kernel<R><<<blocks, FMA_THREADS, 0, st>>>(b, c, guard);
    count_launch();
  }
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_status(err, "FMA rate probe");
  const double fmas = (double)reps * blocks * FMA_THREADS * (double)FMA_CHAINS * FMA_ITERS;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_probe_fma_rate(int dtype, double* tflops, void* stream) {
  if (!tflops) {
    set_error("hdcr_probe_fma_rate: null result pointer");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128) return fma_rate<double>(tflops, as_stream(stream));
  if (dtype == HDCR_C64) return fma_rate<float>(tflops, as_stream(stream));
  set_error("hdcr_probe_fma_rate: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}
