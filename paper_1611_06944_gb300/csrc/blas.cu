// Level-1 kernels of the Krylov solvers (Section 3): inner products with FP64
// accumulation in a deterministic order, and the scratch they need.
#include <mutex>
#include <vector>

#include "blas.cuh"

namespace hdcr {

int red_buffers_alloc(RedBuffers* rb, int nscal) {
  const size_t bytes = sizeof(double) * (RED_MAX_BLOCKS * RED_MAX_NV + nscal) + 256;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    set_error("reduction scratch: cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return HDCR_ERR_NO_MEMORY;
  }
  e = cudaMemset(p, 0, bytes);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_status(e, "cudaMemset(reduction scratch)");
  }
  rb->base = p;
  rb->scal = (double*)p;
  rb->nscal = nscal;
  rb->rs.partials = (double*)p + nscal;
  rb->rs.counter = (unsigned int*)((double*)p + nscal + RED_MAX_BLOCKS * RED_MAX_NV);
  return HDCR_OK;
}

void red_buffers_free(RedBuffers* rb) {
  if (rb->base) cudaFree(rb->base);
  rb->base = nullptr;
}

// ------------------------------------------------------------------ kernels
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cdot_kernel(const cpx<R>* __restrict__ u,
                                                           const cpx<R>* __restrict__ v, long long n,
                                                           RedScratch rs, double* result) {
  double acc[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cpx<R> a = ld(u + i), b = ld(v + i);
    acc[0] = fma((double)a.re, (double)b.re, fma((double)a.im, (double)b.im, acc[0]));
    acc[1] = fma((double)a.re, (double)b.im, fma(-(double)a.im, (double)b.re, acc[1]));
  }
  double tot[2];
  if (grid_reduce<2>(acc, rs, tot)) {
    result[0] = tot[0];
    result[1] = tot[1];
  }
}

// |u|^2 in FP64.  FP32 data: squares summed in FP32 over runs of 16 elements
// (all terms positive: relative error below 16 ulp) and the runs in FP64, which
// keeps the slow FP64 pipe out of the per-element work.
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) norm2_kernel(const cpx<R>* __restrict__ u, long long n,
                                                            RedScratch rs, double* result) {
  double acc[1] = {0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sizeof(R) == 4) {
    while (i < n) {
      float run = 0.f;
#pragma unroll 4
      for (int k = 0; k < 16 && i < n; ++k, i += stride) {
        const cpx<R> a = ld(u + i);
        run = fmaf((float)a.re, (float)a.re, fmaf((float)a.im, (float)a.im, run));
      }
      acc[0] += (double)run;
    }
  } else {
    for (; i < n; i += stride) {
      cpx<R> a = ld(u + i);
      acc[0] = fma((double)a.re, (double)a.re, fma((double)a.im, (double)a.im, acc[0]));
    }
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) result[0] = tot[0];
}

template <typename R>
int launch_cdot(const void* u, const void* v, long long n, RedScratch rs, double* result, cudaStream_t st) {
  cdot_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>((const cpx<R>*)u, (const cpx<R>*)v, n, rs, result); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_cdot<double>(const void*, const void*, long long, RedScratch, double*, cudaStream_t);
template int launch_cdot<float>(const void*, const void*, long long, RedScratch, double*, cudaStream_t);

template <typename R>
int launch_norm2(const void* u, long long n, RedScratch rs, double* result, cudaStream_t st) {
  norm2_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>((const cpx<R>*)u, n, rs, result); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_norm2<double>(const void*, long long, RedScratch, double*, cudaStream_t);
template int launch_norm2<float>(const void*, long long, RedScratch, double*, cudaStream_t);

// Per-device scratch of the standalone reduction calls, created on first use
// and kept until the process exits.
static std::mutex g_dev_mutex;
static std::vector<RedBuffers> g_dev_red;

int device_red_scratch(RedScratch* out) {
  int dev = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_dev_mutex);
  if ((int)g_dev_red.size() <= dev) g_dev_red.resize(dev + 1, RedBuffers{{nullptr, nullptr}, nullptr, 0, nullptr});
  if (!g_dev_red[dev].base) HDCR_TRY(red_buffers_alloc(&g_dev_red[dev], 0));
  *out = g_dev_red[dev].rs;
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_cdot(const void* u, const void* v, size_t n, int dtype, double* result, void* stream) {
  if (!u || !v || !result || n == 0) {
    set_error("hdcr_cdot: null pointer or n == 0");
    return HDCR_ERR_BAD_ARG;
  }
  RedScratch rs;
  HDCR_TRY(device_red_scratch(&rs));
  if (dtype == HDCR_C128) return launch_cdot<double>(u, v, (long long)n, rs, result, as_stream(stream));
  if (dtype == HDCR_C64) return launch_cdot<float>(u, v, (long long)n, rs, result, as_stream(stream));
  set_error("hdcr_cdot: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}

extern "C" int hdcr_norm2(const void* u, size_t n, int dtype, double* result, void* stream) {
  if (!u || !result || n == 0) {
    set_error("hdcr_norm2: null pointer or n == 0");
    return HDCR_ERR_BAD_ARG;
  }
  RedScratch rs;
  HDCR_TRY(device_red_scratch(&rs));
  if (dtype == HDCR_C128) return launch_norm2<double>(u, (long long)n, rs, result, as_stream(stream));
  if (dtype == HDCR_C64) return launch_norm2<float>(u, (long long)n, rs, result, as_stream(stream));
  set_error("hdcr_norm2: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}
